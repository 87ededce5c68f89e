"""Level evaluation without device allocations (vx_csf_eval_level_static).

This entry point serves callers that cannot allocate device memory while they run, such as a
host framework that owns the GPU's memory as a fixed budget, or a latency-bound loop that must
not risk an allocation's synchronisation or out-of-memory failure.  Its scratch lives in a
fixed device array that the library declares; the results must equal those of the allocating
entry point (vx_csf_eval_level) bit for bit, call after call, although every call leaves the
array's contents behind for the next.
"""
import numpy as np
import pytest

from paper_2406_09857_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vx():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2406_09857_gb300 import build
    from paper_2406_09857_gb300 import vx as _vx

    build.build()
    _vx.lib()
    return _vx


def _dev(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _case(vx, k, d, npoly, level, n, seed):
    polys = synth.random_small(k, d, npoly, seed)
    t = synth.random_tuples(k, level, n, seed + 1)
    return polys, vx.System(polys), vx.csf_build(k, level, _dev(t)), int(t.shape[0])


@pytest.mark.parametrize("mode_name", ["FP64", "FP32_MIDRAD"])
def test_static_matches_allocating_entry_point_twice(vx, mode_name):
    import torch

    mode = getattr(vx, mode_name)
    cases = [_case(vx, 3, 6, 2, 5, 6000, 71), _case(vx, 2, 9, 1, 7, 3000, 72)]
    for rep in range(2):  # two calls in a row for each case, interleaved between the cases
        for polys, sysv, c, n in cases:
            keep_ref, lo_ref, hi_ref = vx.csf_eval_level(sysv, c, synth.cube(len(polys[0][0][0])),
                                                         mode, values=True)
            keep = torch.empty(n, dtype=torch.uint8, device="cuda")
            lo = torch.empty((len(polys), n), dtype=torch.float64, device="cuda")
            hi = torch.empty_like(lo)
            vx.csf_eval_level_static(sysv, c, synth.cube(len(polys[0][0][0])), mode, keep, lo, hi)
            torch.cuda.synchronize()
            assert torch.equal(keep, keep_ref)
            assert torch.equal(lo, lo_ref) and torch.equal(hi, hi_ref)


def test_static_rejects_what_does_not_fit(vx):
    import torch

    # one degree-50 surface on 512 x 512 columns: depth-2 blocks of 51 intervals for 262144
    # nodes (214 MB in binary64) exceed the fixed array
    polys = [synth.kostlan_poly(3, 50, 5)]
    i, j = np.meshgrid(np.arange(512, dtype=np.int32), np.arange(512, dtype=np.int32),
                       indexing="ij")
    t = np.stack([i.ravel(), j.ravel(), np.zeros(i.size, dtype=np.int32)], axis=1)
    sysv = vx.System(polys)
    c = vx.csf_build(3, 9, _dev(t))
    keep = torch.empty(t.shape[0], dtype=torch.uint8, device="cuda")
    with pytest.raises(vx.VxError) as e:
        vx.csf_eval_level_static(sysv, c, synth.cube(3), vx.FP64, keep)
    assert e.value.code == vx.ECAPACITY
    assert "scratch" in str(e.value)
    with pytest.raises(vx.VxError) as e:
        vx.csf_eval_level_static(sysv, c, synth.cube(3), vx.FP32, keep)
    assert e.value.code == vx.EINVAL


def _cudart():
    """The CUDA runtime this process has loaded (the one libvx links), through ctypes."""
    import ctypes

    path = None
    with open("/proc/self/maps") as f:
        for line in f:
            if "libcudart.so" in line:
                path = line.split()[-1]
                break
    return ctypes.CDLL(path or "libcudart.so.13")


def _pool_used_high(rt, reset=False):
    """cudaMemPoolAttrUsedMemHigh (0x8) of device 0's default pool, which libvx's stream-ordered
    allocations come from; reset=True first sets the high mark to the current use."""
    import ctypes

    pool = ctypes.c_void_p()
    assert rt.cudaDeviceGetDefaultMemPool(ctypes.byref(pool), 0) == 0
    if reset:
        zero = ctypes.c_uint64(0)
        assert rt.cudaMemPoolSetAttribute(pool, 0x8, ctypes.byref(zero)) == 0
    v = ctypes.c_uint64(0)
    assert rt.cudaMemPoolGetAttribute(pool, 0x8, ctypes.byref(v)) == 0
    return v.value


def test_static_call_allocates_no_device_memory(vx):
    """The defining property, observed from outside: across a warmed-up call the high-water mark
    of the device pool the library allocates from does not move, while the allocating entry
    point on the same level does move it (so the probe sees the library's allocations)."""
    import torch

    polys, sysv, c, n = _case(vx, 3, 6, 2, 5, 6000, 73)
    dom = synth.cube(3)
    keep = torch.empty(n, dtype=torch.uint8, device="cuda")
    lo = torch.empty((len(polys), n), dtype=torch.float64, device="cuda")
    hi = torch.empty_like(lo)
    vx.csf_eval_level_static(sysv, c, dom, vx.FP64, keep, lo, hi)  # warm-up (symbol lookup)
    torch.cuda.synchronize()
    rt = _cudart()
    base = _pool_used_high(rt, reset=True)
    for _ in range(2):
        vx.csf_eval_level_static(sysv, c, dom, vx.FP64, keep, lo, hi)
        vx.csf_eval_level_static(sysv, c, dom, vx.FP32_MIDRAD, keep, lo, hi)
    torch.cuda.synchronize()
    assert _pool_used_high(rt) == base
    vx.csf_eval_level(sysv, c, dom, vx.FP64, values=True)
    torch.cuda.synchronize()
    assert _pool_used_high(rt) > base
