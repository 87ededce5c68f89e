"""C0 on the Taylor form (Def. 3) on the GPU, against the oracle.

- the form's interval on every box, bit for bit (binary64), orders 1-3, k = 1..4, several
  polynomials, a non-symmetric dyadic domain, boxes at the domain's edges;
- Algorithm 3 with the Taylor criterion: the same boxes and per-level counts as the oracle's;
- the certified binary32 form: every C0 / C1 decision and whole enclosures equal binary64's;
- what it refuses: midpoint-radius binary32, orders with more terms than VX_MAXPOLY, batches.
"""
import numpy as np
import pytest

import oracle
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


@pytest.mark.parametrize("k,d,npoly,level,order,n,seed,dom", [
    (1, 12, 1, 6, 3, 64, 1, None),
    (2, 8, 2, 5, 2, 600, 2, None),
    (2, 6, 1, 4, 4, 256, 3, [-2.0, 2.0, 0.0, 1.0]),
    (3, 6, 2, 4, 1, 2000, 4, None),
    (3, 5, 1, 4, 2, 2000, 5, [-1.0, 3.0, -2.0, 2.0, 0.0, 4.0]),
    (4, 4, 1, 3, 2, 1500, 6, None),
    (4, 3, 2, 3, 1, 1500, 7, None),
])
def test_taylor_values_bit_exact(vx, k, d, npoly, level, order, n, seed, dom):
    import torch

    polys = synth.random_small(k, d, npoly, seed)
    dom = synth.cube(k) if dom is None else np.asarray(dom)
    t = synth.random_tuples(k, level, n, seed + 1)
    lo_o, hi_o, keep_o = oracle.taylor_boxes(polys, dom, level, order, t)
    sysv = vx.System(polys)
    c = vx.csf_build(k, level, _dev(t))
    keep, lo, hi = vx.csf_eval_level_taylor(sysv, c, dom, order, values=True)
    torch.cuda.synchronize()
    assert np.array_equal(lo.cpu().numpy(), lo_o)
    assert np.array_equal(hi.cpu().numpy(), hi_o)
    assert np.array_equal(keep.cpu().numpy(), keep_o)


@pytest.mark.parametrize("k,d,npoly,depth,order,seed", [(2, 10, 1, 7, 2, 11), (2, 8, 2, 6, 3, 12),
                                                        (3, 6, 1, 5, 2, 13), (3, 5, 2, 5, 1, 14),
                                                        (4, 3, 1, 4, 2, 15)])
def test_taylor_enclosure_equals_oracle(vx, k, d, npoly, depth, order, seed):
    polys = [synth.kostlan_poly(k, d, 100 * seed + p) for p in range(npoly)]
    dom = synth.cube(k)
    ref = oracle.enclose_taylor(polys, dom, depth, order)
    r = vx.enclose(polys, dom, depth, vx.make_opts(vx.FP64, taylor_order=order))
    assert np.array_equal(r.boxes(), ref["tuples"])
    st = r.stats()
    assert np.array_equal(st["tested"], ref["tested"])
    assert np.array_equal(st["kept"], ref["kept"])


def test_taylor_refusals(vx):
    polys = synth.random_small(3, 4, 1, 20)
    with pytest.raises(vx.VxError) as e:  # the midpoint-radius arithmetic has no Taylor form
        vx.enclose(polys, synth.cube(3), 3, vx.make_opts(vx.FP32_MIDRAD, taylor_order=2))
    assert e.value.code == vx.EINVAL
    with pytest.raises(vx.VxError) as e:  # C(3+3, 3) = 20 > 16 terms
        vx.enclose(polys, synth.cube(3), 3, vx.make_opts(vx.FP64, taylor_order=3))
    assert e.value.code == vx.EINVAL
    with pytest.raises(vx.VxError) as e:
        vx.enclose_batch([(polys, synth.cube(3), 3)], vx.make_opts(vx.FP64, taylor_order=1))
    assert e.value.code == vx.EINVAL


@pytest.mark.parametrize("k,d,npoly,level,order,n,seed,rel", [
    (2, 9, 2, 6, 2, 1500, 31, None),
    (3, 6, 2, 4, 2, 3000, 32, None),
    (3, 5, 3, 4, 1, 3000, 33, [0, 1, 3]),
    (4, 4, 1, 3, 2, 3000, 34, None),
    (2, 12, 1, 7, 3, 3000, 35, [4]),
])
def test_taylor_certified_binary32_level_equals_binary64(vx, k, d, npoly, level, order, n, seed,
                                                           rel):
    """The form's derivatives in certified binary32: every C0 decision (and C1's where C0
    keeps) is the binary64 one, i.e. the oracle's."""
    polys = synth.random_small(k, d, npoly, seed)
    dom = synth.cube(k)
    t = synth.random_tuples(k, level, n, seed + 1)
    sysv = vx.System(polys, rel=rel) if rel else vx.System(polys)
    c = vx.csf_build(k, level, _dev(t))
    if rel is None:
        _, _, keep_o = oracle.taylor_boxes(polys, dom, level, order, t)
    else:
        # the oracle's Taylor C0 per relation: a box is kept iff every form passes its relation
        keep_o = np.ones(t.shape[0], np.uint8)
        for f, p in enumerate(polys):
            lo, hi, _ = oracle.taylor_boxes([p], dom, level, order, t)
            lo, hi = lo[0], hi[0]
            drop = {0: (lo > 0) | (hi < 0), 1: lo > 0, 2: hi < 0, 3: lo >= 0, 4: hi <= 0}[rel[f]]
            keep_o &= (~drop).astype(np.uint8)
    keep, _, nr = vx.csf_taylor_level(sysv, c, dom, order, vx.FP32)
    assert np.array_equal(keep.cpu().numpy(), keep_o)
    keep64, _, nr64 = vx.csf_taylor_level(sysv, c, dom, order, vx.FP64)
    assert np.array_equal(keep64.cpu().numpy(), keep_o) and nr64 == 0
    assert nr < t.shape[0] // 2  # integer coefficients on dyadic boxes: many exact ends


@pytest.mark.parametrize("case", ["circle", "rand2", "rand3"])
def test_taylor_certified_binary32_c1_level(vx, case):
    circle = (np.array([[2, 0], [0, 2], [0, 0]], dtype=np.int32), np.array([1.0, 1.0, -0.5]))
    poly, k, level = {"circle": (circle, 2, 6), "rand2": (synth.random_small(2, 8, 1, 41)[0], 2, 6),
                      "rand3": (synth.kostlan_poly(3, 7, 42), 3, 4)}[case]
    dom = synth.cube(k)
    side = 1 << level
    t = np.stack(np.meshgrid(*[np.arange(side)] * k, indexing="ij"), -1).reshape(-1, k)
    t = np.ascontiguousarray(t.astype(np.int32))
    _, _, keep_o = oracle.taylor_boxes([poly], dom, level, 2, t)
    inc_o = oracle.c1_boxes(poly, dom, level, oracle.C1_TAYLOR, t, 2)
    sysv = vx.System([poly])
    c = vx.csf_build(k, level, _dev(t))
    keep, inc, nr = vx.csf_taylor_level(sysv, c, dom, 2, vx.FP32, c1=True)
    keep = keep.cpu().numpy()
    inc = inc.cpu().numpy()
    assert np.array_equal(keep, keep_o)
    assert np.array_equal(inc[keep == 1], inc_o[keep_o == 1])
    if case == "circle":  # exact zeros of the form at dyadic points: binary64 decides those
        assert nr > 0


@pytest.mark.parametrize("case", ["taylor-c0", "taylor-c1", "vertex-c1"])
def test_taylor_certified_binary32_enclosure_equals_oracle(vx, case):
    if case == "taylor-c0":
        polys = [synth.kostlan_poly(3, 8, 51), synth.kostlan_poly(3, 8, 52)]
        ref = oracle.enclose_taylor(polys, synth.cube(3), 6, 2)
        r = vx.enclose(polys, synth.cube(3), 6, vx.make_opts(vx.FP32, taylor_order=2))
    else:
        poly = synth.random_small(2, 9, 1, 53)[0]
        kind = (oracle.C1_TAYLOR, vx.C1_TAYLOR) if case == "taylor-c1" else \
            (oracle.C1_VERTEX, vx.C1_VERTEX)
        ref = oracle.enclose_c1(poly, synth.cube(2), 10, kind[0], 4, taylor_order=2)
        r = vx.enclose([poly], synth.cube(2), 10,
                       vx.make_opts(vx.FP32, taylor_order=2, c1=kind[1], c1_level=4))
        lev, tup = r.included()
        assert np.array_equal(lev, ref["inc_levels"])
        assert np.array_equal(tup, ref["inc_tuples"])
    assert np.array_equal(r.boxes(), ref["tuples"])
    st = r.stats()
    assert np.array_equal(st["tested"], ref["tested"])
    assert np.array_equal(st["kept"], ref["kept"])
