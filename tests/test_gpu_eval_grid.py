"""vx_csf_eval_grid: Algorithm 2 on explicit per-axis interval lists, against the oracle.

- random interval lists (straddling 0, negative, degenerate points): binary64 values and keep
  bit-exact to orc_eval_grid; certified binary32 keep equal to binary64's; midpoint-radius a
  superset;
- the real special case of the DFT identity of Sec. 3.1 (corrected form): with
  X_j = {[1,1], [-1,-1]} a multilinear polynomial's values on the 2^k sign vectors are the
  Walsh-Hadamard transform of its coefficients, exactly.
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


def _lists(k, n, seed):
    """n intervals per axis: random dyadic ends in [-2, 2], some degenerate, some around 0."""
    st = synth.Stream(seed)
    out = []
    for _ in range(k):
        a = st.uniform_int(-512, 512, n).astype(np.float64) / 256.0
        w = st.uniform_int(0, 96, n).astype(np.float64) / 256.0
        w[::7] = 0.0  # points
        out.append((a, a + w))
    return out


def _dev(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("k,d,npoly,level,n,seed", [(2, 9, 2, 5, 700, 61), (3, 6, 2, 4, 1500, 62),
                                                    (3, 11, 1, 3, 400, 63), (1, 30, 1, 6, 64, 64)])
def test_interval_lists_match_oracle(vx, k, d, npoly, level, n, seed):
    import torch

    polys = synth.random_small(k, d, npoly, seed)
    t = synth.random_tuples(k, level, n, seed + 1)
    xl = _lists(k, 1 << level, seed + 2)
    lo_o, hi_o, keep_o, _ = oracle.eval_grid(polys, xl, t)
    sysv = vx.System(polys)
    c = vx.csf_build(k, level, _dev(t))
    dx = [(_dev(a), _dev(b)) for a, b in xl]
    keep, lo, hi = vx.csf_eval_grid(sysv, c, dx, vx.FP64, values=True)
    torch.cuda.synchronize()
    assert np.array_equal(lo.cpu().numpy(), lo_o)
    assert np.array_equal(hi.cpu().numpy(), hi_o)
    assert np.array_equal(keep.cpu().numpy(), keep_o)
    k32 = vx.csf_eval_grid(sysv, c, dx, vx.FP32)
    assert torch.equal(k32, keep)
    km = vx.csf_eval_grid(sysv, c, dx, vx.FP32_MIDRAD)
    assert torch.all(km >= keep)


@pytest.mark.parametrize("k,seed", [(3, 71), (4, 72)])
def test_walsh_hadamard_special_case(vx, k, seed):
    import torch

    n = 1 << k
    u = synth.Stream(seed).uniform_int(-50, 50, n).astype(np.float64)
    # F = sum_e u[sum_m e_m 2^(m-1)] prod x_m^(e_m), e in {0,1}^k
    exps = np.array([[(i >> m) & 1 for m in range(k)] for i in range(n)], dtype=np.int32)
    polys = [(exps, u)]
    # boxes: every sign vector; label 0 -> [1,1], label 1 -> [-1,-1] on every axis
    t = np.array([[(j >> (k - 1 - m)) & 1 for m in range(k)] for j in range(n)], dtype=np.int32)
    xl = [(np.array([1.0, -1.0]), np.array([1.0, -1.0]))] * k
    sysv = vx.System(polys)
    c = vx.csf_build(k, 1, _dev(t))
    dx = [(_dev(a), _dev(b)) for a, b in xl]
    _, lo, hi = vx.csf_eval_grid(sysv, c, dx, vx.FP64, values=True)
    lo = lo.cpu().numpy()[0]
    hi = hi.cpu().numpy()[0]
    # Walsh-Hadamard: value at sign vector s = sum_i u[i] prod_m s_m^(bit m of i)
    expect = np.array([sum(u[i] * np.prod([(-1.0 if t[j][m] else 1.0) ** ((i >> m) & 1)
                                           for m in range(k)]) for i in range(n))
                       for j in range(n)])
    H = np.array([[1.0]])
    for _ in range(k):
        H = np.block([[H, H], [H, -H]])
    # the same numbers by the Sylvester-Hadamard matrix (bit order of the sign vectors reversed)
    rev = [int(format(j, "0%db" % k)[::-1], 2) for j in range(n)]
    assert np.array_equal(expect, (H @ u)[rev])
    assert np.array_equal(lo, expect) and np.array_equal(hi, expect)
    _, l32, h32 = vx.csf_eval_grid(sysv, c, dx, vx.FP32, values=True)
    assert np.array_equal(l32.cpu().numpy()[0], expect)
    assert np.array_equal(h32.cpu().numpy()[0], expect)
    torch.cuda.synchronize()


def test_rejects_short_lists(vx):
    polys = synth.random_small(2, 3, 1, 80)
    t = synth.random_tuples(2, 3, 20, 81)
    sysv = vx.System(polys)
    c = vx.csf_build(2, 3, _dev(t))
    xl = _lists(2, 7, 82)  # 7 < 2^3
    with pytest.raises(vx.VxError) as e:
        vx.csf_eval_grid(sysv, c, [(_dev(a), _dev(b)) for a, b in xl], vx.FP64)
    assert e.value.code == vx.EINVAL


def test_nesting_order_hand_derived(vx):
    """Algorithm 2's order (x_1 at the root, Sec. 2.2) on non-degenerate boxes: the GPU's
    binary64 values equal the hand-derived enclosures of golden/nesting_order.json, which no
    other nesting order gives."""
    import json
    import os

    import torch

    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                           "nesting_order.json")) as f:
        cases = json.load(f)["cases"]
    for c in cases:
        polys = [(np.asarray(c["exps"], dtype=np.int32), np.asarray(c["coefs"], dtype=np.float64))]
        box = np.asarray(c["box"], dtype=np.float64)
        k = box.shape[0]
        sysv = vx.System(polys)
        cs = vx.csf_build(k, 0, _dev(np.zeros((1, k), dtype=np.int32)))
        dx = [(_dev(box[i, :1].copy()), _dev(box[i, 1:].copy())) for i in range(k)]
        _, lo, hi = vx.csf_eval_grid(sysv, cs, dx, vx.FP64, values=True)
        torch.cuda.synchronize()
        assert (float(lo[0, 0]), float(hi[0, 0])) == tuple(c["expected"]), c["name"]
