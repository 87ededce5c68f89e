"""Systems of equations and inequalities with interval coefficients on the GPU, and k = 5, 6
variables, against the oracle.

- every relation (F = 0, <= 0, >= 0, < 0, > 0) with interval coefficients, one level's values
  and keep bit-exact in binary64, keep equal in certified binary32, a superset in
  midpoint-radius binary32;
- k = 5 and 6 variables: level values bit-exact, Algorithm 3 identical;
- the systems (R) and (A) of the applications section: Algorithm 3 identical to the oracle in
  binary64 and certified binary32 ((A) ends with no box, as the paper reports), and with the
  Taylor form for (R);
- what it refuses: an unknown relation, an interval with lower > upper end, a tensor-core plan
  or C1 on a system with an inequality.
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


def _widen(polys, seed, frac=0.5):
    """Upper ends: some coefficients become intervals [c, c + u] with dyadic u."""
    st = synth.Stream(seed)
    his = []
    for e, c in polys:
        u = st.uniform_int(0, 4, c.shape[0]).astype(np.float64) / 8.0
        mask = st.unit(c.shape[0]) < frac
        his.append(c + np.where(mask, u, 0.0))
    return his


@pytest.mark.parametrize("k,d,level,n,seed", [(2, 8, 5, 900, 1), (3, 6, 4, 3000, 2),
                                              (4, 4, 3, 3000, 3)])
def test_relations_and_intervals_one_level(vx, k, d, level, n, seed):
    import torch

    polys = synth.random_small(k, d, 5, seed)
    his = _widen(polys, seed + 10)
    rel = [vx.EQ, vx.LE, vx.GE, vx.LT, vx.GT]
    t = synth.random_tuples(k, level, n, seed + 1)
    dom = synth.cube(k)
    lo_o, hi_o, keep_o, _ = oracle.eval_csf_gen(polys, dom, level, t, his=his, rel=rel)
    sysv = vx.System(polys, his=his, rel=rel)
    c = vx.csf_build(k, level, _dev(t))
    keep, lo, hi = vx.csf_eval_level(sysv, c, dom, vx.FP64, values=True)
    torch.cuda.synchronize()
    assert np.array_equal(lo.cpu().numpy(), lo_o)
    assert np.array_equal(hi.cpu().numpy(), hi_o)
    assert np.array_equal(keep.cpu().numpy(), keep_o)
    assert 0 < keep_o.sum() < len(keep_o)
    k32 = vx.csf_eval_level(sysv, c, dom, vx.FP32)
    assert torch.equal(k32, keep)
    km = vx.csf_eval_level(sysv, c, dom, vx.FP32_MIDRAD)
    assert torch.all(km >= keep)
    # each relation on its own
    for f, r in enumerate(rel):
        _, _, ko, _ = oracle.eval_csf_gen([polys[f]], dom, level, t, his=[his[f]], rel=[r])
        one = vx.System([polys[f]], his=[his[f]], rel=[r])
        for mode in (vx.FP64, vx.FP32):
            assert np.array_equal(vx.csf_eval_level(one, c, dom, mode).cpu().numpy(), ko)


@pytest.mark.parametrize("k,d,level,n,seed", [(5, 3, 3, 4000, 4), (6, 2, 2, 3000, 5),
                                              (6, 3, 2, 2500, 6)])
def test_five_and_six_variables_one_level(vx, k, d, level, n, seed):
    import torch

    polys = synth.random_small(k, d, 2, seed)
    t = synth.random_tuples(k, level, n, seed + 1)
    dom = synth.cube(k)
    lo_o, hi_o, keep_o, _ = oracle.eval_csf(polys, dom, level, t)
    sysv = vx.System(polys)
    c = vx.csf_build(k, level, _dev(t))
    keep, lo, hi = vx.csf_eval_level(sysv, c, dom, vx.FP64, values=True)
    torch.cuda.synchronize()
    assert np.array_equal(lo.cpu().numpy(), lo_o)
    assert np.array_equal(hi.cpu().numpy(), hi_o)
    assert np.array_equal(keep.cpu().numpy(), keep_o)
    assert torch.equal(vx.csf_eval_level(sysv, c, dom, vx.FP32), keep)


@pytest.mark.parametrize("k,d,depth,seed", [(5, 3, 4, 7), (6, 2, 3, 8)])
def test_five_and_six_variables_enclosure(vx, k, d, depth, seed):
    polys = [synth.kostlan_poly(k, d, 10 * seed + p) for p in range(2)]
    dom = synth.cube(k)
    ref = oracle.enclose(polys, dom, depth)
    for mode in (vx.FP64, vx.FP32):
        r = vx.enclose(polys, dom, depth, vx.make_opts(mode))
        assert np.array_equal(r.boxes(), ref["tuples"])
        st = r.stats()
        assert np.array_equal(st["tested"], ref["tested"])
        assert np.array_equal(st["kept"], ref["kept"])
    assert ref["tuples"].shape[0] > 0


def _enclose_system(vx, s, depth, opts):
    sysv = vx.System(s.polys, his=s.his, rel=s.rel)
    r = vx.enclose_system(sysv, s.domain, depth, opts)
    return r


@pytest.mark.parametrize("depth", [4, 5])
def test_robotics_R_equals_oracle(vx, depth):
    s = synth.robotics()
    ref = oracle.enclose_gen(s.polys, s.domain, depth, s.his, s.rel)
    for mode in (vx.FP64, vx.FP32):
        r = _enclose_system(vx, s, depth, vx.make_opts(mode))
        assert np.array_equal(r.boxes(), ref["tuples"])
        assert np.array_equal(r.stats()["kept"], ref["kept"])
    r = _enclose_system(vx, s, depth, vx.make_opts(vx.FP32_MIDRAD, fp64_final=True))
    assert np.array_equal(r.boxes(), ref["tuples"])


def test_robotics_R_taylor_equals_oracle(vx):
    s = synth.robotics()
    ref = oracle.enclose_gen(s.polys, s.domain, 4, s.his, s.rel, taylor_order=2)
    r = _enclose_system(vx, s, 4, vx.make_opts(vx.FP64, taylor_order=2))
    assert np.array_equal(r.boxes(), ref["tuples"])
    assert np.array_equal(r.stats()["kept"], ref["kept"])


def test_automatic_A_equals_oracle_and_is_empty(vx):
    s = synth.automatic()
    ref = oracle.enclose_gen(s.polys, s.domain, 6, s.his, s.rel)
    assert ref["tuples"].shape[0] == 0
    for mode in (vx.FP64, vx.FP32):
        r = _enclose_system(vx, s, 6, vx.make_opts(mode))
        st = r.stats()
        assert np.array_equal(st["tested"], ref["tested"])
        assert np.array_equal(st["kept"], ref["kept"])
        assert r.boxes().shape[0] == 0


def test_refusals(vx):
    polys = synth.random_small(3, 3, 2, 40)
    with pytest.raises(vx.VxError) as e:
        vx.System(polys, rel=[0, 7])
    assert e.value.code == vx.EINVAL
    with pytest.raises(vx.VxError) as e:
        vx.System(polys, his=[polys[0][1] - 1.0, None])
    assert e.value.code == vx.EINVAL
    ineq = vx.System([synth.gaussian_tensor_poly(3, 12, 41)], rel=[vx.LE])
    with pytest.raises(vx.VxError) as e:
        vx.DensePlan(ineq, 6, synth.cube(3))
    assert e.value.code == vx.EINVAL
    with pytest.raises(vx.VxError) as e:
        vx.enclose_system(ineq, synth.cube(3), 3, vx.make_opts(vx.FP64, c1=vx.C1_VERTEX))
    assert e.value.code == vx.EINVAL
