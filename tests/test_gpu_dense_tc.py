"""The dense full-grid level on the tensor cores (vx_dense_*), against the oracle.

- values: on every box, the device's midpoint-radius enclosure contains the oracle's
  mode-wise power form (binary64, no margins) and is not much wider;
- prefilter: its kept boxes are a superset of the boxes binary64 interval Horner keeps on the
  full grid (vx_csf_eval_level, itself bit-exact to the oracle);
- the exactly decided level (prefilter, then the survivors through the interval path) equals
  the full-grid keep of binary64, in VX_FP64 and in certified VX_FP32, bit for bit;
- the degree-256 boundary of the x3 tile (more than 128 tensor-memory columns), several
  polynomials (AND of their masks), a non-symmetric dyadic domain, the smallest level;
- a bounded wait that gives up is reported and leaves the context usable.
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


def _all_tuples(level):
    n = 1 << level
    g = np.meshgrid(*[np.arange(n, dtype=np.int32)] * 3, indexing="ij")
    return np.stack([x.reshape(-1) for x in g], axis=1)


def _sparse_high_x3(seed):
    """A sparse trivariate polynomial of degree 130 in x3 (more than 128 columns of the
    second contraction) and small degree in x1, x2."""
    st = synth.Stream(seed)
    e = [[0, 0, 0], [1, 0, 0], [0, 2, 0], [0, 0, 130], [2, 1, 7], [0, 1, 64], [1, 1, 129],
         [3, 0, 1]]
    c = st.normal(len(e))
    return np.array(e, dtype=np.int32), c


CASES = {
    "gauss-d12": (lambda: [synth.gaussian_tensor_poly(3, 12, 501)], synth.cube(3), 5),
    "gauss-d20-l6": (lambda: [synth.gaussian_tensor_poly(3, 20, 502)], synth.cube(3), 6),
    "int-d9": (lambda: synth.random_small(3, 9, 1, 503), synth.cube(3), 6),
    "x3-130": (lambda: [_sparse_high_x3(504)], synth.cube(3), 5),
    "box-dom": (lambda: [synth.gaussian_tensor_poly(3, 10, 505)],
                np.array([-1.0, 3.0, 0.0, 2.0, -2.0, 2.0]), 6),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_values_contain_the_power_form(vx, name):
    import torch

    make, dom, level = CASES[name]
    polys = make()
    plan = vx.DensePlan(vx.System(polys), level, dom)
    mid, rad = plan.values(0)
    torch.cuda.synchronize()
    mid = mid.double().cpu().numpy()
    rad = rad.double().cpu().numpy()
    t = _all_tuples(level)
    if t.shape[0] > 40000:  # the oracle is slow: a seeded sample of boxes
        sel = np.unique(synth.Stream(7).uniform_int(0, t.shape[0] - 1, 40000))
        t, mid, rad = t[sel], mid[sel], rad[sel]
    mo, ro = oracle.dense_powerform(polys[0], dom, level, t)
    slack = 1e-9 * (np.abs(mo) + ro) + 1e-300
    assert np.all(np.isfinite(mid)) and np.all(np.isfinite(rad))
    assert np.all(mid - rad <= mo - ro + slack), "device enclosure misses the lower end"
    assert np.all(mo + ro - slack <= mid + rad), "device enclosure misses the upper end"
    # the rounding margins are small next to the exact power form's width
    assert np.median(rad / np.maximum(ro, 1e-300)) < 1.25
    plan.free()


def _full_grid_keep(vx, sysv, dom, level, mode):
    c = vx.csf_full_grid(3, level)
    k = vx.csf_eval_level(sysv, c, dom, mode)
    c.free()
    return k


@pytest.mark.parametrize("name", sorted(CASES))
def test_prefilter_superset_and_exact_level(vx, name):
    import torch

    make, dom, level = CASES[name]
    polys = make()
    sysv = vx.System(polys)
    plan = vx.DensePlan(sysv, level, dom)
    nbox = 1 << (3 * level)
    keep64 = _full_grid_keep(vx, sysv, dom, level, vx.FP64)
    pre = vx.mask_to_bool(plan.prefilter(), nbox)
    assert torch.all(pre | (keep64 == 0)), "the prefilter dropped a box binary64 keeps"
    k64, ns = plan.level_keep(vx.make_opts(vx.FP64))
    assert ns == int(pre.sum().item())
    assert torch.equal(k64, keep64)
    k32, _ = plan.level_keep(vx.make_opts(vx.FP32))
    assert torch.equal(k32, keep64)
    km, _ = plan.level_keep(vx.make_opts(vx.FP32_MIDRAD))
    assert torch.all(km >= keep64)
    plan.free()


def test_two_polynomials_and_of_masks(vx):
    import torch

    polys = [synth.gaussian_tensor_poly(3, 9, 511), synth.random_small(3, 7, 1, 512)[0]]
    dom = synth.cube(3)
    level = 6
    sysv = vx.System(polys)
    plan = vx.DensePlan(sysv, level, dom)
    nbox = 1 << (3 * level)
    pre = vx.mask_to_bool(plan.prefilter(), nbox)
    for f, p in enumerate(polys):
        one = vx.DensePlan(vx.System([p]), level, dom)
        pf = vx.mask_to_bool(one.prefilter(), nbox)
        assert torch.all(pre <= pf)
        one.free()
    keep64 = _full_grid_keep(vx, sysv, dom, level, vx.FP64)
    assert torch.all(pre | (keep64 == 0))
    k32, _ = plan.level_keep(vx.make_opts(vx.FP32))
    assert torch.equal(k32, keep64)
    plan.free()


def test_dense_sweep_cell_level7(vx):
    """The dense-sweep workload's degree-32 tensor on its 128^3 grid."""
    import torch

    s = synth.dense_sweep(32)
    sysv = vx.System(s.polys)
    level = 7
    plan = vx.DensePlan(sysv, level, s.domain)
    keep64 = _full_grid_keep(vx, sysv, s.domain, level, vx.FP64)
    pre = vx.mask_to_bool(plan.prefilter(), 1 << (3 * level))
    assert torch.all(pre | (keep64 == 0))
    k32, ns = plan.level_keep(vx.make_opts(vx.FP32))
    assert torch.equal(k32, keep64)
    assert ns < (1 << (3 * level)) // 2  # the prefilter removes most boxes
    plan.free()


def test_rejects_what_it_does_not_handle(vx):
    polys2 = synth.random_small(2, 5, 1, 520)
    with pytest.raises(vx.VxError) as e:
        vx.DensePlan(vx.System(polys2), 6, synth.cube(2))
    assert e.value.code == vx.EINVAL
    polys3 = [synth.gaussian_tensor_poly(3, 4, 521)]
    with pytest.raises(vx.VxError) as e:
        vx.DensePlan(vx.System(polys3), 4, synth.cube(3))
    assert e.value.code == vx.EINVAL


def test_bounded_wait_gives_up_cleanly(vx):
    import torch

    polys = [synth.gaussian_tensor_poly(3, 12, 530)]
    sysv = vx.System(polys)
    plan = vx.DensePlan(sysv, 6, synth.cube(3))
    good = plan.prefilter().clone()
    vx.lib().vx_set_wait_limit(0)
    try:
        with pytest.raises(vx.VxError) as e:
            plan.prefilter()
        assert e.value.code == vx.ETIMEOUT
    finally:
        vx.lib().vx_set_wait_limit(-1)
    again = plan.prefilter()
    assert torch.equal(again, good)
    plan.free()


def test_prefilter_graph_replay(vx):
    """The prefilter's launches are captured once per mask buffer and replayed: repeated calls
    on one buffer, and a call on another buffer, give the same bits."""
    import torch

    polys = [synth.gaussian_tensor_poly(3, 16, 540), synth.gaussian_tensor_poly(3, 9, 541)]
    plan = vx.DensePlan(vx.System(polys), 6, synth.cube(3))
    m = torch.empty((1 << 18) // 32, dtype=torch.int32, device="cuda")
    first = plan.prefilter(m).clone()
    for _ in range(3):
        m.fill_(0)
        assert torch.equal(plan.prefilter(m), first)
    other = torch.full_like(m, -1)
    assert torch.equal(plan.prefilter(other), first)
    k1, n1 = plan.level_keep(vx.make_opts(vx.FP32))
    k2, n2 = plan.level_keep(vx.make_opts(vx.FP32))
    assert n1 == n2 and torch.equal(k1, k2)
    plan.free()


def _tensor_poly(d, coef_of):
    """The full (d+1)^3 tensor with coefficient coef_of(a1, a2, a3, index)."""
    g = np.meshgrid(*[np.arange(d + 1, dtype=np.int32)] * 3, indexing="ij")
    e = np.stack([x.reshape(-1) for x in g], axis=1)
    return e, coef_of(e)


def _adversarial(name):
    d = 128
    st = synth.Stream({"alternating": 601, "spread": 602, "equal-random-signs": 603}[name])
    if name == "alternating":  # equal magnitudes, signs (-1)^|a|: heavy cancellation near x = 1
        return _tensor_poly(d, lambda e: np.where(e.sum(axis=1) % 2 == 0, 1.0, -1.0))
    if name == "spread":  # magnitudes 2^u, u uniform in [-60, 60], random signs
        def coef(e):
            u = st.uniform_int(-60, 60, e.shape[0]).astype(np.float64)
            s = np.where(st.uniform_int(0, 1, e.shape[0]) == 0, 1.0, -1.0)
            return s * np.ldexp(1.0, u.astype(np.int64))
        return _tensor_poly(d, coef)
    def coef(e):  # equal magnitudes, random signs
        return np.where(st.uniform_int(0, 1, e.shape[0]) == 0, 1.0, -1.0)
    return _tensor_poly(d, coef)


@pytest.mark.parametrize("name", ["alternating", "spread", "equal-random-signs"])
def test_tensor_core_enclosure_at_its_worst_cases(vx, name):
    """Property 1's contractions on the tensor cores at degree 128 (an inner dimension of 136)
    with coefficients chosen against the accumulation model of the TF32 midpoints: equal
    magnitudes with alternating or random signs (cancellation: midpoints far below the sums
    of |products|) and magnitudes spread over 2^-60 .. 2^60.  On sampled boxes the device's
    <mid, rad> contains the oracle's margin-free mode-wise power form, and the midpoint error
    uses less than half of the radius the device adds for rounding (|mid - m| <= (rad - r) / 2):
    the margins of the model hold with a factor 2 to spare."""
    import torch

    polys = [_adversarial(name)]
    dom, level = synth.cube(3), 5
    plan = vx.DensePlan(vx.System(polys), level, dom)
    mid, rad = plan.values(0)
    torch.cuda.synchronize()
    mid = mid.double().cpu().numpy()
    rad = rad.double().cpu().numpy()
    t = _all_tuples(level)
    sel = np.unique(synth.Stream(17).uniform_int(0, t.shape[0] - 1, 300))
    # the boxes next to x = (1, 1, 1) and x = (-1, -1, -1), where the cancellation is largest
    side = 1 << level
    corner = [(side - 1 - i) * side * side + (side - 1 - j) * side + (side - 1 - k)
              for i in range(3) for j in range(3) for k in range(3)]
    sel = np.unique(np.concatenate([sel, corner, np.arange(27)]))
    t, mid, rad = t[sel], mid[sel], rad[sel]
    mo, ro = oracle.dense_powerform(polys[0], dom, level, t)
    assert np.all(np.isfinite(mid)) and np.all(np.isfinite(rad))
    slack = 1e-12 * (np.abs(mo) + ro) + 1e-300
    assert np.all(mid - rad <= mo - ro + slack), "device enclosure misses the lower end"
    assert np.all(mo + ro - slack <= mid + rad), "device enclosure misses the upper end"
    extra = rad - ro
    used = np.abs(mid - mo) / np.maximum(extra, 1e-300)
    print("%s: largest share of the rounding radius used by the midpoint error %.3g "
          "(median %.3g)" % (name, used.max(), np.median(used)))
    assert used.max() < 0.5
    plan.free()
