"""The inclusion criterion C1 (Sec. 3.2) and Algorithm 3 with it on the GPU, against the oracle.

- C1 per box, both tests (vertex signs; the Taylor form of order 2 and 3 at the extremal
  vertices), k = 1..4, bit-exact decisions;
- Algorithm 3 with C0 (interval Horner or Taylor) and C1 from a threshold level: the same
  certified boxes with their levels, the same boxes left at the last level and the same
  per-level counts as the oracle (the circle, whose C1 never certifies the boxes touching it
  at a dyadic vertex; random polynomials; a Table-1 hypersurface);
- what it refuses: several equations, midpoint-radius binary32, the Taylor test without a Taylor form.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2406_09857_gb300 import synth

pytestmark = pytest.mark.gpu

CIRCLE = (np.array([[2, 0], [0, 2], [0, 0]], dtype=np.int32), np.array([1.0, 1.0, -0.5]))


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


@pytest.mark.parametrize("k,d,level,n,seed,dom", [
    (1, 15, 7, 128, 1, None),
    (2, 9, 6, 1500, 2, None),
    (2, 6, 5, 800, 3, [-2.0, 2.0, 0.0, 1.0]),
    (3, 6, 4, 3000, 4, None),
    (4, 4, 3, 3000, 5, None),
])
@pytest.mark.parametrize("kind,order", [("vertex", 0), ("taylor", 2), ("taylor", 3)])
def test_c1_boxes_bit_exact(vx, k, d, level, n, seed, dom, kind, order):
    if kind == "taylor" and math.comb(order + k, k) > 16:
        pytest.skip("C(m+k, k) multi-indices exceed VX_MAXPOLY")
    poly = synth.random_small(k, d, 1, seed)[0]
    dom = synth.cube(k) if dom is None else np.asarray(dom)
    t = synth.random_tuples(k, level, n, seed + 1)
    ok = oracle.C1_VERTEX if kind == "vertex" else oracle.C1_TAYLOR
    ref = oracle.c1_boxes(poly, dom, level, ok, t, order)
    sysv = vx.System([poly])
    c = vx.csf_build(k, level, _dev(t))
    got = vx.csf_c1(sysv, c, dom, vx.C1_VERTEX if kind == "vertex" else vx.C1_TAYLOR, order)
    assert np.array_equal(got.cpu().numpy(), ref)
    assert ref.sum() > 0


def _check_enclosure(vx, poly, dom, depth, kind, c1_level, order):
    ok = oracle.C1_VERTEX if kind == "vertex" else oracle.C1_TAYLOR
    ref = oracle.enclose_c1(poly, dom, depth, ok, c1_level, taylor_order=order)
    opts = vx.make_opts(vx.FP64, taylor_order=order,
                        c1=vx.C1_VERTEX if kind == "vertex" else vx.C1_TAYLOR, c1_level=c1_level)
    r = vx.enclose([poly], dom, depth, opts)
    lev, tup = r.included()
    assert np.array_equal(lev, ref["inc_levels"])
    assert np.array_equal(tup, ref["inc_tuples"])
    assert np.array_equal(r.boxes(), ref["tuples"])
    st = r.stats()
    assert np.array_equal(st["tested"], ref["tested"])
    assert np.array_equal(st["kept"], ref["kept"])
    assert np.array_equal(np.bincount(lev, minlength=depth + 1), ref["included"])
    return ref


@pytest.mark.parametrize("case", ["circle-vertex", "circle-taylor", "rand2-vertex-horner",
                                  "rand2-taylor3", "rand3-vertex-taylor2", "rand3-taylor",
                                  "rand1-vertex", "rand4-taylor"])
def test_enclosure_with_c1_equals_oracle(vx, case):
    cases = {
        "circle-vertex": (CIRCLE, synth.cube(2), 10, "vertex", 3, 0),
        "circle-taylor": (CIRCLE, synth.cube(2), 10, "taylor", 2, 2),
        "rand2-vertex-horner": (synth.random_small(2, 9, 1, 21)[0], synth.cube(2), 10, "vertex",
                                4, 0),
        "rand2-taylor3": (synth.random_small(2, 8, 1, 22)[0], synth.cube(2), 10, "taylor", 3,
                          3),
        "rand3-vertex-taylor2": (synth.random_small(3, 5, 1, 23)[0], synth.cube(3), 6, "vertex",
                                 3, 2),
        "rand3-taylor": (synth.kostlan_poly(3, 8, 24), synth.cube(3), 6, "taylor", 3, 2),
        "rand1-vertex": (synth.kostlan_poly(1, 30, 27), synth.cube(1), 14, "vertex", 2, 0),
        "rand4-taylor": (synth.random_small(4, 3, 1, 26)[0], synth.cube(4), 4, "taylor", 2, 2),
    }
    poly, dom, depth, kind, c1_level, order = cases[case]
    ref = _check_enclosure(vx, poly, dom, depth, kind, c1_level, order)
    assert ref["inc_tuples"].shape[0] > 0


def test_table1_hypersurface_cell(vx):
    s = synth.table1(2, 20, "hypersurfaces")
    ref = _check_enclosure(vx, s.polys[0], s.domain, 12, "taylor", 7, 2)
    assert ref["inc_tuples"].shape[0] > 0


def test_refusals(vx):
    two = synth.random_small(2, 4, 2, 30)
    with pytest.raises(vx.VxError) as e:
        vx.enclose(two, synth.cube(2), 4, vx.make_opts(vx.FP64, c1=vx.C1_VERTEX))
    assert e.value.code == vx.EINVAL
    one = two[:1]
    with pytest.raises(vx.VxError) as e:
        vx.enclose(one, synth.cube(2), 4, vx.make_opts(vx.FP32_MIDRAD, c1=vx.C1_VERTEX))
    assert e.value.code == vx.EINVAL
    with pytest.raises(vx.VxError) as e:
        vx.enclose(one, synth.cube(2), 4, vx.make_opts(vx.FP64, c1=vx.C1_TAYLOR, taylor_order=1))
    assert e.value.code == vx.EINVAL
    with pytest.raises(vx.VxError) as e:
        vx.enclose(one, synth.cube(2), 4, vx.make_opts(vx.FP64, c1=7))
    assert e.value.code == vx.EINVAL
