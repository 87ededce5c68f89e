"""VX_FP32 with recheck_last: the error band's boxes stay in S below the last level and only
the last level is re-decided in binary64.  C0 on interval Horner is inclusion-isotone over the
exact grids (pinned on the oracle: pruning at coarser levels changes no final box), so the
final boxes must be exactly the oracle's, while every level in between keeps at least the
oracle's boxes.

- single systems: a Kostlan curve, integer polynomials whose values at grid points are exact
  (many boxes in the band), a system with relations and interval coefficients, k = 2 and 4;
- the batch engine, where only the finishing trees' band is re-decided;
- what it refuses: binary64 or midpoint-radius modes, the Taylor form, C1.
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


CASES = {
    "curve-d16": ([synth.kostlan_poly(3, 16, 1401), synth.kostlan_poly(3, 16, 1402)], None, None,
                  synth.cube(3), 7),
    "integer-k3": (synth.random_small(3, 6, 2, 1403), None, None, synth.cube(3), 7),
    "integer-k2": (synth.random_small(2, 9, 1, 1404), None, None, synth.cube(2), 9),
    "k4-table1": (synth.table1(4, 6, "curves").polys, None, None, synth.cube(4, -2.0, 2.0), 5),
    "relations": (synth.random_small(3, 5, 3, 1405), None, [0, 1, 4], synth.cube(3), 6),
}
_R = synth.robotics(5)
CASES["robotics-R"] = (_R.polys, _R.his, _R.rel, _R.domain, 5)


@pytest.mark.parametrize("case", sorted(CASES))
def test_recheck_last_final_boxes_equal_oracle(vx, case):
    polys, his, rel, dom, depth = CASES[case]
    ref = oracle.enclose_gen(polys, dom, depth, his=his, rel=rel)
    sysv = vx.System(polys, his=his, rel=rel) if (his or rel) else vx.System(polys)
    every = vx.enclose_system(sysv, dom, depth, vx.make_opts(vx.FP32))
    last = vx.enclose_system(sysv, dom, depth, vx.make_opts(vx.FP32, recheck_last=True))
    try:
        assert np.array_equal(last.boxes(), ref["tuples"])
        assert np.array_equal(every.boxes(), ref["tuples"])
        st, sr = last.stats(), every.stats()
        assert np.array_equal(sr["kept"], ref["kept"])
        assert (st["recheck"][:depth] == 0).all()
        assert (st["kept"][:depth] >= ref["kept"][:depth]).all()
        assert (st["tested"] >= ref["tested"]).all()
        assert st["kept"][depth] == ref["kept"][depth]
    finally:
        last.free()
        every.free()


def test_recheck_last_batch_equals_oracle(vx):
    systems = []
    for i in range(8):
        if i % 2 == 0:
            systems.append((synth.random_small(2, 7, 1, 1410 + i), synth.cube(2), 6 + i % 3))
        else:
            systems.append(([synth.kostlan_poly(3, 8, 1420 + i), synth.kostlan_poly(3, 8, 1430 + i)],
                            synth.cube(3), 4 + i % 3))
    res = vx.enclose_batch(systems, vx.make_opts(vx.FP32, recheck_last=True), nworkers=4)
    for (polys, dom, depth), r in zip(systems, res):
        ref = oracle.enclose(polys, dom, depth)
        assert np.array_equal(r.boxes(), ref["tuples"])
        st = r.stats()
        assert (st["recheck"][:depth] == 0).all()
        assert (st["kept"] >= ref["kept"]).all()


def test_recheck_last_refusals(vx):
    polys = [synth.kostlan_poly(3, 6, 1440)]
    dom = synth.cube(3)
    for opts in (vx.make_opts(vx.FP64, recheck_last=True),
                 vx.make_opts(vx.FP32_MIDRAD, fp64_final=True, recheck_last=True),
                 vx.make_opts(vx.FP32, taylor_order=2, recheck_last=True),
                 vx.make_opts(vx.FP32, taylor_order=2, c1=vx.C1_TAYLOR, c1_level=2,
                              recheck_last=True)):
        with pytest.raises(RuntimeError, match="recheck_last"):
            vx.enclose(polys, dom, 4, opts)
    with pytest.raises(RuntimeError, match="recheck_last"):
        vx.enclose_batch([(polys, dom, 4)], vx.make_opts(vx.FP64, recheck_last=True))
