"""C0 on the Taylor form (Def. 3) on the GPU, against the oracle.

- the form's interval on every box, bit for bit (binary64), orders 1-3, k = 1..4, several
  polynomials, a non-symmetric dyadic domain, boxes at the domain's edges;
- Algorithm 3 with the Taylor criterion: the same boxes and per-level counts as the oracle's;
- what it refuses: binary32 modes, orders with more terms than VX_MAXPOLY, batches.
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
    with pytest.raises(vx.VxError) as e:
        vx.enclose(polys, synth.cube(3), 3, vx.make_opts(vx.FP32, taylor_order=2))
    assert e.value.code == vx.EINVAL
    with pytest.raises(vx.VxError) as e:  # C(3+3, 3) = 20 > 16 terms
        vx.enclose(polys, synth.cube(3), 3, vx.make_opts(vx.FP64, taylor_order=3))
    assert e.value.code == vx.EINVAL
    with pytest.raises(vx.VxError) as e:
        vx.enclose_batch([(polys, synth.cube(3), 3)], vx.make_opts(vx.FP64, taylor_order=1))
    assert e.value.code == vx.EINVAL
