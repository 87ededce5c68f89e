"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Bar: the binary64 path is bit-identical to the oracle (endpoints compared by value, so that
-0 == +0), CSF index arrays and kept sets are identical, and the binary32 midpoint-radius
path encloses the binary64 enclosure box by box (so it keeps a superset), with a binary64
last level giving exactly the binary64 set.
"""
import math

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


def dev(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    return t.cpu().numpy()


# ---------------------------------------------------------------------------------------
# CSF construction (Sec. 2.1) and Algorithm 3's split
# ---------------------------------------------------------------------------------------
@pytest.mark.parametrize("k,level,n,seed", [(1, 5, 20, 1), (2, 6, 700, 2), (3, 5, 5000, 3),
                                            (4, 4, 9000, 4), (3, 9, 40000, 5), (2, 1, 3, 6)])
def test_csf_build_matches_oracle(vx, k, level, n, seed):
    t = synth.random_tuples(k, level, n, seed)
    c = vx.csf_build(k, level, dev(t))
    kk, lv, N = c.nodes()
    N_ref, labs, ptrs = oracle.csf(t, k)
    assert kk == k and lv == level and N.tolist() == N_ref.tolist()
    for depth in range(1, k + 1):
        lab, ptr = c.export(depth)
        assert np.array_equal(host(lab), labs[depth - 1])
        if depth < k:
            assert np.array_equal(host(ptr), ptrs[depth - 1].astype(np.int32))
    assert np.array_equal(host(c.tuples()), t)


def test_csf_build_worked_example(vx):
    import json
    import os

    with open(os.path.join(os.path.dirname(__file__), "golden", "csf_worked_example.json")) as f:
        g = json.load(f)
    c = vx.csf_build(2, 3, dev(np.asarray(g["support"], dtype=np.int32)))
    assert c.nodes()[2].tolist() == g["N"]
    lab1, ptr1 = c.export(1)
    lab2, _ = c.export(2)
    assert host(lab1).tolist() == g["labels_depth1"]
    assert host(ptr1).tolist() == g["ptr_depth1"]
    assert host(lab2).tolist() == g["labels_depth2"]


def test_csf_build_rejects_bad_tuples(vx):
    bad = [np.array([[1, 0], [0, 0]], dtype=np.int32),   # not increasing
           np.array([[0, 0], [0, 0]], dtype=np.int32),   # duplicate
           np.array([[0, 0], [0, 8]], dtype=np.int32)]   # outside [0, 2^3)
    for t in bad:
        with pytest.raises(vx.VxError) as e:
            vx.csf_build(2, 3, dev(t))
        assert e.value.code == vx.EINVAL
    # the context is still fine afterwards
    c = vx.csf_build(2, 3, dev(np.array([[0, 1]], dtype=np.int32)))
    assert c.nodes()[2].tolist() == [1, 1]


def test_csf_build_empty(vx):
    import torch

    c = vx.csf_build(3, 4, torch.empty((0, 3), dtype=torch.int32, device="cuda"))
    assert c.nodes()[2].tolist() == [0, 0, 0]


def _children(kept, k):
    bits = np.array([[(b >> (k - 1 - c)) & 1 for c in range(k)] for b in range(1 << k)],
                    dtype=np.int32)
    ch = (2 * kept[:, None, :] + bits[None, :, :]).reshape(-1, k)
    order = np.lexsort(ch.T[::-1])
    return ch[order]


@pytest.mark.parametrize("k,level,n,p,seed", [(1, 6, 30, 0.5, 1), (2, 6, 900, 0.3, 2),
                                              (3, 5, 6000, 0.2, 3), (4, 3, 3000, 0.4, 4),
                                              (3, 7, 50000, 0.05, 5), (2, 4, 100, 0.0, 6),
                                              (2, 4, 100, 1.0, 7)])
def test_subdivide_matches_definition(vx, k, level, n, p, seed):
    t = synth.random_tuples(k, level, n, seed)
    keep = (synth.Stream(seed + 50).unit(t.shape[0]) < p).astype(np.uint8)
    c = vx.csf_build(k, level, dev(t))
    nxt = vx.csf_subdivide(c, dev(keep))
    kept = t[keep == 1]
    want = _children(kept, k) if kept.shape[0] else np.zeros((0, k), dtype=np.int32)
    _, lv, N = nxt.nodes()
    assert lv == level + 1
    assert np.array_equal(host(nxt.tuples()), want)
    # N_j(next) = 2^j N_j(kept), and the tree equals the one built from scratch
    Nk = oracle.csf(kept, k)[0] if kept.shape[0] else np.zeros(k, dtype=np.int64)
    assert N.tolist() == [int(Nk[j]) << (j + 1) for j in range(k)]
    if want.shape[0]:
        N_ref, labs, ptrs = oracle.csf(want, k)
        for depth in range(1, k + 1):
            lab, ptr = nxt.export(depth)
            assert np.array_equal(host(lab), labs[depth - 1])
            if depth < k:
                assert np.array_equal(host(ptr), ptrs[depth - 1].astype(np.int32))


def _fanout_tuples(k, level, nparents, per, seed):
    """Tuples whose depth-(k-2) nodes have about `per` children each (nparents of them): the
    prune's parent marking takes one thread per node (up to 32 children per node on
    average), a scatter from the children (up to 128) or a warp per node (more)."""
    side = 1 << level
    st = synth.Stream(seed)
    heads = np.unique(st.uniform_int(0, side ** (k - 1) - 1, nparents))
    rows = []
    for h in heads:
        pre = []
        r = int(h)
        for _ in range(k - 1):
            pre.append(r % side)
            r //= side
        pre = pre[::-1]
        last = np.unique(st.uniform_int(0, side - 1, per))
        rows.append(np.column_stack([np.tile(pre, (last.size, 1)), last]))
    return np.concatenate(rows).astype(np.int32)


@pytest.mark.parametrize("k,per,p,seed", [(2, 20, 0.3, 31), (2, 90, 0.05, 32), (2, 400, 0.02, 33),
                                          (3, 90, 0.5, 34), (3, 400, 0.3, 35), (3, 400, 0.0005, 36)])
def test_subdivide_and_compact_across_fanouts(vx, k, per, p, seed):
    """Split and compaction of trees whose leaves hang under few parents with many children
    each, so that every form of the parent marking runs, against the definition."""
    level = 9
    t = _fanout_tuples(k, level, 12, per, seed)
    keep = (synth.Stream(seed + 7).unit(t.shape[0]) < p).astype(np.uint8)
    c = vx.csf_build(k, level, dev(t))
    nxt = vx.csf_subdivide(c, dev(keep))
    kept = t[keep == 1]
    want = _children(kept, k) if kept.shape[0] else np.zeros((0, k), dtype=np.int32)
    assert np.array_equal(host(nxt.tuples()), want)
    if want.shape[0]:
        N_ref, labs, ptrs = oracle.csf(want, k)
        for depth in range(1, k + 1):
            lab, ptr = nxt.export(depth)
            assert np.array_equal(host(lab), labs[depth - 1])
            if depth < k:
                assert np.array_equal(host(ptr), ptrs[depth - 1].astype(np.int32))
    out, idx = vx.csf_compact(c, dev(keep), with_index=True)
    assert np.array_equal(host(out.tuples()), kept)
    assert np.array_equal(host(idx), np.nonzero(keep)[0].astype(np.int32))


@pytest.mark.parametrize("p,seed", [(0.3, 41), (0.002, 42)])
def test_subdivide_and_compact_many_long_parents(vx, p, seed):
    """90 000 depth-0 nodes of 130 children each (k = 2, level 17): enough nodes for the
    parent marking to take a thread per node with long child ranges, with many kept children
    (most nodes settled by their first load) and with few (most ranges read to their end);
    split and compaction against the definition."""
    k, level, npar, per = 2, 17, 90000, 130
    side = 1 << level
    h = np.repeat(np.arange(npar, dtype=np.int64), per)
    j = np.tile(np.arange(per, dtype=np.int64), npar)
    x2 = (j * 997 + h * 13) % side  # distinct within a parent (997 odd, per < side)
    t = np.column_stack([h, x2]).astype(np.int32)
    t = t[np.lexsort(t.T[::-1])]
    keep = (synth.Stream(seed).unit(t.shape[0]) < p).astype(np.uint8)
    c = vx.csf_build(k, level, dev(t))
    nxt = vx.csf_subdivide(c, dev(keep))
    kept = t[keep == 1]
    want = _children(kept, k)
    N_ref, labs, ptrs = oracle.csf(want, k)
    lab0, ptr0 = nxt.export(1)
    lab1, _ = nxt.export(2)
    assert np.array_equal(host(lab0), labs[0]) and np.array_equal(host(lab1), labs[1])
    assert np.array_equal(host(ptr0), ptrs[0].astype(np.int32))
    out, idx = vx.csf_compact(c, dev(keep), with_index=True)
    assert np.array_equal(host(out.tuples()), kept)
    assert np.array_equal(host(idx), np.nonzero(keep)[0].astype(np.int32))


@pytest.mark.parametrize("k,level,n,p,seed", [(2, 6, 900, 0.3, 12), (3, 5, 6000, 0.5, 13),
                                              (4, 3, 2000, 0.1, 14)])
def test_compact_matches_definition(vx, k, level, n, p, seed):
    t = synth.random_tuples(k, level, n, seed)
    keep = (synth.Stream(seed).unit(t.shape[0]) < p).astype(np.uint8)
    c = vx.csf_build(k, level, dev(t))
    out, idx = vx.csf_compact(c, dev(keep), with_index=True)
    assert np.array_equal(host(out.tuples()), t[keep == 1])
    assert np.array_equal(host(idx), np.nonzero(keep)[0].astype(np.int32))


# ---------------------------------------------------------------------------------------
# Algorithm 2 with C0, binary64: bit-identical to the oracle
# ---------------------------------------------------------------------------------------
EVAL_CASES = [
    # k, d, npoly, level, density, n, domain
    (1, 12, 2, 7, 1.0, 100, None),
    (2, 8, 1, 6, 1.0, 2000, None),
    (2, 10, 2, 5, 0.4, 900, None),
    (3, 6, 1, 4, 1.0, 3000, None),
    (3, 7, 2, 5, 0.5, 8000, None),
    (4, 4, 1, 3, 1.0, 3000, None),
    (2, 6, 1, 0, 1.0, 1, None),                           # level 0: the box straddles 0
    (2, 7, 2, 3, 1.0, 60, [-0.75, 1.25, -3.0, 1.0]),      # boxes straddling 0
    (3, 5, 1, 4, 0.7, 2000, [0.0, 1.0, -2.0, 2.0, -0.5, 1.5]),
]


@pytest.mark.parametrize("k,d,npoly,level,density,n,domain", EVAL_CASES)
def test_eval_level_fp64_bitexact(vx, k, d, npoly, level, density, n, domain):
    polys = synth.random_small(k, d, npoly, 1000 + 10 * k + d, density=density)
    dom = np.asarray(domain) if domain is not None else synth.cube(k)
    t = synth.random_tuples(k, level, n, 77 + k)
    sysv = vx.System(polys)
    c = vx.csf_build(k, level, dev(t))
    keep, lo, hi = vx.csf_eval_level(sysv, c, dom, vx.FP64, values=True)
    lo_r, hi_r, keep_r, _ = oracle.eval_csf(polys, dom, level, t)
    assert np.array_equal(host(lo), lo_r)
    assert np.array_equal(host(hi), hi_r)
    assert np.array_equal(host(keep), keep_r)


def test_eval_level_kostlan_high_degree_bitexact(vx):
    # a slice of the degree-100 curve system: 400 random boxes at level 7
    s = synth.curve()
    t = synth.random_tuples(3, 7, 400, 9)
    sysv = vx.System(s.polys)
    c = vx.csf_build(3, 7, dev(t))
    keep, lo, hi = vx.csf_eval_level(sysv, c, s.domain, vx.FP64, values=True)
    lo_r, hi_r, keep_r, _ = oracle.eval_csf(s.polys, s.domain, 7, t)
    assert np.array_equal(host(lo), lo_r) and np.array_equal(host(hi), hi_r)
    assert np.array_equal(host(keep), keep_r)


def test_system_info_counts(vx):
    import math

    s = synth.curve(d=20)
    k, npoly, M = vx.System(s.polys).info()
    assert (k, npoly) == (3, 2)
    assert M[0].tolist() == [math.comb(20 + 3 - j, 3 - j) for j in range(4)]


def test_large_polynomial_packing_checks(vx):
    """A polynomial large enough for its packing loops to be split between host threads
    (62 196 terms): a monomial repeated at the far end (another chunk than its first
    occurrence), a non-finite coefficient or a negative exponent there are still refused, and
    the clean polynomial packs to the dense block sizes."""
    e, c = synth.kostlan_poly(3, 70, 1501)
    k, npoly, M = vx.System([(e, c)]).info()
    assert M[0].tolist() == [math.comb(70 + 3 - j, 3 - j) for j in range(4)]
    e2 = np.concatenate([e, e[:1]])
    with pytest.raises(vx.VxError, match="twice"):
        vx.System([(e2, np.concatenate([c, c[:1]]))])
    c2 = c.copy()
    c2[-1] = np.nan
    with pytest.raises(vx.VxError, match="coefficient"):
        vx.System([(e, c2)])
    e3 = e.copy()
    e3[-1, 2] = -1
    with pytest.raises(vx.VxError, match="exponent"):
        vx.System([(e3, c)])


def test_system_rejects_bad_polynomials(vx):
    e = np.array([[0, 1], [0, 1]], dtype=np.int32)
    with pytest.raises(vx.VxError):
        vx.System([(e, np.array([1.0, 2.0]))])  # same monomial twice
    with pytest.raises(vx.VxError):
        vx.System([(np.array([[0, 1]], dtype=np.int32), np.array([np.inf]))])
    with pytest.raises(vx.VxError):
        vx.System([(np.array([[0, -1]], dtype=np.int32), np.array([1.0]))])


def test_domain_must_be_dyadic(vx):
    polys = synth.random_small(2, 3, 1, 5)
    sysv = vx.System(polys)
    c = vx.csf_build(2, 2, dev(np.array([[0, 0]], dtype=np.int32)))
    with pytest.raises(vx.VxError) as e:
        vx.csf_eval_level(sysv, c, [0.0, 0.1, 0.0, 1.0])
    assert e.value.code == vx.EINVAL


# ---------------------------------------------------------------------------------------
# Algorithm 3
# ---------------------------------------------------------------------------------------
def _circle(k):
    e = np.zeros((k + 1, k), dtype=np.int32)
    for i in range(k):
        e[i, i] = 2
    return [(e, np.array([1.0] * k + [-0.5]))]


ENCLOSE_CASES = {
    "plain-k2-d20-depth8": lambda: (synth.plain().polys, synth.cube(2), 8),
    "k1-d15-2polys": lambda: (synth.random_small(1, 15, 2, 31), synth.cube(1), 12),
    "k2-d9-sparse": lambda: (synth.random_small(2, 9, 1, 32, density=0.5), synth.cube(2), 7),
    "k3-d6-2polys": lambda: (synth.random_small(3, 6, 2, 33), synth.cube(3), 6),
    "k4-d3": lambda: (synth.random_small(4, 3, 1, 34), synth.cube(4), 4),
    "circle": lambda: (_circle(2), synth.cube(2), 9),
    "sphere": lambda: (_circle(3), synth.cube(3), 6),
    "no-zeros": lambda: ([(np.array([[2, 0], [0, 2], [0, 0]], dtype=np.int32),
                           np.array([1.0, 1.0, 1.0]))], synth.cube(2), 6),
    "asym-domain": lambda: (synth.random_small(2, 7, 1, 35), np.array([-0.5, 1.5, -2.0, 0.0]), 7),
    "surface-d12": lambda: ([synth.kostlan_poly(3, 12, 36)], synth.cube(3), 6),
}


@pytest.mark.parametrize("name", sorted(ENCLOSE_CASES))
def test_enclose_fp64_equals_oracle(vx, name):
    polys, dom, depth = ENCLOSE_CASES[name]()
    ref = oracle.enclose(polys, dom, depth)
    res = vx.enclose(polys, dom, depth)
    st = res.stats()
    assert np.array_equal(res.boxes(), ref["tuples"])
    assert np.array_equal(st["tested"], ref["tested"])
    assert np.array_equal(st["kept"], ref["kept"])
    assert np.array_equal(st["nodes"], ref["nodes"])
    assert np.array_equal(st["madds"], ref["work"])


@pytest.mark.parametrize("name", sorted(ENCLOSE_CASES))
def test_enclose_fp32_certified_equals_oracle_every_level(vx, name):
    # binary32 with binary64-certified decisions: every level is the binary64 level
    polys, dom, depth = ENCLOSE_CASES[name]()
    ref = oracle.enclose(polys, dom, depth)
    res = vx.enclose(polys, dom, depth, vx.make_opts(vx.FP32))
    st = res.stats()
    assert np.array_equal(res.boxes(), ref["tuples"])
    assert np.array_equal(st["tested"], ref["tested"])
    assert np.array_equal(st["kept"], ref["kept"])
    assert np.array_equal(st["nodes"], ref["nodes"])
    if name in ("circle", "sphere"):
        # the zero set passes through grid points: some boxes have an endpoint exactly 0 and
        # can only be decided in binary64
        assert st["recheck"].sum() > 0


@pytest.mark.parametrize("k,d,npoly,level,density,n,domain", EVAL_CASES)
def test_eval_level_fp32_certified_decisions(vx, k, d, npoly, level, density, n, domain):
    polys = synth.random_small(k, d, npoly, 1000 + 10 * k + d, density=density)
    dom = np.asarray(domain) if domain is not None else synth.cube(k)
    t = synth.random_tuples(k, level, n, 77 + k)
    sysv = vx.System(polys)
    c = vx.csf_build(k, level, dev(t))
    keep, lo, hi = vx.csf_eval_level(sysv, c, dom, vx.FP32, values=True)
    lo_r, hi_r, keep_r, _ = oracle.eval_csf(polys, dom, level, t)
    assert np.array_equal(host(keep), keep_r)
    # the binary32 bounds are bounds: around the binary64 ones up to rounding
    assert np.all(host(lo) <= hi_r) and np.all(host(hi) >= lo_r)


def test_eval_level_fp32_certified_kostlan_d100(vx):
    s = synth.curve()
    t = synth.random_tuples(3, 8, 3000, 19)
    sysv = vx.System(s.polys)
    c = vx.csf_build(3, 8, dev(t))
    keep = vx.csf_eval_level(sysv, c, s.domain, vx.FP32)
    _, _, keep_r, _ = oracle.eval_csf(s.polys, s.domain, 8, t)
    assert np.array_equal(host(keep), keep_r)


@pytest.mark.parametrize("name", ["plain-k2-d20-depth8", "k3-d6-2polys", "surface-d12",
                                  "asym-domain", "k4-d3"])
def test_enclose_fp32_midrad(vx, name):
    polys, dom, depth = ENCLOSE_CASES[name]()
    ref = oracle.enclose(polys, dom, depth)
    # binary32 below the last level, binary64 last level: exactly the binary64 set
    r1 = vx.enclose(polys, dom, depth, vx.make_opts(vx.FP32_MIDRAD, fp64_final=True))
    assert np.array_equal(r1.boxes(), ref["tuples"])
    # binary32 throughout: a superset at every level
    r2 = vx.enclose(polys, dom, depth, vx.make_opts(vx.FP32_MIDRAD))
    s2 = r2.stats()
    assert np.all(s2["kept"] >= ref["kept"])
    b2 = {tuple(r) for r in r2.boxes().tolist()}
    assert {tuple(r) for r in ref["tuples"].tolist()} <= b2
    # with binary64 rechecks of tight boxes: still a superset, never more than without
    r3 = vx.enclose(polys, dom, depth, vx.make_opts(vx.FP32_MIDRAD, fp64_recheck=True))
    s3 = r3.stats()
    b3 = {tuple(r) for r in r3.boxes().tolist()}
    assert {tuple(r) for r in ref["tuples"].tolist()} <= b3 <= b2
    assert np.all(s3["kept"] >= ref["kept"])


@pytest.mark.parametrize("k,d,level,seed", [(2, 20, 6, 1), (3, 8, 4, 2), (3, 30, 6, 3)])
def test_fp32_box_enclosure_contains_fp64(vx, k, d, level, seed):
    polys = [synth.kostlan_poly(k, d, seed)]
    t = synth.random_tuples(k, level, 3000, seed)
    sysv = vx.System(polys)
    c = vx.csf_build(k, level, dev(t))
    k64, lo64, hi64 = vx.csf_eval_level(sysv, c, synth.cube(k), vx.FP64, values=True)
    k32, lo32, hi32 = vx.csf_eval_level(sysv, c, synth.cube(k), vx.FP32_MIDRAD, values=True)
    lo64, hi64, lo32, hi32 = map(host, (lo64, hi64, lo32, hi32))
    assert np.all(lo32 <= lo64) and np.all(hi32 >= hi64)
    assert np.all(host(k32) >= host(k64))
    # and the binary32 radius is not wildly inflated
    w64 = hi64 - lo64
    w32 = hi32 - lo32
    assert np.median(w32 / np.maximum(w64, 1e-300)) < 1.5


@pytest.mark.parametrize("world", [2, 4, 8])
def test_enclose_from_slab_starts_reproduce_full(vx, world):
    from paper_2406_09857_gb300 import shard

    polys, dom, depth = ENCLOSE_CASES["k3-d6-2polys"]()
    full = oracle.enclose(polys, dom, depth)["tuples"]
    sysv = vx.System(polys)
    parts = []
    for r in range(world):
        s, start = shard.rank_start(3, depth, r, world)
        c = vx.csf_build(3, s, dev(start))
        for mode in (vx.FP64, vx.FP32):
            res = vx.enclose_from(sysv, c, dom, depth, vx.make_opts(mode))
            b = res.boxes()
            if mode == vx.FP64:
                parts.append(b)
            else:
                assert np.array_equal(b, parts[-1])
    assert np.array_equal(np.concatenate(parts, axis=0), full)


def test_bounded_wait_gives_up_cleanly(vx):
    """A TMA-staged stage whose first wait is limited to zero polls records the give-up, waits
    for its copy and returns; the call reports VX_ETIMEOUT and the next call is exact again."""
    import torch

    polys = synth.random_small(3, 8, 1, 91)
    i, j = np.meshgrid(np.arange(512, dtype=np.int32), np.arange(512, dtype=np.int32),
                       indexing="ij")
    t = np.stack([i.ravel(), j.ravel(), (i.ravel() + j.ravel()) % 512], axis=1).astype(np.int32)
    sysv = vx.System(polys)
    c = vx.csf_build(3, 9, dev(t))  # 262144 depth-2 nodes, 512 per parent: TMA-staged stage
    try:
        assert vx.lib().vx_set_wait_limit(0) == 0  # give up without polling
        with pytest.raises(vx.VxError) as e:
            vx.csf_eval_level(sysv, c, synth.cube(3), vx.FP64)
        assert e.value.code == vx.ETIMEOUT
    finally:
        vx.lib().vx_set_wait_limit(-1)
    keep, lo, hi = vx.csf_eval_level(sysv, c, synth.cube(3), vx.FP64, values=True)
    sample = np.arange(0, t.shape[0], 997)
    lo_r, hi_r, keep_r, _ = oracle.eval_boxes(polys, synth.cube(3), 9, t[sample])
    assert np.array_equal(host(lo)[:, sample], lo_r) and np.array_equal(host(hi)[:, sample], hi_r)
    assert np.array_equal(host(keep)[sample], keep_r)


@pytest.mark.parametrize("k,level", [(1, 6), (2, 4), (3, 3), (4, 2)])
def test_full_grid_csf_equals_built(vx, k, level):
    side = 1 << level
    t = np.stack(np.meshgrid(*[np.arange(side, dtype=np.int32)] * k, indexing="ij"),
                 axis=-1).reshape(-1, k)
    a = vx.csf_full_grid(k, level)
    b = vx.csf_build(k, level, dev(t))
    assert a.nodes()[2].tolist() == b.nodes()[2].tolist()
    for depth in range(1, k + 1):
        la, pa = a.export(depth)
        lb, pb = b.export(depth)
        assert torch_equal(la, lb)
        if depth < k:
            assert torch_equal(pa, pb)
    assert np.array_equal(host(a.tuples()), t)


def torch_equal(x, y):
    import torch

    return torch.equal(x, y)


@pytest.mark.parametrize("d,level", [(6, 4), (12, 3)])
def test_dense_level_per_variable_degree(vx, d, level):
    # config-5 shape (degree d in each variable, iid N(0,1)), every box of a level, against
    # per-box nested Horner on a sample and the certified/midpoint-radius invariants on all
    e, cf = synth.gaussian_tensor_poly(3, d, 55)
    polys = [(e, cf)]
    sysv = vx.System(polys)
    c = vx.csf_full_grid(3, level)
    keep, lo, hi = vx.csf_eval_level(sysv, c, synth.cube(3), vx.FP64, values=True)
    t = host(c.tuples())
    sample = np.arange(0, t.shape[0], 7)
    lo_r, hi_r, keep_r, _ = oracle.eval_boxes(polys, synth.cube(3), level, t[sample])
    assert np.array_equal(host(lo)[:, sample], lo_r) and np.array_equal(host(hi)[:, sample], hi_r)
    assert np.array_equal(host(keep)[sample], keep_r)
    k32 = vx.csf_eval_level(sysv, c, synth.cube(3), vx.FP32)
    assert np.array_equal(host(k32), host(keep))
    kmr = vx.csf_eval_level(sysv, c, synth.cube(3), vx.FP32_MIDRAD)
    assert np.all(host(kmr) >= host(keep))


def test_enclose_batch_equals_single_runs(vx):
    """Independent systems of uneven k, degree and depth (the config-4 mix, small): each result
    equals the oracle's enclosure of that system alone, in binary64 and certified binary32."""
    systems = []
    for i in range(12):
        st = synth.Stream(700 + i)
        if i % 2 == 0:
            d = int(st.uniform_int(4, 12, 1)[0])
            systems.append(([synth.kostlan_poly(2, d, 800 + i)], synth.cube(2),
                            int(st.uniform_int(5, 8, 1)[0])))
        else:
            d = int(st.uniform_int(3, 6, 1)[0])
            systems.append(([synth.kostlan_poly(3, d, 900 + i), synth.kostlan_poly(3, d, 950 + i)],
                            synth.cube(3), int(st.uniform_int(3, 5, 1)[0])))
    for mode in (vx.FP64, vx.FP32):
        res = vx.enclose_batch(systems, vx.make_opts(mode), nworkers=4)
        for (polys, dom, depth), r in zip(systems, res):
            ref = oracle.enclose(polys, dom, depth)
            assert np.array_equal(r.boxes(), ref["tuples"])
            assert np.array_equal(r.stats()["tested"], ref["tested"])


def test_dense_level9_all_modes_odd_block(vx):
    """A complete level-9 grid (512^3 boxes) of a degree-(4,4,4) tensor: 262144 depth-2 nodes
    with 512 children per parent, so the stage kernels take their shared-memory-staged form
    where the block layout allows it (binary64, binary32 certified: 16-byte entries) and not
    where a 25-entry midpoint-radius block would start off a 16-byte boundary."""
    e, cf = synth.gaussian_tensor_poly(3, 4, 56)
    polys = [(e, cf)]
    sysv = vx.System(polys)
    c = vx.csf_full_grid(3, 9)
    k64 = host(vx.csf_eval_level(sysv, c, synth.cube(3), vx.FP64))
    k32 = host(vx.csf_eval_level(sysv, c, synth.cube(3), vx.FP32))
    kmr = host(vx.csf_eval_level(sysv, c, synth.cube(3), vx.FP32_MIDRAD))
    assert np.array_equal(k32, k64)
    assert np.all(kmr >= k64)
    rng = synth.Stream(57)
    idx = np.unique(rng.uniform_int(0, (1 << 27) - 1, 4000))
    t = np.stack([idx >> 18, (idx >> 9) & 511, idx & 511], axis=1).astype(np.int32)
    _, _, keep_r, _ = oracle.eval_boxes(polys, synth.cube(3), 9, t)
    assert np.array_equal(k64[idx], keep_r)


def test_enclose_batch_forest_mixed_modes(vx):
    """A larger mixed batch: k = 1, 2 and 3 in one call, depth 0, a system with no zeros in its
    domain (its tree empties at level 0), uneven degrees and depths; binary64 and certified
    binary32 equal the oracle in boxes and per-level counts, midpoint-radius with a binary64
    final level equals it too, and without it is a superset at every level."""
    systems = []
    for i in range(30):
        st = synth.Stream(1700 + i)
        k = 1 + i % 3
        d = int(st.uniform_int(2, 9 if k < 3 else 5, 1)[0])
        npoly = 1 if k == 1 else int(st.uniform_int(1, 2, 1)[0])
        polys = [synth.kostlan_poly(k, d, 1800 + 10 * i + p) for p in range(npoly)]
        depth = int(st.uniform_int(0, 9 - 2 * k, 1)[0]) if i != 4 else 0
        systems.append((polys, synth.cube(k), depth))
    # no zeros: 1 + x^2 + y^2 on [-1,1]^2
    e = np.array([[0, 0], [2, 0], [0, 2]], dtype=np.int32)
    systems.append(([(e, np.array([1.0, 1.0, 1.0]))], synth.cube(2), 6))
    refs = [oracle.enclose(p, dom, depth) for p, dom, depth in systems]
    assert refs[-1]["tuples"].shape[0] == 0
    for opts in (vx.make_opts(vx.FP64), vx.make_opts(vx.FP32),
                 vx.make_opts(vx.FP32_MIDRAD, fp64_final=True)):
        res = vx.enclose_batch(systems, opts)
        for ref, r in zip(refs, res):
            assert np.array_equal(r.boxes(), ref["tuples"])
            st = r.stats()
            assert int(st["kept"][-1]) == ref["tuples"].shape[0]
            if opts.mode == vx.FP32_MIDRAD:  # supersets before the last level
                assert np.all(st["tested"] >= ref["tested"])
            else:
                assert np.array_equal(st["tested"], ref["tested"])
                assert np.array_equal(st["kept"], ref["kept"])
    res = vx.enclose_batch(systems, vx.make_opts(vx.FP32_MIDRAD))
    for ref, r in zip(refs, res):
        b = r.boxes()
        assert b.shape[0] >= ref["tuples"].shape[0]
        got = set(map(tuple, b.tolist()))
        assert all(tuple(t) in got for t in ref["tuples"].tolist())


def test_autotuner_variants_agree_and_cache_round_trips(vx, tmp_path):
    """Every launch variant the autotuner may pick gives the same outputs: enclosures with the
    heuristics only and with tuning (from an empty table) are identical box for box in each
    arithmetic; a cache file written while tuning reloads the same shapes."""
    polys = [synth.kostlan_poly(3, 14, 991), synth.kostlan_poly(3, 14, 992)]
    dom = synth.cube(3)
    path = str(tmp_path / "tune.txt")
    try:
        for mode in (vx.FP64, vx.FP32, vx.FP32_MIDRAD):
            vx.autotune(0)
            ref = vx.enclose(polys, dom, 7, vx.make_opts(mode)).boxes()
            vx.lib().vx_autotune_clear()
            vx.autotune(1, path)
            got = vx.enclose(polys, dom, 7, vx.make_opts(mode)).boxes()
            assert np.array_equal(got, ref)
            again = vx.enclose(polys, dom, 7, vx.make_opts(mode)).boxes()  # cached choices
            assert np.array_equal(again, ref)
        n = vx.autotune_entries()
        assert n > 0
        vx.lib().vx_autotune_clear()
        assert vx.autotune_entries() == 0
        vx.autotune(1, path)
        assert vx.autotune_entries() == n
    finally:
        vx.autotune(1)


@pytest.mark.parametrize("k,d,kind,depth", [(2, 20, "points", 10), (2, 20, "curves", 9),
                                            (3, 20, "points", 6), (3, 20, "curves", 5),
                                            (3, 20, "hypersurfaces", 4), (4, 20, "points", 4),
                                            (4, 20, "curves", 3), (4, 20, "hypersurfaces", 3)])
def test_table1_family_equals_oracle(vx, k, d, kind, depth):
    """The random-polynomial family of the experiments (U[-10,10] coefficients on [-2,2]^k, k
    up to 4), at depths the oracle finishes quickly: binary64 and certified binary32 equal the
    oracle's enclosure."""
    s = synth.table1(k, d, kind)
    ref = oracle.enclose(s.polys, s.domain, depth)
    for mode in (vx.FP64, vx.FP32):
        r = vx.enclose(s.polys, s.domain, depth, vx.make_opts(mode))
        assert np.array_equal(r.boxes(), ref["tuples"])
        assert np.array_equal(r.stats()["tested"], ref["tested"])


@pytest.mark.parametrize("case", ["curve-d14", "three-polys", "mixed-lengths", "relations"])
def test_every_launch_variant_matches_oracle(vx, case):
    """Each launch variant, forced everywhere it exists (one or two boxes per thread, the
    parent's blocks in shared memory or not, more fibre groups, fewer threads, the leaf pairs
    the first polynomial settles skipped with 512 or 1024 leaves per CTA), gives the
    oracle's enclosure in every arithmetic (midpoint-radius with a binary64 last level)."""
    cases = {
        "curve-d14": ([synth.kostlan_poly(3, 14, 1201), synth.kostlan_poly(3, 14, 1202)], None, 7),
        "three-polys": ([synth.kostlan_poly(3, 9, 1203), synth.kostlan_poly(3, 9, 1204),
                         synth.kostlan_poly(3, 7, 1205)], None, 6),
        "mixed-lengths": (synth.random_small(3, 8, 2, 1206, density=0.3), None, 6),
        "relations": (synth.random_small(3, 6, 3, 1207), [0, 1, 4], 6),
    }
    polys, rel, depth = cases[case]
    dom = synth.cube(3)
    ref = oracle.enclose_gen(polys, dom, depth, rel=rel)
    sysv = vx.System(polys, rel=rel) if rel else vx.System(polys)
    try:
        for v in range(5):
            vx.autotune(2 + v)
            for opts in (vx.make_opts(vx.FP32), vx.make_opts(vx.FP64),
                         vx.make_opts(vx.FP32_MIDRAD, fp64_final=True)):
                r = vx.enclose_system(sysv, dom, depth, opts)
                assert np.array_equal(r.boxes(), ref["tuples"]), (case, v)
                r.free()
    finally:
        vx.autotune(1)


def test_small_levels_in_binary64(vx):
    """VX_FP32 with small_level_madds: the levels below the threshold run in binary64 (no band,
    no recheck) and the enclosure is still the oracle's, with or without the Taylor form."""
    polys = [synth.kostlan_poly(3, 10, 1301), synth.kostlan_poly(3, 10, 1302)]
    dom = synth.cube(3)
    ref = oracle.enclose(polys, dom, 7)
    for thr in (1 << 30, 1 << 20):
        r = vx.enclose(polys, dom, 7, vx.make_opts(vx.FP32, small_level_madds=thr))
        assert np.array_equal(r.boxes(), ref["tuples"])
        st = r.stats()
        assert np.array_equal(st["kept"], ref["kept"])
        if thr == 1 << 30:
            assert st["recheck"].sum() == 0
    reft = oracle.enclose_taylor(polys, dom, 6, 2)
    r = vx.enclose(polys, dom, 6, vx.make_opts(vx.FP32, taylor_order=2, small_level_madds=1 << 22))
    assert np.array_equal(r.boxes(), reft["tuples"])


@pytest.mark.parametrize("host_codes", [False, True])
@pytest.mark.parametrize("k,d,depth", [(3, 8, 7), (4, 3, 9), (2, 12, 16)])
def test_box_codes_decode_to_the_boxes(vx, k, d, depth, host_codes):
    """The boxes' grid-index codes, made on request or (host_codes) written into pinned host
    memory by the last level's compaction: increasing, and decoding to the boxes."""
    polys = [synth.kostlan_poly(k, d, 1400 + depth)]
    r = vx.enclose(polys, synth.cube(k), depth, vx.make_opts(vx.FP32, host_codes=host_codes))
    codes = r.box_codes()
    assert codes.dtype == (np.uint32 if k * depth <= 32 else np.uint64)
    assert np.all(codes[1:] > codes[:-1])
    assert np.array_equal(vx.Result.decode_codes(codes, k, depth), r.boxes())
    assert codes.shape[0] > 0


def test_midrad_k4_staged_stage_reads_aligned_blocks(vx):
    """Four variables in binary32 midpoint-radius (8-byte entries): stage 0 writes an odd
    number of entries (5 depth-1 nodes x 27 suffix monomials), so the depth-1 blocks would
    start 8 bytes off a 16-byte boundary if the depths were packed back to back, and depth 2
    has enough nodes (81 920, 128 per parent) for its stage to bring the parents' blocks into
    shared memory by bulk copies.  Every depth's block starts on a 256-byte boundary, so the
    level evaluates; its values equal the allocation-free entry point's (which carves the same
    layout from its own array) bit for bit and contain the oracle's binary64 enclosures."""
    import torch

    polys = synth.random_small(4, 4, 1, 901, density=0.5)
    M = vx.measure(polys)[0]
    assert M[1] % 2 == 1 and (M[2] * 8) % 16 == 0
    x1, x2, x3 = np.meshgrid(np.arange(5), np.arange(128), np.arange(128), indexing="ij")
    x4 = (7 * x1 + 3 * x2 + x3) % 128
    t = np.stack([x1.ravel(), x2.ravel(), x3.ravel(), x4.ravel()], axis=1).astype(np.int32)
    sysv = vx.System(polys)
    c = vx.csf_build(4, 7, dev(t))
    assert c.nodes()[2].tolist() == [5, 640, 81920, 81920]
    dom = synth.cube(4)
    keep, lo, hi = vx.csf_eval_level(sysv, c, dom, vx.FP32_MIDRAD, values=True)
    n = t.shape[0]
    keep_s = torch.empty(n, dtype=torch.uint8, device="cuda")
    lo_s = torch.empty((1, n), dtype=torch.float64, device="cuda")
    hi_s = torch.empty_like(lo_s)
    vx.csf_eval_level_static(sysv, c, dom, vx.FP32_MIDRAD, keep_s, lo_s, hi_s)
    torch.cuda.synchronize()
    assert torch.equal(keep, keep_s) and torch.equal(lo, lo_s) and torch.equal(hi, hi_s)
    lo_o, hi_o, keep_o, _ = oracle.eval_csf(polys, dom, 7, t)
    assert np.all(lo.cpu().numpy() <= lo_o) and np.all(hi.cpu().numpy() >= hi_o)
    assert np.all(keep.cpu().numpy() >= keep_o)


@pytest.mark.parametrize("k,depth", [(1, 10), (2, 7), (3, 5)])
def test_float_pair_tier_decides_the_binary32_band(vx, k, depth):
    """A zero set 2^-30 away from a grid line: x_1 - (3/8 + 2^-30) (+ 2^-40 x_2 ... x_k).  On
    the boxes that meet x_1 = 3/8 the binary32 ends are 0 within their error bound (3/8 + 2^-30
    rounds to 3/8 in binary32), so certified binary32 leaves them to a finer arithmetic; the
    float pairs carry the 2^-30 and decide every one of them, and the enclosure is binary64's."""
    c = 0.375 + 2.0 ** -30
    exps = [[1] + [0] * (k - 1), [0] * k]
    coefs = [1.0, -c]
    if k >= 2:
        exps.append([0] + [1] * (k - 1))
        coefs.append(2.0 ** -40)
    polys = [(np.array(exps, dtype=np.int32), np.array(coefs))]
    dom = synth.cube(k)
    ref = oracle.enclose(polys, dom, depth)
    res = vx.enclose(polys, dom, depth, vx.make_opts(vx.FP32))
    st = res.stats()
    assert np.array_equal(res.boxes(), ref["tuples"])
    assert np.array_equal(st["tested"], ref["tested"])
    assert np.array_equal(st["kept"], ref["kept"])
    assert st["recheck"].sum() > 0
    assert st["recheck64"].sum() == 0
    # only the column of boxes whose x_1-range holds 3/8 + 2^-30 survives
    assert np.all(res.boxes()[:, 0] == ((0.375 + 1.0) * (1 << depth) / 2))


@pytest.mark.parametrize("name,cap,mode_name,recheck_last", [
    ("k3-d6-2polys", 600, "FP64", False), ("k3-d6-2polys", 600, "FP32", True),
    ("k3-d6-2polys", 400, "FP32_MIDRAD", False),
    ("plain-k2-d20-depth8", 700, "FP32", False), ("k4-d3", 8000, "FP64", False)])
def test_enclose_in_x1_ranges_equals_oracle(vx, name, cap, mode_name, recheck_last):
    """A level whose kept boxes would give the next level more than opts.max_level_boxes boxes
    runs in ranges of consecutive x_1 slabs, each through the remaining levels on its own: the
    boxes (as tuples, as codes and as one joined tree) and the per-level counts are the
    oracle's, and no tree of the run held more than the cap."""
    polys, dom, depth = ENCLOSE_CASES[name]()
    ref = oracle.enclose(polys, dom, depth)
    if mode_name == "FP32_MIDRAD":  # a superset of binary64's: the unchunked run is the reference
        whole = vx.enclose(polys, dom, depth, vx.make_opts(vx.FP32_MIDRAD))
        ws = whole.stats()
        ref = {"tuples": whole.boxes(), "tested": ws["tested"], "kept": ws["kept"],
               "nodes": ws["nodes"]}
    k = ref["tuples"].shape[1]
    assert max(ref["kept"][:-1]) << k > cap, "the cap must force a split"
    # host_codes asks for the codes from the last compaction; with the final boxes in several
    # trees they are made on request instead (the same codes)
    o = vx.make_opts(getattr(vx, mode_name), recheck_last=recheck_last, max_level_boxes=cap,
                     host_codes=True)
    res = vx.enclose(polys, dom, depth, o)
    st = res.stats()
    assert np.array_equal(res.boxes(), ref["tuples"])
    assert np.array_equal(st["tested"], ref["tested"]) or recheck_last
    assert st["kept"][-1] == ref["kept"][-1]
    if not recheck_last:
        assert np.array_equal(st["kept"], ref["kept"])
        assert np.array_equal(st["nodes"], ref["nodes"])
    codes = res.box_codes()
    assert np.array_equal(vx.Result.decode_codes(codes, k, depth), ref["tuples"])
    assert np.array_equal(res.csf().tuples().cpu().numpy(), ref["tuples"])


@pytest.mark.parametrize("name,first", [("k3-d6-2polys", 3), ("plain-k2-d20-depth8", 5),
                                        ("k4-d3", 2), ("surface-d12", 4)])
def test_enclose_from_full_grid_level_equals_oracle(vx, name, first):
    """opts.first_level: Algorithm 3 from the full grid of a level gives the oracle's boxes (the
    coarser levels' pruning changes no final box); the levels before it are not evaluated and
    the start level tests its whole grid."""
    polys, dom, depth = ENCLOSE_CASES[name]()
    ref = oracle.enclose(polys, dom, depth)
    k = ref["tuples"].shape[1]
    for mode_name, rl in (("FP64", False), ("FP32", True), ("FP32", False)):
        o = vx.make_opts(getattr(vx, mode_name), recheck_last=rl, first_level=first)
        res = vx.enclose(polys, dom, depth, o)
        st = res.stats()
        assert np.array_equal(res.boxes(), ref["tuples"]), mode_name
        assert np.all(st["tested"][:first] == 0)
        assert st["tested"][first] == 1 << (k * first)
        assert st["kept"][-1] == ref["kept"][-1]
        if not rl:
            assert np.array_equal(st["kept"][first + 1:], ref["kept"][first + 1:])
