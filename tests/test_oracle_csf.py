"""Pins of the oracle's CSF tree, Algorithm 2 and Algorithm 3.

- The CSF of the worked example of Sec. 2.1 (the support printed for the sparse matrix of
  the CSF figure, which is also the exponent set of the example polynomial there).
- Remark 1: N_i(E) is the number of distinct length-i prefixes, counted independently here.
- Algorithm 2 on a CSF gives, box by box, the same doubles as nested Horner on each box alone.
- Theorem 1's operation count: a depth-j node runs one Horner per suffix monomial, so a level
  costs sum_j N_j (M_{j-1} - M_j) interval multiply-adds (M_j = C(d+k-j, k-j) when dense).
- Algorithm 3 returns exactly the boxes of the finest grid that pass the C0 test on their
  own (interval Horner is inclusion-isotone under outward rounding, so pruning at coarser
  levels never drops a box that the finest level keeps).
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2406_09857_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_worked_example_csf():
    with open(os.path.join(GOLDEN, "csf_worked_example.json")) as f:
        g = json.load(f)
    N, labs, ptrs = oracle.csf(g["support"], 2)
    assert N.tolist() == g["N"]
    assert labs[0].tolist() == g["labels_depth1"]
    assert labs[1].tolist() == g["labels_depth2"]
    assert ptrs[0].tolist() == g["ptr_depth1"]


def test_worked_example_polynomial_tree_and_values():
    with open(os.path.join(GOLDEN, "csf_worked_example.json")) as f:
        g = json.load(f)
    exps = np.asarray(g["poly_exps"])
    coefs = np.asarray(g["poly_coefs"], dtype=np.float64)
    # T_F of the polynomial has the same tree as the matrix support
    order = np.lexsort((exps[:, 1], exps[:, 0]))
    N, labs, _ = oracle.csf(exps[order], 2)
    assert N.tolist() == g["N"]
    assert coefs[order].tolist() == g["leaf_values"]
    # and evaluating it at a point (x1, x2) = (1/2, -1/4) (exact dyadics) gives the exact value
    x1, x2 = 0.5, -0.25
    want = sum(c * x1 ** a * x2 ** b for (a, b), c in zip(exps.tolist(), coefs.tolist()))
    lo, hi, _, _ = oracle.eval_grid([(exps, coefs)], [([x1], [x1]), ([x2], [x2])], [[0, 0]])
    assert lo[0, 0] == want == hi[0, 0]


@pytest.mark.parametrize("k,level,n,seed", [(1, 6, 40, 1), (2, 5, 300, 2), (3, 4, 900, 3),
                                            (4, 3, 1500, 4)])
def test_remark1_node_counts(k, level, n, seed):
    t = synth.random_tuples(k, level, n, seed)
    N, labs, ptrs = oracle.csf(t, k)
    for j in range(1, k + 1):
        assert N[j - 1] == len({tuple(r[:j]) for r in t.tolist()})
    # children of each depth-j node are its distinct next coordinates, ascending
    for j in range(k - 1):
        assert ptrs[j][0] == 0 and ptrs[j][-1] == N[j + 1]
        assert np.all(np.diff(ptrs[j]) >= 1)
        for a in range(N[j]):
            ch = labs[j + 1][ptrs[j][a]:ptrs[j][a + 1]]
            assert np.all(np.diff(ch) > 0)


def _same_values(a, b):
    # values compared with == so that -0 == +0 (the sign of a zero endpoint is not part of
    # the enclosure)
    return np.array_equal(a, b)


@pytest.mark.parametrize("k,d,npoly,level,density,seed", [
    (1, 7, 2, 6, 1.0, 10), (2, 6, 1, 5, 1.0, 11), (2, 8, 2, 4, 0.5, 12),
    (3, 4, 1, 4, 1.0, 13), (3, 5, 2, 3, 0.6, 14), (4, 3, 1, 2, 1.0, 15),
    (5, 3, 2, 2, 0.7, 16), (6, 2, 1, 2, 1.0, 17)])
def test_alg2_equals_per_box_nested_horner(k, d, npoly, level, density, seed):
    polys = synth.random_small(k, d, npoly, seed, density=density)
    t = synth.random_tuples(k, level, 400, seed + 100)
    dom = synth.cube(k)
    lo1, hi1, keep1, _ = oracle.eval_csf(polys, dom, level, t)
    lo2, hi2, keep2, _ = oracle.eval_boxes(polys, dom, level, t)
    assert _same_values(lo1, lo2) and _same_values(hi1, hi2)
    assert np.array_equal(keep1, keep2)
    assert np.all(lo1 <= hi1)


@pytest.mark.parametrize("k,d,level,seed", [(1, 9, 5, 1), (2, 7, 4, 2), (3, 5, 3, 3),
                                            (4, 3, 2, 4), (5, 3, 2, 5), (6, 2, 2, 6)])
def test_work_count_theorem1(k, d, level, seed):
    polys = synth.random_small(k, d, 1, seed)
    t = synth.random_tuples(k, level, 500, seed)
    _, _, _, work = oracle.eval_csf(polys, synth.cube(k), level, t)
    N, _, _ = oracle.csf(t, k)
    M = [math.comb(d + k - j, k - j) for j in range(k + 1)]
    assert work == sum(int(N[j - 1]) * (M[j - 1] - M[j]) for j in range(1, k + 1))


@pytest.mark.parametrize("k,d,npoly,depth,seed", [(1, 9, 1, 7, 20), (2, 6, 1, 5, 21),
                                                  (2, 5, 2, 5, 22), (3, 4, 1, 4, 23),
                                                  (3, 3, 2, 3, 24), (4, 3, 2, 3, 25),
                                                  (5, 2, 1, 3, 26), (6, 2, 2, 2, 27)])
def test_alg3_equals_brute_force(k, d, npoly, depth, seed):
    polys = synth.random_small(k, d, npoly, seed)
    dom = synth.cube(k)
    res = oracle.enclose(polys, dom, depth)
    bf = oracle.brute_force(polys, dom, depth)
    want = np.argwhere(bf == 1)  # lexicographic order
    assert np.array_equal(res["tuples"], want.astype(np.int32))
    # bookkeeping of Algorithm 3: each level tests 2^k children of the previous survivors
    for l in range(1, depth + 1):
        assert res["tested"][l] == res["kept"][l - 1] << k
    assert res["tested"][0] == 1


def test_alg3_nontrivial_pruning_happens():
    # the pin above is only meaningful if some boxes are excluded before the last level
    polys = synth.random_small(2, 6, 1, 21)
    res = oracle.enclose(polys, synth.cube(2), 5)
    assert res["kept"][3] < res["tested"][3]
    assert 0 < res["kept"][5] < (1 << 10)


def test_domain_exactness():
    assert oracle.domain_exact([-1.0, 1.0, 0.0, 1.0], 10)
    assert oracle.domain_exact([-2.0, 2.0], 12)
    assert not oracle.domain_exact([0.0, 0.1], 3)
    assert not oracle.domain_exact([1.0, -1.0], 3)


def test_unsorted_or_duplicate_tuples_rejected():
    with pytest.raises(oracle.OracleError):
        oracle.csf([[1, 0], [0, 0]], 2)
    with pytest.raises(oracle.OracleError):
        oracle.csf([[0, 0], [0, 0]], 2)
