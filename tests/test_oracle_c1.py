"""Pins of the oracle's inclusion criterion C1 (Sec. 3.2) and of Algorithm 3 with it.

Checked against what does not use that code:
- a linear polynomial: both tests certify a box exactly when the exact range over the closed
  box has points below and above 0 (the extremes of a linear function are at vertices and its
  Taylor form at a vertex is its value);
- small integer polynomials on dyadic vertices (evaluations exact): the vertex test is exactly
  "two vertices with opposite exact signs"; the Taylor test certifies only such boxes;
- the circle x^2 + y^2 - 1/2: the Taylor test of order 2 equals, box by box, the sign test at
  the two vertices extremal for the gradient at the centre (exact rationals);
- Algorithm 3 with C1 against its level-by-level definition over whole grids (no set
  iteration): a box is certified at level l iff it and its ancestors pass C0, C1 holds on it,
  and no ancestor at a level >= c1_level was certified;
- rational points of the circle lie in a returned box (certified or left at the last level).
"""
from fractions import Fraction
import itertools

import numpy as np
import pytest

import oracle
from exact import grid_box, poly_value
from paper_2406_09857_gb300 import synth


def _all_boxes(k, level):
    n = 1 << level
    return np.array(list(itertools.product(range(n), repeat=k)), dtype=np.int32)


def _vertex_values(exps, coefs, dom, level, tup):
    box = grid_box(dom, level, tup)
    return [poly_value(exps, coefs, [b[(v >> (len(box) - 1 - i)) & 1] for i, b in enumerate(box)])
            for v in range(1 << len(box))]


@pytest.mark.parametrize("kind,order", [(oracle.C1_VERTEX, 0), (oracle.C1_TAYLOR, 2),
                                        (oracle.C1_TAYLOR, 3)])
def test_linear_exact_predicate(kind, order):
    exps = [[1, 0, 0], [0, 1, 0], [0, 0, 1], [0, 0, 0]]
    coefs = [0.75, -1.25, 0.5, -0.125]
    dom = [-1.0, 1.0, -2.0, 2.0, -1.0, 1.0]
    t = _all_boxes(3, 3)
    inc = oracle.c1_boxes((np.array(exps, dtype=np.int32), np.array(coefs)), dom, 3, kind, t,
                          order)
    for i, tup in enumerate(t.tolist()):
        vals = _vertex_values(exps, coefs, dom, 3, tup)
        assert inc[i] == (min(vals) < 0 < max(vals)), tup
    assert 0 < inc.sum() < len(inc)


@pytest.mark.parametrize("k,d,level,seed", [(2, 5, 4, 1), (2, 8, 3, 2), (3, 4, 2, 3)])
def test_vertex_test_is_exact_sign_change(k, d, level, seed):
    (exps, coefs), = synth.random_small(k, d, 1, seed)
    dom = synth.cube(k)
    t = _all_boxes(k, level)
    inc = oracle.c1_boxes((exps, coefs), dom, level, oracle.C1_VERTEX, t)
    for i, tup in enumerate(t.tolist()):
        vals = _vertex_values(exps.tolist(), coefs.tolist(), dom, level, tup)
        assert inc[i] == (min(vals) < 0 < max(vals)), tup
    assert inc.sum() > 0


@pytest.mark.parametrize("k,d,level,order,seed", [(2, 6, 4, 2, 4), (2, 9, 5, 3, 5),
                                                  (3, 5, 3, 2, 6)])
def test_taylor_test_certifies_only_sign_changes(k, d, level, order, seed):
    (exps, coefs), = synth.random_small(k, d, 1, seed)
    dom = synth.cube(k)
    t = _all_boxes(k, level)
    inc = oracle.c1_boxes((exps, coefs), dom, level, oracle.C1_TAYLOR, t, order)
    for i in np.flatnonzero(inc):
        vals = _vertex_values(exps.tolist(), coefs.tolist(), dom, level, t[i].tolist())
        assert min(vals) < 0 < max(vals)
    assert inc.sum() > 0


def test_circle_taylor_order2_closed_form():
    exps = [[2, 0], [0, 2], [0, 0]]
    coefs = [1.0, 1.0, -0.5]
    dom = [-1.0, 1.0, -1.0, 1.0]
    level = 5
    t = _all_boxes(2, level)
    inc = oracle.c1_boxes((np.array(exps, dtype=np.int32), np.array(coefs)), dom, level,
                          oracle.C1_TAYLOR, t, 2)
    for i, tup in enumerate(t.tolist()):
        box = grid_box(dom, level, tup)
        c = [(l + h) / 2 for l, h in box]
        r = [(h - l) / 2 for l, h in box]
        s = [1 if 2 * ci >= 0 else -1 for ci in c]  # sign of the gradient 2c at the centre
        vmax = [ci + si * ri for ci, si, ri in zip(c, s, r)]
        vmin = [ci - si * ri for ci, si, ri in zip(c, s, r)]
        # the order-2 Taylor form of a quadratic at a point is its value there
        expect = poly_value(exps, coefs, vmax) > 0 > poly_value(exps, coefs, vmin)
        assert inc[i] == expect, tup
    assert inc.sum() > 0


def _levelwise(poly, dom, depth, kind, c1_level, order):
    """Certified boxes per level and the boxes left at `depth`, from per-box tests on whole
    grids: B is certified at level l iff every ancestor A (levels < l) and B pass C0, no
    ancestor at a level in [c1_level, l) is certified, and C1 holds on B."""
    k = len(dom) // 2
    c0, c1 = [], []
    for l in range(depth + 1):
        t = _all_boxes(k, l)
        if order:
            _, _, keep = oracle.taylor_boxes([poly], dom, l, order, t)
        else:
            _, _, keep, _ = oracle.eval_csf([poly], dom, l, t)
        c0.append(keep.reshape((1 << l,) * k))
        inc = oracle.c1_boxes(poly, dom, l, kind, t, order) if l >= c1_level else \
            np.zeros(len(t), np.uint8)
        c1.append(inc.reshape((1 << l,) * k))
    alive = np.ones((1,) * k, dtype=bool)  # passed C0 at every level so far, not certified
    cert, left = {}, None
    for l in range(depth + 1):
        if l > 0:
            for ax in range(k):
                alive = np.repeat(alive, 2, axis=ax)
        alive = alive & (c0[l] == 1)
        here = alive & (c1[l] == 1)
        cert[l] = np.argwhere(here).astype(np.int32)
        alive = alive & ~here
        if l == depth:
            left = np.argwhere(alive).astype(np.int32)
    return cert, left


@pytest.mark.parametrize("case", ["circle-vertex", "circle-taylor", "rand-vertex",
                                  "rand-taylor-horner0", "rand3-taylor"])
def test_alg3_with_c1_equals_levelwise_definition(case):
    circle = (np.array([[2, 0], [0, 2], [0, 0]], dtype=np.int32), np.array([1.0, 1.0, -0.5]))
    cases = {
        "circle-vertex": (circle, synth.cube(2), 7, oracle.C1_VERTEX, 3, 0),
        "circle-taylor": (circle, synth.cube(2), 7, oracle.C1_TAYLOR, 2, 2),
        "rand-vertex": (synth.random_small(2, 7, 1, 11)[0], synth.cube(2), 6, oracle.C1_VERTEX,
                        3, 2),
        "rand-taylor-horner0": (synth.random_small(2, 6, 1, 12)[0], synth.cube(2), 6,
                                oracle.C1_VERTEX, 2, 0),
        "rand3-taylor": (synth.random_small(3, 4, 1, 13)[0], synth.cube(3), 4,
                         oracle.C1_TAYLOR, 2, 2),
    }
    poly, dom, depth, kind, c1_level, order = cases[case]
    res = oracle.enclose_c1(poly, dom, depth, kind, c1_level, taylor_order=order)
    cert, left = _levelwise(poly, dom, depth, kind, c1_level, order)
    for l in range(depth + 1):
        got = res["inc_tuples"][res["inc_levels"] == l]
        assert np.array_equal(got, cert[l]), l
        assert res["included"][l] == len(cert[l])
    assert np.array_equal(res["tuples"], left)
    assert res["inc_tuples"].shape[0] > 0


def test_circle_points_are_covered():
    poly = (np.array([[2, 0], [0, 2], [0, 0]], dtype=np.int32), np.array([1.0, 1.0, -0.5]))
    dom = [-1.0, 1.0, -1.0, 1.0]
    depth = 8
    pts = [(Fraction(7, 10), Fraction(1, 10)), (Fraction(1, 10), Fraction(-7, 10)),
           (Fraction(1, 2), Fraction(1, 2)), (Fraction(-17, 26), Fraction(7, 26))]
    for kind, order in ((oracle.C1_VERTEX, 0), (oracle.C1_TAYLOR, 2)):
        res = oracle.enclose_c1(poly, dom, depth, kind, 3, taylor_order=order)
        boxes = [(int(l), tuple(t)) for l, t in zip(res["inc_levels"], res["inc_tuples"].tolist())]
        boxes += [(depth, tuple(t)) for t in res["tuples"].tolist()]
        for x, y in pts:
            assert x * x + y * y == Fraction(1, 2)
            hit = False
            for l, t in boxes:
                (x0, x1), (y0, y1) = grid_box(dom, l, t)
                hit = hit or (x0 <= x <= x1 and y0 <= y <= y1)
            assert hit, (kind, x, y)
        # certified boxes are disjoint across levels: none is inside another one
        for (l1, t1), (l2, t2) in itertools.combinations(boxes, 2):
            if l1 < l2:
                assert tuple(v >> (l2 - l1) for v in t2) != t1


def test_refusals():
    import ctypes

    p = synth.random_small(2, 4, 2, 20)
    k, npoly, off, E, C = oracle.pack(p)  # two equations: C1 is for one
    dom = np.ascontiguousarray(synth.cube(2))
    res = ctypes.c_void_p()
    rc = oracle.lib().orc_enclose_c1(k, npoly, oracle._p(off), oracle._p(E), oracle._p(C),
                                     oracle._p(dom), 3, 0, oracle.C1_VERTEX, 0,
                                     ctypes.byref(res))
    assert rc != 0
    with pytest.raises(oracle.OracleError):
        oracle.enclose_c1(p[0], synth.cube(2), 3, oracle.C1_TAYLOR, 0, taylor_order=1)
