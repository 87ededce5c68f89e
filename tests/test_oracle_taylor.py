"""Pins of the oracle's Taylor form (Def. 3) and of Algorithm 3 with C0 on it.

T_m(F, B) = sum_{|a|<m} G_a(c) (x-c)^a + sum_{|a|=m} []G_a(B) (x-c)^a with G_a = d^a F / a!,
checked against things that do not use that code:
- closed forms written out with Fractions: an affine polynomial (its exact range, any order),
  x^2 at order 1, x^3 at order 2, x*y at order 2;
- containment of exact rational values at rational points of random boxes (orders 1-3);
- Algorithm 3 with the Taylor criterion keeps every box holding a sampled rational zero of the
  circle, and returns a subset of the level's boxes whose own Taylor form contains 0.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from exact import grid_box, poly_value
from paper_2406_09857_gb300 import synth


def _cr(dom, level, tup):
    box = grid_box(dom, level, tup)
    return [(l + h) / 2 for l, h in box], [(h - l) / 2 for l, h in box]


def _ivl_mul(a, b):
    p = [a[0] * b[0], a[0] * b[1], a[1] * b[0], a[1] * b[1]]
    return min(p), max(p)


@pytest.mark.parametrize("order", [1, 2, 3])
def test_affine_is_exact_range(order):
    exps = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], dtype=np.int32)
    coefs = np.array([0.375, -2.5, 1.25, 0.75])
    dom = [-1.0, 1.0] * 3
    t = synth.random_tuples(3, 4, 50, 3)
    lo, hi, _ = oracle.taylor_boxes([(exps, coefs)], dom, 4, order, t)
    for i, tup in enumerate(t.tolist()):
        c, r = _cr(dom, 4, tup)
        v = poly_value(exps.tolist(), coefs.tolist(), c)
        rad = sum(abs(Fraction(b)) * ri for b, ri in zip(coefs[1:], r))
        assert Fraction(lo[0, i]) == v - rad and Fraction(hi[0, i]) == v + rad


def test_square_order1_closed_form():
    exps = np.array([[2]], dtype=np.int32)
    dom = [-1.0, 1.0]
    t = np.arange(16, dtype=np.int32).reshape(-1, 1)
    lo, hi, _ = oracle.taylor_boxes([(exps, np.array([1.0]))], dom, 4, 1, t)
    for i, tup in enumerate(t.tolist()):
        (c,), (r,) = _cr(dom, 4, tup)
        d = _ivl_mul((2 * (c - r), 2 * (c + r)), (-r, r))  # []F'(B) (x - c)
        assert Fraction(lo[0, i]) == c * c + d[0] and Fraction(hi[0, i]) == c * c + d[1]


def test_cube_order2_closed_form():
    exps = np.array([[3]], dtype=np.int32)
    dom = [-2.0, 2.0]
    t = np.arange(32, dtype=np.int32).reshape(-1, 1)
    lo, hi, _ = oracle.taylor_boxes([(exps, np.array([1.0]))], dom, 5, 2, t)
    for i, tup in enumerate(t.tolist()):
        (c,), (r,) = _cr(dom, 5, tup)
        # c^3 + 3c^2 (x-c) + [](3x)(B) (x-c)^2, (x-c)^2 in [0, r^2]
        a = (c ** 3 - 3 * c * c * r, c ** 3 + 3 * c * c * r)
        b = _ivl_mul((3 * (c - r), 3 * (c + r)), (Fraction(0), r * r))
        assert Fraction(lo[0, i]) == a[0] + b[0] and Fraction(hi[0, i]) == a[1] + b[1]


def test_xy_order2_closed_form():
    exps = np.array([[1, 1]], dtype=np.int32)
    dom = [-1.0, 1.0, -1.0, 1.0]
    t = synth.random_tuples(2, 3, 40, 9)
    lo, hi, _ = oracle.taylor_boxes([(exps, np.array([2.0]))], dom, 3, 2, t)
    for i, tup in enumerate(t.tolist()):
        (c1, c2), (r1, r2) = _cr(dom, 3, tup)
        # 2 (c1 c2 + c2 (x-c1) + c1 (y-c2) + (x-c1)(y-c2))
        lo_e = 2 * (c1 * c2 - abs(c2) * r1 - abs(c1) * r2 - r1 * r2)
        hi_e = 2 * (c1 * c2 + abs(c2) * r1 + abs(c1) * r2 + r1 * r2)
        assert Fraction(lo[0, i]) == lo_e and Fraction(hi[0, i]) == hi_e


@pytest.mark.parametrize("k,d,level,order,seed", [(1, 9, 4, 1, 1), (2, 6, 3, 2, 2),
                                                  (3, 4, 2, 2, 3), (2, 7, 4, 3, 4)])
def test_contains_rational_point_values(k, d, level, order, seed):
    (exps, coefs), = synth.random_small(k, d, 1, seed)
    dom = synth.cube(k)
    t = synth.random_tuples(k, level, 30, seed + 5)
    lo, hi, _ = oracle.taylor_boxes([(exps, coefs)], dom, level, order, t)
    st = synth.Stream(seed + 77)
    for i, tup in enumerate(t.tolist()):
        box = grid_box(dom, level, tup)
        for _ in range(5):
            u = st.uniform_int(0, 64, k)
            x = [l + (h - l) * Fraction(int(q), 64) for (l, h), q in zip(box, u)]
            v = poly_value(exps.tolist(), coefs.tolist(), x)
            assert Fraction(lo[0, i]) <= v <= Fraction(hi[0, i])


def test_taylor_enclosure_keeps_zeros_and_is_its_own_criterion():
    # circle x^2 + y^2 - 1/2: rational zeros (3/5, 4/5)/sqrt(2)... use points on x^2+y^2 = 1/2
    # with rational coordinates: (1/2, 1/2), (-1/2, 1/2), (7/10, 1/10), (1/10, -7/10)
    exps = np.array([[2, 0], [0, 2], [0, 0]], dtype=np.int32)
    coefs = np.array([1.0, 1.0, -0.5])
    dom = [-1.0, 1.0, -1.0, 1.0]
    depth = 6
    res = oracle.enclose_taylor([(exps, coefs)], dom, depth, 2)
    kept = set(map(tuple, res["tuples"].tolist()))
    side = 1 << depth
    for x, y in [(Fraction(1, 2), Fraction(1, 2)), (Fraction(-1, 2), Fraction(1, 2)),
                 (Fraction(7, 10), Fraction(1, 10)), (Fraction(1, 10), Fraction(-7, 10))]:
        assert x * x + y * y == Fraction(1, 2)
        i = min(int((x + 1) / 2 * side), side - 1)
        j = min(int((y + 1) / 2 * side), side - 1)
        assert (i, j) in kept
    # the survivors pass the Taylor test on their own level
    _, _, keep = oracle.taylor_boxes([(exps, coefs)], dom, depth, 2, res["tuples"])
    assert keep.all()
    # a box that fails its own test is never returned
    allb = np.stack(np.meshgrid(np.arange(side), np.arange(side), indexing="ij"),
                    -1).reshape(-1, 2).astype(np.int32)
    _, _, kall = oracle.taylor_boxes([(exps, coefs)], dom, depth, 2, allb)
    own = set(map(tuple, allb[kall == 1].tolist()))
    assert kept <= own
