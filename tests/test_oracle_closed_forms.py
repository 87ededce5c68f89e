"""Pins of the oracle's enclosures against closed forms and exact rational arithmetic.

- Containment (Sec. 3.2): {F(x) : x in B} is inside []F(B); checked with exact rational F at
  rational points of random boxes.
- A linear factor x_1 - 3/8: interval Horner of a linear polynomial is exact, so the kept set
  is exactly the boxes whose closed x_1-range contains 3/8.
- The circle x^2 + y^2 - 1/2 and the sphere x^2 + y^2 + z^2 - 1/2 on [-1,1]^k: at level >= 1
  no box straddles 0, nested Horner gives X*X + (Y*Y - 1/2) with exact dyadic squares, so the
  kept set is exactly {B : min_B |x|^2 <= 1/2 <= max_B |x|^2}.
- Products of linear factors with dyadic roots: every closed box containing a zero is kept.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from exact import grid_box, poly_value
from paper_2406_09857_gb300 import synth


@pytest.mark.parametrize("k,d,level,seed", [(1, 8, 4, 1), (2, 5, 3, 2), (3, 3, 2, 3)])
def test_containment_of_rational_points(k, d, level, seed):
    (exps, coefs), = synth.random_small(k, d, 1, seed)
    t = synth.random_tuples(k, level, 40, seed + 7)
    dom = synth.cube(k)
    lo, hi, _, _ = oracle.eval_csf([(exps, coefs)], dom, level, t)
    st = synth.Stream(seed + 1000)
    for b, tup in enumerate(t.tolist()):
        box = grid_box(dom, level, tup)
        for _ in range(6):
            u = st.uniform_int(0, 64, k)
            pt = [a + (c - a) * Fraction(int(x), 64) for (a, c), x in zip(box, u)]
            v = poly_value(exps.tolist(), coefs.tolist(), pt)
            assert Fraction(lo[0, b]) <= v <= Fraction(hi[0, b])


def _all_boxes(k, level):
    side = 1 << level
    g = np.stack(np.meshgrid(*[np.arange(side)] * k, indexing="ij"), axis=-1)
    return g.reshape(-1, k)


@pytest.mark.parametrize("k,depth", [(1, 6), (2, 2), (2, 3), (2, 5), (3, 4)])
def test_linear_factor_closed_form(k, depth):
    e = np.zeros((2, k), dtype=np.int32)
    e[0, 0] = 1
    coefs = np.array([1.0, -0.375])
    dom = synth.cube(k)
    res = oracle.enclose([(e, coefs)], dom, depth)
    root = Fraction(3, 8)
    want = [tuple(b) for b in _all_boxes(k, depth).tolist()
            if grid_box(dom, depth, b)[0][0] <= root <= grid_box(dom, depth, b)[0][1]]
    assert [tuple(r) for r in res["tuples"].tolist()] == sorted(want)
    # on [-1,1], 3/8 is a grid line from level 4 on: two columns, else one
    cols = 2 if depth >= 4 else 1
    assert len(want) == cols * (1 << (depth * (k - 1)))


def _sq_range(a, b):
    lo = Fraction(0) if a <= 0 <= b else min(a * a, b * b)
    return lo, max(a * a, b * b)


@pytest.mark.parametrize("k,depth", [(2, 1), (2, 4), (2, 7), (3, 3), (3, 5)])
def test_circle_sphere_closed_form(k, depth):
    e = np.zeros((k + 1, k), dtype=np.int32)
    for i in range(k):
        e[i, i] = 2
    coefs = np.array([1.0] * k + [-0.5])
    dom = synth.cube(k)
    res = oracle.enclose([(e, coefs)], dom, depth)
    half = Fraction(1, 2)
    want = []
    for b in _all_boxes(k, depth).tolist():
        rngs = [_sq_range(a, c) for a, c in grid_box(dom, depth, b)]
        if sum(r[0] for r in rngs) <= half <= sum(r[1] for r in rngs):
            want.append(tuple(b))
    assert [tuple(r) for r in res["tuples"].tolist()] == want
    # and the enclosure of each kept box is that exact range minus 1/2 (level >= 1)
    lo, hi, _, _ = oracle.eval_csf([(e, coefs)], dom, depth, res["tuples"])
    for i, b in enumerate(res["tuples"].tolist()):
        rngs = [_sq_range(a, c) for a, c in grid_box(dom, depth, b)]
        assert Fraction(lo[0, i]) == sum(r[0] for r in rngs) - half
        assert Fraction(hi[0, i]) == sum(r[1] for r in rngs) - half


def test_circle_rational_zeros_in_kept_boxes():
    # (u+v)/2, (u-v)/2 with u^2 + v^2 = 1 lies on x^2 + y^2 = 1/2
    e = np.array([[2, 0], [0, 2], [0, 0]], dtype=np.int32)
    coefs = np.array([1.0, 1.0, -0.5])
    depth = 6
    dom = synth.cube(2)
    kept = {tuple(r) for r in oracle.enclose([(e, coefs)], dom, depth)["tuples"].tolist()}
    side = 1 << depth
    for (p, q, r) in [(3, 4, 5), (5, 12, 13), (8, 15, 17), (7, 24, 25), (20, 21, 29)]:
        for su in (1, -1):
            for sv in (1, -1):
                u, v = Fraction(su * p, r), Fraction(sv * q, r)
                x, y = (u + v) / 2, (u - v) / 2
                assert x * x + y * y == Fraction(1, 2)
                # every closed grid box containing (x, y) must be kept
                for bx in _boxes_containing(x, side):
                    for by in _boxes_containing(y, side):
                        assert (bx, by) in kept


def _boxes_containing(x, side):
    # box t covers [-1 + 2t/side, -1 + 2(t+1)/side]
    s = (x + 1) * side / 2
    t = int(s)
    out = {min(max(t, 0), side - 1)}
    if s == t and t > 0:
        out.add(t - 1)
    return out


def test_product_of_linear_factors_zeros_kept():
    # f = (x - 1/4)(y + 3/8)(x + y - 1/2), expanded (dyadic coefficients)
    terms = {}

    def mul(p, q):
        r = {}
        for (a, b), c in p.items():
            for (a2, b2), c2 in q.items():
                r[(a + a2, b + b2)] = r.get((a + a2, b + b2), 0) + c * c2
        return r

    f = mul(mul({(1, 0): Fraction(1), (0, 0): Fraction(-1, 4)},
                {(0, 1): Fraction(1), (0, 0): Fraction(3, 8)}),
            {(1, 0): Fraction(1), (0, 1): Fraction(1), (0, 0): Fraction(-1, 2)})
    terms = {k: v for k, v in f.items() if v != 0}
    e = np.array(list(terms.keys()), dtype=np.int32)
    coefs = np.array([float(v) for v in terms.values()])
    depth = 6
    side = 1 << depth
    kept = {tuple(r) for r in oracle.enclose([(e, coefs)], synth.cube(2), depth)["tuples"].tolist()}
    zeros = []
    for i in range(-16, 17):
        s = Fraction(i, 16)
        zeros += [(Fraction(1, 4), s), (s, Fraction(-3, 8)), (s, Fraction(1, 2) - s)]
    for x, y in zeros:
        if abs(x) > 1 or abs(y) > 1:
            continue
        assert poly_value(e.tolist(), coefs.tolist(), [x, y]) == 0
        for bx in _boxes_containing(x, side):
            for by in _boxes_containing(y, side):
                assert (bx, by) in kept
    # and the enclosure is not trivial: far-away boxes are gone
    assert len(kept) < side * side // 4
