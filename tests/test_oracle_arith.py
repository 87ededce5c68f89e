"""Pins of the oracle's interval arithmetic against exact rationals.

Sec. 3.2 ("Exclusion Criterion") asks for an interval []F(B) with {F(x) : x in B} inside it;
the oracle reads this as outward rounding: lower endpoints rounded down, upper rounded up.
These tests check each primitive against the exact rational result rounded by hand, so a
wrong direction, a dropped negation or a compiler that folds -((-a)*b) into a*b fails here.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from exact import rd, ru
from paper_2406_09857_gb300 import synth


def _doubles(seed, n, huge=True):
    st = synth.Stream(seed)
    mant = 1.0 + st.unit(n)
    expo = st.uniform_int(-60, 60, n)
    sign = np.where(st.uniform_int(0, 1, n) == 1, -1.0, 1.0)
    x = sign * np.ldexp(mant, expo)
    # a few special values: zeros of both signs, small integers, subnormal-range results
    specials = np.array([0.0, -0.0, 1.0, -1.0, 3.0, 0.5, 2.0 ** -1070, -(2.0 ** -1060),
                         1e300 if huge else 1e30])
    x[: specials.size] = specials
    return x


@pytest.mark.parametrize("op", [0, 1, 2, 3])
def test_directed_primitives_exact(op):
    a = _doubles(11 + op, 400)
    b = _doubles(101 + op, 400)[::-1].copy()
    b[:9] = np.array([1.0, 2.0 ** -20, -3.0, 0.0, -0.0, 7.0, 2.0 ** -10, 0.75, -1e-300])
    out = oracle.prim(op, a, b)
    for x, y, z in zip(a.tolist(), b.tolist(), out.tolist()):
        q = Fraction(x) * Fraction(y) if op < 2 else Fraction(x) + Fraction(y)
        want = rd(q) if op in (0, 2) else ru(q)
        assert z == want, (op, x, y, z, want)


def test_interval_product_is_outward_rounded_hull():
    st = synth.Stream(7)
    n = 300
    a = _doubles(21, n, huge=False)
    b = _doubles(22, n, huge=False)
    wa = np.abs(_doubles(23, n, huge=False)) * st.unit(n)
    wb = np.abs(_doubles(24, n, huge=False)) * st.unit(n)
    alo, ahi = a, a + wa
    blo, bhi = b, b + wb
    # straddling, one-signed and degenerate intervals
    alo[:4] = [-1.0, -2.0, 0.0, 3.0]
    ahi[:4] = [2.0, -1.0, 0.0, 3.0]
    blo[:4] = [-3.0, -0.5, -1.0, -1.0]
    bhi[:4] = [0.25, 4.0, 1.0, 1.0]
    lo, hi = oracle.imul(alo, ahi, blo, bhi)
    for i in range(n):
        prods = [Fraction(x) * Fraction(y) for x in (alo[i], ahi[i]) for y in (blo[i], bhi[i])]
        assert lo[i] == rd(min(prods)), i
        assert hi[i] == ru(max(prods)), i


def test_horner_univariate_degenerate_dyadic_is_exact():
    # p(x) = 3x^4 - 2x^3 + x - 5 at dyadic points: every intermediate is exact in binary64,
    # so the interval collapses to the exact value (Algorithm 1 on a point interval).
    exps = np.array([[4], [3], [1], [0]])
    coefs = np.array([3.0, -2.0, 1.0, -5.0])
    for num in range(-16, 17):
        x = Fraction(num, 8)
        xl = [float(x)]
        lo, hi, _, work = oracle.eval_grid([(exps, coefs)], [(xl, xl)], [[0]])
        v = 3 * x ** 4 - 2 * x ** 3 + x - 5
        assert Fraction(lo[0, 0]) == v and Fraction(hi[0, 0]) == v
        assert work == 4  # one multiply per degree step: the gap 3->1 costs two


def test_horner_gap_and_trailing_power():
    # x^2 + x^5 has no constant term: the result must still be multiplied by x^2 at the end.
    exps = np.array([[5], [2]])
    coefs = np.array([1.0, 1.0])
    for x in (Fraction(3, 4), Fraction(-5, 8), Fraction(1)):
        lo, hi, _, work = oracle.eval_grid([(exps, coefs)], [([float(x)], [float(x)])], [[0]])
        assert Fraction(lo[0, 0]) == x ** 2 + x ** 5 == Fraction(hi[0, 0])
        assert work == 5


def test_interval_horner_contains_range_and_matches_hand_interval():
    # [a,b] = [1/2, 3/4], p(x) = x^2 - x: by hand, Horner gives ((1*X) - 1)*X with
    # X - 1 = [-1/2, -1/4] and then [-1/2,-1/4]*[1/2,3/4] = [-3/8, -1/8].
    exps = np.array([[2], [1]])
    coefs = np.array([1.0, -1.0])
    lo, hi, _, _ = oracle.eval_grid([(exps, coefs)], [([0.5], [0.75])], [[0]])
    assert lo[0, 0] == -0.375 and hi[0, 0] == -0.125
