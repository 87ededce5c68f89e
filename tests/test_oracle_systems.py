"""Pins of the oracle for systems of equations and inequalities with interval coefficients
(Sec. 4: voxelize takes equations and inequalities; the systems (R) and (A) of Sec. 4.2).

- the five relations on x^2 + y^2 - 1/2 (enclosures exact on sign-definite boxes): the kept
  boxes are exactly those where the relation can hold (exact rationals), strict and non-strict
  told apart on boxes whose range touches 0;
- an interval coefficient: x^2 + y^2 - [c_lo, c_hi] has the enclosure [min - c_hi, max - c_lo];
- (R): the sqrt(3) coefficients as intervals contain the exact values (exact comparison in
  Q(sqrt 3)); the unit quaternions +-e_i solve it and stay in kept boxes;
- (A): the real/imaginary expansion equals exact Gaussian-rational evaluation of the complex
  polynomials; a boundary point solving the first equation stays in kept boxes of it alone;
  the whole system is excluded at depth 6 (the paper reports 0 boxes).
"""
from fractions import Fraction
import itertools
import math

import numpy as np
import pytest

import oracle
from exact import grid_box, poly_value
from paper_2406_09857_gb300 import synth

DISK = (np.array([[2, 0], [0, 2], [0, 0]], dtype=np.int32), np.array([1.0, 1.0, -0.5]))


def _all(k, level):
    n = 1 << level
    return np.array(list(itertools.product(range(n), repeat=k)), dtype=np.int32)


def _sq_range(a, b):
    lo = Fraction(0) if a <= 0 <= b else min(a * a, b * b)
    return lo, max(a * a, b * b)


@pytest.mark.parametrize("rel", [oracle.EQ, oracle.LE, oracle.GE, oracle.LT, oracle.GT])
def test_relations_closed_form(rel):
    dom = [-1.0, 1.0, -1.0, 1.0]
    level = 5
    t = _all(2, level)
    lo, hi, keep, _ = oracle.eval_csf_gen([DISK], dom, level, t, rel=[rel])
    half = Fraction(1, 2)
    strict_cases = 0
    for i, tup in enumerate(t.tolist()):
        (x0, x1), (y0, y1) = grid_box(dom, level, tup)
        a, b = _sq_range(x0, x1)
        c, d = _sq_range(y0, y1)
        mn, mx = a + c - half, b + d - half
        assert Fraction(lo[0, i]) == mn and Fraction(hi[0, i]) == mx
        can = {oracle.EQ: mn <= 0 <= mx, oracle.LE: mn <= 0, oracle.GE: mx >= 0,
               oracle.LT: mn < 0, oracle.GT: mx > 0}[rel]
        assert keep[i] == can, (tup, rel)
        strict_cases += (mn == 0) or (mx == 0)
    assert strict_cases > 0  # boxes whose range touches 0 exist at this level


@pytest.mark.parametrize("rel", [oracle.LE, oracle.GT])
def test_alg3_with_a_relation_closed_form(rel):
    """Relations keep inclusion isotonicity, so Algorithm 3 returns exactly the level's boxes
    where the relation can hold."""
    dom = [-1.0, 1.0, -1.0, 1.0]
    depth = 6
    res = oracle.enclose_gen([DISK], dom, depth, rel=[rel])
    expect = []
    for tup in _all(2, depth).tolist():
        (x0, x1), (y0, y1) = grid_box(dom, depth, tup)
        a, b = _sq_range(x0, x1)
        c, d = _sq_range(y0, y1)
        mn, mx = a + c - Fraction(1, 2), b + d - Fraction(1, 2)
        if (mn <= 0) if rel == oracle.LE else (mx > 0):
            expect.append(tup)
    assert np.array_equal(res["tuples"], np.array(expect, dtype=np.int32))


def test_interval_coefficient_closed_form():
    clo, chi = 0.5 - 2.0 ** -8, 0.5 + 2.0 ** -8
    polys = [(DISK[0], np.array([1.0, 1.0, -chi]))]
    his = [np.array([1.0, 1.0, -clo])]
    dom = [-1.0, 1.0, -1.0, 1.0]
    level = 6
    t = _all(2, level)
    lo, hi, keep, _ = oracle.eval_csf_gen(polys, dom, level, t, his=his)
    for i, tup in enumerate(t.tolist()):
        (x0, x1), (y0, y1) = grid_box(dom, level, tup)
        a, b = _sq_range(x0, x1)
        c, d = _sq_range(y0, y1)
        mn, mx = a + c - Fraction(chi), b + d - Fraction(clo)
        assert Fraction(lo[0, i]) == mn and Fraction(hi[0, i]) == mx
        assert keep[i] == (mn <= 0 <= mx)
    # wider than any point coefficient in it
    _, _, k1, _ = oracle.eval_csf_gen([DISK], dom, level, t)
    assert np.all(keep >= k1) and keep.sum() > k1.sum()


def _ge_sqrt3(A, B, v):
    """A + sqrt(3) B >= v, exactly (Fractions)."""
    u = v - A  # need sqrt(3) B >= u
    if B >= 0 and u <= 0:
        return True
    if B <= 0 and u > 0:
        return False
    if B >= 0:  # both positive
        return 3 * B * B >= u * u
    return 3 * B * B <= u * u  # both negative: sqrt3 B >= u  <=>  3B^2 <= u^2


def test_robotics_sqrt3_enclosures_contain_exact_values():
    R = synth.robotics()
    e, lo_c = R.polys[0]
    hi_c = R.his[0]
    for (c, r3, ex), a, b in zip(synth.ROBOTICS_F1, lo_c, hi_c):
        if r3:  # a <= c sqrt3 <= b, a and b adjacent doubles
            assert _ge_sqrt3(0, Fraction(c), Fraction(a)) and _ge_sqrt3(0, -Fraction(c), -Fraction(b))
            assert math.nextafter(a, math.inf) == b
        else:
            assert a == b == c
    level = 3
    t = synth.random_tuples(4, level, 300, 7)
    lo, hi, _, _ = oracle.eval_csf_gen(R.polys, R.domain, level, t, his=R.his, rel=R.rel)
    st = synth.Stream(8)
    for i, tup in enumerate(t.tolist()):
        box = grid_box(R.domain, level, tup)
        for _ in range(3):
            u = st.uniform_int(0, 16, 4)
            x = [l + (h - l) * Fraction(int(q), 16) for (l, h), q in zip(box, u)]
            A = sum(Fraction(c) * np.prod([xi ** p for xi, p in zip(x, ex)])
                    for c, r3, ex in synth.ROBOTICS_F1 if not r3)
            B = sum(Fraction(c) * np.prod([xi ** p for xi, p in zip(x, ex)])
                    for c, r3, ex in synth.ROBOTICS_F1 if r3)
            assert _ge_sqrt3(A, B, Fraction(lo[0, i]))  # lo <= F(x)
            assert _ge_sqrt3(-A, -B, -Fraction(hi[0, i]))  # F(x) <= hi


def test_robotics_unit_quaternions_kept():
    R = synth.robotics()
    res = oracle.enclose_gen(R.polys, R.domain, 4, R.his, R.rel)
    kept = set(map(tuple, res["tuples"].tolist()))
    side = 16

    def boxes_at(v):  # indices of the closed level-4 boxes of [-1, 1] that contain v
        u = (v + 1) * side / 2
        return sorted({j for j in (int(u) - 1, int(u)) if 0 <= j < side and j <= u <= j + 1})

    for i in range(4):
        for sgn in (-1, 1):
            q = [Fraction(0)] * 4
            q[i] = Fraction(sgn)
            for tup in itertools.product(*[boxes_at(v) for v in q]):
                assert tup in kept, (q, tup)


def _gauss_eval(terms, z):
    """Exact value of sum c z^a with z_j Gaussian rationals (pairs of Fractions)."""
    re, im = Fraction(0), Fraction(0)
    for c, a in terms:
        pr, pi = Fraction(c), Fraction(0)
        for zj, aj in zip(z, a):
            for _ in range(aj):
                pr, pi = pr * zj[0] - pi * zj[1], pr * zj[1] + pi * zj[0]
        re += pr
        im += pi
    return re, im


def test_automatic_expansion_is_exact():
    A = synth.automatic()
    st = synth.Stream(11)
    for _ in range(20):
        v = [Fraction(int(q), 64) for q in st.uniform_int(-64, 64, 6)]
        z = [(v[0], v[1]), (v[2], v[3]), (v[4], v[5])]
        for j, terms in enumerate(synth.AUTOMATIC_Z):
            re, im = _gauss_eval(terms, z)
            for part, val in ((0, re), (1, im)):
                e, c = A.polys[2 * j + part]
                assert poly_value(e.tolist(), c.tolist(), v) == val
    # the inequalities are the three unit disks
    for j in range(3):
        e, c = A.polys[8 + j]
        assert A.rel[8 + j] == synth.REL_LE
        x = [Fraction(0)] * 6
        x[2 * j], x[2 * j + 1] = Fraction(3, 5), Fraction(4, 5)
        assert poly_value(e.tolist(), c.tolist(), x) == 0


def test_automatic_first_equation_boundary_solution_kept():
    A = synth.automatic()
    # z = (1, 1, -1) solves z1 z2^2 - z1 z3 - 2 = 0 on the boundary of the polydisc
    re, im = _gauss_eval(synth.AUTOMATIC_Z[0], [(Fraction(1), Fraction(0))] * 2 +
                         [(Fraction(-1), Fraction(0))])
    assert re == 0 and im == 0
    polys = A.polys[0:2] + A.polys[8:]
    rel = [0, 0, 1, 1, 1]
    res = oracle.enclose_gen(polys, A.domain, 3, rel=rel)
    kept = set(map(tuple, res["tuples"].tolist()))
    # x = (1, 0, 1, 0, -1, 0): the last box on x1, x2; the first on x3; y's at the middle
    assert any(t[0] == 7 and t[2] == 7 and t[4] == 0 and t[1] in (3, 4) and t[3] in (3, 4)
               and t[5] in (3, 4) for t in kept)


def test_automatic_has_no_solution_in_the_polydisc():
    A = synth.automatic()
    res = oracle.enclose_gen(A.polys, A.domain, 6, A.his, A.rel)
    assert res["tuples"].shape[0] == 0
    assert res["kept"][5] > 0  # not trivially empty: boxes survive until level 5


def test_refusals():
    with pytest.raises(oracle.OracleError):
        oracle.eval_csf_gen([DISK], [-1.0, 1.0, -1.0, 1.0], 2, _all(2, 2), rel=[5])
    with pytest.raises(oracle.OracleError):  # lower end above the upper end
        oracle.eval_csf_gen([DISK], [-1.0, 1.0, -1.0, 1.0], 2, _all(2, 2),
                            his=[np.array([1.0, 1.0, -0.75])])
