"""Pins of the oracle's mode-wise midpoint-radius power form (the dense tensor-grid enclosure).

For a box with centre c and half-width r per axis, contracting one variable at a time (the
contractions of Property 1) maps <m_a, q_a> to <sum m_a c^a, sum |m_a|((|c|+r)^a - |c|^a) +
q_a (|c|+r)^a>.  Pinned here against things that do not use that formula:

- a monomial x1^a x2^b x3^c: mid = prod c_i^e_i, rad = prod (|c_i|+r_i)^e_i - prod |c_i|^e_i
  (exact in binary64 on dyadic boxes, checked with Fractions);
- an affine polynomial: the enclosure is its exact range, mid at the centre, rad = sum |b_i| r_i;
- containment: exact rational values at rational points of random boxes lie inside;
- the enclosure contains the nested interval Horner enclosure of the same box (interval Horner
  in midpoint-radius form is contained step by step, and the endpoint form inside that), so a
  box it excludes is excluded by C0 as well.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from exact import grid_box, poly_value
from paper_2406_09857_gb300 import synth


def _boxes(level, n, seed):
    return synth.random_tuples(3, level, n, seed)


def _centre_radius(dom, level, tup):
    box = grid_box(dom, level, tup)
    return [(l + h) / 2 for l, h in box], [(h - l) / 2 for l, h in box]


@pytest.mark.parametrize("e", [(3, 0, 0), (2, 5, 1), (0, 0, 7), (4, 4, 4)])
def test_monomial_closed_form(e):
    dom = [-1.0, 1.0, -0.5, 1.5, -2.0, 2.0]
    level = 4
    t = _boxes(level, 60, 11 + sum(e))
    mid, rad = oracle.dense_powerform((np.array([e], dtype=np.int32), np.array([1.0])), dom,
                                      level, t)
    for i, tup in enumerate(t.tolist()):
        c, r = _centre_radius(dom, level, tup)
        pm = Fraction(1)
        pu = Fraction(1)
        pa = Fraction(1)
        for ci, ri, ei in zip(c, r, e):
            pm *= ci ** ei
            pu *= (abs(ci) + ri) ** ei
            pa *= abs(ci) ** ei
        assert Fraction(mid[i]) == pm
        assert Fraction(rad[i]) == pu - pa


def test_affine_is_exact_range():
    exps = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], dtype=np.int32)
    coefs = np.array([0.375, -2.5, 1.25, 0.75])
    dom = [-1.0, 1.0] * 3
    level = 5
    t = _boxes(level, 80, 5)
    mid, rad = oracle.dense_powerform((exps, coefs), dom, level, t)
    for i, tup in enumerate(t.tolist()):
        c, r = _centre_radius(dom, level, tup)
        assert Fraction(mid[i]) == poly_value(exps.tolist(), coefs.tolist(), c)
        assert Fraction(rad[i]) == sum(abs(Fraction(b)) * ri for b, ri in zip(coefs[1:], r))


@pytest.mark.parametrize("d,level,seed", [(4, 3, 1), (7, 4, 2), (10, 2, 3)])
def test_contains_rational_point_values(d, level, seed):
    (exps, coefs), = synth.random_small(3, d, 1, seed)
    dom = synth.cube(3)
    t = _boxes(level, 25, seed + 3)
    mid, rad = oracle.dense_powerform((exps, coefs), dom, level, t)
    st = synth.Stream(seed + 99)
    for i, tup in enumerate(t.tolist()):
        box = grid_box(dom, level, tup)
        for _ in range(6):
            u = st.uniform_int(0, 64, 3)
            x = [l + (h - l) * Fraction(int(q), 64) for (l, h), q in zip(box, u)]
            v = poly_value(exps.tolist(), coefs.tolist(), x)
            slack = Fraction(1, 10 ** 12) * (abs(Fraction(mid[i])) + Fraction(rad[i]) + 1)
            assert Fraction(mid[i]) - Fraction(rad[i]) - slack <= v
            assert v <= Fraction(mid[i]) + Fraction(rad[i]) + slack


@pytest.mark.parametrize("d,level,seed,dense", [(6, 4, 21, True), (12, 5, 22, True),
                                                 (9, 3, 23, False)])
def test_contains_interval_horner(d, level, seed, dense):
    if dense:
        exps, coefs = synth.gaussian_tensor_poly(3, d, seed)
    else:
        (exps, coefs), = synth.random_small(3, d, 1, seed)
    dom = synth.cube(3)
    t = _boxes(level, 300, seed)
    mid, rad = oracle.dense_powerform((exps, coefs), dom, level, t)
    lo, hi, keep, _ = oracle.eval_boxes([(exps, coefs)], dom, level, t)
    tol = 1e-12 * (np.abs(mid) + rad + 1e-300)
    assert np.all(mid - rad - tol <= lo[0])
    assert np.all(hi[0] <= mid + rad + tol)
    # a box the power form excludes, interval Horner excludes too
    pf_keep = np.abs(mid) <= rad
    assert np.all(pf_keep | (keep == 0))
    assert pf_keep.sum() >= keep.sum()
