"""Pin of the oracle's nesting order against hand-derived values (Algorithm 2, Sec. 2.2).

Algorithm 2 puts x_1 at the root of the tree: Horner in x_1 runs first, once per monomial of
the remaining variables, and its interval coefficients are evaluated in x_2, then x_3.  On a
box that is not a point the order changes the enclosure, so a pin that holds only for points,
for symmetric polynomials or for linear ones cannot see it.  The cases in
``golden/nesting_order.json`` were derived by hand from that definition (the steps are written
out in the file); every operation is exact in binary64, so the oracle must return the values
exactly.  The bivariate case gives [0, 4] in the paper's order and [-1, 4] with x_2 first; the
trivariate cases (an exponent gap and trailing powers in x_1) give values that no other order
of the three variables reproduces.
"""
import json
import os

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
with open(os.path.join(HERE, "golden", "nesting_order.json")) as f:
    GOLD = json.load(f)
CASES = {c["name"]: c for c in GOLD["cases"]}


def _case(name):
    c = CASES[name]
    exps = np.asarray(c["exps"], dtype=np.int32)
    coefs = np.asarray(c["coefs"], dtype=np.float64)
    box = np.asarray(c["box"], dtype=np.float64)
    return [(exps, coefs)], box, np.asarray(c["expected"], dtype=np.float64)


@pytest.mark.parametrize("name", sorted(CASES))
def test_level0_box_equals_hand_derivation(name):
    polys, box, want = _case(name)
    k = box.shape[0]
    t = np.zeros((1, k), dtype=np.int32)
    # the domain itself is the box at level 0
    lo, hi, keep, _ = oracle.eval_csf(polys, box.reshape(-1), 0, t)
    assert (lo[0, 0], hi[0, 0]) == (want[0], want[1])
    assert keep[0] == 1
    # nested Horner per box, and Algorithm 2 on explicit interval lists, agree
    lo, hi, _, _ = oracle.eval_boxes(polys, box.reshape(-1), 0, t)
    assert (lo[0, 0], hi[0, 0]) == (want[0], want[1])
    lo, hi, _, _ = oracle.eval_grid(polys, [(box[i, :1], box[i, 1:]) for i in range(k)], t)
    assert (lo[0, 0], hi[0, 0]) == (want[0], want[1])


@pytest.mark.parametrize("name", sorted(CASES))
def test_box_inside_a_grid(name):
    """The same box as one cell of a larger grid: the level-1 grid of a domain twice as wide
    towards the upper ends holds it as the cell (0, ..., 0), among cells evaluated beside it
    in one tree."""
    polys, box, want = _case(name)
    k = box.shape[0]
    dom = np.stack([box[:, 0], 2 * box[:, 1] - box[:, 0]], axis=1).reshape(-1)
    side = 2
    t = np.stack(np.meshgrid(*[np.arange(side)] * k, indexing="ij"), axis=-1).reshape(-1, k)
    lo, hi, _, _ = oracle.eval_csf(polys, dom, 1, t.astype(np.int32))
    assert (lo[0, 0], hi[0, 0]) == (want[0], want[1])


def test_bivariate_order_distinguishes():
    """The fixture's other order is a different interval: the pin can fail."""
    c = CASES["bivariate x1*x2 + x2"]
    assert c["other_order"]["x2 first"] != c["expected"]
