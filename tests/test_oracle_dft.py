"""Sec. 3.1 ("The Fast Fourier Transform Revisited"): the DFT as an Algorithm-2 evaluation.

As printed, the identity v_j = F(g_{i_1..i_k}) with X_j = {1, w^(2^(k-j))} does not hold for
k >= 2 (checked below).  The reading used here: with
    F = sum_e u_{sum_m e_m 2^(m-1)} prod_m x_m^(e_m),
the DFT is v_j = F(w^j, w^(2j), ..., w^(2^(k-1) j)); coordinate m only depends on
j mod 2^(k-m+1), so with x_k at the root the evaluation points form a sparse subset of a
grid (2^t CSF nodes at depth t) and Algorithm 2 computes the DFT in O(k 2^k) operations.
On the real interval engine the exact special case X_m = {[1,1], [-1,-1]} is the
Walsh-Hadamard transform of integer u.
"""
import numpy as np
import pytest
from scipy.linalg import hadamard

import oracle
from paper_2406_09857_gb300 import synth


def _multilinear(k):
    """Exponent tuples e in {0,1}^k with u-index sum_m e_m 2^(m-1)."""
    e = np.array([[(n >> m) & 1 for m in range(k)] for n in range(1 << k)], dtype=np.int32)
    return e


def test_printed_identity_fails_for_k2():
    k = 2
    u = synth.Stream(5).normal(4) + 0j
    w = np.exp(-2j * np.pi / 4)
    v = np.fft.fft(u)
    # printed: F = sum u_{i1 + i2 2} x1^i1 x2^i2, X_1 = {1, w^2}, X_2 = {1, w}, g = (w^(2 i1), w^i2)
    printed = []
    for j in range(4):
        i1, i2 = (j >> 1) & 1, j & 1
        x1, x2 = w ** (2 * i1), w ** i2
        printed.append(sum(u[a + 2 * b] * x1 ** a * x2 ** b for a in (0, 1) for b in (0, 1)))
    assert not np.allclose(printed, v)


@pytest.mark.parametrize("k", [1, 2, 3, 5, 8])
def test_dft_by_csf_evaluation(k):
    N = 1 << k
    st = synth.Stream(100 + k)
    u = st.normal(N) + 1j * st.normal(N)
    e = _multilinear(k)  # variables x_1..x_k
    # root = x_k: reorder the variables so that y_t = x_{k-t+1}
    ey = e[:, ::-1].copy()
    w = np.exp(-2j * np.pi / N)
    # axis t (1-based) holds y_t = x_{k-t+1} = w^(r 2^(k-t)), r = j mod 2^t
    xl = [np.array([w ** (r << (k - t)) for r in range(1 << t)]) for t in range(1, k + 1)]
    tuples = sorted({tuple(j % (1 << t) for t in range(1, k + 1)) for j in range(N)})
    vals = oracle.eval_grid_complex(ey, u, xl, tuples)
    # map each tuple back to j: the deepest coordinate is j mod 2^k = j
    got = np.empty(N, dtype=np.complex128)
    for tup, v in zip(tuples, vals):
        got[tup[-1]] = v
    N_nodes, _, _ = oracle.csf(np.asarray(tuples), k)
    assert N_nodes.tolist() == [1 << t for t in range(1, k + 1)]
    ref = np.fft.fft(u)
    tol = 8 * k * np.finfo(float).eps * np.abs(u).sum()
    assert np.max(np.abs(got - ref)) <= tol


@pytest.mark.parametrize("k", [1, 2, 3, 4, 6])
def test_walsh_hadamard_exact(k):
    N = 1 << k
    u = synth.Stream(200 + k).uniform_int(-50, 50, N).astype(np.float64)
    e = _multilinear(k)
    xl = [([1.0, -1.0], [1.0, -1.0])] * k
    tuples = np.array([[(j >> m) & 1 for m in range(k)] for j in range(N)], dtype=np.int32)
    order = np.lexsort(tuples.T[::-1])
    tuples = tuples[order]
    lo, hi, _, work = oracle.eval_grid([(e, u)], xl, tuples)
    j = (tuples * (1 << np.arange(k))).sum(axis=1)
    ref = hadamard(N).astype(np.float64) @ u
    assert np.array_equal(lo[0], ref[j]) and np.array_equal(hi[0], ref[j])
    # Property 1 on the 2x...x2 grid: sum_t 2^t * 2^(k-t) = k 2^k multiply-adds
    assert work == k * N
