"""Polynomial packing on the host (vx_system_measure: no device), including the large
polynomials whose loops over their terms run on the library's host thread pool.

- the coefficients each stage reads match the closed forms of dense polynomials: total degree
  d in k variables reads M_j = C(d + k - j, k - j) (Def. 1 with every suffix monomial present),
  degree d per variable (d + 1)^(k - j), on both sides of the size from which the pool is used;
- a repeated monomial, a non-finite coefficient or a negative exponent is refused wherever it
  sits among the terms (another chunk than the first occurrence included);
- repeated and concurrent calls (several host threads at once, so that some find the pool
  busy and pack on their own thread) give the same counts.
"""
import math
import threading

import numpy as np
import pytest

from paper_2406_09857_gb300 import synth


@pytest.fixture(scope="module")
def vx():
    from paper_2406_09857_gb300 import build
    from paper_2406_09857_gb300 import vx as _vx

    build.build()
    _vx.lib()
    return _vx


def _total(k, d):
    return [math.comb(d + k - j, k - j) for j in range(k + 1)]


@pytest.mark.parametrize("k,d", [(2, 30), (3, 20), (3, 70), (4, 14), (2, 400)])
def test_total_degree_counts(vx, k, d):
    e, c = synth.kostlan_poly(k, d, 1600 + d)
    assert vx.measure([(e, c)])[0].tolist() == _total(k, d)


@pytest.mark.parametrize("k,d", [(3, 12), (3, 40)])
def test_per_variable_degree_counts(vx, k, d):
    e, c = synth.gaussian_tensor_poly(k, d, 1700 + d)
    assert vx.measure([(e, c)])[0].tolist() == [(d + 1) ** (k - j) for j in range(k + 1)]


def test_two_polynomials(vx):
    polys = [synth.kostlan_poly(3, 70, 1801), synth.kostlan_poly(3, 9, 1802)]
    M = vx.measure(polys)
    assert M[0].tolist() == _total(3, 70) and M[1].tolist() == _total(3, 9)


@pytest.mark.parametrize("where", [0, 31000, -1])
def test_refusals_anywhere(vx, where):
    e, c = synth.kostlan_poly(3, 70, 1901)  # 62 196 terms: packed on the pool
    e2 = np.concatenate([e, e[where:where + 1] if where != -1 else e[-1:]])
    with pytest.raises(vx.VxError, match="twice"):
        vx.measure([(e2, np.concatenate([c, c[:1]]))])
    c2 = c.copy()
    c2[where] = np.inf
    with pytest.raises(vx.VxError, match="coefficient"):
        vx.measure([(e, c2)])
    e3 = e.copy()
    e3[where, 1] = -2
    with pytest.raises(vx.VxError, match="exponent"):
        vx.measure([(e3, c)])


def test_repeated_and_concurrent_calls(vx):
    polys = [synth.kostlan_poly(3, 60, 2001)]
    want = _total(3, 60)
    for _ in range(5):
        assert vx.measure(polys)[0].tolist() == want
    got, errs = [], []

    def work():
        try:
            for _ in range(3):
                got.append(vx.measure(polys)[0].tolist())
        except Exception as ex:  # reported below
            errs.append(ex)

    th = [threading.Thread(target=work) for _ in range(4)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    assert not errs and len(got) == 12 and all(g == want for g in got)


@pytest.mark.skipif(not hasattr(__import__("os"), "fork"), reason="needs fork")
def test_packing_in_a_forked_child(vx):
    """A process forked after the pool started has none of its threads: it packs on a pool of
    its own and gets the same counts (so does the parent afterwards)."""
    import os
    import warnings

    polys = [synth.kostlan_poly(3, 60, 2101)]
    want = _total(3, 60)
    assert vx.measure(polys)[0].tolist() == want
    r, w = os.pipe()
    with warnings.catch_warnings():
        warnings.simplefilter("ignore", DeprecationWarning)  # fork of a threaded process
        pid = os.fork()
    if pid == 0:
        try:
            ok = vx.measure(polys)[0].tolist() == want
            os.write(w, b"1" if ok else b"0")
        finally:
            os._exit(0)
    os.close(w)
    got = os.read(r, 1)
    os.close(r)
    os.waitpid(pid, 0)
    assert got == b"1"
    assert vx.measure(polys)[0].tolist() == want
