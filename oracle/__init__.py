"""CPU oracle for CSF-amortized interval subdivision -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import this package.  The product library (``paper_2406_09857_gb300``) never imports it and
shares no code with it.

The arithmetic lives in ``vx_oracle.c`` (plain C, FP64, directed rounding through
``fesetround``); this module compiles it with gcc and marshals numpy arrays.  A polynomial
system is a list of ``(exps, coefs)`` pairs: ``exps`` int [nterms, k], ``coefs`` float64
[nterms].
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vx_oracle.c")
_SO = os.path.join(_HERE, "libvx_oracle.so")
# No FMA contraction, rounding-mode-aware optimisation, no fast-math: the oracle must round
# each operation on its own, in the direction the current rounding mode says.
CFLAGS = ["-O2", "-frounding-math", "-ffp-contract=off", "-fno-fast-math", "-std=c11", "-fPIC",
          "-shared"]

_lib = None


def build(force: bool = False) -> str:
    """Compile ``libvx_oracle.so`` next to its source when missing or stale."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".tmp%d" % os.getpid()
        subprocess.run(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"], check=True)
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_SO)
        P = ctypes.c_void_p
        i32, i64 = ctypes.c_int, ctypes.c_int64
        sysargs = [i32, i32, P, P, P]
        L.orc_eval_csf.argtypes = sysargs + [P, i32, P, i64, P, P, P, P]
        L.orc_eval_boxes.argtypes = sysargs + [P, i32, P, i64, P, P, P, P]
        L.orc_eval_grid.argtypes = sysargs + [P, P, P, P, i64, P, P, P, P]
        L.orc_csf.argtypes = [i32, P, i64, P, P, P]
        L.orc_enclose.argtypes = sysargs + [P, i32, ctypes.POINTER(P)]
        L.orc_enclose_from.argtypes = sysargs + [P, i32, P, i64, i32, ctypes.POINTER(P)]
        L.orc_result_count.argtypes = [P]
        L.orc_result_count.restype = i64
        L.orc_result_copy.argtypes = [P, P, P, P, P, P]
        L.orc_result_free.argtypes = [P]
        L.orc_brute_force.argtypes = sysargs + [P, i32, P]
        L.orc_eval_grid_complex.argtypes = [i32, i64, P, P, P, P, P, P, P, i64, P, P]
        L.orc_domain_exact.argtypes = [i32, P, i32]
        L.orc_prim.argtypes = [i32, P, P, i64, P]
        L.orc_imul.argtypes = [P, P, P, P, i64, P, P]
        L.orc_dense_powerform.argtypes = [P, P, i64, P, i32, P, i64, P, P]
        L.orc_taylor_boxes.argtypes = sysargs + [P, i32, i32, P, i64, P, P, P]
        L.orc_enclose_taylor.argtypes = sysargs + [P, i32, i32, ctypes.POINTER(P)]
        L.orc_c1_boxes.argtypes = sysargs + [P, i32, i32, i32, P, i64, P]
        L.orc_eval_csf_gen.argtypes = sysargs + [P, P, P, i32, P, i64, P, P, P, P]
        L.orc_enclose_gen.argtypes = sysargs + [P, P, P, i32, i32, ctypes.POINTER(P)]
        L.orc_enclose_c1.argtypes = sysargs + [P, i32, i32, i32, i32, ctypes.POINTER(P)]
        L.orc_result_inc_count.argtypes = [P]
        L.orc_result_inc_count.restype = i64
        L.orc_result_inc_copy.argtypes = [P, P, P, P]
        for f in ("orc_eval_csf", "orc_eval_boxes", "orc_eval_grid", "orc_csf", "orc_enclose",
                  "orc_enclose_from",
                  "orc_brute_force", "orc_eval_grid_complex", "orc_domain_exact",
                  "orc_dense_powerform", "orc_taylor_boxes", "orc_enclose_taylor",
                  "orc_c1_boxes", "orc_enclose_c1", "orc_eval_csf_gen", "orc_enclose_gen"):
            getattr(L, f).restype = i32
        _lib = L
    return _lib


class OracleError(RuntimeError):
    pass


def _check(rc: int, what: str):
    if rc != 0:
        raise OracleError("%s failed with code %d" % (what, rc))


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def pack(polys):
    """(k, npoly, term_off int64, exps int32 [T,k], coefs float64 [T]) of a system."""
    k = int(np.asarray(polys[0][0]).reshape(-1, np.asarray(polys[0][0]).shape[-1]).shape[1])
    offs = [0]
    E, C = [], []
    for exps, coefs in polys:
        e = np.ascontiguousarray(np.asarray(exps, dtype=np.int32).reshape(-1, k))
        c = np.ascontiguousarray(np.asarray(coefs, dtype=np.float64).reshape(-1))
        assert e.shape[0] == c.shape[0]
        E.append(e)
        C.append(c)
        offs.append(offs[-1] + e.shape[0])
    return (k, len(polys), np.asarray(offs, dtype=np.int64),
            np.ascontiguousarray(np.concatenate(E, axis=0)),
            np.ascontiguousarray(np.concatenate(C)))


def _tuples(tuples, k):
    t = np.ascontiguousarray(np.asarray(tuples, dtype=np.int32).reshape(-1, k))
    return t


def eval_csf(polys, domain, level, tuples):
    """Algorithm 2 on lex-sorted unique box indices of the level-``level`` grid.

    Returns (lo [npoly, n], hi [npoly, n], keep [n] uint8, work) where work counts
    interval multiply-adds."""
    k, npoly, off, E, C = pack(polys)
    t = _tuples(tuples, k)
    n = t.shape[0]
    dom = np.ascontiguousarray(np.asarray(domain, dtype=np.float64).reshape(-1))
    lo = np.empty((npoly, n))
    hi = np.empty((npoly, n))
    keep = np.empty(n, dtype=np.uint8)
    work = np.zeros(1, dtype=np.int64)
    _check(lib().orc_eval_csf(k, npoly, _p(off), _p(E), _p(C), _p(dom), int(level), _p(t), n,
                              _p(lo), _p(hi), _p(keep), _p(work)), "orc_eval_csf")
    return lo, hi, keep, int(work[0])


def eval_boxes(polys, domain, level, tuples):
    """Nested Horner on each box on its own (no sharing); same outputs as eval_csf."""
    k, npoly, off, E, C = pack(polys)
    t = _tuples(tuples, k)
    n = t.shape[0]
    dom = np.ascontiguousarray(np.asarray(domain, dtype=np.float64).reshape(-1))
    lo = np.empty((npoly, n))
    hi = np.empty((npoly, n))
    keep = np.empty(n, dtype=np.uint8)
    work = np.zeros(1, dtype=np.int64)
    _check(lib().orc_eval_boxes(k, npoly, _p(off), _p(E), _p(C), _p(dom), int(level), _p(t), n,
                                _p(lo), _p(hi), _p(keep), _p(work)), "orc_eval_boxes")
    return lo, hi, keep, int(work[0])



def dense_powerform(poly, domain, level, tuples):
    """Mode-wise midpoint-radius power form of one trivariate polynomial on each box:
    (mid, rad) arrays; every value on box i lies in [mid - rad, mid + rad] (binary64, to
    nearest, no margins)."""
    e, c = poly
    E = np.ascontiguousarray(np.asarray(e, dtype=np.int32).reshape(-1, 3))
    C = np.ascontiguousarray(np.asarray(c, dtype=np.float64).reshape(-1))
    t = _tuples(tuples, 3)
    n = t.shape[0]
    dom = np.ascontiguousarray(np.asarray(domain, dtype=np.float64).reshape(-1))
    mid = np.empty(n)
    rad = np.empty(n)
    _check(lib().orc_dense_powerform(_p(E), _p(C), int(E.shape[0]), _p(dom), int(level), _p(t), n,
                                     _p(mid), _p(rad)), "orc_dense_powerform")
    return mid, rad


def eval_grid(polys, xlists, tuples):
    """Algorithm 2 with explicit per-axis interval lists ``xlists[i] = (lo_array, hi_array)``."""
    k, npoly, off, E, C = pack(polys)
    t = _tuples(tuples, k)
    n = t.shape[0]
    xoff = np.zeros(k + 1, dtype=np.int64)
    for i, (a, _) in enumerate(xlists):
        xoff[i + 1] = xoff[i] + len(a)
    xlo = np.ascontiguousarray(np.concatenate([np.asarray(a, dtype=np.float64) for a, _ in xlists]))
    xhi = np.ascontiguousarray(np.concatenate([np.asarray(b, dtype=np.float64) for _, b in xlists]))
    lo = np.empty((npoly, n))
    hi = np.empty((npoly, n))
    keep = np.empty(n, dtype=np.uint8)
    work = np.zeros(1, dtype=np.int64)
    _check(lib().orc_eval_grid(k, npoly, _p(off), _p(E), _p(C), _p(xoff), _p(xlo), _p(xhi), _p(t),
                               n, _p(lo), _p(hi), _p(keep), _p(work)), "orc_eval_grid")
    return lo, hi, keep, int(work[0])


def csf(tuples, k):
    """(N [k], labels per depth, ptr per depth < k) of a lex-sorted unique tuple set."""
    t = _tuples(tuples, k)
    n = t.shape[0]
    N = np.zeros(k, dtype=np.int64)
    _check(lib().orc_csf(k, _p(t), n, _p(N), None, None), "orc_csf")
    labels = np.empty(max(int(N.sum()), 1), dtype=np.int32)
    ptr = np.empty(max(int(N[:-1].sum()) + k - 1, 1), dtype=np.int64)
    _check(lib().orc_csf(k, _p(t), n, _p(N), _p(labels), _p(ptr)), "orc_csf")
    labs, ptrs = [], []
    lo = po = 0
    for j in range(k):
        labs.append(labels[lo:lo + N[j]].copy())
        lo += N[j]
        if j + 1 < k:
            ptrs.append(ptr[po:po + N[j] + 1].copy())
            po += N[j] + 1
    return N, labs, ptrs


def enclose(polys, domain, depth, start_level=0, start=None):
    """Algorithm 3 to ``depth``: survivors of the last level plus per-level statistics.

    With ``start`` (lex-sorted unique box indices of level ``start_level``) the set S starts
    there instead of at the whole domain; the statistics cover levels 0..depth (zeros before
    start_level)."""
    k, npoly, off, E, C = pack(polys)
    dom = np.ascontiguousarray(np.asarray(domain, dtype=np.float64).reshape(-1))
    res = ctypes.c_void_p()
    L = lib()
    if start is None:
        _check(L.orc_enclose(k, npoly, _p(off), _p(E), _p(C), _p(dom), int(depth),
                             ctypes.byref(res)), "orc_enclose")
    else:
        st = _tuples(start, k)
        _check(L.orc_enclose_from(k, npoly, _p(off), _p(E), _p(C), _p(dom), int(start_level),
                                  _p(st), st.shape[0], int(depth), ctypes.byref(res)),
               "orc_enclose_from")
    return _result(res, k, depth)


def _result(res, k, depth):
    L = lib()
    try:
        n = L.orc_result_count(res)
        tup = np.empty((n, k), dtype=np.int32)
        tested = np.empty(depth + 1, dtype=np.int64)
        kept = np.empty(depth + 1, dtype=np.int64)
        nodes = np.empty((depth + 1, k), dtype=np.int64)
        work = np.empty(depth + 1, dtype=np.int64)
        L.orc_result_copy(res, _p(tup), _p(tested), _p(kept), _p(nodes), _p(work))
        ni = L.orc_result_inc_count(res)
        inc_levels = np.empty(ni, dtype=np.int32)
        inc_tuples = np.empty((ni, k), dtype=np.int32)
        included = np.empty(depth + 1, dtype=np.int64)
        L.orc_result_inc_copy(res, _p(inc_levels), _p(inc_tuples), _p(included))
    finally:
        L.orc_result_free(res)
    return {"tuples": tup, "tested": tested, "kept": kept, "nodes": nodes, "work": work,
            "inc_levels": inc_levels, "inc_tuples": inc_tuples, "included": included}


def brute_force(polys, domain, level):
    """Keep flag of every box of the level grid, each box tested on its own: shape (2^level,)*k."""
    k, npoly, off, E, C = pack(polys)
    dom = np.ascontiguousarray(np.asarray(domain, dtype=np.float64).reshape(-1))
    side = 1 << level
    keep = np.empty(side ** k, dtype=np.uint8)
    _check(lib().orc_brute_force(k, npoly, _p(off), _p(E), _p(C), _p(dom), int(level), _p(keep)),
           "orc_brute_force")
    return keep.reshape((side,) * k)


def eval_grid_complex(exps, coefs, xlists, tuples):
    """Algorithm 2 over complex points: ``coefs`` complex [T], ``xlists[i]`` complex arrays."""
    e = np.ascontiguousarray(np.asarray(exps, dtype=np.int32))
    k = e.shape[1]
    c = np.asarray(coefs, dtype=np.complex128)
    cre = np.ascontiguousarray(c.real)
    cim = np.ascontiguousarray(c.imag)
    xoff = np.zeros(k + 1, dtype=np.int64)
    for i, a in enumerate(xlists):
        xoff[i + 1] = xoff[i] + len(a)
    x = np.concatenate([np.asarray(a, dtype=np.complex128) for a in xlists])
    xre = np.ascontiguousarray(x.real)
    xim = np.ascontiguousarray(x.imag)
    t = _tuples(tuples, k)
    n = t.shape[0]
    vre = np.empty(n)
    vim = np.empty(n)
    _check(lib().orc_eval_grid_complex(k, e.shape[0], _p(e), _p(cre), _p(cim), _p(xoff), _p(xre),
                                       _p(xim), _p(t), n, _p(vre), _p(vim)), "orc_eval_grid_complex")
    return vre + 1j * vim


def domain_exact(domain, level):
    dom = np.ascontiguousarray(np.asarray(domain, dtype=np.float64).reshape(-1))
    return bool(lib().orc_domain_exact(len(dom) // 2, _p(dom), int(level)))


def prim(op, a, b):
    """op 0: RD(a*b), 1: RU(a*b), 2: RD(a+b), 3: RU(a+b), element-wise."""
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    out = np.empty_like(a)
    lib().orc_prim(int(op), _p(a), _p(b), a.size, _p(out))
    return out


def imul(alo, ahi, blo, bhi):
    arrs = [np.ascontiguousarray(x, dtype=np.float64) for x in (alo, ahi, blo, bhi)]
    lo = np.empty_like(arrs[0])
    hi = np.empty_like(arrs[0])
    lib().orc_imul(*[_p(x) for x in arrs], arrs[0].size, _p(lo), _p(hi))
    return lo, hi


def taylor_boxes(polys, domain, level, order, tuples):
    """Taylor form of the given order (Def. 3) of each polynomial on each box: lo, hi
    [npoly, n] and keep [n] (0 in every polynomial's form)."""
    k, npoly, off, E, C = pack(polys)
    t = _tuples(tuples, k)
    n = t.shape[0]
    dom = np.ascontiguousarray(np.asarray(domain, dtype=np.float64).reshape(-1))
    lo = np.empty((npoly, n))
    hi = np.empty((npoly, n))
    keep = np.empty(n, dtype=np.uint8)
    _check(lib().orc_taylor_boxes(k, npoly, _p(off), _p(E), _p(C), _p(dom), int(level), int(order),
                                  _p(t), n, _p(lo), _p(hi), _p(keep)), "orc_taylor_boxes")
    return lo, hi, keep


def enclose_taylor(polys, domain, depth, order):
    """Algorithm 3 with C0 on the Taylor form of the given order."""
    k, npoly, off, E, C = pack(polys)
    dom = np.ascontiguousarray(np.asarray(domain, dtype=np.float64).reshape(-1))
    res = ctypes.c_void_p()
    _check(lib().orc_enclose_taylor(k, npoly, _p(off), _p(E), _p(C), _p(dom), int(depth),
                                    int(order), ctypes.byref(res)), "orc_enclose_taylor")
    return _result(res, k, depth)


C1_TAYLOR = 1
C1_VERTEX = 2


def c1_boxes(poly, domain, level, kind, tuples, order=0):
    """Inclusion criterion C1 (Sec. 3.2) of one polynomial on each box: 1 where certified
    (kind C1_VERTEX: certified opposite signs at two vertices; C1_TAYLOR: the Taylor form of
    the given order >= 2 at the vertices extremal for its linear part)."""
    k, npoly, off, E, C = pack([poly])
    t = _tuples(tuples, k)
    n = t.shape[0]
    dom = np.ascontiguousarray(np.asarray(domain, dtype=np.float64).reshape(-1))
    inc = np.empty(n, dtype=np.uint8)
    _check(lib().orc_c1_boxes(k, npoly, _p(off), _p(E), _p(C), _p(dom), int(level), int(kind),
                              int(order), _p(t), n, _p(inc)), "orc_c1_boxes")
    return inc


def enclose_c1(poly, domain, depth, kind, c1_level, taylor_order=0):
    """Algorithm 3 with C0 (interval Horner, or the Taylor form of `taylor_order`) and C1 of
    `kind` from level `c1_level` on; stops when no box is left or after level `depth`.
    inc_levels / inc_tuples: the certified boxes (by level, then lexicographic); tuples: the
    boxes of level `depth` neither excluded nor certified."""
    k, npoly, off, E, C = pack([poly])
    dom = np.ascontiguousarray(np.asarray(domain, dtype=np.float64).reshape(-1))
    res = ctypes.c_void_p()
    _check(lib().orc_enclose_c1(k, npoly, _p(off), _p(E), _p(C), _p(dom), int(depth),
                                int(taylor_order), int(kind), int(c1_level), ctypes.byref(res)),
           "orc_enclose_c1")
    return _result(res, k, depth)


EQ, LE, GE, LT, GT = 0, 1, 2, 3, 4


def _his_rel(polys, his, rel):
    """Upper coefficient ends (concatenated; point coefficients where his[f] is None) and the
    relations (int32), or None for all-point / all-equation systems."""
    H = None
    if his is not None and any(h is not None for h in his):
        H = np.ascontiguousarray(np.concatenate(
            [np.asarray(c if h is None else h, dtype=np.float64).reshape(-1)
             for (_, c), h in zip(polys, his)]))
    R = None if rel is None else np.ascontiguousarray(np.asarray(rel, dtype=np.int32))
    return H, R


def eval_csf_gen(polys, domain, level, tuples, his=None, rel=None):
    """eval_csf for a system of equations and inequalities with interval coefficients:
    his[f] the upper coefficient ends of polynomial f (None: points), rel[f] in EQ, LE, GE,
    LT, GT (F = 0, F <= 0, F >= 0, F < 0, F > 0)."""
    k, npoly, off, E, C = pack(polys)
    H, R = _his_rel(polys, his, rel)
    t = _tuples(tuples, k)
    n = t.shape[0]
    dom = np.ascontiguousarray(np.asarray(domain, dtype=np.float64).reshape(-1))
    lo = np.empty((npoly, n))
    hi = np.empty((npoly, n))
    keep = np.empty(n, dtype=np.uint8)
    work = np.zeros(1, dtype=np.int64)
    _check(lib().orc_eval_csf_gen(k, npoly, _p(off), _p(E), _p(C), _p(H), _p(R), _p(dom),
                                  int(level), _p(t), n, _p(lo), _p(hi), _p(keep), _p(work)),
           "orc_eval_csf_gen")
    return lo, hi, keep, int(work[0])


def enclose_gen(polys, domain, depth, his=None, rel=None, taylor_order=0):
    """Algorithm 3 for a system of equations and inequalities with interval coefficients
    (his, rel as for eval_csf_gen); C0 on interval Horner or the Taylor form."""
    k, npoly, off, E, C = pack(polys)
    H, R = _his_rel(polys, his, rel)
    dom = np.ascontiguousarray(np.asarray(domain, dtype=np.float64).reshape(-1))
    res = ctypes.c_void_p()
    _check(lib().orc_enclose_gen(k, npoly, _p(off), _p(E), _p(C), _p(H), _p(R), _p(dom),
                                 int(depth), int(taylor_order), ctypes.byref(res)),
           "orc_enclose_gen")
    return _result(res, k, depth)
