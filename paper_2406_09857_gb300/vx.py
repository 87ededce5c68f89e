"""ctypes binding of ``libvx`` (``include/vx.h``): argument marshalling only.

Every step of the computation runs in the library's CUDA kernels.  Device buffers are torch
CUDA tensors (passed by ``data_ptr()``) and streams are torch streams (``cuda_stream``).  If the
library has not been built, or no CUDA device is present, the calls raise: there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libvx.so")

OK, EINVAL, ENOMEM, ECAPACITY, EOVERFLOW, ETIMEOUT, ECUDA = 0, -1, -2, -3, -4, -5, -6
KMAX, MAXPOLY, MAXLEVEL = 6, 16, 24
FP64, FP32_MIDRAD, FP32 = 0, 1, 2
C1_TAYLOR, C1_VERTEX = 1, 2
EQ, LE, GE, LT, GT = 0, 1, 2, 3, 4  # relation of a polynomial: F = 0, <= 0, >= 0, < 0, > 0

_lib = None


class VxError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("vx error %d: %s" % (code, msg))
        self.code = code


class Poly(ctypes.Structure):
    _fields_ = [("nvars", ctypes.c_int32), ("nterms", ctypes.c_int32),
                ("exps", ctypes.c_void_p), ("coefs", ctypes.c_void_p)]


class Opts(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("fp64_final", ctypes.c_int32),
                ("fp64_recheck", ctypes.c_int32), ("theta", ctypes.c_float),
                ("timing", ctypes.c_int32), ("taylor_order", ctypes.c_int32),
                ("c1", ctypes.c_int32), ("c1_level", ctypes.c_int32),
                ("small_level_madds", ctypes.c_int32), ("recheck_last", ctypes.c_int32),
                ("max_level_boxes", ctypes.c_int32), ("first_level", ctypes.c_int32),
                ("host_codes", ctypes.c_int32)]


def lib() -> ctypes.CDLL:
    """Loads the in-tree ``libvx.so``; raises ImportError if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError("libvx.so is not built (%s); run paper_2406_09857_gb300/build.py"
                          % LIB_PATH)
    L = ctypes.CDLL(LIB_PATH)
    P, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    PP = ctypes.POINTER(ctypes.c_void_p)
    sig = {
        "vx_last_error": ([], ctypes.c_char_p),
        "vx_system_create": ([P, i32, P, PP], i32),
        "vx_system_create_ex": ([P, P, P, i32, P, PP], i32),
        "vx_system_free": ([P], None),
        "vx_system_info": ([P, P, P, P], i32),
        "vx_system_measure": ([P, i32, P], i32),
        "vx_system_device_bytes": ([P, P], i32),
        "vx_system_upload_bytes": ([P, P], i32),
        "vx_kernel_launches": ([], i64),
        "vx_set_wait_limit": ([i64], i32),
        "vx_autotune": ([i32, ctypes.c_char_p], i32),
        "vx_autotune_entries": ([], i32),
        "vx_autotune_clear": ([], None),
        "vx_csf_build": ([i32, i32, P, i64, P, PP], i32),
        "vx_csf_free": ([P], None),
        "vx_csf_full_grid": ([i32, i32, P, PP], i32),
        "vx_csf_nodes": ([P, P, P, P], i32),
        "vx_csf_export": ([P, i32, P, P, P], i32),
        "vx_csf_tuples": ([P, P, P], i32),
        "vx_csf_eval_level": ([P, P, P, i32, P, P, P, P], i32),
        "vx_csf_eval_level_static": ([P, P, P, i32, P, P, P, P], i32),
        "vx_csf_eval_grid": ([P, P, P, P, P, i32, P, P, P, P], i32),
        "vx_csf_eval_level_taylor": ([P, P, P, i32, P, P, P, P], i32),
        "vx_csf_c1": ([P, P, P, i32, i32, P, P], i32),
        "vx_csf_taylor_level": ([P, P, P, i32, i32, P, P, P, P], i32),
        "vx_result_included": ([P, P, P, P], i32),
        "vx_result_box_codes": ([P, P, P, P], i32),
        "vx_csf_subdivide": ([P, P, P, PP], i32),
        "vx_csf_compact": ([P, P, P, P, PP], i32),
        "vx_enclose_system": ([P, P, i32, P, P, PP], i32),
        "vx_enclose": ([P, i32, P, i32, P, PP], i32),
        "vx_enclose_from": ([P, P, P, i32, P, P, PP], i32),
        "vx_enclose_batch": ([P, P, P, P, i32, P, i32, P], i32),
        "vx_result_boxes": ([P, P, P], i32),
        "vx_result_csf": ([P, PP], i32),
        "vx_result_stats": ([P, P, P, P, P, P, P], i32),
        "vx_result_recheck64": ([P, P], i32),
        "vx_result_timing": ([P, P, P, P, P], i32),
        "vx_kernel_kind_name": ([i32], ctypes.c_char_p),
        "vx_result_elapsed_ms": ([P, P], i32),
        "vx_result_free": ([P], None),
        "vx_dense_plan_create": ([P, i32, P, P, PP], i32),
        "vx_dense_plan_bytes": ([P, P], i32),
        "vx_dense_plan_free": ([P], None),
        "vx_dense_prefilter": ([P, P, P], i32),
        "vx_dense_check_status": ([P], i32),
        "vx_dense_values": ([P, i32, P, P, P], i32),
        "vx_dense_level": ([P, P, P, P, P], i32),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _lib = L
    return L


def autotune(mode=1, cache_path=None):
    """Autotuner of the evaluation kernels: mode 1 tunes each new launch shape, 0 uses the
    heuristics; cache_path (optional) is read now and appended to."""
    _check(lib().vx_autotune(int(mode), cache_path.encode() if cache_path else None))


def autotune_entries() -> int:
    return int(lib().vx_autotune_entries())


def kernel_launches() -> int:
    """Kernels launched by libvx in this process so far."""
    return int(lib().vx_kernel_launches())


def declared_symbols():
    """Names of the functions declared in include/vx.h."""
    import re

    hdr = os.path.join(os.path.dirname(HERE), "include", "vx.h")
    text = open(hdr).read()
    return sorted(set(re.findall(r"\b(vx_[a-z0-9_]+)\s*\(", text)))


def _check(rc: int):
    if rc != OK:
        msg = lib().vx_last_error()
        raise VxError(rc, msg.decode() if msg else "")


def _ptr(t) -> int:
    return 0 if t is None else t.data_ptr()


def _stream(stream) -> int:
    import torch

    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


def _np_ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _polys(polys):
    """Keeps the numpy arrays alive with the vx_poly array that points into them."""
    keep = []
    arr = (Poly * len(polys))()
    for i, (exps, coefs) in enumerate(polys):
        e = np.ascontiguousarray(np.asarray(exps, dtype=np.int32))
        c = np.ascontiguousarray(np.asarray(coefs, dtype=np.float64))
        if e.ndim != 2 or e.shape[0] != c.shape[0]:
            raise ValueError("exps must be [nterms, nvars] and coefs [nterms]")
        keep += [e, c]
        arr[i] = Poly(e.shape[1], e.shape[0], e.ctypes.data, c.ctypes.data)
    return arr, keep


def measure(polys) -> np.ndarray:
    """vx_system_measure: the packing checks and the coefficients each stage reads, M
    [npoly, k+1] as System.info() gives them, on the host only (no device)."""
    arr, keep = _polys(polys)
    k = arr[0].nvars
    M = np.zeros((len(polys), k + 1), dtype=np.int64)
    _check(lib().vx_system_measure(arr, len(polys), M.ctypes.data))
    return M


def _domain(domain) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(domain, dtype=np.float64).reshape(-1))


def make_opts(mode=FP64, fp64_final=False, fp64_recheck=False, theta=0.5, timing=False,
              taylor_order=0, c1=0, c1_level=0, small_level_madds=0, recheck_last=False,
              max_level_boxes=0, first_level=0, host_codes=False) -> Opts:
    o = Opts()
    o.host_codes = int(bool(host_codes))
    o.max_level_boxes = int(max_level_boxes)
    o.first_level = int(first_level)
    o.recheck_last = int(bool(recheck_last))
    o.small_level_madds = int(small_level_madds)
    o.c1 = int(c1)
    o.c1_level = int(c1_level)
    o.mode = int(mode)
    o.fp64_final = int(bool(fp64_final))
    o.fp64_recheck = int(bool(fp64_recheck))
    o.theta = float(theta)
    o.timing = int(bool(timing))
    o.taylor_order = int(taylor_order)
    return o


class System:
    """Polynomials packed and resident on the device (vx_system)."""

    def __init__(self, polys, stream=None, his=None, rel=None):
        """his (optional): per polynomial the upper ends of interval coefficients (None for
        point coefficients); rel (optional): per polynomial EQ, LE, GE, LT or GT."""
        arr, keep = _polys(polys)
        h = ctypes.c_void_p()
        if his is None and rel is None:
            _check(lib().vx_system_create(arr, len(polys), _stream(stream), ctypes.byref(h)))
        else:
            hp = (ctypes.c_void_p * len(polys))()
            for i in range(len(polys)):
                if his is not None and his[i] is not None:
                    a = np.ascontiguousarray(np.asarray(his[i], dtype=np.float64))
                    if a.shape[0] != np.asarray(polys[i][1]).shape[0]:
                        raise ValueError("his[%d] must match the coefficients" % i)
                    keep.append(a)
                    hp[i] = a.ctypes.data
            rl = None if rel is None else np.ascontiguousarray(np.asarray(rel, dtype=np.int32))
            _check(lib().vx_system_create_ex(arr, hp, None if rl is None else _np_ptr(rl),
                                             len(polys), _stream(stream), ctypes.byref(h)))
        self.handle = h
        self.k = int(np.asarray(polys[0][0]).shape[1])
        self.npoly = len(polys)

    def info(self):
        k = ctypes.c_int32()
        n = ctypes.c_int32()
        M = np.zeros((self.npoly, self.k + 1), dtype=np.int64)
        _check(lib().vx_system_info(self.handle, ctypes.byref(k), ctypes.byref(n), _np_ptr(M)))
        return int(k.value), int(n.value), M

    def device_bytes(self) -> int:
        b = ctypes.c_int64()
        _check(lib().vx_system_device_bytes(self.handle, ctypes.byref(b)))
        return int(b.value)

    def upload_bytes(self) -> int:
        """Bytes copied from the host when the system was made."""
        b = ctypes.c_int64()
        _check(lib().vx_system_upload_bytes(self.handle, ctypes.byref(b)))
        return int(b.value)

    def free(self):
        if self.handle:
            lib().vx_system_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Csf:
    """A CSF of box indices of one grid level, on the device (vx_csf)."""

    def __init__(self, handle, owner=None):
        self.handle = handle
        self._owner = owner  # a Result whose tree this borrows

    def nodes(self):
        k = ctypes.c_int32()
        lv = ctypes.c_int32()
        N = np.zeros(KMAX, dtype=np.int64)
        _check(lib().vx_csf_nodes(self.handle, ctypes.byref(k), ctypes.byref(lv), _np_ptr(N)))
        return int(k.value), int(lv.value), N[: k.value].copy()

    def export(self, depth, stream=None):
        import torch

        k, _, N = self.nodes()
        n = int(N[depth - 1])
        lab = torch.empty(max(n, 1), dtype=torch.int32, device="cuda")
        ptr = torch.empty(n + 1, dtype=torch.int32, device="cuda") if depth < k else None
        _check(lib().vx_csf_export(self.handle, depth, _ptr(lab), _ptr(ptr), _stream(stream)))
        return lab[:n], ptr

    def tuples(self, stream=None):
        import torch

        k, _, N = self.nodes()
        n = int(N[k - 1])
        t = torch.empty((max(n, 1), k), dtype=torch.int32, device="cuda")
        _check(lib().vx_csf_tuples(self.handle, _ptr(t), _stream(stream)))
        return t[:n]

    def free(self):
        if self.handle and self._owner is None:
            lib().vx_csf_free(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def csf_build(k, level, tuples, stream=None) -> Csf:
    """CSF of lex-sorted unique int32 box indices ``tuples`` (CUDA tensor [n, k])."""
    n = int(tuples.shape[0])
    h = ctypes.c_void_p()
    _check(lib().vx_csf_build(int(k), int(level), _ptr(tuples) if n else None, n,
                              _stream(stream), ctypes.byref(h)))
    return Csf(h)


def csf_full_grid(k, level, stream=None) -> Csf:
    """The CSF of every box of grid level ``level`` (vx_csf_full_grid)."""
    h = ctypes.c_void_p()
    _check(lib().vx_csf_full_grid(int(k), int(level), _stream(stream), ctypes.byref(h)))
    return Csf(h)


def csf_eval_level(system: System, csf: Csf, domain, mode=FP64, values=False, stream=None):
    """Returns ``keep`` (uint8 [N_k]) and, with ``values``, ``lo``/``hi`` float64 [npoly, N_k]."""
    import torch

    _, _, N = csf.nodes()
    n = int(N[-1])
    keep = torch.empty(max(n, 1), dtype=torch.uint8, device="cuda")
    lo = hi = None
    if values:
        lo = torch.empty((system.npoly, max(n, 1)), dtype=torch.float64, device="cuda")
        hi = torch.empty_like(lo)
    dom = _domain(domain)
    _check(lib().vx_csf_eval_level(system.handle, csf.handle, _np_ptr(dom), int(mode), _ptr(lo),
                                   _ptr(hi), _ptr(keep), _stream(stream)))
    if values:
        return keep[:n], lo[:, :n], hi[:, :n]
    return keep[:n]


STATIC_SCRATCH_BYTES = 64 << 20


def csf_eval_level_taylor(system: System, csf: Csf, domain, order, values=False, stream=None):
    """C0 on the Taylor form of the given order (binary64): keep, or (keep, lo, hi)."""
    import torch

    _, _, N = csf.nodes()
    n = int(N[-1])
    keep = torch.empty(max(n, 1), dtype=torch.uint8, device="cuda")
    lo = hi = None
    if values:
        lo = torch.empty((system.npoly, max(n, 1)), dtype=torch.float64, device="cuda")
        hi = torch.empty_like(lo)
    _check(lib().vx_csf_eval_level_taylor(system.handle, csf.handle, _np_ptr(_domain(domain)),
                                          int(order), _ptr(lo), _ptr(hi), _ptr(keep),
                                          _stream(stream)))
    if values:
        return keep[:n], lo[:, :n], hi[:, :n]
    return keep[:n]


def csf_taylor_level(system: System, csf: Csf, domain, order, mode=FP64, c1=False, stream=None):
    """C0 (and with c1, C1) on the Taylor form of the given order in mode FP64 or FP32
    (certified): (keep uint8 [n], inc uint8 [n] or None, boxes re-decided in binary64)."""
    import torch

    _, _, N = csf.nodes()
    n = int(N[-1])
    keep = torch.empty(max(n, 1), dtype=torch.uint8, device="cuda")
    inc = torch.empty(max(n, 1), dtype=torch.uint8, device="cuda") if c1 else None
    nr = ctypes.c_int64()
    _check(lib().vx_csf_taylor_level(system.handle, csf.handle, _np_ptr(_domain(domain)),
                                     int(order), int(mode), _ptr(keep), _ptr(inc),
                                     ctypes.byref(nr), _stream(stream)))
    return keep[:n], (inc[:n] if c1 else None), int(nr.value)


def csf_c1(system: System, csf: Csf, domain, kind, order=0, stream=None):
    """The inclusion criterion C1 (C1_TAYLOR of the given order >= 2, or C1_VERTEX) of the
    system's one polynomial on every leaf box: uint8 [n], 1 where certified."""
    import torch

    _, _, N = csf.nodes()
    n = int(N[-1])
    inc = torch.empty(max(n, 1), dtype=torch.uint8, device="cuda")
    _check(lib().vx_csf_c1(system.handle, csf.handle, _np_ptr(_domain(domain)), int(kind),
                           int(order), _ptr(inc), _stream(stream)))
    return inc[:n]


def csf_eval_grid(system: System, csf: Csf, xlists, mode=FP64, values=False, stream=None):
    """Level evaluation on explicit per-axis intervals ``xlists[i] = (lo, hi)`` (float64 CUDA
    tensors): keep (uint8 [n]) or (keep, lo, hi) with values=True."""
    import torch

    k, _, N = csf.nodes()
    n = int(N[k - 1])
    los = (ctypes.c_void_p * k)(*[int(a.data_ptr()) for a, _ in xlists])
    his = (ctypes.c_void_p * k)(*[int(b.data_ptr()) for _, b in xlists])
    nx = np.array([int(a.numel()) for a, _ in xlists], dtype=np.int64)
    keep = torch.empty(max(n, 1), dtype=torch.uint8, device="cuda")
    lo = hi = None
    if values:
        lo = torch.empty((system.npoly, max(n, 1)), dtype=torch.float64, device="cuda")
        hi = torch.empty_like(lo)
    _check(lib().vx_csf_eval_grid(system.handle, csf.handle, los, his, _np_ptr(nx), int(mode),
                                  _ptr(lo), _ptr(hi), _ptr(keep), _stream(stream)))
    if values:
        return keep[:n], lo[:, :n], hi[:, :n]
    return keep[:n]


def csf_eval_level_static(system: System, csf: Csf, domain, mode=FP64, keep=None, lo=None,
                          hi=None, stream=None):
    """vx_csf_eval_level_static into caller-provided CUDA tensors: ``keep`` uint8 [N_k] and,
    optionally, ``lo``/``hi`` float64 [npoly, N_k].  Returns ``keep``."""
    dom = _domain(domain)
    _check(lib().vx_csf_eval_level_static(system.handle, csf.handle, _np_ptr(dom), int(mode),
                                          _ptr(lo), _ptr(hi), _ptr(keep), _stream(stream)))
    return keep


def csf_subdivide(csf: Csf, keep, stream=None) -> Csf:
    h = ctypes.c_void_p()
    _check(lib().vx_csf_subdivide(csf.handle, _ptr(keep), _stream(stream), ctypes.byref(h)))
    return Csf(h)


def csf_compact(csf: Csf, keep, with_index=False, stream=None):
    import torch

    _, _, N = csf.nodes()
    idx = torch.empty(max(int(N[-1]), 1), dtype=torch.int32, device="cuda") if with_index else None
    h = ctypes.c_void_p()
    _check(lib().vx_csf_compact(csf.handle, _ptr(keep), _ptr(idx), _stream(stream),
                                ctypes.byref(h)))
    out = Csf(h)
    if with_index:
        n = int(out.nodes()[2][-1])
        return out, idx[:n]
    return out


class Result:
    """Outcome of an enclosure (vx_result)."""

    def __init__(self, handle, k, depth):
        self.handle = handle
        self.k = k
        self.depth = depth

    def boxes(self, copy=True) -> np.ndarray:
        """The surviving boxes [n, k] int32.  copy=False returns a view of the result's own
        (pinned) host buffer, valid until free()."""
        n = ctypes.c_int64()
        p = ctypes.c_void_p()
        _check(lib().vx_result_boxes(self.handle, ctypes.byref(n), ctypes.byref(p)))
        m = int(n.value)
        if m == 0:
            return np.zeros((0, self.k), dtype=np.int32)
        buf = (ctypes.c_int32 * (m * self.k)).from_address(p.value)
        a = np.frombuffer(buf, dtype=np.int32).reshape(m, self.k)
        return a.copy() if copy else a

    def box_codes(self, copy=True) -> np.ndarray:
        """The surviving boxes as grid indices (x_1 most significant), ascending: uint32 when
        k * depth <= 32, else uint64.  copy=False returns a view of the result's pinned host
        buffer, valid until free()."""
        n = ctypes.c_int64()
        cb = ctypes.c_int32()
        p = ctypes.c_void_p()
        _check(lib().vx_result_box_codes(self.handle, ctypes.byref(n), ctypes.byref(cb),
                                         ctypes.byref(p)))
        m = int(n.value)
        dt = np.uint32 if cb.value == 4 else np.uint64
        if m == 0:
            return np.zeros(0, dtype=dt)
        buf = (ctypes.c_uint8 * (m * cb.value)).from_address(p.value)
        a = np.frombuffer(buf, dtype=dt)
        return a.copy() if copy else a

    @staticmethod
    def decode_codes(codes, k, depth) -> np.ndarray:
        """Tuples [n, k] int32 from box codes."""
        c = np.asarray(codes).astype(np.uint64)
        out = np.empty((c.shape[0], k), dtype=np.int32)
        mask = np.uint64((1 << depth) - 1)
        for i in range(k):
            out[:, i] = ((c >> np.uint64(depth * (k - 1 - i))) & mask).astype(np.int32)
        return out

    def included(self):
        """With C1: (levels [n] int32, tuples [n, k] int32) of the certified boxes, ordered by
        level, then lexicographic."""
        n = ctypes.c_int64()
        pl = ctypes.c_void_p()
        pt = ctypes.c_void_p()
        _check(lib().vx_result_included(self.handle, ctypes.byref(n), ctypes.byref(pl),
                                        ctypes.byref(pt)))
        m = int(n.value)
        if m == 0:
            return np.zeros(0, dtype=np.int32), np.zeros((0, self.k), dtype=np.int32)
        lev = np.frombuffer((ctypes.c_int32 * m).from_address(pl.value), dtype=np.int32)
        tup = np.frombuffer((ctypes.c_int32 * (m * self.k)).from_address(pt.value),
                            dtype=np.int32).reshape(m, self.k)
        return lev.copy(), tup.copy()

    def csf(self) -> Csf:
        h = ctypes.c_void_p()
        _check(lib().vx_result_csf(self.handle, ctypes.byref(h)))
        return Csf(h, owner=self)

    def stats(self) -> dict:
        L = self.depth + 1
        nl = ctypes.c_int32()
        tested = np.zeros(L, dtype=np.int64)
        kept = np.zeros(L, dtype=np.int64)
        nodes = np.zeros((L, self.k), dtype=np.int64)
        recheck = np.zeros(L, dtype=np.int64)
        madds = np.zeros(L, dtype=np.int64)
        _check(lib().vx_result_stats(self.handle, ctypes.byref(nl), _np_ptr(tested),
                                     _np_ptr(kept), _np_ptr(nodes), _np_ptr(recheck),
                                     _np_ptr(madds)))
        recheck64 = np.zeros(L, dtype=np.int64)
        _check(lib().vx_result_recheck64(self.handle, _np_ptr(recheck64)))
        return {"tested": tested, "kept": kept, "nodes": nodes, "recheck": recheck,
                "recheck64": recheck64, "madds": madds}

    def timing(self) -> dict:
        nk = ctypes.c_int32()
        ms = np.zeros(32, dtype=np.float64)
        la = np.zeros(32, dtype=np.int64)
        wk = np.zeros(32, dtype=np.int64)
        _check(lib().vx_result_timing(self.handle, ctypes.byref(nk), _np_ptr(ms), _np_ptr(la),
                                      _np_ptr(wk)))
        out = {}
        for i in range(nk.value):
            name = lib().vx_kernel_kind_name(i).decode()
            out[name] = {"ms": float(ms[i]), "launches": int(la[i]), "work": int(wk[i])}
        return out

    def elapsed_ms(self) -> float:
        v = ctypes.c_double()
        _check(lib().vx_result_elapsed_ms(self.handle, ctypes.byref(v)))
        return float(v.value)

    def free(self):
        if self.handle:
            lib().vx_result_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def enclose_system(system: System, domain, depth, opts: Opts | None = None, stream=None) -> Result:
    dom = _domain(domain)
    h = ctypes.c_void_p()
    _check(lib().vx_enclose_system(system.handle, _np_ptr(dom), int(depth),
                                   ctypes.byref(opts) if opts is not None else None,
                                   _stream(stream), ctypes.byref(h)))
    return Result(h, system.k, int(depth))


def enclose_from(system: System, start: Csf, domain, depth, opts: Opts | None = None,
                 stream=None) -> Result:
    """Algorithm 3 from the boxes of ``start`` (vx_enclose_from)."""
    dom = _domain(domain)
    h = ctypes.c_void_p()
    _check(lib().vx_enclose_from(system.handle, start.handle, _np_ptr(dom), int(depth),
                                 ctypes.byref(opts) if opts is not None else None,
                                 _stream(stream), ctypes.byref(h)))
    return Result(h, system.k, int(depth))


def enclose_batch(systems, opts: Opts | None = None, nworkers: int = 16):
    """vx_enclose_batch over ``systems`` = [(polys, domain, depth), ...]; returns Results."""
    n = len(systems)
    arrs, keep = [], []
    ptrs = (ctypes.c_void_p * max(n, 1))()
    npoly = np.zeros(max(n, 1), dtype=np.int32)
    depths = np.zeros(max(n, 1), dtype=np.int32)
    doms = []
    for i, (polys, domain, depth) in enumerate(systems):
        arr, kp = _polys(polys)
        arrs.append(arr)
        keep += kp
        ptrs[i] = ctypes.cast(arr, ctypes.c_void_p)
        npoly[i] = len(polys)
        depths[i] = int(depth)
        doms.append(_domain(domain))
    dom = np.ascontiguousarray(np.concatenate(doms)) if doms else np.zeros(1)
    outs = (ctypes.c_void_p * max(n, 1))()
    _check(lib().vx_enclose_batch(ptrs, _np_ptr(npoly), _np_ptr(dom), _np_ptr(depths), n,
                                  ctypes.byref(opts) if opts is not None else None, int(nworkers),
                                  outs))
    return [Result(ctypes.c_void_p(outs[i]), int(np.asarray(systems[i][0][0][0]).shape[1]),
                   int(systems[i][2])) for i in range(n)]


def enclose(polys, domain, depth, opts: Opts | None = None) -> Result:
    """Algorithm 3 from host polynomials to host boxes (vx_enclose)."""
    arr, keep = _polys(polys)
    dom = _domain(domain)
    h = ctypes.c_void_p()
    _check(lib().vx_enclose(arr, len(polys), _np_ptr(dom), int(depth),
                            ctypes.byref(opts) if opts is not None else None, ctypes.byref(h)))
    k = int(np.asarray(polys[0][0]).shape[1])
    return Result(h, k, int(depth))


class DensePlan:
    """A full-grid level of a trivariate system on the tensor cores (vx_dense_plan): the
    superset prefilter (bit mask), the enclosure values, and the exactly decided level."""

    def __init__(self, system: System, level, domain, stream=None):
        self._system = system  # the plan borrows it
        self.level = int(level)
        self.nbox = 1 << (3 * self.level)
        h = ctypes.c_void_p()
        _check(lib().vx_dense_plan_create(system.handle, self.level, _np_ptr(_domain(domain)),
                                          _stream(stream), ctypes.byref(h)))
        self.handle = h

    def device_bytes(self) -> int:
        b = ctypes.c_int64()
        _check(lib().vx_dense_plan_bytes(self.handle, ctypes.byref(b)))
        return int(b.value)

    def prefilter(self, mask=None, stream=None, check=True):
        """int32 CUDA tensor of nbox/32 words; bit b of word w = box 32 w + b is kept."""
        import torch

        if mask is None:
            mask = torch.empty(self.nbox // 32, dtype=torch.int32, device="cuda")
        _check(lib().vx_dense_prefilter(self.handle, _ptr(mask), _stream(stream)))
        if check:
            _check(lib().vx_dense_check_status(_stream(stream)))
        return mask

    def values(self, poly=0, stream=None):
        """(mid, rad) float32 CUDA tensors [nbox] of polynomial ``poly``."""
        import torch

        mid = torch.empty(self.nbox, dtype=torch.float32, device="cuda")
        rad = torch.empty(self.nbox, dtype=torch.float32, device="cuda")
        _check(lib().vx_dense_values(self.handle, int(poly), _ptr(mid), _ptr(rad),
                                     _stream(stream)))
        return mid, rad

    def level_keep(self, opts: Opts | None = None, keep=None, stream=None):
        """(keep uint8 CUDA tensor [nbox], prefilter survivors): the level decided exactly."""
        import torch

        if keep is None:
            keep = torch.empty(self.nbox, dtype=torch.uint8, device="cuda")
        n = ctypes.c_int64()
        _check(lib().vx_dense_level(self.handle, ctypes.byref(opts) if opts is not None else None,
                                    _ptr(keep), ctypes.byref(n), _stream(stream)))
        return keep, int(n.value)

    def free(self):
        if self.handle:
            lib().vx_dense_plan_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def mask_to_bool(mask, nbox):
    """Unpacks a prefilter bit mask (int32 CUDA tensor) into a bool tensor [nbox]."""
    import torch

    w = mask.view(torch.int32).to(torch.int64) & 0xFFFFFFFF
    bits = torch.arange(32, device=mask.device, dtype=torch.int64)
    return ((w[:, None] >> bits[None, :]) & 1).reshape(-1)[:nbox].to(torch.bool)
