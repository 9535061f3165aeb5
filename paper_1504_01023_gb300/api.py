"""Thin Python binding of the C ABI in include/fe.h (argument marshalling only).

Every step of the integration runs in ``libfe.so``; this module only converts
torch tensors (device memory and streams come from PyTorch) into pointers,
strides and enums. It raises if the library has not been built: there is no
Python or CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np
import torch

from . import build as _build

# enums (values as in include/fe.h)
FE_OK, FE_NOT_READY = 0, 1
TET, PRISM = 0, 1
POISSON, GENERIC = 0, 1
FP64, FP32_MIXED, FP64_DW = 0, 1, 2
QUAD_TET1, QUAD_TET4, QUAD_PRISM6 = 0, 1, 2
PER_ELEMENT, PER_QPOINT, COEF_FN_U = 0, 1, 2
SOA, AOS, INDEXED = 0, 1, 2
MEM_DEVICE, MEM_HOST = 0, 1
NS = {TET: 4, PRISM: 6}
NQ = {QUAD_TET1: 1, QUAD_TET4: 4, QUAD_PRISM6: 6}

_STATUS = {0: "FE_OK", 1: "FE_NOT_READY", -1: "FE_ERR_INVALID_ARG", -2: "FE_ERR_OOM", -3: "FE_ERR_BUDGET",
           -4: "FE_ERR_CUDA", -5: "FE_ERR_TIMEOUT", -6: "FE_ERR_UNSUPPORTED", -7: "FE_ERR_PARTIAL"}


class FeError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class CtxConfig(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("hbm_budget_bytes", ctypes.c_uint64), ("serve_slots", ctypes.c_int),
                ("autotune", ctypes.c_int), ("tuning_cache_path", ctypes.c_char_p)]


class ElemArgs(ctypes.Structure):
    _fields_ = [("n_elem", ctypes.c_int64), ("coords", ctypes.c_void_p), ("coords_layout", ctypes.c_int),
                ("coords_stride", ctypes.c_int64), ("kind", ctypes.c_int), ("quad", ctypes.c_int),
                ("coef_mode", ctypes.c_int), ("coefs", ctypes.c_void_p), ("coefs_layout", ctypes.c_int),
                ("coefs_stride", ctypes.c_int64), ("prec", ctypes.c_int), ("memory", ctypes.c_int),
                ("conn", ctypes.c_void_p), ("n_nodes", ctypes.c_int64), ("ordering", ctypes.c_int),
                ("coef_fn", ctypes.c_void_p)]


class CoefFunction(ctypes.Structure):
    """c_j(u_Q) = p[0][j] + p[1][j] u_Q + p[2][j] u_Q^2 (FE_COEF_FUNCTION_U)."""
    _fields_ = [("p", (ctypes.c_double * 20) * 3)]


class Out(ctypes.Structure):
    _fields_ = [("A", ctypes.c_void_p), ("b", ctypes.c_void_p), ("layout", ctypes.c_int), ("stride", ctypes.c_int64),
                ("flags", ctypes.c_void_p), ("memory", ctypes.c_int), ("packed", ctypes.c_int)]


class BatchItem(ctypes.Structure):
    _fields_ = [("type", ctypes.c_int), ("args", ElemArgs), ("out", Out)]


class LaunchShape(ctypes.Structure):
    _fields_ = [("elems_per_block", ctypes.c_int), ("threads_per_elem", ctypes.c_int), ("persistent", ctypes.c_int)]


class Request(ctypes.Structure):
    _fields_ = [("mesh_id", ctypes.c_int64), ("kind", ctypes.c_int), ("quad", ctypes.c_int), ("coef_mode", ctypes.c_int),
                ("coefs", ctypes.c_void_p), ("prec", ctypes.c_int)]


class Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("type", ctypes.c_int), ("n_elem", ctypes.c_int64), ("A", ctypes.c_void_p),
                ("b", ctypes.c_void_p), ("flags", ctypes.c_void_p), ("t_submit_us", ctypes.c_double),
                ("t_launch_us", ctypes.c_double), ("t_done_us", ctypes.c_double)]


# (name, restype, argtypes) of every exported entry point
_P = ctypes.c_void_p
_SIGS = [
    ("fe_ctx_create", ctypes.c_int, [ctypes.POINTER(CtxConfig), ctypes.POINTER(_P)]),
    ("fe_ctx_destroy", ctypes.c_int, [_P]),
    ("fe_ctx_sync", ctypes.c_int, [_P]),
    ("fe_last_error", ctypes.c_char_p, [_P]),
    ("fe_integrate_tet", ctypes.c_int, [_P, ctypes.POINTER(ElemArgs), ctypes.POINTER(Out), _P]),
    ("fe_integrate_prism", ctypes.c_int, [_P, ctypes.POINTER(ElemArgs), ctypes.POINTER(Out), _P]),
    ("fe_check_args", ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ElemArgs), ctypes.POINTER(Out)]),
    ("fe_bytes_per_element", ctypes.c_int64, [ctypes.c_int] * 5),
    ("fe_mesh_register", ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int64, _P, ctypes.c_int, ctypes.c_int,
                                        ctypes.POINTER(ctypes.c_int64)]),
    ("fe_mesh_release", ctypes.c_int, [_P, ctypes.c_int64]),
    ("fe_batch_submit", ctypes.c_int, [_P, ctypes.POINTER(BatchItem), ctypes.c_int, _P]),
    ("fe_serve_submit", ctypes.c_int, [_P, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_uint64)]),
    ("fe_serve_poll", ctypes.c_int, [_P, ctypes.c_uint64, ctypes.POINTER(Result)]),
    ("fe_serve_release", ctypes.c_int, [_P, ctypes.c_uint64]),
    ("fe_serve_cancel", ctypes.c_int, [_P, ctypes.c_uint64]),
    ("fe_get_launch_shape", ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(ElemArgs), ctypes.POINTER(Out),
                                           ctypes.POINTER(LaunchShape)]),
    ("fe_set_launch_shape", ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(ElemArgs), ctypes.POINTER(Out),
                                           ctypes.POINTER(LaunchShape)]),
    ("fe_batch_set_shape", ctypes.c_int, [_P, ctypes.POINTER(LaunchShape)]),
    ("fe_rule_table", ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                     ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
    ("fe_serve_submit_n", ctypes.c_int, [_P, ctypes.POINTER(Request), ctypes.c_int, ctypes.POINTER(ctypes.c_uint64)]),
    ("fe_serve_release_n", ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_uint64), ctypes.c_int]),
    ("fe_apply_tet", ctypes.c_int, [_P, ctypes.POINTER(ElemArgs), _P, _P, _P, _P, _P]),
    ("fe_apply_prism", ctypes.c_int, [_P, ctypes.POINTER(ElemArgs), _P, _P, _P, _P, _P]),
    ("fe_serve_wait_any", ctypes.c_int, [_P, ctypes.c_int64, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(Result),
                                         ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    ("fe_launch_count", ctypes.c_uint64, []),
    ("fe_ctx_set_profiling", ctypes.c_int, [_P, ctypes.c_int]),
    ("fe_ctx_kernel_time", ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64), ctypes.c_int]),
    ("fe_tune", ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(ElemArgs), ctypes.POINTER(Out), _P]),
    ("fe_get_shape", ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(ElemArgs), ctypes.POINTER(Out),
                                    ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    ("fe_integrate_tet_noalloc", ctypes.c_int, [ctypes.POINTER(ElemArgs), ctypes.POINTER(Out), _P]),
    ("fe_selftest_bounded_wait", ctypes.c_int, [_P, ctypes.c_uint, _P]),
    ("fe_ctx_inject_fault", ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int64, ctypes.c_int64]),
    ("fe_selftest_f64_int", ctypes.c_int, [ctypes.c_int, _P, _P, ctypes.c_int64, _P, _P, _P]),
    ("fe_set_shape", ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(ElemArgs), ctypes.POINTER(Out), ctypes.c_int,
                                    ctypes.c_int]),
]

_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB


def load():
    """Load libfe.so (it must have been built by ``build.build()``)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(_build.LIB):
                raise RuntimeError(f"{_build.LIB} is missing: build it with __graft_entry__.build()")
            lib = ctypes.CDLL(_build.LIB)
            for name, res, args in _SIGS:
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _check(st: int, ctx_handle=None):
    if st != FE_OK:
        msg = load().fe_last_error(ctx_handle)
        raise FeError(st, msg.decode() if msg else "")
    return st


def bytes_per_element(elem_type, kind, quad, coef_mode, prec) -> int:
    return int(load().fe_bytes_per_element(elem_type, kind, quad, coef_mode, prec))


def launch_count() -> int:
    return int(load().fe_launch_count())


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _mem(t):
    return MEM_DEVICE if t.is_cuda else MEM_HOST


def n_coefs(kind, quad, coef_mode):
    return (1 if kind == POISSON else 20) * (NQ[quad] if coef_mode == PER_QPOINT else 1)


FAULT_NONE, FAULT_ALLOC, FAULT_SKIP_TILES = 0, 1, 2   # fe_ctx_inject_fault kinds
QSS, SQS, SSQ = 0, 1, 2   # loop orderings (Sec. 3.3)


def make_args(elem_type, coords, coefs, kind, quad, coef_mode, prec, layout, conn=None, ordering=QSS, coef_fn=None):
    """ElemArgs for torch tensors. SOA: coords (3*NS, E) and coefs (NC, E), unit
    stride along elements, any plane stride. AOS: coords (E, NS, 3), coefs (E, ...).
    INDEXED: coords = nodes (N, 3), conn (E, NS) int32, coefs (E, ...)."""
    a = ElemArgs()
    a.ordering = ordering
    if coef_mode == COEF_FN_U:
        assert coef_fn is not None, "COEF_FN_U needs the parameter array coef_fn [3, 20]"
        P = np.ascontiguousarray(np.asarray(coef_fn, dtype=np.float64).reshape(3, 20))
        fn = CoefFunction()
        for i in range(3):
            for j in range(20):
                fn.p[i][j] = float(P[i, j])
        a._fn = fn                       # kept alive with the arguments
        a.coef_fn = ctypes.addressof(fn)
    if layout == INDEXED:
        assert conn is not None and conn.dtype == torch.int32 and conn.is_contiguous()
        assert conn.dim() == 2 and conn.shape[1] == NS[elem_type]
        assert coords.dim() == 2 and coords.shape[1] == 3 and coords.is_contiguous() and coefs.is_contiguous()
        assert coords.dtype == torch.float64
        want = torch.float32 if prec == FP32_MIXED else torch.float64
        assert coefs.dtype == want, f"coefficients must be {want}"
        a.n_elem = conn.shape[0]
        a.coords = coords.data_ptr()
        a.coords_layout = INDEXED
        a.kind, a.quad, a.coef_mode, a.prec = kind, quad, coef_mode, prec
        a.coefs = coefs.data_ptr()
        a.coefs_layout = AOS
        a.memory = _mem(coords)
        a.conn = conn.data_ptr()
        a.n_nodes = coords.shape[0]
        return a
    if layout == SOA:
        assert coords.dim() == 2 and coords.shape[0] == 3 * NS[elem_type]
        n = coords.shape[1]
        cf = coefs.reshape(-1, n) if coefs.dim() == 1 else coefs
        # size-1 dimensions may report any stride: only a real element axis must be unit-stride
        assert n <= 1 or (coords.stride(1) == 1 and cf.stride(-1) == 1)
        a.coords_stride = coords.stride(0) if n > 1 else 0
        # a single plane has no plane stride (size-1 dimensions may report any stride)
        a.coefs_stride = cf.stride(0) if cf.shape[0] > 1 else 0
    else:
        assert coords.is_contiguous() and coefs.is_contiguous()
        n = coords.shape[0]
        a.coords_stride = 0
        a.coefs_stride = 0
    assert coords.dtype == torch.float64
    want = torch.float32 if prec == FP32_MIXED else torch.float64
    assert coefs.dtype == want, f"coefficients must be {want}"
    a.n_elem = n
    a.coords = coords.data_ptr()
    a.coords_layout = layout
    a.kind, a.quad, a.coef_mode, a.prec = kind, quad, coef_mode, prec
    a.coefs = coefs.data_ptr()
    a.coefs_layout = layout
    a.memory = _mem(coords)
    return a


def rule_table(quad):
    """The library's quadrature as its kernels use it: (weights [n], reference
    shape-function values [n, NS]) at the rule's points."""
    ns = 4 if quad in (QUAD_TET1, QUAD_TET4) else 6
    n = ctypes.c_int()
    w = (ctypes.c_double * 64)()
    phi = (ctypes.c_double * (64 * ns))()
    _check(load().fe_rule_table(quad, 64, ctypes.byref(n), w, phi), None)
    return np.array(w[:n.value]), np.array(phi[:n.value * ns]).reshape(n.value, ns)


def packed_size(elem_type):
    """Entries of the packed upper triangle of A^e (10 or 21)."""
    ns = NS[elem_type]
    return ns * (ns + 1) // 2


def alloc_out(elem_type, n, prec, out_layout, device, with_flags=True, pin=False, packed=False):
    """A, b, flags. A is (n, NS, NS) element-contiguous or (NS*NS, n) plane-major;
    packed: (n, NP) or (NP, n), NP = NS*(NS+1)/2 upper-triangle entries."""
    ns = NS[elem_type]
    na = packed_size(elem_type) if packed else ns * ns
    dt = torch.float32 if prec == FP32_MIXED else torch.float64
    kw = dict(dtype=dt, device=device)
    if out_layout == SOA:
        # A and b share one plane stride: one (NA + NS, n) buffer
        buf = torch.empty((na + ns, n), **kw, pin_memory=pin) if pin else torch.empty((na + ns, n), **kw)
        A, b = buf[:na], buf[na:]
    else:
        shape = (n, na) if packed else (n, ns, ns)
        A = torch.empty(shape, **kw, pin_memory=pin) if pin else torch.empty(shape, **kw)
        b = torch.empty((n, ns), **kw, pin_memory=pin) if pin else torch.empty((n, ns), **kw)
    flags = None
    if with_flags:
        flags = (torch.empty(n, dtype=torch.uint8, device=device, pin_memory=pin) if pin
                 else torch.empty(n, dtype=torch.uint8, device=device))
    return A, b, flags


def make_out(A, b, flags, out_layout, packed=False):
    o = Out()
    o.packed = 1 if packed else 0
    o.A, o.b = A.data_ptr(), b.data_ptr()
    o.layout = out_layout
    if out_layout == SOA:
        n = A.shape[1]
        assert n <= 1 or (A.stride(0) == b.stride(0) and A.stride(1) == 1 and b.stride(1) == 1)
        o.stride = A.stride(0) if n > 1 else 0
    o.flags = flags.data_ptr() if flags is not None else None
    o.memory = _mem(A)
    return o


# Largest n_elem fe_integrate_tet_noalloc accepts (its static scratch holds one
# list entry per element).
NOALLOC_MAX_ELEMS = (4 << 20) // 8 - 32


def integrate_tet_noalloc(coords, coefs, kind, quad, coef_mode, layout, out_layout, out, stream=None):
    """Mixed-precision tetrahedra through fe_integrate_tet_noalloc: the caller
    provides every buffer (``out`` = (A, b, flags)); the library allocates nothing.
    Returns after the kernels finish."""
    args = make_args(TET, coords, coefs, kind, quad, coef_mode, FP32_MIXED, layout)
    o = make_out(*out, out_layout)
    s = ctypes.c_void_p(stream.cuda_stream if stream is not None else torch.cuda.current_stream().cuda_stream)
    _check(load().fe_integrate_tet_noalloc(ctypes.byref(args), ctypes.byref(o), s))
    return out


class _DeviceArray:
    """__cuda_array_interface__ view of a device pointer owned by the library."""

    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = {"data": (int(ptr), False), "shape": tuple(shape), "typestr": typestr,
                                         "version": 3, "strides": None}


def device_view(ptr, shape, dtype, device=0):
    """Zero-copy torch view of library-owned device memory (e.g. served outputs)."""
    typestr = {torch.float32: "<f4", torch.float64: "<f8", torch.uint8: "|u1"}[dtype]
    return torch.as_tensor(_DeviceArray(ptr, shape, typestr), device=f"cuda:{device}")


def context_settings(autotune=None, tuning_cache=None, environ=None):
    """Autotuning and the tuning-cache path of a new context: the arguments when
    given, else the environment (FE_AUTOTUNE=1, FE_TUNING_CACHE=<path>), else off
    and no cache."""
    env = os.environ if environ is None else environ
    if autotune is None:
        autotune = env.get("FE_AUTOTUNE", "0").strip() not in ("", "0", "false", "False", "no")
    if tuning_cache is None:
        tuning_cache = env.get("FE_TUNING_CACHE") or None
    return bool(autotune), tuning_cache


class Context:
    """One library context on one CUDA device."""

    def __init__(self, device: int = 0, autotune: bool | None = None, tuning_cache: str | None = None,
                 hbm_budget: int = 0, serve_slots: int = 0):
        lib = load()
        autotune, tuning_cache = context_settings(autotune, tuning_cache)
        cfg = CtxConfig(device, hbm_budget, serve_slots, int(autotune),
                        tuning_cache.encode() if tuning_cache else None)
        h = ctypes.c_void_p()
        _check(lib.fe_ctx_create(ctypes.byref(cfg), ctypes.byref(h)))
        self.h = h
        self.device = device
        self._keep = {}

    def close(self):
        if self.h:
            load().fe_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def sync(self):
        _check(load().fe_ctx_sync(self.h), self.h)

    def _stream(self, stream, on_device):
        if stream is not None:
            return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
        if on_device:
            return ctypes.c_void_p(torch.cuda.current_stream(self.device).cuda_stream)
        return ctypes.c_void_p(0)

    def integrate(self, elem_type, coords, coefs, kind, quad, coef_mode=PER_ELEMENT, prec=FP32_MIXED, layout=SOA,
                  out_layout=SOA, out=None, with_flags=True, stream=None, conn=None, packed=False, ordering=QSS,
                  coef_fn=None):
        """Integrate one element set; returns (A, b, flags) tensors (allocated if
        ``out`` is None, on the device of ``coords``; pinned host memory for host inputs).
        With layout=INDEXED, coords is the node array and conn the element -> node table."""
        args = make_args(elem_type, coords, coefs, kind, quad, coef_mode, prec, layout, conn, ordering, coef_fn)
        if out is None:
            on_host = not coords.is_cuda
            out = alloc_out(elem_type, args.n_elem, prec, out_layout, coords.device, with_flags, pin=on_host,
                            packed=packed)
        A, b, flags = out
        o = make_out(A, b, flags, out_layout, packed)
        fn = load().fe_integrate_tet if elem_type == TET else load().fe_integrate_prism
        _check(fn(self.h, ctypes.byref(args), ctypes.byref(o), self._stream(stream, coords.is_cuda)), self.h)
        return A, b, flags

    def apply(self, elem_type, nodes, conn, coefs, kind, quad, x, y, f=None, coef_mode=PER_ELEMENT, prec=FP32_MIXED,
              flags=None, stream=None):
        """Matrix-free y += sum_e P_e^T A^e P_e x (and f += sum_e P_e^T b^e if f is
        given) over the elements of a node table; y and f accumulate."""
        args = make_args(elem_type, nodes, coefs, kind, quad, coef_mode, prec, INDEXED, conn)
        want = torch.float32 if prec == FP32_MIXED else torch.float64
        for v in (x, y) + ((f,) if f is not None else ()):
            assert v.dtype == want and v.is_contiguous() and v.numel() == nodes.shape[0]
        fn = load().fe_apply_tet if elem_type == TET else load().fe_apply_prism
        _check(fn(self.h, ctypes.byref(args), x.data_ptr(), y.data_ptr(), f.data_ptr() if f is not None else None,
                  flags.data_ptr() if flags is not None else None, self._stream(stream, True)), self.h)

    def tune(self, elem_type, coords, coefs, kind, quad, coef_mode=PER_ELEMENT, prec=FP32_MIXED, layout=SOA,
             out_layout=SOA, out=None, stream=None, conn=None, packed=False, ordering=QSS, coef_fn=None):
        args = make_args(elem_type, coords, coefs, kind, quad, coef_mode, prec, layout, conn, ordering, coef_fn)
        if out is None:
            out = alloc_out(elem_type, args.n_elem, prec, out_layout, coords.device, packed=packed)
        o = make_out(*out, out_layout, packed)
        _check(load().fe_tune(self.h, elem_type, ctypes.byref(args), ctypes.byref(o), self._stream(stream, True)), self.h)
        return self.shape(elem_type, coords, coefs, kind, quad, coef_mode, prec, layout, out_layout, out, conn, packed,
                          ordering, coef_fn)

    def set_shape(self, block, persistent, elem_type, coords, coefs, kind, quad, coef_mode=PER_ELEMENT,
                  prec=FP32_MIXED, layout=SOA, out_layout=SOA, out=None, conn=None, packed=False, tpe=1):
        """Pin the launch shape: `block` elements per tile, `tpe` threads per element."""
        args = make_args(elem_type, coords, coefs, kind, quad, coef_mode, prec, layout, conn)
        if out is None:
            out = alloc_out(elem_type, args.n_elem, prec, out_layout, coords.device, packed=packed)
        o = make_out(*out, out_layout, packed)
        sh = LaunchShape(block, tpe, persistent)
        _check(load().fe_set_launch_shape(self.h, elem_type, ctypes.byref(args), ctypes.byref(o), ctypes.byref(sh)),
               self.h)

    def shape(self, elem_type, coords, coefs, kind, quad, coef_mode=PER_ELEMENT, prec=FP32_MIXED, layout=SOA,
              out_layout=SOA, out=None, conn=None, packed=False, ordering=QSS, coef_fn=None):
        args = make_args(elem_type, coords, coefs, kind, quad, coef_mode, prec, layout, conn, ordering, coef_fn)
        if out is None:
            out = alloc_out(elem_type, args.n_elem, prec, out_layout, coords.device, packed=packed)
        o = make_out(*out, out_layout, packed)
        sh = LaunchShape()
        _check(load().fe_get_launch_shape(self.h, elem_type, ctypes.byref(args), ctypes.byref(o), ctypes.byref(sh)),
               self.h)
        return sh.elems_per_block, sh.persistent, sh.threads_per_elem

    def selftest_bounded_wait(self, polls: int = 1 << 16) -> int:
        """Run the failure-detection self-test; returns the status (FE_ERR_TIMEOUT expected)."""
        return int(load().fe_selftest_bounded_wait(self.h, polls, self._stream(None, True)))

    def inject_fault(self, kind: int, count: int = 1, param: int = 1):
        """Host-side fault injection for failure-detection tests (FAULT_ALLOC: the next
        `count` device allocations fail as out of memory; FAULT_SKIP_TILES: the next
        `count` main-kernel launches skip every tile whose index is a multiple of
        `param` and the next sync reports FE_ERR_PARTIAL; FAULT_NONE clears both)."""
        _check(load().fe_ctx_inject_fault(self.h, kind, count, param), self.h)

    def set_profiling(self, on: bool):
        _check(load().fe_ctx_set_profiling(self.h, int(on)), self.h)

    def kernel_time(self, reset: bool = True):
        ms, n = ctypes.c_double(), ctypes.c_int64()
        _check(load().fe_ctx_kernel_time(self.h, ctypes.byref(ms), ctypes.byref(n), int(reset)), self.h)
        return ms.value, n.value

    # -- resident meshes, batching, serving ---------------------------------
    def mesh_register(self, elem_type, coords, layout=AOS) -> int:
        mid = ctypes.c_int64()
        n = coords.shape[0] if layout == AOS else coords.shape[1]
        _check(load().fe_mesh_register(self.h, elem_type, n, _ptr(coords), layout, _mem(coords), ctypes.byref(mid)),
               self.h)
        return mid.value

    def mesh_release(self, mesh_id: int):
        _check(load().fe_mesh_release(self.h, mesh_id), self.h)

    def batch_set_shape(self, block=None, tpe=1, persistent=1):
        """Pin the shape of new batch plans (block elements per tile, tpe threads per
        prism element, persistent grids or one block per tile), or return to
        tuned/default shapes with block=None."""
        if block is None:
            _check(load().fe_batch_set_shape(self.h, None), self.h)
        else:
            sh = LaunchShape(block, tpe, persistent)
            _check(load().fe_batch_set_shape(self.h, ctypes.byref(sh)), self.h)

    def batch_submit(self, items, stream=None):
        """items: list of (elem_type, ElemArgs, Out)."""
        arr = (BatchItem * len(items))()
        for i, (t, a, o) in enumerate(items):
            arr[i].type, arr[i].args, arr[i].out = t, a, o
        _check(load().fe_batch_submit(self.h, arr, len(items), self._stream(stream, True)), self.h)

    def serve_submit(self, mesh_id, kind, quad, coef_mode, coefs, prec=FP32_MIXED) -> int:
        req = Request(mesh_id, kind, quad, coef_mode, coefs.data_ptr(), prec)
        t = ctypes.c_uint64()
        _check(load().fe_serve_submit(self.h, ctypes.byref(req), ctypes.byref(t)), self.h)
        self._keep[t.value] = (coefs, prec)
        return t.value

    def serve_submit_many(self, requests) -> list:
        """Several requests in one call (they can share one launch): a list of
        (mesh_id, kind, quad, coef_mode, coefs[, prec]) tuples. All or nothing."""
        n = len(requests)
        arr = (Request * max(n, 1))()
        for i, rq in enumerate(requests):
            mesh_id, kind, quad, cm, coefs = rq[:5]
            prec = rq[5] if len(rq) > 5 else FP32_MIXED
            arr[i] = Request(mesh_id, kind, quad, cm, coefs.data_ptr(), prec)
        tks = (ctypes.c_uint64 * max(n, 1))()
        _check(load().fe_serve_submit_n(self.h, arr, n, tks), self.h)
        out = list(tks[:n])
        for t, rq in zip(out, requests):
            self._keep[t] = (rq[4], rq[5] if len(rq) > 5 else FP32_MIXED)
        return out

    def serve_release_many(self, tickets):
        """Release several finished requests in one call. All or nothing."""
        n = len(tickets)
        arr = (ctypes.c_uint64 * max(n, 1))(*tickets)
        _check(load().fe_serve_release_n(self.h, arr, n), self.h)
        for t in tickets:
            self._keep.pop(t, None)

    def serve_result_tensors(self, ticket, res):
        """(A [n,NS,NS], b [n,NS], flags [n]) views of a finished request's outputs."""
        prec = self._keep[ticket][1]
        dt = torch.float32 if prec == FP32_MIXED else torch.float64
        ns, n = NS[res.type], res.n_elem
        return (device_view(res.A, (n, ns, ns), dt, self.device), device_view(res.b, (n, ns), dt, self.device),
                device_view(res.flags, (n,), torch.uint8, self.device))

    def serve_poll(self, ticket):
        """None while running, else the Result structure."""
        res = Result()
        st = load().fe_serve_poll(self.h, ticket, ctypes.byref(res))
        if st == FE_NOT_READY:
            return None
        _check(st, self.h)
        return res

    def serve_wait_any(self, timeout_us=1000, max_results=64):
        """Finished requests not yet returned by this call, in completion order:
        a list of (ticket, Result), empty on timeout."""
        if getattr(self, "_wait_bufs", None) is None or len(self._wait_bufs[0]) < max_results:
            self._wait_bufs = ((ctypes.c_uint64 * max_results)(), (Result * max_results)())
        tks, res = self._wait_bufs
        n = ctypes.c_int()
        _check(load().fe_serve_wait_any(self.h, int(timeout_us), tks, res, max_results, ctypes.byref(n)), self.h)
        out = []
        for i in range(n.value):
            r = Result()
            ctypes.pointer(r)[0] = res[i]
            out.append((tks[i], r))
        return out

    def serve_cancel(self, ticket):
        """Withdraw a request that has not been launched yet."""
        _check(load().fe_serve_cancel(self.h, ticket), self.h)
        self._keep.pop(ticket, None)

    def serve_release(self, ticket):
        self._keep.pop(ticket, None)
        _check(load().fe_serve_release(self.h, ticket), self.h)
