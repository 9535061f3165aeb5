"""Plain FP64 CPU oracle for finite-element numerical integration (arXiv 1504.01023).

TEST INFRASTRUCTURE ONLY. Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package. It shares no code, table
or constant with the CUDA library in ``paper_1504_01023_gb300``; the two are
compared on the same seeded inputs.

``oracle.c`` restates Algorithm 1 (Sec. 2.3) literally in C, compiled with
``-O2 -ffp-contract=off``; ``exact.py`` gives exact-rational closed forms used to
pin it. Functions here only marshal numpy arrays.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

TET, PRISM = 0, 1
POISSON, GENERIC = 0, 1
Q_TET1, Q_TET4, Q_PRISM6, Q_TET_COLLAPSED, Q_PRISM_TENSOR = 0, 1, 2, 3, 4
NS = {TET: 4, PRISM: 6}


def compile_source(src: str, out: str) -> str:
    """Compile an oracle source file into a shared library (gcc, OpenMP, no contraction)."""
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-shared", "-fPIC", "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so next to it."""
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    return compile_source(_SRC, _LIB_PATH)


def load_library(path: str):
    """ctypes handle of an oracle library with its signatures declared."""
    lib = ctypes.CDLL(path)
    i32, i64, p = ctypes.c_int, ctypes.c_int64, ctypes.c_void_p
    lib.oracle_quad_size.argtypes = [i32, i32]
    lib.oracle_quad_size.restype = i32
    lib.oracle_quad_rule.argtypes = [i32, i32, p, p]
    lib.oracle_quad_rule.restype = i32
    lib.oracle_integrate.argtypes = [i32, i32, i32, i32, i32, i64, p, p, p, p, p, i32]
    lib.oracle_integrate.restype = i32
    lib.oracle_quality.argtypes = [i32, i64, p, p, i32]
    lib.oracle_coefs_from_u.argtypes = [i32, i32, i32, i64, p, p, p]
    lib.oracle_coefs_from_u.restype = i32
    lib.oracle_quality.restype = i32
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = load_library(build())
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def quad_rule(rule: int, order: int = 0):
    """Points [n,3] and weights [n] of a rule (Eq. quadrature)."""
    lib = _load()
    n = lib.oracle_quad_size(rule, order)
    if n <= 0:
        raise ValueError(f"bad rule {rule} order {order}")
    pts = np.zeros((n, 3))
    wts = np.zeros(n)
    lib.oracle_quad_rule(rule, order, _ptr(pts), _ptr(wts))
    return pts, wts


def integrate(elem_type: int, kind: int, rule: int, coords, coefs, coef_per_q: bool = False,
              order: int = 0, n_threads: int = 1, lib=None):
    """Element matrices of Algorithm 1 in FP64.

    coords: [E, NS, 3]; coefs: Poisson [E] or [E, NQ], generic [E, 20] or [E, NQ, 20].
    Returns (A [E,NS,NS], b [E,NS], flags [E] uint8: bit1 det<0, bit2 degenerate).
    ``lib`` selects another compiled oracle (planted-mistake tests).
    """
    lib = lib or _load()
    coords = np.ascontiguousarray(coords, dtype=np.float64)
    coefs = np.ascontiguousarray(coefs, dtype=np.float64)
    n = coords.shape[0]
    ns = NS[elem_type]
    assert coords.shape == (n, ns, 3), coords.shape
    nq = lib.oracle_quad_size(rule, order)
    per = (1 if kind == POISSON else 20) * (nq if coef_per_q else 1)
    assert coefs.size == n * per, (coefs.shape, n, per)
    A = np.zeros((n, ns, ns))
    b = np.zeros((n, ns))
    flags = np.zeros(n, dtype=np.uint8)
    rc = lib.oracle_integrate(elem_type, kind, rule, order, int(coef_per_q), n, _ptr(coords), _ptr(coefs),
                              _ptr(A), _ptr(b), _ptr(flags), int(n_threads))
    if rc != 0:
        raise ValueError("oracle_integrate rejected its arguments")
    return A, b, flags


def coefs_from_u(elem_type: int, kind: int, rule: int, u, P, lib=None):
    """Per-point coefficients of the function c_j(u_Q) = P[0][j] + P[1][j] u_Q +
    P[2][j] u_Q^2, u_Q interpolated from the nodal values u [E, NS] at the rule's
    points. Returns generic [E, NQ, 20] or Poisson [E, NQ] (slot 16: d^0)."""
    lib = lib or _load()
    u = np.ascontiguousarray(u, dtype=np.float64)
    P = np.ascontiguousarray(P, dtype=np.float64).reshape(3, 20)
    n = u.shape[0]
    assert u.shape == (n, NS[elem_type])
    nq = lib.oracle_quad_size(rule, 0)
    out = np.zeros((n, nq, 20) if kind == GENERIC else (n, nq))
    if lib.oracle_coefs_from_u(elem_type, kind, rule, n, _ptr(u), _ptr(P), _ptr(out)) != 0:
        raise ValueError("oracle_coefs_from_u rejected its arguments")
    return out


def quality(elem_type: int, coords, n_threads: int = 1, lib=None):
    """Single-precision mean-ratio quality per element (min over PRISM6 points for
    prisms). ``lib`` selects another compiled oracle (planted-mistake tests)."""
    lib = lib or _load()
    coords = np.ascontiguousarray(coords, dtype=np.float64)
    n = coords.shape[0]
    q = np.zeros(n, dtype=np.float32)
    if lib.oracle_quality(elem_type, n, _ptr(coords), _ptr(q), int(n_threads)) != 0:
        raise ValueError("oracle_quality rejected its arguments")
    return q


def rel_frobenius(x, ref):
    """Per-element relative Frobenius error ||x-ref||_F / max(||ref||_F, 1e-300)."""
    x = np.asarray(x, dtype=np.float64).reshape(len(x), -1)
    ref = np.asarray(ref, dtype=np.float64).reshape(len(ref), -1)
    num = np.sqrt(np.sum((x - ref) ** 2, axis=1))
    den = np.maximum(np.sqrt(np.sum(ref ** 2, axis=1)), 1e-300)
    return num / den
