"""fe_integrate_tet_noalloc: mixed-precision tetrahedra for callers that cannot
allocate device memory (code inside a device-memory arena that a host application
owns, real-time loops that forbid allocator calls, plugins without a context of
this library). Its scratch is a static device array; its results must be the same
bits as those of fe_integrate_tet on the same inputs, call after call, and within
the mixed tolerance of the FP64 oracle.

Collected last on purpose: if it fails, a run that stops at the first failure
has already run every other test."""
import ctypes

import numpy as np
import pytest
import torch

from helpers import TOL, gpu_outputs_to_numpy, make_inputs, run_oracle, to_device_inputs
import oracle
from paper_1504_01023_gb300 import api, build, meshgen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    build.build()
    c = api.Context(0)
    yield c
    c.close()


def _case(seed, fraction, layout, n_cubes=20, n_elem=None, t_range=meshgen.SLIVER_T_RANGE):
    mesh = meshgen.tet_cube_mesh(n_cubes, seed=seed)                   # 48,000 elements for 20 cubes
    if n_elem is not None:
        mesh = np.ascontiguousarray(mesh[:n_elem])
    meshgen.make_slivers(mesh, fraction, seed=seed + 1, t_range=t_range)   # some take the double pass
    _, c = make_inputs(api.TET, api.GENERIC, api.QUAD_TET4, 0, mesh=mesh, seed=seed)
    X, C, c_used = to_device_inputs(api.TET, mesh, c, api.FP32_MIXED, layout)
    return mesh, X, C, c_used


def _both(ctx, X, C, n, layout, out_layout):
    ref = ctx.integrate(api.TET, X, C, api.GENERIC, api.QUAD_TET4, api.PER_ELEMENT, api.FP32_MIXED, layout,
                        out_layout)
    ctx.sync()
    out = api.alloc_out(api.TET, n, api.FP32_MIXED, out_layout, X.device)
    api.integrate_tet_noalloc(X, C, api.GENERIC, api.QUAD_TET4, api.PER_ELEMENT, layout, out_layout, out)
    return gpu_outputs_to_numpy(api.TET, *ref, out_layout), gpu_outputs_to_numpy(api.TET, *out, out_layout)


@pytest.mark.parametrize("layout,out_layout", [(api.AOS, api.AOS), (api.SOA, api.SOA)])
def test_noalloc_matches_context_path_two_calls(ctx, layout, out_layout):
    for call, (seed, fraction) in enumerate([(101, 0.05), (202, 0.2)]):   # two calls in a row
        mesh, X, C, c_used = _case(seed, fraction, layout)
        n = len(mesh)
        (Ar, br, fr), (An, bn, fn) = _both(ctx, X, C, n, layout, out_layout)
        assert (fn & 1).sum() > 0, "the case must exercise the scratch list"
        # the same kernels, one thread per element: the same bits
        assert np.array_equal(An, Ar) and np.array_equal(bn, br) and np.array_equal(fn, fr), call
        Ao, bo, _ = run_oracle(api.TET, api.GENERIC, api.QUAD_TET4, 0, mesh, c_used)
        assert oracle.rel_frobenius(An, Ao).max() <= TOL[api.FP32_MIXED]
        assert oracle.rel_frobenius(bn, bo).max() <= TOL[api.FP32_MIXED]


def test_noalloc_at_capacity_every_element_flagged(ctx):
    """Exactly the static list's capacity, every element sent to the double pass:
    the list fills to its last slot without overflow (a clean status, FE_OK), the
    results equal the context path's bits and the oracle within the tolerance. A
    mismatch between the capacity the binding states and the library's would make
    this call fail or the next test's call at capacity + 1 succeed."""
    n = api.NOALLOC_MAX_ELEMS
    # every element flattened to a height of 0.2-0.8% (mean ratio 0.007-0.09)
    mesh, X, C, c_used = _case(303, 1.0, api.AOS, n_cubes=45, n_elem=n, t_range=(0.002, 0.008))
    (Ar, br, fr), (An, bn, fn) = _both(ctx, X, C, n, api.AOS, api.AOS)
    assert (fn & 1).all()
    assert np.array_equal(An, Ar) and np.array_equal(bn, br) and np.array_equal(fn, fr)
    Ao, bo, _ = run_oracle(api.TET, api.GENERIC, api.QUAD_TET4, 0, mesh, c_used)
    assert oracle.rel_frobenius(An, Ao).max() <= TOL[api.FP32_MIXED]
    assert oracle.rel_frobenius(bn, bo).max() <= TOL[api.FP32_MIXED]


def _raw_args(n, ordering=0):
    a = api.ElemArgs()
    a.n_elem = n
    a.coords, a.coefs = 4096, 8192
    a.kind, a.quad, a.coef_mode, a.prec = api.GENERIC, api.QUAD_TET4, api.PER_ELEMENT, api.FP32_MIXED
    a.coords_layout = a.coefs_layout = api.AOS
    a.ordering = ordering
    o = api.Out()
    o.A, o.b = 16384, 32768
    o.layout = api.AOS
    return a, o


def test_noalloc_rejects_too_many_elements():
    build.build()
    lib = api.load()
    a, o = _raw_args(api.NOALLOC_MAX_ELEMS + 1)
    st = lib.fe_integrate_tet_noalloc(ctypes.byref(a), ctypes.byref(o), None)
    assert st == -1
    assert b"capacity" in lib.fe_last_error(None)


def test_noalloc_rejects_other_orderings():
    """The SQS and SSQ study kernels are not this entry point's: rejected before any
    GPU work, as the context path would run them."""
    build.build()
    lib = api.load()
    for ordering in (1, 2):
        a, o = _raw_args(1000, ordering)
        st = lib.fe_integrate_tet_noalloc(ctypes.byref(a), ctypes.byref(o), None)
        assert st == -6, ordering
        assert b"ordering" in lib.fe_last_error(None)
