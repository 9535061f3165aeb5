"""fe_integrate_tet_noalloc: mixed-precision tetrahedra for callers that cannot
allocate device memory (arena-owned memory, allocator-free real-time loops,
plugins without a context). Its scratch is a static device array; the results
must equal those of fe_integrate_tet on the same inputs, call after call.

Collected last on purpose: if it fails, a run that stops at the first failure
has already run every other test."""
import ctypes

import numpy as np
import pytest
import torch

from helpers import TOL, gpu_outputs_to_numpy, make_inputs, to_device_inputs
import oracle
from paper_1504_01023_gb300 import api, build, meshgen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    build.build()
    c = api.Context(0)
    yield c
    c.close()


def _case(seed, fraction, layout, out_layout):
    mesh = meshgen.tet_cube_mesh(20, seed=seed)                        # 48,000 elements
    meshgen.make_slivers(mesh, fraction, seed=seed + 1)                # some take the double pass
    _, c = make_inputs(api.TET, api.GENERIC, api.QUAD_TET4, 0, mesh=mesh, seed=seed)
    X, C, _ = to_device_inputs(api.TET, mesh, c, api.FP32_MIXED, layout)
    return X, C


@pytest.mark.parametrize("layout,out_layout", [(api.AOS, api.AOS), (api.SOA, api.SOA)])
def test_noalloc_matches_context_path_two_calls(ctx, layout, out_layout):
    for call, (seed, fraction) in enumerate([(101, 0.05), (202, 0.2)]):   # two calls in a row
        X, C = _case(seed, fraction, layout, out_layout)
        n = X.shape[0] if layout == api.AOS else X.shape[1]
        ref = ctx.integrate(api.TET, X, C, api.GENERIC, api.QUAD_TET4, api.PER_ELEMENT, api.FP32_MIXED, layout,
                            out_layout)
        ctx.sync()
        out = api.alloc_out(api.TET, n, api.FP32_MIXED, out_layout, X.device)
        api.integrate_tet_noalloc(X, C, api.GENERIC, api.QUAD_TET4, api.PER_ELEMENT, layout, out_layout, out)
        Ar, br, fr = gpu_outputs_to_numpy(api.TET, *ref, out_layout)
        An, bn, fn = gpu_outputs_to_numpy(api.TET, *out, out_layout)
        assert (fn & 1).sum() > 0, "the case must exercise the scratch list"
        assert oracle.rel_frobenius(An, Ar).max() <= TOL[api.FP32_MIXED]
        assert oracle.rel_frobenius(bn, br).max() <= TOL[api.FP32_MIXED]
        assert np.array_equal(fn, fr)


def test_noalloc_rejects_too_many_elements():
    build.build()
    lib = api.load()
    n = api.NOALLOC_MAX_ELEMS + 1
    a = api.ElemArgs()
    a.n_elem = n
    a.coords, a.coefs = 4096, 8192
    a.kind, a.quad, a.coef_mode, a.prec = api.GENERIC, api.QUAD_TET4, api.PER_ELEMENT, api.FP32_MIXED
    o = api.Out()
    o.A, o.b = 16384, 32768
    st = lib.fe_integrate_tet_noalloc(ctypes.byref(a), ctypes.byref(o), None)
    assert st == -1
    assert b"capacity" in lib.fe_last_error(None)
