"""The Python binding's argument marshalling, on host tensors (no GPU): the
ElemArgs / Out structures it builds for every layout are accepted by the
library's own host-side validation (fe_check_args), carry the right strides and
memory kind, and the output allocations have the documented shapes."""
import ctypes
import itertools

import numpy as np
import pytest
import torch

from paper_1504_01023_gb300 import api, build, meshgen


@pytest.fixture(scope="module")
def lib():
    build.build()
    return api.load()


def _check(lib, et, a, o):
    return lib.fe_check_args(et, ctypes.byref(a), ctypes.byref(o))


CASES = list(itertools.product([api.TET, api.PRISM], [api.FP64, api.FP32_MIXED, api.FP64_DW], [api.SOA, api.AOS],
                               [api.SOA, api.AOS]))


@pytest.mark.parametrize("et,prec,il,ol", CASES, ids=["t%d-p%d-i%d-o%d" % c for c in CASES])
def test_structures_pass_host_validation(lib, et, prec, il, ol):
    n = 37
    ns = api.NS[et]
    mesh = (meshgen.tet_cube_mesh(3) if et == api.TET else meshgen.prism_slab_mesh(5))[:n]
    quad = api.QUAD_TET4 if et == api.TET else api.QUAD_PRISM6
    dt = torch.float32 if prec == api.FP32_MIXED else torch.float64
    if il == api.SOA:
        X = torch.from_numpy(meshgen.soa(mesh))
        C = torch.zeros((20, n), dtype=dt)
    else:
        X = torch.from_numpy(np.ascontiguousarray(mesh))
        C = torch.zeros((n, 20), dtype=dt)
    a = api.make_args(et, X, C, api.GENERIC, quad, api.PER_ELEMENT, prec, il)
    A, b, f = api.alloc_out(et, n, prec, ol, "cpu")
    o = api.make_out(A, b, f, ol)
    assert _check(lib, et, a, o) == 0, api.load().fe_last_error(None)
    assert a.n_elem == n and a.memory == api.MEM_HOST and o.memory == api.MEM_HOST
    if il == api.SOA:
        assert a.coords_stride == n and a.coefs_stride == n
    if ol == api.SOA:
        assert A.shape == (ns * ns, n) and b.shape == (ns, n) and o.stride == n
        assert A.stride(0) == b.stride(0)           # one plane stride for both outputs
    else:
        assert A.shape == (n, ns, ns) and b.shape == (n, ns)
    assert A.dtype == dt and f.shape == (n,) and f.dtype == torch.uint8


def test_node_table_and_packed_structures(lib):
    nodes, conn = meshgen.tet_cube_indexed(3)
    n = len(conn)
    X, K = torch.from_numpy(nodes), torch.from_numpy(conn)
    C = torch.zeros((n, 20), dtype=torch.float32)
    a = api.make_args(api.TET, X, C, api.GENERIC, api.QUAD_TET4, api.PER_ELEMENT, api.FP32_MIXED, api.INDEXED, conn=K)
    assert a.coords_layout == api.INDEXED and a.n_nodes == len(nodes) and a.conn == K.data_ptr()
    full = api.make_out(*api.alloc_out(api.TET, n, api.FP32_MIXED, api.AOS, "cpu"), api.AOS)
    assert _check(lib, api.TET, a, full) == -6                   # node tables need device memory
    a.memory = full.memory = api.MEM_DEVICE                      # (validation does not dereference pointers)
    assert _check(lib, api.TET, a, full) == 0, api.load().fe_last_error(None)
    # packed (upper-triangle) output: the Laplace kind with element-contiguous coordinates
    A, b, f = api.alloc_out(api.TET, n, api.FP32_MIXED, api.AOS, "cpu", packed=True)
    assert A.shape == (n, api.packed_size(api.TET)) == (n, 10)
    o = api.make_out(A, b, f, api.AOS, packed=True)
    assert o.packed == 1
    o.memory = api.MEM_DEVICE
    assert _check(lib, api.TET, a, o) == -6                      # not with a node table
    o.memory = api.MEM_HOST
    mesh = meshgen.tet_cube_mesh(3)[:n]
    Xe = torch.from_numpy(np.ascontiguousarray(mesh))
    lap = api.make_args(api.TET, Xe, torch.zeros(n, dtype=torch.float32), api.POISSON, api.QUAD_TET1,
                        api.PER_ELEMENT, api.FP32_MIXED, api.AOS)
    assert _check(lib, api.TET, lap, o) == 0, api.load().fe_last_error(None)
    gen = api.make_args(api.TET, Xe, torch.zeros((n, 20), dtype=torch.float32), api.GENERIC, api.QUAD_TET4,
                        api.PER_ELEMENT, api.FP32_MIXED, api.AOS)
    assert _check(lib, api.TET, gen, o) != 0                     # not for the generic kind


def test_wrong_dtypes_are_caught_before_the_library(lib):
    mesh = meshgen.tet_cube_mesh(2)
    X = torch.from_numpy(np.ascontiguousarray(mesh))
    with pytest.raises(AssertionError):
        api.make_args(api.TET, X, torch.zeros((len(mesh), 20), dtype=torch.float64), api.GENERIC,
                      api.QUAD_TET4, api.PER_ELEMENT, api.FP32_MIXED, api.AOS)
    with pytest.raises(AssertionError):
        api.make_args(api.TET, X.float(), torch.zeros((len(mesh), 20), dtype=torch.float32), api.GENERIC,
                      api.QUAD_TET4, api.PER_ELEMENT, api.FP32_MIXED, api.AOS)


def test_context_settings_from_arguments_and_environment():
    assert api.context_settings(environ={}) == (False, None)
    assert api.context_settings(environ={"FE_AUTOTUNE": "1", "FE_TUNING_CACHE": "/tmp/t.txt"}) == (True, "/tmp/t.txt")
    assert api.context_settings(environ={"FE_AUTOTUNE": "0"}) == (False, None)
    # explicit arguments win over the environment
    assert api.context_settings(False, "a.txt", environ={"FE_AUTOTUNE": "1", "FE_TUNING_CACHE": "b"}) == (False, "a.txt")
