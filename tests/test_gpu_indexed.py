"""Connectivity-indexed geometry (FE_LAYOUT_INDEXED): a node array plus an
element -> node table. Parity against the FP64 oracle on the gathered
coordinates (nodes[conn]), bit-identity with the element-contiguous path on the
same coordinates, and elements whose node index is out of range."""
import itertools

import numpy as np
import pytest
import torch

from helpers import TOL, gpu_outputs_to_numpy, make_inputs, max_errors, run_oracle
from paper_1504_01023_gb300 import api, meshgen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1504_01023_gb300 import build
    build.build()
    c = api.Context(0)
    yield c
    c.close()


def _indexed(et, n):
    if et == api.TET:
        nodes, conn = meshgen.tet_cube_indexed(8, seed=meshgen.SEED_BASE + 61)
    else:
        nodes, conn = meshgen.prism_slab_indexed(40, seed=meshgen.SEED_BASE + 62)
    return nodes, np.ascontiguousarray(conn[:n])


def _run(ctx, et, kind, quad, cpq, prec, olay, nodes, conn, c, layout=api.INDEXED):
    n = len(conn)
    cdt = np.float32 if prec == api.FP32_MIXED else np.float64
    C = torch.from_numpy(np.ascontiguousarray(c.astype(cdt).reshape(n, -1))).cuda()
    cm = api.PER_QPOINT if cpq else api.PER_ELEMENT
    if layout == api.INDEXED:
        X = torch.from_numpy(nodes).cuda()
        K = torch.from_numpy(conn).cuda()
        A, b, f = ctx.integrate(et, X, C, kind, quad, cm, prec, api.INDEXED, olay, conn=K)
    else:
        X = torch.from_numpy(np.ascontiguousarray(nodes[conn])).cuda()
        A, b, f = ctx.integrate(et, X, C, kind, quad, cm, prec, api.AOS, olay)
    ctx.sync()
    An, bn, fn = gpu_outputs_to_numpy(et, A, b, f, olay)
    return An, bn, fn, c.astype(cdt).astype(np.float64)


PRECS = [api.FP64, api.FP32_MIXED, api.FP64_DW]
CASES = ([(api.TET, k, q, c, p, o) for k, q, c, p, o in itertools.product(
            [api.POISSON, api.GENERIC], [api.QUAD_TET1, api.QUAD_TET4], [0, 1], PRECS, [api.SOA, api.AOS])] +
         [(api.PRISM, k, api.QUAD_PRISM6, c, p, o) for k, c, p, o in itertools.product(
            [api.POISSON, api.GENERIC], [0, 1], PRECS, [api.SOA, api.AOS])])


@pytest.mark.parametrize("et,kind,quad,cpq,prec,olay", CASES, ids=["t%d-k%d-q%d-c%d-p%d-o%d" % c for c in CASES])
def test_indexed_parity(ctx, et, kind, quad, cpq, prec, olay):
    n = 2999 if et == api.TET else 1999
    nodes, conn = _indexed(et, n)
    _, c = make_inputs(et, kind, quad, cpq, mesh=nodes[conn], seed=23)
    An, bn, fn, cu = _run(ctx, et, kind, quad, cpq, prec, olay, nodes, conn, c)
    Ar, br, fr = run_oracle(et, kind, quad, cpq, nodes[conn], cu)
    ea, eb = max_errors(An, bn, Ar, br)
    assert ea <= TOL[prec] and eb <= TOL[prec], (ea, eb)
    assert (fn == fr).all()
    # the element-contiguous path on the same coordinates does the same arithmetic
    Aa, ba, fa, _ = _run(ctx, et, kind, quad, cpq, prec, olay, nodes, conn, c, layout=api.AOS)
    assert np.array_equal(An, Aa) and np.array_equal(bn, ba) and np.array_equal(fn, fa)


@pytest.mark.parametrize("et", [api.TET, api.PRISM])
def test_out_of_range_node_indices(ctx, et):
    """Indices outside [0, n_nodes) are not followed: those elements get zero
    results and flag bit 3; every other element is unaffected."""
    quad = api.QUAD_TET4 if et == api.TET else api.QUAD_PRISM6
    nodes, conn = _indexed(et, 1000)
    conn = conn.copy()
    bad = np.array([3, 64, 65, 500, 999])
    conn[3, 1] = -1
    conn[64, 0] = len(nodes)
    conn[65, -1] = 2 ** 31 - 1
    conn[500, 2] = -2 ** 31
    conn[999, 0] = len(nodes) + 7
    _, c = make_inputs(et, api.GENERIC, quad, 0, mesh=nodes[np.clip(conn, 0, len(nodes) - 1)], seed=24)
    for prec in PRECS:
        An, bn, fn, cu = _run(ctx, et, api.GENERIC, quad, 0, prec, api.AOS, nodes, conn, c)
        assert (fn[bad] == 8).all() and not An[bad].any() and not bn[bad].any()
        ok = np.setdiff1d(np.arange(1000), bad)
        Ar, br, fr = run_oracle(et, api.GENERIC, quad, 0, nodes[conn[ok]], cu[ok])
        ea, eb = max_errors(An[ok], bn[ok], Ar, br)
        assert ea <= TOL[prec] and eb <= TOL[prec], (prec, ea, eb)
        assert (fn[ok] == fr).all()


@pytest.mark.parametrize("et", [api.TET, api.PRISM])
def test_indexed_small_sizes_and_shapes(ctx, et):
    """Ragged sizes, every tuned launch shape, and the tuner itself."""
    quad = api.QUAD_TET4 if et == api.TET else api.QUAD_PRISM6
    nodes, conn_all = _indexed(et, 3000)
    X = torch.from_numpy(nodes).cuda()
    for n in [1, 2, 31, 33, 129, 257, 3000]:
        conn = np.ascontiguousarray(conn_all[:n])
        _, c = make_inputs(et, api.GENERIC, quad, 0, mesh=nodes[conn], seed=n)
        C = torch.from_numpy(c.astype(np.float32).reshape(n, -1)).cuda()
        K = torch.from_numpy(conn).cuda()
        kw = dict(kind=api.GENERIC, quad=quad, coef_mode=api.PER_ELEMENT, prec=api.FP32_MIXED, layout=api.INDEXED,
                  out_layout=api.AOS, conn=K)
        Ar, br, _ = run_oracle(et, api.GENERIC, quad, 0, nodes[conn], c.astype(np.float32).astype(np.float64))
        for shape in [(64, 0), (128, 1), (256, 0)]:
            ctx.set_shape(shape[0], shape[1], et, X, C, **kw)
            A, b, f = ctx.integrate(et, X, C, **kw)
            ctx.sync()
            ea, eb = max_errors(A.double().cpu().numpy(), b.double().cpu().numpy(), Ar, br)
            assert ea <= TOL[api.FP32_MIXED] and eb <= TOL[api.FP32_MIXED], (n, shape, ea, eb)
    # the tuner picks a shape and keeps the results
    ctx.tune(et, X, C, **kw)
    A, b, f = ctx.integrate(et, X, C, **kw)
    ctx.sync()
    ea, eb = max_errors(A.double().cpu().numpy(), b.double().cpu().numpy(), Ar, br)
    assert ea <= TOL[api.FP32_MIXED] and eb <= TOL[api.FP32_MIXED]


def test_indexed_slivers_fixup(ctx):
    """Poorly shaped elements of an indexed mesh take the double path (bit 0) in the
    mixed and double-word forms: their fix-up gathers coordinates through the table."""
    nodes, conn = meshgen.tet_cube_indexed(12, seed=meshgen.SEED_BASE + 63)
    nodes = nodes.copy()
    # flatten some tetrahedra: move node 3 of every 9th element onto the plane of the others
    rng = np.random.default_rng(5)
    sel = np.arange(0, len(conn), 97)
    for e in sel:
        a, b_, c_, d = conn[e]
        cen = (nodes[a] + nodes[b_] + nodes[c_]) / 3
        nodes[d] = cen + rng.uniform(0.002, 0.02) * (nodes[d] - cen)
    _, c = make_inputs(api.TET, api.GENERIC, api.QUAD_TET4, 0, mesh=nodes[conn], seed=25)
    for prec in (api.FP32_MIXED, api.FP64_DW):
        An, bn, fn, cu = _run(ctx, api.TET, api.GENERIC, api.QUAD_TET4, 0, prec, api.AOS, nodes, conn, c)
        Ar, br, fr = run_oracle(api.TET, api.GENERIC, api.QUAD_TET4, 0, nodes[conn], cu)
        ea, eb = max_errors(An, bn, Ar, br)
        assert ea <= TOL[prec] and eb <= TOL[prec], (prec, ea, eb)
        assert (fn & 1).sum() > 0
        assert ((fn & 6) == fr).all()
