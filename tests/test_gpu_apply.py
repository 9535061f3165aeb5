"""Matrix-free application (fe_apply_*): y += sum_e P_e^T A^e P_e x and
f += sum_e P_e^T b^e over the elements of a node table, against the same sums
formed with numpy from the FP64 oracle's element matrices.

Atomic accumulation makes the order of the sums vary, so the comparison is per
node against a bound: the element tolerance times sum_e ||A^e||_F ||x_e||, plus
a few units of rounding of the accumulation precision times the magnitudes of
everything summed into the node."""
import itertools

import numpy as np
import pytest
import torch

from helpers import TOL, make_inputs, run_oracle
from paper_1504_01023_gb300 import api, meshgen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1504_01023_gb300 import build
    build.build()
    c = api.Context(0)
    yield c
    c.close()


def _mesh(et, n):
    if et == api.TET:
        nodes, conn = meshgen.tet_cube_indexed(8, seed=meshgen.SEED_BASE + 71)
    else:
        nodes, conn = meshgen.prism_slab_indexed(40, seed=meshgen.SEED_BASE + 72)
    return nodes, np.ascontiguousarray(conn[:n])


def _reference(A, b, conn, x, y0, f0, keep):
    """numpy: y0 + sum_e P_e^T A_e x_e, f0 + sum_e P_e^T b_e over elements `keep`,
    and per node the two parts of the bound."""
    A, b, c = A[keep], b[keep], conn[keep]
    xe = x[c]                                                         # [E, NS]
    contrib = np.einsum("ers,es->er", A, xe)
    y = y0.copy()
    np.add.at(y, c, contrib)
    f = f0.copy()
    np.add.at(f, c, b)
    scale_y = np.zeros_like(y0)
    np.add.at(scale_y, c, (np.linalg.norm(A.reshape(len(A), -1), axis=1) * np.linalg.norm(xe, axis=1))[:, None]
              * np.ones_like(contrib))
    mag_y = np.abs(y0).copy()
    np.add.at(mag_y, c, np.einsum("ers,es->er", np.abs(A), np.abs(xe)))
    scale_f = np.zeros_like(f0)
    np.add.at(scale_f, c, np.linalg.norm(b, axis=1)[:, None] * np.ones_like(b))
    mag_f = np.abs(f0).copy()
    np.add.at(mag_f, c, np.abs(b))
    return y, f, scale_y, mag_y, scale_f, mag_f


def _check(got, ref, scale, mag, prec):
    u = 2.0 ** -24 if prec == api.FP32_MIXED else 2.0 ** -53
    bound = TOL[prec] * scale + 64 * u * mag
    err = np.abs(got - ref)
    assert (err <= bound).all(), float((err / np.maximum(bound, 1e-300)).max())


def _vectors(n_nodes, prec, seed):
    rng = np.random.default_rng(seed)
    x = rng.uniform(-1, 1, n_nodes)
    y0 = rng.uniform(-1, 1, n_nodes)
    f0 = rng.uniform(-1, 1, n_nodes)
    dt = np.float32 if prec == api.FP32_MIXED else np.float64
    return [v.astype(dt) for v in (x, y0, f0)]


def _apply(ctx, et, kind, quad, cpq, prec, nodes, conn, c, x, y0, f0, with_f=True):
    n = len(conn)
    cdt = np.float32 if prec == api.FP32_MIXED else np.float64
    C = torch.from_numpy(np.ascontiguousarray(c.astype(cdt).reshape(n, -1))).cuda()
    X = torch.from_numpy(nodes).cuda()
    K = torch.from_numpy(conn).cuda()
    xt, yt, ft = (torch.from_numpy(v.copy()).cuda() for v in (x, y0, f0))
    flags = torch.zeros(n, dtype=torch.uint8, device="cuda")
    ctx.apply(et, X, K, C, kind, quad, xt, yt, ft if with_f else None,
              api.PER_QPOINT if cpq else api.PER_ELEMENT, prec, flags)
    ctx.sync()
    return yt.cpu().numpy().astype(np.float64), ft.cpu().numpy().astype(np.float64), flags.cpu().numpy(), \
        c.astype(cdt).astype(np.float64)


PRECS = [api.FP64, api.FP32_MIXED, api.FP64_DW]
CASES = ([(api.TET, k, q, c, p) for k, q, c, p in itertools.product(
            [api.POISSON, api.GENERIC], [api.QUAD_TET1, api.QUAD_TET4], [0, 1], PRECS)] +
         [(api.PRISM, k, api.QUAD_PRISM6, c, p) for k, c, p in itertools.product(
            [api.POISSON, api.GENERIC], [0, 1], PRECS)])


@pytest.mark.parametrize("et,kind,quad,cpq,prec", CASES, ids=["t%d-k%d-q%d-c%d-p%d" % c for c in CASES])
def test_apply_matches_oracle_sums(ctx, et, kind, quad, cpq, prec):
    n = 2999 if et == api.TET else 1999
    nodes, conn = _mesh(et, n)
    _, c = make_inputs(et, kind, quad, cpq, mesh=nodes[conn], seed=33)
    x, y0, f0 = _vectors(len(nodes), prec, 34)
    y, f, fl, cu = _apply(ctx, et, kind, quad, cpq, prec, nodes, conn, c, x, y0, f0)
    Ao, bo, fo = run_oracle(et, kind, quad, cpq, nodes[conn], cu)
    keep = np.arange(n)
    yr, fr, sy, my, sf, mf = _reference(Ao, bo, conn, x.astype(np.float64), y0.astype(np.float64),
                                        f0.astype(np.float64), keep)
    _check(y, yr, sy, my, prec)
    _check(f, fr, sf, mf, prec)
    assert ((fl & 6) == fo).all()


@pytest.mark.parametrize("prec", PRECS)
def test_apply_without_load_vector_and_twice(ctx, prec):
    """f = NULL leaves f alone; two calls accumulate twice."""
    nodes, conn = _mesh(api.TET, 3072)
    _, c = make_inputs(api.TET, api.GENERIC, api.QUAD_TET4, 0, mesh=nodes[conn], seed=35)
    x, y0, f0 = _vectors(len(nodes), prec, 36)
    n = len(conn)
    cdt = np.float32 if prec == api.FP32_MIXED else np.float64
    C = torch.from_numpy(np.ascontiguousarray(c.astype(cdt).reshape(n, -1))).cuda()
    X, K = torch.from_numpy(nodes).cuda(), torch.from_numpy(conn).cuda()
    xt, yt = torch.from_numpy(x.copy()).cuda(), torch.from_numpy(y0.copy()).cuda()
    for _ in range(2):
        ctx.apply(api.TET, X, K, C, api.GENERIC, api.QUAD_TET4, xt, yt, None, api.PER_ELEMENT, prec)
    ctx.sync()
    Ao, bo, _ = run_oracle(api.TET, api.GENERIC, api.QUAD_TET4, 0, nodes[conn], c.astype(cdt).astype(np.float64))
    yr, _, sy, my, _, _ = _reference(np.concatenate([Ao, Ao]), np.concatenate([bo, bo]), np.concatenate([conn, conn]),
                                     x.astype(np.float64), y0.astype(np.float64), f0.astype(np.float64),
                                     np.arange(2 * n))
    _check(yt.cpu().numpy().astype(np.float64), yr, sy, my, prec)


@pytest.mark.parametrize("et", [api.TET, api.PRISM])
def test_apply_out_of_range_indices_add_nothing(ctx, et):
    quad = api.QUAD_TET4 if et == api.TET else api.QUAD_PRISM6
    nodes, conn = _mesh(et, 1000)
    conn = conn.copy()
    bad = np.array([0, 77, 512, 999])
    conn[0, 1] = -5
    conn[77, 2] = len(nodes)
    conn[512, 0] = 2 ** 31 - 1
    conn[999, -1] = -2 ** 31
    safe = np.clip(conn, 0, len(nodes) - 1)
    _, c = make_inputs(et, api.GENERIC, quad, 0, mesh=nodes[safe], seed=37)
    for prec in PRECS:
        x, y0, f0 = _vectors(len(nodes), prec, 38)
        y, f, fl, cu = _apply(ctx, et, api.GENERIC, quad, 0, prec, nodes, conn, c, x, y0, f0)
        assert (fl[bad] == 8).all()
        keep = np.setdiff1d(np.arange(1000), bad)
        Ao, bo, _ = run_oracle(et, api.GENERIC, quad, 0, nodes[conn[keep]], cu[keep])
        Af = np.zeros((1000,) + Ao.shape[1:])
        bf = np.zeros((1000,) + bo.shape[1:])
        Af[keep], bf[keep] = Ao, bo
        yr, fr, sy, my, sf, mf = _reference(Af, bf, safe, x.astype(np.float64), y0.astype(np.float64),
                                            f0.astype(np.float64), keep)
        _check(y, yr, sy, my, prec)
        _check(f, fr, sf, mf, prec)


def test_apply_slivers_go_through_the_double_path(ctx):
    """Flagged elements add their double-precision results once."""
    nodes, conn = meshgen.tet_cube_indexed(12, seed=meshgen.SEED_BASE + 73)
    nodes = nodes.copy()
    rng = np.random.default_rng(9)
    for e in range(0, len(conn), 89):
        a, b_, c_, d = conn[e]
        cen = (nodes[a] + nodes[b_] + nodes[c_]) / 3
        nodes[d] = cen + rng.uniform(0.002, 0.02) * (nodes[d] - cen)
    _, c = make_inputs(api.TET, api.GENERIC, api.QUAD_TET4, 0, mesh=nodes[conn], seed=39)
    for prec in (api.FP32_MIXED, api.FP64_DW):
        x, y0, f0 = _vectors(len(nodes), prec, 40)
        y, f, fl, cu = _apply(ctx, api.TET, api.GENERIC, api.QUAD_TET4, 0, prec, nodes, conn, c, x, y0, f0)
        assert (fl & 1).sum() > 0
        Ao, bo, fo = run_oracle(api.TET, api.GENERIC, api.QUAD_TET4, 0, nodes[conn], cu)
        yr, fr, sy, my, sf, mf = _reference(Ao, bo, conn, x.astype(np.float64), y0.astype(np.float64),
                                            f0.astype(np.float64), np.arange(len(conn)))
        _check(y, yr, sy, my, prec)
        _check(f, fr, sf, mf, prec)


def test_apply_rejects_element_contiguous_geometry(ctx):
    nodes, conn = _mesh(api.TET, 100)
    X = torch.from_numpy(np.ascontiguousarray(nodes[conn])).cuda()
    C = torch.zeros((100, 20), dtype=torch.float32, device="cuda")
    a = api.make_args(api.TET, X, C, api.GENERIC, api.QUAD_TET4, api.PER_ELEMENT, api.FP32_MIXED, api.AOS)
    v = torch.zeros(100, dtype=torch.float32, device="cuda")
    st = api.load().fe_apply_tet(ctx.h, __import__("ctypes").byref(a), v.data_ptr(), v.data_ptr(), None, None, None)
    assert st == -6


def _fan_mesh(layers=30, ring=12):
    """Stacked fans of tetrahedra around the z axis: layer L has apex (0, 0, L),
    top (0, 0, L + 1) and a ring of `ring` nodes at height L + 1/2; its elements
    are (apex, ring_i, ring_i+1, top). Every element of a layer holds the apex in
    slot 0 and the top in slot 3, the top is the next layer's apex (slot 0), and
    each ring node sits in slot 1 of one element and slot 2 of its neighbour."""
    th = 2 * np.pi * np.arange(ring) / ring
    nodes = [(0.0, 0.0, float(L)) for L in range(layers + 1)]
    conn = []
    for L in range(layers):
        base = len(nodes)
        nodes += [(np.cos(t), np.sin(t), L + 0.5) for t in th]
        for i in range(ring):
            conn.append((L, base + i, base + (i + 1) % ring, L + 1))
    return np.asarray(nodes, dtype=np.float64), np.asarray(conn, dtype=np.int32)


@pytest.mark.parametrize("prec", PRECS)
def test_apply_nodes_shared_across_a_warp(ctx, prec):
    """Many lanes of a warp add to the same node, from the same slot and from
    different slots; the sums are those of the oracle's element matrices."""
    nodes, conn = _fan_mesh()
    _, c = make_inputs(api.TET, api.GENERIC, api.QUAD_TET4, 0, mesh=nodes[conn], seed=41)
    x, y0, f0 = _vectors(len(nodes), prec, 42)
    y, f, fl, cu = _apply(ctx, api.TET, api.GENERIC, api.QUAD_TET4, 0, prec, nodes, conn, c, x, y0, f0)
    Ao, bo, fo = run_oracle(api.TET, api.GENERIC, api.QUAD_TET4, 0, nodes[conn], cu)
    assert ((fl & 6) == fo).all()
    yr, fr, sy, my, sf, mf = _reference(Ao, bo, conn, x.astype(np.float64), y0.astype(np.float64),
                                        f0.astype(np.float64), np.arange(len(conn)))
    _check(y, yr, sy, my, prec)
    _check(f, fr, sf, mf, prec)
