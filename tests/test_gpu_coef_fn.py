"""Coefficients from a function of a nodal field (FE_COEF_FUNCTION_U): the kernels
interpolate u at the integration points and evaluate c_j(u_Q) = P0_j + P1_j u_Q +
P2_j u_Q^2; the oracle does the same at its own rule points with its own shape
functions (oracle.coefs_from_u) and integrates with per-point coefficients."""
import itertools

import numpy as np
import pytest
import torch

import oracle
from helpers import ORACLE_RULE, TOL, gpu_outputs_to_numpy, max_errors
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
        return meshgen.tet_cube_mesh(8, seed=meshgen.SEED_BASE + 81)[:n]
    return meshgen.prism_slab_mesh(40, seed=meshgen.SEED_BASE + 82)[:n]


def _field(mesh):
    """A smooth field evaluated at every element's vertices: u in about [-1, 2]."""
    x, y, z = mesh[..., 0], mesh[..., 1], mesh[..., 2]
    return np.sin(3.0 * x) + y * y - 0.5 * z


def _params(seed):
    rng = np.random.default_rng(seed)
    P = rng.uniform(-1.0, 1.0, (3, 20))
    # keep the diffusion block dominant, as for a physical c(u)
    for i in (5, 10, 15):
        P[0, i] += 4.0
    return P


def _run(ctx, et, kind, quad, prec, olay, mesh, u, P):
    n = len(mesh)
    dt = np.float32 if prec == api.FP32_MIXED else np.float64
    X = torch.from_numpy(np.ascontiguousarray(mesh)).cuda()
    U = torch.from_numpy(np.ascontiguousarray(u.astype(dt))).cuda()
    A, b, f = ctx.integrate(et, X, U, kind, quad, api.COEF_FN_U, prec, api.AOS, olay, coef_fn=P)
    ctx.sync()
    return (*gpu_outputs_to_numpy(et, A, b, f, olay), u.astype(dt).astype(np.float64))


PRECS = [api.FP64, api.FP32_MIXED, api.FP64_DW]
CASES = ([(api.TET, k, q, p, o) for k, q, p, o in itertools.product(
            [api.POISSON, api.GENERIC], [api.QUAD_TET1, api.QUAD_TET4], PRECS, [api.SOA, api.AOS])] +
         [(api.PRISM, k, api.QUAD_PRISM6, p, o) for k, p, o in itertools.product(
            [api.POISSON, api.GENERIC], PRECS, [api.SOA, api.AOS])])


@pytest.mark.parametrize("et,kind,quad,prec,olay", CASES, ids=["t%d-k%d-q%d-p%d-o%d" % c for c in CASES])
def test_coef_function_parity(ctx, et, kind, quad, prec, olay):
    mesh = _mesh(et, 2999 if et == api.TET else 1999)
    u = _field(mesh)
    P = _params(91)
    An, bn, fn, uu = _run(ctx, et, kind, quad, prec, olay, mesh, u, P)
    rule = ORACLE_RULE[quad]
    cq = oracle.coefs_from_u(et, kind, rule, uu, P)
    Ar, br, fr = oracle.integrate(et, kind, rule, mesh, cq, coef_per_q=True, n_threads=8)
    ea, eb = max_errors(An, bn, Ar, br)
    assert ea <= TOL[prec] and eb <= TOL[prec], (ea, eb)
    assert (fn == fr).all()


@pytest.mark.parametrize("prec", [api.FP32_MIXED, api.FP64_DW])
def test_coef_function_slivers(ctx, prec):
    mesh = meshgen.tet_cube_mesh(12, seed=meshgen.SEED_BASE + 2)
    meshgen.make_slivers(mesh, 0.1, seed=meshgen.SEED_BASE + 23)
    u = _field(mesh)
    P = _params(92)
    An, bn, fn, uu = _run(ctx, api.TET, api.GENERIC, api.QUAD_TET4, prec, api.AOS, mesh, u, P)
    cq = oracle.coefs_from_u(api.TET, api.GENERIC, oracle.Q_TET4, uu, P)
    Ar, br, fr = oracle.integrate(api.TET, api.GENERIC, oracle.Q_TET4, mesh, cq, coef_per_q=True, n_threads=8)
    ea, eb = max_errors(An, bn, Ar, br)
    assert ea <= TOL[prec] and eb <= TOL[prec], (ea, eb)
    assert (fn & 1).sum() > 0 and ((fn & 6) == fr).all()


def test_coef_function_rejected_where_unsupported(ctx):
    mesh = _mesh(api.TET, 100)
    X = torch.from_numpy(np.ascontiguousarray(mesh)).cuda()
    U = torch.zeros((100, 4), dtype=torch.float32, device="cuda")
    P = np.zeros((3, 20))
    # plane-major coordinates
    Xs = torch.from_numpy(meshgen.soa(mesh)).cuda()
    with pytest.raises(api.FeError) as e:
        ctx.integrate(api.TET, Xs, U.T.contiguous(), api.GENERIC, api.QUAD_TET4, api.COEF_FN_U, api.FP32_MIXED,
                      api.SOA, api.AOS, coef_fn=P)
    assert e.value.status == -6
    # batched
    out = api.alloc_out(api.TET, 100, api.FP32_MIXED, api.AOS, "cuda")
    a = api.make_args(api.TET, X, U, api.GENERIC, api.QUAD_TET4, api.COEF_FN_U, api.FP32_MIXED, api.AOS, coef_fn=P)
    with pytest.raises(api.FeError) as e:
        ctx.batch_submit([(api.TET, a, api.make_out(*out, api.AOS))])
    assert e.value.status == -6
