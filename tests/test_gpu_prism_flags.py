"""The shape test of prisms (not in the paper; it routes poorly shaped elements to
the double-precision Jacobian pass): flag bit 0 of the mixed and double-word forms
against the oracle's single-precision mean ratio (minimum over the six points) on
every element clear of the 0.1 threshold, with one and two threads per element,
for both kinds; and the results within each form's tolerance."""
import numpy as np
import pytest
import torch

import oracle
from helpers import TOL, make_inputs, max_errors, run_oracle
from paper_1504_01023_gb300 import api, build, meshgen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    build.build()
    c = api.Context(0)
    yield c
    c.close()


def flattened_prisms(seed):
    """3,200 prisms of the slab (legs and height 1/40), each top flattened towards
    its bottom by a factor log-uniform in [0.015, 0.7] and 30% of them sheared
    sideways: mean ratios from about 0.003 to 0.85, a fifth below 0.1 (a few of the
    thinnest sheared ones invert at some points over their jittered bottoms). Every
    element is moved to start at the origin, which keeps the oracle's Jacobian
    (formed from absolute coordinates) well conditioned."""
    x = meshgen.prism_slab_mesh(40, seed=seed).copy()
    n = len(x)
    rng = np.random.default_rng(seed + 1)
    s = np.exp(rng.uniform(np.log(0.015), np.log(0.7), n))
    x[:, 3:, 2] = x[:, :3, 2] + s[:, None] * (x[:, 3:, 2] - x[:, :3, 2])
    x[:, 3:, :2] += rng.uniform(-0.02, 0.02, (n, 1, 2)) * (rng.random((n, 1, 1)) < 0.3)
    return np.ascontiguousarray(x - x[:, :1])


@pytest.mark.parametrize("tpe", [1, 2])
@pytest.mark.parametrize("prec", [api.FP32_MIXED, api.FP64_DW])
@pytest.mark.parametrize("kind", [api.GENERIC, api.POISSON])
def test_prism_flag_matches_oracle_quality(ctx, kind, prec, tpe):
    mesh = flattened_prisms(81)
    n = len(mesh)
    _, c = make_inputs(api.PRISM, kind, api.QUAD_PRISM6, 1, mesh=mesh, seed=82)
    cdt = np.float32 if prec == api.FP32_MIXED else np.float64
    X = torch.from_numpy(mesh).cuda()
    C = torch.from_numpy(np.ascontiguousarray(c.astype(cdt).reshape(n, -1))).cuda()
    kw = dict(kind=kind, quad=api.QUAD_PRISM6, coef_mode=api.PER_QPOINT, prec=prec, layout=api.AOS,
              out_layout=api.AOS)
    out = api.alloc_out(api.PRISM, n, prec, api.AOS, "cuda")
    ctx.set_shape(64, 0, api.PRISM, X, C, tpe=tpe, out=out, **kw)
    A, b, f = ctx.integrate(api.PRISM, X, C, out=out, **kw)
    ctx.sync()
    fn = f.cpu().numpy()
    q = oracle.quality(oracle.PRISM, mesh, n_threads=8)
    flagged = (fn & 1).astype(bool)
    clear = np.abs(q - 0.1) > 1e-3 * 0.1
    assert clear.sum() >= n - 5
    assert (q < 0.1).sum() > 300 and (q >= 0.1).sum() > 2000
    assert np.array_equal(flagged[clear], q[clear] < 0.1), np.flatnonzero(flagged[clear] != (q[clear] < 0.1))[:10]
    cu = c.astype(cdt).astype(np.float64)
    Ao, bo, fo = run_oracle(api.PRISM, kind, api.QUAD_PRISM6, 1, mesh, cu)
    # the thinnest sheared prisms over a sloped bottom invert at some points (bit 1)
    assert np.array_equal(fn & 6, fo)
    ea, eb = max_errors(A.double().cpu().numpy(), b.double().cpu().numpy(), Ao, bo)
    assert ea <= TOL[prec] and eb <= TOL[prec], (ea, eb)
