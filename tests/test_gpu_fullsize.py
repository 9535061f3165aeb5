"""Parity at the full workload sizes, in the launch configuration the benchmark
uses (tuned shape, natural element-contiguous order), on elements sampled at
random and recomputed one by one by the FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle
from helpers import TOL, max_errors
from paper_1504_01023_gb300 import api, meshgen

pytestmark = pytest.mark.gpu

SAMPLE = 4000


@pytest.fixture(scope="module")
def ctx():
    from paper_1504_01023_gb300 import build
    build.build()
    c = api.Context(0)
    yield c
    c.close()


def _run_aos(ctx, et, mesh, coefs, kind, quad, cm, prec, tune=True):
    n = len(mesh)
    cdt = np.float32 if prec == api.FP32_MIXED else np.float64
    X = torch.from_numpy(np.ascontiguousarray(mesh)).cuda()
    C = torch.from_numpy(np.ascontiguousarray(coefs.reshape(n, -1).astype(cdt))).cuda()
    out = api.alloc_out(et, n, prec, api.AOS, "cuda")
    kw = dict(kind=kind, quad=quad, coef_mode=cm, prec=prec, layout=api.AOS, out_layout=api.AOS, out=out)
    if tune:
        ctx.tune(et, X, C, **kw)
    A, b, f = ctx.integrate(et, X, C, **kw)
    ctx.sync()
    return A, b, f, coefs.reshape(n, -1).astype(cdt).astype(np.float64)


def _check_sample(et, A, b, f, mesh, c, kind, rule, cpq, tol, seed):
    n = len(mesh)
    idx = np.sort(np.random.default_rng(seed).choice(n, size=min(SAMPLE, n), replace=False))
    it = torch.from_numpy(idx).cuda()
    An = A[it].double().cpu().numpy()
    bn = b[it].double().cpu().numpy()
    cs = c[idx]
    if cpq:
        cs = cs.reshape(len(idx), -1 if kind == api.POISSON else 6, *(() if kind == api.POISSON else (20,)))
    Ar, br, fr = oracle.integrate(et, kind, rule, mesh[idx], cs, coef_per_q=bool(cpq), n_threads=8)
    ea, eb = max_errors(An, bn, Ar, br)
    assert ea <= tol and eb <= tol, (ea, eb)
    assert ((f[it].cpu().numpy() & 6) == fr).all()


def test_poisson_tets_48k_fp64_every_element(ctx):
    """20^3 x 6 = 48,000 Poisson tetrahedra, 1-point rule, d^0 = 1, FP64: all elements."""
    mesh = meshgen.tet_cube_mesh(20, 0.2, seed=meshgen.SEED_BASE + 1)
    d0 = meshgen.poisson_coefs(len(mesh), 1, 1.0)
    A, b, f, cu = _run_aos(ctx, api.TET, mesh, d0, api.POISSON, api.QUAD_TET1, api.PER_ELEMENT, api.FP64)
    Ar, br, fr = oracle.integrate(api.TET, api.POISSON, oracle.Q_TET1, mesh, cu.reshape(-1), n_threads=8)
    ea, eb = max_errors(A.cpu().numpy(), b.cpu().numpy(), Ar, br)
    assert ea <= TOL[api.FP64] and eb <= TOL[api.FP64], (ea, eb)
    assert (f.cpu().numpy() == fr).all()


def test_generic_tets_6M_mixed_sampled(ctx):
    mesh = meshgen.tet_cube_mesh(100, 0.2, seed=meshgen.SEED_BASE + 2)
    c = meshgen.generic_coefs(len(mesh), 1, seed=meshgen.SEED_BASE + 2)
    A, b, f, cu = _run_aos(ctx, api.TET, mesh, c, api.GENERIC, api.QUAD_TET4, api.PER_ELEMENT, api.FP32_MIXED)
    assert not (f.cpu().numpy() & 1).any()     # no element of this mesh is poorly shaped
    _check_sample(api.TET, A, b, f, mesh, cu, api.GENERIC, oracle.Q_TET4, 0, TOL[api.FP32_MIXED], 1)


def test_generic_tets_6M_fp64_sampled(ctx):
    """The benchmark's step: the default shape, the autotuner's choice (as the
    benchmark times it) and the two tile sizes the tuner picks between."""
    mesh = meshgen.tet_cube_mesh(100, 0.2, seed=meshgen.SEED_BASE + 2)
    c = meshgen.generic_coefs(len(mesh), 1, seed=meshgen.SEED_BASE + 2)
    A, b, f, cu = _run_aos(ctx, api.TET, mesh, c, api.GENERIC, api.QUAD_TET4, api.PER_ELEMENT, api.FP64, tune=False)
    _check_sample(api.TET, A, b, f, mesh, cu, api.GENERIC, oracle.Q_TET4, 0, TOL[api.FP64], 2)
    A, b, f, cu = _run_aos(ctx, api.TET, mesh, c, api.GENERIC, api.QUAD_TET4, api.PER_ELEMENT, api.FP64, tune=True)
    _check_sample(api.TET, A, b, f, mesh, cu, api.GENERIC, oracle.Q_TET4, 0, TOL[api.FP64], 3)
    n = len(mesh)
    X = torch.from_numpy(np.ascontiguousarray(mesh)).cuda()
    C = torch.from_numpy(np.ascontiguousarray(c.reshape(n, -1))).cuda()
    kw = dict(kind=api.GENERIC, quad=api.QUAD_TET4, coef_mode=api.PER_ELEMENT, prec=api.FP64, layout=api.AOS,
              out_layout=api.AOS)
    for block, seed in ((64, 4), (128, 5)):
        ctx.set_shape(block, 0, api.TET, X, C, **kw)
        A, b, f = ctx.integrate(api.TET, X, C, **kw)
        ctx.sync()
        _check_sample(api.TET, A, b, f, mesh, cu, api.GENERIC, oracle.Q_TET4, 0, TOL[api.FP64], seed)


def test_generic_prisms_2M_mixed_sampled(ctx):
    mesh = meshgen.prism_slab_mesh(1000, None, 0.1, seed=meshgen.SEED_BASE + 3)
    c = meshgen.generic_coefs(len(mesh), 6, seed=meshgen.SEED_BASE + 3)
    A, b, f, cu = _run_aos(ctx, api.PRISM, mesh, c, api.GENERIC, api.QUAD_PRISM6, api.PER_QPOINT, api.FP32_MIXED)
    _check_sample(api.PRISM, A, b, f, mesh, cu, api.GENERIC, oracle.Q_PRISM6, 1, TOL[api.FP32_MIXED], 3)


def test_generic_tets_with_slivers_6M_mixed(ctx):
    """1% of the 6M elements flattened to mean ratio < 0.1: they take the double
    Jacobian path; sampled parity over flagged and unflagged elements."""
    mesh = meshgen.tet_cube_mesh(100, 0.2, seed=meshgen.SEED_BASE + 2)
    sl = meshgen.make_slivers(mesh, 0.01, seed=meshgen.SEED_BASE + 20)
    c = meshgen.generic_coefs(len(mesh), 1, seed=meshgen.SEED_BASE + 2)
    A, b, f, cu = _run_aos(ctx, api.TET, mesh, c, api.GENERIC, api.QUAD_TET4, api.PER_ELEMENT, api.FP32_MIXED, tune=False)
    fl = f.cpu().numpy()
    assert (fl & 1).sum() >= 0.5 * len(sl)
    _check_sample(api.TET, A, b, f, mesh, cu, api.GENERIC, oracle.Q_TET4, 0, TOL[api.FP32_MIXED], 4)
    # and all flagged elements (double Jacobian path)
    idx = np.nonzero(fl & 1)[0]
    it = torch.from_numpy(idx).cuda()
    Ar, br, _ = oracle.integrate(api.TET, api.GENERIC, oracle.Q_TET4, mesh[idx], cu[idx], n_threads=8)
    ea, eb = max_errors(A[it].double().cpu().numpy(), b[it].double().cpu().numpy(), Ar, br)
    assert ea <= TOL[api.FP32_MIXED] and eb <= TOL[api.FP32_MIXED], (ea, eb)


def test_batched_256_meshes_sampled():
    """The 256-mesh batch (sizes log-uniform [1e3, 2e6]) through the captured graph;
    every mesh checked on a sample against the oracle."""
    import bench
    from paper_1504_01023_gb300 import build
    build.build()
    dev = torch.device("cuda", 0)
    specs = meshgen.batch_mix(256, 1e3, 2e6, seed=meshgen.SEED_BASE + 4)
    pool = bench.DevicePool(2_000_000, meshgen.SEED_BASE + 40, dev)
    ctx = api.Context(0, autotune=True)
    items, keep = [], []
    for n, et, kind in specs:
        X, C, quad, cpq = pool.mesh(et, kind, n)
        out = api.alloc_out(et, n, api.FP32_MIXED, api.AOS, dev)
        cm = api.PER_QPOINT if cpq else api.PER_ELEMENT
        items.append((et, api.make_args(et, X, C, kind, quad, cm, api.FP32_MIXED, api.AOS), api.make_out(*out, api.AOS)))
        keep.append((et, kind, quad, cpq, X, C, out))
    ctx.batch_submit(items)
    ctx.batch_submit(items)                    # graph replay
    ctx.sync()
    rule = {api.QUAD_TET1: oracle.Q_TET1, api.QUAD_TET4: oracle.Q_TET4, api.QUAD_PRISM6: oracle.Q_PRISM6}
    rng = np.random.default_rng(5)
    for et, kind, quad, cpq, X, C, (A, b, f) in keep:
        n = X.shape[0]
        idx = np.sort(rng.choice(n, size=min(64, n), replace=False))
        it = torch.from_numpy(idx).cuda()
        x = X[it].cpu().numpy()
        cs = C[it].double().cpu().numpy()
        if kind == api.POISSON:
            cs = cs.reshape(len(idx), -1) if cpq else cs.reshape(-1)
        else:
            cs = cs.reshape(len(idx), 6, 20) if cpq else cs.reshape(len(idx), 20)
        Ar, br, _ = oracle.integrate(et, kind, rule[quad], x, cs, coef_per_q=bool(cpq), n_threads=8)
        ea, eb = max_errors(A[it].double().cpu().numpy(), b[it].double().cpu().numpy(), Ar, br)
        assert ea <= TOL[api.FP32_MIXED] and eb <= TOL[api.FP32_MIXED], (et, kind, quad, cpq, ea, eb)
    ctx.close()


def test_poisson_tets_48k_double_word_every_element(ctx):
    """The 48,000-element Poisson workload in the double-word form: every element
    against the oracle at the double-precision tolerance."""
    mesh = meshgen.tet_cube_mesh(20, 0.2, seed=meshgen.SEED_BASE + 1)
    d0 = meshgen.poisson_coefs(len(mesh), 1, 1.0)
    A, b, f, cu = _run_aos(ctx, api.TET, mesh, d0, api.POISSON, api.QUAD_TET1, api.PER_ELEMENT, api.FP64_DW)
    Ar, br, fr = oracle.integrate(api.TET, api.POISSON, oracle.Q_TET1, mesh, cu.reshape(-1), n_threads=8)
    ea, eb = max_errors(A.cpu().numpy(), b.cpu().numpy(), Ar, br)
    assert ea <= TOL[api.FP64_DW] and eb <= TOL[api.FP64_DW], (ea, eb)
    assert ((f.cpu().numpy() & 6) == fr).all()


def test_poisson_tets_6M_double_word_sampled(ctx):
    """100^3 x 6 Poisson tetrahedra (the double-precision benchmark workload), tuned
    shape, double-word form."""
    mesh = meshgen.tet_cube_mesh(100, 0.2, seed=meshgen.SEED_BASE + 2)
    d0 = meshgen.poisson_coefs(len(mesh), 1, 1.0)
    A, b, f, cu = _run_aos(ctx, api.TET, mesh, d0, api.POISSON, api.QUAD_TET1, api.PER_ELEMENT, api.FP64_DW)
    _check_sample(api.TET, A, b, f, mesh, cu.reshape(-1), api.POISSON, oracle.Q_TET1, 0, TOL[api.FP64_DW], 3)


def test_generic_tets_6M_double_word_sampled(ctx):
    mesh = meshgen.tet_cube_mesh(100, 0.2, seed=meshgen.SEED_BASE + 2)
    c = meshgen.generic_coefs(len(mesh), 1, seed=meshgen.SEED_BASE + 2)
    A, b, f, cu = _run_aos(ctx, api.TET, mesh, c, api.GENERIC, api.QUAD_TET4, api.PER_ELEMENT, api.FP64_DW)
    _check_sample(api.TET, A, b, f, mesh, cu, api.GENERIC, oracle.Q_TET4, 0, TOL[api.FP64_DW], 4)
