"""Prisms with two threads per element (each thread one zeta level of the point
loop, the pair adding its partial results): every kind, precision form and
coefficient mode against the FP64 oracle, on ragged tiles; the same flags as one
thread per element; the launch-shape rules; the autotuner's choice."""
import itertools

import numpy as np
import pytest
import torch

from helpers import TOL, make_inputs, max_errors, run_oracle
from paper_1504_01023_gb300 import api, meshgen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1504_01023_gb300 import build
    build.build()
    c = api.Context(0)
    yield c
    c.close()


def _run(ctx, mesh, c, kind, cpq, prec, block, tpe, persistent=0):
    n = len(mesh)
    cdt = np.float32 if prec == api.FP32_MIXED else np.float64
    X = torch.from_numpy(np.ascontiguousarray(mesh)).cuda()
    C = torch.from_numpy(np.ascontiguousarray(c.astype(cdt).reshape(n, -1))).cuda()
    cm = api.PER_QPOINT if cpq else api.PER_ELEMENT
    out = api.alloc_out(api.PRISM, n, prec, api.AOS, "cuda")
    kw = dict(kind=kind, quad=api.QUAD_PRISM6, coef_mode=cm, prec=prec, layout=api.AOS, out_layout=api.AOS, out=out)
    ctx.set_shape(block, persistent, api.PRISM, X, C, tpe=tpe, **kw)
    assert ctx.shape(api.PRISM, X, C, **kw) == (block, persistent, tpe)
    A, b, f = ctx.integrate(api.PRISM, X, C, **kw)
    ctx.sync()
    return A.double().cpu().numpy(), b.double().cpu().numpy(), f.cpu().numpy(), c.astype(cdt).astype(np.float64)


PRECS = [api.FP64, api.FP32_MIXED, api.FP64_DW]
CASES = list(itertools.product([api.POISSON, api.GENERIC], [0, 1], PRECS))


@pytest.mark.parametrize("kind,cpq,prec", CASES, ids=["k%d-c%d-p%d" % c for c in CASES])
def test_pair_matches_oracle_and_single_thread(ctx, kind, cpq, prec):
    mesh, c = make_inputs(api.PRISM, kind, api.QUAD_PRISM6, cpq, n=1999, seed=51)
    for block, pers in ((64, 0), (128, 1), (32, 0)):
        An, bn, fn, cu = _run(ctx, mesh, c, kind, cpq, prec, block, 2, pers)
        Ao, bo, fo = run_oracle(api.PRISM, kind, api.QUAD_PRISM6, cpq, mesh, cu)
        ea, eb = max_errors(An, bn, Ao, bo)
        assert ea <= TOL[prec] and eb <= TOL[prec], (block, pers, ea, eb)
        assert ((fn & 6) == fo).all()
    A1, b1, f1, _ = _run(ctx, mesh, c, kind, cpq, prec, 128, 1)
    assert np.array_equal(f1, fn)
    if kind == api.POISSON:
        assert np.allclose(An, An.transpose(0, 2, 1), rtol=0, atol=0)   # both lanes hold the same sums


@pytest.mark.parametrize("prec", [api.FP32_MIXED, api.FP64_DW])
def test_pair_poor_and_inverted_prisms(ctx, prec):
    """Flattened prisms take the double-precision fix-up (one thread each), inverted
    ones are flagged, in both launch shapes alike."""
    mesh, c = make_inputs(api.PRISM, api.GENERIC, api.QUAD_PRISM6, 1, n=1500, seed=52)
    mesh = mesh.copy()
    rng = np.random.default_rng(53)
    flat = rng.choice(len(mesh), size=60, replace=False)
    # height 0.5% of the element's size (mean ratio ~0.04), moved next to the origin
    # so that the oracle's absolute-coordinate Jacobian stays well conditioned
    mesh[flat, 3:, 2] = mesh[flat, :3, 2] + 5e-3 * (mesh[flat, 3:, 2] - mesh[flat, :3, 2])
    mesh[flat] -= mesh[flat, :1, :]
    inv = np.setdiff1d(rng.choice(len(mesh), size=40, replace=False), flat)
    mesh[inv] = mesh[inv][:, [3, 4, 5, 0, 1, 2]]
    An, bn, fn, cu = _run(ctx, mesh, c, api.GENERIC, 1, prec, 64, 2)
    A1, b1, f1, _ = _run(ctx, mesh, c, api.GENERIC, 1, prec, 64, 1)
    assert (fn[flat] & 1).all() and (fn[inv] & 2).all()
    assert np.array_equal(fn, f1)
    Ao, bo, fo = run_oracle(api.PRISM, api.GENERIC, api.QUAD_PRISM6, 1, mesh, cu)
    ea, eb = max_errors(An, bn, Ao, bo)
    assert ea <= TOL[prec] and eb <= TOL[prec], (ea, eb)


def test_pair_shape_rules(ctx):
    mesh, c = make_inputs(api.PRISM, api.GENERIC, api.QUAD_PRISM6, 0, n=100, seed=54)
    X = torch.from_numpy(np.ascontiguousarray(mesh)).cuda()
    C = torch.from_numpy(np.ascontiguousarray(c.astype(np.float32).reshape(100, -1))).cuda()
    kw = dict(kind=api.GENERIC, quad=api.QUAD_PRISM6, coef_mode=api.PER_ELEMENT, prec=api.FP32_MIXED)
    # plane-major output or coordinates: one thread per element only
    with pytest.raises(api.FeError) as e:
        ctx.set_shape(64, 0, api.PRISM, X, C, layout=api.AOS, out_layout=api.SOA, tpe=2, **kw)
    assert e.value.status == -6
    # tetrahedra: one thread per element only
    tm, tc = make_inputs(api.TET, api.GENERIC, api.QUAD_TET4, 0, n=100, seed=55)
    Xt = torch.from_numpy(np.ascontiguousarray(tm)).cuda()
    Ct = torch.from_numpy(np.ascontiguousarray(tc.astype(np.float32).reshape(100, -1))).cuda()
    with pytest.raises(api.FeError) as e:
        ctx.set_shape(64, 0, api.TET, Xt, Ct, kind=api.GENERIC, quad=api.QUAD_TET4, prec=api.FP32_MIXED,
                      layout=api.AOS, out_layout=api.AOS, tpe=2)
    assert e.value.status == -6
    # three threads, or more threads per block than the kernel allows
    for block, tpe in ((64, 3), (256, 2), (24, 1)):
        with pytest.raises(api.FeError) as e:
            ctx.set_shape(block, 0, api.PRISM, X, C, layout=api.AOS, out_layout=api.AOS, tpe=tpe, **kw)
        assert e.value.status == -1


def test_tuner_considers_two_threads_per_element(ctx):
    mesh, c = make_inputs(api.PRISM, api.GENERIC, api.QUAD_PRISM6, 1, n=20000, seed=56)
    for prec in PRECS:
        cdt = np.float32 if prec == api.FP32_MIXED else np.float64
        X = torch.from_numpy(np.ascontiguousarray(mesh)).cuda()
        C = torch.from_numpy(np.ascontiguousarray(c.astype(cdt).reshape(len(mesh), -1))).cuda()
        kw = dict(kind=api.GENERIC, quad=api.QUAD_PRISM6, coef_mode=api.PER_QPOINT, prec=prec, layout=api.AOS,
                  out_layout=api.AOS)
        block, pers, tpe = ctx.tune(api.PRISM, X, C, **kw)
        # one, two or six threads per prism (whole warps of groups, at most 256 threads)
        assert tpe in (1, 2, 6) and pers in (0, 1) and block % (32 // tpe) == 0 and block // (32 // tpe) * 32 <= 256
        A, b, f = ctx.integrate(api.PRISM, X, C, **kw)
        ctx.sync()
        Ao, bo, _ = run_oracle(api.PRISM, api.GENERIC, api.QUAD_PRISM6, 1, mesh, c.astype(cdt).astype(np.float64))
        ea, eb = max_errors(A.double().cpu().numpy(), b.double().cpu().numpy(), Ao, bo)
        assert ea <= TOL[prec] and eb <= TOL[prec]
