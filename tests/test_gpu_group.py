"""Several threads per element, one row each (4 per tetrahedron, 6 per prism) or
one entry each (16 per tetrahedron; the intra-element parallelism of Sec. 3.3
with the QSS loop order kept): every
kind, precision form, rule and coefficient mode against the FP64 oracle on
ragged tiles, persistent and not; the same flags as one thread per element;
slivers and inverted elements through the fix-up; the launch-shape rules; the
autotuner's choice among one, two, four, six and sixteen threads per element."""
import itertools

import numpy as np
import pytest
import torch

import oracle
from helpers import TOL, make_inputs, max_errors, run_oracle
from paper_1504_01023_gb300 import api, meshgen

pytestmark = pytest.mark.gpu

PRECS = [api.FP64, api.FP32_MIXED, api.FP64_DW]
NS_OF = {api.TET: 4, api.PRISM: 6}


@pytest.fixture(scope="module")
def ctx():
    from paper_1504_01023_gb300 import build
    build.build()
    c = api.Context(0)
    yield c
    c.close()


def _run(ctx, et, mesh, c, kind, quad, cpq, prec, block, tpe, persistent=0):
    n = len(mesh)
    cdt = np.float32 if prec == api.FP32_MIXED else np.float64
    X = torch.from_numpy(np.ascontiguousarray(mesh)).cuda()
    C = torch.from_numpy(np.ascontiguousarray(c.astype(cdt).reshape(n, -1))).cuda()
    cm = api.PER_QPOINT if cpq else api.PER_ELEMENT
    out = api.alloc_out(et, n, prec, api.AOS, "cuda")
    kw = dict(kind=kind, quad=quad, coef_mode=cm, prec=prec, layout=api.AOS, out_layout=api.AOS, out=out)
    ctx.set_shape(block, persistent, et, X, C, tpe=tpe, **kw)
    assert ctx.shape(et, X, C, **kw) == (block, persistent, tpe)
    A, b, f = ctx.integrate(et, X, C, **kw)
    ctx.sync()
    return A.double().cpu().numpy(), b.double().cpu().numpy(), f.cpu().numpy(), c.astype(cdt).astype(np.float64)


CASES = [(api.TET, q, t) for q in (api.QUAD_TET1, api.QUAD_TET4) for t in (4, 16)] + [(api.PRISM, api.QUAD_PRISM6, 6)]


@pytest.mark.parametrize("et,quad,tpe", CASES)
@pytest.mark.parametrize("kind,cpq,prec", list(itertools.product([api.POISSON, api.GENERIC], [0, 1], PRECS)))
def test_rows_per_lane_match_oracle(ctx, et, quad, tpe, kind, cpq, prec):
    n = 1234 if et == api.TET else 777                 # ragged last tile
    mesh, c = make_inputs(et, kind, quad, cpq, n=n, seed=71 + kind + 2 * cpq)
    epw = 32 // tpe
    for block, pers in ((8 * epw, 0), (2 * epw, 1)):
        An, bn, fn, cu = _run(ctx, et, mesh, c, kind, quad, cpq, prec, block, tpe, pers)
        Ao, bo, fo = run_oracle(et, kind, quad, cpq, mesh, cu)
        ea, eb = max_errors(An, bn, Ao, bo)
        assert ea <= TOL[prec] and eb <= TOL[prec], (block, pers, ea, eb)
        assert np.array_equal(fn & 6, fo)
        # one thread per element flags the same elements
        A1, b1, f1, _ = _run(ctx, et, mesh, c, kind, quad, cpq, prec, 64, 1)
        assert np.array_equal(fn, f1)


@pytest.mark.parametrize("prec", [api.FP32_MIXED, api.FP64_DW, api.FP64])
def test_rows_per_lane_slivers_and_inverted(ctx, prec):
    """Poorly shaped elements take the double-precision fix-up (one thread each) in
    the mixed and double-word forms; inverted ones are flagged; every element meets
    the form's tolerance."""
    # tetrahedra: 10% slivers, a few inverted
    mesh = meshgen.tet_cube_mesh(9, seed=73)
    sl = meshgen.make_slivers(mesh, 0.1, seed=74)
    inv = np.arange(5, len(mesh), 97)
    mesh[inv] = mesh[inv][:, [0, 2, 1, 3]]
    _, c = make_inputs(api.TET, api.GENERIC, api.QUAD_TET4, 0, mesh=mesh, seed=75)
    for tpe, block in ((4, 64), (16, 16)):
        An, bn, fn, cu = _run(ctx, api.TET, mesh, c, api.GENERIC, api.QUAD_TET4, 0, prec, block, tpe)
        Ao, bo, fo = run_oracle(api.TET, api.GENERIC, api.QUAD_TET4, 0, mesh, cu)
        ea, eb = max_errors(An, bn, Ao, bo)
        assert ea <= TOL[prec] and eb <= TOL[prec], (tpe, ea, eb)
        assert np.array_equal(fn & 6, fo)
        if prec != api.FP64:
            q = oracle.quality(oracle.TET, mesh, n_threads=8)
            clear = np.abs(q - 0.1) > 1e-3 * 0.1
            assert np.array_equal((fn & 1).astype(bool)[clear], q[clear] < 0.1)
            assert (fn & 1).sum() >= 0.5 * len(sl)
    # prisms: flattened and inverted ones
    pm, pc = make_inputs(api.PRISM, api.GENERIC, api.QUAD_PRISM6, 1, n=1500, seed=76)
    pm = pm.copy()
    rng = np.random.default_rng(77)
    flat = rng.choice(len(pm), size=60, replace=False)
    pm[flat, 3:, 2] = pm[flat, :3, 2] + 5e-3 * (pm[flat, 3:, 2] - pm[flat, :3, 2])
    pm[flat] -= pm[flat, :1, :]
    pinv = np.setdiff1d(rng.choice(len(pm), size=40, replace=False), flat)
    pm[pinv] = pm[pinv][:, [3, 4, 5, 0, 1, 2]]
    An, bn, fn, cu = _run(ctx, api.PRISM, pm, pc, api.GENERIC, api.QUAD_PRISM6, 1, prec, 40, 6)
    Ao, bo, fo = run_oracle(api.PRISM, api.GENERIC, api.QUAD_PRISM6, 1, pm, cu)
    ea, eb = max_errors(An, bn, Ao, bo)
    assert ea <= TOL[prec] and eb <= TOL[prec], (ea, eb)
    assert np.array_equal(fn & 6, fo) and (fn[pinv] & 2).all()
    if prec != api.FP64:
        assert (fn[flat] & 1).all()


def test_rows_per_lane_shape_rules(ctx):
    tm, tc = make_inputs(api.TET, api.GENERIC, api.QUAD_TET4, 0, n=100, seed=78)
    pm, pc = make_inputs(api.PRISM, api.GENERIC, api.QUAD_PRISM6, 0, n=100, seed=79)
    T = (torch.from_numpy(np.ascontiguousarray(tm)).cuda(),
         torch.from_numpy(np.ascontiguousarray(tc.astype(np.float32).reshape(100, -1))).cuda(), api.TET, api.QUAD_TET4)
    P = (torch.from_numpy(np.ascontiguousarray(pm)).cuda(),
         torch.from_numpy(np.ascontiguousarray(pc.astype(np.float32).reshape(100, -1))).cuda(), api.PRISM,
         api.QUAD_PRISM6)
    kw = dict(kind=api.GENERIC, coef_mode=api.PER_ELEMENT, prec=api.FP32_MIXED)
    # the wrong group size for the type, or plane-major outputs: unsupported
    for (X, C, et, quad), tpe, block, outl in ((T, 6, 10, api.AOS), (P, 4, 16, api.AOS), (T, 4, 16, api.SOA),
                                               (P, 6, 10, api.SOA), (P, 16, 4, api.AOS), (T, 16, 4, api.SOA)):
        with pytest.raises(api.FeError) as e:
            ctx.set_shape(block, 0, et, X, C, quad=quad, layout=api.AOS, out_layout=outl, tpe=tpe, **kw)
        assert e.value.status == -6, (et, tpe, outl)
    # not whole warps of groups, or more than 256 threads
    for (X, C, et, quad), tpe, block in ((T, 4, 12, ), (T, 4, 72), (P, 6, 12), (P, 6, 45), (T, 16, 3), (T, 16, 18)):
        with pytest.raises(api.FeError) as e:
            ctx.set_shape(block, 0, et, X, C, quad=quad, layout=api.AOS, out_layout=api.AOS, tpe=tpe, **kw)
        assert e.value.status == -1, (et, tpe, block)


def test_tuner_considers_rows_per_lane(ctx):
    """The autotuner's candidates include four and sixteen threads per tetrahedron
    and two and six per prism; whatever it keeps gives oracle-accurate results."""
    for et, quad, cpq in ((api.TET, api.QUAD_TET4, 0), (api.PRISM, api.QUAD_PRISM6, 1)):
        mesh, c = make_inputs(et, api.GENERIC, quad, cpq, n=20000 if et == api.TET else 8000, seed=80)
        for prec in PRECS:
            cdt = np.float32 if prec == api.FP32_MIXED else np.float64
            X = torch.from_numpy(np.ascontiguousarray(mesh)).cuda()
            C = torch.from_numpy(np.ascontiguousarray(c.astype(cdt).reshape(len(mesh), -1))).cuda()
            kw = dict(kind=api.GENERIC, quad=quad, coef_mode=api.PER_QPOINT if cpq else api.PER_ELEMENT, prec=prec,
                      layout=api.AOS, out_layout=api.AOS)
            block, pers, tpe = ctx.tune(et, X, C, **kw)
            assert tpe in ((1, 4, 16) if et == api.TET else (1, 2, 6)) and pers in (0, 1)
            A, b, f = ctx.integrate(et, X, C, **kw)
            ctx.sync()
            Ao, bo, _ = run_oracle(et, api.GENERIC, quad, cpq, mesh, c.astype(cdt).astype(np.float64))
            ea, eb = max_errors(A.double().cpu().numpy(), b.double().cpu().numpy(), Ao, bo)
            assert ea <= TOL[prec] and eb <= TOL[prec]
