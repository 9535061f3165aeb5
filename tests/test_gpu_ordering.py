"""Loop-ordering study kernels (SQS, SSQ; Algorithms 4-7) in the mixed form:
the same element matrices as the oracle within the mixed tolerance, and the same
shape-test flags as the QSS kernels."""
import itertools

import numpy as np
import pytest
import torch

import oracle
from helpers import TOL, gpu_outputs_to_numpy, make_inputs, max_errors, run_oracle, to_device_inputs
from paper_1504_01023_gb300 import api, meshgen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1504_01023_gb300 import build
    build.build()
    c = api.Context(0)
    yield c
    c.close()


def _run(ctx, et, kind, quad, cpq, ordering, mesh, c):
    X, C, cu = to_device_inputs(et, mesh, c, api.FP32_MIXED, api.AOS)
    cm = api.PER_QPOINT if cpq else api.PER_ELEMENT
    A, b, f = ctx.integrate(et, X, C, kind, quad, cm, api.FP32_MIXED, api.AOS, api.AOS, ordering=ordering)
    ctx.sync()
    return (*gpu_outputs_to_numpy(et, A, b, f, api.AOS), cu)


CASES = ([(api.TET, k, q, c, o) for k, q, c, o in itertools.product(
            [api.POISSON, api.GENERIC], [api.QUAD_TET1, api.QUAD_TET4], [0, 1], [api.SQS, api.SSQ])] +
         [(api.PRISM, k, api.QUAD_PRISM6, c, o) for k, c, o in itertools.product(
            [api.POISSON, api.GENERIC], [0, 1], [api.SQS, api.SSQ])])


@pytest.mark.parametrize("et,kind,quad,cpq,ordering", CASES, ids=["t%d-k%d-q%d-c%d-o%d" % c for c in CASES])
def test_ordering_parity(ctx, et, kind, quad, cpq, ordering):
    mesh, c = make_inputs(et, kind, quad, cpq, n=2999 if et == api.TET else 1999, seed=61)
    An, bn, fn, cu = _run(ctx, et, kind, quad, cpq, ordering, mesh, c)
    Ar, br, fr = run_oracle(et, kind, quad, cpq, mesh, cu)
    ea, eb = max_errors(An, bn, Ar, br)
    assert ea <= TOL[api.FP32_MIXED] and eb <= TOL[api.FP32_MIXED], (ea, eb)
    assert (fn == fr).all()
    Aq, bq, fq, _ = _run(ctx, et, kind, quad, cpq, api.QSS, mesh, c)
    assert np.array_equal(fn, fq)


@pytest.mark.parametrize("ordering", [api.SQS, api.SSQ])
def test_ordering_slivers_take_the_double_path(ctx, ordering):
    mesh = meshgen.tet_cube_mesh(12, seed=meshgen.SEED_BASE + 2)
    meshgen.make_slivers(mesh, 0.1, seed=meshgen.SEED_BASE + 22)
    _, c = make_inputs(api.TET, api.GENERIC, api.QUAD_TET4, 0, mesh=mesh, seed=62)
    An, bn, fn, cu = _run(ctx, api.TET, api.GENERIC, api.QUAD_TET4, 0, ordering, mesh, c)
    Ar, br, fr = run_oracle(api.TET, api.GENERIC, api.QUAD_TET4, 0, mesh, cu)
    ea, eb = max_errors(An, bn, Ar, br)
    assert ea <= TOL[api.FP32_MIXED] and eb <= TOL[api.FP32_MIXED], (ea, eb)
    q = oracle.quality(oracle.TET, mesh, n_threads=8)
    clear = np.abs(q - 0.1) > 1e-4
    assert (((fn & 1) > 0)[clear] == (q[clear] < 0.1)).all()
