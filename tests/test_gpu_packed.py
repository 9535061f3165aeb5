"""Packed (upper-triangle) output of the symmetric Laplace A^e: bit-identical to
the upper triangle of the full output, in every layout, precision and memory."""
import itertools

import numpy as np
import pytest
import torch

from helpers import make_inputs, to_device_inputs
from paper_1504_01023_gb300 import api

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1504_01023_gb300 import build
    build.build()
    c = api.Context(0)
    yield c
    c.close()


def _upper(A, ns):
    r, s = np.triu_indices(ns)
    return A[:, r, s]


def _full_and_packed(ctx, et, quad, cpq, prec, lay, olay, n, device="cuda"):
    mesh, c = make_inputs(et, api.POISSON, quad, cpq, n=n, seed=51)
    X, C, _ = to_device_inputs(et, mesh, c, prec, lay, device)
    cm = api.PER_QPOINT if cpq else api.PER_ELEMENT
    A, b, f = ctx.integrate(et, X, C, api.POISSON, quad, cm, prec, lay, olay)
    Ap, bp, fp = ctx.integrate(et, X, C, api.POISSON, quad, cm, prec, lay, olay, packed=True)
    ctx.sync()
    ns = api.NS[et]
    if olay == api.SOA:
        A = A.T.reshape(-1, ns, ns)
        Ap, b, bp = Ap.T, b.T, bp.T
    A, Ap, b, bp = (t.cpu().numpy() for t in (A, Ap, b, bp))
    return _upper(A, ns), Ap, b, bp, f.cpu().numpy(), fp.cpu().numpy()


PRECS = [api.FP64, api.FP32_MIXED, api.FP64_DW]
CASES = ([(api.TET, q, c, p, i, o) for q, c, p, i, o in itertools.product(
            [api.QUAD_TET1, api.QUAD_TET4], [0, 1], PRECS, [api.SOA, api.AOS], [api.SOA, api.AOS])] +
         [(api.PRISM, api.QUAD_PRISM6, c, p, i, o) for c, p, i, o in itertools.product(
            [0, 1], PRECS, [api.SOA, api.AOS], [api.SOA, api.AOS])])


@pytest.mark.parametrize("et,quad,cpq,prec,lay,olay", CASES, ids=["t%d-q%d-c%d-p%d-i%d-o%d" % c for c in CASES])
def test_packed_is_the_upper_triangle(ctx, et, quad, cpq, prec, lay, olay):
    n = 2999 if et == api.TET else 1999
    Au, Ap, b, bp, f, fp = _full_and_packed(ctx, et, quad, cpq, prec, lay, olay, n)
    assert Ap.shape == Au.shape
    assert np.array_equal(Au, Ap) and np.array_equal(b, bp) and np.array_equal(f, fp)


@pytest.mark.parametrize("pinned", [True, False])
def test_packed_host_buffers(ctx, pinned):
    """The chunked host pipeline and the mapped path copy NP entries per element."""
    mesh, c = make_inputs(api.TET, api.POISSON, api.QUAD_TET4, 0, n=3000, seed=52)
    ref = None
    for dev in ("cuda", "cpu"):
        X, C, _ = to_device_inputs(api.TET, mesh, c, api.FP32_MIXED, api.AOS, dev)
        if dev == "cpu" and pinned:
            X, C = X.pin_memory(), C.pin_memory()
        out = api.alloc_out(api.TET, 3000, api.FP32_MIXED, api.AOS, dev, pin=(dev == "cpu" and pinned), packed=True)
        A, b, f = ctx.integrate(api.TET, X, C, api.POISSON, api.QUAD_TET4, api.PER_ELEMENT, api.FP32_MIXED, api.AOS,
                                api.AOS, out=out, packed=True)
        ctx.sync()
        got = (A.cpu().numpy(), b.cpu().numpy(), f.cpu().numpy())
        if ref is None:
            ref = got
        else:
            assert all(np.array_equal(x, y) for x, y in zip(ref, got))


def test_packed_tuned_shapes(ctx):
    mesh, c = make_inputs(api.PRISM, api.POISSON, api.QUAD_PRISM6, 1, n=3000, seed=53)
    X, C, _ = to_device_inputs(api.PRISM, mesh, c, api.FP32_MIXED, api.SOA)
    kw = dict(kind=api.POISSON, quad=api.QUAD_PRISM6, coef_mode=api.PER_QPOINT, prec=api.FP32_MIXED, layout=api.SOA,
              out_layout=api.SOA)
    Af, bf, _ = ctx.integrate(api.PRISM, X, C, **kw)
    ctx.sync()
    ref = _upper(Af.T.reshape(-1, 6, 6).cpu().numpy(), 6)
    for shape in [(64, 0), (128, 1), (256, 0)]:
        ctx.set_shape(shape[0], shape[1], api.PRISM, X, C, packed=True, **kw)
        Ap, bp, _ = ctx.integrate(api.PRISM, X, C, packed=True, **kw)
        ctx.sync()
        assert np.array_equal(Ap.T.cpu().numpy(), ref), shape


def test_packed_needs_the_laplace_kind(ctx):
    mesh, c = make_inputs(api.TET, api.GENERIC, api.QUAD_TET4, 0, n=100, seed=54)
    X, C, _ = to_device_inputs(api.TET, mesh, c, api.FP32_MIXED, api.AOS)
    with pytest.raises(api.FeError) as e:
        ctx.integrate(api.TET, X, C, api.GENERIC, api.QUAD_TET4, api.PER_ELEMENT, api.FP32_MIXED, api.AOS, api.AOS,
                      packed=True)
    assert e.value.status == -6
