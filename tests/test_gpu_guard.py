"""Guard bands: output arrays sit inside larger buffers filled with a sentinel
byte pattern; after each launch the bytes before and after every output (and
the flags) must be unchanged. Ragged sizes (tiles not full), every element type,
precision form, input and output layout, packed output, two threads per prism
element and one row per lane (four threads per tetrahedron, six per prism)."""
import itertools

import numpy as np
import pytest
import torch

from helpers import make_inputs, to_device_inputs
from paper_1504_01023_gb300 import api

pytestmark = pytest.mark.gpu

GUARD = 4096                    # bytes of guard band on each side (a multiple of 16)
SENTINEL = 0xA5


@pytest.fixture(scope="module")
def ctx():
    from paper_1504_01023_gb300 import build
    build.build()
    c = api.Context(0)
    yield c
    c.close()


def _guarded(nbytes, dtype, shape):
    """A view of `shape` in the middle of a byte buffer with guard bands."""
    raw = torch.full((GUARD + nbytes + GUARD,), SENTINEL, dtype=torch.uint8, device="cuda")
    view = raw[GUARD:GUARD + nbytes].view(dtype).view(*shape)
    return raw, view


def _check_guards(raw, nbytes):
    head = raw[:GUARD].cpu().numpy()
    tail = raw[GUARD + nbytes:].cpu().numpy()
    assert (head == SENTINEL).all(), "write before the output"
    assert (tail == SENTINEL).all(), "write after the output"


def _outputs(et, n, prec, lay, packed):
    ns = api.NS[et]
    na = ns * (ns + 1) // 2 if packed else ns * ns
    dt = torch.float32 if prec == api.FP32_MIXED else torch.float64
    es = 4 if prec == api.FP32_MIXED else 8
    shapeA = (na, n) if lay == api.SOA else (n, na) if packed else (n, ns, ns)
    shapeB = (ns, n) if lay == api.SOA else (n, ns)
    rA, A = _guarded(n * na * es, dt, shapeA)
    rB, B = _guarded(n * ns * es, dt, shapeB)
    rF, F = _guarded(n, torch.uint8, (n,))
    return (rA, n * na * es), (rB, n * ns * es), (rF, n), (A, B, F)


CASES = ([(api.TET, k, q, p, il, ol, False) for k, q, p, il, ol in itertools.product(
            [api.POISSON, api.GENERIC], [api.QUAD_TET1, api.QUAD_TET4], [api.FP64, api.FP32_MIXED, api.FP64_DW],
            [api.SOA, api.AOS], [api.SOA, api.AOS])] +
         [(api.PRISM, k, api.QUAD_PRISM6, p, il, ol, False) for k, p, il, ol in itertools.product(
            [api.POISSON, api.GENERIC], [api.FP64, api.FP32_MIXED, api.FP64_DW], [api.SOA, api.AOS],
            [api.SOA, api.AOS])] +
         [(et, api.POISSON, q, p, api.AOS, ol, True) for (et, q), p, ol in itertools.product(
            [(api.TET, api.QUAD_TET1), (api.PRISM, api.QUAD_PRISM6)], [api.FP32_MIXED, api.FP64_DW],
            [api.SOA, api.AOS])])


@pytest.mark.parametrize("et,kind,quad,prec,il,ol,packed", CASES,
                         ids=["t%d-k%d-q%d-p%d-i%d-o%d-%s" % (c[:6] + ("pk" if c[6] else "full",)) for c in CASES])
def test_no_write_outside_outputs(ctx, et, kind, quad, prec, il, ol, packed):
    n = 997 if et == api.TET else 611                # ragged: no tile is full at the end
    cpq = 1 if et == api.PRISM else 0
    mesh, c = make_inputs(et, kind, quad, cpq, n=n, seed=61)
    X, C, _ = to_device_inputs(et, mesh, c, prec, il)
    ga, gb, gf, (A, B, F) = _outputs(et, n, prec, ol, packed)
    cm = api.PER_QPOINT if cpq else api.PER_ELEMENT
    ctx.integrate(et, X, C, kind, quad, cm, prec, il, ol, out=(A, B, F), packed=packed)
    ctx.sync()
    for raw, nbytes in (ga, gb, gf):
        _check_guards(raw, nbytes)
    assert torch.isfinite(A).all() and torch.isfinite(B).all()


@pytest.mark.parametrize("prec", [api.FP64, api.FP32_MIXED, api.FP64_DW])
def test_no_write_outside_outputs_two_threads_per_prism(ctx, prec):
    n = 611
    mesh, c = make_inputs(api.PRISM, api.GENERIC, api.QUAD_PRISM6, 1, n=n, seed=62)
    X, C, _ = to_device_inputs(api.PRISM, mesh, c, prec, api.AOS)
    ga, gb, gf, (A, B, F) = _outputs(api.PRISM, n, prec, api.AOS, False)
    kw = dict(kind=api.GENERIC, quad=api.QUAD_PRISM6, coef_mode=api.PER_QPOINT, prec=prec, layout=api.AOS,
              out_layout=api.AOS, out=(A, B, F))
    for block, pers in ((64, 0), (32, 1)):
        ctx.set_shape(block, pers, api.PRISM, X, C, tpe=2, **kw)
        ctx.integrate(api.PRISM, X, C, **kw)
        ctx.sync()
        for raw, nbytes in (ga, gb, gf):
            _check_guards(raw, nbytes)


@pytest.mark.parametrize("et,kind", [(api.TET, api.GENERIC), (api.TET, api.POISSON), (api.PRISM, api.GENERIC),
                                     (api.PRISM, api.POISSON)])
@pytest.mark.parametrize("prec", [api.FP64, api.FP32_MIXED, api.FP64_DW])
def test_no_write_outside_outputs_rows_per_lane(ctx, et, kind, prec):
    """Four threads per tetrahedron and six per prism (one row of A^e each; five
    groups per warp for prisms, two lanes idle): ragged tiles, persistent and not."""
    n = 997 if et == api.TET else 611
    quad = api.QUAD_TET4 if et == api.TET else api.QUAD_PRISM6
    cpq = 1 if et == api.PRISM else 0
    mesh, c = make_inputs(et, kind, quad, cpq, n=n, seed=63)
    X, C, _ = to_device_inputs(et, mesh, c, prec, api.AOS)
    ga, gb, gf, (A, B, F) = _outputs(et, n, prec, api.AOS, False)
    kw = dict(kind=kind, quad=quad, coef_mode=api.PER_QPOINT if cpq else api.PER_ELEMENT, prec=prec,
              layout=api.AOS, out_layout=api.AOS, out=(A, B, F))
    tpe = 4 if et == api.TET else 6
    epw = 32 // tpe
    for block, pers in ((8 * epw, 0), (2 * epw, 1), (4 * epw, 0)):
        ctx.set_shape(block, pers, et, X, C, tpe=tpe, **kw)
        ctx.integrate(et, X, C, **kw)
        ctx.sync()
        for raw, nbytes in (ga, gb, gf):
            _check_guards(raw, nbytes)
        assert torch.isfinite(A).all() and torch.isfinite(B).all()
