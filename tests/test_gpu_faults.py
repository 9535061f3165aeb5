"""Failure detection by host-side fault injection (fe_ctx_inject_fault): a
simulated allocation failure returns FE_ERR_OOM and leaves the context usable,
and a launch told to skip tiles writes nothing for them and makes fe_ctx_sync
report FE_ERR_PARTIAL. Nothing here faults, traps or hangs the GPU: the skipped
tiles are simply not processed, and no allocation is attempted for a failed one."""
import numpy as np
import pytest
import torch

from helpers import TOL, make_inputs, max_errors, run_oracle, to_device_inputs
from paper_1504_01023_gb300 import api, build, meshgen

pytestmark = pytest.mark.gpu


@pytest.fixture()
def ctx():
    build.build()
    c = api.Context(0)
    yield c
    c.close()


def _inputs(n, prec, seed=61):
    mesh, c = make_inputs(api.TET, api.GENERIC, api.QUAD_TET4, 0, seed=seed,
                          mesh=meshgen.tet_cube_mesh(30, seed=seed)[:n])
    X, C, c_used = to_device_inputs(api.TET, mesh, c, prec, api.AOS)
    return mesh, X, C, c_used


KW = dict(kind=api.GENERIC, quad=api.QUAD_TET4, coef_mode=api.PER_ELEMENT, layout=api.AOS, out_layout=api.AOS)


def test_injected_allocation_failure_then_recovery(ctx):
    """The first mixed-precision call of 100,000 elements must grow the fix-up list
    (the context starts with room for 1,024): with one injected failure it returns
    FE_ERR_OOM; the same call then succeeds and matches the oracle. A resident mesh
    fails and then registers the same way."""
    n = 100_000
    mesh, X, C, c_used = _inputs(n, api.FP32_MIXED)
    ctx.inject_fault(api.FAULT_ALLOC, count=1)
    with pytest.raises(api.FeError) as e:
        ctx.integrate(api.TET, X, C, prec=api.FP32_MIXED, **KW)
    assert e.value.status == -2 and "injected" in str(e.value)
    A, b, f = ctx.integrate(api.TET, X, C, prec=api.FP32_MIXED, **KW)
    ctx.sync()
    Ao, bo, _ = run_oracle(api.TET, api.GENERIC, api.QUAD_TET4, 0, mesh, c_used)
    ea, eb = max_errors(A.double().cpu().numpy(), b.double().cpu().numpy(), Ao, bo)
    assert ea <= TOL[api.FP32_MIXED] and eb <= TOL[api.FP32_MIXED]
    ctx.inject_fault(api.FAULT_ALLOC, count=1)
    with pytest.raises(api.FeError) as e:
        ctx.mesh_register(api.TET, X, api.AOS)
    assert e.value.status == -2
    mid = ctx.mesh_register(api.TET, X, api.AOS)
    ctx.mesh_release(mid)
    ctx.sync()


@pytest.mark.parametrize("prec", [api.FP32_MIXED, api.FP64])
def test_injected_tile_skip_reports_partial(ctx, prec):
    """One launch skipping every third tile of 128 elements: those elements keep the
    sentinel their outputs were filled with, every other element matches the oracle,
    and fe_ctx_sync reports FE_ERR_PARTIAL once; the next call is complete again."""
    n = 20_000
    mesh, X, C, c_used = _inputs(n, prec)
    dt = torch.float32 if prec == api.FP32_MIXED else torch.float64
    out = (torch.full((n, 4, 4), float("nan"), dtype=dt, device="cuda"),
           torch.full((n, 4), float("nan"), dtype=dt, device="cuda"),
           torch.full((n,), 255, dtype=torch.uint8, device="cuda"))
    ctx.set_shape(128, 0, api.TET, X, C, prec=prec, out=out, **KW)
    ctx.inject_fault(api.FAULT_SKIP_TILES, count=1, param=3)
    ctx.integrate(api.TET, X, C, prec=prec, out=out, **KW)
    with pytest.raises(api.FeError) as e:
        ctx.sync()
    assert e.value.status == -7
    A = out[0].double().cpu().numpy()
    b = out[1].double().cpu().numpy()
    f = out[2].cpu().numpy()
    tile = np.arange(n) // 128
    skipped = tile % 3 == 0
    assert np.isnan(A[skipped]).all() and np.isnan(b[skipped]).all() and (f[skipped] == 255).all()
    Ao, bo, _ = run_oracle(api.TET, api.GENERIC, api.QUAD_TET4, 0, mesh, c_used)
    ea, eb = max_errors(A[~skipped], b[~skipped], Ao[~skipped], bo[~skipped])
    assert ea <= TOL[prec] and eb <= TOL[prec]
    ctx.integrate(api.TET, X, C, prec=prec, out=out, **KW)
    ctx.sync()
    ea, eb = max_errors(out[0].double().cpu().numpy(), out[1].double().cpu().numpy(), Ao, bo)
    assert ea <= TOL[prec] and eb <= TOL[prec]


def test_inject_fault_rejects_bad_arguments(ctx):
    for kind, count, param in ((api.FAULT_SKIP_TILES, 1, 0), (api.FAULT_ALLOC, -1, 1), (9, 1, 1)):
        with pytest.raises(api.FeError) as e:
            ctx.inject_fault(kind, count, param)
        assert e.value.status == -1
    ctx.inject_fault(api.FAULT_ALLOC, count=5)
    ctx.inject_fault(api.FAULT_NONE)
    mesh, X, C, _ = _inputs(5000, api.FP32_MIXED)
    ctx.integrate(api.TET, X, C, prec=api.FP32_MIXED, **KW)
    ctx.sync()
