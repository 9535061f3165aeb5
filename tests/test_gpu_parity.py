"""Parity of the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances (relative Frobenius per element, A and b separately): 1e-12 for the
FP64 and double-word forms, 2e-5 for the mixed form. Inputs span several tiles
with a ragged tail.
"""
import itertools

import numpy as np
import pytest
import torch

import oracle
from helpers import TOL, make_inputs, max_errors, run_gpu, run_oracle
from paper_1504_01023_gb300 import api, meshgen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1504_01023_gb300 import build
    build.build()
    c = api.Context(0)
    yield c
    c.close()


PRECS = [api.FP64, api.FP32_MIXED, api.FP64_DW]
TET_CASES = list(itertools.product([api.POISSON, api.GENERIC], [api.QUAD_TET1, api.QUAD_TET4], [0, 1],
                                   PRECS, [api.SOA, api.AOS], [api.SOA, api.AOS]))
PRISM_CASES = list(itertools.product([api.POISSON, api.GENERIC], [api.QUAD_PRISM6], [0, 1],
                                     PRECS, [api.SOA, api.AOS], [api.SOA, api.AOS]))


def _ids(cases):
    return ["k%d-q%d-c%d-p%d-i%d-o%d" % c for c in cases]


@pytest.mark.parametrize("kind,quad,cpq,prec,lay,olay", TET_CASES, ids=_ids(TET_CASES))
def test_tet_parity(ctx, kind, quad, cpq, prec, lay, olay):
    mesh, c = make_inputs(api.TET, kind, quad, cpq, n=2999, seed=11)
    An, bn, fn, cu = run_gpu(ctx, api.TET, kind, quad, cpq, prec, lay, olay, mesh, c)
    Ar, br, fr = run_oracle(api.TET, kind, quad, cpq, mesh, cu)
    ea, eb = max_errors(An, bn, Ar, br)
    assert ea <= TOL[prec] and eb <= TOL[prec], (ea, eb)
    assert (fn == fr).all()      # no element here is poor, inverted or degenerate


@pytest.mark.parametrize("kind,quad,cpq,prec,lay,olay", PRISM_CASES, ids=_ids(PRISM_CASES))
def test_prism_parity(ctx, kind, quad, cpq, prec, lay, olay):
    mesh, c = make_inputs(api.PRISM, kind, quad, cpq, n=1999, seed=13)
    An, bn, fn, cu = run_gpu(ctx, api.PRISM, kind, quad, cpq, prec, lay, olay, mesh, c)
    Ar, br, fr = run_oracle(api.PRISM, kind, quad, cpq, mesh, cu)
    ea, eb = max_errors(An, bn, Ar, br)
    assert ea <= TOL[prec] and eb <= TOL[prec], (ea, eb)
    assert (fn == fr).all()


@pytest.mark.parametrize("prec", PRECS)
def test_thin_prisms_far_from_origin(ctx, prec):
    """h = 1e-3 elements at coordinates up to 1: the mixed form must form its edge
    vectors without the cancellation of rounding absolute coordinates."""
    full = meshgen.prism_slab_mesh(1000, seed=meshgen.SEED_BASE + 3, n_elem=1_999_000)
    mesh = full[-3001:].copy()        # elements near (1, 1)
    _, c = make_inputs(api.PRISM, api.GENERIC, api.QUAD_PRISM6, 1, mesh=mesh, seed=17)
    An, bn, fn, cu = run_gpu(ctx, api.PRISM, api.GENERIC, api.QUAD_PRISM6, 1, prec, api.SOA, api.SOA, mesh, c)
    Ar, br, _ = run_oracle(api.PRISM, api.GENERIC, api.QUAD_PRISM6, 1, mesh, cu)
    ea, eb = max_errors(An, bn, Ar, br)
    assert ea <= TOL[prec] and eb <= TOL[prec], (ea, eb)


@pytest.mark.parametrize("et", [api.TET, api.PRISM])
def test_small_and_ragged_sizes(ctx, et):
    quad = api.QUAD_TET4 if et == api.TET else api.QUAD_PRISM6
    for n in [1, 2, 31, 33, 255, 257, 513]:
        mesh, c = make_inputs(et, api.GENERIC, quad, 0, n=n, seed=n)
        for prec in PRECS:
            for lay, olay in [(api.SOA, api.SOA), (api.AOS, api.AOS)]:
                An, bn, fn, cu = run_gpu(ctx, et, api.GENERIC, quad, 0, prec, lay, olay, mesh, c)
                Ar, br, _ = run_oracle(et, api.GENERIC, quad, 0, mesh, cu)
                ea, eb = max_errors(An, bn, Ar, br)
                assert ea <= TOL[prec] and eb <= TOL[prec], (n, prec, lay, ea, eb)


def test_zero_elements(ctx):
    X = torch.empty((12, 0), dtype=torch.float64, device="cuda")
    C = torch.empty((20, 0), dtype=torch.float32, device="cuda")
    A, b, f = ctx.integrate(api.TET, X, C, api.GENERIC, api.QUAD_TET4)
    ctx.sync()
    assert A.numel() == 0


def test_inverted_and_degenerate_elements(ctx):
    mesh, c = make_inputs(api.TET, api.GENERIC, api.QUAD_TET4, 0, n=300, seed=3)
    mesh = mesh.copy()
    inv = np.arange(0, 300, 7)
    mesh[inv] = mesh[inv][:, [0, 2, 1, 3]]                 # inverted
    deg = np.arange(3, 300, 11)
    mesh[deg, 3] = mesh[deg, 0]                            # vertex 3 on vertex 0: zero volume
    for prec in PRECS:
        An, bn, fn, cu = run_gpu(ctx, api.TET, api.GENERIC, api.QUAD_TET4, 0, prec, api.SOA, api.SOA, mesh, c)
        Ar, br, fr = run_oracle(api.TET, api.GENERIC, api.QUAD_TET4, 0, mesh, cu)
        ea, eb = max_errors(An, bn, Ar, br)
        assert ea <= TOL[prec] and eb <= TOL[prec]
        assert ((fn & 6) == fr).all()                      # bits 1, 2 agree with the oracle
        assert (fn[deg] & 4).all() and not An[deg].any()
        if prec != api.FP64:
            assert (fn[deg] & 1).all()                     # degenerate -> double path


def test_nan_coordinates_do_not_fault(ctx):
    mesh, c = make_inputs(api.TET, api.GENERIC, api.QUAD_TET4, 0, n=200, seed=4)
    mesh = mesh.copy()
    mesh[5, 2, 1] = np.nan
    mesh[9, 0, 0] = np.inf
    for prec in PRECS:
        An, bn, fn, cu = run_gpu(ctx, api.TET, api.GENERIC, api.QUAD_TET4, 0, prec, api.SOA, api.SOA, mesh, c)
        ok = np.ones(200, bool)
        ok[[5, 9]] = False
        Ar, br, _ = run_oracle(api.TET, api.GENERIC, api.QUAD_TET4, 0, mesh[ok], cu[ok])
        ea, eb = max_errors(An[ok], bn[ok], Ar, br)
        assert ea <= TOL[prec] and eb <= TOL[prec]


@pytest.mark.parametrize("fraction", [0.01, 0.1])
def test_sliver_stress_mixed(ctx, fraction):
    """Poorly shaped elements (mean ratio < 0.1) take the double-precision Jacobian
    path; the flag decision is the float mean ratio, compared with the oracle's
    float quality away from the threshold."""
    mesh = meshgen.tet_cube_mesh(12, seed=meshgen.SEED_BASE + 2)
    sl = meshgen.make_slivers(mesh, fraction, seed=meshgen.SEED_BASE + 20)
    _, c = make_inputs(api.TET, api.GENERIC, api.QUAD_TET4, 0, mesh=mesh, seed=5)
    An, bn, fn, cu = run_gpu(ctx, api.TET, api.GENERIC, api.QUAD_TET4, 0, api.FP32_MIXED, api.SOA, api.SOA, mesh, c)
    Ar, br, _ = run_oracle(api.TET, api.GENERIC, api.QUAD_TET4, 0, mesh, cu)
    ea, eb = max_errors(An, bn, Ar, br)
    assert ea <= 2e-5 and eb <= 2e-5, (ea, eb)
    q = oracle.quality(oracle.TET, mesh, n_threads=8)
    flagged = (fn & 1).astype(bool)
    clear = np.abs(q - 0.1) > 1e-3 * 0.1
    assert (flagged[clear] == (q[clear] < 0.1)).all()
    assert flagged.sum() >= 0.5 * len(sl)


@pytest.mark.parametrize("pinned", [True, False])
@pytest.mark.parametrize("lay", [api.SOA, api.AOS])
def test_host_buffers_match_device_path(ctx, pinned, lay):
    """Host buffers: pinned ones are read and written in place (zero copy),
    pageable ones go through the chunked staging pipeline (n > one chunk)."""
    n = 2_200_000 if not pinned else 5000
    mesh = meshgen.tet_cube_mesh(72, seed=8)[:n]
    _, c = make_inputs(api.TET, api.GENERIC, api.QUAD_TET4, 0, mesh=mesh, seed=8)
    from helpers import to_device_inputs
    Xd, Cd, _ = to_device_inputs(api.TET, mesh, c, api.FP32_MIXED, lay)
    Xh, Ch = Xd.cpu(), Cd.cpu()
    if pinned:
        Xh, Ch = Xh.pin_memory(), Ch.pin_memory()
    rd = ctx.integrate(api.TET, Xd, Cd, api.GENERIC, api.QUAD_TET4, api.PER_ELEMENT, api.FP32_MIXED, lay, lay)
    ctx.sync()
    outh = api.alloc_out(api.TET, n, api.FP32_MIXED, lay, "cpu", True, pin=pinned)
    rh = ctx.integrate(api.TET, Xh, Ch, api.GENERIC, api.QUAD_TET4, api.PER_ELEMENT, api.FP32_MIXED, lay, lay, out=outh)
    for td, th in zip(rd, rh):
        assert torch.equal(td.cpu(), th)


def test_autotune_keeps_results(ctx):
    mesh, c = make_inputs(api.TET, api.GENERIC, api.QUAD_TET4, 0, n=20000, seed=9)
    from helpers import to_device_inputs, gpu_outputs_to_numpy
    X, C, cu = to_device_inputs(api.TET, mesh, c, api.FP32_MIXED, api.SOA)
    r0 = gpu_outputs_to_numpy(api.TET, *ctx.integrate(api.TET, X, C, api.GENERIC, api.QUAD_TET4), api.SOA)
    shape = ctx.tune(api.TET, X, C, api.GENERIC, api.QUAD_TET4)
    assert shape[0] in (64, 128, 256, 512)
    r1 = gpu_outputs_to_numpy(api.TET, *ctx.integrate(api.TET, X, C, api.GENERIC, api.QUAD_TET4), api.SOA)
    ctx.sync()
    assert np.array_equal(r0[0], r1[0]) and np.array_equal(r0[1], r1[1])


def test_profiling_records_kernel_time(ctx):
    mesh, c = make_inputs(api.TET, api.GENERIC, api.QUAD_TET4, 0, n=10000, seed=10)
    from helpers import to_device_inputs
    X, C, _ = to_device_inputs(api.TET, mesh, c, api.FP32_MIXED, api.SOA)
    ctx.set_profiling(True)
    n0 = api.launch_count()
    for _ in range(3):
        ctx.integrate(api.TET, X, C, api.GENERIC, api.QUAD_TET4)
    ms, k = ctx.kernel_time()
    ctx.set_profiling(False)
    assert k == 3 and ms > 0
    assert api.launch_count() - n0 == 6          # main + fix-up per call


def test_bounded_wait_times_out_and_context_survives(ctx):
    """A bulk-copy wait that can never complete gives up after its poll limit and
    reports FE_ERR_TIMEOUT; the context then integrates normally."""
    st = ctx.selftest_bounded_wait(1 << 14)
    assert st == -5
    mesh, c = make_inputs(api.TET, api.GENERIC, api.QUAD_TET4, 0, n=500, seed=21)
    An, bn, fn, cu = run_gpu(ctx, api.TET, api.GENERIC, api.QUAD_TET4, 0, api.FP32_MIXED, api.AOS, api.AOS, mesh, c)
    Ar, br, _ = run_oracle(api.TET, api.GENERIC, api.QUAD_TET4, 0, mesh, cu)
    ea, eb = max_errors(An, bn, Ar, br)
    assert ea <= TOL[api.FP32_MIXED] and eb <= TOL[api.FP32_MIXED]


def test_sliver_stress_double_word(ctx):
    """Double-word form: elements with mean ratio < 0.1 (flag bit 0) are computed in
    double; every element meets the double-precision tolerance."""
    mesh = meshgen.tet_cube_mesh(12, seed=meshgen.SEED_BASE + 2)
    sl = meshgen.make_slivers(mesh, 0.1, seed=meshgen.SEED_BASE + 21)
    for kind, quad in [(api.POISSON, api.QUAD_TET1), (api.GENERIC, api.QUAD_TET4)]:
        _, c = make_inputs(api.TET, kind, quad, 0, mesh=mesh, seed=6)
        An, bn, fn, cu = run_gpu(ctx, api.TET, kind, quad, 0, api.FP64_DW, api.AOS, api.AOS, mesh, c)
        Ar, br, fr = run_oracle(api.TET, kind, quad, 0, mesh, cu)
        ea, eb = max_errors(An, bn, Ar, br)
        assert ea <= 1e-12 and eb <= 1e-12, (kind, ea, eb)
        q = oracle.quality(oracle.TET, mesh, n_threads=8)
        flagged = (fn & 1).astype(bool)
        clear = np.abs(q - 0.1) > 1e-3 * 0.1
        assert (flagged[clear] == (q[clear] < 0.1)).all()
        assert flagged.sum() >= 0.5 * len(sl)
        assert ((fn & 6) == fr).all()


@pytest.mark.parametrize("et", [api.TET, api.PRISM])
def test_double_word_windows(ctx, et):
    """Elements outside the double-word window go to the double path (flag bit 0)
    and still meet the double-precision tolerance: coordinates scaled by 2^-30 and
    2^30 (|det J| outside [2^-60, 2^60]), all coefficients scaled by 1e-20 and
    1e20, one coefficient set to 1e-17 (below 2^-50); untouched elements stay in
    double-word (bit 0 clear). The scaling is about the origin: the oracle forms
    J from absolute coordinates, and for prisms (inexact reference derivatives)
    its rounding grows like |x| / h."""
    quad = api.QUAD_TET4 if et == api.TET else api.QUAD_PRISM6
    mesh, c = make_inputs(et, api.GENERIC, quad, 0, n=600, seed=41)
    mesh, c = mesh.copy(), c.copy()
    mesh[100:200] *= 2.0 ** -30
    mesh[200:300] *= 2.0 ** 30
    c[300:400] *= 1e-20
    c[400:500] *= 1e20
    c.reshape(600, -1)[500:600, 5] = 1e-17
    An, bn, fn, cu = run_gpu(ctx, et, api.GENERIC, quad, 0, api.FP64_DW, api.AOS, api.AOS, mesh, c)
    Ar, br, fr = run_oracle(et, api.GENERIC, quad, 0, mesh, cu)
    ea, eb = max_errors(An, bn, Ar, br)
    assert ea <= 1e-12 and eb <= 1e-12, (ea, eb)
    assert not (fn[:100] & 1).any()
    assert (fn[100:] & 1).all()
    assert ((fn & 6) == fr).all()


SOA_TMA_CASES = list(itertools.product([api.TET, api.PRISM], [api.POISSON, api.GENERIC], [0, 1], PRECS))


@pytest.mark.parametrize("et,kind,cpq,prec", SOA_TMA_CASES, ids=["t%d-k%d-c%d-p%d" % c for c in SOA_TMA_CASES])
def test_plane_major_tensor_copy_path(ctx, et, kind, cpq, prec):
    """n = 3000: every plane pitch is a 16-byte multiple, so plane-major tiles move
    as 2-D tensor copies (the n = 2999 cases above take the per-plane fallback);
    3000 = 46 x 64 + 56 leaves a ragged last tile (zero-filled loads, clipped stores)."""
    quad = api.QUAD_TET4 if et == api.TET else api.QUAD_PRISM6
    mesh, c = make_inputs(et, kind, quad, cpq, n=3000, seed=31)
    for shape in [(64, 0), (128, 1)]:
        from helpers import to_device_inputs, gpu_outputs_to_numpy
        X, C, cu = to_device_inputs(et, mesh, c, prec, api.SOA)
        cm = api.PER_QPOINT if cpq else api.PER_ELEMENT
        ctx.set_shape(shape[0], shape[1], et, X, C, kind, quad, cm, prec, api.SOA, api.SOA)
        A, b, f = ctx.integrate(et, X, C, kind, quad, cm, prec, api.SOA, api.SOA)
        ctx.sync()
        An, bn, fn = gpu_outputs_to_numpy(et, A, b, f, api.SOA)
        Ar, br, fr = run_oracle(et, kind, quad, cpq, mesh, cu)
        ea, eb = max_errors(An, bn, Ar, br)
        assert ea <= TOL[prec] and eb <= TOL[prec], (shape, ea, eb)
        assert (fn == fr).all()
