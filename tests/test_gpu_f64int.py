"""The double multiplications and additions that the FP64 kernels run in integer
instructions, against the GPU's double-precision instructions, bit for bit
(fe_selftest_f64_int): random operands over the whole range, ties,
cancellations, every exponent difference, zeros, subnormals, infinities and
NaNs; and the FP64 tetrahedron arithmetic built on them against the same
arithmetic on the double pipe, on jittered, sliver, inverted and degenerate
elements with coefficients of many magnitudes (zeros included)."""
import ctypes

import numpy as np
import pytest
import torch

from paper_1504_01023_gb300 import api, build, meshgen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    build.build()
    return api.load()


def _run(lib, what, x, y, n, width):
    X = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()
    Y = torch.from_numpy(np.ascontiguousarray(y, dtype=np.float64)).cuda()
    oi = torch.empty(n * width, dtype=torch.float64, device="cuda")
    oh = torch.empty(n * width, dtype=torch.float64, device="cuda")
    st = lib.fe_selftest_f64_int(what, X.data_ptr(), Y.data_ptr(), n, oi.data_ptr(), oh.data_ptr(), None)
    assert st == 0, lib.fe_last_error(None)
    return oi.cpu().numpy().view(np.uint64), oh.cpu().numpy().view(np.uint64)


def _operands(rng, n):
    mant = rng.uniform(1.0, 2.0, n) * rng.choice([-1.0, 1.0], n)
    return mant * 2.0 ** rng.integers(-1075, 1024, n).astype(float)


def test_operations_bit_for_bit(lib):
    rng = np.random.default_rng(11)
    n = 1 << 22
    with np.errstate(all="ignore"):
        a = _operands(rng, n)
        b = _operands(rng, n)
        # a quarter of the pairs close in magnitude (cancellation, small exponent gaps)
        q = n // 4
        b[:q] = a[:q] * (1.0 + rng.uniform(-1e-3, 1e-3, q)) * rng.choice([-1.0, 1.0], q)
        # exponent gaps 0..70
        g = slice(q, 2 * q)
        b[g] = a[g] * rng.uniform(1.0, 2.0, q) * 2.0 ** -rng.integers(0, 71, q).astype(float)
        # short significands: exact products and sums with half-ulp tails (ties)
        t = slice(2 * q, 2 * q + q // 2)
        a[t] = rng.integers(1 << 26, 1 << 27, q // 2) * 2.0 ** rng.integers(-60, 60, q // 2).astype(float)
        b[t] = rng.integers(1 << 26, 1 << 27, q // 2) * 2.0 ** rng.integers(-60, 60, q // 2).astype(float)
    special = np.array([0.0, -0.0, 5e-324, -5e-324, 2.2250738585072014e-308, 1e-310, np.inf, -np.inf, np.nan,
                        1.7976931348623157e308, 1.0, -1.0, 0.5, 3.0])
    sa, sb = np.meshgrid(special, special)
    a = np.concatenate([a, sa.ravel()])
    b = np.concatenate([b, sb.ravel()])
    m = len(a)
    oi, oh = _run(lib, 0, a, b, m, 2)
    nan = np.isnan(oh.view(np.float64))
    assert np.array_equal(np.isnan(oi.view(np.float64)), nan)
    diff = np.flatnonzero((oi != oh) & ~nan)
    assert diff.size == 0, [(a[i % m], b[i % m], "mul" if i < m else "add") for i in diff[:5]]
    # the forms that report special cases (zeros handled in integer instructions)
    for what in (3, 4):
        oi, oh = _run(lib, what, a, b, m, 1)
        nan = np.isnan(oh.view(np.float64))
        assert np.array_equal(np.isnan(oi.view(np.float64)), nan)
        diff = np.flatnonzero((oi != oh) & ~nan)
        assert diff.size == 0, [(what, a[i], b[i]) for i in diff[:5]]


def _tets(seed):
    rng = np.random.default_rng(seed)
    mesh = meshgen.tet_cube_mesh(30, seed=seed)               # 162,000 elements
    meshgen.make_slivers(mesh, 0.1, seed=seed + 1)
    mesh[::37] = mesh[::37][:, [0, 2, 1, 3]]                  # inverted
    mesh[5::101, 3] = mesh[5::101, 0]                         # degenerate
    n = len(mesh)
    # element sizes from 1e-6 to 1e6 times the mesh's
    mesh = (mesh - mesh[:, :1]) * 10.0 ** rng.uniform(-6, 6, (n, 1, 1)) + mesh[:, :1]
    c = meshgen.generic_coefs(n, 1, seed=seed + 2)
    c *= 10.0 ** rng.uniform(-8, 8, (n, 1))
    c[rng.random(c.shape) < 0.1] = 0.0                        # zero coefficients
    return mesh, c


def test_tetrahedron_arithmetic_bit_for_bit(lib):
    mesh, c = _tets(21)
    n = len(mesh)
    oi, oh = _run(lib, 1, mesh.reshape(n, 12), c, n, 20)
    assert np.array_equal(oi, oh)
    oi, oh = _run(lib, 2, mesh.reshape(n, 12), c[:, 16], n, 20)
    assert np.array_equal(oi, oh)


def test_selftest_rejects_bad_arguments(lib):
    assert lib.fe_selftest_f64_int(5, None, None, 1, None, None, None) == -1
    assert lib.fe_selftest_f64_int(0, None, None, -1, None, None, None) == -1
    assert lib.fe_selftest_f64_int(0, None, None, 0, None, None, None) == 0


@pytest.mark.parametrize("et,kind,quad,cpq,tpe", [
    (api.TET, api.GENERIC, api.QUAD_TET4, 0, 1), (api.TET, api.POISSON, api.QUAD_TET1, 0, 1),
    (api.PRISM, api.GENERIC, api.QUAD_PRISM6, 1, 1), (api.PRISM, api.GENERIC, api.QUAD_PRISM6, 1, 2),
    (api.PRISM, api.POISSON, api.QUAD_PRISM6, 1, 1), (api.PRISM, api.POISSON, api.QUAD_PRISM6, 1, 2)])
def test_special_operands_in_the_fp64_kernels(lib, et, kind, quad, cpq, tpe):
    """Coefficients that send the integer-instruction products of the FP64 kernels
    to their special cases (a subnormal operand, a product that underflows, signed
    zeros): those elements are redone on the double pipe, and every element still
    matches the oracle within the FP64 tolerance."""
    from helpers import TOL, make_inputs, run_oracle, to_device_inputs
    mesh, c = make_inputs(et, kind, quad, cpq, n=997 if et == api.TET else 611, seed=71)
    n = len(mesh)
    flat = c.reshape(n, -1)
    specials = [1e-310, -1e-310, 1e-307, -1e-307, 0.0, -0.0]
    for j, e in enumerate(range(0, n, 5)):
        flat[e, j % flat.shape[1]] = specials[j % len(specials)]
    X, C, c_used = to_device_inputs(et, mesh, c, api.FP64, api.AOS)
    kw = dict(kind=kind, quad=quad, coef_mode=api.PER_QPOINT if cpq else api.PER_ELEMENT, prec=api.FP64,
              layout=api.AOS, out_layout=api.AOS)
    with api.Context(0) as ctx:
        ctx.set_shape(32 * 2 // tpe, 0, et, X, C, tpe=tpe, **kw)
        A, b, _ = ctx.integrate(et, X, C, **kw)
        ctx.sync()
    ns = api.NS[et]
    An = A.double().cpu().numpy().reshape(n, ns, ns)
    bn = b.double().cpu().numpy().reshape(n, ns)
    Ar, br, _ = run_oracle(et, kind, quad, cpq, mesh, c_used)
    assert np.isfinite(An).all() and np.isfinite(bn).all()
    # relative per element, with an absolute floor far below the normal range for
    # the load vectors made of subnormal values alone (a Laplace kind whose d^0 is
    # one of the specials: its rounding there is coarser than 1e-12 in any order)
    for G, R in ((An.reshape(n, -1), Ar.reshape(n, -1)), (bn, br)):
        err = np.linalg.norm(G - R, axis=1)
        ref = np.linalg.norm(R, axis=1)
        bad = np.flatnonzero(err > TOL[api.FP64] * ref + 1e-300)
        assert bad.size == 0, (bad[:5], err[bad[:5]], ref[bad[:5]])
