"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Every check here is independent of the oracle's own code path: exact-rational
closed forms (``oracle/exact.py``), exact monomial integrals, invariants of the
weak form of Sec. 2.1 (Eq. weak_form) under the element integrals of Sec. 2.2
(Eqs. sm_local, lv_local), and a textbook mean-ratio formula. No GPU.
"""
from fractions import Fraction as F

import numpy as np
import pytest

import oracle
from oracle import exact
from paper_1504_01023_gb300 import meshgen
from prism_quality_ref import affine_prism_quality, prism_quality_per_point

TET, PRISM = oracle.TET, oracle.PRISM
POI, GEN = oracle.POISSON, oracle.GENERIC


def _rand_rational_tet(rng):
    while True:
        x = [[F(int(rng.integers(-8, 9)), int(rng.integers(1, 5))) for _ in range(3)] for _ in range(4)]
        v = exact._det3(exact._sub(x[1], x[0]), exact._sub(x[2], x[0]), exact._sub(x[3], x[0]))
        if v > 0:
            return x


def _rand_rational_coefs(rng, symmetric=False):
    C = [[F(int(rng.integers(-9, 10)), int(rng.integers(1, 4))) for _ in range(4)] for _ in range(4)]
    if symmetric:
        C = [[C[min(a, b)][max(a, b)] for b in range(4)] for a in range(4)]
    D = [F(int(rng.integers(-9, 10)), int(rng.integers(1, 4))) for _ in range(4)]
    return C, D


def _to_np(x):
    return np.array([[float(v) for v in row] for row in x])


def _coef_vec(C, D):
    return np.array([float(C[a][b]) for a in range(4) for b in range(4)] + [float(d) for d in D])


def _relerr(x, ref):
    x, ref = np.asarray(x, float), np.asarray(ref, float)
    return np.linalg.norm(x - ref) / max(np.linalg.norm(ref), 1e-300)


# ---------------------------------------------------------------------------
# Quadrature tables (Eq. quadrature): exactness up to the stated degree
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("rule,elem,deg", [
    (oracle.Q_TET1, "tet", 1), (oracle.Q_TET4, "tet", 2), (oracle.Q_PRISM6, "prism", 2),
])
def test_rules_integrate_monomials_exactly(rule, elem, deg):
    pts, wts = oracle.quad_rule(rule)
    for a in range(deg + 1):
        for b in range(deg + 1 - a):
            for c in range(deg + 1 - a - b):
                got = np.sum(wts * pts[:, 0] ** a * pts[:, 1] ** b * pts[:, 2] ** c)
                ref = float(exact.monomial_integral(elem, a, b, c))
                assert abs(got - ref) <= 1e-15 * max(1.0, abs(ref)), (a, b, c, got, ref)


def test_rules_stated_degree_is_sharp():
    # one degree higher than stated must fail somewhere (guards a wrong table that
    # happens to be "too good", e.g. a different rule than the one documented)
    pts, wts = oracle.quad_rule(oracle.Q_TET4)
    got = np.sum(wts * pts[:, 0] ** 3)
    assert abs(got - float(exact.monomial_integral("tet", 3, 0, 0))) > 1e-6
    pts, wts = oracle.quad_rule(oracle.Q_PRISM6)
    # PRISM6 is exact to degree 3 in zeta and degree 2 in (xi, eta)
    assert abs(np.sum(wts * pts[:, 2] ** 2) - float(exact.monomial_integral("prism", 0, 0, 2))) < 1e-15
    assert abs(np.sum(wts * pts[:, 2] ** 4) - float(exact.monomial_integral("prism", 0, 0, 4))) > 1e-3
    assert abs(np.sum(wts * pts[:, 0] ** 3) - float(exact.monomial_integral("prism", 3, 0, 0))) > 1e-4


@pytest.mark.parametrize("rule,elem,order", [(oracle.Q_TET_COLLAPSED, "tet", 6), (oracle.Q_PRISM_TENSOR, "prism", 6)])
def test_high_order_rules(rule, elem, order):
    pts, wts = oracle.quad_rule(rule, order)
    for a in range(6):
        for b in range(6 - a):
            for c in range(6 - a - b):
                got = np.sum(wts * pts[:, 0] ** a * pts[:, 1] ** b * pts[:, 2] ** c)
                ref = float(exact.monomial_integral(elem, a, b, c))
                assert abs(got - ref) <= 1e-14, (a, b, c)


def test_exact_rational_rules_are_exact():
    # the rational rules behind exact.element_by_rational_rule, against exact integrals
    pts, wts = exact._tet_rule_deg3()
    for a, b, c in [(0, 0, 0), (1, 0, 0), (1, 1, 1), (3, 0, 0), (0, 2, 1)]:
        assert sum(w * p[0] ** a * p[1] ** b * p[2] ** c for p, w in zip(pts, wts)) == exact.monomial_integral("tet", a, b, c)
    pts, wts = exact._prism_rule()
    for a, b, c in [(0, 0, 0), (3, 0, 0), (1, 2, 0), (2, 1, 4), (0, 0, 5)]:
        assert sum(w * p[0] ** a * p[1] ** b * p[2] ** c for p, w in zip(pts, wts)) == exact.monomial_integral("prism", a, b, c)


# ---------------------------------------------------------------------------
# Tetrahedra: exact closed forms
# ---------------------------------------------------------------------------
def test_two_exact_statements_agree():
    rng = np.random.default_rng(7)
    for _ in range(3):
        x = _rand_rational_tet(rng)
        C, D = _rand_rational_coefs(rng)
        A1, b1 = exact.tet_closed_form(x, C, D, "TET4")
        A2, b2 = exact.element_by_rational_rule("tet", x, C, D)
        assert A1 == A2 and b1 == b2


@pytest.mark.parametrize("rule,name", [(oracle.Q_TET4, "TET4"), (oracle.Q_TET1, "TET1")])
def test_tet_generic_matches_exact_closed_form(rule, name):
    rng = np.random.default_rng(11 + rule)
    xs, cs, refs = [], [], []
    for _ in range(20):
        x = _rand_rational_tet(rng)
        C, D = _rand_rational_coefs(rng)
        A, b = exact.tet_closed_form(x, C, D, name)
        xs.append(_to_np(x))
        cs.append(_coef_vec(C, D))
        refs.append((_to_np(A), np.array([float(v) for v in b])))
    A, b, flags = oracle.integrate(TET, GEN, rule, np.stack(xs), np.stack(cs))
    assert not flags.any()
    for e, (Ar, br) in enumerate(refs):
        assert _relerr(A[e], Ar) < 1e-13
        assert _relerr(b[e], br) < 1e-13


def test_tet_poisson_matches_exact_closed_form():
    rng = np.random.default_rng(5)
    C = [[F(1) if (a == b and a > 0) else F(0) for b in range(4)] for a in range(4)]
    xs, d0s, refs = [], [], []
    for _ in range(10):
        x = _rand_rational_tet(rng)
        d0 = F(int(rng.integers(-5, 6)), 3)
        A, b = exact.tet_closed_form(x, C, [d0, F(0), F(0), F(0)], "TET4")
        xs.append(_to_np(x))
        d0s.append(float(d0))
        refs.append((_to_np(A), np.array([float(v) for v in b])))
    for rule in (oracle.Q_TET1, oracle.Q_TET4):
        A, b, _ = oracle.integrate(TET, POI, rule, np.stack(xs), np.array(d0s))
        for e, (Ar, br) in enumerate(refs):
            assert _relerr(A[e], Ar) < 1e-13
            assert _relerr(b[e], br) < 1e-13


def test_tet_mass_matrix_closed_form():
    """c^{0;0} = 1 only: A = |T|/20 (1 + delta_rs) and sum A = |T| (TET4)."""
    x = meshgen.tet_cube_mesh(3, seed=3)
    coefs = np.zeros((len(x), 20))
    coefs[:, 0] = 1.0
    A, b, _ = oracle.integrate(TET, GEN, oracle.Q_TET4, x, coefs)
    e1, e2, e3 = x[:, 1] - x[:, 0], x[:, 2] - x[:, 0], x[:, 3] - x[:, 0]
    vol = np.abs(np.einsum("ni,ni->n", e1, np.cross(e2, e3))) / 6.0
    ref = vol[:, None, None] * (np.ones((4, 4)) + np.eye(4))[None] / 20.0
    assert np.max(np.abs(A - ref) / vol[:, None, None]) < 1e-13
    assert np.max(np.abs(A.sum(axis=(1, 2)) - vol) / vol) < 1e-13


def test_tet_per_point_coefficients_equal_per_element_when_constant():
    x = meshgen.tet_cube_mesh(2, seed=4)
    c = meshgen.generic_coefs(len(x), 1, seed=4)
    A1, b1, _ = oracle.integrate(TET, GEN, oracle.Q_TET4, x, c)
    A2, b2, _ = oracle.integrate(TET, GEN, oracle.Q_TET4, x, np.repeat(c[:, None, :], 4, axis=1), coef_per_q=True)
    assert np.max(oracle.rel_frobenius(A1, A2)) < 1e-14
    assert np.max(oracle.rel_frobenius(b1, b2)) < 1e-14


# ---------------------------------------------------------------------------
# Prisms
# ---------------------------------------------------------------------------
def _rational_prism(rng, affine):
    """Bottom triangle counter-clockwise, top = bottom + (0,0,height) (+ z noise if not affine)."""
    while True:
        base = [[F(int(rng.integers(-6, 7)), 2), F(int(rng.integers(-6, 7)), 2), F(int(rng.integers(-2, 3)), 4)]
                for _ in range(3)]
        e1, e2 = exact._sub(base[1], base[0]), exact._sub(base[2], base[0])
        if e1[0] * e2[1] - e1[1] * e2[0] > 0:
            break
    hgt = F(int(rng.integers(2, 7)), 2)
    top = []
    for v in base:
        dz = F(0) if affine else F(int(rng.integers(-2, 3)), 8)
        top.append([v[0], v[1], v[2] + hgt + dz])
    return base + top


@pytest.mark.parametrize("symmetric", [False, True])
def test_affine_prism_matches_exact_rational(symmetric):
    rng = np.random.default_rng(21 + symmetric)
    xs, cs, refs = [], [], []
    for _ in range(6):
        x = _rational_prism(rng, affine=True)
        C, D = _rand_rational_coefs(rng, symmetric)
        A, b = exact.element_by_rational_rule("prism", x, C, D)
        xs.append(_to_np(x))
        cs.append(_coef_vec(C, D))
        refs.append((_to_np(A), np.array([float(v) for v in b])))
    A, b, _ = oracle.integrate(PRISM, GEN, oracle.Q_PRISM6, np.stack(xs), np.stack(cs))
    for e, (Ar, br) in enumerate(refs):
        assert _relerr(A[e], Ar) < 1e-13
        assert _relerr(b[e], br) < 1e-13
        if symmetric:
            assert np.max(np.abs(A[e] - A[e].T)) <= 1e-14 * np.max(np.abs(A[e]))


def test_nonaffine_prism_mass_and_convection_exact_with_high_order_rule():
    """Mass and convection integrands stay polynomial on a z-jittered prism, so the
    brute-force tensor rule must reproduce the exact rational values."""
    rng = np.random.default_rng(31)
    xs, cs, refs = [], [], []
    for _ in range(4):
        x = _rational_prism(rng, affine=False)
        C, D = _rand_rational_coefs(rng)
        for i in range(1, 4):
            for j in range(1, 4):
                C[i][j] = F(0)
        A, b = exact.element_by_rational_rule("prism", x, C, D, terms=("conv", "mass"))
        xs.append(_to_np(x))
        cs.append(_coef_vec(C, D))
        refs.append((_to_np(A), np.array([float(v) for v in b])))
    A, b, _ = oracle.integrate(PRISM, GEN, oracle.Q_PRISM_TENSOR, np.stack(xs), np.stack(cs), order=6)
    for e, (Ar, br) in enumerate(refs):
        assert _relerr(A[e], Ar) < 1e-13
        assert _relerr(b[e], br) < 1e-13


def test_prism_volume_exact():
    rng = np.random.default_rng(41)
    xs, vols = [], []
    for _ in range(5):
        x = _rational_prism(rng, affine=False)
        xs.append(_to_np(x))
        vols.append(float(exact.prism_volume(x)))
    coefs = np.zeros((5, 20))
    coefs[:, 0] = 1.0
    for rule, order in [(oracle.Q_PRISM6, 0), (oracle.Q_PRISM_TENSOR, 8)]:
        A, _, _ = oracle.integrate(PRISM, GEN, rule, np.stack(xs), coefs, order=order)
        assert np.max(np.abs(A.sum(axis=(1, 2)) - vols) / np.array(vols)) < 1e-14


def test_jittered_prism_diffusion_brute_force():
    """On z-jittered prisms the stiffness integrand is rational; the tensor rule must
    converge (orders 10 and 14 agree) and PRISM6 must be within quadrature error of it."""
    x = meshgen.prism_slab_mesh(4, seed=5)[:12]
    c = meshgen.generic_coefs(len(x), 1, seed=6)
    A10, _, _ = oracle.integrate(PRISM, GEN, oracle.Q_PRISM_TENSOR, x, c, order=10)
    A14, _, _ = oracle.integrate(PRISM, GEN, oracle.Q_PRISM_TENSOR, x, c, order=14)
    A6, _, _ = oracle.integrate(PRISM, GEN, oracle.Q_PRISM6, x, c)
    assert np.max(oracle.rel_frobenius(A10, A14)) < 1e-13
    err6 = np.max(oracle.rel_frobenius(A6, A14))
    assert err6 < 1e-2                        # O(jitter^2) quadrature error, jitter = 0.1 h
    # an unjittered slab is affine: PRISM6 is then exact
    xa = meshgen.prism_slab_mesh(4, zjitter=0.0, seed=5)[:12]
    A6a, _, _ = oracle.integrate(PRISM, GEN, oracle.Q_PRISM6, xa, c)
    A14a, _, _ = oracle.integrate(PRISM, GEN, oracle.Q_PRISM_TENSOR, xa, c, order=14)
    assert np.max(oracle.rel_frobenius(A6a, A14a)) < 1e-13


def test_tet_against_collapsed_brute_force():
    x = meshgen.tet_cube_mesh(2, seed=8)[:10]
    c = meshgen.generic_coefs(len(x), 1, seed=8)
    A4, b4, _ = oracle.integrate(TET, GEN, oracle.Q_TET4, x, c)
    Ah, bh, _ = oracle.integrate(TET, GEN, oracle.Q_TET_COLLAPSED, x, c, order=5)
    assert np.max(oracle.rel_frobenius(A4, Ah)) < 1e-13
    assert np.max(oracle.rel_frobenius(b4, bh)) < 1e-13


# ---------------------------------------------------------------------------
# Invariants (any element, any rule)
# ---------------------------------------------------------------------------
def _meshes():
    return [(TET, oracle.Q_TET4, meshgen.tet_cube_mesh(3, seed=12)[:60]),
            (TET, oracle.Q_TET1, meshgen.tet_cube_mesh(3, seed=13)[:60]),
            (PRISM, oracle.Q_PRISM6, meshgen.prism_slab_mesh(6, seed=14)[:60])]


@pytest.mark.parametrize("case", range(3))
def test_laplace_row_and_column_sums_vanish(case):
    et, rule, x = _meshes()[case]
    A, _, _ = oracle.integrate(et, POI, rule, x, np.ones(len(x)))
    scale = np.abs(A).max(axis=(1, 2))
    assert np.max(np.abs(A.sum(axis=2)) / scale[:, None]) < 1e-13
    assert np.max(np.abs(A.sum(axis=1)) / scale[:, None]) < 1e-13


@pytest.mark.parametrize("case", range(3))
def test_symmetric_coefficients_give_symmetric_matrix(case):
    et, rule, x = _meshes()[case]
    c = meshgen.generic_coefs(len(x), 1, seed=15)
    C = c[:, :16].reshape(-1, 4, 4)
    C = 0.5 * (C + C.transpose(0, 2, 1))
    c[:, :16] = C.reshape(-1, 16)
    A, _, _ = oracle.integrate(et, GEN, rule, x, c)
    assert np.max(np.abs(A - A.transpose(0, 2, 1)) / np.abs(A).max(axis=(1, 2))[:, None, None]) < 1e-14
    # and a non-symmetric c^{i;0} != c^{0;i} must break it
    c2 = c.copy()
    c2[:, 4] += 1.0
    A2, _, _ = oracle.integrate(et, GEN, rule, x, c2)
    assert np.max(np.abs(A2 - A2.transpose(0, 2, 1))) > 1e-6


def _rotation(rng):
    q, r = np.linalg.qr(rng.standard_normal((3, 3)))
    q = q * np.sign(np.diag(r))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


@pytest.mark.parametrize("case", range(3))
def test_rigid_motion_invariance(case):
    et, rule, x = _meshes()[case]
    rng = np.random.default_rng(16)
    c = meshgen.generic_coefs(len(x), 1, seed=17)
    A, b, _ = oracle.integrate(et, GEN, rule, x, c)
    # translation: unchanged for any coefficients
    At, bt, _ = oracle.integrate(et, GEN, rule, x + np.array([0.3, -0.7, 1.1]), c)
    assert np.max(oracle.rel_frobenius(At, A)) < 1e-12 and np.max(oracle.rel_frobenius(bt, b)) < 1e-12
    # rotation with the coefficients transformed as tensors and vectors
    R = _rotation(rng)
    xr = x @ R.T
    C = c[:, :16].reshape(-1, 4, 4).copy()
    D = c[:, 16:].copy()
    Cr = C.copy()
    Cr[:, 1:, 1:] = R @ C[:, 1:, 1:] @ R.T
    Cr[:, 1:, 0] = C[:, 1:, 0] @ R.T
    Cr[:, 0, 1:] = C[:, 0, 1:] @ R.T
    Dr = D.copy()
    Dr[:, 1:] = D[:, 1:] @ R.T
    cr = np.concatenate([Cr.reshape(-1, 16), Dr], axis=1)
    Ar, br, _ = oracle.integrate(et, GEN, rule, xr, cr)
    assert np.max(oracle.rel_frobenius(Ar, A)) < 1e-12 and np.max(oracle.rel_frobenius(br, b)) < 1e-12


@pytest.mark.parametrize("case", range(3))
def test_scaling_powers(case):
    """x -> s x: Laplace stiffness scales by s, convection by s^2, mass by s^3."""
    et, rule, x = _meshes()[case]
    s = 2.5
    base = np.zeros((len(x), 20))
    diff, conv, mass = base.copy(), base.copy(), base.copy()
    diff[:, [5, 10, 15]] = 1.0
    conv[:, [1, 4, 8]] = [0.3, -0.2, 0.5]
    mass[:, 0] = 1.0
    for cf, p in [(diff, 1), (conv, 2), (mass, 3)]:
        A1, _, _ = oracle.integrate(et, GEN, rule, x, cf)
        A2, _, _ = oracle.integrate(et, GEN, rule, s * x, cf)
        assert np.max(oracle.rel_frobenius(A2, s ** p * A1)) < 1e-13


@pytest.mark.parametrize("case", range(3))
def test_linear_field_consistency(case):
    """With only c^{i;j}: sum_s A_rs u(x_s) = b_r for u = a.x + beta, when
    d^i = c^{ij} a_j and d^0 = 0 (both bases reproduce linear fields)."""
    et, rule, x = _meshes()[case]
    c = meshgen.generic_coefs(len(x), 1, seed=18)
    C = c[:, :16].reshape(-1, 4, 4)
    C[:, 0, :] = 0.0
    C[:, :, 0] = 0.0
    a = np.array([0.7, -1.3, 0.4])
    c2 = np.concatenate([C.reshape(-1, 16), np.zeros((len(x), 4))], axis=1)
    c2[:, 17:20] = np.einsum("nij,j->ni", C[:, 1:, 1:], a)
    A, b, _ = oracle.integrate(et, GEN, rule, x, c2)
    u = x @ a + 0.25
    lhs = np.einsum("nrs,ns->nr", A, u)
    assert np.max(np.abs(lhs - b) / np.abs(A).max(axis=(1, 2))[:, None]) < 1e-12


# ---------------------------------------------------------------------------
# Orientation and degenerate elements
# ---------------------------------------------------------------------------
def test_inverted_and_degenerate_elements():
    x = meshgen.tet_cube_mesh(1, jitter=0.0, seed=1)[:2].copy()
    c = meshgen.generic_coefs(2, 1, seed=2)
    A, b, f = oracle.integrate(TET, GEN, oracle.Q_TET4, x, c)
    assert not f.any()
    # swapping vertices 1 and 2 inverts the element: same matrix up to the permutation
    xi = x[:, [0, 2, 1, 3], :]
    Ai, bi, fi = oracle.integrate(TET, GEN, oracle.Q_TET4, xi, c)
    assert (fi == 2).all()
    perm = [0, 2, 1, 3]
    assert np.max(oracle.rel_frobenius(Ai, A[:, perm][:, :, perm])) < 1e-14
    assert np.max(oracle.rel_frobenius(bi, b[:, perm])) < 1e-14
    # a flat element: zeros and bit 2
    xd = x.copy()
    xd[:, 3] = xd[:, 0] + 0.5 * (xd[:, 1] - xd[:, 0]) + 0.5 * (xd[:, 2] - xd[:, 0])
    xd[:, :, 2] = 0.0
    Ad, bd, fd = oracle.integrate(TET, GEN, oracle.Q_TET4, xd, c)
    assert (fd == 4).all() and not Ad.any() and not bd.any()


# ---------------------------------------------------------------------------
# Shape quality (single precision, not in the paper)
# ---------------------------------------------------------------------------
def _liu_joe(x):
    """Mean ratio of a tetrahedron by the edge-length formula 12 (3V)^{2/3} / sum l^2."""
    e1, e2, e3 = x[:, 1] - x[:, 0], x[:, 2] - x[:, 0], x[:, 3] - x[:, 0]
    v = np.abs(np.einsum("ni,ni->n", e1, np.cross(e2, e3))) / 6.0
    l2 = sum(np.sum((x[:, i] - x[:, j]) ** 2, axis=1) for i in range(4) for j in range(i + 1, 4))
    return 12.0 * (3.0 * v) ** (2.0 / 3.0) / l2


def test_tet_quality_matches_edge_length_formula():
    x = meshgen.tet_cube_mesh(4, seed=9)
    xs = x.copy()
    meshgen.make_slivers(xs, 0.3, seed=10)
    for arr in (x, xs):
        q = oracle.quality(TET, arr)
        ref = _liu_joe(arr)
        assert np.max(np.abs(q - ref) / ref) < 2e-5


def test_quality_ideal_elements_and_invariance():
    s3 = np.sqrt(3.0)
    eq = np.array([[[0, 0, 0], [1, 0, 0], [0.5, s3 / 2, 0], [0.5, s3 / 6, np.sqrt(2.0 / 3.0)]]])
    assert abs(oracle.quality(TET, eq)[0] - 1.0) < 1e-6
    pr = np.array([[[0, 0, 0], [1, 0, 0], [0.5, s3 / 2, 0], [0, 0, 1], [1, 0, 1], [0.5, s3 / 2, 1]]])
    assert abs(oracle.quality(PRISM, pr)[0] - 1.0) < 1e-6
    R = _rotation(np.random.default_rng(3))
    for et, x in [(TET, eq), (PRISM, pr)]:
        assert abs(oracle.quality(et, 3.7 * x @ R.T + 0.4)[0] - 1.0) < 1e-5
    # the unjittered Kuhn tetrahedron
    k = meshgen.tet_cube_mesh(1, jitter=0.0)[:1]
    assert abs(oracle.quality(TET, k)[0] - _liu_joe(k)[0]) < 1e-6


# ---------------------------------------------------------------------------
# Coefficients from a function of a nodal field (c_j(u_Q) = P0_j + P1_j u_Q + P2_j u_Q^2)
# ---------------------------------------------------------------------------
def test_coef_function_constant_field_is_per_element():
    """u constant over the element: every point sees the same coefficients
    P(u), so the element matrices equal those with per-element coefficients."""
    from paper_1504_01023_gb300 import meshgen
    rng = np.random.default_rng(71)
    P = rng.uniform(-1, 1, (3, 20))
    for et, rule, mesh in ((oracle.TET, oracle.Q_TET4, meshgen.tet_cube_mesh(3, seed=5)[:40]),
                           (oracle.PRISM, oracle.Q_PRISM6, meshgen.prism_slab_mesh(5, seed=6)[:40])):
        n, ns = len(mesh), mesh.shape[1]
        uv = rng.uniform(-2, 2, n)
        u = np.repeat(uv[:, None], ns, axis=1)
        cq = oracle.coefs_from_u(et, oracle.GENERIC, rule, u, P)
        ce = P[0][None, :] + P[1][None, :] * uv[:, None] + P[2][None, :] * uv[:, None] ** 2
        Aq, bq, _ = oracle.integrate(et, oracle.GENERIC, rule, mesh, cq, coef_per_q=True)
        Ae, be, _ = oracle.integrate(et, oracle.GENERIC, rule, mesh, ce)
        assert np.abs(Aq - Ae).max() <= 1e-12 * np.abs(Ae).max()
        assert np.abs(bq - be).max() <= 1e-12 * np.abs(be).max()


def test_coef_function_linear_field_load_tet():
    """d^0 = u_Q (P1_16 = 1, all else 0): b_r = int u phi_r = |T|/20 (sum u + u_r)
    for a linear field on a tetrahedron (TET4 is exact for this quadratic)."""
    from paper_1504_01023_gb300 import meshgen
    mesh = meshgen.tet_cube_mesh(3, seed=7)[:50]
    rng = np.random.default_rng(72)
    u = rng.uniform(-1, 1, (50, 4))
    P = np.zeros((3, 20))
    P[1, 16] = 1.0
    cq = oracle.coefs_from_u(oracle.TET, oracle.GENERIC, oracle.Q_TET4, u, P)
    A, b, _ = oracle.integrate(oracle.TET, oracle.GENERIC, oracle.Q_TET4, mesh, cq, coef_per_q=True)
    e = mesh[:, 1:] - mesh[:, :1]
    vol = np.abs(np.einsum("ei,ei->e", e[:, 0], np.cross(e[:, 1], e[:, 2]))) / 6.0
    ref = vol[:, None] / 20.0 * (u.sum(1, keepdims=True) + u)
    assert np.abs(A).max() == 0.0
    assert np.abs(b - ref).max() <= 1e-13 * np.abs(ref).max()


def test_coef_function_field_through_thickness_prism():
    """A right prism (triangle of area 1/2, height 0.3) with u = 0 on the bottom
    nodes and 1 on the top ones, d^0 = u_Q: b = |T_a| h / 18 at the bottom nodes
    and |T_a| h / 9 at the top ones (PRISM6 is exact here)."""
    tri = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]])
    h = 0.3
    mesh = np.zeros((1, 6, 3))
    mesh[0, :3, :2] = tri
    mesh[0, 3:, :2] = tri
    mesh[0, 3:, 2] = h
    u = np.array([[0.0, 0.0, 0.0, 1.0, 1.0, 1.0]])
    P = np.zeros((3, 20))
    P[1, 16] = 1.0
    cq = oracle.coefs_from_u(oracle.PRISM, oracle.POISSON, oracle.Q_PRISM6, u, P)
    A, b, _ = oracle.integrate(oracle.PRISM, oracle.POISSON, oracle.Q_PRISM6, mesh, cq, coef_per_q=True)
    ref = np.array([h * 0.5 / 18] * 3 + [h * 0.5 / 9] * 3)
    assert np.abs(b[0] - ref).max() <= 1e-15


def test_coef_function_quadratic_term_poisson_kind():
    """The quadratic term of the coefficient function in the Laplace kind
    (d^0 = u_Q^2, P2_16 = 1, all else 0), against closed forms:
    - a right prism (triangle area |T_a|, height h) with u = 0 on the bottom nodes
      and 1 on the top ones: u = t (t = z/h) and u^2 phi is cubic in t and linear
      in the triangle, which PRISM6 integrates exactly, so
      b_bottom = |T_a| h / 3 * int t^2 (1 - t) dt = |T_a| h / 36 and
      b_top = |T_a| h / 3 * int t^3 dt = |T_a| h / 12;
    - a tetrahedron with TET1, whose one point is the centroid, where u is the mean
      of the nodal values: b_r = |T| / 4 * mean(u)^2;
    - a tetrahedron with TET4 and a constant field c: b_r = |T| / 4 * c^2.
    The generic kind reads d^0 from the same slot and must give the same b."""
    tri = np.array([[0.0, 0.0], [0.8, 0.1], [0.2, 0.7]])
    area = 0.5 * abs((tri[1, 0] - tri[0, 0]) * (tri[2, 1] - tri[0, 1]) - (tri[1, 1] - tri[0, 1]) * (tri[2, 0] - tri[0, 0]))
    h = 0.4
    prism = np.zeros((1, 6, 3))
    prism[0, :3, :2] = tri
    prism[0, 3:, :2] = tri
    prism[0, 3:, 2] = h
    u = np.array([[0.0, 0.0, 0.0, 1.0, 1.0, 1.0]])
    P = np.zeros((3, 20))
    P[2, 16] = 1.0
    ref = np.array([area * h / 36] * 3 + [area * h / 12] * 3)
    for kind in (oracle.POISSON, oracle.GENERIC):
        cq = oracle.coefs_from_u(oracle.PRISM, kind, oracle.Q_PRISM6, u, P)
        A, b, _ = oracle.integrate(oracle.PRISM, kind, oracle.Q_PRISM6, prism, cq, coef_per_q=True)
        assert np.abs(b[0] - ref).max() <= 1e-15 * 8, (kind, b[0], ref)
        if kind == oracle.GENERIC:
            assert np.abs(A).max() == 0.0
    mesh = meshgen.tet_cube_mesh(2, seed=31)[:24]
    e = mesh[:, 1:] - mesh[:, :1]
    vol = np.abs(np.einsum("ei,ei->e", e[:, 0], np.cross(e[:, 1], e[:, 2]))) / 6.0
    rng = np.random.default_rng(32)
    uf = rng.uniform(-2, 2, (24, 4))
    uc = np.repeat(rng.uniform(-2, 2, (24, 1)), 4, axis=1)
    for rule, field, ubar in ((oracle.Q_TET1, uf, uf.mean(axis=1)), (oracle.Q_TET4, uc, uc[:, 0])):
        ref = np.repeat((vol * ubar ** 2 / 4)[:, None], 4, axis=1)
        for kind in (oracle.POISSON, oracle.GENERIC):
            cq = oracle.coefs_from_u(oracle.TET, kind, rule, field, P)
            _, b, _ = oracle.integrate(oracle.TET, kind, rule, mesh, cq, coef_per_q=True)
            assert np.abs(b - ref).max() <= 1e-14 * np.abs(ref).max(), (rule, kind)


def test_prism_quality_affine_closed_form():
    """oracle.quality on prisms whose top is a translate of the bottom (J constant):
    right and oblique, from flat to tall, rotated and moved; against the edge-length
    formula of prism_quality_ref (single precision on the oracle's side)."""
    rng = np.random.default_rng(41)
    n = 400
    base = rng.uniform(-1, 1, (n, 3, 3))
    base[:, :, 2] = 0.0
    normal = np.cross(base[:, 1] - base[:, 0], base[:, 2] - base[:, 0])
    normal /= np.linalg.norm(normal, axis=1, keepdims=True)
    height = 10.0 ** rng.uniform(-2.5, 0.5, n)
    shear = rng.uniform(-0.7, 0.7, (n, 3)) * height[:, None] * (rng.random((n, 1)) < 0.5)
    d = height[:, None] * normal + shear
    x = np.concatenate([base, base + d[:, None, :]], axis=1)
    R = _rotation(rng)
    x = x @ R.T + rng.uniform(-3, 3, 3)
    q = oracle.quality(PRISM, x)
    e1, e2 = x[:, 1] - x[:, 0], x[:, 2] - x[:, 0]
    ref = affine_prism_quality(e1, e2, x[:, 3] - x[:, 0])
    assert ref.min() < 0.05 and ref.max() > 0.5
    assert np.max(np.abs(q - ref) / ref) < 5e-5


def test_prism_quality_min_over_points_non_affine():
    """Prisms with independently jittered top nodes (J varies): the oracle's quality
    is the minimum over the six PRISM6 points of the mean ratio of J there. The test
    takes J at each point by central differences of the map and applies the affine
    closed form to the prism with the same Jacobian (prism_quality_ref)."""
    rng = np.random.default_rng(43)
    x = meshgen.prism_slab_mesh(12, seed=44).copy()
    n = len(x)
    x[:, 3:] += rng.uniform(-0.06, 0.06, (n, 3, 3))
    x = x - x[:, :1]
    per_point = prism_quality_per_point(x)
    ref = per_point.min(axis=0)
    assert np.mean(per_point.argmin(axis=0) != per_point.argmax(axis=0)) > 0.9   # the points differ
    q = oracle.quality(PRISM, x)
    assert np.max(np.abs(q - ref) / ref) < 5e-5
