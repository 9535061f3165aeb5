"""The regrouping behind the FP64 and double-word generic tetrahedron kernels with
per-element coefficients (tet_generic_aug): every entry of A^e is one bilinear
form at_r M at_s^T of the augmented cofactor rows at_r = (a_r, 1), plus a
diagonal mass correction, and b^e is at_r . (sW d, e). Checked here in numpy, in
double precision, against the FP64 oracle (Algorithm 1 as written) on random
tetrahedra of both orientations, for both tetrahedral rules; and the reciprocal
the FP64 kernel uses (recip_scaled: a float reciprocal of the leading bits scaled
by the exponent, then one third-order Newton step), emulated bit for bit up to
the float reciprocal, against 1 / v. These test the identities the kernels rely
on; the kernels themselves are tested against the oracle on the GPU."""
import numpy as np
import pytest

import oracle
from paper_1504_01023_gb300 import meshgen

W = 1.0 / 6.0
M2 = {oracle.Q_TET1: (1.0 / 96.0, 1.0 / 96.0), oracle.Q_TET4: (2.0 / 120.0, 1.0 / 120.0)}   # (diagonal, off)


def augmented(x, c, rule):
    """A^e, b^e of one tetrahedron by the augmented bilinear form."""
    e = x[1:] - x[0]
    a = np.array([np.cross(e[1], e[2]), np.cross(e[2], e[0]), np.cross(e[0], e[1])])   # det J grad phi_1..3
    det = e[0] @ a[0]
    V, sg = abs(det), np.sign(det)
    C = c[:16].reshape(4, 4)
    d0, d = c[16], c[17:20]
    m2d, m2o = M2[rule]
    M = np.zeros((4, 4))
    M[:3, :3] = W / V * C[1:, 1:]
    M[:3, 3] = sg * W / 4 * C[1:, 0]        # c^{i;0}, with the test function's gradient
    M[3, :3] = sg * W / 4 * C[0, 1:]        # c^{0;j}, with the trial function's gradient
    M[3, 3] = V * C[0, 0] * m2o
    at = np.ones((4, 4))
    at[1:, :3] = a
    at[0, :3] = -a.sum(axis=0)
    A = at @ M @ at.T + np.eye(4) * V * C[0, 0] * (m2d - m2o)
    b = at @ np.concatenate([sg * W * d, [V * d0 * W / 4]])
    return A, b


@pytest.mark.parametrize("rule", [oracle.Q_TET1, oracle.Q_TET4])
def test_augmented_form_matches_oracle(rule):
    mesh = meshgen.tet_cube_mesh(3, seed=91)[:120].copy()
    meshgen.make_slivers(mesh, 0.2, seed=92)
    mesh[::3] = mesh[::3][:, [0, 2, 1, 3]]                                # a third inverted
    c = meshgen.generic_coefs(len(mesh), 1, seed=93)
    c[:, 1:4] *= np.random.default_rng(94).uniform(-3, 3, (len(mesh), 3))  # c^{0i} unlike c^{i0}
    Ao, bo, fo = oracle.integrate(oracle.TET, oracle.GENERIC, rule, mesh, c)
    assert (fo == 2).sum() == 40
    for k in range(len(mesh)):
        A, b = augmented(mesh[k], c[k], rule)
        assert np.linalg.norm(A - Ao[k]) <= 1e-13 * np.linalg.norm(Ao[k]), k
        assert np.linalg.norm(b - bo[k]) <= 1e-13 * np.linalg.norm(bo[k]), k


def recip_scaled(v, w):
    """The kernel's w / v: bits of v -> float in [1, 2) from its leading 24 bits,
    its float reciprocal (round to nearest), rescaled by v's exponent into a
    double, then y0 w (1 + e + e^2) with e = 1 - v y0 by fused multiply-adds
    (numpy has no fma: the products are formed exactly with float128 where
    available, else with the exact splitting below)."""
    bits = np.array([v], dtype=np.float64).view(np.uint64)[0]
    hw, lw = int(bits >> 32), int(bits & 0xFFFFFFFF)
    ev = (hw >> 20) & 0x7FF
    mb = 0x3F800000 | ((hw & 0xFFFFF) << 3) | (lw >> 29)
    m = np.array([mb], dtype=np.uint32).view(np.float32)[0]
    r = np.float32(1.0) / m                                               # correctly rounded in numpy
    rb = int(np.array([r], dtype=np.float32).view(np.uint32)[0])
    er = (rb >> 23) & 0xFF
    yh = ((er + 1919 - ev) << 20) | ((rb & 0x7FFFFF) >> 3)
    y0 = np.array([(yh << 32) | ((rb << 29) & 0xFFFFFFFF)], dtype=np.uint64).view(np.float64)[0]
    from fractions import Fraction as F
    # fused multiply-adds: exact rational arithmetic, one rounding each
    e = float(1 - F(v) * F(y0))
    wy0 = float(F(w) * F(y0))
    e2 = float(F(e) * F(e) + F(e))
    return float(F(wy0) * F(e2) + F(wy0))


def test_recip_scaled_within_an_ulp():
    rng = np.random.default_rng(95)
    vs = np.concatenate([10.0 ** rng.uniform(-299, 299, 400), rng.uniform(0.5, 4.0, 200),
                         [1.0, 2.0, 0.75, 1.0 - 2 ** -52, 1.0 + 2 ** -52, 1e-300, 2.0 ** -1000, 2.0 ** 1000]])
    for w in (1.0, 1.0 / 6.0):
        for v in vs:
            y = recip_scaled(float(v), w)
            ref = w / v
            assert abs(y - ref) <= 1.0 * np.spacing(ref), (v, w, y, ref)
