"""The regrouping behind the generic prism kernels (level_generic): the PRISM6 sum
of vol Phi_r^T C_q Phi_s (Phi_0s = phi_s, Phi_is = d phi_s / d x_i) equals a
fixed combination of per-level sums of the reference-space coefficient matrix
Gamma_q = vol_q B_q^T C_q B_q, B_q = diag(1, J^{-T}): the reference derivatives
of the prism's shape functions are the same at the three points of a level up to
lambda_k(t), so the 6 x 6 expansion happens once per level instead of once per
point. Checked here in numpy, in double precision, against the direct sum over
the points with global gradients (J^{-T} times the reference gradients), on
random prisms with per-point coefficients; the load vector likewise. This tests
the identity the kernels rely on; the kernels themselves are tested against the
oracle on the GPU."""
import numpy as np
import pytest

S3 = 1.0 / np.sqrt(3.0)
ZB = [0.5 * (1 + S3), 0.5 * (1 - S3)]      # (1 - zeta)/2 at zeta = -1/sqrt3, +1/sqrt3
ZT = [0.5 * (1 - S3), 0.5 * (1 + S3)]
W = 1.0 / 6.0                               # PRISM6 weight (reference volume 1)
DL = [(-1.0, -1.0), (1.0, 0.0), (0.0, 1.0)]  # (d lambda_k / d xi, d lambda_k / d eta)


def lam(t, k):
    return 2.0 / 3.0 if t == k else 1.0 / 6.0


def direct(x, C, d):
    """sum_Q |det J| w (Phi^T C_q Phi, Phi^T d_q), Phi from J^{-T} and the reference gradients.
    C: (6, 4, 4), d: (6, 4) per point q = 3 l + t."""
    A = np.zeros((6, 6))
    b = np.zeros(6)
    for l in range(2):
        for t in range(3):
            q = 3 * l + t
            dr = np.zeros((6, 3))
            ph = np.zeros(6)
            for k in range(3):
                dr[k] = [DL[k][0] * ZB[l], DL[k][1] * ZB[l], -lam(t, k) / 2]
                dr[k + 3] = [DL[k][0] * ZT[l], DL[k][1] * ZT[l], lam(t, k) / 2]
                ph[k], ph[k + 3] = lam(t, k) * ZB[l], lam(t, k) * ZT[l]
            J = x.T @ dr
            g = dr @ np.linalg.inv(J)           # rows: global gradients
            Phi = np.vstack([ph, g.T])          # 4 x 6
            vol = abs(np.linalg.det(J)) * W
            A += vol * Phi.T @ C[q] @ Phi
            b += vol * Phi.T @ d[q]
    return A, b


def level_sums(x, C, d, l):
    """The kernel's per-level steps: per point the cofactor rows a_i (J^{-1} = rows
    a_i / det), Gamma from the scaled coefficients, gathered into the per-level sums
    SF, SP, SQ, SG (3 x 3) and BU, BR (3) of zeta level l."""
    r = x - x[0]
    ub, ut, vb, vt = r[1] - r[0], r[4] - r[3], r[2] - r[0], r[5] - r[3]
    w = [r[3] - r[0], r[4] - r[1], r[5] - r[2]]
    wm = (w[0] + w[1] + w[2]) / 12.0
    D = np.array(DL)                             # D[k] = (D_k1, D_k2)
    zb, zt = ZB[l], ZT[l]
    cx, cy = zb * ub + zt * ut, zb * vb + zt * vt
    a3 = np.cross(cx, cy)
    SF, SP, SQ, SG = np.zeros((3, 3)), np.zeros((3, 3)), np.zeros((3, 3)), np.zeros((3, 3))
    S4 = np.zeros((2, 2))
    BU, BR = np.zeros(3), np.zeros(3)
    for t in range(3):
        q = 3 * l + t
        h = np.array([1 / 3 if t == k else 1 / 12 for k in range(3)])   # lambda_k(t) / 2
        cz = wm + 0.25 * w[t]
        a1, a2 = np.cross(cy, cz), np.cross(cz, cx)
        det = cx @ a1
        s2, s1, s0 = W / abs(det), np.copysign(W, det), W * abs(det)
        c = C[q]
        Ct = np.empty((4, 4))
        Ct[0, 0] = s0 * c[0, 0]
        Ct[0, 1:], Ct[1:, 0] = s1 * c[0, 1:], s1 * c[1:, 0]
        Ct[1:, 1:] = s2 * c[1:, 1:]
        dt0, dtv = s0 * d[q][0], s1 * d[q][1:]
        a = [None, a1, a2, a3]
        G = np.empty((4, 4))
        G[0, 0] = Ct[0, 0]
        for j in range(1, 4):
            Ca = Ct[1:, 1:] @ a[j]
            G[0, j] = Ct[0, 1:] @ a[j]
            G[j, 0] = a[j] @ Ct[1:, 0]
            for i in range(1, 4):
                G[i, j] = a[i] @ Ca
        xk = D @ G[0, 1:3]                   # x_k' = sum_j D_k'j Gamma_0j
        yk = D @ G[1:3, 0]                   # y_k = sum_i D_ki Gamma_i0
        e = 2 * h * G[0, 0] + xk
        SF += 2 * np.outer(h, e) + 2 * np.outer(yk, h)
        S4 += G[1:3, 1:3]
        p = 2 * h * G[0, 3] + D @ G[1:3, 3]
        qv = 2 * h * G[3, 0] + D @ G[3, 1:3]
        SP += np.outer(p, h)
        SQ += np.outer(h, qv)
        SG += np.outer(h, h) * G[3, 3]
        dl = np.array([dtv @ a1, dtv @ a2, dtv @ a3])
        BU += 2 * h * dt0 + D @ dl[:2]
        BR += h * dl[2]
    SF += D @ S4 @ D.T
    return SF, SP, SQ, SG, BU, BR


def regrouped(x, C, d):
    """One thread per element: per level the sums, then the level's share of the
    6 x 6 expansion into A and b."""
    A = np.zeros((6, 6))
    b = np.zeros(6)
    for l in range(2):
        zb, zt = ZB[l], ZT[l]
        SF, SP, SQ, SG, BU, BR = level_sums(x, C, d, l)
        for k in range(3):
            for kk in range(3):
                A[k, kk] += zb * (zb * SF[k, kk] - SP[k, kk] - SQ[k, kk]) + SG[k, kk]
                A[k, kk + 3] += zb * (zt * SF[k, kk] + SP[k, kk]) - zt * SQ[k, kk] - SG[k, kk]
                A[k + 3, kk] += zt * (zb * SF[k, kk] - SP[k, kk]) + zb * SQ[k, kk] - SG[k, kk]
                A[k + 3, kk + 3] += zt * (zt * SF[k, kk] + SP[k, kk] + SQ[k, kk]) + SG[k, kk]
            b[k] += zb * BU[k] - BR[k]
            b[k + 3] += zt * BU[k] + BR[k]
    return A, b


def regrouped_pair(x, C, d):
    """Two threads per element, one zeta level each: with zb = 1/2 + s c, zt = 1/2 - s c
    (c = 1/(2 sqrt 3), s = +1 on level 0 and -1 on level 1), so that zb^2 = 1/3 + s c,
    zt^2 = 1/3 - s c and zb zt = 1/6, each lane forms from its level's sums
      X = SF/3 + SG - s c (SP + SQ),  Y = s c SF - (SP + SQ)/2,
      U = SF/6 - SG + s c (SP + SQ),  V = (SP - SQ)/2,
      Bx = BU/2,  By = s c BU - BR,
    and the blocks of A are sums over the two levels of
      A_00 = X + Y,  A_11 = X - Y,  A_01 = U + V,  A_10 = U - V,
    and b_k = Bx + By, b_(k+3) = Bx - By. Lane 0 keeps X, Y (blocks 00, 11) and the
    bottom entries of b, lane 1 U, V (blocks 01, 10) and the top ones; each sends
    the other the two combinations it needs."""
    c = 0.5 / np.sqrt(3.0)
    parts = []
    for l in range(2):
        sg = 1.0 if l == 0 else -1.0
        SF, SP, SQ, SG, BU, BR = level_sums(x, C, d, l)
        Sp, Sm = SP + SQ, SP - SQ
        parts.append(dict(X=SF / 3 + SG - sg * c * Sp, Y=sg * c * SF - Sp / 2, U=SF / 6 - SG + sg * c * Sp,
                          V=Sm / 2, Bx=BU / 2, By=sg * c * BU - BR))
    X, Y, U, V, Bx, By = (parts[0][k] + parts[1][k] for k in ("X", "Y", "U", "V", "Bx", "By"))
    A = np.zeros((6, 6))
    A[:3, :3], A[3:, 3:], A[:3, 3:], A[3:, :3] = X + Y, X - Y, U + V, U - V
    return A, np.concatenate([Bx + By, Bx - By])


def _prism(rng, scale=1.0, shift=0.0):
    tri = np.array([[0.0, 0.0], [1.0, 0.0], [0.3, 0.9]]) + rng.uniform(-0.15, 0.15, (3, 2))
    x = np.zeros((6, 3))
    x[:3, :2] = tri
    x[3:, :2] = tri + rng.uniform(-0.2, 0.2, (3, 2))
    x[:3, 2] = rng.uniform(-0.1, 0.1, 3)
    x[3:, 2] = 1.0 + rng.uniform(-0.3, 0.3, 3)
    return scale * x + shift


@pytest.mark.parametrize("form", [regrouped, regrouped_pair])
@pytest.mark.parametrize("seed", range(6))
def test_regrouped_generic_prism_equals_direct_sum(seed, form):
    rng = np.random.default_rng(seed)
    x = _prism(rng, scale=rng.uniform(0.01, 10.0), shift=rng.uniform(-50, 50, 3))
    C = rng.uniform(-1, 1, (6, 4, 4))
    d = rng.uniform(-1, 1, (6, 4))
    A0, b0 = direct(x, C, d)
    A1, b1 = form(x, C, d)
    assert np.linalg.norm(A1 - A0) <= 1e-12 * np.linalg.norm(A0)
    assert np.linalg.norm(b1 - b0) <= 1e-12 * np.linalg.norm(b0)


@pytest.mark.parametrize("form", [regrouped, regrouped_pair])
def test_regrouped_inverted_prism(form):
    """Negative det J (top below the base): |det J| in vol, the sign in vol J^{-1}."""
    rng = np.random.default_rng(11)
    x = _prism(rng)
    x[3:, 2] = -x[3:, 2]
    C = rng.uniform(-1, 1, (6, 4, 4))
    d = rng.uniform(-1, 1, (6, 4))
    A0, b0 = direct(x, C, d)
    A1, b1 = form(x, C, d)
    assert np.linalg.norm(A1 - A0) <= 1e-12 * np.linalg.norm(A0)
    assert np.linalg.norm(b1 - b0) <= 1e-12 * np.linalg.norm(b0)


@pytest.mark.parametrize("form", [regrouped, regrouped_pair])
def test_each_coefficient_slot_separately(form):
    """One coefficient slot at a time (each of c^{00}, c^{0j}, c^{i0}, c^{ij}, d^a), so
    that a dropped or transposed term cannot hide behind the others."""
    rng = np.random.default_rng(5)
    x = _prism(rng)
    for a in range(4):
        for bb in range(4):
            C = np.zeros((6, 4, 4))
            C[:, a, bb] = rng.uniform(0.5, 1.5, 6)
            A0, _ = direct(x, C, np.zeros((6, 4)))
            A1, _ = form(x, C, np.zeros((6, 4)))
            assert np.linalg.norm(A1 - A0) <= 1e-12 * np.linalg.norm(A0), (a, bb)
        d = np.zeros((6, 4))
        d[:, a] = rng.uniform(0.5, 1.5, 6)
        _, b0 = direct(x, np.zeros((6, 4, 4)), d)
        _, b1 = form(x, np.zeros((6, 4, 4)), d)
        assert np.linalg.norm(b1 - b0) <= 1e-12 * np.linalg.norm(b0), a
