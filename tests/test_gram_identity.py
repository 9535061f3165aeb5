"""The regrouping behind the Laplace prism kernels (prism_laplace_assemble):
sum over the six points of vol grad phi_m . grad phi_n equals a fixed
combination of per-level and per-point Gram terms of the rows of J^{-1}. Checked
here in numpy, in double precision, against the direct sum over the points of
the products of global gradients (J^{-T} times the reference gradients), on
random prisms. This tests the identity the kernels rely on; the kernels
themselves are tested against the oracle on the GPU."""
import numpy as np

S3 = 1.0 / np.sqrt(3.0)
ZB = [0.5 * (1 + S3), 0.5 * (1 - S3)]      # (1 - zeta)/2 at zeta = -1/sqrt3, +1/sqrt3
ZT = [0.5 * (1 - S3), 0.5 * (1 + S3)]


def lam(t, k):
    return 2.0 / 3.0 if t == k else 1.0 / 6.0


def direct(x):
    """sum_Q |det J| w grad phi_m . grad phi_n from reference gradients."""
    A = np.zeros((6, 6))
    dl = [(-1.0, -1.0), (1.0, 0.0), (0.0, 1.0)]
    for l in range(2):
        for t in range(3):
            d = np.zeros((6, 3))
            for k in range(3):
                d[k] = [dl[k][0] * ZB[l], dl[k][1] * ZB[l], -lam(t, k) / 2]
                d[k + 3] = [dl[k][0] * ZT[l], dl[k][1] * ZT[l], lam(t, k) / 2]
            J = x.T @ d
            G = d @ np.linalg.inv(J)
            A += abs(np.linalg.det(J)) / 6.0 * G @ G.T
    return A


def regrouped(x):
    r = x - x[0]
    ub, ut, vb, vt = r[1] - r[0], r[4] - r[3], r[2] - r[0], r[5] - r[3]
    w = [r[3] - r[0], r[4] - r[1], r[5] - r[2]]
    L = np.zeros((2, 3))
    v = np.zeros((2, 3, 2))
    c3 = np.zeros(3)
    for l in range(2):
        cx, cy = ZB[l] * ub + ZT[l] * ut, ZB[l] * vb + ZT[l] * vt
        a3 = np.cross(cx, cy)
        for t in range(3):
            h = [1 / 3 if t == k else 1 / 12 for k in range(3)]
            cz = h[0] * w[0] + h[1] * w[1] + h[2] * w[2]
            a1, a2 = np.cross(cy, cz), np.cross(cz, cx)
            sw = (1 / 6) / abs(cx @ a1)
            L[l] += sw * np.array([a1 @ a1, a1 @ a2, a2 @ a2])
            v[l, t] = sw * np.array([a1 @ a3, a2 @ a3])
            c3[t] += sw * (a3 @ a3)
    Pi = np.zeros((3, 3, 3))
    for kind in range(3):
        w0 = [ZB[0] ** 2, ZT[0] ** 2, ZB[0] * ZT[0]][kind]
        w1 = [ZB[1] ** 2, ZT[1] ** 2, ZB[1] * ZT[1]][kind]
        g = w0 * L[0] + w1 * L[1]
        P = np.array([[g[0] + 2 * g[1] + g[2], -(g[0] + g[1]), -(g[1] + g[2])],
                      [-(g[0] + g[1]), g[0], g[1]],
                      [-(g[1] + g[2]), g[1], g[2]]])
        Pi[kind] = P
    pi = np.zeros((2, 3, 3))
    for side in range(2):
        z0, z1 = (ZT[0], ZT[1]) if side else (ZB[0], ZB[1])
        V = z0 / 12 * v[0].sum(0) + z1 / 12 * v[1].sum(0)
        for b in range(3):
            n = V + z0 / 4 * v[0][b] + z1 / 4 * v[1][b]
            pi[side, :, b] = [-(n[0] + n[1]), n[0], n[1]]
    C = c3.sum() / 144
    H = np.array([[C + (15 / 144 if a == b else 3 / 144) * (c3[a] if a == b else c3[a] + c3[b])
                   for b in range(3)] for a in range(3)])
    A = np.zeros((6, 6))
    for m in range(6):
        for n in range(6):
            a, b, tm, tn = m % 3, n % 3, m >= 3, n >= 3
            p = Pi[(1 if tm else 0) if tm == tn else 2][a][b]
            x1, y1 = pi[1 if tm else 0][a][b], pi[1 if tn else 0][b][a]
            A[m, n] = p + (x1 if tn else -x1) + (y1 if tm else -y1) + (H[a][b] if tm == tn else -H[a][b])
    return A


def test_regrouping_equals_gradient_products():
    rng = np.random.default_rng(2024)
    for _ in range(200):
        base = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], float) + rng.uniform(-0.2, 0.2, (3, 3))
        top = base + np.array([0, 0, 1.0]) + rng.uniform(-0.3, 0.3, (3, 3))
        x = np.vstack([base, top]) * rng.uniform(0.1, 3) + rng.uniform(-5, 5, 3)
        Ad, Ag = direct(x), regrouped(x)
        assert np.linalg.norm(Ad - Ag) <= 1e-13 * np.linalg.norm(Ad)
        assert np.allclose(Ag, Ag.T, rtol=0, atol=1e-14 * np.abs(Ag).max())
