"""Exact-rational reference values used to pin the FP64 oracle (test infrastructure).

Nothing here calls the oracle or the CUDA library. Two independent statements of
the element integrals of Sec. 2.2 (Eqs. sm_local, lv_local), in exact rational
arithmetic (``fractions.Fraction``):

* ``tet_closed_form`` -- linear tetrahedron without any Jacobian inverse: the
  gradients of the barycentric functions come from the outward face-area vectors,
  grad(lambda_k) = -S_k / (3|T|); the integrals of products of barycentric
  functions are the textbook ones, int lambda_r = |T|/4 and
  int lambda_r lambda_s = |T| (1 + delta_rs) / 20 (for the 1-point rule the mass
  term is |T|/16 in every entry, what that rule gives).
* ``element_by_rational_rule`` -- any tetrahedron or prism, evaluated with
  rational-point rules that integrate the polynomial integrands exactly (Boole's
  rule on the line, the degree-3 seven-point triangle rule, and a collapsed-cube
  product of Boole rules on the tetrahedron), with the Jacobian inverse by
  Cramer's rule.
  Polynomial integrands are integrated exactly; this is exact for tetrahedra and
  for prisms whose Jacobian is constant (top face a translate of the bottom face),
  and for the mass and convection terms of any prism.
"""
from __future__ import annotations

from fractions import Fraction as F
from itertools import product


def _sub(a, b):
    return [a[i] - b[i] for i in range(3)]


def _cross(a, b):
    return [a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]]


def _dot(a, b):
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]


def _det3(c0, c1, c2):
    """Determinant of the matrix with columns c0, c1, c2."""
    return _dot(c0, _cross(c1, c2))


def tet_closed_form(x, C, D, rule: str = "TET4"):
    """Exact A (4x4) and b (4) of a linear tetrahedron with per-element coefficients.

    x: 4 vertices (3 Fractions each); C: 4x4 (C[a][b] = c^{a;b}); D: 4 (d^a).
    rule: "TET4" (exact integrals) or "TET1" (mass term as the centroid rule gives).
    """
    vol6 = _det3(_sub(x[1], x[0]), _sub(x[2], x[0]), _sub(x[3], x[0]))
    V = abs(vol6) / 6
    grads = []
    for k in range(4):
        a, b, c = [x[j] for j in range(4) if j != k]
        S = [v / 2 for v in _cross(_sub(b, a), _sub(c, a))]
        if _dot(S, _sub(x[k], a)) > 0:      # points toward vertex k: flip to outward
            S = [-v for v in S]
        grads.append([-v / (3 * V) for v in S])
    Cd = [[C[i][j] for j in range(1, 4)] for i in range(1, 4)]
    ci0 = [C[i][0] for i in range(1, 4)]
    c0i = [C[0][i] for i in range(1, 4)]
    A = [[F(0)] * 4 for _ in range(4)]
    b = [F(0)] * 4
    for r in range(4):
        for s in range(4):
            Cg = [_dot(Cd[i], grads[s]) for i in range(3)]
            diff = V * _dot(grads[r], Cg)
            conv = V / 4 * _dot(ci0, grads[r]) + V / 4 * _dot(c0i, grads[s])
            if rule == "TET4":
                mass = C[0][0] * V * (1 + (1 if r == s else 0)) / 20
            else:
                mass = C[0][0] * V / 16
            A[r][s] = diff + conv + mass
        b[r] = V * _dot([D[1], D[2], D[3]], grads[r]) + D[0] * V / 4
    return A, b


# ---------------------------------------------------------------------------
# Rational-point rules
# ---------------------------------------------------------------------------
def _boole():
    """5-point closed Newton-Cotes (Boole) rule on [-1,1], exact to degree 5."""
    pts = [F(-1), F(-1, 2), F(0), F(1, 2), F(1)]
    wts = [F(7 * 2, 90), F(32 * 2, 90), F(12 * 2, 90), F(32 * 2, 90), F(7 * 2, 90)]
    return pts, wts


def _triangle_deg3():
    """Seven-point rule on the unit right triangle (area 1/2), exact to degree 3:
    |T| (1/20 * vertices + 2/15 * edge midpoints + 9/20 * centroid)."""
    area = F(1, 2)
    verts = [(F(0), F(0)), (F(1), F(0)), (F(0), F(1))]
    mids = [(F(1, 2), F(0)), (F(1, 2), F(1, 2)), (F(0), F(1, 2))]
    cen = [(F(1, 3), F(1, 3))]
    pts = verts + mids + cen
    wts = [area * F(1, 20)] * 3 + [area * F(2, 15)] * 3 + [area * F(9, 20)]
    return pts, wts


def _tet_rule_deg3():
    """Rational rule exact to degree 3 on the unit tetrahedron: collapsed-cube
    tensor product of Boole rules mapped to [0,1] (xi = u, eta = v(1-u),
    zeta = t(1-u)(1-v), Jacobian (1-u)^2 (1-v); a degree-d integrand becomes
    degree d+2 in u, d+1 in v, d in t, and Boole is exact to degree 5)."""
    lp, lw = _boole()
    u01 = [(p + 1) / 2 for p in lp]
    w01 = [w / 2 for w in lw]
    pts, wts = [], []
    for (u, wu), (v, wv), (t, wt) in product(zip(u01, w01), zip(u01, w01), zip(u01, w01)):
        pts.append((u, v * (1 - u), t * (1 - u) * (1 - v)))
        wts.append(wu * wv * wt * (1 - u) * (1 - u) * (1 - v))
    return pts, wts


def _prism_rule():
    tp, tw = _triangle_deg3()
    lp, lw = _boole()
    pts, wts = [], []
    for (p, wp) in zip(tp, tw):
        for (z, wz) in zip(lp, lw):
            pts.append((p[0], p[1], z))
            wts.append(wp * wz)
    return pts, wts


def _tet_shape(xi):
    phi = [1 - xi[0] - xi[1] - xi[2], xi[0], xi[1], xi[2]]
    dphi = [[F(-1), F(-1), F(-1)], [F(1), F(0), F(0)], [F(0), F(1), F(0)], [F(0), F(0), F(1)]]
    return phi, dphi


def _prism_shape(xi):
    lam = [1 - xi[0] - xi[1], xi[0], xi[1]]
    dlam = [[F(-1), F(-1)], [F(1), F(0)], [F(0), F(1)]]
    zb, zt = (1 - xi[2]) / 2, (1 + xi[2]) / 2
    phi = [lam[k] * zb for k in range(3)] + [lam[k] * zt for k in range(3)]
    dphi = ([[dlam[k][0] * zb, dlam[k][1] * zb, -lam[k] / 2] for k in range(3)]
            + [[dlam[k][0] * zt, dlam[k][1] * zt, lam[k] / 2] for k in range(3)])
    return phi, dphi


def element_by_rational_rule(elem: str, x, C, D, terms=("diff", "conv", "mass")):
    """Exact A and b (lists of Fractions) by exact rational quadrature.

    elem: "tet" or "prism"; x: vertices; C 4x4, D 4 per element. ``terms`` selects
    which parts of A to include (the load vector is always complete). Exact when
    every selected integrand is a polynomial within the rule's degree.
    """
    if elem == "tet":
        pts, wts = _tet_rule_deg3()
        shape, ns = _tet_shape, 4
    else:
        pts, wts = _prism_rule()
        shape, ns = _prism_shape, 6
    A = [[F(0)] * ns for _ in range(ns)]
    b = [F(0)] * ns
    for xi, w in zip(pts, wts):
        phi, dphi = shape(xi)
        J = [[sum(x[k][i] * dphi[k][m] for k in range(ns)) for m in range(3)] for i in range(3)]
        cols = [[J[i][m] for i in range(3)] for m in range(3)]
        det = _det3(cols[0], cols[1], cols[2])
        # Cramer: rows of J^{-1} are cross products of columns over det
        inv_rows = [_cross(cols[1], cols[2]), _cross(cols[2], cols[0]), _cross(cols[0], cols[1])]
        inv = [[v / det for v in row] for row in inv_rows]          # inv[m][i] = (J^-1)_{mi}
        grad = [[sum(dphi[k][m] * inv[m][i] for m in range(3)) for i in range(3)] for k in range(ns)]
        vol = abs(det) * w
        Phi = [[phi[k]] + grad[k] for k in range(ns)]               # Phi[k][a]
        for r in range(ns):
            for s in range(ns):
                acc = F(0)
                for a in range(4):
                    for bb in range(4):
                        part = "mass" if (a == 0 and bb == 0) else ("diff" if (a > 0 and bb > 0) else "conv")
                        if part in terms:
                            acc += C[a][bb] * Phi[r][a] * Phi[s][bb]
                A[r][s] += vol * acc
            b[r] += vol * sum(D[a] * Phi[r][a] for a in range(4))
    return A, b


def prism_volume(x):
    """Exact volume of a prism element: det J is of degree 1 in (xi, eta) and 2 in
    zeta, integrated exactly by the rational rule."""
    pts, wts = _prism_rule()
    vol = F(0)
    for xi, w in zip(pts, wts):
        _, dphi = _prism_shape(xi)
        J = [[sum(x[k][i] * dphi[k][m] for k in range(6)) for m in range(3)] for i in range(3)]
        cols = [[J[i][m] for i in range(3)] for m in range(3)]
        vol += abs(_det3(cols[0], cols[1], cols[2])) * w
    return vol


def monomial_integral(elem: str, a: int, b: int, c: int):
    """Exact integral of xi^a eta^b zeta^c over the reference element."""
    from math import factorial
    if elem == "tet":
        return F(factorial(a) * factorial(b) * factorial(c), factorial(a + b + c + 3))
    tri = F(factorial(a) * factorial(b), factorial(a + b + 2))
    line = F(0) if c % 2 else F(2, c + 1)
    return tri * line
