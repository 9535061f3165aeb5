"""Mean ratio of prisms by formulas written for the tests (independent of the
oracle's Jacobian-based computation): an affine prism by its edge lengths and
volume, and a general prism as the minimum over the PRISM6 points of the affine
prism with the same Jacobian, the Jacobian taken by central differences of the
map."""
import numpy as np


def affine_prism_quality(e1, e2, d):
    """Mean ratio of an affine prism (bottom triangle with edge vectors e1, e2 from
    vertex 0, top = bottom + d); the ideal is the unit-edge equilateral triangle
    times unit height. T = J S^{-1} maps the triangle part by an affine M and the
    height direction to d, so
      det T = 2|T_a| (n . d) / (sqrt3 / 2) = 4 |T_a| (n . d) / sqrt3,
      ||T||_F^2 = ||M||_F^2 + |d|^2 = (2/3) (sum of the squared edge lengths) + |d|^2
    (the three edge vectors of the equilateral triangle have sum u u^T = 3/2 I), and
    q = 3 |det T|^{2/3} / ||T||_F^2."""
    c = np.cross(e1, e2)                      # 2 |T_a| n
    vol_term = 2.0 * np.abs(np.einsum("ni,ni->n", c, d)) / np.sqrt(3.0)
    l2 = np.sum(e1 ** 2, 1) + np.sum(e2 ** 2, 1) + np.sum((e2 - e1) ** 2, 1)
    return 3.0 * vol_term ** (2.0 / 3.0) / (2.0 / 3.0 * l2 + np.sum(d ** 2, 1))


def prism_map(x, xi, eta, zeta):
    """Point of the physical prism at reference coordinates: the bottom and top
    triangles interpolated linearly in (xi, eta), then linearly in zeta."""
    lam = np.array([1.0 - xi - eta, xi, eta])
    bot = np.einsum("k,nki->ni", lam, x[:, :3])
    top = np.einsum("k,nki->ni", lam, x[:, 3:])
    return 0.5 * (1.0 - zeta) * bot + 0.5 * (1.0 + zeta) * top


def prism_quality_per_point(x):
    """[6, E] mean ratios at the PRISM6 points (triangle points (1/6,1/6), (2/3,1/6),
    (1/6,2/3) at zeta = -+1/sqrt3): J by central differences (exact for this map,
    which is linear in each reference coordinate), then the affine prism with edges
    J_xi, J_eta and top offset 2 J_zeta."""
    pts = [(1 / 6, 1 / 6), (2 / 3, 1 / 6), (1 / 6, 2 / 3)]
    out = []
    hstep = 0.125
    for zeta in (-1 / np.sqrt(3.0), 1 / np.sqrt(3.0)):
        for xi, eta in pts:
            jx = (prism_map(x, xi + hstep, eta, zeta) - prism_map(x, xi - hstep, eta, zeta)) / (2 * hstep)
            jy = (prism_map(x, xi, eta + hstep, zeta) - prism_map(x, xi, eta - hstep, zeta)) / (2 * hstep)
            jz = (prism_map(x, xi, eta, zeta + hstep) - prism_map(x, xi, eta, zeta - hstep)) / (2 * hstep)
            out.append(affine_prism_quality(jx, jy, 2.0 * jz))
    return np.array(out)
