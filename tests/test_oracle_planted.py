"""The pins must catch plausible mistakes: each case plants one mistake in a copy
of the oracle source (on the CPU), rebuilds it, and checks that the exact-rational
pins reject the result. The shipped oracle is never modified."""
import os
from fractions import Fraction as F

import numpy as np
import pytest

import oracle
from oracle import exact
from prism_quality_ref import prism_quality_per_point

SRC = os.path.join(os.path.dirname(oracle.__file__), "oracle.c")

# (description, text in oracle.c, replacement)
MUTATIONS = [
    ("transposed coefficient operand", "vol[iQ] * CC(iD, jD, iQ)", "vol[iQ] * CC(jD, iD, iQ)"),
    ("dropped load term d^3", "for (int iD = 0; iD <= ND; iD++) {\n                b[iS]",
     "for (int iD = 0; iD < ND; iD++) {\n                b[iS]"),
    ("wrong sign of a prism derivative", "dphi[k + 3][2] = 0.5 * lam[k];", "dphi[k + 3][2] = -0.5 * lam[k];"),
    ("transposed Jacobian inverse", "s = s + dphat[iS][m] * inv[m][i];", "s = s + dphat[iS][m] * inv[i][m];"),
    ("wrong TET4 weight", "wts[q] = 1.0 / 24.0;", "wts[q] = 1.0 / 20.0;"),
    ("signed instead of absolute det", "vol[iQ] = fabs(det) * wts[iQ];", "vol[iQ] = det * wts[iQ];"),
    ("swapped prism point coordinates", "pts[3 * q + 0] = tri[t][0];", "pts[3 * q + 0] = tri[t][1];"),
]


def _cases():
    rng = np.random.default_rng(99)
    tets, prisms = [], []
    for _ in range(4):
        while True:
            x = [[F(int(rng.integers(-8, 9)), int(rng.integers(1, 4))) for _ in range(3)] for _ in range(4)]
            v = exact._det3(exact._sub(x[1], x[0]), exact._sub(x[2], x[0]), exact._sub(x[3], x[0]))
            if v != 0:
                break
        C = [[F(int(rng.integers(-9, 10)), 2) for _ in range(4)] for _ in range(4)]
        D = [F(int(rng.integers(-9, 10)), 2) for _ in range(4)]
        tets.append((x, C, D))
    for _ in range(3):
        base = [[F(0), F(0), F(0)], [F(int(rng.integers(2, 5))), F(0), F(1, 4)], [F(1, 2), F(int(rng.integers(2, 5))), F(0)]]
        top = [[v[0], v[1], v[2] + F(3, 2)] for v in base]
        C = [[F(int(rng.integers(-9, 10)), 2) for _ in range(4)] for _ in range(4)]
        D = [F(int(rng.integers(-9, 10)), 2) for _ in range(4)]
        prisms.append((base + top, C, D))
    return tets, prisms


def _pins_pass(lib):
    tets, prisms = _cases()
    for elem, cases, rule in [(oracle.TET, tets, oracle.Q_TET4), (oracle.PRISM, prisms, oracle.Q_PRISM6)]:
        xs = np.array([[[float(v) for v in p] for p in x] for x, _, _ in cases])
        cs = np.array([[float(C[a][b]) for a in range(4) for b in range(4)] + [float(d) for d in D] for _, C, D in cases])
        A, b, _ = oracle.integrate(elem, oracle.GENERIC, rule, xs, cs, lib=lib)
        for e, (x, C, D) in enumerate(cases):
            if elem == oracle.TET:
                Ar, br = exact.tet_closed_form(x, C, D, "TET4")
            else:
                Ar, br = exact.element_by_rational_rule("prism", x, C, D)
            Ar = np.array([[float(v) for v in row] for row in Ar])
            br = np.array([float(v) for v in br])
            if np.linalg.norm(A[e] - Ar) > 1e-12 * np.linalg.norm(Ar) or np.linalg.norm(b[e] - br) > 1e-12 * np.linalg.norm(br):
                return False
    return True


def test_unmodified_oracle_passes():
    assert _pins_pass(oracle._load())


@pytest.mark.parametrize("desc,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_is_caught(tmp_path, desc, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor not unique/not found: {desc}"
    mutated = tmp_path / "oracle_mut.c"
    mutated.write_text(src.replace(old, new))
    lib = oracle.load_library(oracle.compile_source(str(mutated), str(tmp_path / "liboracle_mut.so")))
    assert not _pins_pass(lib), f"pins did not catch: {desc}"


# Mistakes in the coefficient function and in the shape quality, each against
# the pins of its own part (the closed forms of tests/test_oracle_pins.py).
MUTATIONS_AUX = [
    ("coefficient function: quadratic term of d^0 from the wrong slot (Laplace kind)",
     "P[40 + 16] * uq * uq", "P[40 + 17] * uq * uq", "coef_fn"),
    ("coefficient function: linear term squared (Laplace kind)",
     "P[20 + 16] * uq + P[40 + 16]", "P[20 + 16] * uq * uq + P[40 + 16]", "coef_fn"),
    ("prism quality: ideal height 1/2 instead of 1", "{0.0, 0.0, 0.5}};", "{0.0, 0.0, 1.0}};", "quality"),
    ("prism quality: maximum over the points instead of the minimum", "if (!(qq >= qmin)) qmin = qq;",
     "if (!(qq <= qmin) || qmin > 1e29f) qmin = qq;", "quality"),
]


def _coef_fn_pins_pass(lib):
    """Laplace-kind coefficient function against the closed forms of the quadratic
    and linear terms: a right prism with u = 0 below and 1 above (PRISM6 exact)."""
    tri = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]])
    h = 0.5
    prism = np.zeros((1, 6, 3))
    prism[0, :3, :2] = tri
    prism[0, 3:, :2] = tri
    prism[0, 3:, 2] = h
    u = np.array([[0.0, 0.0, 0.0, 1.0, 1.0, 1.0]])
    for slot, ref in ((2, [0.5 * h / 36] * 3 + [0.5 * h / 12] * 3), (1, [0.5 * h / 18] * 3 + [0.5 * h / 9] * 3)):
        P = np.zeros((3, 20))
        P[slot, 16] = 1.0
        cq = oracle.coefs_from_u(oracle.PRISM, oracle.POISSON, oracle.Q_PRISM6, u, P, lib=lib)
        _, b, _ = oracle.integrate(oracle.PRISM, oracle.POISSON, oracle.Q_PRISM6, prism, cq, coef_per_q=True)
        if np.abs(b[0] - np.array(ref)).max() > 1e-14:
            return False
    return True


def _quality_pins_pass(lib):
    """Prism quality against the affine closed form on right prisms of the unit-edge
    equilateral triangle, and against the minimum over the points of the per-point
    closed form on prisms with a tilted top (prism_quality_ref)."""
    s3 = np.sqrt(3.0)
    tri = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.5, s3 / 2, 0.0]])
    out = []
    for hgt in (0.25, 1.0, 3.0):
        x = np.concatenate([tri, tri + [0.0, 0.0, hgt]])[None]
        # det T = 4 |T_a| h / sqrt3 = h, ||T||_F^2 = 2 + h^2
        ref = 3.0 * hgt ** (2.0 / 3.0) / (2.0 + hgt ** 2)
        out.append(abs(oracle.quality(oracle.PRISM, x, lib=lib)[0] - ref) <= 1e-5 * ref)
    # top vertex 3 lifted by different amounts: the points differ
    x = np.repeat(np.concatenate([tri, tri + [0.0, 0.0, 1.0]])[None], 4, axis=0)
    x[:, 3, 2] += np.array([0.3, 0.8, 1.5, 2.5])
    ref = prism_quality_per_point(x).min(axis=0)
    q = oracle.quality(oracle.PRISM, x, lib=lib)
    out.append(bool(np.all(np.abs(q - ref) <= 5e-5 * ref)))
    return all(out)


def test_unmodified_oracle_passes_aux_pins():
    assert _coef_fn_pins_pass(oracle._load())
    assert _quality_pins_pass(oracle._load())


@pytest.mark.parametrize("desc,old,new,part", MUTATIONS_AUX, ids=[m[0] for m in MUTATIONS_AUX])
def test_planted_mistake_in_aux_part_is_caught(tmp_path, desc, old, new, part):
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor not unique/not found: {desc}"
    mutated = tmp_path / "oracle_mut.c"
    mutated.write_text(src.replace(old, new))
    lib = oracle.load_library(oracle.compile_source(str(mutated), str(tmp_path / "liboracle_mut.so")))
    check = _coef_fn_pins_pass if part == "coef_fn" else _quality_pins_pass
    assert not check(lib), f"pins did not catch: {desc}"
