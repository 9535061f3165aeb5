"""The pins must catch plausible mistakes: each case plants one mistake in a copy
of the oracle source (on the CPU), rebuilds it, and checks that the exact-rational
pins reject the result. The shipped oracle is never modified."""
import os
from fractions import Fraction as F

import numpy as np
import pytest

import oracle
from oracle import exact

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
