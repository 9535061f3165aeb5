"""Error statistics of every precision form against the FP64 oracle, over every
element of mid-size seeded meshes: relative Frobenius error per element of A^e
and of b^e, its maximum and 99.9th percentile, split into elements that took the
double-precision path (flag bit 0) and elements that did not.

Each statistic must be within the form's tolerance. With FE_ERROR_REPORT set to a
file path, the statistics are also appended there, one JSON object per case."""
import json
import os

import numpy as np
import pytest
import torch

import oracle
from helpers import ORACLE_RULE, TOL
from paper_1504_01023_gb300 import api, meshgen

pytestmark = pytest.mark.gpu

PRECS = {"fp64": api.FP64, "mixed": api.FP32_MIXED, "double_word": api.FP64_DW}


@pytest.fixture(scope="module")
def ctx():
    from paper_1504_01023_gb300 import build
    build.build()
    c = api.Context(0)
    yield c
    c.close()


def _workload(name):
    """(element type, kind, rule, per-point coefficients, mesh, coefficients)."""
    if name == "poisson_tet1_48k":
        mesh = meshgen.tet_cube_mesh(20, 0.2, seed=meshgen.SEED_BASE + 1)
        return api.TET, api.POISSON, api.QUAD_TET1, 0, mesh, meshgen.poisson_coefs(len(mesh), 1, 1.0)
    if name.startswith("generic_tet4_384k"):
        mesh = meshgen.tet_cube_mesh(40, 0.2, seed=meshgen.SEED_BASE + 2)
        frac = {"generic_tet4_384k": 0.0, "generic_tet4_384k_slivers1": 0.01, "generic_tet4_384k_slivers10": 0.10}[name]
        if frac:
            meshgen.make_slivers(mesh, frac, seed=meshgen.SEED_BASE + 20)
        return api.TET, api.GENERIC, api.QUAD_TET4, 0, mesh, meshgen.generic_coefs(len(mesh), 1,
                                                                                    seed=meshgen.SEED_BASE + 2)
    if name == "generic_prism6_180k":
        mesh = meshgen.prism_slab_mesh(300, None, 0.1, seed=meshgen.SEED_BASE + 3)
        return api.PRISM, api.GENERIC, api.QUAD_PRISM6, 1, mesh, meshgen.generic_coefs(len(mesh), 6,
                                                                                        seed=meshgen.SEED_BASE + 3)
    raise KeyError(name)


def _stats(err, sel):
    e = err[sel]
    if len(e) == 0:
        return {"n": 0, "max": None, "p99.9": None}
    return {"n": int(len(e)), "max": float(e.max()), "p99.9": float(np.quantile(e, 0.999))}


WORKLOADS = ["poisson_tet1_48k", "generic_tet4_384k", "generic_tet4_384k_slivers1", "generic_tet4_384k_slivers10",
             "generic_prism6_180k"]
CASES = [(w, p) for w in WORKLOADS for p in PRECS]


@pytest.mark.parametrize("wl,pname", CASES, ids=[f"{w}-{p}" for w, p in CASES])
def test_error_statistics(ctx, wl, pname):
    et, kind, quad, cpq, mesh, c = _workload(wl)
    prec = PRECS[pname]
    n = len(mesh)
    cdt = np.float32 if prec == api.FP32_MIXED else np.float64
    cu = c.astype(cdt)
    X = torch.from_numpy(np.ascontiguousarray(mesh)).cuda()
    C = torch.from_numpy(np.ascontiguousarray(cu.reshape(n, -1))).cuda()
    A, b, f = ctx.integrate(et, X, C, kind, quad, api.PER_QPOINT if cpq else api.PER_ELEMENT, prec, api.AOS, api.AOS)
    ctx.sync()
    An, bn, fl = A.double().cpu().numpy(), b.double().cpu().numpy(), f.cpu().numpy()
    cref = cu.astype(np.float64)
    if kind == api.POISSON:
        cref = cref.reshape(-1)
    Ar, br, fr = oracle.integrate(et, kind, ORACLE_RULE[quad], mesh, cref, coef_per_q=bool(cpq), n_threads=8)
    ea, eb = oracle.rel_frobenius(An, Ar), oracle.rel_frobenius(bn, br)
    flagged = (fl & 1) != 0
    rec = {"workload": wl, "n_elem": n, "precision": pname, "tolerance": TOL[prec],
           "A": {"unflagged": _stats(ea, ~flagged), "flagged": _stats(ea, flagged)},
           "b": {"unflagged": _stats(eb, ~flagged), "flagged": _stats(eb, flagged)}}
    path = os.environ.get("FE_ERROR_REPORT")
    if path:
        with open(path, "a") as fh:
            fh.write(json.dumps(rec) + "\n")
    print(json.dumps(rec))
    assert ((fl & 6) == fr).all()
    if prec == api.FP64:
        assert not flagged.any()
    if "slivers" in wl and prec != api.FP64:
        assert flagged.sum() > 0
    for part in ("A", "b"):
        for grp in ("unflagged", "flagged"):
            s = rec[part][grp]
            if s["n"]:
                assert s["max"] <= TOL[prec] and s["p99.9"] <= TOL[prec], (part, grp, s)
