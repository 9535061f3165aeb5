"""Shared helpers of the GPU parity tests: run the CUDA path through the C ABI
and the FP64 oracle on the same seeded inputs, and compare per element."""
from __future__ import annotations

import numpy as np
import torch

import oracle
from paper_1504_01023_gb300 import api, meshgen

TOL = {api.FP64: 1e-12, api.FP64_DW: 1e-12, api.FP32_MIXED: 2e-5}
ORACLE_RULE = {api.QUAD_TET1: oracle.Q_TET1, api.QUAD_TET4: oracle.Q_TET4, api.QUAD_PRISM6: oracle.Q_PRISM6}


def make_inputs(et, kind, quad, cpq, n=None, seed=1, mesh=None):
    """Seeded mesh (numpy [E,NS,3]) and coefficients in the oracle's shape."""
    if mesh is None:
        mesh = meshgen.tet_cube_mesh(8, seed=seed) if et == api.TET else meshgen.prism_slab_mesh(40, seed=seed)
        if n is not None:
            mesh = mesh[:n]
    n = len(mesh)
    nq = api.NQ[quad]
    if kind == api.GENERIC:
        c = meshgen.generic_coefs(n, nq if cpq else 1, seed=seed + 100)
    else:
        c = meshgen.poisson_coefs(n, nq if cpq else 1, value=None, seed=seed + 200)
    return mesh, c


def to_device_inputs(et, mesh, c, prec, layout, device="cuda"):
    """Torch tensors in the layout the ABI expects; coefficients narrowed to the
    precision of the form (the oracle then reads the same narrowed values)."""
    n = len(mesh)
    cdt = np.float32 if prec == api.FP32_MIXED else np.float64
    c_used = c.astype(cdt)
    if layout == api.SOA:
        X = torch.from_numpy(meshgen.soa(mesh))
        C = torch.from_numpy(np.ascontiguousarray(c_used.reshape(n, -1).T))
    else:
        X = torch.from_numpy(np.ascontiguousarray(mesh))
        C = torch.from_numpy(np.ascontiguousarray(c_used.reshape(n, -1)))
    if device is not None:
        X, C = X.to(device), C.to(device)
    return X, C, c_used.astype(np.float64)


def gpu_outputs_to_numpy(et, A, b, flags, out_layout):
    ns = api.NS[et]
    if out_layout == api.SOA:
        n = A.shape[1]
        An = A.T.reshape(n, ns, ns).double().cpu().numpy()
        bn = b.T.double().cpu().numpy()
    else:
        An = A.double().cpu().numpy()
        bn = b.double().cpu().numpy()
    fn = flags.cpu().numpy() if flags is not None else None
    return An, bn, fn


def run_gpu(ctx, et, kind, quad, cpq, prec, layout, out_layout, mesh, c, device="cuda"):
    X, C, c_used = to_device_inputs(et, mesh, c, prec, layout, device)
    A, b, flags = ctx.integrate(et, X, C, kind, quad, api.PER_QPOINT if cpq else api.PER_ELEMENT, prec, layout,
                                out_layout)
    ctx.sync()
    An, bn, fn = gpu_outputs_to_numpy(et, A, b, flags, out_layout)
    return An, bn, fn, c_used


def run_oracle(et, kind, quad, cpq, mesh, c_used):
    return oracle.integrate(et, kind, ORACLE_RULE[quad], mesh, c_used, coef_per_q=bool(cpq), n_threads=8)


def max_errors(An, bn, Ar, br):
    return float(oracle.rel_frobenius(An, Ar).max()), float(oracle.rel_frobenius(bn, br).max())
