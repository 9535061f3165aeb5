"""Seeded synthetic workloads (meshes and coefficients) for the integration kernels.

This module holds input generation only: node grids, element connectivity,
jitter, random coefficients. It computes no Jacobian, no shape function and no
element integral, so the CUDA path and the CPU oracle can both be fed from it
without sharing any of the method's arithmetic.

The paper describes no mesh (Sec. 5 gives timings per element only), so the
workloads are synthetic: jittered Kuhn-split cubes for tetrahedra, an extruded
triangulated square for prisms, and coefficients drawn per element or per
integration point. Seeds are ``SEED_BASE + workload number``.
"""
from __future__ import annotations

import numpy as np

SEED_BASE = 1504010230

# Kuhn split of the unit cube into 6 tetrahedra sharing the (0,0,0)-(1,1,1)
# diagonal: one tetrahedron per permutation of the axes, listed so that every
# tetrahedron has positive orientation (odd permutations have vertices 1 and 2
# swapped).
_PERMS = [(0, 1, 2), (1, 2, 0), (2, 0, 1), (0, 2, 1), (2, 1, 0), (1, 0, 2)]
_PARITY = [0, 0, 0, 1, 1, 1]


def _kuhn_corner_offsets():
    out = []
    for perm, odd in zip(_PERMS, _PARITY):
        v = [np.zeros(3, dtype=np.int64)]
        for ax in perm:
            nxt = v[-1].copy()
            nxt[ax] += 1
            v.append(nxt)
        if odd:
            v[1], v[2] = v[2], v[1]
        out.append(np.stack(v))
    return np.stack(out)                       # [6, 4, 3] corner offsets in {0,1}


def tet_cube_mesh(n: int, jitter: float = 0.2, seed: int = SEED_BASE + 1, n_elem: int | None = None):
    """Unit cube split into n^3 cubes x 6 Kuhn tetrahedra; every node moved by
    U[-jitter*h, jitter*h] per coordinate (h = 1/n). Returns coords [E, 4, 3]
    (float64), elements ordered cube by cube (x fastest). ``n_elem`` keeps the
    first n_elem elements."""
    nodes, conn = tet_cube_indexed(n, jitter, seed, n_elem)
    return nodes[conn]


def tet_cube_indexed(n: int, jitter: float = 0.2, seed: int = SEED_BASE + 1, n_elem: int | None = None):
    """The mesh of tet_cube_mesh as a node array [(n+1)^3, 3] (node id = i +
    (n+1)(j + (n+1)k)) and an element -> node table [E, 4] (int32);
    nodes[conn] is exactly tet_cube_mesh's coordinates."""
    rng = np.random.default_rng(seed)
    h = 1.0 / n
    m = n + 1
    grid = np.stack(np.meshgrid(np.arange(m), np.arange(m), np.arange(m), indexing="ij"), -1)
    nodes = grid.transpose(2, 1, 0, 3).reshape(-1, 3).astype(np.float64) * h    # node id = i + m*(j + m*k)
    nodes += rng.uniform(-jitter * h, jitter * h, size=nodes.shape)
    total = 6 * n ** 3
    if n_elem is None:
        n_elem = total
    assert 0 <= n_elem <= total
    cubes = np.arange((n_elem + 5) // 6, dtype=np.int64)
    ci = cubes % n
    cj = (cubes // n) % n
    ck = cubes // (n * n)
    off = _kuhn_corner_offsets()                                        # [6,4,3]
    ii = ci[:, None, None] + off[None, :, :, 0]
    jj = cj[:, None, None] + off[None, :, :, 1]
    kk = ck[:, None, None] + off[None, :, :, 2]
    nid = (ii + m * (jj + m * kk)).reshape(-1, 4)[:n_elem]
    return nodes, np.ascontiguousarray(nid.astype(np.int32))


def prism_slab_mesh(n: int, hz: float | None = None, zjitter: float = 0.1, seed: int = SEED_BASE + 3,
                    n_elem: int | None = None):
    """[0,1]^2 split into n x n squares, each cut into two triangles along the same
    diagonal, extruded to one layer z in [0, hz] (hz = 1/n by default); every
    node's z moved by U[-zjitter*hz, zjitter*hz]. Returns coords [E, 6, 3]:
    bottom triangle (counter-clockwise seen from +z), then the top vertices above
    them."""
    nodes, conn = prism_slab_indexed(n, hz, zjitter, seed, n_elem)
    return nodes[conn]


def prism_slab_indexed(n: int, hz: float | None = None, zjitter: float = 0.1, seed: int = SEED_BASE + 3,
                       n_elem: int | None = None):
    """The mesh of prism_slab_mesh as a node array [2 (n+1)^2, 3] (bottom nodes
    i + (n+1) j, then the top ones) and an element -> node table [E, 6] (int32);
    nodes[conn] is exactly prism_slab_mesh's coordinates."""
    rng = np.random.default_rng(seed)
    h = 1.0 / n
    if hz is None:
        hz = h
    m = n + 1
    total = 2 * n * n
    if n_elem is None:
        n_elem = total
    assert 0 <= n_elem <= total
    jy, ix = np.meshgrid(np.arange(m), np.arange(m), indexing="ij")
    xy = np.stack([ix.reshape(-1) * h, jy.reshape(-1) * h], -1)           # node id = i + m*j
    zb = rng.uniform(-zjitter * hz, zjitter * hz, size=m * m)
    zt = hz + rng.uniform(-zjitter * hz, zjitter * hz, size=m * m)
    sq = np.arange((n_elem + 1) // 2, dtype=np.int64)
    i = sq % n
    j = sq // n
    p00 = i + m * j
    p10 = p00 + 1
    p01 = p00 + m
    p11 = p01 + 1
    tri = np.stack([np.stack([p00, p10, p11], -1), np.stack([p00, p11, p01], -1)], 1).reshape(-1, 3)[:n_elem]
    nodes = np.empty((2 * m * m, 3))
    nodes[:m * m, :2] = xy
    nodes[m * m:, :2] = xy
    nodes[:m * m, 2] = zb
    nodes[m * m:, 2] = zt
    conn = np.concatenate([tri, tri + m * m], axis=1).astype(np.int32)
    return nodes, np.ascontiguousarray(conn)


def _haar_orthogonal(rng, n: int):
    """n Haar-distributed 3x3 orthogonal matrices: Gram-Schmidt (QR with positive
    R diagonal) of Gaussian matrices, columns in order."""
    g = rng.standard_normal((n, 3, 3))
    q = np.empty_like(g)
    for c in range(3):
        v = g[:, :, c].copy()
        for p in range(c):
            v -= np.sum(q[:, :, p] * v, axis=1, keepdims=True) * q[:, :, p]
        q[:, :, c] = v / np.linalg.norm(v, axis=1, keepdims=True)
    return q


def generic_coefs(n_elem: int, n_points: int = 1, seed: int = SEED_BASE + 2, chunk: int = 1 << 20):
    """Convection-diffusion-reaction coefficients, 20 per element and point,
    packed C[4][4] row-major (C[a][b] = c^{a;b}) then D[4] (d^a):
    c^{ij} = Q diag(l) Q^T with l ~ U[0.1, 10]^3 and Q Haar-orthogonal,
    c^{i0}, c^{0i} ~ U[-1,1]^3, c^{00} ~ U[0,1], d^0 ~ U[-1,1], d^i ~ U[-1,1]^3.
    Returns [E, 20] (n_points == 1) or [E, n_points, 20], float64."""
    rng = np.random.default_rng(seed)
    total = n_elem * n_points
    out = np.empty((total, 20))
    for s in range(0, total, chunk):
        k = min(chunk, total - s)
        lam = rng.uniform(0.1, 10.0, size=(k, 3))
        q = _haar_orthogonal(rng, k)
        cd = np.einsum("nij,nj,nkj->nik", q, lam, q)
        C = np.zeros((k, 4, 4))
        C[:, 1:, 1:] = cd
        C[:, 1:, 0] = rng.uniform(-1.0, 1.0, size=(k, 3))
        C[:, 0, 1:] = rng.uniform(-1.0, 1.0, size=(k, 3))
        C[:, 0, 0] = rng.uniform(0.0, 1.0, size=k)
        out[s:s + k, :16] = C.reshape(k, 16)
        out[s:s + k, 16] = rng.uniform(-1.0, 1.0, size=k)
        out[s:s + k, 17:20] = rng.uniform(-1.0, 1.0, size=(k, 3))
    return out.reshape(n_elem, 20) if n_points == 1 else out.reshape(n_elem, n_points, 20)


def poisson_coefs(n_elem: int, n_points: int = 1, value: float | None = 1.0, seed: int = SEED_BASE + 1):
    """d^0 per element (n_points == 1, shape [E]) or per point ([E, n_points]):
    the constant ``value``, or U[-1,1] when value is None."""
    shape = (n_elem,) if n_points == 1 else (n_elem, n_points)
    if value is not None:
        return np.full(shape, float(value))
    return np.random.default_rng(seed).uniform(-1.0, 1.0, size=shape)


# Flattening factors for the sliver stress set: vertex 3 is moved toward the
# centroid of the opposite face to t times its height. For jittered Kuhn
# tetrahedra t log-uniform in this range puts the single-precision mean-ratio
# quality mostly in [0.01, 0.1).
SLIVER_T_RANGE = (2e-3, 2e-2)


def make_slivers(coords: np.ndarray, fraction: float, seed: int = SEED_BASE + 20,
                 t_range=SLIVER_T_RANGE):
    """Flatten a seeded random subset of tetrahedra in place: x3 <- c + t (x3 - c)
    with c the centroid of vertices 0..2 and t log-uniform in t_range. Returns the
    sorted indices of the flattened elements."""
    rng = np.random.default_rng(seed)
    n = coords.shape[0]
    k = int(round(fraction * n))
    idx = np.sort(rng.choice(n, size=k, replace=False)) if k else np.zeros(0, dtype=np.int64)
    t = np.exp(rng.uniform(np.log(t_range[0]), np.log(t_range[1]), size=k))
    c = coords[idx, :3, :].mean(axis=1)
    coords[idx, 3, :] = c + t[:, None] * (coords[idx, 3, :] - c)
    return idx


def loguniform_sizes(n: int, lo: float, hi: float, seed: int):
    """n integer sizes log-uniform in [lo, hi]."""
    rng = np.random.default_rng(seed)
    return np.round(np.exp(rng.uniform(np.log(lo), np.log(hi), size=n))).astype(np.int64)


def batch_mix(n_meshes: int = 256, lo: float = 1e3, hi: float = 2e6, seed: int = SEED_BASE + 4):
    """Mesh sizes and (type, kind) of the batched workload: sizes log-uniform in
    [lo, hi], type 50/50 tetrahedron/prism, kind 50/50 Poisson/generic.
    Returns a list of (n_elem, elem_type, kind) with 0 = tet/Poisson, 1 = prism/generic."""
    rng = np.random.default_rng(seed)
    sizes = np.round(np.exp(rng.uniform(np.log(lo), np.log(hi), size=n_meshes))).astype(np.int64)
    types = rng.integers(0, 2, size=n_meshes)
    kinds = rng.integers(0, 2, size=n_meshes)
    return [(int(s), int(t), int(k)) for s, t, k in zip(sizes, types, kinds)]


def mesh_for_size(elem_type: int, n_elem: int, seed: int):
    """A cube (tet) or slab (prism) mesh with exactly n_elem elements: the smallest
    grid that holds them, first n_elem elements kept."""
    if elem_type == 0:
        n = max(1, int(np.ceil((n_elem / 6.0) ** (1.0 / 3.0))))
        while 6 * n ** 3 < n_elem:
            n += 1
        return tet_cube_mesh(n, 0.2, seed=seed, n_elem=n_elem)
    n = max(1, int(np.ceil(np.sqrt(n_elem / 2.0))))
    while 2 * n * n < n_elem:
        n += 1
    return prism_slab_mesh(n, None, 0.1, seed=seed, n_elem=n_elem)


class MixPool:
    """Seeded base data for workloads of many meshes of uneven size: one
    tetrahedral and one prism base mesh of at least `max_elems` elements, a pool of
    independent generic coefficient draws and of Poisson right-hand sides. A mesh
    of n elements is a window of n consecutive elements of its base mesh at a
    seeded offset; its per-element or per-point coefficients are consecutive pool
    entries from a seeded offset (cyclically)."""

    def __init__(self, max_elems: int, seed: int, pool_size: int = 1 << 22):
        n = max(1, int(np.ceil((max_elems / 6.0) ** (1.0 / 3.0))))
        while 6 * n ** 3 < max_elems:
            n += 1
        self.tet = tet_cube_mesh(n, 0.2, seed=seed)
        m = max(1, int(np.ceil(np.sqrt(max_elems / 2.0))))
        while 2 * m * m < max_elems:
            m += 1
        self.prism = prism_slab_mesh(m, None, 0.1, seed=seed + 1)
        self.generic = generic_coefs(pool_size, 1, seed=seed + 2)
        self.poisson = np.random.default_rng(seed + 3).uniform(-1.0, 1.0, size=pool_size)
        self.rng = np.random.default_rng(seed + 4)

    def window(self, elem_type: int, n: int):
        base = self.tet if elem_type == 0 else self.prism
        off = int(self.rng.integers(0, len(base) - n + 1))
        return off

    def coef_offset(self):
        return int(self.rng.integers(0, len(self.poisson)))


def mix_spec(elem_type: int, kind: int):
    """Rule and coefficient mode of each (type, kind) in the mixed workloads:
    tetrahedra Poisson TET1 with d^0 per element, generic TET4 per element;
    prisms PRISM6 with d^0 per point (Poisson) or 20 coefficients per point."""
    if elem_type == 0:
        return (0, 0) if kind == 0 else (1, 0)       # (quad, per-point)
    return (2, 1)


def soa(a: np.ndarray) -> np.ndarray:
    """[E, ...] -> [K, E] planes (structure of arrays), contiguous."""
    return np.ascontiguousarray(a.reshape(a.shape[0], -1).T)
