"""C ABI checks that need no GPU: the library loads, exports every entry point
declared in include/fe.h, and validates arguments on the host."""
import ctypes
import os
import re

import pytest

from paper_1504_01023_gb300 import api, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "fe.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fe_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return api.load()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 18
    for n in names:
        assert hasattr(lib, n), n
    # and the binding declares a signature for each of them
    assert set(names) <= {s[0] for s in api._SIGS}


def test_bytes_per_element_matches_table3(lib):
    """Table 3 (Sec. 4.1): DP words per element 36, 66, 52, 80 (Poisson tet and
    prism with d^0 per point, conv-diff tet and prism with 20 per-element
    coefficients) -> 288, 528, 416, 640 bytes."""
    b = api.bytes_per_element
    assert b(api.TET, api.POISSON, api.QUAD_TET4, api.PER_QPOINT, api.FP64) == 288
    assert b(api.PRISM, api.POISSON, api.QUAD_PRISM6, api.PER_QPOINT, api.FP64) == 528
    assert b(api.TET, api.GENERIC, api.QUAD_TET4, api.PER_ELEMENT, api.FP64) == 416
    assert b(api.PRISM, api.GENERIC, api.QUAD_PRISM6, api.PER_ELEMENT, api.FP64) == 640
    # the workloads of this library
    assert b(api.TET, api.POISSON, api.QUAD_TET1, api.PER_ELEMENT, api.FP64) == 264
    assert b(api.TET, api.GENERIC, api.QUAD_TET4, api.PER_ELEMENT, api.FP32_MIXED) == 256
    assert b(api.PRISM, api.GENERIC, api.QUAD_PRISM6, api.PER_QPOINT, api.FP32_MIXED) == 792
    # the double-word form moves the bytes of the FP64 form
    for et, q in [(api.TET, api.QUAD_TET1), (api.TET, api.QUAD_TET4), (api.PRISM, api.QUAD_PRISM6)]:
        for kind in (api.POISSON, api.GENERIC):
            for cm in (api.PER_ELEMENT, api.PER_QPOINT):
                assert b(et, kind, q, cm, api.FP64_DW) == b(et, kind, q, cm, api.FP64)
    assert b(api.TET, api.POISSON, api.QUAD_TET1, api.PER_ELEMENT, 3) == -1
    assert b(api.TET, 7, api.QUAD_TET4, 0, 0) == -1


def _args(n=10, et=api.TET, quad=api.QUAD_TET4, prec=api.FP32_MIXED):
    a = api.ElemArgs()
    a.n_elem = n
    a.coords = 4096
    a.coefs = 8192
    a.kind, a.quad, a.coef_mode, a.prec = api.GENERIC, quad, api.PER_ELEMENT, prec
    o = api.Out()
    o.A, o.b = 16384, 32768
    return a, o


def _chk(lib, et, a, o):
    return lib.fe_check_args(et, ctypes.byref(a), ctypes.byref(o))


def test_argument_validation(lib):
    a, o = _args()
    assert _chk(lib, api.TET, a, o) == 0
    bad = []
    a2, o2 = _args(); a2.n_elem = -1; bad.append((api.TET, a2, o2))
    a2, o2 = _args(); a2.quad = api.QUAD_PRISM6; bad.append((api.TET, a2, o2))
    a2, o2 = _args(); bad.append((api.PRISM, a2, o2))                       # tet rule on a prism
    a2, o2 = _args(); a2.coords = 0; bad.append((api.TET, a2, o2))
    a2, o2 = _args(); a2.coords = 4100; bad.append((api.TET, a2, o2))        # misaligned double
    a2, o2 = _args(); a2.coords_stride = 5; bad.append((api.TET, a2, o2))    # SOA stride < n
    a2, o2 = _args(); o2.stride = 3; bad.append((api.TET, a2, o2))
    a2, o2 = _args(); a2.kind = 9; bad.append((api.TET, a2, o2))
    a2, o2 = _args(); a2.prec = 5; bad.append((api.TET, a2, o2))
    a2, o2 = _args(); o2.layout = 4; bad.append((api.TET, a2, o2))
    a2, o2 = _args(); a2.memory = 3; bad.append((api.TET, a2, o2))
    for et, a2, o2 in bad:
        assert _chk(lib, et, a2, o2) == -1, (a2.n_elem, a2.quad)
    assert lib.fe_check_args(api.TET, None, ctypes.byref(o)) == -1
    # coefficient layout must follow the coordinate layout
    a2, o2 = _args(); a2.coefs_layout = api.AOS
    assert _chk(lib, api.TET, a2, o2) == -6
    # zero elements is valid even with null pointers
    a2, o2 = _args(0); a2.coords = 0; a2.coefs = 0; o2.A = 0; o2.b = 0
    assert _chk(lib, api.TET, a2, o2) == 0
    assert lib.fe_last_error(None)


def test_node_table_validation(lib):
    """FE_LAYOUT_INDEXED: node array + int32 element -> node table, device memory,
    element-contiguous coefficients."""
    def idx(**kw):
        a, o = _args()
        a.coords_layout, a.coefs_layout = api.INDEXED, api.AOS
        a.conn, a.n_nodes = 65536, 100
        for k, v in kw.items():
            setattr(a, k, v)
        return a, o
    a, o = idx()
    assert _chk(lib, api.TET, a, o) == 0
    assert _chk(lib, api.TET, *idx(conn=0)) == -1                 # no table
    assert _chk(lib, api.TET, *idx(conn=65538)) == -1             # misaligned int32
    assert _chk(lib, api.TET, *idx(n_nodes=0)) == -1
    assert _chk(lib, api.TET, *idx(n_nodes=1 << 31)) == -1        # indices are int32
    assert _chk(lib, api.TET, *idx(coefs_layout=api.SOA)) == -6   # coefficients element-contiguous
    assert _chk(lib, api.TET, *idx(memory=api.MEM_HOST)) == -6    # device memory only
    a, o = idx()
    o.memory = api.MEM_HOST
    assert _chk(lib, api.TET, a, o) == -6
    # the output side has no indexed layout
    a, o = idx()
    o.layout = api.INDEXED
    assert _chk(lib, api.TET, a, o) == -1
    # no allocation-free call with a node table (rejected before any GPU work)
    assert lib.fe_integrate_tet_noalloc(ctypes.byref(idx()[0]), ctypes.byref(o), None) in (-1, -6)


def test_packed_output_validation(lib):
    """packed = 1 (upper triangle) for the symmetric Laplace kind only."""
    a, o = _args()
    a.kind = api.POISSON
    o.packed = 1
    assert _chk(lib, api.TET, a, o) == 0
    a.kind = api.GENERIC
    assert _chk(lib, api.TET, a, o) == -6
    a.kind, o.packed = api.POISSON, 2
    assert _chk(lib, api.TET, a, o) == -1
    o.packed = 1
    a.coords_layout, a.coefs_layout, a.conn, a.n_nodes = api.INDEXED, api.AOS, 65536, 10
    assert _chk(lib, api.TET, a, o) == -6


def test_ordering_validation(lib):
    """SQS / SSQ (study orderings): mixed form, element-contiguous in and out."""
    a, o = _args()
    a.coords_layout = a.coefs_layout = o.layout = api.AOS
    for ordering in (api.QSS, api.SQS, api.SSQ):
        a.ordering = ordering
        assert _chk(lib, api.TET, a, o) == 0
    a.ordering = 3
    assert _chk(lib, api.TET, a, o) == -1
    a.ordering = api.SQS
    a.prec = api.FP64
    assert _chk(lib, api.TET, a, o) == -6
    a.prec = api.FP32_MIXED
    o.layout = api.SOA
    assert _chk(lib, api.TET, a, o) == -6


def test_coef_function_validation(lib):
    """FE_COEF_FUNCTION_U: a parameter block, element-contiguous coordinates."""
    fn = api.CoefFunction()
    a, o = _args()
    a.coords_layout = a.coefs_layout = o.layout = api.AOS
    a.coef_mode = api.COEF_FN_U
    assert _chk(lib, api.TET, a, o) == -1                  # no parameter block
    a.coef_fn = ctypes.addressof(fn)
    assert _chk(lib, api.TET, a, o) == 0
    a.coords_layout = a.coefs_layout = api.SOA
    assert _chk(lib, api.TET, a, o) == -6
    a.coords_layout = a.coefs_layout = api.AOS
    a.ordering = api.SQS
    assert _chk(lib, api.TET, a, o) == -6
    # per element: coordinates, the NS nodal values, outputs
    b = api.bytes_per_element
    assert b(api.TET, api.GENERIC, api.QUAD_TET4, api.COEF_FN_U, api.FP32_MIXED) == 96 + 16 + 80
    assert b(api.PRISM, api.GENERIC, api.QUAD_PRISM6, api.COEF_FN_U, api.FP32_MIXED) == 144 + 24 + 168


def test_null_context_rejected(lib):
    a, o = _args()
    assert lib.fe_integrate_tet(None, ctypes.byref(a), ctypes.byref(o), None) == -1
    assert lib.fe_ctx_sync(None) == -1


def _ref_shape_values(elem, pts):
    """Reference shape functions at reference points (vertex k <-> phi_k): the tet
    (1 - xi - eta - zeta, xi, eta, zeta); the prism lambda_k(xi, eta) (1 -/+ zeta) / 2
    with lambda = (1 - xi - eta, xi, eta) on the bottom and top triangles."""
    import numpy as np
    xi, eta, zeta = pts[:, 0], pts[:, 1], pts[:, 2]
    if elem == "tet":
        return np.stack([1 - xi - eta - zeta, xi, eta, zeta], axis=1)
    lam = np.stack([1 - xi - eta, xi, eta], axis=1)
    return np.concatenate([lam * ((1 - zeta) / 2)[:, None], lam * ((1 + zeta) / 2)[:, None]], axis=1)


@pytest.mark.parametrize("quad,elem", [(api.QUAD_TET1, "tet"), (api.QUAD_TET4, "tet"), (api.QUAD_PRISM6, "prism")])
def test_rule_tables_match_the_oracle(lib, quad, elem):
    """The kernels' quadrature (weights and shape values at the points, compile-time
    constants of the library) against the oracle's rule, typed in separately: the
    same points, up to order, and the same weights."""
    import numpy as np
    import oracle
    w, phi = api.rule_table(quad)
    rule = {api.QUAD_TET1: oracle.Q_TET1, api.QUAD_TET4: oracle.Q_TET4, api.QUAD_PRISM6: oracle.Q_PRISM6}[quad]
    pts, wts = oracle.quad_rule(rule)
    ref = _ref_shape_values(elem, pts)
    assert len(w) == len(wts)
    used = set()
    for q in range(len(w)):
        d = np.abs(ref - phi[q]).max(axis=1)
        j = int(np.argmin(d))
        assert d[j] < 1e-15 and j not in used, (q, d)
        used.add(j)
        assert abs(w[q] - wts[j]) < 1e-16
    # partition of unity and the reference measure
    assert np.allclose(phi.sum(axis=1), 1.0, rtol=0, atol=1e-15)
    assert abs(w.sum() - (1 / 6 if elem == "tet" else 1.0)) < 1e-15
    with pytest.raises(api.FeError):
        n = ctypes.c_int()
        arr = (ctypes.c_double * 1)()
        api._check(lib.fe_rule_table(quad, 0 if quad == api.QUAD_TET1 else 1, ctypes.byref(n), arr, None))


def test_validation_fuzz(lib):
    """Host-only fuzzing of the argument validation: valid argument sets with up to
    three fields replaced by random values (enums in and out of range, negative and
    huge sizes and strides, null and misaligned pointers, which are never
    dereferenced) give FE_OK, FE_ERR_INVALID_ARG or FE_ERR_UNSUPPORTED, never a
    crash; and FE_OK only for arguments that meet the documented rules."""
    import numpy as np
    rng = np.random.default_rng(2024)
    sizes = [-5, -1, 0, 1, 7, 1000, (1 << 31) + 3, (1 << 32) - 1, 1 << 32, 1 << 40]
    strides = [0, 1, 999, 1000, 1 << 20, (1 << 40), (1 << 40) + 1, 1 << 62, -3]
    ptrs = [0, 4096, 4097, 4100, 8192, 1 << 40]
    fields = {
        "et": lambda: int(rng.integers(-1, 3)), "n_elem": lambda: int(rng.choice(sizes)),
        "coords": lambda: int(rng.choice(ptrs)), "coefs": lambda: int(rng.choice(ptrs)),
        "A": lambda: int(rng.choice(ptrs)), "b": lambda: int(rng.choice(ptrs)),
        "coords_layout": lambda: int(rng.integers(-1, 4)), "coefs_layout": lambda: int(rng.integers(-1, 4)),
        "layout": lambda: int(rng.integers(-1, 4)), "coords_stride": lambda: int(rng.choice(strides)),
        "coefs_stride": lambda: int(rng.choice(strides)), "stride": lambda: int(rng.choice(strides)),
        "kind": lambda: int(rng.integers(-1, 4)), "quad": lambda: int(rng.integers(-1, 4)),
        "coef_mode": lambda: int(rng.integers(-1, 4)), "prec": lambda: int(rng.integers(-1, 4)),
        "memory": lambda: int(rng.integers(-1, 3)), "omemory": lambda: int(rng.integers(-1, 3)),
        "conn": lambda: int(rng.choice(ptrs)), "n_nodes": lambda: int(rng.choice(sizes)),
        "ordering": lambda: int(rng.integers(-1, 4)), "packed": lambda: int(rng.integers(-1, 3)),
    }
    names = list(fields)
    seen = {0: 0, -1: 0, -6: 0}
    for _ in range(20000):
        et = int(rng.integers(0, 2))
        lay = int(rng.integers(0, 2))
        v = dict(et=et, n_elem=int(rng.integers(1, 5000)), coords=4096, coefs=8192, A=12288, b=16384,
                 coords_layout=lay, coefs_layout=lay, layout=int(rng.integers(0, 2)), coords_stride=0,
                 coefs_stride=0, stride=0, kind=int(rng.integers(0, 2)),
                 quad=int(rng.integers(0, 2)) if et == 0 else 2, coef_mode=int(rng.integers(0, 2)),
                 prec=int(rng.integers(0, 3)), memory=0, omemory=0, conn=0, n_nodes=0, ordering=0, packed=0)
        k = int(rng.integers(0, 4))
        for f in (rng.choice(names, size=k, replace=False) if k else []):
            v[f] = fields[f]()
        a = api.ElemArgs()
        o = api.Out()
        a.n_elem, a.coords, a.coefs, o.A, o.b = v["n_elem"], v["coords"], v["coefs"], v["A"], v["b"]
        a.coords_layout, a.coefs_layout, o.layout = v["coords_layout"], v["coefs_layout"], v["layout"]
        a.coords_stride, a.coefs_stride, o.stride = v["coords_stride"], v["coefs_stride"], v["stride"]
        a.kind, a.quad, a.coef_mode, a.prec = v["kind"], v["quad"], v["coef_mode"], v["prec"]
        a.memory, o.memory, a.conn, a.n_nodes = v["memory"], v["omemory"], v["conn"], v["n_nodes"]
        a.ordering, o.packed, a.coef_fn = v["ordering"], v["packed"], None
        st = lib.fe_check_args(v["et"], ctypes.byref(a), ctypes.byref(o))
        assert st in (0, -1, -6), st
        seen[st] += 1
        if st == 0:
            et = v["et"]
            assert et in (0, 1) and a.kind in (0, 1) and a.prec in (0, 1, 2) and a.coef_mode in (0, 1)
            assert a.quad in ((0, 1) if et == 0 else (2,))
            assert 0 <= a.n_elem < (1 << 32) and a.ordering in (0, 1, 2) and o.packed in (0, 1)
            assert o.layout in (0, 1) and a.coords_layout in (0, 1, 2) and a.memory in (0, 1) and o.memory in (0, 1)
            if a.n_elem > 0:
                assert a.coords and a.coefs and o.A and o.b and a.coords % 8 == 0
                used = ([a.coords_stride, a.coefs_stride] if a.coords_layout == 0 else []) + \
                       ([o.stride] if o.layout == 0 else [])
                for s in used:
                    assert s == 0 or a.n_elem <= s <= (1 << 40)
                if a.coords_layout == 2:
                    assert a.conn and a.conn % 4 == 0 and 0 < a.n_nodes < (1 << 31)
    assert min(seen.values()) > 100, seen
