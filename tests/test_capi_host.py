"""The C-ABI library without a GPU: it loads, exports every function that
include/lcmg.h declares, and its host-only calls (L-curve corner, lambda
window, defaults, argument errors) agree with the oracle."""
import numpy as np
import pytest

import problemgen as pg
from oracle import lcurve

L = pytest.importorskip("paper_2306_11067_gb300.lcmg")


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2306_11067_gb300 import build
    build.build()


def test_library_exports_every_header_function():
    lib = L.lib()
    names = L.header_functions()
    assert len(names) >= 20
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(L._SIGS), set(names) ^ set(L._SIGS)


def test_default_params():
    p = L.lcmg_default_params()
    assert (p.nu, p.coarse_max, p.maxit, p.check_every, p.graphs) == (1, 16, 10000, 16, 1)
    assert (p.tol, p.q, p.d_min) == (1e-6, 2.0, 1e-3)
    # execution-path options: the measured-fastest combination on GB300
    assert (p.vfuse, p.mode, p.precision) == (1, L.MODE_SEQUENTIAL, L.PREC_FP64)
    assert L.lcmg_version().startswith("lcmg")


def test_cull_matches_oracle_exhaustive():
    for m in range(10, 65):
        assert L.lcmg_cull_lambdas(m, 0) == (1, m)
        for i in range(1, m + 1):
            assert L.lcmg_cull_lambdas(m, i) == lcurve.lambda_window(m, i)
    with pytest.raises(L.LcmgError):
        L.lcmg_cull_lambdas(10, 11)


def test_corner_matches_oracle_random_curves():
    g = pg.rng(5)
    for trial in range(300):
        k = int(g.integers(3, 40))
        rho = np.sort(10.0 ** g.uniform(-2, 3, k))
        eta = np.sort(10.0 ** g.uniform(-2, 3, k))[::-1].copy()
        assert L.lcmg_lcurve_corner(rho, eta) == lcurve.corner(rho, eta), trial


@pytest.mark.parametrize("eps", [0.0, 1e-15, -1e-15])
def test_corner_ties_go_to_the_smaller_lambda(eps):
    """A staircase in (log rho, log eta) with two identical corners, one of
    them moved by a relative 1e-15 either way: curvatures within a relative
    1e-12 are a tie, and a tie goes to the smaller lambda (index 1), in the
    library as in the oracle."""
    from oracle import lcurve
    u = np.array([0.0, 0.0, 1.0, 1.0 + eps, 2.0])
    v = np.array([2.0, 1.0, 1.0, 0.0, 0.0])
    rho, eta = 10.0 ** u, 10.0 ** v
    kap = lcurve.menger_curvature(rho, eta)
    assert abs(kap[3] - kap[1]) <= 1e-12 * kap[1]
    assert lcurve.corner(rho, eta) == 1
    assert L.lcmg_lcurve_corner(rho, eta) == 1


def test_corner_argument_errors():
    with pytest.raises(L.LcmgError) as e:
        L.lcmg_lcurve_corner([1.0, 2.0], [2.0, 1.0])
    assert e.value.status == L.LCMG_ERR_INVALID_ARG
    with pytest.raises(L.LcmgError):
        L.lcmg_lcurve_corner([1.0, -2.0, 3.0], [3.0, 2.0, 1.0])


def test_server_rejects_bad_arguments_without_a_device():
    """Argument checks of the serving entry points run before any CUDA call."""
    import ctypes as C
    h = C.c_void_p()
    p = L.lcmg_default_params()
    assert L.lib().lcmg_server_create(C.byref(h), 0, 1 << 30, 0, C.byref(p)) == L.LCMG_ERR_INVALID_ARG
    assert L.lib().lcmg_server_create(C.byref(h), 0, 0, 2, C.byref(p)) == L.LCMG_ERR_INVALID_ARG
    assert L.lib().lcmg_server_create(None, 0, 1 << 30, 2, C.byref(p)) == L.LCMG_ERR_INVALID_ARG
    assert b"bad arguments" in L.lib().lcmg_server_last_error()
    assert L.lib().lcmg_server_destroy(None) == L.LCMG_OK


def _amg_levels(n_v, n_h, d, max_coarse=16):
    from oracle import amg, operators as ops, multigrid as mg
    return amg.hierarchy(mg.weighted_laplacian(ops.gradient(n_v, n_h), d), max_coarse=max_coarse)


@pytest.mark.parametrize("n_v,n_h,seed", [(16, 16, 1), (32, 28, 2), (48, 52, 3), (9, 31, 4)])
@pytest.mark.parametrize("weights", ["random", "ones"])
def test_rs_split_and_interpolation_match_oracle(n_v, n_h, seed, weights):
    """Classical AMG on the host (lcmg_rs_split / lcmg_rs_interp) on every
    level of the oracle's hierarchy of L^T D^2 L: the C/F split is the same
    bit for bit (integer work), P within 1e-14."""
    import scipy.sparse as sp
    from oracle import operators as ops
    ne = ops.n_edges(n_v, n_h)
    d = pg.random_weights(ne, seed, d_min=0.02) if weights == "random" else np.ones(ne)
    Ks, Ps, cfs = _amg_levels(n_v, n_h, d)
    assert len(Ps) >= 2
    for k, P in enumerate(Ps):
        cf = L.lcmg_rs_split(Ks[k])
        assert (cf == cfs[k]).all(), (k, int((cf != cfs[k]).sum()))
        rp, ci, v, nc = L.lcmg_rs_interp(Ks[k], cf)
        Pl = sp.csr_matrix((v, ci, rp), shape=(Ks[k].shape[0], nc))
        assert nc == P.shape[1]
        assert abs(Pl - P).max() <= 1e-14


def test_rs_host_argument_errors():
    import scipy.sparse as sp
    K = sp.csr_matrix(np.array([[2.0, -1.0], [-1.0, 2.0]]))
    with pytest.raises(L.LcmgError) as e:
        L.lcmg_rs_split(K, theta=1.5)
    assert e.value.status == L.LCMG_ERR_INVALID_ARG
    n, rp, ci, v = L._csr_in(K)
    bad = ci.copy()
    bad[0], bad[1] = bad[1], bad[0]                       # unsorted row
    cf = np.empty(2, np.int8)
    assert L.lib().lcmg_rs_split(n, L._ptr(rp), L._ptr(bad), L._ptr(v), 0.25, L._ptr(cf)) == L.LCMG_ERR_INVALID_ARG
    with pytest.raises(L.LcmgError):                     # an F point without a strong C connection
        L.lcmg_rs_interp(K, np.array([0, 0], np.int8))


def _edge_case_matrices():
    import scipy.sparse as sp
    yield "diagonal", sp.csr_matrix(np.diag([2.0, 3.0, 1.0, 4.0]))
    yield "positive off-diagonals", sp.csr_matrix(np.array([[2.0, 0.5, 0.0], [0.5, 2.0, 0.5], [0.0, 0.5, 2.0]]))
    A = np.zeros((6, 6))
    for a, b in ((0, 1), (1, 2), (3, 4), (4, 5)):      # two components
        A[a, b] = A[b, a] = -1.0
    A[np.arange(6), np.arange(6)] = -A.sum(axis=1)
    yield "two components", sp.csr_matrix(A)
    yield "one point", sp.csr_matrix(np.array([[1.0]]))
    g = pg.rng(7)
    n = 12
    perm = g.permutation(n)
    K = np.zeros((n, n))
    for i in range(n - 1):                               # 1-D chain, shuffled numbering
        a, b = perm[i], perm[i + 1]
        K[a, b] = K[b, a] = -1.0
    K[np.arange(n), np.arange(n)] = -K.sum(axis=1)
    yield "shuffled chain", sp.csr_matrix(K)
    for name, K, _, _ in _HAND_WORKED:
        yield name, sp.csr_matrix(K)


# Strength counts only negative couplings, and a coupling exactly at the
# threshold is weak.  In both matrices each end point then depends strongly
# on the middle point alone, the middle point on both ends: the first pass
# takes the middle point (measure 2) and its two dependants become F.  Each F
# point interpolates from the middle point, its other neighbour (weak, F)
# lumped into the diagonal: -(-1)/(6 + 5) and -(-4)/(6 - 1).
_HAND_WORKED = [
    ("large positive coupling",
     np.array([[6.0, -1.0, 5.0], [-1.0, 2.0, -1.0], [5.0, -1.0, 6.0]]),
     [0, 1, 0], np.array([[1.0 / 11.0], [1.0], [1.0 / 11.0]])),
    ("coupling at the threshold",
     np.array([[6.0, -4.0, -1.0], [-4.0, 9.0, -4.0], [-1.0, -4.0, 6.0]]),
     [0, 1, 0], np.array([[0.8], [1.0], [0.8]])),
]


@pytest.mark.parametrize("name,K,cf_hand,P_hand", _HAND_WORKED, ids=[c[0] for c in _HAND_WORKED])
def test_rs_strength_cases_worked_by_hand(name, K, cf_hand, P_hand):
    """Sec. 3.1's strength test, the first pass and the interpolation
    formula on two 3x3 matrices worked by hand: the oracle and the host
    library give the split and the weights above."""
    import scipy.sparse as sp
    from oracle import amg
    Ks = sp.csr_matrix(K)
    cf_ref, S = amg.split(Ks)
    assert list(cf_ref) == cf_hand
    assert np.allclose(amg.interpolation(Ks, S, cf_ref).toarray(), P_hand, rtol=1e-15, atol=0)
    cf = L.lcmg_rs_split(Ks)
    assert list(cf) == cf_hand
    rp, ci, v, nc = L.lcmg_rs_interp(Ks, cf)
    assert np.allclose(sp.csr_matrix((v, ci, rp), shape=(3, nc)).toarray(), P_hand, rtol=1e-15, atol=0)


@pytest.mark.parametrize("name,K", list(_edge_case_matrices()), ids=lambda v: v if isinstance(v, str) else "")
def test_rs_amg_edge_cases_match_oracle(name, K):
    """Degenerate inputs of the host AMG calls: the same split and
    interpolation as the oracle (no strong connection at all: every point
    C and P the identity)."""
    import scipy.sparse as sp
    from oracle import amg
    cf_ref, S = amg.split(K)
    cf = L.lcmg_rs_split(K)
    assert np.array_equal(cf, cf_ref), (name, cf, cf_ref)
    rp, ci, v, nc = L.lcmg_rs_interp(K, cf)
    P_ref = amg.interpolation(K, S, cf_ref)
    P = sp.csr_matrix((v, ci, rp), shape=(K.shape[0], nc))
    assert P.shape == P_ref.shape and abs(P - P_ref).max() <= 1e-15 if P.nnz else P_ref.nnz == 0
    if name in ("diagonal", "positive off-diagonals", "one point"):
        assert cf.all() and np.allclose(P.toarray(), np.eye(K.shape[0]))


def _header_struct_fields(name):
    """(type, name) of every field of a typedef'd struct of include/lcmg.h,
    in order; pointer types as 'ptr'."""
    import re
    txt = open(L.HEADER).read()
    end = txt.index("} " + name + ";")
    start = txt.rindex("typedef struct", 0, end)
    body = re.sub(r"/\*.*?\*/", "", txt[txt.index("{", start) + 1:end], flags=re.S)
    out = []
    for decl in body.split(";"):
        decl = " ".join(decl.split())
        if not decl:
            continue
        m = re.match(r"(?:const\s+)?(\w+)\s*(\*?)\s*(.*)", decl)
        base, star, names = m.group(1), m.group(2), m.group(3)
        for nm in names.split(","):
            nm = nm.strip()
            ptr = bool(star) or nm.startswith("*")
            out.append(("ptr" if ptr else base, nm.lstrip("*").strip()))
    return out


@pytest.mark.parametrize("name", ["lcmg_params", "lcmg_stats", "lcmg_problem", "lcmg_request", "lcmg_result",
                                  "lcmg_server_stats"])
def test_abi_structs_match_the_header_field_by_field(name):
    import ctypes as C
    want = _header_struct_fields(name)
    got = getattr(L, name)._fields_
    # a C field named after a Python keyword carries a trailing underscore
    assert [n for _, n in want] == [n.rstrip("_") for n, _ in got]
    cmap = {"int32_t": C.c_int32, "int64_t": C.c_int64, "double": C.c_double, "size_t": C.c_size_t,
            "ptr": C.c_void_p}
    for (t, n), (n2, ct) in zip(want, got):
        assert cmap[t] == ct, (name, n)


def test_default_params_write_exactly_the_struct():
    """The library fills sizeof(lcmg_params) bytes: guard bytes after the
    binding's struct stay untouched and the last fields hold their defaults."""
    import ctypes as C
    size = C.sizeof(L.lcmg_params)
    buf = (C.c_ubyte * (size + 64))(*([0xA5] * (size + 64)))
    L.lib().lcmg_default_params(C.cast(buf, C.POINTER(L.lcmg_params)))
    assert bytes(buf[size:]) == bytes([0xA5]) * 64
    p = L.lcmg_params.from_buffer(buf)
    assert (p.amg_coarse_max, p.compact_cols, p.alpha_fuse, p.beta_fuse, p.spmv_variant_at) == \
        (256, 1, 1, 1, 0)
