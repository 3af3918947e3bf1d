"""The allocation-free operator entry point, lcmg_apply_normal_noalloc.

Callers that cannot allocate device memory where they need the operator
(code under an external memory manager that owns the device memory, a
real-time loop that cannot pay an allocation's synchronisation) use this
entry point instead of a context.  Its only intermediate lives in a fixed
array of the library that every call shares, so the test makes two calls
in a row with different sizes and data and checks each result against the
context-based entry point lcmg_apply_normal_dev, within the 1e-13 relative
tolerance of the other operator parity tests.  It is collected last so a
run that stops at the first failure has already run every other test.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import problemgen as pg

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2306_11067_gb300 import lcmg as L  # noqa: E402
from paper_2306_11067_gb300 import Solver  # noqa: E402


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _dev_csr(A):
    """A and A^T as device CSR tensors with A's value type."""
    M = sp.csr_matrix((A.val, A.col, A.row_ptr), shape=(A.m, A.n))
    T = M.T.tocsr()
    T.sort_indices()
    cu = lambda a, dt: torch.tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")
    vt = torch.float32 if A.val.dtype == np.float32 else torch.float64
    return (cu(A.row_ptr, torch.int64), cu(A.col, torch.int32), cu(A.val, vt),
            cu(T.indptr.astype(np.int64), torch.int64), cu(T.indices.astype(np.int32), torch.int32),
            cu(T.data, vt))


def _context_apply(A, n_v, n_h, d, lams, X):
    s = Solver(n_v, n_h)
    s.set_forward_csr(A)
    s.set_weights(d)
    xd = torch.tensor(X, dtype=torch.float64, device="cuda")
    yd = torch.empty_like(xd)
    L.lcmg_apply_normal_dev(s.ctx, lams, xd, yd)
    out = yd.cpu().numpy()
    s.close()
    return out


@pytest.mark.parametrize("workload", ["ct", "blur_fp64"])
def test_noalloc_matches_context_apply_two_calls(workload):
    if workload == "ct":
        P = pg.make_problem("ct256", size=48)          # FP32 values
    else:
        P = pg.make_problem("deblur32_csr")            # FP64 values
    A, n_v, n_h = P.A, P.n_v, P.n_h
    n_edges = n_h * (n_v - 1) + (n_h - 1) * n_v
    d = pg.random_weights(n_edges, 3)
    rp, ci, va, rpT, ciT, vaT = _dev_csr(A)
    dd = torch.tensor(d, dtype=torch.float64, device="cuda")
    calls = [(np.array([1e-3, 0.3, 7.0]), pg.rng(5).standard_normal((3, P.n))),
             (np.array([0.05, 2.0]), pg.rng(6).standard_normal((2, P.n)))]
    for lams, X in calls:
        p = torch.tensor(X, dtype=torch.float64, device="cuda")
        q = torch.full_like(p, float("nan"))
        L.lcmg_apply_normal_noalloc(0, None, n_v, n_h, A.m, rp, ci, va, rpT, ciT, vaT, dd, lams, p, q)
        torch.cuda.synchronize()
        got = q.cpu().numpy()
        ref = _context_apply(A, n_v, n_h, d, lams, X)
        for j in range(len(lams)):
            assert _rel(got[j], ref[j]) <= 1e-13, (workload, lams[j], _rel(got[j], ref[j]))


def test_noalloc_rejects_sizes_beyond_the_scratch():
    P = pg.make_problem("ct256", size=48)
    A = P.A
    rp, ci, va, rpT, ciT, vaT = _dev_csr(A)
    d = torch.ones(P.n_h * (P.n_v - 1) + (P.n_h - 1) * P.n_v, dtype=torch.float64, device="cuda")
    # a declared row count with n_cols * m just above 2^19: rejected before
    # any pointer is read
    ncols = 2
    m_big = (1 << 18) + 1
    lams = np.full(ncols, 0.1)
    p = torch.zeros((ncols, P.n), dtype=torch.float64, device="cuda")
    q = torch.zeros_like(p)
    with pytest.raises(L.LcmgError) as e:
        L.lcmg_apply_normal_noalloc(0, None, P.n_v, P.n_h, m_big, rp, ci, va, rpT, ciT, vaT, d, lams, p, q)
    assert e.value.status == L.LCMG_ERR_INVALID_ARG
    assert "scratch" in L.lcmg_last_error()


def test_noalloc_allocates_no_device_memory():
    """After one call has loaded the library's device image on the GPU, two
    more calls leave the free device memory and the caching allocator's
    counters unchanged: nothing is allocated on the device."""
    P = pg.make_problem("ct256", size=48)
    A, n_v, n_h = P.A, P.n_v, P.n_h
    rp, ci, va, rpT, ciT, vaT = _dev_csr(A)
    d = torch.tensor(pg.random_weights(n_h * (n_v - 1) + (n_h - 1) * n_v, 3), dtype=torch.float64, device="cuda")
    lams = np.array([0.1, 1.0])
    p = torch.tensor(pg.rng(7).standard_normal((2, P.n)), dtype=torch.float64, device="cuda")
    q = torch.empty_like(p)
    L.lcmg_apply_normal_noalloc(0, None, n_v, n_h, A.m, rp, ci, va, rpT, ciT, vaT, d, lams, p, q)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_stats().get("allocation.all.allocated", 0)
    for _ in range(2):
        L.lcmg_apply_normal_noalloc(0, None, n_v, n_h, A.m, rp, ci, va, rpT, ciT, vaT, d, lams, p, q)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    alloc1 = torch.cuda.memory_stats().get("allocation.all.allocated", 0)
    assert free1 == free0
    assert alloc1 == alloc0


def test_noalloc_rejects_overlapping_p_and_q():
    P = pg.make_problem("ct256", size=48)
    A = P.A
    rp, ci, va, rpT, ciT, vaT = _dev_csr(A)
    d = torch.ones(P.n_h * (P.n_v - 1) + (P.n_h - 1) * P.n_v, dtype=torch.float64, device="cuda")
    buf = torch.zeros((3, P.n), dtype=torch.float64, device="cuda")
    with pytest.raises(L.LcmgError) as e:
        L.lcmg_apply_normal_noalloc(0, None, P.n_v, P.n_h, A.m, rp, ci, va, rpT, ciT, vaT, d, np.array([0.1, 1.0]),
                                    buf[0:2], buf[1:3])
    assert e.value.status == L.LCMG_ERR_INVALID_ARG
    assert "overlap" in L.lcmg_last_error()
