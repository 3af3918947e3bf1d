"""The library's host-only calls against stored fixtures (tests/golden/,
written by tests/golden/make_golden.py from the oracle alone): the L-curve
corner (Sec. 1), Algorithm 2's lambda window (the paper's 30-lambda grid,
Sec. 4) and classical AMG's split and interpolation (Sec. 3.1).  Integer
results bit for bit; interpolation weights within 1e-14."""
import os

import numpy as np
import pytest
import scipy.sparse as sp

L = pytest.importorskip("paper_2306_11067_gb300.lcmg")
GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2306_11067_gb300 import build
    build.build()


def _lines(name):
    with open(os.path.join(GOLD, name)) as f:
        return [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]


def test_corners_match_fixture():
    rows = _lines("corners.txt")
    assert len(rows) == 30
    for r in rows:
        k = int(r[0])
        rho = np.array([float(v) for v in r[1:1 + k]])
        eta = np.array([float(v) for v in r[1 + k:1 + 2 * k]])
        assert L.lcmg_lcurve_corner(rho, eta) == int(r[1 + 2 * k])


def test_windows_match_fixture():
    rows = _lines("windows.txt")
    assert len(rows) == 31
    for i, lo, hi in ((int(a), int(b), int(c)) for a, b, c in rows):
        assert L.lcmg_cull_lambdas(30, i) == (lo, hi)


def test_rs_amg_matches_fixture():
    rec = {r[0]: r[1:] for r in _lines("rs_amg_12x10.txt")}
    n, nnz = int(rec["K"][0]), int(rec["K"][1])
    K = sp.csr_matrix((np.array([float(v) for v in rec["v"]]), np.array([int(v) for v in rec["ci"]]),
                       np.array([int(v) for v in rec["rp"]])), shape=(n, n))
    assert K.nnz == nnz
    cf = L.lcmg_rs_split(K)
    assert "".join(str(int(v)) for v in cf) == rec["cf"][0]
    rp, ci, v, nc = L.lcmg_rs_interp(K, cf)
    assert (n, nc, rp[-1]) == tuple(int(x) for x in rec["P"])
    assert np.array_equal(rp, np.array([int(x) for x in rec["prp"]]))
    assert np.array_equal(ci, np.array([int(x) for x in rec["pci"]]))
    assert np.abs(v - np.array([float(x) for x in rec["pv"]])).max() <= 1e-14
