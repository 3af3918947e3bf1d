"""Pins of the outer-loop ingredients (Sec. 1, 3.3-3.5, Algorithm 2).

* corner: a hyperbola sampled symmetrically about its vertex selects the
  vertex; an L made of two straight legs selects the joint; the sign
  convention (positive at the L-shaped corner for increasing lambda).
* update_weights (eq. (g)): a single vertical step edge gets d = d_min on
  exactly that column of horizontal edges; a ramp gives the closed form
  1 - (|v| / max|v|)^q; a constant image leaves D unchanged; the update is
  multiplicative in D.
* lambda_window: the formula of Algorithm 2 against the prose of Sec. 3.4
  (ten indices i-2 .. i+7, shifted to the smallest or largest ten near the
  ends), exhaustively for m in [10, 64].
* should_stop: three equal consecutive selections.
"""
import numpy as np
import pytest

import problemgen as pg
from oracle import operators as ops
from oracle import lcurve


def test_corner_hyperbola_vertex():
    # u v = 1 in log-log coordinates; u increases with lambda, v decreases
    for k in (3, 5, 7):
        t = 2.0 ** (np.arange(-k, k + 1) / 2.0)
        rho, eta = 10.0 ** t, 10.0 ** (1.0 / t)
        assert lcurve.corner(rho, eta) == k


def test_corner_two_legs_joint():
    # steep leg (u fixed, v falling) then flat leg (u rising, v fixed)
    u = np.array([0.0, 0.01, 0.02, 0.03, 0.5, 1.0, 1.5, 2.0])
    v = np.array([3.0, 2.0, 1.0, 0.0, -0.01, -0.02, -0.03, -0.04])
    assert lcurve.corner(10.0 ** u, 10.0 ** v) == 3


def test_corner_sign_and_fallback():
    # a curve that first runs flat and then falls steeply turns clockwise:
    # no positive curvature; the fallback still returns an interior point
    u = np.array([0.0, 1.0, 2.0, 2.01, 2.02])
    v = np.array([2.0, 1.99, 1.98, 1.0, 0.0])
    kap = lcurve.menger_curvature(10.0 ** u, 10.0 ** v)
    assert np.all(kap[1:-1] <= 0)
    assert 1 <= lcurve.corner(10.0 ** u, 10.0 ** v) <= 3


def test_corner_tie_goes_to_smaller_lambda():
    # a symmetric staircase with two identical corners
    u = np.array([0.0, 0.0, 1.0, 1.0, 2.0])
    v = np.array([2.0, 1.0, 1.0, 0.0, 0.0])
    kap = lcurve.menger_curvature(10.0 ** u, 10.0 ** v)
    assert kap[1] == pytest.approx(kap[3])
    assert lcurve.corner(10.0 ** u, 10.0 ** v) == 1


@pytest.mark.parametrize("q", [1.0, 2.0])
def test_update_weights_step_edge(q):
    n_v, n_h = 6, 5
    img = np.zeros((n_v, n_h))
    img[:, 3:] = 2.0                      # step between columns 2 and 3
    L = ops.gradient(n_v, n_h)
    d0 = np.ones(ops.n_edges(n_v, n_h))
    d = lcurve.update_weights(d0, L, pg.vec(img), q=q, d_min=1e-3)
    nvert = n_h * (n_v - 1)
    # horizontal edge (i, j)-(i, j+1) has index nvert + i + j n_v
    on_edge = np.zeros_like(d, dtype=bool)
    for i in range(n_v):
        on_edge[nvert + i + 2 * n_v] = True
    assert np.all(d[on_edge] == 1e-3)
    assert np.all(d[~on_edge] == 1.0)


@pytest.mark.parametrize("q", [1.0, 2.0, 0.5])
def test_update_weights_closed_form(q):
    n_v, n_h = 5, 4
    img = np.outer(np.array([0.0, 1.0, 3.0, 6.0, 10.0]), np.ones(n_h))   # diffs 1,2,3,4
    L = ops.gradient(n_v, n_h)
    d0 = np.full(ops.n_edges(n_v, n_h), 0.5)
    d = lcurve.update_weights(d0, L, pg.vec(img), q=q, d_min=1e-3)
    nvert = n_h * (n_v - 1)
    g = np.tile(np.array([1.0, 2.0, 3.0, 4.0]) / 4.0, n_h)
    expect = 0.5 * np.maximum(1.0 - g ** q, 1e-3)
    assert np.allclose(d[:nvert], expect, rtol=1e-15)
    assert np.all(d[nvert:] == 0.5)           # zero horizontal gradient: d = 1


def test_update_weights_constant_image_is_identity():
    L = ops.gradient(4, 4)
    d0 = pg.random_weights(ops.n_edges(4, 4), 1)
    assert np.array_equal(lcurve.update_weights(d0, L, np.full(16, 3.0)), d0)


def _window_from_prose(m, i):
    """Ten consecutive indices i-2 .. i+7 shifted to lie inside 1..m."""
    lo, hi = i - 2, i + 7
    if lo < 1:
        lo, hi = 1, 10
    if hi > m:
        lo, hi = m - 9, m
    return max(lo, 1), min(hi, m)


def test_lambda_window_exhaustive():
    for m in range(10, 65):
        assert lcurve.lambda_window(m, 0) == (1, m)
        for i in range(1, m + 1):
            lo, hi = lcurve.lambda_window(m, i)
            assert (lo, hi) == _window_from_prose(m, i)
            assert hi - lo + 1 == 10
            assert lo <= i <= hi or i < lo + 2


def test_lambda_window_examples():
    # m = 30 (the paper's lambda count)
    assert lcurve.lambda_window(30, 1) == (1, 10)
    assert lcurve.lambda_window(30, 12) == (10, 19)
    assert lcurve.lambda_window(30, 29) == (21, 30)
    assert lcurve.lambda_window(8, 5) == (1, 8)       # fewer than ten lambdas


def test_should_stop():
    assert lcurve.should_stop([3, 3, 3])
    assert not lcurve.should_stop([3, 4, 4])
    assert not lcurve.should_stop([2, 2])


def test_should_stop_lx_stops_at_the_first_decrease():
    assert not lcurve.should_stop_lx([5.0])
    assert not lcurve.should_stop_lx([5.0, 5.0])        # equal is not a decrease
    assert not lcurve.should_stop_lx([5.0, 6.0])
    assert lcurve.should_stop_lx([5.0, 6.0, 5.9])
    assert lcurve.should_stop_lx([5.0, 4.0])
    assert lcurve.should_stop([1, 2, 2, 2])
    assert not lcurve.should_stop([5, 5, 6, 6])


def test_weight_update_uses_the_current_weights_by_hand():
    """Eq. (g) on v = D^(l) L x: L x = (1, 0.8), D^(l) = diag(0.5, 1) give
    v = (0.5, 0.8), g = (0.625, 1), d = (1 - 0.625^2, d_min) and
    D^(l+1) = diag(d) D^(l) = (0.3046875, 0.001)."""
    import numpy as np
    from oracle import operators as ops
    L = ops.gradient(3, 1)                       # two vertical edges
    x = np.array([0.0, 1.0, 1.8])
    assert np.allclose(L @ x, [1.0, 0.8])
    d = lcurve.update_weights(np.array([0.5, 1.0]), L, x, q=2.0, d_min=1e-3)
    assert np.allclose(d, [0.3046875, 1e-3], rtol=1e-15, atol=0)
