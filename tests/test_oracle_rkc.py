"""Pins for the oracle's RKC integrator (explicit Runge-Kutta-Chebyshev of
order 2, Sommeijer, Shampine & Verwer 1998), the alternative integrator the
paper's network/integrator separation admits (Software design section, ¶4).
The stage recursion is checked against the method's closed-form stability
polynomial, built here independently from numpy's Chebyshev basis; the
adaptive integrator against closed forms and published values."""
import os

import numpy as np
import pytest
from numpy.polynomial import chebyshev as cheb

import oracle
from mc_inputs import network_13, robertson_cells, robertson_network, synthetic_cells

EPS = 2.0 / 13.0
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _closed_form(s):
    """P_s(z) = 1 - b_s T_s(w0) + b_s T_s(w0 + w1 z) and beta_s = (1 + w0)/w1."""
    Ts = cheb.Chebyshev.basis(s)
    d1, d2 = Ts.deriv(1), Ts.deriv(2)
    w0 = 1.0 + EPS / s ** 2
    w1 = d1(w0) / d2(w0)
    bs = d2(w0) / d1(w0) ** 2
    return (lambda z: 1.0 - bs * Ts(w0) + bs * Ts(w0 + w1 * z)), (1.0 + w0) / w1


@pytest.mark.parametrize("s", [2, 3, 5, 10, 40, 150])
def test_one_step_on_y_lambda_y_is_the_stability_polynomial(s):
    # rounding in the stage recursion grows like s^2 eps (internal stability of
    # the three-term recursion); a wrong coefficient misses by far more
    P, beta = _closed_form(s)
    for z in np.linspace(-beta, 0.2, 23):
        y = oracle.rkc_linear_step([[z]], [[0.0]], [1.0], 0.0, 1.0, s)
        assert abs(y[0] - P(z)) <= 1e-13 * s * s * max(1.0, abs(P(z)))


@pytest.mark.parametrize("s", [2, 7, 30])
def test_the_step_is_bounded_on_the_stability_interval(s):
    _, beta = _closed_form(s)
    assert 0.6 * (s * s - 1) < beta < 0.7 * s * s
    for z in np.linspace(-0.999 * beta, 0.0, 200):
        y = oracle.rkc_linear_step([[z]], [[0.0]], [1.0], 0.0, 1.0, s)
        assert abs(y[0]) <= 1.0 + 1e-12


@pytest.mark.parametrize("s", [2, 5, 20])
def test_local_error_is_third_order(s):
    """Order 2: y1 - exp(z) = O(z^3), so halving z divides the error by ~8."""
    errs = []
    for z in (-2e-2, -1e-2):
        y = oracle.rkc_linear_step([[z]], [[0.0]], [1.0], 0.0, 1.0, s)
        errs.append(abs(y[0] - np.exp(z)))
    assert 7.0 < errs[0] / errs[1] < 9.0


@pytest.mark.parametrize("s", [2, 4, 17])
def test_stage_times_integrate_linear_forcing_exactly(s):
    """y' = c0 + c1 t: an order-2 step with the right stage times is exact (up
    to rounding over the s stages); a wrong stage time misses by ~c1 h^2 dc."""
    c = [[0.3], [-1.7]]
    t, h = 0.4, 0.25
    y = oracle.rkc_linear_step([[0.0]], c, [2.0], t, h, s)
    exact = 2.0 + 0.3 * h - 1.7 * ((t + h) ** 2 - t ** 2) / 2.0
    assert abs(y[0] - exact) < 2e-15 * s * s


def test_vector_step_is_the_polynomial_of_the_matrix():
    rng = np.random.default_rng(2)
    Q = np.linalg.qr(rng.normal(size=(3, 3)))[0]
    lam = np.array([-3.0, -40.0, -0.5])
    A = Q @ np.diag(lam) @ Q.T
    s, h = 9, 0.8
    P, beta = _closed_form(s)
    assert (-lam * h < beta).all()
    y0 = np.array([1.0, -2.0, 0.5])
    y = oracle.rkc_linear_step(A, np.zeros((1, 3)), y0, 0.0, h, s)
    ref = Q @ (np.array([P(z) for z in lam * h]) * (Q.T @ y0))
    np.testing.assert_allclose(y, ref, rtol=1e-11, atol=1e-13)


@pytest.mark.parametrize("k1,k2", [(1.0, 1000.0), (2.0, 0.5)])
def test_adaptive_rkc_on_the_chain_closed_form(k1, k2):
    K = np.array([[-k1, 0.0, 0.0], [k1, -k2, 0.0], [0.0, k2, 0.0]])
    t1 = 3.0
    y, s, st = oracle.rkc_linear_integrate(K, np.zeros((1, 3)), [1.0, 0.0, 0.0], 0.0, t1, rtol=1e-8, atol=1e-14)
    a = np.exp(-k1 * t1)
    b = k1 / (k2 - k1) * (np.exp(-k1 * t1) - np.exp(-k2 * t1))
    assert s == 0
    # global error of an order-2 method whose local error is held at rtol
    np.testing.assert_allclose(y, [a, b, 1 - a - b], rtol=1e-5, atol=1e-7)
    y2, _, _ = oracle.rkc_linear_integrate(K, np.zeros((1, 3)), [1.0, 0.0, 0.0], 0.0, t1, rtol=1e-10, atol=1e-16)
    assert np.abs(y2 - [a, b, 1 - a - b]).max() < np.abs(y - [a, b, 1 - a - b]).max()
    if k2 == 1000.0:
        assert st[7] > 2          # the stiff rate forces more than two stages


def test_adaptive_rkc_error_tracks_the_tolerance():
    """Order 2 with the local error held at the tolerance: steps scale like
    tol^(1/3), so the global error scales like tol^(2/3) -- a factor ~21.5 per
    factor 100 of tolerance."""
    errs = []
    for rtol in (1e-4, 1e-6, 1e-8):
        y, s, _ = oracle.rkc_linear_integrate([[-1.0]], [[0.0]], [1.0], 0.0, 2.0, rtol=rtol, atol=rtol * 1e-4)
        assert s == 0
        errs.append(abs(y[0] - np.exp(-2.0)))
        assert errs[-1] < 10.0 * rtol ** (2.0 / 3.0)
    for a, b in zip(errs, errs[1:]):
        assert 10.0 < a / b < 40.0


def test_rkc_reaches_robertson_reference_values():
    ref = {}
    with open(os.path.join(GOLDEN, "robertson_t40.txt")) as f:
        for line in f:
            p = line.split()
            if p and not p[0].startswith("#"):
                ref[p[0]] = (float(p[1]), float(p[2]))
    on = oracle.OracleNetwork(robertson_network())
    cells = robertson_cells(1, 1)
    cells["rate_scale"][:] = 1.0
    x, _, s, st, _ = oracle.burn_ladder(on, cells, 40.0, [dict(method="rkc", rtol=1e-7, atol=1e-12)])
    assert s[0] == 0
    for i, name in enumerate(("y1", "y2", "y3")):
        v, tol = ref[name]
        assert abs(x[i, 0] - v) <= tol
    assert abs(x[:, 0].sum() - 1.0) < 1e-12


def test_rkc_on_network_cells_is_accurate_where_it_succeeds():
    """Against a tight BDF result: cells RKC finishes are accurate in
    distribution; the stiff ones stop at the step cap instead of returning a
    wrong state."""
    net = network_13()
    on = oracle.OracleNetwork(net)
    cells = synthetic_cells(net, 96, seed=3)
    x, T, s, _, _ = oracle.burn_ladder(on, cells, 1e10, [dict(method="rkc", max_steps=5000)])
    tx, tT, ts, _ = oracle.burn(on, cells, 1e10, rtol=1e-10, atol=1e-16)
    assert set(np.unique(s)) <= {0, 1}
    ok = (s == 0) & (ts == 0)
    assert ok.mean() > 0.7
    within = (np.abs(x - tx) <= 1e-3 * np.abs(tx) + 1e-7).all(axis=0)
    assert within[ok].mean() > 0.95
    assert np.max(np.abs(T - tT)[ok] / tT[ok]) < 1e-3
