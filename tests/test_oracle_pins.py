"""Pins for the CPU oracle: each test checks the oracle against something
other than itself -- published values, closed forms, invariants, brute force
or exact polynomial arithmetic -- so that a dropped term, a wrong sign or index
or a transposed operand in it fails one of them."""
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from mc_inputs import network_13, network_33, robertson_network, robertson_cells, synthetic_cells
from mc_inputs.networks import K_B_EV

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


# ---------------------------------------------------------------- coefficients
def test_constant_step_corrector_matches_gear_table():
    for row in _read_golden("gear_nordsieck_l.txt"):
        q = int(row[0])
        ref = np.array([float(Fraction(v)) for v in row[1:]])
        l, _ = oracle.bdf_coeffs(q, np.arange(1, q + 2, dtype=float))
        np.testing.assert_allclose(l / l[1], ref, rtol=1e-14)


def _interp_nordsieck(poly, t_pts, t0, h, q):
    """Nordsieck array at t0 (scale h) of the degree-q polynomial through
    (t_pts, poly(t_pts))."""
    P = np.polynomial.Polynomial.fit(t_pts, poly(t_pts), q, domain=[t_pts.min(), t_pts.max()]).convert()
    z = np.zeros((q + 1, 1))
    d = P
    fact = 1.0
    for j in range(q + 1):
        if j > 0:
            d = d.deriv()
            fact *= j
        z[j, 0] = h ** j * d(t0) / fact
    return z


def _poly_ode(y):
    """y' = p(t) with p = y', as (A, c) for the linear test ODE."""
    dp = y.deriv()
    c = np.zeros((max(len(dp.coef), 1), 1))
    c[: len(dp.coef), 0] = dp.coef
    return np.zeros((1, 1)), c


@pytest.mark.parametrize("q", [1, 2, 3, 4, 5])
def test_textbook_error_constants(q):
    """Constant steps, y = t^(q+1), exact back values: the step's true error
    equals C_q h^(q+1) y^(q+1) with the textbook C_q, and the oracle's
    constant-step error coefficient is that C_q."""
    Cq = {int(r[0]): float(Fraction(r[1])) for r in _read_golden("bdf_error_constants.txt")}[q]
    y = np.polynomial.Polynomial([0.0] * (q + 1) + [1.0])
    h, t0 = 0.1, 1.0
    pts = t0 - h * np.arange(q + 1)
    z = _interp_nordsieck(y, pts, t0, h, q)
    A, c = _poly_ode(y)
    z1, _, e, est = oracle.linear_fixed_steps(A, c, q, [h], t0, z, [h] * (q + 1))
    true_err = z1[0, 0] - y(t0 + h)
    deriv = float(np.prod(np.arange(1, q + 2)))  # y^(q+1) = (q+1)!
    assert true_err == pytest.approx(Cq * h ** (q + 1) * deriv, rel=1e-8)
    _, cq = oracle.bdf_coeffs(q, np.arange(1, q + 2, dtype=float))
    assert cq == pytest.approx(Cq, rel=1e-14)


@pytest.mark.parametrize("q", [1, 2, 3, 4, 5])
def test_error_estimate_exact_at_variable_steps(q):
    """Random past step sizes and a random degree-(q+1) solution: cq times the
    predictor's miss equals the true local error of one step from exact back
    values (the variable-coefficient formula)."""
    rng = np.random.default_rng(100 + q)
    y = np.polynomial.Polynomial(rng.uniform(-1, 1, q + 2))
    hist = rng.uniform(0.05, 0.3, q + 1)
    h, t0 = 0.17, 0.4
    pts = t0 - np.concatenate([[0.0], np.cumsum(hist[:q])])
    z = _interp_nordsieck(y, pts, t0, h, q)
    miss = y(t0 + h) - oracle.predict(z)[0, 0]
    A, c = _poly_ode(y)
    z1, _, e, est = oracle.linear_fixed_steps(A, c, q, [h], t0, z, hist)
    true_err = z1[0, 0] - y(t0 + h)
    assert est[0, 0] / e[0, 0] * miss == pytest.approx(true_err, rel=1e-7, abs=1e-14)


@pytest.mark.parametrize("q", [1, 2, 3, 4, 5])
def test_error_estimate_in_steady_running(q):
    """y' = y at constant steps: after 40 steps the estimate cq*e of the last
    step matches the true local error of a step from exact back values (to
    O(h); h is large enough that roundoff stays far below the error)."""
    h, m = 0.01, 40
    A, c = np.array([[1.0]]), np.zeros((1, 1))
    pts = -h * np.arange(q + 1)
    P = np.polynomial.Polynomial.fit(pts, np.exp(pts), q).convert()
    z = np.array([[h ** j * P.deriv(j)(0.0) / np.prod(np.arange(1, j + 1))] for j in range(q + 1)])
    _, _, e, est = oracle.linear_fixed_steps(A, c, q, [h] * m, 0.0, z, [h] * (q + 2))
    t1 = (m - 1) * h
    pts2 = t1 - h * np.arange(q + 1)
    P2 = np.polynomial.Polynomial.fit(pts2, np.exp(pts2), q).convert()
    z2 = np.array([[h ** j * P2.deriv(j)(t1) / np.prod(np.arange(1, j + 1))] for j in range(q + 1)])
    zz, _, _, _ = oracle.linear_fixed_steps(A, c, q, [h], t1, z2, [h] * (q + 2))
    true_err = zz[0, 0] - np.exp(t1 + h)
    assert est[m - 1, 0] / true_err == pytest.approx(1.0, abs=0.06)


@pytest.mark.parametrize("q", [1, 2, 3, 4, 5])
def test_polynomial_solutions_are_exact(q):
    """A solution of degree <= q is reproduced exactly by order q over a
    variable step sequence (all Nordsieck components)."""
    rng = np.random.default_rng(200 + q)
    y = np.polynomial.Polynomial(rng.uniform(-1, 1, q + 1))
    hs = rng.uniform(0.05, 0.4, 7)
    t0 = 0.3
    z = np.zeros((q + 1, 1))
    d, fact = y, 1.0
    for j in range(q + 1):
        if j:
            d, fact = d.deriv(), fact * j
        z[j, 0] = hs[0] ** j * d(t0) / fact
    A, c = _poly_ode(y)
    # one step at a time so the array can be rescaled to the next step size
    hist = list(rng.uniform(0.05, 0.4, q + 1))
    t = t0
    for k in range(len(hs)):
        z, h8, e, est = oracle.linear_fixed_steps(A, c, q, [hs[k]], t, z, hist)
        hist = list(h8[: q + 1])
        t += hs[k]
        assert z[0, 0] == pytest.approx(y(t), rel=1e-12, abs=1e-12)
        if k + 1 < len(hs):
            eta = hs[k + 1] / hs[k]
            z = z * (eta ** np.arange(q + 1))[:, None]
    assert z[1, 0] == pytest.approx(hs[-1] * y.deriv()(t), rel=1e-10, abs=1e-12)


@pytest.mark.parametrize("q", [2, 3, 4, 5])
def test_order_down_estimate_is_exact(q):
    """est_{q-1} = c * z_q (after an order-q step on a degree-q solution)
    equals the true error of an order q-1 step from exact back values."""
    rng = np.random.default_rng(300 + q)
    y = np.polynomial.Polynomial(rng.uniform(-1, 1, q + 1))
    hist = rng.uniform(0.05, 0.3, q + 1)
    h, t0 = 0.21, 0.5
    A, c = _poly_ode(y)
    pts = t0 - np.concatenate([[0.0], np.cumsum(hist[:q])])
    zq, h8, _, _ = oracle.linear_fixed_steps(A, c, q, [h], t0, _interp_nordsieck(y, pts, t0, h, q), hist)
    xi = np.cumsum(h8[:q]) / h
    est = oracle.err_coef_qm1(q, xi) * zq[q, 0]
    zl, _, _, _ = oracle.linear_fixed_steps(A, c, q - 1, [h], t0, _interp_nordsieck(y, pts[:q], t0, h, q - 1), hist)
    true_err = zl[0, 0] - y(t0 + h)
    assert est == pytest.approx(true_err, rel=1e-7, abs=1e-14)


@pytest.mark.parametrize("q", [1, 2, 3])
def test_order_up_estimate_converges(q):
    """est_{q+1} from two consecutive order-q corrections approaches the true
    error of an order q+1 step as h -> 0 (smooth solution y = exp(t)). The
    corrections are taken after 40 constant steps, once the sequence of
    corrections is smooth."""
    ratios = []
    A = np.array([[1.0]])
    c = np.zeros((1, 1))
    ex = np.exp
    for h in (0.02, 0.01):
        m = 40
        pts = -h * np.arange(q + 1)
        P = np.polynomial.Polynomial.fit(pts, ex(pts), q).convert()
        z = np.array([[h ** j * P.deriv(j)(0.0) / np.prod(np.arange(1, j + 1))] for j in range(q + 1)])
        _, _, e, _ = oracle.linear_fixed_steps(A, c, q, [h] * m, 0.0, z, [h] * (q + 2))
        est = oracle.err_coef_qp1(q) * (e[m - 1, 0] - e[m - 2, 0])
        # true error of an order q+1 step from exact back values, from t_m
        t1 = m * h
        pts2 = t1 - h * np.arange(q + 2)
        P2 = np.polynomial.Polynomial.fit(pts2, ex(pts2), q + 1).convert()
        z2 = np.array([[h ** j * P2.deriv(j)(t1) / np.prod(np.arange(1, j + 1))] for j in range(q + 2)])
        zz, _, _, _ = oracle.linear_fixed_steps(A, c, q + 1, [h], t1, z2, [h] * (q + 2))
        true_err = zz[0, 0] - ex(t1 + h)
        ratios.append(est / true_err)
    # a coefficient off by G_q/G_(q+1) (0.67, 0.82, 0.88) fails this
    assert abs(ratios[0] - 1.0) < 0.05 and abs(ratios[1] - 1.0) < 0.05


@pytest.mark.parametrize("q", [1, 2, 3, 4])
def test_order_raise_builds_the_next_interpolant(q):
    """After a step at order q, z + C * coefs(x prod(x + xi_i)) * e is the
    degree-(q+1) polynomial through the new value and q+1 back values."""
    rng = np.random.default_rng(400 + q)
    y = np.polynomial.Polynomial(rng.uniform(-1, 1, q + 3))
    hist = rng.uniform(0.05, 0.3, q + 2)
    h, t0 = 0.19, 0.2
    A, c = _poly_ode(y)
    pts = t0 - np.concatenate([[0.0], np.cumsum(hist[:q])])
    z1, h8, e, _ = oracle.linear_fixed_steps(A, c, q, [h], t0, _interp_nordsieck(y, pts, t0, h, q), hist)
    xi = np.cumsum(h8[: q + 1]) / h
    C = oracle.order_raise_coef(q, xi)
    co = oracle.order_lower_coefs(q + 1, xi)
    zr = np.zeros((q + 2, 1))
    zr[: q + 1] = z1
    zr[:, 0] += co * C * e[0, 0]
    t1 = t0 + h
    back = t1 - np.concatenate([[0.0], np.cumsum(h8[: q + 1])])
    vals = y(back)
    vals[0] = z1[0, 0]
    Q = np.polynomial.Polynomial.fit(back, vals, q + 1).convert()
    ref = np.array([h ** j * Q.deriv(j)(t1) / np.prod(np.arange(1, j + 1)) for j in range(q + 2)])
    np.testing.assert_allclose(zr[:, 0], ref, rtol=1e-7, atol=1e-10)


@pytest.mark.parametrize("q", [2, 3, 4, 5])
def test_order_lower_keeps_q_points(q):
    """Dropping a degree-q Nordsieck polynomial to degree q-1 gives the
    polynomial through the current point and the q-1 previous ones."""
    rng = np.random.default_rng(500 + q)
    P = np.polynomial.Polynomial(rng.uniform(-1, 1, q + 1))
    hist = rng.uniform(0.1, 0.4, q)
    h, t0 = 0.23, 0.0
    z = np.array([h ** j * P.deriv(j)(t0) / np.prod(np.arange(1, j + 1)) for j in range(q + 1)])
    xi = np.cumsum(hist) / h
    co = oracle.order_lower_coefs(q, xi)
    zl = z[:q] - co[:q] * z[q]
    back = t0 - np.concatenate([[0.0], np.cumsum(hist[: q - 1])])
    R = np.polynomial.Polynomial.fit(back, P(back), q - 1).convert()
    ref = np.array([h ** j * R.deriv(j)(t0) / np.prod(np.arange(1, j + 1)) for j in range(q)])
    np.testing.assert_allclose(zl, ref, rtol=1e-9, atol=1e-12)


def test_predict_is_taylor_shift_and_retract_undoes_it():
    rng = np.random.default_rng(7)
    q, h, t0 = 5, 0.3, 0.1
    P = np.polynomial.Polynomial(rng.uniform(-1, 1, q + 1))
    z = np.array([[h ** j * P.deriv(j)(t0) / np.prod(np.arange(1, j + 1))] for j in range(q + 1)])
    zp = oracle.predict(z)
    ref = np.array([h ** j * P.deriv(j)(t0 + h) / np.prod(np.arange(1, j + 1)) for j in range(q + 1)])
    np.testing.assert_allclose(zp[:, 0], ref, rtol=1e-12)
    np.testing.assert_allclose(oracle.retract(zp), z, rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("q", [1, 2, 3, 4, 5])
def test_empirical_order_on_linear_decay(q):
    """y' = -y at constant step from exact back values: global error at t = 1
    falls like h^q."""
    errs = []
    for nsteps in (40, 80):
        h = 1.0 / nsteps
        pts = -h * np.arange(q + 1)
        P = np.polynomial.Polynomial.fit(pts, np.exp(-pts), q).convert()
        z = np.array([[h ** j * P.deriv(j)(0.0) / np.prod(np.arange(1, j + 1))] for j in range(q + 1)])
        zz, _, _, _ = oracle.linear_fixed_steps(np.array([[-1.0]]), np.zeros((1, 1)), q, [h] * nsteps, 0.0, z, [h] * (q + 1))
        errs.append(abs(zz[0, 0] - np.exp(-1.0)))
    order = np.log2(errs[0] / errs[1])
    assert abs(order - q) < 0.25


# ---------------------------------------------------------------- integrator
def test_robertson_reference_values():
    ref = {r[0]: (float(r[1]), float(r[2])) for r in _read_golden("robertson_t40.txt")}
    on = oracle.OracleNetwork(robertson_network())
    cells = robertson_cells(1, 1)
    cells["rate_scale"][:] = 1.0
    x, _, status, _ = oracle.burn(on, cells, 40.0, rtol=1e-10, atol=1e-14)
    assert status[0] == 0
    for i, name in enumerate(("y1", "y2", "y3")):
        v, tol = ref[name]
        assert abs(x[i, 0] - v) <= tol
    # the invariant y1 + y2 + y3 = 1 holds to roundoff at any tolerance
    for rtol in (1e-4, 1e-6, 1e-10):
        x, _, _, _ = oracle.burn(on, cells, 40.0, rtol=rtol, atol=rtol * 1e-4)
        assert abs(x[:, 0].sum() - 1.0) < 1e-13


def test_robertson_error_tracks_tolerance():
    on = oracle.OracleNetwork(robertson_network())
    cells = robertson_cells(8, 1)
    tight, _, _, _ = oracle.burn(on, cells, 40.0, rtol=1e-12, atol=1e-18)
    loose, _, s, _ = oracle.burn(on, cells, 40.0, rtol=1e-6, atol=1e-10)
    assert (s == 0).all()
    rel = np.abs(loose - tight) / np.maximum(np.abs(tight), 1e-8)
    assert rel.max() < 2e-5


@pytest.mark.parametrize("k1,k2", [(1.0, 1000.0), (2.0, 2.0), (5.0, 0.3)])
def test_chain_closed_form(k1, k2):
    """A -> B -> C first-order chain against its closed form."""
    K = np.array([[-k1, 0.0, 0.0], [k1, -k2, 0.0], [0.0, k2, 0.0]])
    t1 = 3.0
    y, s, _ = oracle.linear_integrate(K, np.zeros((1, 3)), [1.0, 0.0, 0.0], 0.0, t1, rtol=1e-9, atol=1e-14)
    a = np.exp(-k1 * t1)
    if k1 == k2:
        b = k1 * t1 * np.exp(-k1 * t1)
    else:
        b = k1 / (k2 - k1) * (np.exp(-k1 * t1) - np.exp(-k2 * t1))
    ref = np.array([a, b, 1.0 - a - b])
    assert s == 0
    np.testing.assert_allclose(y, ref, rtol=2e-7, atol=1e-12)


def test_chain_as_reaction_network():
    """The same chain through the reaction-table right-hand side."""
    from mc_inputs.networks import Network
    z = np.zeros(2)
    net = Network(name="chain", n_species=3, n_elements=1, energy_eq=False,
                  react=np.array([[0, -1], [1, -1]], dtype=np.int32),
                  prod=np.array([[1, -1], [2, -1]], dtype=np.int32),
                  composition=np.ones((3, 1), dtype=np.int32),
                  A_f=np.array([1.0, 1000.0]), b_f=z.copy(), C_f=z.copy(),
                  A_r=z.copy(), b_r=z.copy(), C_r=z.copy(), dE_eV=z.copy())
    on = oracle.OracleNetwork(net)
    cells = {"x": np.array([[1.0], [0.0], [0.0]]), "T": None, "ndens": None, "rate_scale": None}
    x, _, s, _ = oracle.burn(on, cells, 3.0, rtol=1e-9, atol=1e-14)
    a = np.exp(-3.0)
    b = 1.0 / 999.0 * (np.exp(-3.0) - np.exp(-3000.0))
    np.testing.assert_allclose(x[:, 0], [a, b, 1 - a - b], rtol=2e-7, atol=1e-12)


def _robertson_f(y, k):
    return np.array([-k[0] * y[0] + k[2] * y[1] * y[2],
                     k[0] * y[0] - k[2] * y[1] * y[2] - k[1] * y[1] ** 2,
                     k[1] * y[1] ** 2])


def _robertson_J(y, k):
    return np.array([[-k[0], k[2] * y[2], k[2] * y[1]],
                     [k[0], -k[2] * y[2] - 2 * k[1] * y[1], -k[2] * y[1]],
                     [0.0, 2 * k[1] * y[1], 0.0]])


def test_robertson_rhs_and_jacobian_closed_form():
    on = oracle.OracleNetwork(robertson_network())
    rng = np.random.default_rng(3)
    for _ in range(5):
        y = rng.uniform(0, 1, 3)
        s = rng.uniform(0.5, 2, 3)
        k = np.array([0.04, 3e7, 1e4]) * s
        f, J = on.eval(y, rate_scale=s)
        np.testing.assert_allclose(f, _robertson_f(y, k), rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(J, _robertson_J(y, k), rtol=1e-12, atol=1e-12)


def _backward_euler(y0, k, t1, n):
    h = t1 / n
    y = np.array(y0, dtype=float)
    for _ in range(n):
        x = y.copy()
        for _ in range(20):
            G = x - y - h * _robertson_f(x, k)
            dx = np.linalg.solve(np.eye(3) - h * _robertson_J(x, k), -G)
            x += dx
            if np.abs(dx).max() < 1e-15:
                break
        y = x
    return y


@pytest.mark.parametrize("scale", [1.0, 0.6, 1.8])
def test_robertson_brute_force_backward_euler(scale):
    """Tiny-step backward Euler with Richardson extrapolation (a different
    method, written here in numpy) agrees with the oracle to its O(h^2)."""
    k = np.array([0.04, 3e7, 1e4]) * scale
    t1 = 0.5
    y1 = _backward_euler([1, 0, 0], k, t1, 2000)
    y2 = _backward_euler([1, 0, 0], k, t1, 4000)
    rich = 2 * y2 - y1
    on = oracle.OracleNetwork(robertson_network())
    cells = {"x": np.array([[1.0], [0.0], [0.0]]), "T": None, "ndens": None,
             "rate_scale": np.full((3, 1), scale)}
    x, _, s, _ = oracle.burn(on, cells, t1, rtol=1e-11, atol=1e-16)
    np.testing.assert_allclose(x[:, 0], rich, rtol=2e-6, atol=1e-12)
    # and the first-order BE error itself is visible (the comparison is sharp)
    assert np.abs(y1 - x[:, 0]).max() > 10 * np.abs(rich - x[:, 0]).max()


@pytest.mark.parametrize("make", [network_13, network_33])
def test_network_rhs_conserves_elements_and_energy(make):
    net = make()
    on = oracle.OracleNetwork(net)
    rng = np.random.default_rng(11)
    S = net.n_species
    for _ in range(4):
        x = rng.uniform(0.0, 1.0, S)
        T = np.exp(rng.uniform(np.log(50), np.log(2e4)))
        u = x.sum() * K_B_EV * T / (net.gamma - 1)
        f = on.eval(np.concatenate([x, [u]]), ndens=10 ** rng.uniform(0, 8), jac=False)
        scale = np.abs(f).max() + 1e-300
        assert np.abs(net.composition.T @ f[:S]).max() <= 1e-12 * scale
        assert abs(f[S] + net.species_energy_eV @ f[:S]) <= 1e-12 * scale * 10


def test_network_rhs_single_reaction_by_hand():
    """One reaction A + B <=> C + D with energy: every term of the right-hand
    side checked against the rate law written out here."""
    from mc_inputs.networks import Network
    net = Network(name="one", n_species=4, n_elements=2, energy_eq=True,
                  react=np.array([[0, 1]], dtype=np.int32), prod=np.array([[2, 3]], dtype=np.int32),
                  composition=np.array([[1, 0], [0, 2], [1, 1], [0, 1]], dtype=np.int32),
                  A_f=np.array([2e-10]), b_f=np.array([0.5]), C_f=np.array([300.0]),
                  A_r=np.array([5e-11]), b_r=np.array([-0.3]), C_r=np.array([1200.0]),
                  dE_eV=np.array([1.7]), gamma=5.0 / 3.0)
    on = oracle.OracleNetwork(net)
    x = np.array([0.3, 0.2, 0.4, 0.1])
    T, n = 800.0, 1e6
    u = x.sum() * K_B_EV * T / (2.0 / 3.0)
    f = on.eval(np.concatenate([x, [u]]), ndens=n, jac=False)
    kf = 2e-10 * T ** 0.5 * np.exp(-300.0 / T)
    kr = 5e-11 * T ** -0.3 * np.exp(-1200.0 / T)
    w = kf * n * x[0] * x[1] - kr * n * x[2] * x[3]
    np.testing.assert_allclose(f, [-w, -w, w, w, 1.7 * w], rtol=1e-12)


@pytest.mark.parametrize("make", [robertson_network, network_13, network_33])
def test_jacobian_matches_finite_differences(make):
    net = make()
    on = oracle.OracleNetwork(net)
    rng = np.random.default_rng(5)
    S = net.n_species
    for _ in range(3):
        x = rng.uniform(0.05, 1.0, S)
        if net.energy_eq:
            T = np.exp(rng.uniform(np.log(200), np.log(2e4)))
            y = np.concatenate([x, [x.sum() * K_B_EV * T / (net.gamma - 1)]])
            nd = 10 ** rng.uniform(0, 6)
        else:
            y, nd = x, 1.0
        f, J = on.eval(y, ndens=nd)
        Jfd = np.zeros_like(J)
        for j in range(y.size):
            d = 1e-6 * max(abs(y[j]), 1e-3)
            yp, ym = y.copy(), y.copy()
            yp[j] += d
            ym[j] -= d
            Jfd[:, j] = (on.eval(yp, ndens=nd, jac=False) - on.eval(ym, ndens=nd, jac=False)) / (2 * d)
        scale = np.abs(J).max()
        np.testing.assert_allclose(J, Jfd, rtol=1e-5, atol=1e-7 * scale)


@pytest.mark.parametrize("make", [network_13, network_33])
def test_burn_conserves_elements_and_energy(make):
    """Element totals and total energy (thermal + chemical) are linear
    invariants of the energy-form state; the BDF step keeps them up to the
    roundoff of each linear solve (backward error ~ eps |L||U| |delta|, larger
    for stiffer cells), so the drift is bounded per step, not absolutely: a
    dropped or mis-signed term drifts by 1e-6 or more."""
    net = make()
    on = oracle.OracleNetwork(net)
    cells = synthetic_cells(net, 128, seed=21)
    x, T, s, st = oracle.burn(on, cells, 1e10, max_steps=20000)
    ok = s == 0
    assert ok.sum() >= 120
    x0, T0 = cells["x"], cells["T"]
    el0 = net.composition.T @ x0
    el1 = net.composition.T @ x
    drift = (np.abs(el1 - el0) / np.abs(el0)).max(axis=0)[ok]
    steps = st[0][ok]
    assert np.median(drift) < 1e-14
    assert np.mean(drift < 1e-12) >= 0.95
    assert (drift <= 1e-13 * steps).all()
    eps = net.species_energy_eV
    E0 = x0.sum(0) * K_B_EV * T0 / (net.gamma - 1) + eps @ x0
    E1 = x.sum(0) * K_B_EV * T / (net.gamma - 1) + eps @ x
    scale = np.abs(eps) @ np.abs(x0) + x0.sum(0) * K_B_EV * T0
    de = (np.abs(E1 - E0) / scale)[ok]
    assert np.median(de) < 1e-14
    assert np.mean(de < 1e-12) >= 0.95
    assert (de <= 1e-13 * steps).all()


def test_failure_paths_report_status():
    on = oracle.OracleNetwork(network_13())
    cells = synthetic_cells(network_13(), 4, seed=3)
    cells["T"] = cells["T"].copy()
    cells["T"][0] = -5.0
    cells["T"][1] = np.nan
    _, _, s, _ = oracle.burn(on, cells, 1e10)
    assert s[0] == 4 and s[1] == 4
    _, _, s, st = oracle.burn(on, synthetic_cells(network_13(), 4, seed=3), 1e10, max_steps=3)
    assert (s == 1).all() and (st[0] <= 3).all()


# ---------------------------------------------------------------- LU
def test_lu_against_definition_and_solve():
    rng = np.random.default_rng(9)
    for n in (3, 13, 33):
        A = rng.normal(size=(n, n))
        lu, piv, rc = oracle.lu_factor(A)
        assert rc == 0
        L = np.tril(lu, -1) + np.eye(n)
        U = np.triu(lu)
        PA = A.copy()
        for k in range(n):
            PA[[k, piv[k]]] = PA[[piv[k], k]]
        np.testing.assert_allclose(L @ U, PA, rtol=1e-12, atol=1e-12)
        b = rng.normal(size=n)
        np.testing.assert_allclose(oracle.lu_solve(lu, piv, b), np.linalg.solve(A, b), rtol=1e-9)


def test_lu_pivot_ties_take_the_first_row():
    A = np.array([[1.0, 2.0, 0.0], [-3.0, 1.0, 1.0], [3.0, 0.0, 2.0]])
    _, piv, _ = oracle.lu_factor(A)
    assert piv[0] == 1
    _, _, rc = oracle.lu_factor(np.array([[1.0, 2.0], [2.0, 4.0]]))
    assert rc == 1


# ---------------------------------------------------------------- starting step
def test_starting_step_closed_form_on_scalar_problems():
    """Hairer, Norsett & Wanner's starting step (Solving ODEs I, II.4) with
    p = 1 on y' = lam y, worked by hand. With w = rtol |y0| + atol:
    d0 = |y0|/w, d1 = |lam y0|/w, h0 = 0.01 d0/d1 = 0.01/|lam| (both norms
    above 1e-5), the Euler trial gives d2 = |f(y0 + h0 f0) - f0|/(w h0)
    = lam^2 |y0|/w, and h = min(100 h0, sqrt(0.01 / max(d1, d2)), span)."""
    # lam = -1000, y0 = 1: w = 1.0001e-6, d2 = 1e6/w dominates, h = sqrt(0.01 w / 1e6)
    h = oracle.linear_initial_step([[-1000.0]], [1.0])
    assert abs(h / np.sqrt(1.0001e-14) - 1) < 1e-14
    # lam = -0.5, y0 = 2: w = 2.0001e-6, d1 = 1/w exceeds d2 = 0.5/w,
    # h = sqrt(0.01 w) = sqrt(2.0001e-8) < 100 h0 = 2
    h = oracle.linear_initial_step([[-0.5]], [2.0])
    assert abs(h / np.sqrt(2.0001e-8) - 1) < 1e-14
    # the span clips h0 and then h
    h = oracle.linear_initial_step([[-1000.0]], [1.0], span=1e-8)
    assert h == 1e-8
    # y0 = 0: both norms vanish, h0 = 1e-6, and with d1 = d2 = 0 the rule takes
    # max(1e-6, 1e-3 h0) = 1e-6
    h = oracle.linear_initial_step([[-3.0]], [0.0])
    assert h == 1e-6


def test_starting_step_on_a_diagonal_system():
    """Two decoupled modes lam = (-1000, -1), y0 = (1, 1): the WRMS norms are
    the root-mean-squares of the two components, d1 = sqrt((1e6 + 1)/2)/w,
    d2 = sqrt((1e12 + 1)/2)/w, h0 = 0.01 sqrt(2/(1e6 + 1))."""
    w = 1.0001e-6
    h0 = 0.01 * np.sqrt(2.0 / (1e6 + 1.0))
    h1 = np.sqrt(0.01 * w / np.sqrt((1e12 + 1.0) / 2.0))
    h = oracle.linear_initial_step(np.diag([-1000.0, -1.0]), [1.0, 1.0])
    assert abs(h / min(100 * h0, h1) - 1) < 1e-13


# ---------------------------------------------------------------- Newton
def test_newton_with_a_current_matrix_is_exact_on_a_linear_problem():
    """For y' = A y the corrector equation h A (z0 + e) - z1 - l1 e = 0 is
    linear, and P = I - (h/l1) A is its exact Jacobian divided by -l1: the
    first modified-Newton correction from e = 0 is the solution
    e* = (l1 I - h A)^-1 (h A z0 - z1), and the second finds nothing left."""
    A = np.array([[-1000.0, 1.0, 0.0], [2.0, -3.0, 0.5], [0.0, 40.0, -7.0]])
    z0 = np.array([1.0, 0.5, 0.25])
    z1 = np.array([0.3, -0.2, 0.1])
    for l1, h in ((1.0, 0.01), (1.5, 0.02)):
        want = np.linalg.solve(l1 * np.eye(3) - h * A, h * A @ z0 - z1)
        tr, res = oracle.linear_newton(A, z0, z1, l1, h, 1.0, w=np.full(3, 1e-30))
        np.testing.assert_allclose(tr[0], want, rtol=1e-13, atol=1e-16)
        np.testing.assert_allclose(tr[1], want, rtol=1e-13, atol=1e-16)
        # loose weights: the first correction already passes the convergence test
        tr, res = oracle.linear_newton(A, z0, z1, l1, h, 1.0, w=np.full(3, 1e6))
        assert res == 0 and tr.shape[0] == 1


def test_stale_matrix_correction_contracts_at_its_closed_form_rate():
    """Scalar y' = lam y with the matrix formed at gamma_P = r gamma: each
    correction delta = c (1 - gamma_P lam)^-1 [(h lam (z0 + e) - z1)/l1 - e],
    c = 2 / (1 + gamma/gamma_P), so the error e - e* is multiplied by
    rho = 1 - c (1 - gamma lam) / (1 - gamma_P lam) and e_k = e* (1 - rho^k).
    With lam = -1e4, h = 0.01, l1 = 1 (gamma lam = -100): r = 1.2 gives
    c = 12/11, rho = 1 - (12/11)(101/121) = 119/1331; r = 0.8 gives c = 8/9,
    rho = 1 - (8/9)(101/81) = -79/729. Tiny weights keep the convergence test
    from stopping the three corrections."""
    lam, h, l1, z0, z1 = -1e4, 0.01, 1.0, 0.7, -0.2
    e_star = (h * lam * z0 - z1) / (l1 - h * lam)
    for r, rho in ((1.2, 119.0 / 1331.0), (0.8, -79.0 / 729.0)):
        tr, res = oracle.linear_newton([[lam]], [z0], [z1], l1, h, r, w=[1e-30])
        assert res == 1 and tr.shape[0] == 3
        for k in range(3):
            assert abs(tr[k, 0] - e_star * (1 - rho ** (k + 1))) <= 1e-14 * abs(e_star)


def _settled_estimate(log, k0, settle):
    """Error estimates of the accepted steps from k0 + settle on, up to the
    next step change (or the last step before the clipped final one)."""
    h, E = log[:, 1], log[:, 3]
    k1 = k0 + 1
    while k1 < len(h) - 1 and abs(h[k1] / h[k0] - 1.0) < 1e-12:
        k1 += 1
    return E[k0 + settle:k1]


def test_step_size_rule_targets_the_bias_at_order_one():
    """The step-size rule aims the next step's error estimate at 1/BIAS_q of
    the tolerance: a local error that scales as h^(q+1) and a new step of
    h (BIAS E)^(-1/(q+1)) leave E' = 1/BIAS. On y' = -y with order 1 (the
    error in the error-test norm, with weights rtol |y|, then stays constant
    from step to step) the estimates after the first step change must sit at
    1/6 once the step history holds the new step only."""
    y, s, st, log = oracle.linear_integrate_steps(np.array([[-1.0]]), np.zeros((1, 1)), [1.0], 0.0, 5.0,
                                                  rtol=1e-6, atol=1e-14, max_order=1)
    assert s == 0 and np.all(log[:, 2] == 1)
    h = log[:, 1]
    changes = [k for k in range(1, len(h) - 1) if abs(h[k] / h[k - 1] - 1.0) > 1e-12]
    assert changes, "no step change to check"
    k0 = changes[0]
    eta = h[k0] / h[k0 - 1]
    assert 1.5 <= eta < 1e4  # a change neither below the threshold nor at the first-change cap
    E = _settled_estimate(log, k0, 1)
    assert len(E) > 100
    np.testing.assert_allclose(E, 1.0 / 6.0, rtol=2e-3)


def test_order_raise_targets_the_raised_bias():
    """An order raise is taken with the order-(q+1) estimate and its own bias
    (10) and exponent 1/(q+2): once the history has settled at the new order,
    the order-2 estimates of y' = -y sit at 1/10."""
    y, s, st, log = oracle.linear_integrate_steps(np.array([[-1.0]]), np.zeros((1, 1)), [1.0], 0.0, 5.0,
                                                  rtol=1e-6, atol=1e-14, max_order=2)
    assert s == 0
    h, q = log[:, 1], log[:, 2]
    raises = [k for k in range(1, len(h) - 1) if q[k] == 2 and q[k - 1] == 1]
    assert raises, "no order raise"
    k0 = raises[0]
    assert abs(h[k0] / h[k0 - 1] - 1.0) > 1e-12  # the raise came with a step change
    E = _settled_estimate(log, k0, 8)
    assert len(E) > 100
    np.testing.assert_allclose(E, 1.0 / 10.0, rtol=1e-2)
