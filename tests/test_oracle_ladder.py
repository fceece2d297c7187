"""Pins for the oracle's failure-retry pieces (Software design section, ¶3: a
zone whose integration fails may be integrated again on its own under other
tolerances or with an approximate Jacobian): the forward-difference Jacobian and
the retry ladder. Each check is against something other than the code under
test -- a closed form, exactness on a linear system, published values, or the
oracle's plain burn."""
import os

import numpy as np
import pytest

import oracle
from mc_inputs import network_13, network_33, robertson_cells, robertson_network, synthetic_cells
from mc_inputs.networks import K_B_EV, Network

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
SQRT_EPS = np.sqrt(np.finfo(np.float64).eps)


def _fd_increment(y, rtol, atol):
    """The increment the forward difference is defined with: sqrt(eps) times
    (|y_j| + atol/rtol), taken as the difference actually represented."""
    d = SQRT_EPS * (np.abs(y) + atol / rtol)
    return (y + d) - y


def test_fd_jacobian_is_exact_on_a_linear_chain():
    """A -> B -> C: f = K y, so forward differences give K up to the cancellation
    of rounding in f: |J_ij - K_ij| <= c eps sum_k |K_ik y_k| / d_j. A wrong
    column, a transposed matrix or a wrong increment misses by O(1)."""
    z = np.zeros(2)
    net = Network(name="chain", n_species=3, n_elements=1, energy_eq=False,
                  react=np.array([[0, -1], [1, -1]], dtype=np.int32),
                  prod=np.array([[1, -1], [2, -1]], dtype=np.int32),
                  composition=np.ones((3, 1), dtype=np.int32),
                  A_f=np.array([1.0, 1000.0]), b_f=z.copy(), C_f=z.copy(),
                  A_r=z.copy(), b_r=z.copy(), C_r=z.copy(), dE_eV=z.copy())
    on = oracle.OracleNetwork(net)
    K = np.array([[-1.0, 0.0, 0.0], [1.0, -1000.0, 0.0], [0.0, 1000.0, 0.0]])
    rng = np.random.default_rng(0)
    eps = np.finfo(np.float64).eps
    for _ in range(5):
        y = rng.uniform(0.0, 1.0, 3)
        J = on.fd_jac(y)
        d = _fd_increment(y, 1e-6, 1e-10)
        terms = np.abs(K) @ np.abs(y) + np.abs(K) @ np.abs(d)
        bound = 8 * eps * terms[:, None] / d[None, :]
        assert np.all(np.abs(J - K) <= bound), (J - K) / bound


def test_fd_jacobian_error_on_robertson_is_half_the_curvature_times_the_increment():
    """Robertson's f is quadratic, so the forward difference is J + H_jj d_j / 2
    exactly: only the y2^2 terms (H = -+2 k2) leave an error, -+k2 d_2. This pins
    both the column orientation and the increment rule."""
    on = oracle.OracleNetwork(robertson_network())
    k1, k2, k3 = 0.04, 3.0e7, 1.0e4
    rtol, atol = 1e-6, 1e-10
    rng = np.random.default_rng(1)
    for _ in range(5):
        y = np.array([rng.uniform(0.5, 1.0), rng.uniform(1e-6, 4e-5), rng.uniform(0.0, 0.5)])
        Jx = np.array([[-k1, k3 * y[2], k3 * y[1]],
                       [k1, -k3 * y[2] - 2 * k2 * y[1], -k3 * y[1]],
                       [0.0, 2 * k2 * y[1], 0.0]])
        d = _fd_increment(y, rtol, atol)
        expected = Jx.copy()
        expected[1, 1] += -k2 * d[1]
        expected[2, 1] += k2 * d[1]
        J = on.fd_jac(y, rtol=rtol, atol=atol)
        scale = np.abs(Jx).max(axis=1, keepdims=True)
        assert np.all(np.abs(J - expected) <= 1e-7 * scale + 1e-12)
        # and the error term is really there (the increment is not zero or tiny)
        assert abs(J[1, 1] - Jx[1, 1]) > 0.5 * k2 * d[1]


@pytest.mark.parametrize("make", [network_13, network_33])
def test_fd_jacobian_agrees_with_the_analytic_one_on_energy_networks(make):
    net = make()
    on = oracle.OracleNetwork(net)
    cells = synthetic_cells(net, 6, seed=11)
    for c in range(6):
        xs = cells["x"][:, c]
        y = np.concatenate([xs, [xs.sum() * K_B_EV * cells["T"][c] / (net.gamma - 1.0)]])
        _, J = on.eval(y, ndens=cells["ndens"][c])
        Jf = on.fd_jac(y, ndens=cells["ndens"][c])
        scale = np.abs(J).max(axis=1, keepdims=True) + 1e-300
        assert np.max(np.abs(Jf - J) / scale) < 1e-4


def _golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


def test_robertson_with_fd_jacobian_reaches_the_reference_values():
    ref = {r[0]: (float(r[1]), float(r[2])) for r in _golden("robertson_t40.txt")}
    on = oracle.OracleNetwork(robertson_network())
    cells = robertson_cells(1, 1)
    cells["rate_scale"][:] = 1.0
    x, _, status, stats, rung = oracle.burn_ladder(
        on, cells, 40.0, [dict(rtol=1e-10, atol=1e-14, jac="fd")])
    assert status[0] == 0 and rung[0] == 0 and stats[4, 0] > 0
    for i, name in enumerate(("y1", "y2", "y3")):
        v, tol = ref[name]
        assert abs(x[i, 0] - v) <= tol
    assert abs(x[:, 0].sum() - 1.0) < 1e-13


def test_ladder_outputs_are_the_direct_burn_of_the_rung_that_gave_them():
    net = network_13()
    on = oracle.OracleNetwork(net)
    cells = synthetic_cells(net, 400, seed=3)
    rungs = [dict(max_steps=300), dict(max_steps=100000)]
    x, T, s, st, rung = oracle.burn_ladder(on, cells, 1e10, rungs)
    d0 = oracle.burn(on, cells, 1e10, max_steps=300)
    d1 = oracle.burn(on, cells, 1e10, max_steps=100000)
    retry = np.isin(d0[2], [1, 2, 3, 5])
    assert retry.any() and (~retry).any()
    np.testing.assert_array_equal(rung, retry.astype(np.int32))
    for out, a, b in zip((x, T, s, st), d0, d1):
        want = np.where(retry, b, a)
        np.testing.assert_array_equal(out, want)


def test_ladder_never_retries_rejected_inputs_and_leaves_them_untouched():
    net = network_13()
    on = oracle.OracleNetwork(net)
    cells = synthetic_cells(net, 4, seed=5)
    cells["T"][0] = -1.0
    cells["ndens"][1] = 0.0
    x, T, s, _, rung = oracle.burn_ladder(on, cells, 1e10, [dict(), dict(rtol=1e-4), dict(jac="fd")])
    assert list(s[:2]) == [4, 4] and list(rung[:2]) == [0, 0]
    np.testing.assert_array_equal(x[:, :2], cells["x"][:, :2])
    assert T[0] == -1.0
    assert (s[2:] == 0).all() and (rung[2:] == 0).all()


def test_ladder_rejects_bad_rung_lists():
    on = oracle.OracleNetwork(robertson_network())
    cells = robertson_cells(2, 1)
    with pytest.raises(ValueError):
        oracle.burn_ladder(on, cells, 40.0, [])
    with pytest.raises(ValueError):
        oracle.burn_ladder(on, cells, 40.0, [dict()] * 9)
    with pytest.raises(ValueError):
        oracle.burn_ladder(on, cells, 40.0, [dict(max_order=6)])
