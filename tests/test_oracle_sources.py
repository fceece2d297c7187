"""Pins for the oracle's constant source terms: the coupling of a burn to a
hydrodynamics step by spectral deferred corrections (Software design section,
¶4) integrates dy/dt = f(y) + s with s constant over the step. Each check is
against a closed form or an invariant, not against the oracle itself."""
import dataclasses

import numpy as np
import pytest
from scipy.linalg import expm

import oracle
from mc_inputs import network_13, synthetic_cells
from mc_inputs.networks import K_B_EV, Network


def _chain(k1, k2):
    z = np.zeros(2)
    return Network(name="chain", n_species=3, n_elements=1, energy_eq=False,
                   react=np.array([[0, -1], [1, -1]], dtype=np.int32),
                   prod=np.array([[1, -1], [2, -1]], dtype=np.int32),
                   composition=np.ones((3, 1), dtype=np.int32),
                   A_f=np.array([k1, k2], dtype=np.float64), b_f=z.copy(), C_f=z.copy(),
                   A_r=z.copy(), b_r=z.copy(), C_r=z.copy(), dE_eV=z.copy())


def test_source_alone_gives_the_straight_line():
    """All rates zero: y(t) = y0 + s t, which the BDF method integrates exactly."""
    on = oracle.OracleNetwork(_chain(0.0, 0.0))
    x0 = np.array([[0.5, 0.2], [0.3, 0.1], [0.2, 0.7]])
    s = np.array([[1e-3, -2e-3], [-4e-4, 1e-3], [2e-4, 5e-4]])
    cells = {"x": x0, "T": None, "ndens": None, "rate_scale": None}
    x, _, st, _ = oracle.burn(on, cells, 50.0, rtol=1e-8, atol=1e-14, source=s)
    assert (st == 0).all()
    np.testing.assert_allclose(x, x0 + 50.0 * s, rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("k1,k2", [(1.0, 1000.0), (2.0, 0.5)])
def test_chain_with_source_against_the_matrix_exponential(k1, k2):
    """y' = K y + s: [y(t); 1] = exp(t [[K, s], [0, 0]]) [y0; 1]."""
    on = oracle.OracleNetwork(_chain(k1, k2))
    K = np.array([[-k1, 0.0, 0.0], [k1, -k2, 0.0], [0.0, k2, 0.0]])
    s = np.array([0.3, -0.05, 0.01])
    y0 = np.array([1.0, 0.0, 0.0])
    t1 = 3.0
    M = np.zeros((4, 4))
    M[:3, :3] = K
    M[:3, 3] = s
    ref = (expm(t1 * M) @ np.concatenate([y0, [1.0]]))[:3]
    cells = {"x": y0[:, None].copy(), "T": None, "ndens": None, "rate_scale": None}
    x, _, st, _ = oracle.burn(on, cells, t1, rtol=1e-9, atol=1e-14, source=s[:, None])
    assert st[0] == 0
    np.testing.assert_allclose(x[:, 0], ref, rtol=2e-7, atol=1e-12)


def test_energy_form_with_source_and_no_reactions():
    """Rates zero in the energy form: x and u move on straight lines, and T
    comes out of the ideal-gas inversion of the final state."""
    net = network_13()
    R = net.A_f.size
    quiet = dataclasses.replace(net, A_f=np.zeros(R), A_r=np.zeros(R))
    on = oracle.OracleNetwork(quiet)
    cells = synthetic_cells(net, 5, seed=7)
    S, dt = net.n_species, 1e4
    rng = np.random.default_rng(3)
    src = np.zeros((S + 1, 5))
    src[:S] = rng.uniform(-1e-6, 1e-6, (S, 5)) * cells["x"] / dt
    X0 = cells["x"].sum(axis=0)
    u0 = X0 * K_B_EV * cells["T"] / (net.gamma - 1.0)
    src[S] = rng.uniform(-0.3, 0.3, 5) * u0 / dt
    x, T, st, _ = oracle.burn(on, cells, dt, rtol=1e-9, atol=1e-16, source=src)
    assert (st == 0).all()
    x_ref = cells["x"] + dt * src[:S]
    u_ref = u0 + dt * src[S]
    T_ref = (net.gamma - 1.0) * u_ref / (K_B_EV * x_ref.sum(axis=0))
    np.testing.assert_allclose(x, x_ref, rtol=1e-12, atol=0)
    np.testing.assert_allclose(T, T_ref, rtol=1e-12)


def test_zero_source_is_the_plain_burn():
    net = network_13()
    on = oracle.OracleNetwork(net)
    cells = synthetic_cells(net, 64, seed=3)
    a = oracle.burn(on, cells, 1e10)
    b = oracle.burn(on, cells, 1e10, source=np.zeros((net.n_ode, 64)))
    for u, v in zip(a, b):
        np.testing.assert_array_equal(u, v)


def test_element_neutral_source_keeps_element_totals():
    """Reactions keep every element total; a source that moves atoms between
    species of the same composition (C^T s = 0) must keep them too."""
    net = network_13()
    on = oracle.OracleNetwork(net)
    C = net.composition.astype(np.float64)              # [S, E]
    cells = synthetic_cells(net, 32, seed=9)
    S = net.n_species
    # pairs of species with equal composition, or else a species and its atoms
    src = np.zeros((S + 1, 32))
    rng = np.random.default_rng(5)
    mono = [int(np.flatnonzero((net.composition == np.eye(net.n_elements, dtype=np.int32)[e]).all(axis=1))[0])
            for e in range(net.n_elements)]
    for c in range(32):
        j = int(rng.integers(0, S))
        rate = 1e-12 * rng.uniform(0.5, 1.0)
        src[j, c] -= rate                                 # take one molecule of species j ...
        for e in range(net.n_elements):
            src[mono[e], c] += rate * C[j, e]             # ... and return its atoms
    assert np.allclose(C.T @ src[:S], 0.0, atol=1e-24)
    x, _, st, _ = oracle.burn(on, cells, 1e10, source=src)
    ok = st == 0
    assert ok.mean() > 0.9
    e0 = C.T @ cells["x"]
    e1 = C.T @ x
    assert np.max(np.abs(e1 - e0)[:, ok] / np.abs(e0[:, ok])) < 1e-10
