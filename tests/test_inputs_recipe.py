"""The seeded input recipes stated for the workloads hold: network shapes,
rate-parameter ranges, element balance, cell distributions, hot fractions,
the mixed batch's split and the AMR-box request stream (CPU)."""
import numpy as np
import pytest

from mc_inputs import (box_request_stream, mixed_batch, network_13, network_33, robertson_cells,
                       synthetic_cells, synthetic_sources)


@pytest.mark.parametrize("make,S,E,R", [(network_13, 12, 3, 40), (network_33, 32, 4, 120)])
def test_network_shapes_ranges_and_balance(make, S, E, R):
    net = make()
    assert (net.n_species, net.n_elements, net.n_reactions, net.n_ode) == (S, E, R, S + 1)
    assert net.gamma == pytest.approx(5.0 / 3.0)
    for A in (net.A_f, net.A_r):
        assert np.all((A >= 1e-12) & (A <= 1e-8))
    for b in (net.b_f, net.b_r):
        assert np.all((b >= -1.0) & (b <= 1.0))
    for C in (net.C_f, net.C_r):
        assert np.all((C >= 0.0) & (C <= 5e4))
    assert np.all(np.abs(net.dE_eV) <= 5.0)
    comp = net.composition
    for r in range(R):
        lhs = sum(comp[s] for s in net.react[r] if s >= 0)
        rhs = sum(comp[s] for s in net.prod[r] if s >= 0)
        np.testing.assert_array_equal(lhs, rhs)
    # the same seed gives the same network
    again = make()
    np.testing.assert_array_equal(again.react, net.react)
    np.testing.assert_array_equal(again.A_f, net.A_f)


def test_cell_distributions():
    net = network_13()
    c = synthetic_cells(net, 200_000, seed=4)
    lt, ln = np.log10(c["T"]), np.log10(c["ndens"])
    assert lt.min() >= 1.0 and lt.max() <= 4.0 and abs(lt.mean() - 2.5) < 0.01
    assert ln.min() >= 0.0 and ln.max() <= 8.0 and abs(ln.mean() - 4.0) < 0.02
    np.testing.assert_allclose(c["x"].sum(axis=0), 1.0, rtol=1e-12)
    assert np.all(c["x"] >= 1e-6)
    hot = synthetic_cells(net, 200_000, seed=4, hot_fraction=0.01)
    frac = hot["hot"].mean()
    assert abs(frac - 0.01) < 0.001
    th = np.log10(hot["T"][hot["hot"]])
    assert th.min() >= 4.0 and th.max() <= 5.0


def test_robertson_rate_factors():
    c = robertson_cells(100_000, 1)
    f = np.log(c["rate_scale"])
    assert f.shape == (3, 100_000)
    assert f.min() >= np.log(0.5) and f.max() <= np.log(2.0) and abs(f.mean()) < 0.01
    np.testing.assert_array_equal(c["x"][:, 0], [1.0, 0.0, 0.0])


def test_mixed_batch_split_and_hot_cells():
    b = mixed_batch(300_000, seed=6, hot_fraction=0.01)
    counts = np.bincount(b["net_id"], minlength=3) / 300_000
    np.testing.assert_allclose(counts, 1 / 3, atol=0.005)
    covered = np.sort(np.concatenate([idx for _, _, idx in b["groups"]]))
    np.testing.assert_array_equal(covered, np.arange(300_000))
    for net, cells, idx in b["groups"][1:]:
        assert abs(cells["hot"].mean() - 0.01) < 0.002


def test_box_request_stream():
    reqs = box_request_stream(20_000, 2.0, seed=7, edge_range=(16, 128))
    L = np.array([r["edge"] for r in reqs])
    assert L.min() >= 16 and L.max() <= 128
    assert all(r["n_cells"] == r["edge"] ** 3 for r in reqs[:100])
    nets = np.array([r["net"] for r in reqs])
    assert abs((nets == "net13").mean() - 0.5) < 0.02
    gaps = np.diff([0.0] + [r["t_arrive"] for r in reqs])
    assert abs(gaps.mean() - 0.5) < 0.02 and abs(gaps.std() / gaps.mean() - 1.0) < 0.05  # exponential


def test_sources_scale_with_the_state():
    net = network_13()
    c = synthetic_cells(net, 10_000, seed=3)
    s = synthetic_sources(net, c, 1e10, seed=22, scale=0.05)
    assert s.shape == (net.n_ode, 10_000)
    assert np.all(np.abs(s[:-1] * 1e10) <= 0.05 * c["x"] + 1e-30)
    assert np.all(np.abs(s[-1] * 1e10) <= 0.05 * 1e-4 * c["T"] + 1e-30)
