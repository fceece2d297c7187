"""Parity of the CUDA burn (through the C ABI) with the CPU FP64 oracle."""
import numpy as np
import pytest

import oracle
from mc_inputs import network_13, network_33, robertson_cells, robertson_network, synthetic_cells
from parity import classify, compare

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mc():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2608_06466_b300 as mc
    return mc


def _run(mc, net, cells, dt, **opt):
    h = mc.Network(net)
    o = mc.mc_burn_opts_default(**opt)
    return mc.burn(h, cells, dt, o)


def _oracle(net, cells, dt, **kw):
    return oracle.burn(oracle.OracleNetwork(net), cells, dt, **kw)


def _reference(net, cells, dt, index=None):
    """Oracle result, stability mask and tight-tolerance oracle result."""
    on = oracle.OracleNetwork(net)
    (ox, oT, os_, ost), stable = classify(on, cells, dt, oracle.burn, index=index)
    tx, tT, _, _ = oracle.burn(on, cells, dt, rtol=1e-10, atol=1e-16, index=index)
    return ox, oT, os_, ost, stable, (tx, tT)


@pytest.mark.parametrize("variant", [1, 2])
@pytest.mark.parametrize("lu", [64, 32])
def test_robertson_4096(mc, variant, lu):
    net, cells = robertson_network(), robertson_cells(4096, 1)
    gx, gT, gs, gst = _run(mc, net, cells, 40.0, variant=variant, lu_precision=lu)
    ox, oT, os_, ost = _oracle(net, cells, 40.0)
    rep = compare(gx, gT, gs, ox, oT, os_, ost)
    print(rep)
    assert rep["pass"], rep
    assert (gs == 0).all()
    if lu == 64:
        # same algorithm, same decisions: step counts agree on nearly every cell
        assert np.mean(gst[0] == ost[0]) > 0.95


@pytest.mark.parametrize("make,n", [(network_13, 4096), (network_33, 1024)])
@pytest.mark.parametrize("lu", [64, 32])
def test_synthetic_networks(mc, make, n, lu):
    net = make()
    cells = synthetic_cells(net, n, seed=3)
    gx, gT, gs, gst = _run(mc, net, cells, 1e10, lu_precision=lu)
    ox, oT, os_, ost, stable, tight = _reference(net, cells, 1e10)
    rep = compare(gx, gT, gs, ox, oT, os_, ost, stable=stable, tight=tight)
    print(net.name, lu, rep, "same step count:", np.mean(gst[0] == ost[0]))
    assert rep["pass"], rep
    assert rep["stable"] >= 0.9 * n


def test_full_size_sampled(mc):
    """2^20 cells of the 13-ODE network in the default (benchmark) launch
    configuration; 512 sampled cells recomputed by the oracle."""
    net = network_13()
    cells = synthetic_cells(net, 1 << 20, seed=3)
    gx, gT, gs, gst = _run(mc, net, cells, 1e10)
    idx = np.sort(np.random.default_rng(0).choice(1 << 20, 512, replace=False))
    ox, oT, os_, ost, stable, tight = _reference(net, cells, 1e10, index=idx)
    rep = compare(gx[:, idx], gT[idx], gs[idx], ox, oT, os_, ost, stable=stable, tight=tight)
    print(rep)
    assert rep["pass"], rep
    assert np.mean(gs == 0) > 0.99


@pytest.mark.parametrize("variant", [1, 2])
def test_ragged_and_degenerate_sizes(mc, variant):
    net = network_13()
    h = mc.Network(net)
    for n in (1, 37, 129):
        cells = synthetic_cells(net, n, seed=11)
        gx, gT, gs, gst = mc.burn(h, cells, 1e10, mc.mc_burn_opts_default(variant=variant))
        ox, oT, os_, ost, stable, tight = _reference(net, cells, 1e10)
        rep = compare(gx, gT, gs, ox, oT, os_, ost, stable=stable, tight=tight)
        assert rep["pass"], (n, rep)
    # zero cells is a no-op
    import torch
    x = torch.zeros((12, 0), dtype=torch.float64, device="cuda")
    mc.mc_burn_batch(h, None, 0, 1e10, x, 0, x, None, None, x, None)


def test_leading_dimension_larger_than_count(mc):
    import torch
    net = network_13()
    h = mc.Network(net)
    cells = synthetic_cells(net, 100, seed=12)
    ld = 160
    x = torch.zeros((12, ld), dtype=torch.float64, device="cuda")
    x[:, :100] = torch.as_tensor(cells["x"])
    x[:, 100:] = 7.0
    T = torch.full((ld,), 3.0, dtype=torch.float64, device="cuda")
    T[:100] = torch.as_tensor(cells["T"])
    nd = torch.ones(ld, dtype=torch.float64, device="cuda")
    nd[:100] = torch.as_tensor(cells["ndens"])
    st = torch.full((ld,), -9, dtype=torch.int32, device="cuda")
    mc.mc_burn_batch(h, None, 100, 1e10, x, ld, T, nd, None, st, None)
    torch.cuda.synchronize()
    assert (x[:, 100:] == 7.0).all() and (T[100:] == 3.0).all() and (st[100:] == -9).all()
    ox, oT, os_, ost, stable, tight = _reference(net, cells, 1e10)
    rep = compare(x[:, :100].cpu().numpy(), T[:100].cpu().numpy(), st[:100].cpu().numpy(), ox, oT, os_, ost,
                  stable=stable, tight=tight)
    assert rep["pass"], rep


def test_bad_inputs_and_step_cap(mc):
    net = network_13()
    cells = synthetic_cells(net, 8, seed=13)
    cells["x"] = cells["x"].copy()
    cells["T"] = cells["T"].copy()
    cells["ndens"] = cells["ndens"].copy()
    cells["x"][0, 0] = np.nan
    cells["T"][1] = -1.0
    cells["ndens"][2] = 0.0
    cells["T"][3] = np.inf
    gx, gT, gs, gst = _run(mc, net, cells, 1e10)
    ox, oT, os_, ost, stable, tight = _reference(net, cells, 1e10)
    assert list(gs[:4]) == [4, 4, 4, 4] and list(os_[:4]) == [4, 4, 4, 4]
    np.testing.assert_array_equal(gT[1], -1.0)  # rejected cells are left untouched
    rep = compare(gx, gT, gs, ox, oT, os_, ost, stable=stable, tight=tight)
    assert rep["pass"], rep
    gx, gT, gs, gst = _run(mc, net, synthetic_cells(net, 64, seed=14), 1e10, max_steps=7)
    ox, oT, os_, ost = _oracle(net, synthetic_cells(net, 64, seed=14), 1e10, max_steps=7)
    np.testing.assert_array_equal(gs, os_)
    assert (gs == 1).any()
    np.testing.assert_allclose(gx, ox, rtol=1e-9, atol=1e-15)


def test_host_pointer_path_matches_device_path(mc):
    net = network_13()
    h = mc.Network(net)
    cells = synthetic_cells(net, 300, seed=15)
    x = np.ascontiguousarray(cells["x"]).copy()
    T = cells["T"].copy()
    nd = cells["ndens"].copy()
    st = np.zeros(300, dtype=np.int32)
    stats = np.zeros((8, 300), dtype=np.int32)
    mc.mc_burn_batch(h, None, 300, 1e10, x, 300, T, nd, None, st, stats)
    gx, gT, gs, gst = mc.burn(h, cells, 1e10)
    np.testing.assert_array_equal(x, gx)
    np.testing.assert_array_equal(T, gT)
    np.testing.assert_array_equal(st, gs)
    np.testing.assert_array_equal(stats, gst)


def test_isothermal_rate_scale_matches_oracle(mc):
    """Robertson with per-cell rate factors and an explicit temperature array
    (ignored by its T-independent rates)."""
    net = robertson_network()
    cells = robertson_cells(257, seed=5)
    cells["T"] = np.full(257, 300.0)
    gx, gT, gs, gst = _run(mc, net, cells, 40.0)
    ox, oT, os_, ost = _oracle(net, cells, 40.0)
    rep = compare(gx, None, gs, ox, None, os_, ost)
    assert rep["pass"], rep
