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
    """Oracle result, stability mask, tight-tolerance oracle result and the
    classification's re-probe (tests/parity.py)."""
    on = oracle.OracleNetwork(net)
    (ox, oT, os_, ost), stable, reprobe = classify(on, cells, dt, oracle.burn, index=index, with_reprobe=True)
    tx, tT, _, _ = oracle.burn(on, cells, dt, rtol=1e-10, atol=1e-16, index=index)
    return ox, oT, os_, ost, stable, (tx, tT), reprobe


@pytest.mark.parametrize("variant", [1, 2, 3])
@pytest.mark.parametrize("lu", [64, 32])
def test_robertson_4096(mc, variant, lu):
    net, cells = robertson_network(), robertson_cells(4096, 1)
    gx, gT, gs, gst = _run(mc, net, cells, 40.0, variant=variant, lu_precision=lu)
    ox, oT, os_, ost = _oracle(net, cells, 40.0)
    tx, _, _, _ = _oracle(net, cells, 40.0, rtol=1e-11, atol=1e-17)
    rep = compare(gx, gT, gs, ox, oT, os_, ost, tight=(tx, None))
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
    ox, oT, os_, ost, stable, tight, rp = _reference(net, cells, 1e10)
    rep = compare(gx, gT, gs, ox, oT, os_, ost, stable=stable, tight=tight, reprobe=rp)
    print(net.name, lu, rep, "same step count:", np.mean(gst[0] == ost[0]))
    assert rep["pass"], rep
    assert rep["stable"] >= 0.75 * n


@pytest.mark.parametrize("lu,n_log2,variant", [(32, 22, 2), (64, 20, 1)])
def test_full_size_sampled(mc, lu, n_log2, variant):
    """The 13-ODE network at the workloads' full sizes in the launch
    configurations the benchmark times: the FP32-matrix persistent path on
    2^22 cells (its headline) and the plain FP64 path on 2^20 cells; 4096
    sampled cells recomputed by the oracle."""
    net = network_13()
    n = 1 << n_log2
    cells = synthetic_cells(net, n, seed=3)
    gx, gT, gs, gst = _run(mc, net, cells, 1e10, lu_precision=lu, variant=variant)
    idx = np.sort(np.random.default_rng(0).choice(n, 4096, replace=False))
    ox, oT, os_, ost, stable, tight, rp = _reference(net, cells, 1e10, index=idx)
    rep = compare(gx[:, idx], gT[idx], gs[idx], ox, oT, os_, ost, stable=stable, tight=tight, reprobe=rp)
    print(lu, n, rep)
    assert rep["pass"], rep
    assert np.mean(gs == 0) > 0.99


@pytest.mark.parametrize("variant", [1, 2, 3])
def test_ragged_and_degenerate_sizes(mc, variant):
    net = network_13()
    h = mc.Network(net)
    for n in (1, 37, 129):
        cells = synthetic_cells(net, n, seed=11)
        gx, gT, gs, gst = mc.burn(h, cells, 1e10, mc.mc_burn_opts_default(variant=variant))
        ox, oT, os_, ost, stable, tight, rp = _reference(net, cells, 1e10)
        rep = compare(gx, gT, gs, ox, oT, os_, ost, stable=stable, tight=tight, reprobe=rp)
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
    ox, oT, os_, ost, stable, tight, rp = _reference(net, cells, 1e10)
    rep = compare(x[:, :100].cpu().numpy(), T[:100].cpu().numpy(), st[:100].cpu().numpy(), ox, oT, os_, ost,
                  stable=stable, tight=tight, reprobe=rp)
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
    ox, oT, os_, ost, stable, tight, rp = _reference(net, cells, 1e10)
    assert list(gs[:4]) == [4, 4, 4, 4] and list(os_[:4]) == [4, 4, 4, 4]
    np.testing.assert_array_equal(gT[1], -1.0)  # rejected cells are left untouched
    rep = compare(gx, gT, gs, ox, oT, os_, ost, stable=stable, tight=tight, reprobe=rp)
    assert rep["pass"], rep
    # the step cap: same statuses and attempt counts. The states are compared
    # loosely: after 7 attempts they sit at slightly different times, because
    # the starting step uses the difference quotient |f(y0 + h0 f0) - f0| / h0,
    # whose rounding depends on the last bits of the rate exponential (table
    # form here, libm in the oracle) and moves h by ~0.1 % on some cells.
    gx, gT, gs, gst = _run(mc, net, synthetic_cells(net, 64, seed=14), 1e10, max_steps=7)
    ox, oT, os_, ost = _oracle(net, synthetic_cells(net, 64, seed=14), 1e10, max_steps=7)
    np.testing.assert_array_equal(gs, os_)
    assert (gs == 1).any()
    np.testing.assert_array_equal(gst[0] + gst[1] + gst[2], ost[0] + ost[1] + ost[2])
    same = (gst[:7] == ost[:7]).all(axis=0)
    assert same.mean() >= 0.8
    np.testing.assert_allclose(gx[:, same], ox[:, same], rtol=1e-2, atol=1e-8)


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


@pytest.mark.parametrize("make,n,lu", [(network_13, 2048, 64), (network_13, 2048, 32), (network_33, 512, 32),
                                       (robertson_network, 1024, 64)])
def test_straggler_handoff_parity(mc, make, n, lu):
    """A low hand-off threshold sends most cells through the warp-cooperative
    form part-way; results must still match the oracle."""
    net = make()
    if make is robertson_network:
        cells, dt = robertson_cells(n, 1), 40.0
    else:
        cells, dt = synthetic_cells(net, n, seed=3), 1e10
    gx, gT, gs, gst = _run(mc, net, cells, dt, lu_precision=lu, variant=2, straggler_steps=40)
    ox, oT, os_, ost, stable, tight, rp = _reference(net, cells, dt)
    rep = compare(gx, gT, gs, ox, oT, os_, ost, stable=stable, tight=tight, reprobe=rp)
    print(net.name, lu, rep, "handed off:", np.mean(ost[0] + ost[1] + ost[2] > 40))
    assert rep["pass"], rep


def test_fused_launch_matches_two_launches(mc):
    """Bulk and hand-off in one cooperative launch (128-thread blocks) against
    the bulk launch followed by the straggler launch (64-thread blocks): with
    every qualifying cell fitting the record list, each cell's arithmetic is
    the same, so the results agree bit for bit (no record lost or repeated)."""
    net = network_13()
    cells = synthetic_cells(net, 16384, seed=3)
    a = _run(mc, net, cells, 1e10, lu_precision=32, variant=2, straggler_steps=1024, block_threads=128)
    b = _run(mc, net, cells, 1e10, lu_precision=32, variant=2, straggler_steps=1024, block_threads=64)
    att = a[3][0] + a[3][1] + a[3][2]
    print("handed off:", np.mean(att > 1024))
    assert 0.01 < np.mean(att > 1024) < 0.125
    for u, v in zip(a, b):
        assert np.array_equal(u, v)


def _segments(mc, batch, dts):
    segs, keep = [], []
    for (net, cells, idx), dt in zip(batch["groups"], dts):
        h = mc.Network(net)
        from paper_2608_06466_b300.api import to_device
        d = to_device(cells)
        keep.append((h, d, net, cells))
        n = cells["x"].shape[1]
        segs.append(mc.segment(h, n, n, d["x"], d["T"], d["ndens"], d["rate_scale"], d["status"], d["stats"], dt=dt))
    return segs, keep


def _snapshot(keep):
    return [(d["x"].cpu().numpy().copy(), None if d["T"] is None else d["T"].cpu().numpy().copy(),
             d["status"].cpu().numpy().copy(), d["stats"].cpu().numpy().copy()) for (_, d, _, _) in keep]


def _reset(keep):
    import torch
    for (h, d, net, cells) in keep:
        d["x"].copy_(torch.as_tensor(cells["x"]))
        if d["T"] is not None:
            d["T"].copy_(torch.as_tensor(cells["T"]))


MIXED_DTS = [40.0, 1e10, 1e10]   # Robertson to t = 40, the energy networks over 1e10 s


def test_mixed_batch_and_graph(mc):
    """Robertson (3 ODEs, its own dt), net13 and net33 with 1 % hot cells in ONE
    persistent launch; each segment against the oracle; a CUDA-graph replay of
    the same launch reproduces it bit for bit, twice."""
    import torch
    from mc_inputs import mixed_batch
    batch = mixed_batch(3 * 700, seed=6, hot_fraction=0.01)
    segs, keep = _segments(mc, batch, MIXED_DTS)
    opts = mc.mc_burn_opts_default(lu_precision=32)
    mc.mc_burn_mixed(segs, opts, 1e10)
    torch.cuda.synchronize()
    first = _snapshot(keep)
    for (h, d, net, cells), (gx, gT, gs, gst), dt in zip(keep, first, MIXED_DTS):
        ox, oT, os_, ost, stable, tight, rp = _reference(net, cells, dt)
        rep = compare(gx, gT, gs, ox, oT, os_, ost, stable=stable, tight=tight, reprobe=rp)
        assert rep["pass"], (net.name, rep)
    totals = torch.zeros(8, dtype=torch.int64, device="cuda")
    g = mc.mc_graph_create(segs, opts, 1e10, totals)
    for rep_i in range(2):
        _reset(keep)
        g.launch()
        torch.cuda.synchronize()
        for (h, d, net, cells), (gx, gT, gs, gst) in zip(keep, first):
            np.testing.assert_array_equal(d["x"].cpu().numpy(), gx)
            np.testing.assert_array_equal(d["status"].cpu().numpy(), gs)
        want = sum(d["stats"].cpu().numpy().astype(np.int64).sum(axis=1) for (_, d, _, _) in keep)
        np.testing.assert_array_equal(totals.cpu().numpy(), want)
    g.close()


@pytest.mark.parametrize("lu", [32, 64])
def test_mixed_handoff_parity(mc, lu):
    """A low hand-off threshold sends most thread-per-cell cells of the mixed
    launch through its record lists and the warp-per-cell pass."""
    import torch
    from mc_inputs import mixed_batch
    batch = mixed_batch(3 * 400, seed=8, hot_fraction=0.01)
    segs, keep = _segments(mc, batch, MIXED_DTS)
    mc.mc_burn_mixed(segs, mc.mc_burn_opts_default(lu_precision=lu, straggler_steps=40), 1e10)
    torch.cuda.synchronize()
    for (h, d, net, cells), (gx, gT, gs, gst), dt in zip(keep, _snapshot(keep), MIXED_DTS):
        ox, oT, os_, ost, stable, tight, rp = _reference(net, cells, dt)
        rep = compare(gx, gT, gs, ox, oT, os_, ost, stable=stable, tight=tight, reprobe=rp)
        print(net.name, lu, rep)
        assert rep["pass"], (net.name, rep)


def test_results_do_not_depend_on_the_mix(mc):
    """Each cell's result is the same burned alone, in a larger batch and in
    another variant of the persistent launch (bitwise)."""
    import torch
    net = network_13()
    h = mc.Network(net)
    cells = synthetic_cells(net, 3000, seed=31)
    alone = {k: (v[:, :100] if (v is not None and v.ndim == 2) else (None if v is None else v[:100]))
             for k, v in cells.items() if k != "hot"}
    ax, aT, as_, _ = mc.burn(h, alone, 1e10, mc.mc_burn_opts_default(lu_precision=32))
    bx, bT, bs, _ = mc.burn(h, cells, 1e10, mc.mc_burn_opts_default(lu_precision=32, blocks_per_sm=1))
    np.testing.assert_array_equal(ax, bx[:, :100])
    np.testing.assert_array_equal(aT, bT[:100])
    np.testing.assert_array_equal(as_, bs[:100])


def test_autotune_returns_a_measured_shape(mc):
    import torch
    from paper_2608_06466_b300.api import to_device
    net = network_13()
    h = mc.Network(net)
    d = to_device(synthetic_cells(net, 2048, seed=41))
    x0 = d["x"].clone()
    best = mc.mc_autotune(h, mc.mc_burn_opts_default(lu_precision=32), 2048, 1e10, d["x"], 2048, d["T"], d["ndens"])
    torch.cuda.synchronize()
    assert best.variant in (1, 2, 3) and best.block_threads in (64, 128, 256)
    assert best.staging in (mc.MC_STAGING_SHARED, mc.MC_STAGING_LANE)
    assert best.straggler_steps in (2048, 8192, 32768, -1)
    assert torch.equal(d["x"], x0)  # the sample is not modified


@pytest.mark.parametrize("lu", [64, 32])
def test_lane_staging_parity(mc, lu):
    """The persistent worker with each lane doing its own matrix work (the
    autotuner's other staging) against the oracle."""
    net = network_13()
    cells = synthetic_cells(net, 2048, seed=5)
    gx, gT, gs, gst = _run(mc, net, cells, 1e10, lu_precision=lu, variant=mc.MC_VARIANT_PERSISTENT,
                           staging=mc.MC_STAGING_LANE)
    ox, oT, os_, ost, stable, tight, rp = _reference(net, cells, 1e10)
    rep = compare(gx, gT, gs, ox, oT, os_, ost, stable=stable, tight=tight, reprobe=rp)
    print(lu, rep)
    assert rep["pass"], rep
