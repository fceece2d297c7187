"""Serving loop (continuous batching) through the C ABI: results equal lone
burns bit for bit and the oracle on sampled cells, per-request options, work
of several requests overlapping on the device, and FIFO admission under the
HBM budget (state plus the stream scratch each burn needs)."""
import numpy as np
import pytest

import oracle
from mc_inputs import network_13, network_33, synthetic_cells
from parity import classify, compare

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mc():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2608_06466_b300 as mc
    return mc


def _requests(rng, nets, k):
    out = []
    for i in range(k):
        which = int(rng.integers(0, len(nets)))
        edge = int(rng.integers(5, 13))
        cells = synthetic_cells(nets[which], edge ** 3, seed=1000 + i)
        out.append((which, cells))
    return out


def test_results_same_alone_and_in_the_mix(mc):
    """Ten requests of both networks, alternating FP32 and FP64 matrices and
    host and device buffers, submitted at once: each result equals the same
    request burned alone with the same options, bit for bit."""
    import torch
    nets = [network_13(), network_33()]
    handles = [mc.Network(n) for n in nets]
    reqs = _requests(np.random.default_rng(0), nets, 10)
    opts = [mc.mc_burn_opts_default(lu_precision=32), mc.mc_burn_opts_default(lu_precision=64)]
    alone = [mc.burn(handles[w], cells, 1e10, opts[i % 2]) for i, (w, cells) in enumerate(reqs)]
    srv = mc.Server(0, 8 << 30, opts[0])
    bufs, ids = [], []
    for i, (which, cells) in enumerate(reqs):
        n = cells["x"].shape[1]
        if i % 3 == 0:
            b = {"x": cells["x"].copy(), "T": cells["T"].copy(), "nd": cells["ndens"].copy(),
                 "st": np.full(n, -1, dtype=np.int32)}
        else:
            b = {"x": torch.as_tensor(cells["x"], device="cuda").clone(),
                 "T": torch.as_tensor(cells["T"], device="cuda").clone(),
                 "nd": torch.as_tensor(cells["ndens"], device="cuda"),
                 "st": torch.full((n,), -1, dtype=torch.int32, device="cuda")}
        bufs.append(b)
        ids.append(srv.submit(handles[which], n, 1e10, b["x"], n, b["T"], b["nd"], b["st"], opts=opts[i % 2]))
    srv.drain(600)
    torch.cuda.synchronize()
    for i, rid in enumerate(ids):
        rc, info = srv.poll(rid)
        assert rc == 0 and info.state == 0
        assert info.t_submit <= info.t_admit <= info.t_done
        assert 0.0 <= info.gpu_start <= info.gpu_end
        b = bufs[i]
        get = (lambda v: v.cpu().numpy()) if hasattr(b["x"], "cpu") else (lambda v: v)
        ax, aT, as_, _ = alone[i]
        np.testing.assert_array_equal(get(b["x"]), ax)
        np.testing.assert_array_equal(get(b["T"]), aT)
        np.testing.assert_array_equal(get(b["st"]), as_)
        assert info.n_failed == int((as_ != 0).sum())
    srv.close()
    # the served results against the oracle on sampled cells of each network
    for which in (0, 1):
        k = [i for i, (w, _) in enumerate(reqs) if w == which][0]
        cells = reqs[k][1]
        n = cells["x"].shape[1]
        idx = np.sort(np.random.default_rng(k).choice(n, min(n, 128), replace=False))
        on = oracle.OracleNetwork(nets[which])
        o, stable, rp = classify(on, cells, 1e10, oracle.burn, index=idx, with_reprobe=True)
        t = oracle.burn(on, cells, 1e10, rtol=1e-10, atol=1e-16, index=idx)
        get = (lambda v: v.cpu().numpy()) if hasattr(bufs[k]["x"], "cpu") else (lambda v: v)
        rep = compare(get(bufs[k]["x"])[:, idx], get(bufs[k]["T"])[idx], get(bufs[k]["st"])[idx], *o,
                      stable=stable, tight=(t[0], t[1]), reprobe=rp)
        assert rep["pass"], (nets[which].name, rep)


def test_requests_overlap_on_the_device(mc):
    """Requests submitted together run on different streams at the same time:
    some pair's [gpu_start, gpu_end] intervals overlap."""
    net = network_13()
    h = mc.Network(net)
    srv = mc.Server(0, 8 << 30, mc.mc_burn_opts_default(lu_precision=32))
    keep, ids = [], []
    for i in range(8):
        c = synthetic_cells(net, 4096, seed=70 + i)
        b = (c["x"].copy(), c["T"].copy(), c["ndens"].copy(), np.zeros(4096, dtype=np.int32))
        keep.append(b)
        ids.append(srv.submit(h, 4096, 1e10, b[0], 4096, b[1], b[2], b[3]))
    srv.drain(600)
    infos = [srv.poll(r)[1] for r in ids]
    srv.close()
    spans = [(i.gpu_start, i.gpu_end) for i in infos]
    assert all(0.0 <= a <= b for a, b in spans)
    overlap = max(min(b1, b2) - max(a1, a2) for k, (a1, b1) in enumerate(spans) for (a2, b2) in spans[k + 1:])
    assert overlap > 0.0, spans


def test_budget_admission_is_fifo_and_bounded(mc):
    net = network_13()
    h = mc.Network(net)
    opts = mc.mc_burn_opts_default(lu_precision=32)
    state, scratch = mc.Server.request_bytes(net_h := h, 512, opts)
    assert state >= (12 + 2) * 8 * 512 and scratch > 4 * 512
    # room for two requests' state and one stream's scratch
    srv = mc.Server(0, 2 * state + scratch + 100, opts)
    ids, keep = [], []
    for i in range(6):
        c = synthetic_cells(net, 512, seed=50 + i)
        b = (c["x"].copy(), c["T"].copy(), c["ndens"].copy(), np.zeros(512, dtype=np.int32))
        keep.append(b)
        ids.append(srv.submit(net_h, 512, 1e10, b[0], 512, b[1], b[2], b[3]))
    with pytest.raises(mc.MCError, match="MC_E_BUDGET"):
        big = synthetic_cells(net, 4096, seed=99)
        srv.submit(net_h, 4096, 1e10, big["x"].copy(), 4096, big["T"].copy(), big["ndens"].copy(),
                   np.zeros(4096, dtype=np.int32))
    srv.drain(600)
    infos = [srv.poll(r)[1] for r in ids]
    admits = [i.t_admit for i in infos]
    assert admits == sorted(admits)
    # at most two requests were ever admitted and unfinished at the same time
    for i in infos:
        live = sum(1 for j in infos if j.t_admit <= i.t_admit < j.t_done)
        assert live <= 2
    with pytest.raises(mc.MCError, match="MC_E_NOTFOUND"):
        srv.poll(123456789)
    srv.close()
