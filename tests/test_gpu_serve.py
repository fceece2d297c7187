"""Serving loop (continuous batching) through the C ABI."""
import numpy as np
import pytest

from mc_inputs import network_13, network_33, synthetic_cells

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
        cells = synthetic_cells(nets[which][0], edge ** 3, seed=1000 + i)
        out.append((which, cells))
    return out


def test_results_same_alone_and_in_the_mix(mc):
    import torch
    nets = [(network_13(), None), (network_33(), None)]
    handles = [mc.Network(n) for n, _ in nets]
    reqs = _requests(np.random.default_rng(0), nets, 10)
    opts = mc.mc_burn_opts_default(lu_precision=32)
    # alone: each request burned by itself
    alone = []
    for which, cells in reqs:
        alone.append(mc.burn(handles[which], cells, 1e10, opts))
    # in the mix: all submitted at once, half from host arrays and half from device tensors
    srv = mc.Server(0, 8 << 30, opts)
    bufs, ids = [], []
    for i, (which, cells) in enumerate(reqs):
        n = cells["x"].shape[1]
        if i % 2 == 0:
            b = {"x": cells["x"].copy(), "T": cells["T"].copy(), "nd": cells["ndens"].copy(),
                 "st": np.full(n, -1, dtype=np.int32)}
        else:
            b = {"x": torch.as_tensor(cells["x"], device="cuda").clone(), "T": torch.as_tensor(cells["T"], device="cuda").clone(),
                 "nd": torch.as_tensor(cells["ndens"], device="cuda"), "st": torch.full((n,), -1, dtype=torch.int32, device="cuda")}
        bufs.append(b)
        ids.append(srv.submit(handles[which], n, 1e10, b["x"], n, b["T"], b["nd"], b["st"]))
    srv.drain(600)
    torch.cuda.synchronize()
    for i, rid in enumerate(ids):
        rc, info = srv.poll(rid)
        assert rc == 0 and info.state == 0
        assert info.t_submit <= info.t_admit <= info.t_done
        b = bufs[i]
        get = (lambda v: v.cpu().numpy()) if hasattr(b["x"], "cpu") else (lambda v: v)
        ax, aT, as_, _ = alone[i]
        np.testing.assert_array_equal(get(b["x"]), ax)
        np.testing.assert_array_equal(get(b["T"]), aT)
        np.testing.assert_array_equal(get(b["st"]), as_)
        assert info.n_failed == int((as_ != 0).sum())
    srv.close()


def test_budget_admission_is_fifo_and_bounded(mc):
    net = network_13()
    h = mc.Network(net)
    one = (12 + 2) * 8 * 512 + 4 * 512 + 1024
    srv = mc.Server(0, 2 * one + 100, mc.mc_burn_opts_default(lu_precision=32))
    ids, keep = [], []
    for i in range(6):
        c = synthetic_cells(net, 512, seed=50 + i)
        b = (c["x"].copy(), c["T"].copy(), c["ndens"].copy(), np.zeros(512, dtype=np.int32))
        keep.append(b)
        ids.append(srv.submit(h, 512, 1e10, b[0], 512, b[1], b[2], b[3]))
    with pytest.raises(mc.MCError, match="MC_E_BUDGET"):
        big = synthetic_cells(net, 4096, seed=99)
        srv.submit(h, 4096, 1e10, big["x"].copy(), 4096, big["T"].copy(), big["ndens"].copy(),
                   np.zeros(4096, dtype=np.int32))
    srv.drain(600)
    infos = [srv.poll(r)[1] for r in ids]
    admits = [i.t_admit for i in infos]
    assert admits == sorted(admits)
    # at most two requests were ever admitted and unfinished at the same time
    for k, i in enumerate(infos):
        live = sum(1 for j in infos if j.t_admit <= i.t_admit < j.t_done)
        assert live <= 2
    with pytest.raises(mc.MCError, match="MC_E_NOTFOUND"):
        srv.poll(123456789)
    srv.close()
