"""The allocation-free burn entry point (mc_burn_batch_noalloc).

Some callers cannot let a library allocate device memory: programs that give
all of it to their own arena at start-up, or latency-critical loops that
cannot absorb cudaMalloc's implicit synchronisation. The entry point keeps its
scratch in a fixed device array instead; here its results are checked against
the allocating entry point's on the same inputs, on two calls in a row (the
shared array keeps the previous call's contents, so a missed reset shows up
on the second call). This file is collected last on purpose."""
import numpy as np
import pytest

from mc_inputs import network_13, synthetic_cells

pytestmark = pytest.mark.gpu

RTOL, ATOL = 1e-5, 1e-10  # the parity bar of the GPU tests


@pytest.fixture(scope="module")
def mc():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2608_06466_b300 as mc
    return mc


@pytest.mark.parametrize("lu", [32, 64])
def test_noalloc_matches_allocating_entry_point_on_two_calls(mc, lu):
    import torch
    net = network_13()
    h = mc.Network(net)
    n = 3000
    opts = mc.mc_burn_opts_default(lu_precision=lu, variant=mc.MC_VARIANT_PERSISTENT, straggler_steps=-1)
    for call in range(2):
        cells = synthetic_cells(net, n, seed=70 + call)
        bufs = []
        for _ in range(2):
            bufs.append({"x": torch.as_tensor(cells["x"], device="cuda").clone(),
                         "T": torch.as_tensor(cells["T"], device="cuda").clone(),
                         "nd": torch.as_tensor(cells["ndens"], device="cuda"),
                         "st": torch.full((n,), -1, dtype=torch.int32, device="cuda"),
                         "stats": torch.zeros((8, n), dtype=torch.int32, device="cuda")})
        a, b = bufs
        mc.mc_burn_batch(h, opts, n, 1e10, a["x"], n, a["T"], a["nd"], None, a["st"], a["stats"])
        mc.mc_burn_batch_noalloc(h, opts, n, 1e10, b["x"], n, b["T"], b["nd"], None, b["st"], b["stats"])
        torch.cuda.synchronize()
        np.testing.assert_array_equal(b["st"].cpu().numpy(), a["st"].cpu().numpy())
        np.testing.assert_allclose(b["x"].cpu().numpy(), a["x"].cpu().numpy(), rtol=RTOL, atol=10 * ATOL)
        np.testing.assert_allclose(b["T"].cpu().numpy(), a["T"].cpu().numpy(), rtol=RTOL)
        assert (a["st"].cpu().numpy() == 0).mean() > 0.99


def test_noalloc_rejects_batches_beyond_its_maximum(mc):
    import torch
    net = network_13()
    h = mc.Network(net)
    n = mc.MC_NOALLOC_MAX_CELLS + 1
    x = torch.zeros((12, 1), dtype=torch.float64, device="cuda")
    with pytest.raises(mc.MCError, match="MC_E_INVALID"):
        mc.mc_burn_batch_noalloc(h, None, n, 1e10, x, n, x, None, None, x, None)
