"""The burn with constant source terms (mc_burn_batch_sdc) against the CPU
oracle: dy/dt = f(y) + s with s fixed per cell and component over the burn,
the burn inside a step coupled by spectral deferred corrections (Software
design section, paragraph 4)."""
import numpy as np
import pytest

import oracle
from mc_inputs import network_13, synthetic_cells, synthetic_sources
from mc_inputs.networks import Network
from parity import classify, compare

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mc():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2608_06466_b300 as mc
    return mc


def _burn_sdc(mc, net, cells, src, dt, **opt):
    import torch
    from paper_2608_06466_b300.api import to_device
    h = mc.Network(net)
    d = to_device(cells)
    s = torch.as_tensor(np.ascontiguousarray(src), device="cuda")
    n = cells["x"].shape[1]
    mc.mc_burn_batch_sdc(h, mc.mc_burn_opts_default(**opt), n, dt, d["x"], n, d["T"], d["ndens"], d["rate_scale"],
                         s, d["status"], d["stats"])
    torch.cuda.synchronize()
    T = None if d["T"] is None else d["T"].cpu().numpy()
    return d["x"].cpu().numpy(), T, d["status"].cpu().numpy(), d["stats"].cpu().numpy()


@pytest.mark.parametrize("lu,variant", [(64, 2), (32, 2), (64, 1)])
def test_sources_match_the_oracle(mc, lu, variant):
    net = network_13()
    cells = synthetic_cells(net, 2048, seed=21)
    src = synthetic_sources(net, cells, 1e10, seed=22, scale=0.05)
    gx, gT, gs, gst = _burn_sdc(mc, net, cells, src, 1e10, lu_precision=lu, variant=variant)
    on = oracle.OracleNetwork(net)
    (ox, oT, os_, ost), stable, rp = classify(on, cells, 1e10, oracle.burn, with_reprobe=True, source=src)
    tx, tT, _, _ = oracle.burn(on, cells, 1e10, rtol=1e-10, atol=1e-16, source=src)
    rep = compare(gx, gT, gs, ox, oT, os_, ost, stable=stable, tight=(tx, tT), reprobe=rp)
    print(lu, variant, rep)
    assert rep["pass"], rep
    assert rep["stable"] >= 0.75 * 2048


def test_source_alone_gives_the_straight_line(mc):
    """All rates zero: y(t) = y0 + s t, integrated exactly by the BDF method."""
    z = np.zeros(2)
    quiet = Network(name="quiet", n_species=3, n_elements=1, energy_eq=False,
                    react=np.array([[0, -1], [1, -1]], dtype=np.int32),
                    prod=np.array([[1, -1], [2, -1]], dtype=np.int32),
                    composition=np.ones((3, 1), dtype=np.int32),
                    A_f=z.copy(), b_f=z.copy(), C_f=z.copy(), A_r=z.copy(), b_r=z.copy(), C_r=z.copy(),
                    dE_eV=z.copy())
    x0 = np.array([[0.5, 0.2], [0.3, 0.1], [0.2, 0.7]])
    s = np.array([[1e-3, -2e-3], [-4e-4, 1e-3], [2e-4, 5e-4]])
    cells = {"x": x0, "T": None, "ndens": None, "rate_scale": None}
    gx, _, gs, _ = _burn_sdc(mc, quiet, cells, s, 50.0, rtol=1e-8, atol=1e-14)
    assert (gs == 0).all()
    np.testing.assert_allclose(gx, x0 + 50.0 * s, rtol=1e-13, atol=1e-15)


def test_zero_source_is_the_plain_burn(mc):
    net = network_13()
    cells = synthetic_cells(net, 512, seed=23)
    a = _burn_sdc(mc, net, cells, np.zeros((net.n_ode, 512)), 1e10, variant=2)
    h = mc.Network(net)
    b = mc.burn(h, cells, 1e10, mc.mc_burn_opts_default(variant=2))
    for u, v in zip(a, b):
        np.testing.assert_array_equal(u, v)
