"""The retry ladder (mc_burn_ladder) and the RKC integrator on the GPU against
the CPU oracle (Software design section: paragraph 3, a zone that fails is
integrated again under other tolerances or with an approximate Jacobian; paragraphs 2
and 4, RKC beside VODE on the same network interface)."""
import numpy as np
import pytest

import oracle
from mc_inputs import network_13, synthetic_cells
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


def _ladder_gpu(mc, net, cells, dt, rungs):
    import torch
    from paper_2608_06466_b300.api import to_device
    h = mc.Network(net)
    d = to_device(cells)
    n = cells["x"].shape[1]
    rung = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    mc.mc_burn_ladder(h, rungs, n, dt, d["x"], n, d["T"], d["ndens"], d["rate_scale"], d["status"], d["stats"], rung)
    torch.cuda.synchronize()
    T = None if d["T"] is None else d["T"].cpu().numpy()
    return d["x"].cpu().numpy(), T, d["status"].cpu().numpy(), d["stats"].cpu().numpy(), rung.cpu().numpy()


def _ladder_oracle(rungs):
    def burn(onet, cells, dt, index=None, **kw):
        return oracle.burn_ladder(onet, cells, dt, rungs, index=index)[:4]
    return burn


@pytest.mark.parametrize("lu", [32, 64])
def test_ladder_matches_the_oracle_ladder(mc, lu):
    """Rung 0 caps the steps at 60, so most cells fail and are retried by rung
    1 with the forward-difference Jacobian; statuses, the rung that finished
    each cell and the results follow the oracle's ladder."""
    net = network_13()
    cells = synthetic_cells(net, 1024, seed=31)
    gx, gT, gs, gst, grung = _ladder_gpu(mc, net, cells, 1e10, [
        mc.rung(max_steps=60, lu_precision=lu),
        mc.rung(jacobian=mc.MC_JAC_FD, lu_precision=lu)])
    o_rungs = [{"max_steps": 60}, {"jac": "fd"}]
    on = oracle.OracleNetwork(net)
    ox, oT, os_, ost, orung = oracle.burn_ladder(on, cells, 1e10, o_rungs)
    assert (orung == 1).mean() > 0.3 and (grung == 1).mean() > 0.3
    # the rung that finished a cell follows from rung 0's deterministic cap
    near = np.abs(ost[0] + ost[1] + ost[2] - 60) <= 1
    assert np.mean(grung[~near] == orung[~near]) > 0.99
    (o, stable, rp) = classify(on, cells, 1e10, _ladder_oracle(o_rungs), twin=False, with_reprobe=True)
    t = oracle.burn(on, cells, 1e10, rtol=1e-10, atol=1e-16)
    rep = compare(gx, gT, gs, o[0], o[1], o[2], o[3], stable=stable & (grung == orung), tight=(t[0], t[1]),
                  reprobe=rp)
    print(lu, rep)
    assert rep["pass"], rep


def test_rkc_rung_matches_the_oracle_rkc(mc):
    """A ladder of one RKC rung is a plain RKC burn: cells that finish within
    the step cap match the oracle's RKC, the stiff ones stop at the cap in
    both."""
    net = network_13()
    cells = synthetic_cells(net, 256, seed=32)
    gx, gT, gs, gst, grung = _ladder_gpu(mc, net, cells, 1e10, [mc.rung(method=mc.MC_METHOD_RKC, max_steps=200)])
    o_rungs = [{"method": "rkc", "max_steps": 200}]
    on = oracle.OracleNetwork(net)
    (o, stable, rp) = classify(on, cells, 1e10, _ladder_oracle(o_rungs), twin=False, with_reprobe=True)
    ox, oT, os_, ost = o
    assert (os_ == 0).mean() > 0.2 and (os_ == 1).any()
    np.testing.assert_array_equal(gst[0][os_ == 0], ost[0][os_ == 0])  # same accepted steps
    rep = compare(gx, gT, gs, ox, oT, os_, ost, stable=stable, tight=None if stable.all() else
                  oracle.burn(on, cells, 1e10, rtol=1e-10, atol=1e-16)[:2], reprobe=rp, max_steps=200)
    print(rep)
    assert rep["pass"], rep


def test_rkc_on_a_linear_chain_against_the_matrix_exponential(mc):
    """A -> B -> C with mild rates: the adaptive RKC result against
    exp(K t) y0 within the tolerance's reach."""
    from scipy.linalg import expm
    z = np.zeros(2)
    chain = Network(name="chain", n_species=3, n_elements=1, energy_eq=False,
                    react=np.array([[0, -1], [1, -1]], dtype=np.int32),
                    prod=np.array([[1, -1], [2, -1]], dtype=np.int32),
                    composition=np.ones((3, 1), dtype=np.int32),
                    A_f=np.array([1.0, 30.0]), b_f=z.copy(), C_f=z.copy(),
                    A_r=z.copy(), b_r=z.copy(), C_r=z.copy(), dE_eV=z.copy())
    y0 = np.array([[1.0, 0.6], [0.0, 0.3], [0.0, 0.1]])
    cells = {"x": y0, "T": None, "ndens": None, "rate_scale": None}
    gx, _, gs, _, _ = _ladder_gpu(mc, chain, cells, 2.0,
                                  [mc.rung(method=mc.MC_METHOD_RKC, rtol=1e-8, atol=1e-12)])
    assert (gs == 0).all()
    K = np.array([[-1.0, 0.0, 0.0], [1.0, -30.0, 0.0], [0.0, 30.0, 0.0]])
    ref = expm(2.0 * K) @ y0
    # the global error of an order-2 method whose local error is held at rtol
    np.testing.assert_allclose(gx, ref, rtol=1e-5, atol=1e-7)
    # and the same integration as the oracle's RKC, step for step
    ox, _, os_, _, _ = oracle.burn_ladder(oracle.OracleNetwork(chain), cells, 2.0,
                                          [{"method": "rkc", "rtol": 1e-8, "atol": 1e-12}])
    assert (os_ == 0).all()
    np.testing.assert_allclose(gx, ox, rtol=1e-11, atol=1e-16)
