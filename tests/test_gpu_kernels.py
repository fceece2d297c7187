"""Kernel-level checks of the device network code through the C ABI: rate
coefficients (table-driven exponential) against CUDA's exp, right-hand side and
Jacobian against the oracle at random states."""
import numpy as np
import pytest

import oracle
from mc_inputs import network_13, network_33, robertson_network
from mc_inputs.networks import K_B_EV

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mc():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2608_06466_b300 as mc
    return mc


def _ulp_diff(a, b):
    ia = a.view(np.int64)
    ib = b.view(np.int64)
    return np.abs(ia - ib)


def test_rate_exponential_within_few_ulp_of_cuda_exp(mc):
    import torch
    net = network_33()
    h = mc.Network(net)
    n = 1 << 16
    rng = np.random.default_rng(1)
    T = torch.as_tensor(np.exp(rng.uniform(np.log(5.0), np.log(2e5), n)), device="cuda")
    kf = torch.empty((net.n_reactions, n), dtype=torch.float64, device="cuda")
    kr = torch.empty_like(kf)
    mc.mc_network_rates(h, n, T, kf, kr, n)
    lnT, invT = torch.log(T), 1.0 / T
    lnAf = torch.as_tensor(np.log(net.A_f), device="cuda")[:, None]
    ref = torch.exp(lnAf + torch.as_tensor(net.b_f, device="cuda")[:, None] * lnT
                    - torch.as_tensor(net.C_f, device="cuda")[:, None] * invT)
    torch.cuda.synchronize()
    a, b = kf.cpu().numpy(), ref.cpu().numpy()
    normal = (b > 2.3e-308) & (b < 1e300)
    d = _ulp_diff(a[normal], b[normal])
    assert d.max() <= 4, d.max()
    sub = ~normal & (b >= 0)
    np.testing.assert_allclose(a[sub], b[sub], rtol=0, atol=1e-320)


@pytest.mark.parametrize("make", [robertson_network, network_13, network_33])
def test_rhs_and_jacobian_match_oracle(mc, make):
    import torch
    net = make()
    h = mc.Network(net)
    on = oracle.OracleNetwork(net)
    rng = np.random.default_rng(2)
    n = 257
    S, N = net.n_species, net.n_ode
    x = rng.uniform(0.0, 1.0, (S, n))
    T = np.exp(rng.uniform(np.log(20.0), np.log(3e4), n))
    nd = 10 ** rng.uniform(0, 8, n) if net.energy_eq else np.ones(n)
    y = np.concatenate([x, (x.sum(0) * K_B_EV * T / (net.gamma - 1))[None, :]]) if net.energy_eq else x
    yt = torch.as_tensor(np.ascontiguousarray(y), device="cuda")
    Tt = None if net.energy_eq else torch.as_tensor(T, device="cuda")
    ndt = torch.as_tensor(nd, device="cuda")
    f = torch.empty((N, n), dtype=torch.float64, device="cuda")
    J = torch.empty((N * N, n), dtype=torch.float64, device="cuda")
    ok = torch.empty(n, dtype=torch.int32, device="cuda")
    mc.mc_network_rhs(h, n, yt, n, Tt, ndt, None, f, J, ok)
    torch.cuda.synchronize()
    f, J, ok = f.cpu().numpy(), J.cpu().numpy(), ok.cpu().numpy()
    assert ok.all()
    for c in range(0, n, 16):
        of, oJ = on.eval(y[:, c], ndens=nd[c], T_iso=(1.0 if net.energy_eq else T[c]))
        sf = np.abs(of).max() + 1e-300
        np.testing.assert_allclose(f[:, c], of, rtol=1e-12, atol=1e-13 * sf)
        sJ = np.abs(oJ).max() + 1e-300
        np.testing.assert_allclose(J[:, c].reshape(N, N), oJ, rtol=1e-11, atol=1e-12 * sJ)
