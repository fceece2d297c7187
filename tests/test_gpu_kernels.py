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
    """With b = C = 0 a rate coefficient is exactly exp(ln A) of the stored
    ln A, so the table-driven exponential can be compared with CUDA's exp on
    bit-identical arguments, over the whole double range (normal and
    subnormal results)."""
    import torch
    from mc_inputs.networks import Network
    R = 512
    rng = np.random.default_rng(1)
    v = np.concatenate([rng.uniform(-744.0, 709.0, R - 64), rng.uniform(-745.0, -700.0, 32),
                        rng.uniform(-1.0, 1.0, 32)])
    A = np.exp(v)
    A[A == 0] = 5e-324
    z = np.zeros(R)
    net = Network(name="exptest", n_species=2, n_elements=1, energy_eq=False,
                  react=np.tile(np.array([[0, -1]], dtype=np.int32), (R, 1)),
                  prod=np.tile(np.array([[1, -1]], dtype=np.int32), (R, 1)),
                  composition=np.ones((2, 1), dtype=np.int32), A_f=A, b_f=z.copy(), C_f=z.copy(),
                  A_r=z.copy(), b_r=z.copy(), C_r=z.copy(), dE_eV=z.copy())
    h = mc.Network(net)
    n = 64
    T = torch.full((n,), 300.0, dtype=torch.float64, device="cuda")
    kf = torch.empty((R, n), dtype=torch.float64, device="cuda")
    kr = torch.empty_like(kf)
    mc.mc_network_rates(h, n, T, kf, kr, n)
    ref = torch.exp(torch.log(torch.as_tensor(A, device="cuda")))[:, None].expand(R, n)
    torch.cuda.synchronize()
    a, b = kf.cpu().numpy(), ref.cpu().numpy()
    normal = b > 2.2250738585072014e-308
    assert _ulp_diff(a[normal], b[normal]).max() <= 2
    # subnormal results: within one unit of the smallest subnormal spacing
    assert np.abs(a[~normal] - b[~normal]).max() <= 1e-323
    assert (kr.cpu().numpy() == 0).all()


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
