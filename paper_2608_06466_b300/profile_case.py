"""Single cases for profiling the library with ncu (one GPU, small enough
that a capture ends by itself).

    python -m paper_2608_06466_b300.profile_case eval
        mc_network_rates on net13 and net33 and mc_network_rhs (with the
        Jacobian) on net13, 2^18 states each: the evaluation kernels k_rates,
        k_rhs and k_jac, whose FP64 instruction counters give the per-unit
        flops of the roofline model.

    python -m paper_2608_06466_b300.profile_case burn --cells 1048576 --lu 32 \\
        --variant 2 --max-steps 3000 --straggler -1 [--staging 1|2] [--bps K]
        One burn of net13 cells (seed 3) with those options; prints the time
        and the summed per-cell counters.
"""
from __future__ import annotations

import argparse
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def run_eval(n: int = 1 << 18) -> None:
    import torch

    import paper_2608_06466_b300 as mc
    from mc_inputs import network_13, network_33, synthetic_cells
    from mc_inputs.networks import K_B_EV
    rng = np.random.default_rng(1)
    for make in (network_13, network_33):
        net = make()
        h = mc.Network(net)
        T = torch.as_tensor(np.exp(rng.uniform(np.log(10.0), np.log(1e4), n)), device="cuda")
        kf = torch.empty((net.n_reactions, n), dtype=torch.float64, device="cuda")
        kr = torch.empty_like(kf)
        mc.mc_network_rates(h, n, T, kf, kr, n)
        torch.cuda.synchronize()
    net = network_13()
    h = mc.Network(net)
    c = synthetic_cells(net, n, seed=3)
    y = np.concatenate([c["x"], (c["x"].sum(0) * K_B_EV * c["T"] / (net.gamma - 1))[None, :]])
    yt = torch.as_tensor(np.ascontiguousarray(y), device="cuda")
    nd = torch.as_tensor(c["ndens"], device="cuda")
    f = torch.empty((net.n_ode, n), dtype=torch.float64, device="cuda")
    J = torch.empty((net.n_ode ** 2, n), dtype=torch.float64, device="cuda")
    ok = torch.empty(n, dtype=torch.int32, device="cuda")
    mc.mc_network_rhs(h, n, yt, n, None, nd, None, f, J, ok)
    torch.cuda.synchronize()
    print("evaluated", n, "states; finite:", int(ok.sum()))


def run_burn(n: int, lu: int, variant: int, max_steps: int, straggler: int, staging: int = 0, bps: int = 0) -> None:
    import torch

    import paper_2608_06466_b300 as mc
    from paper_2608_06466_b300.api import to_device
    from mc_inputs import network_13, synthetic_cells
    net = network_13()
    h = mc.Network(net)
    d = to_device(synthetic_cells(net, n, seed=3))
    o = mc.mc_burn_opts_default(lu_precision=lu, variant=variant, max_steps=max_steps, straggler_steps=straggler,
                                staging=staging, blocks_per_sm=bps)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    mc.mc_burn_batch(h, o, n, 1e10, d["x"], n, d["T"], d["ndens"], None, d["status"], d["stats"])
    e1.record()
    torch.cuda.synchronize()
    st = d["stats"].cpu().numpy().astype(np.int64)
    print("ms", e0.elapsed_time(e1), "attempts", int((st[0] + st[1] + st[2]).sum()), "rhs", int(st[3].sum()),
          "jac", int(st[4].sum()), "lu", int(st[5].sum()), "newton", int(st[6].sum()))


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("case", choices=["eval", "burn"])
    ap.add_argument("--cells", type=int, default=1 << 20)
    ap.add_argument("--lu", type=int, default=32)
    ap.add_argument("--variant", type=int, default=2)
    ap.add_argument("--max-steps", type=int, default=100000)
    ap.add_argument("--straggler", type=int, default=0)
    ap.add_argument("--staging", type=int, default=0, help="0 auto, 1 shared, 2 lane")
    ap.add_argument("--bps", type=int, default=0, help="persistent blocks per SM (0 = autotuned)")
    a = ap.parse_args()
    if a.case == "eval":
        run_eval()
    else:
        run_burn(a.cells, a.lu, a.variant, a.max_steps, a.straggler, a.staging, a.bps)


if __name__ == "__main__":
    main()
