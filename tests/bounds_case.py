"""Small burns over every launch form of the library, for the bounds-check
build: run in a child process with MC_LIBRARY naming libmc_check.so
(`python tests/bounds_case.py out.npz`), and in the test's own process with
the normal library, so that the two builds' results can be compared and the
check build's record read.

Forms: the cost-ordered persistent launch with a low hand-off threshold (many
straggler records) and the FP64 retry pass, the plain and warp-per-cell
variants, the 33-ODE network, Robertson with per-cell rate factors, host
buffers with ld > n, constant sources, a three-rung retry ladder with a
forward-difference and an RKC rung, and a mixed launch over three networks.
"""
from __future__ import annotations

import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
for p in (ROOT, os.path.join(ROOT, "tests")):
    if p not in sys.path:
        sys.path.insert(0, p)

HANDOFF = 1024       # hand-off threshold of the "fused" case
HANDOFF_CAP = 512    # its record list: max(256, cells / 8)

# (name, cells) of the calls whose stores the check build verifies
VERIFIED = [("fused", 4096), ("plain", 2048), ("warp", 512), ("net33", 512), ("robertson", 4096),
            ("host", 1000), ("sdc", 1024), ("ladder", 1024)]


def _dev(cells, ld, torch):
    """Device copies with leading dimension ld (columns past n hold NaN)."""
    n = cells["x"].shape[1]
    S = cells["x"].shape[0]
    x = torch.full((S, ld), float("nan"), dtype=torch.float64, device="cuda")
    x[:, :n] = torch.as_tensor(cells["x"], device="cuda")
    T = nd = None
    if cells.get("T") is not None:
        T = torch.full((ld,), float("nan"), dtype=torch.float64, device="cuda")
        T[:n] = torch.as_tensor(cells["T"], device="cuda")
        nd = torch.ones(ld, dtype=torch.float64, device="cuda")
        nd[:n] = torch.as_tensor(cells["ndens"], device="cuda")
    ks = None
    if cells.get("rate_scale") is not None:
        R = cells["rate_scale"].shape[0]
        ks = torch.ones((R, ld), dtype=torch.float64, device="cuda")
        ks[:, :n] = torch.as_tensor(cells["rate_scale"], device="cuda")
    st = torch.full((ld,), -7, dtype=torch.int32, device="cuda")
    sx = torch.zeros((8, ld), dtype=torch.int32, device="cuda")
    return {"x": x, "T": T, "nd": nd, "ks": ks, "st": st, "sx": sx}


def _out(d):
    return {k: d[k].cpu().numpy() for k in ("x", "T", "st", "sx") if d.get(k) is not None}


def run_cases(mc) -> dict:
    import torch
    from mc_inputs import (mixed_batch, network_13, network_33, robertson_cells, robertson_network,
                           synthetic_cells, synthetic_sources)
    n13, n33, rob = network_13(), network_33(), robertson_network()
    h13, h33, hrob = mc.Network(n13), mc.Network(n33), mc.Network(rob)
    out = {}

    def put(name, d):
        for k, v in _out(d).items():
            out[f"{name}.{k}"] = v

    # cost-ordered persistent launch, FP32 matrix with its FP64 retry, hand-off
    # after 1024 attempts (the record list, 512 entries here, takes every cell
    # that reaches it, so which cells are handed off does not depend on timing)
    c = synthetic_cells(n13, 4096, seed=11)
    d = _dev(c, 4096 + 5, torch)
    o = mc.mc_burn_opts_default(lu_precision=32, variant=mc.MC_VARIANT_PERSISTENT, straggler_steps=HANDOFF)
    mc.mc_burn_batch(h13, o, 4096, 1e10, d["x"], 4096 + 5, d["T"], d["nd"], None, d["st"], d["sx"])
    put("fused", d)
    # plain FP64 and warp-per-cell
    c = synthetic_cells(n13, 2048, seed=12)
    d = _dev(c, 2048, torch)
    mc.mc_burn_batch(h13, mc.mc_burn_opts_default(lu_precision=64, variant=mc.MC_VARIANT_PLAIN), 2048, 1e10,
                     d["x"], 2048, d["T"], d["nd"], None, d["st"], d["sx"])
    put("plain", d)
    c = synthetic_cells(n13, 512, seed=13)
    d = _dev(c, 512, torch)
    mc.mc_burn_batch(h13, mc.mc_burn_opts_default(lu_precision=64, variant=mc.MC_VARIANT_WARP), 512, 1e10,
                     d["x"], 512, d["T"], d["nd"], None, d["st"], d["sx"])
    put("warp", d)
    # 33-ODE network (warp-per-cell), FP32 matrix with retry
    c = synthetic_cells(n33, 512, seed=14)
    d = _dev(c, 512, torch)
    mc.mc_burn_batch(h33, mc.mc_burn_opts_default(lu_precision=32), 512, 1e10, d["x"], 512, d["T"], d["nd"], None,
                     d["st"], d["sx"])
    put("net33", d)
    # Robertson with per-cell rate factors
    c = robertson_cells(4096, 15)
    d = _dev(c, 4096, torch)
    mc.mc_burn_batch(hrob, mc.mc_burn_opts_default(lu_precision=64), 4096, 40.0, d["x"], 4096, d["T"], d["nd"],
                     d["ks"], d["st"], d["sx"])
    put("robertson", d)
    # host buffers, ld > n
    c = synthetic_cells(n13, 1000, seed=16)
    ld = 1003
    hx = np.full((n13.n_species, ld), np.nan)
    hx[:, :1000] = c["x"]
    hT = np.full(ld, np.nan)
    hT[:1000] = c["T"]
    hnd = np.ones(ld)
    hnd[:1000] = c["ndens"]
    hst = np.full(ld, -7, dtype=np.int32)
    hsx = np.zeros((8, ld), dtype=np.int32)
    mc.mc_burn_batch(h13, mc.mc_burn_opts_default(lu_precision=32), 1000, 1e10, hx, ld, hT, hnd, None, hst, hsx)
    out.update({"host.x": hx, "host.T": hT, "host.st": hst, "host.sx": hsx})
    # constant sources
    c = synthetic_cells(n13, 1024, seed=17)
    src = torch.as_tensor(synthetic_sources(n13, c, 1e10, seed=18, scale=0.05), device="cuda")
    d = _dev(c, 1024, torch)
    mc.mc_burn_batch_sdc(h13, mc.mc_burn_opts_default(lu_precision=64), 1024, 1e10, d["x"], 1024, d["T"], d["nd"],
                         None, src, d["st"], d["sx"])
    put("sdc", d)
    # retry ladder: a tight step cap, then a forward-difference Jacobian, then RKC
    c = synthetic_cells(n13, 1024, seed=19)
    d = _dev(c, 1024, torch)
    rg = torch.full((1024,), -1, dtype=torch.int32, device="cuda")
    rungs = [mc.rung(max_steps=60, lu_precision=32), mc.rung(max_steps=300, jacobian=mc.MC_JAC_FD),
             mc.rung(method=mc.MC_METHOD_RKC, max_steps=400)]
    mc.mc_burn_ladder(h13, rungs, 1024, 1e10, d["x"], 1024, d["T"], d["nd"], None, d["st"], d["sx"], rg)
    put("ladder", d)
    out["ladder.rung"] = rg.cpu().numpy()
    # mixed launch over three networks (bounds checked; stores are not counted here)
    mb = mixed_batch(3 * 256, seed=20, hot_fraction=0.01)
    segs, keep = [], []
    for (net, cc, idx), h, dt in zip(mb["groups"], (hrob, h13, h33), (40.0, 1e10, 1e10)):
        n = len(idx)
        dd = _dev(cc, n, torch)
        keep.append((net.name, dd))
        segs.append(mc.segment(h, n, n, dd["x"], dd["T"], dd["nd"], dd["ks"], dd["st"], dd["sx"], dt=dt))
    mc.mc_burn_mixed(segs, mc.mc_burn_opts_default(lu_precision=64), 1e10)
    for name, dd in keep:
        put("mixed_" + name, dd)
    torch.cuda.synchronize()
    return out


if __name__ == "__main__":
    import torch

    import paper_2608_06466_b300 as mc
    torch.cuda.set_device(0)
    mc.mc_bounds_reset(0)
    res = run_cases(mc)
    rep = mc.mc_bounds_report(0)
    res.update({"report." + k: np.array(v) for k, v in rep.items()})
    res["library"] = np.array(mc.LIB_PATH)
    np.savez(sys.argv[1], **res)
