"""Convenience layer over the C ABI: move a cell batch into device memory
(torch tensors), call mc_burn_batch, bring results back. Marshalling only."""
from __future__ import annotations

import numpy as np

from . import _mc


def to_device(cells: dict, device="cuda"):
    """Cell dict (numpy SoA as produced by mc_inputs) -> dict of torch tensors."""
    import torch

    out = {}
    for k in ("x", "T", "ndens", "rate_scale"):
        v = cells.get(k)
        out[k] = None if v is None else torch.as_tensor(np.ascontiguousarray(v, dtype=np.float64), device=device)
    n = cells["x"].shape[1]
    out["status"] = torch.full((n,), -1, dtype=torch.int32, device=device)
    out["stats"] = torch.zeros((_mc.MC_NSTAT, n), dtype=torch.int32, device=device)
    return out


def burn_device(net: "_mc.Network", d: dict, dt: float, opts=None, stream=None):
    """Burn a device-resident cell dict (from to_device) in place."""
    n = d["x"].shape[1]
    return _mc.mc_burn_batch(net, opts, n, dt, d["x"], n, d["T"], d["ndens"], d["rate_scale"], d["status"],
                             d["stats"], stream)


def burn(net: "_mc.Network", cells: dict, dt: float, opts=None, device="cuda"):
    """Burn numpy cells on the GPU; returns (x, T, status, stats) as numpy."""
    import torch

    d = to_device(cells, device)
    burn_device(net, d, dt, opts)
    torch.cuda.synchronize()
    T = None if d["T"] is None else d["T"].cpu().numpy()
    return d["x"].cpu().numpy(), T, d["status"].cpu().numpy(), d["stats"].cpu().numpy()
