"""Seeded stream of AMR-box burn requests for the serving loop."""
from __future__ import annotations

import numpy as np


def box_request_stream(n_requests: int, rate_per_s: float, seed: int = 7,
                       edge_range=(16, 128), nets=("net13", "net33")) -> list[dict]:
    """Poisson arrivals at ``rate_per_s``; each request is a cubic box with edge
    L log-uniform in ``edge_range`` (rounded to an integer, cells = L^3) on a
    network drawn 50/50 from ``nets``, with its own cell seed."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_per_s, size=n_requests)
    t = np.cumsum(gaps)
    L = np.rint(np.exp(rng.uniform(np.log(edge_range[0]), np.log(edge_range[1]), n_requests))).astype(int)
    which = rng.integers(0, len(nets), size=n_requests)
    cell_seed = rng.integers(1, 2**31 - 1, size=n_requests)
    return [{"t_arrive": float(t[i]), "edge": int(L[i]), "n_cells": int(L[i]) ** 3,
             "net": nets[which[i]], "cell_seed": int(cell_seed[i])} for i in range(n_requests)]
