"""Seeded per-cell initial states (structure-of-arrays, species-major)."""
from __future__ import annotations

import numpy as np

from .networks import Network, robertson_network, network_13, network_33


def _log_uniform(rng: np.random.Generator, lo: float, hi: float, n: int) -> np.ndarray:
    return np.exp(rng.uniform(np.log(lo), np.log(hi), size=n))


def robertson_cells(n_cells: int, seed: int = 1) -> dict:
    """Robertson cells: y0 = (1, 0, 0); each of k1, k2, k3 scaled per cell by an
    independent factor log-uniform in [0.5, 2] (``rate_scale`` [3, n])."""
    rng = np.random.default_rng(seed)
    scale = _log_uniform(rng, 0.5, 2.0, 3 * n_cells).reshape(3, n_cells)
    x = np.zeros((3, n_cells))
    x[0] = 1.0
    return {"x": x, "T": None, "ndens": None, "rate_scale": scale}


def synthetic_cells(net: Network, n_cells: int, seed: int, hot_fraction: float = 0.0,
                    T_range=(10.0, 1.0e4), n_range=(1.0, 1.0e8),
                    hot_T_range=(1.0e4, 1.0e5)) -> dict:
    """Cells for an energy-equation network.

    T log-uniform in ``T_range`` K, n log-uniform in ``n_range`` cm^-3. Element
    abundances are uniform in [0.1, 1] per cell and element (then normalised);
    each element's share sits on its monatomic species, and every species also
    starts with a 1e-6 share, so the number fractions sum to 1. A fraction
    ``hot_fraction`` of the cells instead draws T log-uniform in ``hot_T_range``.
    """
    rng = np.random.default_rng(seed)
    S, E = net.n_species, net.n_elements
    T = _log_uniform(rng, *T_range, n_cells)
    nd = _log_uniform(rng, *n_range, n_cells)
    ab = rng.uniform(0.1, 1.0, size=(E, n_cells))
    ab /= ab.sum(axis=0, keepdims=True)
    floor = 1.0e-6
    x = np.full((S, n_cells), floor)
    mono = [int(np.flatnonzero((net.composition == np.eye(E, dtype=np.int32)[e]).all(axis=1))[0])
            for e in range(E)]
    for e in range(E):
        x[mono[e]] += ab[e] * (1.0 - S * floor)
    if hot_fraction > 0.0:
        hot = rng.random(n_cells) < hot_fraction
        T[hot] = _log_uniform(rng, *hot_T_range, int(hot.sum()))
    else:
        hot = np.zeros(n_cells, dtype=bool)
    return {"x": x, "T": T, "ndens": nd, "rate_scale": None, "hot": hot}


def mixed_batch(n_cells: int, seed: int = 6, hot_fraction: float = 0.01) -> dict:
    """Mixed batch: each cell carries a network id drawn evenly from
    {Robertson-3, net13, net33}; 1 % of the energy-network cells are hot.

    Returns ``{"net_id": int8 [n], "groups": [(Network, cells_dict, index)]}``
    where ``index`` lists the global cell numbers of each group in order."""
    rng = np.random.default_rng(seed)
    net_id = rng.integers(0, 3, size=n_cells).astype(np.int8)
    nets = [robertson_network(), network_13(), network_33()]
    groups = []
    for g, net in enumerate(nets):
        idx = np.flatnonzero(net_id == g)
        if g == 0:
            cells = robertson_cells(len(idx), seed=seed * 7 + 1)
        else:
            cells = synthetic_cells(net, len(idx), seed=seed * 7 + 1 + g, hot_fraction=hot_fraction)
        groups.append((net, cells, idx))
    return {"net_id": net_id, "groups": groups}


def synthetic_sources(net: Network, cells: dict, dt: float, seed: int, scale: float = 0.1) -> np.ndarray:
    """Constant per-cell sources [n_ode, n] of the size an advective coupling
    term has: each species' source moves it by up to ``scale`` of its initial
    fraction over dt (uniform in [-scale, scale], relative); the energy
    component's source is uniform in [-scale, scale] x 1e-4 T / dt (eV per unit
    density and second; 1e-4 T is of the order of u for fractions summing to 1)."""
    rng = np.random.default_rng(seed)
    x = np.asarray(cells["x"], dtype=np.float64)
    ref = [x]
    if net.energy_eq:
        ref.append(1e-4 * np.asarray(cells["T"], dtype=np.float64)[None, :])
    ref = np.concatenate(ref, axis=0)
    return rng.uniform(-scale, scale, size=ref.shape) * ref / dt
