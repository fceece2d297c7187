"""Seeded synthetic inputs for the per-cell burn.

This package is the only code shared by the CPU oracle tests and the CUDA
path. It generates data and nothing else: reaction networks (species,
stoichiometry, rate parameters, reaction energies), per-cell initial states
constant source terms and request streams. None of the burn's arithmetic (rates, right-hand side,
Jacobian, integrator) lives here.
"""
from .networks import Network, robertson_network, synthetic_network, network_13, network_33
from .cells import robertson_cells, synthetic_cells, synthetic_sources, mixed_batch
from .requests import box_request_stream

__all__ = [
    "Network", "robertson_network", "synthetic_network", "network_13", "network_33",
    "robertson_cells", "synthetic_cells", "synthetic_sources", "mixed_batch", "box_request_stream",
]
