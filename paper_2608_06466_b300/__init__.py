"""B300-native per-cell stiff burn: VODE-style BDF integration of reaction
networks (with an ideal-gas energy equation) over an operator-split step, one
cell per GPU lane, behind the C ABI in include/mc.h.

The Python layer only marshals arguments into libmc.so; importing it without
the built library raises ImportError (there is no CPU fallback).
"""
from ._mc import (  # noqa: F401
    CELL_STATUS, MC_NOALLOC_MAX_CELLS, MC_NSTAT, MC_VARIANT_AUTO, MC_VARIANT_PERSISTENT, MC_VARIANT_PLAIN, MC_VARIANT_WARP, STAT_NAMES,
    Graph, MCError, Network, Server, check, lib, mc_burn_batch, mc_burn_batch_noalloc, mc_burn_batch_sdc, mc_burn_mixed, mc_burn_opts,
    mc_autotune, mc_burn_opts_default, mc_graph_create, mc_last_error, mc_launch_count, mc_alloc_count, mc_network_create,
    mc_network_destroy, mc_network_rates, mc_network_rhs, mc_probe_fma_rate, mc_server_create, segment,
    MC_JAC_ANALYTIC, MC_JAC_FD, MC_METHOD_BDF, MC_METHOD_RKC, mc_burn_ladder, mc_rung, rung,
    LIB_PATH, mc_bounds_report, mc_bounds_reset, MC_STAGING_AUTO, MC_STAGING_SHARED, MC_STAGING_LANE,
)
from .api import burn  # noqa: F401
