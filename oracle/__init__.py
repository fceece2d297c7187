"""CPU FP64 oracle for the per-cell burn -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package. It shares no code with the CUDA path
(``paper_2608_06466_b300``), and the CUDA path never imports it.

The arithmetic lives in ``mc_oracle.c`` (plain C, IEEE double, no FMA
contraction); this module compiles it with gcc and binds it with ctypes.
"""
from .oracle import (  # noqa: F401
    OracleNetwork, build, burn, burn_ladder, lib, linear_integrate, linear_integrate_steps, linear_fixed_steps,
    bdf_coeffs,
    err_coef_qm1, err_coef_qp1, order_raise_coef, order_lower_coefs, lu_factor, lu_solve,
    predict, retract, rkc_linear_step, rkc_linear_integrate, linear_initial_step, linear_newton,
    NSTAT, STATUS,
)
