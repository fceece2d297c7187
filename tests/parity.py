"""Parity rule between the CUDA path and the CPU oracle (used by the GPU
tests, the smoke check and the benchmark's sampled check).

Both sides run the same integrator spec, but a stiff burn with an energy
equation can amplify a last-bit difference (FMA contraction, a libm ulp) into
a different step sequence: then two correct integrations differ by their own
integration error, which at rtol = 1e-6 can exceed 1e-5 (the oracle compiled
with and without FMA contraction differs that much on ~3 % of the 13-ODE
cells). So each cell is classified by the oracle itself:

  stable     the oracle's result moves by < 1e-8 (relative) both when the
             inputs move by a small relative amount (1e-13 for the FP64 path,
             whose differences are roundoff; 1e-9 for the FP32-matrix path,
             whose Newton iterates differ at ~1e-7 of a correction, i.e. ~1e-13
             of the state, and may stop one iteration apart) and when the
             oracle is recompiled with FMA contraction (its rounding twin): the
             result is a well-defined function of the inputs at this level, and
             the CUDA path must match it:
             |g - o| <= 1e-5 |o| + 10 atol (abundances), |g - o| <= 1e-5 |o| (T).
  sensitive  otherwise: several results are correct, and a single run's error
             against the true solution is random-like (the FMA-compiled oracle
             has the same error distribution as the oracle, cell by cell ratios
             up to 1000x). So the CUDA path must be as accurate as the oracle in
             distribution against a tight-tolerance oracle t, with
             e = max_i |a_i - t_i| / (|t_i| + 1e-4) per cell (and |T - t_T|/t_T):
             every cell e_g <= 10 max(e_o) + 1e-4, median(e_g) <= 3 median(e_o)
             + 1e-6, p90(e_g) <= 3 p90(e_o) + 1e-5 (the floors keep samples of a
             few dozen cells from failing on noise; they sit well below the
             ~1e-5..1e-3 global errors of these cells).

Statuses must agree except for cells whose oracle attempt count is within 1 %
of the step cap.

The FP32-matrix form is a different integration, not a rounding variant of
the oracle's: with an FP32 iteration matrix the Newton iterates differ from the
FP64 ones, so the iteration stops at a different point inside its convergence
bound (CORTES = 0.1 of the local tolerance, ~1e-7 of the state per step), and
over a cell's history those differences add up like a global error (measured:
up to ~2e-4 on the 33-ODE network). So for it every finished cell gets the
distribution check above (as accurate as the oracle against the tight
solution), stable cells must stay within 1000 (rtol |o| + atol) of the oracle,
i.e. 1000 error weights (a gross-error bar above the oracle's own integration
error, which reaches ~1e-4 relative on stable 33-ODE cells), and the
per-result deviation from the FP64 oracle is reported
(stable_within_1e-5_frac, max_rel_x_stable)."""
from __future__ import annotations

import numpy as np

RTOL = 1e-5
STABLE_MOVE = 1e-8
PERTURB = 1e-13


def _agree(a, o):
    move = np.abs(a[0] - o[0]) / (np.abs(o[0]) + 1e-4)
    ok = (move < STABLE_MOVE).all(axis=0) & (a[2] == o[2])
    if o[1] is not None:
        ok &= np.abs(a[1] - o[1]) < STABLE_MOVE * np.abs(o[1])
    return ok


def classify(onet, cells, dt, burn, index=None, perturb=PERTURB, twin=True, **kw):
    """Oracle result and the stability mask (see module doc); ``burn`` is
    oracle.burn, ``onet`` its network. twin=True also runs the oracle's
    FMA-contracted rounding twin where the host supports it."""
    o = burn(onet, cells, dt, index=index, **kw)
    pc = dict(cells)
    pc["x"] = np.asarray(cells["x"]) * (1.0 + perturb)
    if cells.get("T") is not None:
        pc["T"] = np.asarray(cells["T"]) * (1.0 - perturb)
    stable = _agree(burn(onet, pc, dt, index=index, **kw), o)
    if twin:
        import platform
        if platform.machine() in ("x86_64", "AMD64"):
            import oracle
            tw = oracle.oracle.rounding_twin()
            stable &= _agree(tw.burn(tw.OracleNetwork(onet.net), cells, dt, index=index, **kw), o)
    return o, stable


def compare(g_x, g_T, g_s, o_x, o_T, o_s, o_stats, stable=None, tight=None, atol=1e-10,
            max_steps=100000, rtol=RTOL, fp32_matrix=False):
    """g_*: CUDA results; o_*: oracle; stable: mask from classify (None = all
    cells stable); tight: (x, T) of a tight-tolerance oracle run, needed when
    some cells are sensitive."""
    n = g_s.size
    if stable is None:
        stable = np.ones(n, dtype=bool)
    near_cap = o_stats[0] + o_stats[1] + o_stats[2] >= 0.99 * max_steps
    status_bad = (g_s != o_s) & ~near_cap
    both_ok = (g_s == 0) & (o_s == 0)
    dx = np.abs(g_x - o_x)
    strict = both_ok & stable
    if fp32_matrix:
        x_bad = ((dx > 1e3 * (1e-6 * np.abs(o_x) + atol)) & strict[None, :]).any(axis=0)
        bar = 1e-3
    else:
        x_bad = ((dx > rtol * np.abs(o_x) + 10.0 * atol) & strict[None, :]).any(axis=0)
        bar = rtol
    within = ((dx <= rtol * np.abs(o_x) + 10.0 * atol) | ~strict[None, :]).all(axis=0)
    big = (np.abs(o_x) >= atol / 1e-6) & strict[None, :]
    rel = np.where(big, dx / np.maximum(np.abs(o_x), 1e-300), 0.0)
    T_bad = np.zeros(n, dtype=bool)
    rep = {"cells": int(n), "status_mismatch": int(status_bad.sum()), "stable": int(strict.sum()),
           "sensitive": int((both_ok & ~stable).sum()),
           "max_rel_x_stable": float(rel.max()) if rel.size else 0.0}
    if g_T is not None and o_T is not None:
        relT = np.where(strict, np.abs(g_T - o_T) / np.abs(o_T), 0.0)
        T_bad |= relT > bar
        within &= relT <= rtol
        rep["max_rel_T_stable"] = float(relT.max())
    rep["stable_within_1e-5_frac"] = float(within[strict].mean()) if strict.any() else 1.0
    sens = both_ok if fp32_matrix else (both_ok & ~stable)
    rep["sensitive_pass"] = True
    if sens.any():
        if tight is None:
            raise ValueError("sensitive cells need a tight-tolerance oracle result")
        tx, tT = tight
        eg = (np.abs(g_x - tx) / (np.abs(tx) + 1e-4)).max(axis=0)
        eo = (np.abs(o_x - tx) / (np.abs(tx) + 1e-4)).max(axis=0)
        if g_T is not None:
            eg = np.maximum(eg, np.abs(g_T - tT) / tT)
            eo = np.maximum(eo, np.abs(o_T - tT) / tT)
        eg, eo = eg[sens], eo[sens]
        worst = eg > 10.0 * eo.max() + 1e-4
        med_ok = np.median(eg) <= 3.0 * np.median(eo) + 1e-6
        p90_ok = np.percentile(eg, 90) <= 3.0 * np.percentile(eo, 90) + 1e-5
        rep["sensitive_err_gpu_p50_p90_max"] = [float(np.median(eg)), float(np.percentile(eg, 90)), float(eg.max())]
        rep["sensitive_err_oracle_p50_p90_max"] = [float(np.median(eo)), float(np.percentile(eo, 90)), float(eo.max())]
        rep["sensitive_pass"] = bool(med_ok and p90_ok and not worst.any())
        x_bad[np.flatnonzero(sens)[worst]] = True
    rep["x_fail"] = int(x_bad.sum())
    rep["T_fail"] = int(T_bad.sum())
    rep["pass"] = (rep["status_mismatch"] == 0 and rep["x_fail"] == 0 and rep["T_fail"] == 0
                   and rep["sensitive_pass"])
    return rep
