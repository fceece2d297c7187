"""Benchmark of the per-cell burn on B300.

Workload (one "step" = one burn of the whole batch): the precision form on the
13-ODE synthetic network (12 species from 3 elements + the energy equation, 40
reversible reactions), 2^22 cells per GPU, T log-uniform [10, 1e4] K, n
log-uniform [1, 1e8] cm^-3, dt = 1e10 s, rtol = 1e-6, atol = 1e-10. The
headline arm is the FP32-iteration-matrix persistent path (FP32 LU refined
with FP64 residuals, FP64 retry of the cells it cannot serve). Beside it, on
one GPU: the FP64-matrix persistent path on the same cells (same scheduling,
so the pair isolates the matrix precision) and the plain FP64 path (one
thread per cell, one launch, no refill) on the 2^20-cell plain FP64 workload.
Inputs are reset from a device-resident copy before every step (inside the
timed region); the inputs (470 MB) exceed L2 and L2 is flushed between steps.

``--config mixed`` times the batched uneven-work form instead: one persistent
launch over 2^22 cells split evenly over Robertson (3 ODEs, t = 40), net13 and
net33 (33 ODEs), 1 % hot cells, replayed from a captured CUDA graph.

Prints one JSON line (rank 0). ``--impl reference`` times the CPU FP64 oracle
on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cells/s at rtol=1e-6 (FP32-LU persistent vs FP64 plain); p50/p99 burn latency"
N_CELLS = 1 << 22          # the precision form's workload
N_PLAIN = 1 << 20          # the plain FP64 workload
DT = 1.0e10
CELL_SEED = 4              # precision-form cells
PLAIN_SEED = 3             # plain-FP64 cells
ORACLE_SAMPLE = 131072     # cells of the oracle's timed sample (baseline and reference arm)
PARITY_SAMPLE = 4096       # cells of each timed burn recomputed by the oracle

# ---- FP64-pipe roofline model ---------------------------------------------
# FP64 flops per unit of work (an FMA is 2 flops, an add or a multiply 1).
# Measured by ncu's thread-level DFMA/DADD/DMUL counters on the library's own
# evaluation kernels (python -m paper_2608_06466_b300.profile_case eval, 2^18
# states each):
#   RHS_FLOPS_PER_REACTION   one reaction of a right-hand side: two table
#                            exponentials and their arguments, the mass-action
#                            products, the scatter and the energy term
#   RHS_FLOPS_FIXED          the rest of a right-hand side (EOS temperature,
#                            log T, 1/T, sums)
# Counted from the code (no transcendental inside):
#   Jacobian   a right-hand side's rates plus 22 flops per reaction for the
#              derivatives and n (S + 1) for the EOS chain rule
#   FP64 LU    (2/3) n^3 + n^2 / 2; an FP32 LU costs the FP64 pipe nothing
#   solve      FP64: 2 n^2; FP32: one refinement sweep, 2 n^2 + 5 n (further
#              sweeps are not counted, so the FP32 figure is a lower bound)
#   attempt    (q(q+1)/2 + 2(q+1) + 3) n with q = 3, the weights' n reciprocals
#              charged 1 flop each
RHS_FLOPS_PER_REACTION = 51.75   # k_rates slope 38.8 (two exponentials with their arguments) + 13
RHS_FLOPS_FIXED = 47.0           # k_rhs on net13: 2117 flops per right-hand side = 47 + 40 x 51.75


def fp64_flops(S, R, n, stats, lu_precision):
    """Algorithmic FP64 flops of the work the per-cell counters record."""
    st = stats.astype(np.float64)
    attempts = st[0] + st[1] + st[2]
    f_rhs = RHS_FLOPS_FIXED + R * RHS_FLOPS_PER_REACTION
    f_jac = f_rhs + 22.0 * R + n * (S + 1)
    f_lu = (2.0 / 3.0) * n ** 3 + 0.5 * n * n if lu_precision == 64 else 0.0
    f_solve = 2.0 * n * n if lu_precision == 64 else 2.0 * n * n + 5.0 * n
    q = 3
    f_step = (q * (q + 1) / 2 + 2 * (q + 1) + 3) * n + n
    return float((st[3] * f_rhs + st[4] * f_jac + st[5] * f_lu + st[6] * f_solve + attempts * f_step).sum())


# DRAM traffic of the headline kernel (k_burn_fused<13, float>) per step
# attempt, from an ncu capture of one launch on 2^20 net13 cells
# (python -m paper_2608_06466_b300.profile_case burn --cells 1048576 --lu 32
# --variant 2 --max-steps 3000: 2005.7 GB read + written over 243.8 M
# attempts); the traffic is lane state evicted past L2 and grows with
# attempts, not cells, so the timed run's attempts scale it.
DRAM_BYTES_PER_ATTEMPT = 8228.0

# where the nvidia-smi clock samples of the timed region are written
LOG_DIR = os.environ.get("MC_BENCH_LOG_DIR", os.path.join(tempfile.gettempdir(), "mc_bench"))


# ---- multi-rank bookkeeping (one process per GPU; the cells shard with no
# exchange, so the only collectives are a barrier and a max of the timings)
def shard_seed(rank: int) -> int:
    """Cell seed of a rank's shard: every rank burns its own, independent cells."""
    return CELL_SEED + 1000 * rank


def max_over_ranks(x: float, world: int, device: str = "cpu") -> float:
    """Largest x over all ranks: the slowest rank sets the job's time. Needs an
    initialised process group when world > 1 (NCCL wants device="cuda")."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(cells_per_rank: int, world: int, ms: float) -> float:
    """Whole-job cells/s: the cells of every rank over the slowest rank's time."""
    return cells_per_rank * world / (ms / 1e3)


def clock_sampler_start(path):
    q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")
    try:
        f = open(path, "w")
        return subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits", "-lms", "200"],
                                stdout=f, stderr=subprocess.DEVNULL), f
    except Exception:
        return None, None


def clock_sampler_stop(proc, f, path, device_index=0):
    if proc is None:
        return None
    proc.terminate()
    try:
        proc.wait(timeout=5)
    except Exception:
        proc.kill()
    f.close()
    sm, mx, reasons = [], 0.0, set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in open(path):
        p = [v.strip() for v in line.split(",")]
        if len(p) < 9 or not p[0].isdigit() or int(p[0]) != device_index:
            continue
        try:
            sm.append(float(p[1]))
            mx = max(mx, float(p[2]))
        except ValueError:
            continue
        for name, v in zip(names, p[5:9]):
            if v.lower() == "active":
                reasons.add(name)
    if not sm:
        return None
    return {"sm_mhz": float(statistics.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
            "samples": len(sm)}


def cpu_baseline(net, n_sample, seed):
    """The oracle as it stands, on a bounded sample of the workload, all host cores."""
    import oracle
    from mc_inputs import synthetic_cells
    cells = synthetic_cells(net, n_sample, seed=seed)
    on = oracle.OracleNetwork(net)
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    _, _, status, _ = oracle.burn(on, cells, DT, nthreads=cores)
    dt = time.perf_counter() - t0
    return {"value": n_sample / dt, "unit": "cells/s", "cores": cores, "kind": "oracle",
            "sample": f"{n_sample} cells of the same workload (seed {seed}), FP64 oracle, "
                      f"{cores} threads, {dt:.1f} s; cells/s extrapolates linearly",
            "ok_fraction": float(np.mean(status == 0))}


def parity_sample(net, cells, idx, gx, gT, gs):
    """The oracle's verdict on sampled cells of a timed burn (tests/parity.py)."""
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import oracle
    from parity import classify, compare
    on = oracle.OracleNetwork(net)
    o, stable, reprobe = classify(on, cells, DT, oracle.burn, index=idx, with_reprobe=True)
    t = oracle.burn(on, cells, DT, rtol=1e-10, atol=1e-16, index=idx)
    rep = compare(gx, gT, gs, o[0], o[1], o[2], o[3], stable=stable, tight=(t[0], t[1]), reprobe=reprobe)
    # the largest relative difference over every sampled result (stable and
    # sensitive cells, abundances with |o| above 10 atol, and T), status OK on both sides
    both = (gs == 0) & (o[2] == 0)
    ox, gx_ = o[0][:, both], gx[:, both]
    big = np.abs(ox) > 1e-9
    rel_all = float((np.abs(gx_ - ox)[big] / np.abs(ox)[big]).max()) if big.any() else 0.0
    relT_all = None
    if gT is not None and o[1] is not None and both.any():
        relT_all = float((np.abs(gT[both] - o[1][both]) / np.abs(o[1][both])).max())
    # the same figure for the oracle's own rounding twin (the same algorithm with
    # FMA contraction): how far two correct integrations of these cells can differ
    tw = oracle.oracle.rounding_twin()
    w = tw.burn(tw.OracleNetwork(net), cells, DT, index=idx)
    both_t = (w[2] == 0) & (o[2] == 0)
    bt = np.abs(o[0][:, both_t]) > 1e-9
    rel_twin = float((np.abs(w[0][:, both_t] - o[0][:, both_t])[bt] / np.abs(o[0][:, both_t])[bt]).max()) \
        if bt.any() else 0.0
    return {"sampled_cells": int(idx.size), "pass": rep["pass"], "stable": rep["stable"],
            "max_rel_x_all": rel_all, "max_rel_T_all": relT_all, "max_rel_x_all_oracle_twin": rel_twin,
            "sensitive": rep["sensitive"], "reclassified": rep["reclassified"],
            "max_rel_x_stable": rep["max_rel_x_stable"], "max_rel_T_stable": rep.get("max_rel_T_stable"),
            "status_mismatch": rep["status_mismatch"],
            "sensitive_err_gpu_p50_p90_max": rep.get("sensitive_err_gpu_p50_p90_max"),
            "sensitive_err_oracle_p50_p90_max": rep.get("sensitive_err_oracle_p50_p90_max")}


def steady_throughput(done, window_s):
    """Cells per second of a closed loop from its completions [(time, cells)]:
    the cells completed after the first completion and inside the window,
    over the time between the two (the ramp-up before the first completion
    and the work in flight at the window's end are left out). With fewer than
    two completions inside the window, every request over the time to the
    last completion. Returns (cells/s, completions inside the window)."""
    done = sorted(done)
    inside = [d for d in done if d[0] <= window_s]
    if len(inside) >= 2:
        return sum(c for _, c in inside[1:]) / max(window_s - inside[0][0], 1e-9), len(inside)
    if not done:
        return 0.0, 0
    return sum(c for _, c in done) / max(done[-1][0], 1e-9), len(inside)


def serving_measurement(mc, window_s=40.0, seed=7, edge_range=(16, 48), concurrency=8):
    """Serving loop on AMR-box requests (edge L log-uniform in edge_range,
    cells = L^3, 50/50 net13 / net33, FP32 iteration matrix, 150 GB budget).

    Saturation: a closed loop that keeps `concurrency` requests in flight for
    window_s seconds; capacity = cells of the requests completed after the
    first completion and inside the window / the time between the two (the
    ramp-up before the first completion and the work still in flight at the
    end are both left out). Then Poisson arrivals at 0.5x and 0.9x of that
    capacity for window_s seconds each, drained after the window; latency =
    completion minus submission, per request."""
    import time as _t
    from mc_inputs import box_request_stream, network_13, network_33, synthetic_cells
    nets = {"net13": network_13(), "net33": network_33()}
    handles = {k: mc.Network(v) for k, v in nets.items()}
    opts = mc.mc_burn_opts_default(lu_precision=32)

    def make(r):
        net = nets[r["net"]]
        c = synthetic_cells(net, r["n_cells"], seed=r["cell_seed"])
        return (r["net"], r["n_cells"], np.ascontiguousarray(c["x"]), c["T"].copy(), c["ndens"].copy(),
                np.zeros(r["n_cells"], dtype=np.int32))

    def submit(srv, b):
        name, n, x, T, nd, st = b
        return srv.submit(handles[name], n, DT, x, n, T, nd, st)

    # warm the kernels and the per-stream scratch once (the host buffers must
    # outlive their requests)
    srv = mc.Server(0, 150 << 30, opts)
    warm = [make(r) for r in box_request_stream(2, 1.0, seed=seed + 99, edge_range=(16, 16),
                                                nets=("net13", "net33"))]
    for b in warm:
        submit(srv, b)
    srv.drain(600)
    srv.close()
    del warm

    # saturation: closed loop
    pool = box_request_stream(4096, 1.0, seed=seed, edge_range=edge_range)
    srv = mc.Server(0, 150 << 30, opts)
    live, done, k = {}, [], 0
    t0 = _t.perf_counter()
    while True:
        now = _t.perf_counter() - t0
        while now < window_s and len(live) < concurrency:
            b = make(pool[k])
            k += 1
            live[submit(srv, b)] = b
        for rid in list(live):
            rc, info = srv.poll(rid)
            if rc == 0:
                done.append((_t.perf_counter() - t0, live[rid][1]))
                del live[rid]
        if not live and now >= window_s:
            break
        _t.sleep(0.002)
    srv.drain(3600)
    srv.close()
    lam_cells, done_n = steady_throughput(done, window_s)
    mean_cells = float(np.mean([r["n_cells"] for r in pool]))
    out = {"lambda_sat_cells_per_s": lam_cells, "saturation_requests_completed": done_n,
           "mean_cells_per_request": mean_cells, "edge_range": list(edge_range), "window_s": window_s,
           "concurrency": concurrency, "lu_precision": 32, "loads": []}
    if not lam_cells > 0.0:
        return out  # nothing completed: no load levels to offer
    for load in (0.5, 0.9):
        rate = load * lam_cells / mean_cells
        reqs = box_request_stream(max(1, int(rate * window_s * 3) + 8), rate, seed=seed + int(load * 100),
                                  edge_range=edge_range)
        reqs = [r for r in reqs if r["t_arrive"] <= window_s] or reqs[:1]
        bufs = [make(r) for r in reqs]
        srv = mc.Server(0, 150 << 30, opts)
        ids = []
        t0 = _t.perf_counter()
        for r, b in zip(reqs, bufs):
            wait = r["t_arrive"] - (_t.perf_counter() - t0)
            if wait > 0:
                _t.sleep(wait)
            ids.append(submit(srv, b))
        srv.drain(3600)
        span = _t.perf_counter() - t0
        infos = [srv.poll(i)[1] for i in ids]
        srv.close()
        lat = np.array([i.t_done - i.t_submit for i in infos])
        cells = sum(b[1] for b in bufs)
        out["loads"].append({"load": load, "requests": len(ids), "rate_req_per_s": rate,
                             "p50_latency_s": float(np.percentile(lat, 50)),
                             "p99_latency_s": float(np.percentile(lat, 99)),
                             "cells_per_s": cells / span, "failed_cells": int(sum(i.n_failed for i in infos))})
    return out


def run_reference(args, rank, world):
    from mc_inputs import network_13
    net = network_13()
    if rank != 0:
        return
    n_sample = int(os.environ.get("MC_REF_SAMPLE", str(ORACLE_SAMPLE)))
    times = []
    for i in range(args.warmup + args.steps):
        b = cpu_baseline(net, n_sample, seed=CELL_SEED + 100 * i)
        if i >= args.warmup:
            times.append(n_sample / b["value"])
    ms = 1e3 * float(np.mean(times))
    value = n_sample / (ms / 1e3)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "cells/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "net13 synthetic kinetics, 12 species + energy, 40 reactions; "
                                   f"bounded sample of {n_sample} cells per step (seeds {CELL_SEED} + 100 i)",
                       "n_cells_per_step": n_sample, "dt_s": DT, "rtol": 1e-6, "atol": 1e-10},
            "cpu_baseline": {"value": value, "unit": "cells/s", "cores": os.cpu_count(), "kind": "oracle",
                             "sample": f"{n_sample} cells per step"},
            "e2e": {"value": value, "unit": "cells/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


MIXED_CELLS = 1 << 22
MIXED_SEED = 6
MIXED_DTS = (40.0, DT, DT)   # Robertson to t = 40, the energy networks over dt


def run_mixed(args, mc, world, rank, local, stream, flush, barrier, fp64_peak, fp32_peak):
    """The batched uneven-work form: 2^22 cells split evenly over Robertson,
    net13 and net33 (1 % hot cells), one persistent launch captured in a CUDA
    graph and replayed each step; inputs reset from device copies inside the
    timed region."""
    import torch
    from paper_2608_06466_b300.api import to_device
    from mc_inputs import mixed_batch
    n = args.cells
    batch = mixed_batch(n, seed=MIXED_SEED + 1000 * rank, hot_fraction=0.01)
    segs, keep = [], []
    for (net, cells, idx), dt in zip(batch["groups"], MIXED_DTS):
        h = mc.Network(net)
        d = to_device(cells)
        x0 = d["x"].clone()
        T0 = None if d["T"] is None else d["T"].clone()
        m = cells["x"].shape[1]
        segs.append(mc.segment(h, m, m, d["x"], d["T"], d["ndens"], d["rate_scale"], d["status"], d["stats"], dt=dt))
        keep.append((h, d, x0, T0, net, cells))
    # the FP64 iteration matrix: on this GPU the faster form for these networks
    # (cooperative FP64 LU; the 33-ODE matrices defeat FP32 refinement late in
    # a burn and send those cells to the FP64 retry)
    opts = mc.mc_burn_opts_default(lu_precision=64)
    # the mixed launch takes its grid, staging and hand-off from the
    # autotuner's pick for its thread-per-cell network with the most cells
    # (net13), timed here on a bounded sample of that segment (step cap 2000
    # per trial, so that the search ends in seconds)
    lead = max((k for k in keep if k[4].n_ode <= 16), key=lambda k: k[5]["x"].shape[1])
    lh, ld_, lnet = lead[0], lead[1], lead[4]
    m_lead = ld_["x"].shape[1]
    ns = min(16384, m_lead)
    t0 = time.perf_counter()
    best = mc.mc_autotune(lh, mc.mc_burn_opts_default(lu_precision=64, max_steps=2000), ns, DT, ld_["x"], m_lead,
                          ld_["T"], ld_["ndens"])
    tuned = {"network": lnet.name, "sample_cells": ns, "trial_max_steps": 2000,
             "seconds": round(time.perf_counter() - t0, 2), "variant": int(best.variant),
             "block_threads": int(best.block_threads), "blocks_per_sm": int(best.blocks_per_sm),
             "staging": int(best.staging), "straggler_steps": int(best.straggler_steps)}
    g = mc.mc_graph_create(segs, opts, DT)

    def reset():
        for (h, d, x0, T0, net, cells) in keep:
            d["x"].copy_(x0)
            if T0 is not None:
                d["T"].copy_(T0)

    def step():
        reset()
        g.launch(stream)

    ms, per, launches, clocks, k_timed, w_run = timed_steps(step, args.steps, args.warmup, stream, flush, barrier,
                                                           rank, local, True, args.max_timed_s, world)
    ms = max_over_ranks(ms, world, "cuda")
    flops, attempts, ok = 0.0, 0.0, 0
    results = []
    for (h, d, x0, T0, net, cells) in keep:
        st = d["stats"].cpu().numpy()
        flops += fp64_flops(net.n_species, net.n_reactions, net.n_ode, st, 64)
        attempts += float((st[0].astype(np.int64) + st[1] + st[2]).sum())
        s = d["status"].cpu().numpy()
        ok += int((s == 0).sum())
        results.append((d["x"].cpu().numpy(), None if d["T"] is None else d["T"].cpu().numpy(), s))
    # end to end: inputs from pinned host memory, graph replay, results back
    hosts = []
    for (h, d, x0, T0, net, cells) in keep:
        hx = torch.from_numpy(np.ascontiguousarray(cells["x"])).pin_memory()
        hT = None if T0 is None else torch.from_numpy(np.ascontiguousarray(cells["T"])).pin_memory()
        ox = torch.empty_like(hx).pin_memory()
        oT = None if hT is None else torch.empty_like(hT).pin_memory()
        os_ = torch.empty(d["status"].shape, dtype=torch.int32).pin_memory()
        hosts.append((hx, hT, ox, oT, os_))
    e2e_ms = []
    h2d = d2h = 0
    for i in range(1 + max(1, min(args.steps, 2))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for (h, d, x0, T0, net, cells), (hx, hT, ox, oT, os_) in zip(keep, hosts):
            d["x"].copy_(hx, non_blocking=True)
            if hT is not None:
                d["T"].copy_(hT, non_blocking=True)
        g.launch(stream)
        for (h, d, x0, T0, net, cells), (hx, hT, ox, oT, os_) in zip(keep, hosts):
            ox.copy_(d["x"], non_blocking=True)
            if oT is not None:
                oT.copy_(d["T"], non_blocking=True)
            os_.copy_(d["status"], non_blocking=True)
        torch.cuda.synchronize()
        if i > 0:
            e2e_ms.append((time.perf_counter() - t0) * 1e3)
    for (hx, hT, ox, oT, os_) in hosts:
        h2d += hx.numel() * 8 + (0 if hT is None else hT.numel() * 8)
        d2h += ox.numel() * 8 + (0 if oT is None else oT.numel() * 8) + os_.numel() * 4
    g.close()
    e2e_v = job_throughput(n, world, max_over_ranks(float(np.mean(e2e_ms)), world, "cuda"))
    parity, cpu = None, None

    def oracle_legs():
        import oracle
        parity = []
        for (h, d, x0, T0, net, cells), (gx, gT, gs), dt in zip(keep, results, MIXED_DTS):
            sys.path.insert(0, os.path.join(ROOT, "tests"))
            from parity import classify, compare
            m = cells["x"].shape[1]
            idx = np.sort(np.random.default_rng(2).choice(m, 128, replace=False))
            on = oracle.OracleNetwork(net)
            o, stable, rp = classify(on, cells, dt, oracle.burn, index=idx, with_reprobe=True)
            t = oracle.burn(on, cells, dt, rtol=1e-10, atol=1e-16, index=idx)
            rep = compare(gx[:, idx], None if gT is None else gT[idx], gs[idx], *o, stable=stable,
                          tight=(t[0], t[1]), reprobe=rp)
            parity.append({"network": net.name, "sampled_cells": 128, "pass": rep["pass"], "stable": rep["stable"],
                           "max_rel_x_stable": rep["max_rel_x_stable"], "status_mismatch": rep["status_mismatch"]})
        # the oracle on a bounded sample of each segment (a third of the sample each)
        cores = os.cpu_count() or 1
        sample = 3 * 21846
        t0 = time.perf_counter()
        for (h, d, x0, T0, net, cells), dt in zip(keep, MIXED_DTS):
            sub = {k: (None if v is None else (v[..., :sample // 3] if k != "hot" else v[:sample // 3]))
                   for k, v in cells.items()}
            oracle.burn(oracle.OracleNetwork(net), sub, dt, nthreads=cores)
        el = time.perf_counter() - t0
        cpu = {"value": sample / el, "unit": "cells/s", "cores": cores, "kind": "oracle",
               "sample": f"{sample} cells, a third of each network's segment, FP64 oracle, {cores} threads, "
                         f"{el:.1f} s; cells/s extrapolates linearly"}
        return parity, cpu

    if rank == 0 and not args.no_cpu_baseline:
        try:
            parity, cpu = oracle_legs()
        except Exception as exc:  # noqa: BLE001 -- recorded, the line still prints
            parity = cpu = {"error": f"{type(exc).__name__}: {exc}"}
    achieved = flops / (ms / 1e3) / 1e12
    return {
        "metric": METRIC, "value": job_throughput(n, world, ms), "unit": "cells/s", "n_gpus": world,
        "steps": k_timed, "warmup": w_run, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "steps_requested": args.steps, "warmup_requested": args.warmup,
        "config": {"workload": "batched uneven work: Robertson (3 ODEs, t = 40) + net13 (13 ODEs) + net33 "
                               "(33 ODEs, 4 elements, 120 reactions), a third each, 1 % hot cells T log-U[1e4, 1e5] K",
                   "n_cells_per_gpu": n, "seed": MIXED_SEED + 1000 * rank, "dt_s": list(MIXED_DTS),
                   "rtol": 1e-6, "atol": 1e-10, "lu_precision": 64,
                   "variant": "one persistent launch over all networks (cost-ordered queues, hand-off and "
                              "warp-per-cell record pass), CUDA graph replay",
                   "autotuned": tuned,
                   "l2": "inputs exceed L2 and L2 is flushed between steps",
                   "parallelism": f"independent shards x{world}"},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": fp64_peak, "unit": "TFLOP/s",
                     "frac": achieved / fp64_peak,
                     "traffic": None, "peak_source": "FP64 FMA rate measured in this run (mc_probe_fma_rate)",
                     "attempts": attempts},
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_v, "unit": "cells/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": int(launches), "clocks": clocks, "status_ok_fraction": ok / n,
        "parity_sample": parity, "per_step_ms": per,
    }


def _build_if_missing():
    if not os.path.exists(os.path.join(ROOT, "paper_2608_06466_b300", "libmc.so")):
        # a fresh checkout: build the library (loading the build script by path,
        # since importing the package needs the library)
        import importlib.util
        spec = importlib.util.spec_from_file_location("_mc_build",
                                                      os.path.join(ROOT, "paper_2608_06466_b300", "build.py"))
        mod = importlib.util.module_from_spec(spec)
        spec.loader.exec_module(mod)
        mod.build()


def timed_steps(step, steps, warmup, stream, flush, barrier, rank, local, sample_clocks, budget_s=None, world=1):
    """W untimed and K timed steps, CUDA events on the launching stream, a
    barrier and a device synchronize on both sides, L2 flushed before each.
    With budget_s, at most 3 warm-up steps run and K is cut to what the last
    warm-up step's time fits in budget_s (never below 3, never above the K
    asked for; the same on every rank); the count actually timed is returned."""
    import torch
    import paper_2608_06466_b300 as mc
    if budget_s is not None:
        warmup = min(warmup, 3)
    t_last = 0.0
    for _ in range(warmup):
        t0 = time.perf_counter()
        step()
        torch.cuda.synchronize()
        t_last = time.perf_counter() - t0
    if budget_s is not None and t_last > 0.0:
        fit = int(max_over_ranks(budget_s / t_last, world, "cuda") if world == 1 else
                  -max_over_ranks(-budget_s / t_last, world, "cuda"))
        steps = min(steps, max(3, fit))
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    mc.mc_launch_count(reset=True)
    path = os.path.join(LOG_DIR, f"bench_clocks_r{rank}.csv")
    proc, fh = clock_sampler_start(path) if sample_clocks else (None, None)
    per = []
    for _ in range(steps):
        flush.zero_()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        e1.synchronize()
        per.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    barrier()
    launches = mc.mc_launch_count()
    clocks = clock_sampler_stop(proc, fh, path, local) if sample_clocks else None
    return float(np.mean(per)), per, launches, clocks, steps, warmup


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="precision", choices=["precision", "mixed"])
    ap.add_argument("--cells", type=int, default=N_CELLS)
    ap.add_argument("--max-timed-s", type=float, default=100.0,
                    help="cut the timed steps to what fits this many seconds (at least 3) and the warm-up to 3; "
                         "0 times exactly --steps after exactly --warmup")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true", help="skip the FP64 comparison arms")
    ap.add_argument("--serving-window-s", type=float, default=40.0,
                    help="seconds of each serving phase (saturation, 0.5x and 0.9x load)")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving-loop measurement")
    args = ap.parse_args()
    if args.max_timed_s <= 0:
        args.max_timed_s = None

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    import torch.distributed as dist
    _build_if_missing()
    import paper_2608_06466_b300 as mc
    from paper_2608_06466_b300.api import to_device
    from mc_inputs import network_13, synthetic_cells

    torch.cuda.set_device(local)
    if world > 1:
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    os.makedirs(LOG_DIR, exist_ok=True)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    fp64_peak, fp32_peak = mc.mc_probe_fma_rate()
    if args.config == "mixed":
        line = run_mixed(args, mc, world, rank, local, stream, flush, barrier, fp64_peak, fp32_peak)
        if rank == 0:
            print(json.dumps(line), flush=True)
        if world > 1:
            dist.destroy_process_group()
        return

    net = network_13()
    h = mc.Network(net)
    n = args.cells
    cells = synthetic_cells(net, n, seed=shard_seed(rank))
    d = to_device(cells)
    x0, T0 = d["x"].clone(), d["T"].clone()
    opts32 = mc.mc_burn_opts_default(lu_precision=32, variant=mc.MC_VARIANT_PERSISTENT)
    opts64p = mc.mc_burn_opts_default(lu_precision=64, variant=mc.MC_VARIANT_PERSISTENT)
    opts64 = mc.mc_burn_opts_default(lu_precision=64, variant=mc.MC_VARIANT_PLAIN)

    def burn(opts):
        d["x"].copy_(x0)
        d["T"].copy_(T0)
        mc.mc_burn_batch(h, opts, n, DT, d["x"], n, d["T"], d["ndens"], None, d["status"], d["stats"], stream)

    ms32, per32, launches, clocks, k_timed, w_run = timed_steps(lambda: burn(opts32), args.steps, args.warmup, stream,
                                                                flush, barrier, rank, local, True, args.max_timed_s,
                                                                world)
    ms32 = max_over_ranks(ms32, world, "cuda")
    gx, gT = d["x"].cpu().numpy(), d["T"].cpu().numpy()
    status = d["status"].cpu().numpy()
    stats = d["stats"].cpu().numpy()
    flops = fp64_flops(net.n_species, net.n_reactions, net.n_ode, stats, 32)
    attempts = float((stats[0].astype(np.int64) + stats[1] + stats[2]).sum())
    value = job_throughput(n, world, ms32)

    # FP64 comparison arms: same scheduling with the FP64 matrix on the same
    # cells, and the plain one-thread-per-cell FP64 path on the plain
    # workload's 2^20 cells; one timed step each after a small warm-up burn
    arms = None
    if not args.no_plain and world == 1:
        small = min(n, 4096)
        for o in (opts64p, opts64):
            mc.mc_burn_batch(h, o, small, DT, d["x"], n, d["T"], d["ndens"], None, d["status"], d["stats"], stream)
        ms64p = timed_steps(lambda: burn(opts64p), 1, 0, stream, flush, barrier, rank, local, False)[0]
        st64p = d["stats"].cpu().numpy()
        cells_p = synthetic_cells(net, N_PLAIN, seed=PLAIN_SEED)
        dp = to_device(cells_p)
        xp0, Tp0 = dp["x"].clone(), dp["T"].clone()

        def burn_plain():
            dp["x"].copy_(xp0)
            dp["T"].copy_(Tp0)
            mc.mc_burn_batch(h, opts64, N_PLAIN, DT, dp["x"], N_PLAIN, dp["T"], dp["ndens"], None, dp["status"],
                             dp["stats"], stream)

        ms64 = timed_steps(burn_plain, 1, 0, stream, flush, barrier, rank, local, False)[0]
        st64 = dp["stats"].cpu().numpy()
        arms = {
            "fp64_persistent": {
                "value": n / (ms64p / 1e3), "unit": "cells/s", "ms_per_step": ms64p, "cells": n,
                "fp64_tflops_algorithmic": fp64_flops(net.n_species, net.n_reactions, net.n_ode, st64p, 64)
                / (ms64p / 1e3) / 1e12,
                "note": "same cells and scheduling as the headline, FP64 iteration matrix"},
            "fp64_plain": {
                "value": N_PLAIN / (ms64 / 1e3), "unit": "cells/s", "ms_per_step": ms64, "cells": N_PLAIN,
                "fp64_tflops_algorithmic": fp64_flops(net.n_species, net.n_reactions, net.n_ode, st64, 64)
                / (ms64 / 1e3) / 1e12,
                "ok_fraction": float(np.mean(dp["status"].cpu().numpy() == 0)),
                "note": f"plain FP64 workload: 2^20 cells (seed {PLAIN_SEED}), one thread per cell, one launch"},
        }
        del dp

    # end to end through the C ABI with host buffers (pinned), copies inside
    xh = torch.from_numpy(np.ascontiguousarray(cells["x"])).pin_memory()
    Th = torch.from_numpy(np.ascontiguousarray(cells["T"])).pin_memory()
    nh = torch.from_numpy(np.ascontiguousarray(cells["ndens"])).pin_memory()
    xw, Tw = xh.clone().pin_memory(), Th.clone().pin_memory()
    sh = torch.zeros(n, dtype=torch.int32).pin_memory()
    # one timed call: the kernels, scratch and allocator pool are warm from the
    # device-resident steps above
    e2e_ms = []
    for _ in range(1):
        xw.copy_(xh)
        Tw.copy_(Th)
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        mc.mc_burn_batch(h, opts32, n, DT, xw.numpy(), n, Tw.numpy(), nh.numpy(), None, sh.numpy(), None, None)
        t1 = time.perf_counter()
        e2e_ms.append((t1 - t0) * 1e3)
    e2e_v = job_throughput(n, world, max_over_ranks(float(np.mean(e2e_ms)), world, "cuda"))
    h2d = (net.n_species + 2) * 8 * n
    d2h = (net.n_species + 1) * 8 * n + 4 * n

    # the legs after the timed region: a failure in one is recorded in its key
    # and does not cost the line
    def leg(fn):
        try:
            return fn()
        except Exception as exc:  # noqa: BLE001
            return {"error": f"{type(exc).__name__}: {exc}"}

    parity = None
    cpu = None
    serving = None
    if rank == 0 and not args.no_cpu_baseline:
        idx = np.sort(np.random.default_rng(1).choice(n, PARITY_SAMPLE, replace=False))
        parity = leg(lambda: parity_sample(net, cells, idx, gx[:, idx], gT[idx], status[idx]))
    if rank == 0 and world == 1 and not args.no_serving:
        serving = leg(lambda: serving_measurement(mc, window_s=args.serving_window_s))
    if rank == 0 and not args.no_cpu_baseline:
        cpu = leg(lambda: cpu_baseline(net, int(os.environ.get("MC_CPU_SAMPLE", str(ORACLE_SAMPLE))), CELL_SEED))

    if rank == 0:
        achieved = flops / (ms32 / 1e3) / 1e12
        traffic = None if DRAM_BYTES_PER_ATTEMPT is None else DRAM_BYTES_PER_ATTEMPT * attempts
        line = {
            "metric": METRIC, "value": value, "unit": "cells/s", "n_gpus": world, "steps": k_timed,
            "warmup": w_run, "ms_per_step": ms32, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "steps_requested": args.steps, "warmup_requested": args.warmup,
            "config": {"workload": "precision form: net13 synthetic kinetics, 12 species from 3 elements + energy "
                                   "equation (13 ODEs), 40 reversible reactions, ideal gas gamma=5/3",
                       "n_cells_per_gpu": n, "cell_seed": shard_seed(rank), "dt_s": DT, "rtol": 1e-6, "atol": 1e-10,
                       "T_K": "log-uniform [10, 1e4]", "n_cm3": "log-uniform [1, 1e8]",
                       "lu_precision": 32, "variant": "persistent (cost-ordered queue, one cooperative launch "
                                                      "with hand-off, FP64 retry pass)",
                       "max_steps": 100000,
                       "l2": "inputs exceed L2 (470 MB) and L2 is flushed between steps (256 MB write)",
                       "parallelism": f"independent shards x{world}"},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": fp64_peak, "unit": "TFLOP/s",
                         "frac": achieved / fp64_peak, "traffic": traffic,
                         "peak_source": "FP64 FMA rate measured in this run (mc_probe_fma_rate)",
                         "model": "FP64 flops per unit from ncu counters on the evaluation kernels x the run's "
                                  "per-cell counters",
                         "attempts": attempts, "fp32_fma_peak_tflops": fp32_peak},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_v, "unit": "cells/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": int(launches),
            "clocks": clocks,
            "fp64_arms": arms,
            "status_ok_fraction": float(np.mean(status == 0)),
            "parity_sample": parity,
            "serving": serving,
            "per_step_ms": per32,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
