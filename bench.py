"""Benchmark of the per-cell burn on B300.

Workload (one "step" = one burn of the whole batch): the 13-ODE synthetic
network (12 species from 3 elements + the energy equation, 40 reversible
reactions), 2^20 cells per GPU, T log-uniform [10, 1e4] K, n log-uniform
[1, 1e8] cm^-3, dt = 1e10 s, rtol = 1e-6, atol = 1e-10. The headline arm is the
FP32-iteration-matrix persistent path; the plain FP64 path on the same inputs
is reported beside it. Inputs are reset from a device-resident copy before
every step (inside the timed region) and L2 is flushed between steps.

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
N_CELLS = 1 << 20
DT = 1.0e10
CELL_SEED = 3

# FP64-pipe cost model of the algorithm (operations per unit, each a fused or
# plain FP64 arithmetic instruction; an FMA is 2 flops, anything else 1):
# exp/log/div/sqrt/pow are charged the FP64 instruction counts of the CUDA
# math routines the kernels call, measured once by throughput against the FMA
# rate (exp 20, log 36, div 8). The table-driven exp costs about 11, so the
# model slightly overstates the work; it is kept fixed so numbers compare.
EXP_OPS, LOG_OPS, DIV_OPS = 20, 36, 8

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


def fp64_ops_per_cell(S, R, n, stats):
    """FP64 operations of the work the per-cell counters record."""
    rhs, jac, lu, newton, steps = (stats[3].astype(np.float64), stats[4].astype(np.float64),
                                   stats[5].astype(np.float64), stats[6].astype(np.float64),
                                   stats[0].astype(np.float64))
    attempts = steps + stats[1] + stats[2]
    f_rhs = S + 3 + DIV_OPS + LOG_OPS + DIV_OPS + R * (2 * EXP_OPS + 4 + 5 + 2 + 4 + 1)
    f_jac = f_rhs + R * (16 + 6 + 10) + n * (S + 1)
    f_lu = n * n + (2.0 / 3.0) * n ** 3 + n * DIV_OPS
    f_solve = 2.0 * n * n + n * DIV_OPS + 3 * n + 2 * n + 1
    f_step = 15 * n + 2 * n + n * DIV_OPS + 4 * n + 60
    return rhs * f_rhs + jac * f_jac + lu * f_lu + newton * f_solve + attempts * f_step


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


def serving_measurement(mc, n_sat=6, n_load=8, seed=7, edge_range=(16, 64)):
    """Serving loop on AMR-box requests (edge L log-uniform in edge_range, cells
    = L^3, 50/50 net13 / net33, FP32-matrix path, 150 GB budget): closed-loop
    saturation, then Poisson arrivals at 0.5x and 0.9x of it. Bounded request
    counts and box sizes keep the run within minutes."""
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

    def run(stream_reqs, arrivals):
        srv = mc.Server(0, 150 << 30, opts)
        bufs = [make(r) for r in stream_reqs]
        ids = []
        t0 = _t.perf_counter()
        for (name, n, x, T, nd, st), ta in zip(bufs, arrivals):
            wait = ta - (_t.perf_counter() - t0)
            if wait > 0:
                _t.sleep(wait)
            ids.append(srv.submit(handles[name], n, DT, x, n, T, nd, st))
        srv.drain(3600)
        span = _t.perf_counter() - t0
        infos = [srv.poll(i)[1] for i in ids]
        srv.close()
        lat = np.array([i.t_done - i.t_submit for i in infos])
        cells = sum(b[1] for b in bufs)
        return lat, cells, span, sum(i.n_failed for i in infos)

    sat_reqs = box_request_stream(n_sat, 1.0, seed=seed, edge_range=edge_range)
    lat, cells, span, _ = run(sat_reqs, [0.0] * n_sat)
    lam_cells = cells / span
    sizes = np.array([r["n_cells"] for r in box_request_stream(4096, 1.0, seed=seed + 1, edge_range=edge_range)])
    mean_cells = float(sizes.mean())
    out = {"lambda_sat_cells_per_s": lam_cells, "mean_cells_per_request": mean_cells,
           "edge_range": list(edge_range),
           "saturation_requests": n_sat, "loads": [],
           "note": f"{n_load} Poisson requests per load level (bounded so the run ends in minutes)"}
    for load in (0.5, 0.9):
        rate = load * lam_cells / mean_cells
        reqs = box_request_stream(n_load, rate, seed=seed + int(load * 100), edge_range=edge_range)
        arrivals = [r["t_arrive"] for r in reqs]
        lat, cells, span, failed = run(reqs, arrivals)
        out["loads"].append({"load": load, "requests": n_load, "rate_req_per_s": rate,
                             "p50_latency_s": float(np.percentile(lat, 50)),
                             "p99_latency_s": float(np.percentile(lat, 99)),
                             "cells_per_s": cells / span, "failed_cells": int(failed)})
    return out


def run_reference(args, rank, world):
    from mc_inputs import network_13
    net = network_13()
    if rank != 0:
        return
    n_sample = int(os.environ.get("MC_REF_SAMPLE", "4096"))
    times = []
    for i in range(args.warmup + args.steps):
        b = cpu_baseline(net, n_sample, seed=CELL_SEED + i)
        if i >= args.warmup:
            times.append(n_sample / b["value"])
    ms = 1e3 * float(np.mean(times))
    value = n_sample / (ms / 1e3)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "cells/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "net13 synthetic kinetics, 12 species + energy, 40 reactions; "
                                   f"bounded sample of {n_sample} cells per step (seeds {CELL_SEED}..)",
                       "n_cells_per_step": n_sample, "dt_s": DT, "rtol": 1e-6, "atol": 1e-10},
            "cpu_baseline": {"value": value, "unit": "cells/s", "cores": os.cpu_count(), "kind": "oracle",
                             "sample": f"{n_sample} cells per step"},
            "e2e": {"value": value, "unit": "cells/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cells", type=int, default=N_CELLS)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--serving", action="store_true",
                    help="add the serving-loop measurement (AMR-box requests, a few minutes)")
    ap.add_argument("--no-serving", action="store_true", help="no serving measurement (the default)")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    import torch.distributed as dist
    if not os.path.exists(os.path.join(ROOT, "paper_2608_06466_b300", "libmc.so")):
        # a fresh checkout: build the library (loading the build script by path,
        # since importing the package needs the library)
        import importlib.util
        spec = importlib.util.spec_from_file_location("_mc_build",
                                                      os.path.join(ROOT, "paper_2608_06466_b300", "build.py"))
        mod = importlib.util.module_from_spec(spec)
        spec.loader.exec_module(mod)
        mod.build()
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

    net = network_13()
    h = mc.Network(net)
    n = args.cells
    cells = synthetic_cells(net, n, seed=shard_seed(rank))
    d = to_device(cells)
    x0, T0 = d["x"].clone(), d["T"].clone()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    opts32 = mc.mc_burn_opts_default(lu_precision=32, variant=mc.MC_VARIANT_PERSISTENT)
    opts64 = mc.mc_burn_opts_default(lu_precision=64, variant=mc.MC_VARIANT_PLAIN)

    def one_step(opts):
        d["x"].copy_(x0)
        d["T"].copy_(T0)
        mc.mc_burn_batch(h, opts, n, DT, d["x"], n, d["T"], d["ndens"], None, d["status"], d["stats"], stream)

    def timed(opts, steps, warmup, sample_clocks=False):
        for _ in range(warmup):
            one_step(opts)
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        mc.mc_launch_count(reset=True)
        proc, fh = clock_sampler_start(os.path.join(LOG_DIR, f"bench_clocks_r{rank}.csv")) \
            if sample_clocks else (None, None)
        total = 0.0
        per = []
        for _ in range(steps):
            flush.zero_()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            one_step(opts)
            e1.record(stream)
            e1.synchronize()
            ms = e0.elapsed_time(e1)
            per.append(ms)
            total += ms
        torch.cuda.synchronize()
        barrier()
        launches = mc.mc_launch_count()
        clocks = clock_sampler_stop(proc, fh, os.path.join(LOG_DIR, f"bench_clocks_r{rank}.csv"),
                                    local) if sample_clocks else None
        ms = max_over_ranks(total / steps, world, "cuda")
        return ms, per, launches, clocks

    os.makedirs(LOG_DIR, exist_ok=True)
    fp64_peak, fp32_peak = mc.mc_probe_fma_rate()

    ms32, per32, launches, clocks = timed(opts32, args.steps, args.warmup, sample_clocks=True)
    status = d["status"].cpu().numpy()
    stats = d["stats"].cpu().numpy()
    ops = float(fp64_ops_per_cell(net.n_species, net.n_reactions, net.n_ode, stats).sum())
    value = job_throughput(n, world, ms32)

    plain = None
    if not args.no_plain:
        ms64, _, _, _ = timed(opts64, 1, 1)
        st64 = d["stats"].cpu().numpy()
        ops64 = float(fp64_ops_per_cell(net.n_species, net.n_reactions, net.n_ode, st64).sum())
        plain = {"value": job_throughput(n, world, ms64), "unit": "cells/s", "ms_per_step": ms64,
                 "fp64_tflops_algorithmic": 2 * ops64 / (ms64 / 1e3) / 1e12,
                 "ok_fraction": float(np.mean(d["status"].cpu().numpy() == 0))}

    # end to end through the C ABI with host buffers (pinned), copies inside
    xh = torch.from_numpy(np.ascontiguousarray(cells["x"])).pin_memory()
    Th = torch.from_numpy(np.ascontiguousarray(cells["T"])).pin_memory()
    nh = torch.from_numpy(np.ascontiguousarray(cells["ndens"])).pin_memory()
    xw, Tw = xh.clone().pin_memory(), Th.clone().pin_memory()
    sh = torch.zeros(n, dtype=torch.int32).pin_memory()
    e2e_ms = []
    for i in range(1 + max(1, min(args.steps, 2))):
        xw.copy_(xh)
        Tw.copy_(Th)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        mc.mc_burn_batch(h, opts32, n, DT, xw.numpy(), n, Tw.numpy(), nh.numpy(), None, sh.numpy(), None, None)
        t1 = time.perf_counter()
        if i > 0:
            e2e_ms.append((t1 - t0) * 1e3)
    e2e_v = job_throughput(n, world, max_over_ranks(float(np.mean(e2e_ms)), world, "cuda"))
    h2d = (net.n_species + 2) * 8 * n
    d2h = (net.n_species + 1) * 8 * n + 4 * n

    # sampled parity of the timed results against the oracle
    parity = None
    if rank == 0 and not args.no_cpu_baseline:
        sys.path.insert(0, os.path.join(ROOT, "tests"))
        import oracle
        from parity import classify, compare
        idx = np.sort(np.random.default_rng(1).choice(n, 128, replace=False))
        one_step(opts32)
        torch.cuda.synchronize()
        on = oracle.OracleNetwork(net)
        (o, stable) = classify(on, cells, DT, oracle.burn, index=idx, perturb=1e-9)
        t = oracle.burn(on, cells, DT, rtol=1e-10, atol=1e-16, index=idx)
        gx = d["x"].cpu().numpy()[:, idx]
        gT = d["T"].cpu().numpy()[idx]
        gs = d["status"].cpu().numpy()[idx]
        rep = compare(gx, gT, gs, o[0], o[1], o[2], o[3], stable=stable, tight=(t[0], t[1]), fp32_matrix=True)
        parity = {"sampled_cells": 128, "pass": rep["pass"], "stable": rep["stable"],
                  "max_rel_x_stable": rep["max_rel_x_stable"], "status_mismatch": rep["status_mismatch"],
                  "stable_within_1e-5_frac": rep["stable_within_1e-5_frac"]}

    serving = None
    if rank == 0 and args.serving and not args.no_serving:
        serving = serving_measurement(mc)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline(net, int(os.environ.get("MC_CPU_SAMPLE", "262144")), CELL_SEED)

    if rank == 0:
        achieved = 2 * ops / (ms32 / 1e3) / 1e12
        line = {
            "metric": METRIC, "value": value, "unit": "cells/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms32, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "net13 synthetic kinetics: 12 species from 3 elements + energy equation "
                                   "(13 ODEs), 40 reversible reactions, ideal gas gamma=5/3",
                       "n_cells_per_gpu": n, "dt_s": DT, "rtol": 1e-6, "atol": 1e-10,
                       "T_K": "log-uniform [10, 1e4]", "n_cm3": "log-uniform [1, 1e8]",
                       "lu_precision": 32, "variant": "persistent (cost-ordered queue, one cooperative launch with hand-off)", "max_steps": 100000,
                       "l2": "flushed between steps (256 MB write)", "parallelism": f"independent shards x{world}"},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": fp64_peak, "unit": "TFLOP/s",
                         "frac": achieved / fp64_peak, "traffic": None,
                         "peak_source": "FP64 FMA rate measured in this run (mc_probe_fma_rate)",
                         "fp32_fma_peak_tflops": fp32_peak},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_v, "unit": "cells/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": int(launches),
            "clocks": clocks,
            "fp64_plain": plain,
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
