// mc_mixed.cu -- mixed-network persistent launch (one launch over several
// networks' cells), its CUDA-graph capture, per-launch counter totals, and the
// measured launch-shape autotuner.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "mc_internal.h"
#include "mc_warp.cuh"

using namespace mc;

namespace {

__global__ void k_stats_total(const int32_t *stats, int64_t ld, int64_t n, long long *totals) {
  for (int k = 0; k < NSTAT; ++k) {
    long long s = 0;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x)
      s += stats[k * ld + c];
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if ((threadIdx.x & 31) == 0 && s) atomicAdd((unsigned long long *)&totals[k], (unsigned long long)s);
  }
}

int bucket_of(int n) { return (n == 3 || n == 13 || n == 33) ? n : 40; }

mc_status validate_segments(const mc_segment *segs, int32_t nseg, int dev) {
  if (!segs || nseg < 1 || nseg > MIXED_MAX_SEGS || nseg > MAX_QUEUES)
    return set_error(MC_E_INVALID, "mixed batch: 1..%d segments", MIXED_MAX_SEGS);
  for (int s = 0; s < nseg; ++s) {
    const mc_segment &g = segs[s];
    if (!g.net || g.n_cells < 0 || g.ld < g.n_cells || g.n_cells > (int64_t)INT32_MAX)
      return set_error(MC_E_INVALID, "segment %d: bad network or sizes", s);
    if (g.n_cells > 0 && (!g.x || !g.status || (g.net->energy && !g.T)))
      return set_error(MC_E_INVALID, "segment %d: x, status (and T for energy networks) are required", s);
    if (g.net->device != dev) return set_error(MC_E_INVALID, "segment %d: network on another device", s);
  }
  return MC_OK;
}

// Queue resets and kernels of one mixed burn on stream st (capturable).
mc_status mixed_launch(const mc_segment *segs, int32_t nseg, const mc_burn_opts &ob, double dt,
                       cudaStream_t st) {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int64_t total = 0;
  for (int s = 0; s < nseg; ++s) total += segs[s].n_cells;
  unsigned long long *next;
  uint32_t *rcount;
  int32_t *retry;
  scratch_stream(st);
  mc_status rs = scratch_get(dev, ob.lu_precision == 32 ? total : 0, &next, &rcount, &retry);
  if (rs != MC_OK) return rs;
  MixedArgs m{};
  m.nseg = nseg;
  int64_t off = 0;
  int nmax = 0;
  for (int s = 0; s < nseg; ++s) {
    const mc_segment &g = segs[s];
    SegDev &d = m.seg[s];
    d.net = dnet_of(g.net);
    d.bucket = bucket_of(g.net->n);
    nmax = std::max(nmax, g.net->n);
    CellArgs &a = d.a;
    a = CellArgs{};
    a.n_cells = g.n_cells;
    a.ld = g.ld;
    a.dt = dt;
    a.x = g.x;
    a.T = g.T;
    a.nd = g.ndens;
    a.ks = g.rate_scale;
    a.status = g.status;
    a.stats = g.stats;
    if (ob.lu_precision == 32) {
      a.retry = retry + off;
      a.retry_count = rcount + s;
      off += g.n_cells;
    }
  }
  Tuned tu = autotune_pick(nullptr, ob);
  const Opts o{ob.rtol, ob.atol, ob.max_order, ob.max_steps};
  // shared workspace of the warp-per-cell segments (the largest one)
  size_t per_warp = 16;
  for (int s = 0; s < nseg; ++s) {
    const int b = m.seg[s].bucket, R = segs[s].net->R;
    if (b == 33) per_warp = std::max(per_warp, ob.lu_precision == 64 ? wsh_bytes<33, double>(R) : wsh_bytes<33, float>(R));
    if (b == 40) per_warp = std::max(per_warp, ob.lu_precision == 64 ? wsh_bytes<40, double>(R) : wsh_bytes<40, float>(R));
  }
  m.smem_per_warp = (int)per_warp;
  const int mthreads = 128;
  const int msmem = (int)per_warp * (mthreads / 32);
  {
    // both precisions run in one call (FP32 pass, FP64 retry pass)
    static thread_local DevAttrCache configured;
    if (configured.below(dev, msmem)) {
      cudaError_t ea = cudaFuncSetAttribute(k_burn_mixed<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, msmem);
      if (ea == cudaSuccess)
        ea = cudaFuncSetAttribute(k_burn_mixed<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, msmem);
      if (ea != cudaSuccess) return cuda_error(ea, "mixed smem attribute");
      configured.raise(dev, msmem);
    }
  }
  cudaError_t e = cudaMemsetAsync(next, 0, sizeof(unsigned long long) * nseg, st);
  if (e == cudaSuccess && ob.lu_precision == 32) e = cudaMemsetAsync(rcount, 0, sizeof(uint32_t) * nseg, st);
  if (e != cudaSuccess) return cuda_error(e, "mixed queue reset");
  const unsigned blocks = (unsigned)std::max(1, sms * tu.blocks_per_sm);
  if (ob.lu_precision == 64) {
    k_burn_mixed<double><<<blocks, mthreads, msmem, st>>>(m, o, next);
  } else {
    k_burn_mixed<float><<<blocks, mthreads, msmem, st>>>(m, o, next);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, "mixed launch");
    count_launch(1);
    // FP64 pass over every segment's retry list (lengths read on the device)
    MixedArgs r = m;
    off = 0;
    for (int s = 0; s < nseg; ++s) {
      CellArgs &a = r.seg[s].a;
      a.index = retry + off;
      a.n_dev = rcount + s;
      a.retry = nullptr;
      a.retry_count = nullptr;
      off += segs[s].n_cells;
    }
    e = cudaMemsetAsync(next, 0, sizeof(unsigned long long) * nseg, st);
    if (e != cudaSuccess) return cuda_error(e, "mixed queue reset");
    k_burn_mixed<double><<<blocks, mthreads, msmem, st>>>(r, o, next);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_error(e, "mixed launch");
  count_launch(1);
  (void)nmax;
  return MC_OK;
}

}  // namespace

extern "C" mc_status mc_burn_mixed(const mc_segment *segs, int32_t n_segs, const mc_burn_opts *opts,
                                   double dt, void *stream) {
  mc_burn_opts o;
  mc_status s = check_opts(opts, &o);
  if (s != MC_OK) return s;
  if (!(dt > 0.0) || !std::isfinite(dt)) return set_error(MC_E_INVALID, "mc_burn_mixed: dt must be positive");
  int dev = 0;
  cudaGetDevice(&dev);
  s = validate_segments(segs, n_segs, dev);
  if (s != MC_OK) return s;
  return mixed_launch(segs, n_segs, o, dt, (cudaStream_t)stream);
}

// ---------------------------------------------------------------- graph
struct mc_graph {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int64_t kernels = 0;
  int device = 0;
  void *scratch = nullptr;   // scratch set the captured kernels use
};

extern "C" mc_status mc_graph_create(const mc_segment *segs, int32_t n_segs, const mc_burn_opts *opts,
                                     double dt, int64_t *totals, void *stream, mc_graph **out) {
  (void)stream;
  if (!out) return set_error(MC_E_INVALID, "mc_graph_create: null out");
  *out = nullptr;
  mc_burn_opts o;
  mc_status s = check_opts(opts, &o);
  if (s != MC_OK) return s;
  if (!(dt > 0.0) || !std::isfinite(dt)) return set_error(MC_E_INVALID, "mc_graph_create: dt must be positive");
  int dev = 0;
  cudaGetDevice(&dev);
  s = validate_segments(segs, n_segs, dev);
  if (s != MC_OK) return s;
  // allocate scratch before capture (capture must not allocate or synchronise)
  int64_t total = 0;
  for (int k = 0; k < n_segs; ++k) total += segs[k].n_cells;
  unsigned long long *next;
  uint32_t *rcount;
  int32_t *retry;
  cudaStream_t cs;
  cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (e != cudaSuccess) return cuda_error(e, "capture stream");
  // the graph keeps the scratch set of its capture stream (allocated here, before capture)
  scratch_stream(cs);
  s = scratch_get(dev, o.lu_precision == 32 ? total : 0, &next, &rcount, &retry);
  if (s != MC_OK) {
    cudaStreamDestroy(cs);
    return s;
  }
  mc_graph *g = new mc_graph();
  g->device = dev;
  const int64_t before = mc_launch_count(0);
  e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed);
  if (e != cudaSuccess) {
    cudaStreamDestroy(cs);
    delete g;
    return cuda_error(e, "begin capture");
  }
  s = MC_OK;
  if (totals) {
    e = cudaMemsetAsync(totals, 0, sizeof(int64_t) * MC_NSTAT, cs);
    if (e != cudaSuccess) s = cuda_error(e, "totals reset");
  }
  if (s == MC_OK) s = mixed_launch(segs, n_segs, o, dt, cs);
  if (s == MC_OK && totals) {
    for (int k = 0; k < n_segs; ++k) {
      if (!segs[k].stats || segs[k].n_cells == 0) continue;
      k_stats_total<<<296, 256, 0, cs>>>(segs[k].stats, segs[k].ld, segs[k].n_cells, (long long *)totals);
      count_launch(1);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) s = cuda_error(e, "totals kernel");
  }
  e = cudaStreamEndCapture(cs, &g->graph);
  if (s == MC_OK && e != cudaSuccess) s = cuda_error(e, "end capture");
  if (s == MC_OK) {
    e = cudaGraphInstantiate(&g->exec, g->graph, 0);
    if (e != cudaSuccess) s = cuda_error(e, "graph instantiate");
  }
  g->scratch = scratch_detach(dev, cs);
  cudaStreamDestroy(cs);
  g->kernels = mc_launch_count(0) - before;
  mc_launch_count(1);
  count_launch(before);  // captured launches did not run
  if (s != MC_OK) {
    if (g->graph) cudaGraphDestroy(g->graph);
    scratch_free(g->scratch);
    delete g;
    return s;
  }
  *out = g;
  return MC_OK;
}

extern "C" mc_status mc_graph_launch(mc_graph *g, void *stream) {
  if (!g || !g->exec) return set_error(MC_E_INVALID, "mc_graph_launch: null graph");
  cudaError_t e = cudaGraphLaunch(g->exec, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_error(e, "graph launch");
  count_launch(g->kernels);
  return MC_OK;
}

extern "C" mc_status mc_graph_destroy(mc_graph *g) {
  if (!g) return MC_OK;
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  cudaDeviceSynchronize();  // replays may still be using the scratch set
  scratch_free(g->scratch);
  delete g;
  return MC_OK;
}
