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
    if (!(g.dt >= 0.0) || !std::isfinite(g.dt))
      return set_error(MC_E_INVALID, "segment %d: dt must be finite and not negative", s);
    if (g.net->device != dev) return set_error(MC_E_INVALID, "segment %d: network on another device", s);
  }
  return MC_OK;
}

// Hand-off threshold and record capacity of a thread-per-cell segment of n
// cells (the single-network path's defaults).
constexpr int MIXED_STRAG_STEPS = 2048;

int64_t mixed_rec_cap(int64_t n) { return std::max<int64_t>(256, n / 8); }

template <int N, typename LT>
size_t rec_bytes(int64_t cap) {
  return (sizeof(Lane<N, LT>) * (size_t)cap + 255) & ~(size_t)255;
}

// Straggler record bytes of every thread-per-cell segment, laid out one after
// the other (FP32 pass only takes hand-offs in the FP32 matrix form).
size_t mixed_rec_total(const mc_segment *segs, int32_t nseg, int lu) {
  size_t t = 0;
  for (int s = 0; s < nseg; ++s) {
    const int b = bucket_of(segs[s].net->n);
    const int64_t cap = mixed_rec_cap(segs[s].n_cells);
    if (b == 3) t += lu == 32 ? rec_bytes<3, float>(cap) : rec_bytes<3, double>(cap);
    if (b == 13) t += lu == 32 ? rec_bytes<13, float>(cap) : rec_bytes<13, double>(cap);
  }
  return t;
}

// Grow every scratch buffer a mixed burn on stream st uses (queue counters,
// retry lists, cost order, straggler records), so that the launch itself
// neither allocates nor synchronises (it may then be captured).
mc_status mixed_reserve(const mc_segment *segs, int32_t nseg, const mc_burn_opts &ob, cudaStream_t st) {
  int dev = 0;
  cudaGetDevice(&dev);
  int64_t total = 0;
  for (int s = 0; s < nseg; ++s) total += segs[s].n_cells;
  unsigned long long *next;
  uint32_t *rcount;
  int32_t *retry;
  scratch_stream(st);
  mc_status rs = scratch_get(dev, ob.lu_precision == 32 ? total : 0, &next, &rcount, &retry);
  if (rs != MC_OK) return rs;
  int32_t *order;
  uint8_t *bkt;
  uint32_t *hist;
  rs = order_scratch(dev, std::max<int64_t>(1, total), &order, &bkt, &hist);
  if (rs != MC_OK) return rs;
  const size_t rb = mixed_rec_total(segs, nseg, ob.lu_precision);
  if (rb > 0) {
    void *rec;
    uint32_t *cnt;
    rs = straggler_scratch(rb, &rec, &cnt);
    if (rs != MC_OK) return rs;
  }
  return MC_OK;
}

template <int N, typename LT>
mc_status launch_records(const DNet &d, const Opts &o, const CellArgs &a, const StragArgs &sa,
                         unsigned long long *next, int sms, cudaStream_t st) {
  const int per_warp = (int)wsh_bytes<N, LT>(d.R);
  static thread_local DevAttrCache configured;
  int dev = 0;
  cudaGetDevice(&dev);
  if (configured.below(dev, per_warp)) {
    cudaError_t e = cudaFuncSetAttribute(k_burn_straggler<N, LT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         per_warp);
    if (e != cudaSuccess) return cuda_error(e, "mixed straggler smem attribute");
    configured.raise(dev, per_warp);
  }
  const int wblocks = std::max(1, std::min(sms * 16, (int)sa.cap));
  k_burn_straggler<N, LT><<<wblocks, 32, per_warp, st>>>(d, o, a, (const Lane<N, LT> *)sa.rec, sa.count, sa.cap,
                                                          nullptr, next, per_warp);
  count_launch(1);
  return MC_OK;
}

// One pass of the mixed kernel in matrix precision LT: cost-ordered queues,
// the persistent launch with hand-off, then the warp-per-cell pass over each
// thread-per-cell segment's records.
template <typename LT>
mc_status mixed_pass(const mc_segment *segs, MixedArgs m, const Opts &o, int blocks, int mthreads, int msmem,
                     bool handoff, unsigned long long *next, uint32_t *rcnt, char *rec, int sms, cudaStream_t st) {
  const int nseg = m.nseg;
  cudaError_t e = cudaMemsetAsync(next, 0, sizeof(unsigned long long) * 2 * MIXED_MAX_SEGS, st);
  if (e == cudaSuccess && handoff) e = cudaMemsetAsync(rcnt, 0, sizeof(uint32_t) * 4 * MIXED_MAX_SEGS, st);
  if (e != cudaSuccess) return cuda_error(e, "mixed queue reset");
  size_t off = 0;
  for (int s = 0; s < nseg; ++s) {
    m.sa[s] = StragArgs{nullptr, nullptr, 0u, 0, nullptr};
    const int b = m.seg[s].bucket;
    if (!handoff || (b != 3 && b != 13) || segs[s].n_cells == 0) continue;
    const int64_t cap = mixed_rec_cap(segs[s].n_cells);
    m.sa[s] = StragArgs{rec + off, rcnt + 4 * s, (uint32_t)cap, MIXED_STRAG_STEPS, nullptr};
    off += (b == 3) ? rec_bytes<3, LT>(cap) : rec_bytes<13, LT>(cap);
  }
  k_burn_mixed<LT><<<(unsigned)blocks, mthreads, msmem, st>>>(m, o, next);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_error(e, "mixed launch");
  count_launch(1);
  for (int s = 0; s < nseg; ++s) {
    if (!m.sa[s].rec) continue;
    const SegDev &g = m.seg[s];
    mc_status r = (g.bucket == 3)
                      ? launch_records<3, LT>(g.net, o, g.a, m.sa[s], next + MIXED_MAX_SEGS + s, sms, st)
                      : launch_records<13, LT>(g.net, o, g.a, m.sa[s], next + MIXED_MAX_SEGS + s, sms, st);
    if (r != MC_OK) return r;
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_error(e, "mixed record pass");
  return MC_OK;
}

// Queue resets and kernels of one mixed burn on stream st (capturable once
// mixed_reserve has sized the scratch).
mc_status mixed_launch(const mc_segment *segs, int32_t nseg, const mc_burn_opts &ob, double dt,
                       cudaStream_t st) {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  mc_status rs = mixed_reserve(segs, nseg, ob, st);
  if (rs != MC_OK) return rs;
  int64_t total = 0;
  for (int s = 0; s < nseg; ++s) total += segs[s].n_cells;
  unsigned long long *next;
  uint32_t *rcount;
  int32_t *retry;
  scratch_stream(st);
  rs = scratch_get(dev, ob.lu_precision == 32 ? total : 0, &next, &rcount, &retry);
  if (rs != MC_OK) return rs;
  int32_t *order;
  uint8_t *bkt;
  uint32_t *hist;
  rs = order_scratch(dev, std::max<int64_t>(1, total), &order, &bkt, &hist);
  if (rs != MC_OK) return rs;
  void *rec = nullptr;
  uint32_t *rcnt = nullptr;
  const size_t rb = mixed_rec_total(segs, nseg, ob.lu_precision);
  if (rb > 0) {
    rs = straggler_scratch(rb, &rec, &rcnt);
    if (rs != MC_OK) return rs;
  }
  // launch shape and staging: the autotuner's pick for the thread-per-cell
  // network with the most cells (the warp-per-cell segments share the grid)
  const mc_network *lead = nullptr;
  int64_t most = -1;
  for (int s = 0; s < nseg; ++s)
    if (segs[s].net->n <= 16 && segs[s].n_cells > most) {
      most = segs[s].n_cells;
      lead = segs[s].net;
    }
  const Tuned tu = autotune_pick(lead, ob);
  const Opts o{ob.rtol, ob.atol, ob.max_order, ob.max_steps, ob.jacobian == MC_JAC_FD ? 1 : 0,
               tu.staging == MC_STAGING_LANE ? 1 : 0};
  MixedArgs m{};
  m.nseg = nseg;
  int64_t off = 0;
  for (int s = 0; s < nseg; ++s) {
    const mc_segment &g = segs[s];
    SegDev &d = m.seg[s];
    d.net = dnet_of(g.net);
    d.bucket = bucket_of(g.net->n);
    CellArgs &a = d.a;
    a = CellArgs{};
    a.n_cells = g.n_cells;
    a.ld = g.ld;
    a.dt = g.dt > 0.0 ? g.dt : dt;
    a.x = g.x;
    a.T = g.T;
    a.nd = g.ndens;
    a.ks = g.rate_scale;
    a.status = g.status;
    a.stats = g.stats;
    bc_attach(a);
    // each segment's queue hands out its cells in decreasing cost order
    if (g.n_cells > 0) {
      rs = order_cells(g.net, o, a, order + off, bkt + off, hist, st);
      if (rs != MC_OK) return rs;
      a.index = order + off;
    }
    if (ob.lu_precision == 32) {
      a.retry = retry + off;
      a.retry_count = rcount + s;
      a.retry_mask = FP32_RETRY_MASK;
    }
    off += g.n_cells;
  }
  // warp workspace (the largest one): the warp-per-cell segments' state, the
  // thread-per-cell segments' cooperative matrix work
  size_t per_warp = 16;
  for (int s = 0; s < nseg; ++s) {
    const int b = m.seg[s].bucket, R = segs[s].net->R;
    const bool f = ob.lu_precision == 32;
    if (b == 3) per_warp = std::max(per_warp, f ? wsh_bytes<3, float>(R) : wsh_bytes<3, double>(R));
    if (b == 13) per_warp = std::max(per_warp, f ? wsh_bytes<13, float>(R) : wsh_bytes<13, double>(R));
    if (b == 33) per_warp = std::max(per_warp, f ? wsh_bytes<33, float>(R) : wsh_bytes<33, double>(R));
    if (b == 40) per_warp = std::max(per_warp, f ? wsh_bytes<40, float>(R) : wsh_bytes<40, double>(R));
  }
  // the FP64 retry pass runs on the same workspace size (its matrices are
  // larger than the FP32 pass's)
  for (int s = 0; s < nseg; ++s) {
    const int b = m.seg[s].bucket, R = segs[s].net->R;
    if (b == 3) per_warp = std::max(per_warp, wsh_bytes<3, double>(R));
    if (b == 13) per_warp = std::max(per_warp, wsh_bytes<13, double>(R));
    if (b == 33) per_warp = std::max(per_warp, wsh_bytes<33, double>(R));
    if (b == 40) per_warp = std::max(per_warp, wsh_bytes<40, double>(R));
  }
  m.smem_per_warp = (int)per_warp;
  int smem_max = 0;
  if (cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return set_error(MC_E_CUDA, "mixed: shared memory limit");
  // four warps a block unless their workspaces exceed a block's shared memory
  const int mthreads = std::max(32, std::min(128, 32 * (smem_max / (int)per_warp)));
  const int msmem = (int)per_warp * (mthreads / 32);
  {
    static thread_local DevAttrCache configured;
    if (configured.below(dev, msmem)) {
      cudaError_t ea = cudaFuncSetAttribute(k_burn_mixed<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, msmem);
      if (ea == cudaSuccess)
        ea = cudaFuncSetAttribute(k_burn_mixed<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, msmem);
      if (ea != cudaSuccess) return cuda_error(ea, "mixed smem attribute");
      configured.raise(dev, msmem);
    }
  }
  if (ob.lu_precision == 32) {
    cudaError_t e = cudaMemsetAsync(rcount, 0, sizeof(uint32_t) * nseg, st);
    if (e != cudaSuccess) return cuda_error(e, "mixed retry reset");
  }
  const int blocks = std::max(1, sms * tu.blocks_per_sm * (128 / mthreads));
  const bool handoff = tu.strag_steps >= 0;
  if (ob.lu_precision == 64)
    return mixed_pass<double>(segs, m, o, blocks, mthreads, msmem, handoff, next, rcnt, (char *)rec, sms, st);
  rs = mixed_pass<float>(segs, m, o, blocks, mthreads, msmem, handoff, next, rcnt, (char *)rec, sms, st);
  if (rs != MC_OK) return rs;
  // FP64 pass over every segment's retry list (lengths read on the device), no hand-off
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
  return mixed_pass<double>(segs, r, o, blocks, mthreads, msmem, false, next, rcnt, (char *)rec, sms, st);
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
  if (s == MC_OK) s = mixed_reserve(segs, n_segs, o, cs);
  if (s == MC_OK) {
    // the stream-ordered scratch must exist before replays on other streams use it
    e = cudaStreamSynchronize(cs);
    if (e != cudaSuccess) s = cuda_error(e, "capture stream set-up");
  }
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
