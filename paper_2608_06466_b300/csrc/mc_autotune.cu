// mc_autotune.cu -- measured launch-shape selection. mc_autotune times
// candidates on a sample of the caller's cells in three passes -- variant x
// threads per block x persistent blocks per SM; then, for a thread-per-cell
// persistent winner, the staging of the matrix work (the warp's shared memory
// or the lane's own state); then the straggler hand-off threshold -- and
// keeps the fastest per (device, ODE count, reactions, energy form, matrix
// precision); mc_burn_* with zero shape fields use the stored winner. Winners
// persist in a JSON-lines file when MC_AUTOTUNE_CACHE names one.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "mc_internal.h"
#include "mc_kernels.cuh"

using namespace mc;

namespace {
// default straggler hand-off threshold (attempts): on 2^22 net13 cells the
// fused burn took 30.6 s handing off at 2048 attempts, 29.9 s at 8192, and
// 46.7 s with no hand-off (the cells that run to the step cap then finish one
// lane at a time after the bulk)
constexpr int kHandoff = 8192;
using Key = std::tuple<std::string, int, int, int, int>;
std::mutex g_mu;
std::map<Key, Tuned> g_table;
bool g_loaded = false;

std::string device_name() {
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceProp p;
  if (cudaGetDeviceProperties(&p, dev) != cudaSuccess) return "unknown";
  std::string s = p.name;
  for (char &c : s)
    if (c == ' ' || c == '"') c = '_';
  return s;
}

Key key_of(const mc_network *net, int lu) {
  return Key(device_name(), net ? net->n : 0, net ? net->R : 0, net ? net->energy : 0, lu);
}

void load_cache() {
  if (g_loaded) return;
  g_loaded = true;
  const char *path = std::getenv("MC_AUTOTUNE_CACHE");
  if (!path) return;
  FILE *f = std::fopen(path, "r");
  if (!f) return;
  char line[512];
  while (std::fgets(line, sizeof line, f)) {
    char dev[256];
    int n, R, en, lu, var, thr, bps, stg, strag;
    if (std::sscanf(line,
                    "{\"device\": \"%255[^\"]\", \"n\": %d, \"R\": %d, \"energy\": %d, \"lu\": %d, "
                    "\"variant\": %d, \"threads\": %d, \"blocks_per_sm\": %d, \"staging\": %d, "
                    "\"straggler_steps\": %d}",
                    dev, &n, &R, &en, &lu, &var, &thr, &bps, &stg, &strag) == 10)
      g_table[Key(dev, n, R, en, lu)] = Tuned{var, thr, bps, strag, stg};
  }
  std::fclose(f);
}

void save_entry(const Key &k, const Tuned &t) {
  const char *path = std::getenv("MC_AUTOTUNE_CACHE");
  if (!path) return;
  FILE *f = std::fopen(path, "a");
  if (!f) return;
  std::fprintf(f,
               "{\"device\": \"%s\", \"n\": %d, \"R\": %d, \"energy\": %d, \"lu\": %d, \"variant\": %d, "
               "\"threads\": %d, \"blocks_per_sm\": %d, \"staging\": %d, \"straggler_steps\": %d}\n",
               std::get<0>(k).c_str(), std::get<1>(k), std::get<2>(k), std::get<3>(k), std::get<4>(k), t.variant,
               t.threads, t.blocks_per_sm, t.staging, t.strag_steps);
  std::fclose(f);
}
}  // namespace

Tuned mc::autotune_pick(const mc_network *net, const mc_burn_opts &o) {
  // defaults: thread-per-cell with hand-off for small networks, warp-per-cell
  // above 16 ODEs (the per-cell matrices no longer fit a lane's share of L1)
  Tuned t{(net && net->n > 16) ? MC_VARIANT_WARP : MC_VARIANT_PERSISTENT, 128, 2, kHandoff, MC_STAGING_SHARED};
  {
    std::lock_guard<std::mutex> lk(g_mu);
    load_cache();
    auto it = g_table.find(key_of(net, o.lu_precision));
    if (it != g_table.end()) t = it->second;
  }
  if (o.variant != MC_VARIANT_AUTO) t.variant = o.variant;
  if (o.block_threads) t.threads = o.block_threads;
  if (o.blocks_per_sm) t.blocks_per_sm = o.blocks_per_sm;
  if (o.straggler_steps) t.strag_steps = o.straggler_steps;
  if (o.staging) t.staging = o.staging;
  return t;
}

extern "C" mc_status mc_autotune(const mc_network *net, const mc_burn_opts *opts, int64_t n_sample, double dt,
                                 const double *x, int64_t ld, const double *T, const double *ndens,
                                 void *stream, mc_burn_opts *best) {
  if (!net || !x || n_sample <= 0 || ld < n_sample || (net->energy && !T))
    return set_error(MC_E_INVALID, "mc_autotune: bad arguments");
  mc_burn_opts o;
  mc_status s = check_opts(opts, &o);
  if (s != MC_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t n = n_sample;
  double *wx = nullptr, *wT = nullptr;
  int32_t *ws = nullptr;
  cudaError_t e = dev_malloc((void **)&wx, sizeof(double) * net->S * n);
  if (e == cudaSuccess && T) e = dev_malloc((void **)&wT, sizeof(double) * n);
  if (e == cudaSuccess) e = dev_malloc((void **)&ws, sizeof(int32_t) * n);
  if (e != cudaSuccess) {
    cudaFree(wx);
    cudaFree(wT);
    return cuda_error(e, "autotune buffers");
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  struct Cand { int var, thr, bps, stg, strag; };
  // one timed burn of the sample with a candidate; returns false on an error
  auto trial = [&](const Cand &c, float *ms_out) -> bool {
    e = cudaMemcpy2DAsync(wx, sizeof(double) * n, x, sizeof(double) * ld, sizeof(double) * n, net->S,
                          cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess && T) e = cudaMemcpyAsync(wT, T, sizeof(double) * n, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return false;
    mc_burn_opts t = o;
    t.variant = c.var;
    t.block_threads = c.thr;
    t.blocks_per_sm = c.bps ? c.bps : 1;
    t.staging = c.stg;
    t.straggler_steps = c.strag;
    CellArgs a{};
    a.n_cells = n;
    a.ld = n;
    a.dt = dt;
    a.x = wx;
    a.T = wT;
    a.nd = ndens;
    a.status = ws;
    cudaEventRecord(e0, st);
    s = burn_device(net, t, a, st);
    cudaEventRecord(e1, st);
    if (s != MC_OK) return false;
    e = cudaEventSynchronize(e1);
    if (e != cudaSuccess) return false;
    cudaEventElapsedTime(ms_out, e0, e1);
    return true;
  };
  float best_ms = 1e30f;
  Cand win{MC_VARIANT_PLAIN, 64, 0, MC_STAGING_SHARED, kHandoff};
  bool failed = false;
  auto consider = [&](const Cand &c) {
    if (failed) return;
    float ms = 0.f;
    if (!trial(c, &ms)) {
      failed = true;
      return;
    }
    if (ms < best_ms) {
      best_ms = ms;
      win = c;
    }
  };
  // first pass: variant x threads x blocks per SM
  for (int thr : {64, 128, 256}) consider({MC_VARIANT_PLAIN, thr, 0, MC_STAGING_SHARED, kHandoff});
  for (int thr : {64, 128, 256})
    for (int bps : {1, 2, 4}) consider({MC_VARIANT_PERSISTENT, thr, bps, MC_STAGING_SHARED, kHandoff});
  for (int bps : {1, 2, 4}) consider({MC_VARIANT_WARP, 128, bps, MC_STAGING_SHARED, kHandoff});
  if (win.var == MC_VARIANT_PERSISTENT) {
    // second pass: staging of the matrix work; third: hand-off threshold
    Cand c = win;
    c.stg = MC_STAGING_LANE;
    consider(c);
    for (int strag : {2048, 32768, -1}) {
      c = win;
      c.strag = strag;
      consider(c);
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(wx);
  cudaFree(wT);
  cudaFree(ws);
  if (s != MC_OK) return s;
  if (e != cudaSuccess) return cuda_error(e, "autotune trial");
  Tuned t{win.var, win.thr, win.bps ? win.bps : 1, win.strag, win.stg};
  {
    std::lock_guard<std::mutex> lk(g_mu);
    load_cache();
    const Key k = key_of(net, o.lu_precision);
    g_table[k] = t;
    save_entry(k, t);
  }
  if (best) {
    *best = o;
    best->variant = t.variant;
    best->block_threads = t.threads;
    best->blocks_per_sm = t.blocks_per_sm;
    best->staging = t.staging;
    best->straggler_steps = t.strag_steps;
  }
  return MC_OK;
}
