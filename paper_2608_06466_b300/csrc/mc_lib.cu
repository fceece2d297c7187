// mc_lib.cu -- C ABI of the per-cell burn (see include/mc.h): network upload,
// batch burns (plain / persistent, FP64 / FP32 iteration matrix with an FP64
// retry pass), host-pointer staging, error reporting.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <atomic>
#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "mc.h"
#include "mc_kernels.cuh"
#include "mc_internal.h"

using namespace mc;

// ---------------------------------------------------------------- errors
static thread_local std::string g_err;
static thread_local int64_t g_launches = 0;

mc_status mc::set_error(mc_status code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

mc_status mc::cuda_error(cudaError_t e, const char *what) {
  return set_error(MC_E_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

void mc::count_launch(int64_t k) { g_launches += k; }

static std::atomic<int64_t> g_allocs{0};

cudaError_t mc::dev_malloc(void **p, size_t bytes) {
  g_allocs.fetch_add(1);
  return cudaMalloc(p, bytes);
}

cudaError_t mc::dev_malloc_async(void **p, size_t bytes, cudaStream_t st) {
  g_allocs.fetch_add(1);
  return cudaMallocAsync(p, bytes, st);
}

cudaError_t mc::host_malloc_pinned(void **p, size_t bytes) {
  g_allocs.fetch_add(1);
  return cudaMallocHost(p, bytes);
}

extern "C" int64_t mc_alloc_count(void) { return g_allocs.load(); }

extern "C" const char *mc_last_error(void) { return g_err.c_str(); }
extern "C" int32_t mc_version(void) { return 1; }
extern "C" int64_t mc_launch_count(int32_t reset) {
  const int64_t v = g_launches;
  if (reset) g_launches = 0;
  return v;
}

extern "C" void mc_burn_opts_default(mc_burn_opts *o) {
  if (!o) return;
  o->rtol = 1e-6;
  o->atol = 1e-10;
  o->max_order = 5;
  o->max_steps = 100000;
  o->lu_precision = 64;
  o->variant = MC_VARIANT_AUTO;
  o->block_threads = 0;
  o->blocks_per_sm = 0;
  o->straggler_steps = 0;
  o->jacobian = MC_JAC_ANALYTIC;
  o->staging = MC_STAGING_AUTO;
}

// ---------------------------------------------------------------- networks
extern "C" mc_status mc_network_create(const mc_network_desc *d, mc_network **out) {
  if (!d || !out) return set_error(MC_E_INVALID, "mc_network_create: null argument");
  *out = nullptr;
  const int S = d->n_species, R = d->n_reactions;
  const int n = S + (d->energy_eq ? 1 : 0);
  if (S < 1 || R < 0 || (R > 0 && (!d->react || !d->prod || !d->A_f || !d->b_f || !d->C_f ||
                                   !d->A_r || !d->b_r || !d->C_r || !d->dE_eV)))
    return set_error(MC_E_INVALID, "mc_network_create: bad sizes or null arrays");
  if (n > NMAX_ODE || R > RMAX_REACT)
    return set_error(MC_E_UNSUPPORTED, "mc_network_create: %d ODEs / %d reactions exceed %d / %d", n,
                     R, NMAX_ODE, RMAX_REACT);
  if (d->energy_eq && !(d->gamma > 1.0) )
    return set_error(MC_E_INVALID, "mc_network_create: gamma must exceed 1");
  std::vector<int4> side(R > 0 ? R : 1);
  std::vector<RxPar> par(R > 0 ? R : 1);
  for (int r = 0; r < R; ++r) {
    int v[4] = {d->react[2 * r], d->react[2 * r + 1], d->prod[2 * r], d->prod[2 * r + 1]};
    for (int k = 0; k < 4; ++k)
      if (v[k] < -1 || v[k] >= S) return set_error(MC_E_INVALID, "reaction %d: species index out of range", r);
    if (v[0] < 0 || v[2] < 0) return set_error(MC_E_INVALID, "reaction %d: slot 0 of a side is empty", r);
    side[r] = make_int4(v[0], v[1], v[2], v[3]);
    const double Af = d->A_f[r], Ar = d->A_r[r];
    if (!(Af >= 0.0) || !(Ar >= 0.0) || !std::isfinite(Af) || !std::isfinite(Ar) ||
        !std::isfinite(d->b_f[r]) || !std::isfinite(d->C_f[r]) || !std::isfinite(d->b_r[r]) ||
        !std::isfinite(d->C_r[r]) || !std::isfinite(d->dE_eV[r]))
      return set_error(MC_E_INVALID, "reaction %d: rate parameters must be finite, A >= 0", r);
    par[r].lnAf = Af > 0.0 ? std::log(Af) : -INFINITY;
    par[r].bf = d->b_f[r];
    par[r].Cf = d->C_f[r];
    par[r].lnAr = Ar > 0.0 ? std::log(Ar) : -INFINITY;
    par[r].br = d->b_r[r];
    par[r].Cr = d->C_r[r];
    par[r].dE = d->dE_eV[r];
    par[r].rev = Ar > 0.0 ? 1.0 : 0.0;
  }
  mc_network *net = new (std::nothrow) mc_network();
  if (!net) return set_error(MC_E_NOMEM, "mc_network_create: host allocation");
  net->S = S;
  net->R = R;
  net->n = n;
  net->energy = d->energy_eq ? 1 : 0;
  net->gamma = d->gamma;
  net->side_h = side;
  net->par_h = par;
  cudaError_t e = cudaGetDevice(&net->device);
  if (e != cudaSuccess) { delete net; return cuda_error(e, "cudaGetDevice"); }
  e = dev_malloc((void **)&net->side_d, sizeof(int4) * side.size());
  if (e == cudaSuccess) e = dev_malloc((void **)&net->par_d, sizeof(RxPar) * par.size());
  if (e == cudaSuccess) e = cudaMemcpy(net->side_d, side.data(), sizeof(int4) * side.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(net->par_d, par.data(), sizeof(RxPar) * par.size(), cudaMemcpyHostToDevice);
  // occurrence lists in the order the right-hand side scatters: per reaction
  // reactant 0, product 0, reactant 1, product 1
  std::vector<std::vector<int>> occ(S);
  for (int r = 0; r < R; ++r) {
    const int4 q = side[r];
    const int sp[4] = {q.x, q.z, q.y, q.w};
    const int slot[4] = {0, 2, 1, 3};
    for (int k = 0; k < 4; ++k)
      if (sp[k] >= 0) occ[sp[k]].push_back(4 * r + slot[k]);
  }
  std::vector<int> csr(S + 1);
  csr[0] = 0;
  for (int i = 0; i < S; ++i) csr[i + 1] = csr[i] + (int)occ[i].size();
  for (int i = 0; i < S; ++i) csr.insert(csr.end(), occ[i].begin(), occ[i].end());
  net->csr_len = (int)csr.size();
  // 2^(j/64) for the table-driven exponential, rounded once from extended precision
  double tab[64];
  for (int j = 0; j < 64; ++j) tab[j] = (double)exp2l((long double)j / 64.0L);
  if (e == cudaSuccess) e = dev_malloc((void **)&net->exptab_d, sizeof tab);
  if (e == cudaSuccess) e = cudaMemcpy(net->exptab_d, tab, sizeof tab, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = dev_malloc((void **)&net->csr_d, sizeof(int) * csr.size());
  if (e == cudaSuccess) e = cudaMemcpy(net->csr_d, csr.data(), sizeof(int) * csr.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(net->side_d);
    cudaFree(net->par_d);
    cudaFree(net->csr_d);
    cudaFree(net->exptab_d);
    delete net;
    return cuda_error(e, "mc_network_create upload");
  }
  *out = net;
  return MC_OK;
}

extern "C" mc_status mc_network_destroy(mc_network *net) {
  if (!net) return MC_OK;
  cudaFree(net->side_d);
  cudaFree(net->par_d);
  cudaFree(net->csr_d);
  cudaFree(net->exptab_d);
  delete net;
  return MC_OK;
}

extern "C" int32_t mc_network_n_ode(const mc_network *net) { return net ? net->n : 0; }

DNet mc::dnet_of(const mc_network *net) {
  DNet d;
  d.S = net->S;
  d.R = net->R;
  d.n = net->n;
  d.energy = net->energy;
  d.gm1 = net->gamma - 1.0;
  d.side = (const int4 *)net->side_d;
  d.par = (const RxPar *)net->par_d;
  d.csr_ptr = (const int *)net->csr_d;
  d.csr_ent = (const int *)net->csr_d + (net->S + 1);
  d.exptab = (const double *)net->exptab_d;
  return d;
}

// ---------------------------------------------------------------- device scratch
// Library-owned scratch, one set per (device, stream) so burns issued on
// different streams never share queue counters or lists: the persistent queue
// counters, the FP32 pass's retry lists, the cost order, the straggler records
// and the retry ladder's lists (each grown on demand, never shrunk).
namespace {
struct DevScratch {
  unsigned long long *next = nullptr;   // [MAX_QUEUES] queue counters
  uint32_t *retry_count = nullptr;      // [MAX_QUEUES] retry-list lengths
  int32_t *retry = nullptr;             // retry lists (cells)
  int64_t retry_cap = 0;
  void *rec = nullptr;                  // straggler records
  uint32_t *rec_count = nullptr;
  size_t rec_bytes = 0;
  void *order = nullptr;                // cost order: list, bucket bytes, histogram
  int64_t order_cap = 0;
  void *ladder = nullptr;               // retry ladder: two cell lists and their counts
  int64_t ladder_cap = 0;
};
std::mutex g_scratch_mu;
std::map<std::pair<int, uintptr_t>, DevScratch> g_scratch;

thread_local cudaStream_t g_cur_stream = nullptr;

DevScratch &scratch_of(int dev) {
  return g_scratch[std::make_pair(dev, (uintptr_t)g_cur_stream)];
}

// Scratch grows by stream-ordered allocation on its own stream: the old
// buffer is freed after the work already queued on the stream (which may
// still read it), and neither step synchronises the device, so a burn on one
// stream never waits for burns on others.
cudaError_t retire(void *p) {
  if (!p) return cudaSuccess;
  return cudaFreeAsync(p, g_cur_stream);
}

cudaError_t grow(void **p, size_t bytes) { return dev_malloc_async(p, bytes, g_cur_stream); }
}  // namespace

void mc::scratch_stream(cudaStream_t st) { g_cur_stream = st; }

// Hand the scratch set of (dev, st) to the caller (a graph that keeps using it
// after its capture stream is gone); free it with scratch_free.
void *mc::scratch_detach(int dev, cudaStream_t st) {
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  auto it = g_scratch.find(std::make_pair(dev, (uintptr_t)st));
  if (it == g_scratch.end()) return nullptr;
  DevScratch *d = new DevScratch(it->second);
  g_scratch.erase(it);
  return d;
}

void mc::scratch_free(void *h) {
  DevScratch *d = (DevScratch *)h;
  if (!d) return;
  cudaFree(d->next);
  cudaFree(d->retry);
  cudaFree(d->rec);
  cudaFree(d->rec_count);
  cudaFree(d->order);
  cudaFree(d->ladder);
  delete d;
}

mc_status mc::scratch_get(int dev, int64_t retry_cells, unsigned long long **next, uint32_t **rcount,
                          int32_t **retry) {
  if (dev < 0) return set_error(MC_E_INVALID, "device %d out of range", dev);
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  DevScratch &s = scratch_of(dev);
  cudaError_t e;
  if (!s.next) {
    e = grow((void **)&s.next, (sizeof(unsigned long long) + sizeof(uint32_t)) * MAX_QUEUES);
    if (e != cudaSuccess) return cuda_error(e, "scratch allocation");
    s.retry_count = (uint32_t *)(s.next + MAX_QUEUES);
  }
  if (retry_cells > s.retry_cap) {
    e = retire(s.retry);
    s.retry = nullptr;
    s.retry_cap = 0;
    if (e != cudaSuccess) return cuda_error(e, "scratch grow sync");
    e = grow((void **)&s.retry, sizeof(int32_t) * retry_cells);
    if (e != cudaSuccess) return cuda_error(e, "retry list allocation");
    s.retry_cap = retry_cells;
  }
  *next = s.next;
  *rcount = s.retry_count;
  *retry = s.retry;
  return MC_OK;
}

mc_status mc::straggler_scratch(size_t bytes, void **rec, uint32_t **count) {
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  DevScratch &s = scratch_of(dev);
  cudaError_t e;
  if (!s.rec_count) {
    e = grow((void **)&s.rec_count, 256);
    if (e != cudaSuccess) return cuda_error(e, "straggler counter allocation");
  }
  if (bytes > s.rec_bytes) {
    e = retire(s.rec);
    s.rec = nullptr;
    s.rec_bytes = 0;
    if (e != cudaSuccess) return cuda_error(e, "straggler grow sync");
    e = grow((void **)&s.rec, bytes);
    if (e != cudaSuccess) return cuda_error(e, "straggler record allocation");
    s.rec_bytes = bytes;
  }
  *rec = s.rec;
  *count = s.rec_count;
  return MC_OK;
}

mc_status mc::ladder_scratch(int dev, int64_t n, int32_t **lists, uint32_t **counts) {
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  DevScratch &s = scratch_of(dev);
  if (n > s.ladder_cap) {
    cudaError_t e = retire(s.ladder);
    s.ladder = nullptr;
    s.ladder_cap = 0;
    if (e != cudaSuccess) return cuda_error(e, "ladder grow sync");
    e = grow(&s.ladder, 256 + sizeof(int32_t) * 2 * (size_t)n);
    if (e != cudaSuccess) return cuda_error(e, "ladder list allocation");
    s.ladder_cap = n;
  }
  *counts = (uint32_t *)s.ladder;
  *lists = (int32_t *)((char *)s.ladder + 256);
  return MC_OK;
}

mc_status mc::order_scratch(int dev, int64_t n, int32_t **index, uint8_t **bkt, uint32_t **hist) {
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  DevScratch &s = scratch_of(dev);
  const size_t list = ((size_t)n * sizeof(int32_t) + 255) & ~(size_t)255;
  const size_t bytes = ((size_t)n + 255) & ~(size_t)255;
  if (n > s.order_cap) {
    cudaError_t e = retire(s.order);
    s.order = nullptr;
    s.order_cap = 0;
    if (e != cudaSuccess) return cuda_error(e, "order grow sync");
    e = grow((void **)&s.order, list + bytes + sizeof(uint32_t) * ORDER_BUCKETS);
    if (e != cudaSuccess) return cuda_error(e, "order buffer allocation");
    s.order_cap = n;
  }
  // the layout follows the capacity, so a smaller n reuses the same offsets
  const size_t cl = ((size_t)s.order_cap * sizeof(int32_t) + 255) & ~(size_t)255;
  const size_t cb = ((size_t)s.order_cap + 255) & ~(size_t)255;
  *index = (int32_t *)s.order;
  *bkt = (uint8_t *)s.order + cl;
  *hist = (uint32_t *)((uint8_t *)s.order + cl + cb);
  return MC_OK;
}

// ---------------------------------------------------------------- launches
namespace {

template <typename LT>
mc_status dispatch(const mc_network *net, const DNet &d, const Opts &o, const CellArgs &a,
                   int variant, int threads, int bps, int strag, unsigned long long *next, cudaStream_t st) {
  switch (net->n) {
    case 3: return launch_one<3, LT>(d, o, a, variant, threads, bps, strag, next, st);
    case 13: return launch_one<13, LT>(d, o, a, variant, threads, bps, strag, next, st);
    case 33: return launch_one<33, LT>(d, o, a, variant, threads, bps, strag, next, st);
    default: break;
  }
  if (net->n <= 8) return launch_one<8, LT>(d, o, a, variant, threads, bps, strag, next, st);
  if (net->n <= 16) return launch_one<16, LT>(d, o, a, variant, threads, bps, strag, next, st);
  if (net->n <= 24) return launch_one<24, LT>(d, o, a, variant, threads, bps, strag, next, st);
  return launch_one<NMAX_ODE, LT>(d, o, a, variant, threads, bps, strag, next, st);
}

bool is_device_ptr(const void *p) {
  if (!p) return true;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

mc_status mc::check_opts(const mc_burn_opts *opts, mc_burn_opts *o) {
  mc_burn_opts_default(o);
  if (opts) *o = *opts;
  if (!(o->rtol > 0.0) || !(o->atol > 0.0) || !std::isfinite(o->rtol) || !std::isfinite(o->atol))
    return set_error(MC_E_INVALID, "rtol and atol must be positive and finite");
  if (o->max_order < 1 || o->max_order > QMAX) return set_error(MC_E_INVALID, "max_order must be 1..5");
  if (o->max_steps < 1) return set_error(MC_E_INVALID, "max_steps must be positive");
  if (o->lu_precision != 64 && o->lu_precision != 32)
    return set_error(MC_E_INVALID, "lu_precision must be 64 or 32");
  if (o->variant < 0 || o->variant > MC_VARIANT_WARP) return set_error(MC_E_INVALID, "unknown variant");
  if (o->block_threads < 0 || o->block_threads > 1024 || (o->block_threads % 32) != 0)
    return set_error(MC_E_INVALID, "block_threads must be a multiple of 32 up to 1024");
  if (o->blocks_per_sm < 0 || o->blocks_per_sm > 32) return set_error(MC_E_INVALID, "blocks_per_sm must be 0..32");
  if (o->straggler_steps < -1) return set_error(MC_E_INVALID, "straggler_steps must be -1, 0 or positive");
  if (o->jacobian != MC_JAC_ANALYTIC && o->jacobian != MC_JAC_FD)
    return set_error(MC_E_INVALID, "jacobian must be MC_JAC_ANALYTIC or MC_JAC_FD");
  if (o->staging < MC_STAGING_AUTO || o->staging > MC_STAGING_LANE)
    return set_error(MC_E_INVALID, "staging must be MC_STAGING_AUTO, _SHARED or _LANE");
  return MC_OK;
}

// Burn one segment on the device (device pointers) with the given scratch:
// queue counters next[0..1], the FP32 pass's retry count and list (n_cells
// entries). Runs the FP32 pass and, when it leaves Newton failures behind, the
// FP64 retry pass over them. Straggler hand-off only when allow_strag.
mc_status mc::burn_device_scratch(const mc_network *net, const mc_burn_opts &ob, const CellArgs &a0,
                                  cudaStream_t st, unsigned long long *next, uint32_t *rcount, int32_t *retry,
                                  bool allow_strag) {
  Tuned tu = autotune_pick(net, ob);
  if (!allow_strag) tu.strag_steps = 0;
  Opts o{ob.rtol, ob.atol, ob.max_order, ob.max_steps, ob.jacobian == MC_JAC_FD ? 1 : 0,
         tu.staging == MC_STAGING_LANE ? 1 : 0};
  const DNet d = dnet_of(net);
  if (ob.lu_precision == 64)
    return dispatch<double>(net, d, o, a0, tu.variant, tu.threads, tu.blocks_per_sm, tu.strag_steps, next, st);
  CellArgs a = a0;
  a.retry = retry;
  a.retry_count = rcount;
  a.retry_mask = FP32_RETRY_MASK;
  cudaError_t e = cudaMemsetAsync(rcount, 0, sizeof(uint32_t), st);
  if (e != cudaSuccess) return cuda_error(e, "retry counter reset");
  mc_status s = dispatch<float>(net, d, o, a, tu.variant, tu.threads, tu.blocks_per_sm, tu.strag_steps, next, st);
  if (s != MC_OK) return s;
  // FP64 pass over the list; its length is read on the device
  CellArgs b = a0;
  b.index = retry;
  b.n_dev = rcount;
  b.n_cells = a0.n_cells;
  return dispatch<double>(net, d, o, b, MC_VARIANT_PERSISTENT, tu.threads, tu.blocks_per_sm, 0, next, st);
}

// Burn with the library scratch set of stream st.
mc_status mc::burn_device(const mc_network *net, const mc_burn_opts &ob, const CellArgs &a0,
                          cudaStream_t st) {
  int dev = 0;
  cudaGetDevice(&dev);
  scratch_stream(st);
  unsigned long long *next;
  uint32_t *rcount;
  int32_t *retry;
  mc_status s = scratch_get(dev, ob.lu_precision == 32 ? a0.n_cells : 0, &next, &rcount, &retry);
  if (s != MC_OK) return s;
  // queue-fed launches hand out the cells in decreasing cost order
  CellArgs a = a0;
  bc_attach(a);
  if (!a0.index && !a0.n_dev && autotune_pick(net, ob).variant != MC_VARIANT_PLAIN) {
    int32_t *order;
    uint8_t *bkt;
    uint32_t *hist;
    s = order_scratch(dev, a0.n_cells, &order, &bkt, &hist);
    if (s != MC_OK) return s;
    s = order_cells(net, Opts{ob.rtol, ob.atol, ob.max_order, ob.max_steps, 0}, a0, order, bkt, hist, st);
    if (s != MC_OK) return s;
    a.index = order;
  }
  return burn_device_scratch(net, ob, a, st, next, rcount, retry, true);
}

// Shared argument checks of the batch entry points. *on_dev tells whether the
// cell arrays are device (true) or host memory.
mc_status mc::check_batch(const mc_network *net, int64_t n_cells, double dt, double *x, int64_t ld, double *T,
                          const double *ndens, const double *rate_scale, int32_t *status, int32_t *stats,
                          bool *on_dev) {
  if (!net) return set_error(MC_E_INVALID, "null network");
  if (n_cells < 0 || ld < n_cells || n_cells > (int64_t)INT32_MAX)
    return set_error(MC_E_INVALID, "need 0 <= n_cells <= ld and n_cells < 2^31");
  if (!(dt > 0.0) || !std::isfinite(dt)) return set_error(MC_E_INVALID, "dt must be positive");
  if (n_cells == 0) {
    *on_dev = true;
    return MC_OK;
  }
  if (!x || !status) return set_error(MC_E_INVALID, "x and status are required");
  if (net->energy && !T) return set_error(MC_E_INVALID, "energy networks need T");
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev != net->device) return set_error(MC_E_INVALID, "network lives on device %d, current is %d", net->device, dev);
  const bool d = is_device_ptr(x);
  if (d != is_device_ptr(status) || (T && d != is_device_ptr(T)) || (ndens && d != is_device_ptr(ndens)) ||
      (rate_scale && d != is_device_ptr(rate_scale)) || (stats && d != is_device_ptr(stats)))
    return set_error(MC_E_INVALID, "mix of host and device arrays");
  *on_dev = d;
  return MC_OK;
}

namespace {

mc_status burn_batch_impl(const mc_network *net, const mc_burn_opts *opts, int64_t n_cells, double dt, double *x,
                          int64_t ld, double *T, const double *ndens, const double *rate_scale, const double *source,
                          int32_t *status, int32_t *stats, void *stream) {
  mc_burn_opts o;
  mc_status s = check_opts(opts, &o);
  if (s != MC_OK) return s;
  bool on_dev = true;
  s = check_batch(net, n_cells, dt, x, ld, T, ndens, rate_scale, status, stats, &on_dev);
  if (s != MC_OK) return s;
  if (n_cells == 0) return MC_OK;
  if (source && is_device_ptr(source) != on_dev) return set_error(MC_E_INVALID, "mix of host and device arrays");
  cudaStream_t st = (cudaStream_t)stream;
  CellArgs a{};
  a.n_cells = n_cells;
  a.ld = ld;
  a.dt = dt;
  if (on_dev) {
    a.x = x;
    a.T = T;
    a.nd = ndens;
    a.ks = rate_scale;
    a.src = source;
    a.status = status;
    a.stats = stats;
    s = bc_begin(n_cells, st);
    if (s == MC_OK) s = burn_device(net, o, a, st);
    if (s == MC_OK) s = bc_end(n_cells, st);
    return s;
  }
  // host arrays: stage through device memory, packed with ld = n_cells
  const int64_t nc = n_cells;
  const size_t bx = sizeof(double) * net->S * nc, b1 = sizeof(double) * nc;
  const size_t bks = rate_scale ? sizeof(double) * net->R * nc : 0;
  const size_t bsr = source ? sizeof(double) * net->n * nc : 0;
  const size_t bst = sizeof(int32_t) * nc, bsx = stats ? sizeof(int32_t) * MC_NSTAT * nc : 0;
  char *buf = nullptr;
  const size_t total = bx + (T ? b1 : 0) + (ndens ? b1 : 0) + bks + bsr + bst + bsx + 256 * 9;
  cudaError_t e = dev_malloc_async((void **)&buf, total, st);
  if (e != cudaSuccess) return cuda_error(e, "staging allocation");
  size_t off = 0;
  auto take = [&](size_t b) { char *p = buf + off; off += (b + 255) & ~(size_t)255; return p; };
  a.x = (double *)take(bx);
  a.T = T ? (double *)take(b1) : nullptr;
  a.nd = ndens ? (const double *)take(b1) : nullptr;
  a.ks = rate_scale ? (const double *)take(bks) : nullptr;
  a.src = source ? (const double *)take(bsr) : nullptr;
  a.status = (int32_t *)take(bst);
  a.stats = stats ? (int32_t *)take(bsx) : nullptr;
  a.ld = nc;
  auto h2d = [&](void *dst, const void *src, int rows) -> cudaError_t {
    return cudaMemcpy2DAsync(dst, sizeof(double) * nc, src, sizeof(double) * ld, sizeof(double) * nc, rows,
                             cudaMemcpyHostToDevice, st);
  };
  e = h2d(a.x, x, net->S);
  if (e == cudaSuccess && T) e = h2d(a.T, T, 1);
  if (e == cudaSuccess && ndens) e = h2d((void *)a.nd, ndens, 1);
  if (e == cudaSuccess && rate_scale) e = h2d((void *)a.ks, rate_scale, net->R);
  if (e == cudaSuccess && source) e = h2d((void *)a.src, source, net->n);
  if (e != cudaSuccess) { cudaFreeAsync(buf, st); return cuda_error(e, "host to device copy"); }
  s = bc_begin(n_cells, st);
  if (s == MC_OK) s = burn_device(net, o, a, st);
  if (s == MC_OK) s = bc_end(n_cells, st);
  if (s != MC_OK) { cudaFreeAsync(buf, st); return s; }
  e = cudaMemcpy2DAsync(x, sizeof(double) * ld, a.x, sizeof(double) * nc, sizeof(double) * nc, net->S,
                        cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && T)
    e = cudaMemcpyAsync(T, a.T, b1, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(status, a.status, bst, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && stats)
    e = cudaMemcpy2DAsync(stats, sizeof(int32_t) * ld, a.stats, sizeof(int32_t) * nc, sizeof(int32_t) * nc,
                          MC_NSTAT, cudaMemcpyDeviceToHost, st);
  cudaFreeAsync(buf, st);
  if (e != cudaSuccess) return cuda_error(e, "device to host copy");
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_error(e, "mc_burn_batch host round trip");
  return MC_OK;
}

}  // namespace

extern "C" mc_status mc_burn_batch(const mc_network *net, const mc_burn_opts *opts, int64_t n_cells,
                                   double dt, double *x, int64_t ld, double *T, const double *ndens,
                                   const double *rate_scale, int32_t *status, int32_t *stats,
                                   void *stream) {
  return burn_batch_impl(net, opts, n_cells, dt, x, ld, T, ndens, rate_scale, nullptr, status, stats, stream);
}

extern "C" mc_status mc_burn_batch_sdc(const mc_network *net, const mc_burn_opts *opts, int64_t n_cells,
                                       double dt, double *x, int64_t ld, double *T, const double *ndens,
                                       const double *rate_scale, const double *source, int32_t *status,
                                       int32_t *stats, void *stream) {
  if (!source && n_cells > 0) return set_error(MC_E_INVALID, "mc_burn_batch_sdc: source is required");
  return burn_batch_impl(net, opts, n_cells, dt, x, ld, T, ndens, rate_scale, source, status, stats, stream);
}

// ---------------------------------------------------------------- scratch size
namespace {
template <typename LT>
size_t lane_bytes(int n) {
  if (n <= 3) return sizeof(Lane<3, LT>);
  if (n <= 8) return sizeof(Lane<8, LT>);
  if (n <= 13) return sizeof(Lane<13, LT>);
  if (n <= 16) return sizeof(Lane<16, LT>);
  if (n <= 24) return sizeof(Lane<24, LT>);
  if (n <= 33) return sizeof(Lane<33, LT>);
  return sizeof(Lane<NMAX_ODE, LT>);
}
}  // namespace

size_t mc::burn_scratch_bytes(const mc_network *net, const mc_burn_opts &o, int64_t n) {
  size_t b = 2048;                                   // queue counters, retry count, record counts
  if (o.lu_precision == 32) b += sizeof(int32_t) * (size_t)n;  // FP64 retry list
  const Tuned tu = autotune_pick(net, o);
  if (tu.variant != MC_VARIANT_PLAIN)
    b += 5 * (size_t)n + 512 + sizeof(uint32_t) * ORDER_BUCKETS;  // cost order
  if (tu.variant == MC_VARIANT_PERSISTENT && tu.strag_steps > 0 && tu.strag_steps < o.max_steps) {
    const size_t lane = o.lu_precision == 32 ? lane_bytes<float>(net->n) : lane_bytes<double>(net->n);
    const int64_t rec_max = (int64_t)((2ull << 30) / lane);
    const int64_t cap = std::min<int64_t>(rec_max, std::max<int64_t>(256, n / 8));
    b += ((lane * (size_t)cap + 255) & ~(size_t)255) + sizeof(uint32_t) * (size_t)cap;
  }
  return b;
}

// ---------------------------------------------------------------- retry ladder
extern "C" mc_status mc_burn_ladder(const mc_network *net, const mc_rung *rungs, int32_t n_rungs, int64_t n_cells,
                                    double dt, double *x, int64_t ld, double *T, const double *ndens,
                                    const double *rate_scale, int32_t *status, int32_t *stats, int32_t *rung,
                                    void *stream) {
  if (!rungs || n_rungs < 1 || n_rungs > 8) return set_error(MC_E_INVALID, "mc_burn_ladder: 1..8 rungs");
  std::vector<mc_burn_opts> ro(n_rungs);
  for (int k = 0; k < n_rungs; ++k) {
    mc_status s = check_opts(&rungs[k].opts, &ro[k]);
    if (s != MC_OK) return s;
    if (rungs[k].method != MC_METHOD_BDF && rungs[k].method != MC_METHOD_RKC)
      return set_error(MC_E_INVALID, "mc_burn_ladder: rung %d: unknown method", k);
  }
  bool on_dev = true;
  mc_status s = check_batch(net, n_cells, dt, x, ld, T, ndens, rate_scale, status, stats, &on_dev);
  if (s != MC_OK) return s;
  if (n_cells == 0) return MC_OK;
  if (!on_dev || (rung && !is_device_ptr(rung)))
    return set_error(MC_E_INVALID, "mc_burn_ladder: cell arrays must be device memory");
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0;
  cudaGetDevice(&dev);
  scratch_stream(st);
  int32_t *lists;
  uint32_t *cnt;
  s = ladder_scratch(dev, n_cells, &lists, &cnt);
  if (s != MC_OK) return s;
  CellArgs base{};
  base.n_cells = n_cells;
  base.ld = ld;
  base.dt = dt;
  base.x = x;
  base.T = T;
  base.nd = ndens;
  base.ks = rate_scale;
  base.status = status;
  base.stats = stats;
  base.rung = rung;
  bc_attach(base);
  s = bc_begin(n_cells, st);
  if (s != MC_OK) return s;
  for (int k = 0; k < n_rungs; ++k) {
    CellArgs a = base;
    a.rung_id = k;
    const int cur = k & 1, nxt = cur ^ 1;
    if (k > 0) {
      // the previous rung's failures, counted on the device
      a.index = lists + cur * n_cells;
      a.n_dev = cnt + cur;
    }
    if (k + 1 < n_rungs) {
      cudaError_t e = cudaMemsetAsync(cnt + nxt, 0, sizeof(uint32_t), st);
      if (e != cudaSuccess) return cuda_error(e, "ladder list reset");
      a.lretry = lists + nxt * n_cells;
      a.lretry_count = cnt + nxt;
      a.lretry_mask = LADDER_MASK;
    }
    s = (rungs[k].method == MC_METHOD_RKC) ? burn_rkc_device(net, ro[k], a, st) : burn_device(net, ro[k], a, st);
    if (s != MC_OK) return s;
  }
  return bc_end(n_cells, st);
}
