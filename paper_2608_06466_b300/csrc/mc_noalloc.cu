// mc_noalloc.cu -- a burn entry point that allocates no memory.
//
// Some callers cannot let a library call cudaMalloc: applications that hand all
// device memory to their own arena up front (an AMR framework's pool, a fixed
// per-rank budget) and must not see allocations appear later, and latency-
// critical loops where cudaMalloc's implicit device synchronisation is not
// acceptable. For them, mc_burn_batch_noalloc runs the persistent burn with its
// scratch (queue counters, the FP32 pass's retry count and list) in a
// file-scope device array of fixed size instead of library-allocated buffers.
#include <cmath>
#include <mutex>

#include "mc_internal.h"
#include "mc_kernels.cuh"

using namespace mc;

namespace {

constexpr size_t kHead = 256;  // queue counters (2 x 8 bytes) at 0, retry count at 128
// Part of this file's device code: CUDA allocates it on a device when it
// loads that code there (lazily, at the first call's address look-up below),
// and it stays until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kHead + sizeof(int32_t) * MC_NOALLOC_MAX_CELLS];

std::mutex g_mu;
void *g_addr[256] = {};  // device address of the array, per device (set-up once)

}  // namespace

extern "C" mc_status mc_burn_batch_noalloc(const mc_network *net, const mc_burn_opts *opts, int64_t n_cells,
                                           double dt, double *x, int64_t ld, double *T, const double *ndens,
                                           const double *rate_scale, int32_t *status, int32_t *stats,
                                           void *stream) {
  mc_burn_opts o;
  mc_status s = check_opts(opts, &o);
  if (s != MC_OK) return s;
  if (n_cells > MC_NOALLOC_MAX_CELLS)
    return set_error(MC_E_INVALID, "mc_burn_batch_noalloc: %lld cells exceed its fixed maximum of %d",
                     (long long)n_cells, MC_NOALLOC_MAX_CELLS);
  bool on_dev = true;
  s = check_batch(net, n_cells, dt, x, ld, T, ndens, rate_scale, status, stats, &on_dev);
  if (s != MC_OK) return s;
  if (n_cells == 0) return MC_OK;
  if (!on_dev) return set_error(MC_E_INVALID, "mc_burn_batch_noalloc: cell arrays must be device memory");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_error(e, "mc_burn_batch_noalloc: device");
  if (dev < 0 || dev >= 256) return set_error(MC_E_INVALID, "device %d out of range", dev);
  char *base;
  {
    // set-up, once per device with that device current: the array's name is a
    // host-side stand-in, so its device address must come from the runtime
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
      void *p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess) return cuda_error(e, "mc_burn_batch_noalloc: scratch address");
      g_addr[dev] = p;
    }
    base = (char *)g_addr[dev];
  }
  unsigned long long *next = (unsigned long long *)base;
  uint32_t *rcount = (uint32_t *)(base + 128);
  int32_t *retry = (int32_t *)(base + kHead);
  CellArgs a{};
  a.n_cells = n_cells;
  a.ld = ld;
  a.dt = dt;
  a.x = x;
  a.T = T;
  a.nd = ndens;
  a.ks = rate_scale;
  a.status = status;
  a.stats = stats;
  bc_attach(a);
  mc_burn_opts q = o;
  q.variant = MC_VARIANT_PERSISTENT;
  // the counters and the retry count are cleared on the stream by the launches
  return burn_device_scratch(net, q, a, (cudaStream_t)stream, next, rcount, retry, false);
}
