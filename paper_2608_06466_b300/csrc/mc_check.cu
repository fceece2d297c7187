// mc_check.cu -- host side of the bounds-check build: one check record per
// device, the per-call verification that every cell was stored exactly once,
// and the report (mc_bounds_report / mc_bounds_reset, exported by both builds;
// the normal build reports enabled = 0 and checks nothing).
#include <mutex>

#include "mc_internal.h"
#include "mc_kernels.cuh"

using namespace mc;

#ifdef MC_BOUNDS_CHECK
namespace {

constexpr int kMaxDevices = 64;
std::mutex g_bc_mu;
BoundsCheck *g_bc[kMaxDevices] = {};
unsigned int *g_stores[kMaxDevices] = {};
int64_t g_stores_cap[kMaxDevices] = {};

BoundsCheck *record_of(int dev) {
  if (dev < 0 || dev >= kMaxDevices) return nullptr;
  std::lock_guard<std::mutex> lk(g_bc_mu);
  if (!g_bc[dev]) {
    BoundsCheck *p = nullptr;
    if (dev_malloc((void **)&p, sizeof(BoundsCheck)) != cudaSuccess) return nullptr;
    if (cudaMemset(p, 0, sizeof(BoundsCheck)) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) {
      cudaFree(p);
      return nullptr;
    }
    g_bc[dev] = p;
  }
  return g_bc[dev];
}

__global__ void k_bc_begin(BoundsCheck *bc, unsigned int *stores, long long n) {
  bc->stores = stores;
  bc->cells = n;
}

// cells of the call whose store count is not exactly one
__global__ void k_bc_verify(BoundsCheck *bc, long long n) {
  unsigned long long bad = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    bad += (bc->stores[i] != 1u) ? 1ull : 0ull;
  for (int o = 16; o > 0; o >>= 1) bad += __shfl_xor_sync(0xffffffffu, bad, o);
  if ((threadIdx.x & 31) == 0 && bad) atomicAdd((unsigned long long *)&bc->not_once, bad);
}

__global__ void k_bc_end(BoundsCheck *bc, long long n) {
  bc->calls += 1;
  bc->cells_checked += n;
  bc->stores = nullptr;
  bc->cells = 0;
}

}  // namespace

void mc::bc_attach(CellArgs &a) {
  if (a.bc) return;
  int dev = 0;
  cudaGetDevice(&dev);
  a.bc = record_of(dev);
}

mc_status mc::bc_begin(int64_t n, cudaStream_t st) {
  int dev = 0;
  cudaGetDevice(&dev);
  BoundsCheck *bc = record_of(dev);
  if (!bc) return set_error(MC_E_CUDA, "bounds-check record allocation");
  {
    std::lock_guard<std::mutex> lk(g_bc_mu);
    if (n > g_stores_cap[dev]) {
      if (g_stores[dev]) {
        cudaDeviceSynchronize();
        cudaFree(g_stores[dev]);
      }
      g_stores[dev] = nullptr;
      g_stores_cap[dev] = 0;
      if (dev_malloc((void **)&g_stores[dev], sizeof(unsigned int) * (size_t)n) != cudaSuccess)
        return set_error(MC_E_NOMEM, "bounds-check store counters");
      g_stores_cap[dev] = n;
    }
  }
  cudaError_t e = cudaMemsetAsync(g_stores[dev], 0, sizeof(unsigned int) * (size_t)n, st);
  if (e != cudaSuccess) return cuda_error(e, "bounds-check reset");
  k_bc_begin<<<1, 1, 0, st>>>(bc, g_stores[dev], (long long)n);
  e = cudaGetLastError();
  return e == cudaSuccess ? MC_OK : cuda_error(e, "bounds-check begin");
}

mc_status mc::bc_end(int64_t n, cudaStream_t st) {
  int dev = 0;
  cudaGetDevice(&dev);
  BoundsCheck *bc = record_of(dev);
  if (!bc) return set_error(MC_E_CUDA, "bounds-check record allocation");
  const int blocks = (int)std::min<int64_t>(1184, (n + 255) / 256);
  if (n > 0) k_bc_verify<<<blocks, 256, 0, st>>>(bc, (long long)n);
  k_bc_end<<<1, 1, 0, st>>>(bc, (long long)n);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? MC_OK : cuda_error(e, "bounds-check verify");
}

extern "C" mc_status mc_bounds_report(int32_t device, mc_bounds_info *out) {
  if (!out) return set_error(MC_E_INVALID, "mc_bounds_report: null out");
  *out = mc_bounds_info{};
  out->enabled = 1;
  cudaError_t e = cudaSetDevice(device);
  if (e != cudaSuccess) return cuda_error(e, "mc_bounds_report: device");
  BoundsCheck *bc = record_of(device);
  if (!bc) return set_error(MC_E_CUDA, "bounds-check record allocation");
  BoundsCheck h{};
  e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(&h, bc, sizeof h, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_error(e, "mc_bounds_report");
  out->refused = h.refused;
  out->first_site = h.site;
  out->first_index = h.index;
  out->first_bound = h.bound;
  out->calls_checked = h.calls;
  out->cells_checked = h.cells_checked;
  out->cells_not_once = h.not_once;
  return MC_OK;
}

extern "C" mc_status mc_bounds_reset(int32_t device) {
  cudaError_t e = cudaSetDevice(device);
  if (e != cudaSuccess) return cuda_error(e, "mc_bounds_reset: device");
  BoundsCheck *bc = record_of(device);
  if (!bc) return set_error(MC_E_CUDA, "bounds-check record allocation");
  e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemset(bc, 0, sizeof(BoundsCheck));
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  return e == cudaSuccess ? MC_OK : cuda_error(e, "mc_bounds_reset");
}

#else  // the normal build: no checks, nothing recorded

void mc::bc_attach(CellArgs &) {}
mc_status mc::bc_begin(int64_t, cudaStream_t) { return MC_OK; }
mc_status mc::bc_end(int64_t, cudaStream_t) { return MC_OK; }

extern "C" mc_status mc_bounds_report(int32_t, mc_bounds_info *out) {
  if (!out) return set_error(MC_E_INVALID, "mc_bounds_report: null out");
  *out = mc_bounds_info{};
  return MC_OK;
}

extern "C" mc_status mc_bounds_reset(int32_t) { return MC_OK; }

#endif
