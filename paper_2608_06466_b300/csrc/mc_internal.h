// mc_internal.h -- host-side internals shared by the library's translation units.
#pragma once

#include <cstdarg>
#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "mc.h"
#include "mc_device.cuh"

namespace mc {
struct CellArgs;
}

struct mc_network {
  int S = 0, R = 0, n = 0, energy = 0, device = 0;
  double gamma = 5.0 / 3.0;
  std::vector<int4> side_h;
  std::vector<mc::RxPar> par_h;
  void *side_d = nullptr;
  void *par_d = nullptr;
  void *csr_d = nullptr;          // csr_ptr[S+1] then csr_ent[...]
  void *exptab_d = nullptr;       // 2^(j/64), j = 0..63
  int csr_len = 0;
};

namespace mc {

constexpr int NMAX_ODE = 40;      // largest ODE count compiled
constexpr int RMAX_REACT = 512;   // largest reaction count accepted
constexpr int MAX_QUEUES = 16;    // persistent queue counters per device

mc_status set_error(mc_status code, const char *fmt, ...);
// Every device or pinned-host allocation of the library goes through these,
// so mc_alloc_count can report them.
cudaError_t dev_malloc(void **p, size_t bytes);
cudaError_t dev_malloc_async(void **p, size_t bytes, cudaStream_t st);
cudaError_t host_malloc_pinned(void **p, size_t bytes);
mc_status cuda_error(cudaError_t e, const char *what);
void count_launch(int64_t k);
DNet dnet_of(const mc_network *net);
mc_status check_opts(const mc_burn_opts *in, mc_burn_opts *out);
// Scratch of the stream most recently named by scratch_stream() on this thread.
void scratch_stream(cudaStream_t st);
void *scratch_detach(int dev, cudaStream_t st);
void scratch_free(void *h);
mc_status scratch_get(int dev, int64_t retry_cells, unsigned long long **next, uint32_t **rcount,
                      int32_t **retry);
mc_status burn_device(const mc_network *net, const mc_burn_opts &o, const CellArgs &a, cudaStream_t st);
// Bounds-check build (mc_check.cu; no-ops in the normal build): give a
// launch's cell arguments the device's check record, and bracket a call whose
// every cell must be stored exactly once.
void bc_attach(CellArgs &a);
mc_status bc_begin(int64_t n_cells, cudaStream_t st);
mc_status bc_end(int64_t n_cells, cudaStream_t st);
// Burn with the explicit Runge-Kutta-Chebyshev integrator (mc_rkc.cu).
mc_status burn_rkc_device(const mc_network *net, const mc_burn_opts &o, const CellArgs &a, cudaStream_t st);
mc_status burn_device_scratch(const mc_network *net, const mc_burn_opts &o, const CellArgs &a, cudaStream_t st,
                              unsigned long long *next, uint32_t *rcount, int32_t *retry, bool allow_strag);
mc_status check_batch(const mc_network *net, int64_t n_cells, double dt, double *x, int64_t ld, double *T,
                      const double *ndens, const double *rate_scale, int32_t *status, int32_t *stats,
                      bool *on_dev);

// Device bytes a burn of n cells of this network with these options makes the
// library scratch of its stream grow to (queue counters, FP32 retry list, cost
// order, straggler records), for budgeted admission.
size_t burn_scratch_bytes(const mc_network *net, const mc_burn_opts &o, int64_t n);

// launch shape chosen for a network and options
struct Tuned {
  int variant;        // MC_VARIANT_PLAIN, MC_VARIANT_PERSISTENT or MC_VARIANT_WARP
  int threads;        // threads per block
  int blocks_per_sm;  // persistent grid size per SM
  int strag_steps;    // attempts before a persistent lane hands its cell off (<= 0: never)
  int staging;        // MC_STAGING_SHARED or MC_STAGING_LANE
};
Tuned autotune_pick(const mc_network *net, const mc_burn_opts &o);

// Kernel attributes belong to a device. Per device, the largest value this
// thread has already raised an attribute to, so each (thread, device) sets it
// once and a second device on the same thread is not skipped.
struct DevAttrCache {
  static constexpr int kDevices = 64;
  int value[kDevices] = {};
  bool below(int dev, int v) const { return dev < 0 || dev >= kDevices || value[dev] < v; }
  void raise(int dev, int v) {
    if (dev >= 0 && dev < kDevices && value[dev] < v) value[dev] = v;
  }
};

// Launch the burn kernel of ODE-count bucket N (network n <= N) with matrix
// precision LT; defined in mc_launch.cuh, instantiated in mc_inst_<N>.cu.
template <int N, typename LT>
mc_status launch_one(const DNet &d, const Opts &o, const CellArgs &a, int variant, int threads,
                     int blocks_per_sm, int strag_steps, unsigned long long *next, cudaStream_t st);

// Library-owned retry-ladder lists of the current stream's scratch set: two
// lists of n cells each (lists, lists + n) and their two counts.
mc_status ladder_scratch(int dev, int64_t n, int32_t **lists, uint32_t **counts);

// Library-owned record buffer for straggler hand-off (grown on demand) and its
// claim counter, on the current device.
mc_status straggler_scratch(size_t bytes, void **rec, uint32_t **count);

// Library-owned cost-order buffers for n cells on device dev, scratch set of
// the current stream: the queue's cell list, one bucket byte per cell and the
// bucket histogram.
mc_status order_scratch(int dev, int64_t n, int32_t **index, uint8_t **bkt, uint32_t **hist);

// Write into index the cells 0..a.n_cells-1 ordered by decreasing cost key
// (mc_order.cu); four operations on stream st, no host synchronisation.
mc_status order_cells(const mc_network *net, const Opts &o, const CellArgs &a, int32_t *index, uint8_t *bkt,
                      uint32_t *hist, cudaStream_t st);

}  // namespace mc
