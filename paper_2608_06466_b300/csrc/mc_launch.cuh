// mc_launch.cuh -- launch of the burn kernels for one compiled ODE-count
// bucket N and matrix precision LT; instantiated once per bucket in
// mc_inst_<N>.cu so the buckets compile in parallel.
#pragma once

#include <algorithm>

#include "mc_internal.h"
#include "mc_kernels.cuh"

namespace mc {

template <int N, typename LT>
mc_status launch_one(const DNet &d, const Opts &o, const CellArgs &a, int variant, int threads,
                     int blocks_per_sm, unsigned long long *next, cudaStream_t st) {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaError_t e;
  if (variant == MC_VARIANT_PLAIN) {
    if (a.n_cells <= 0) return MC_OK;
    const int64_t blocks = (a.n_cells + threads - 1) / threads;
    k_burn_plain<N, LT><<<(unsigned)blocks, threads, 0, st>>>(d, o, a);
  } else {
    e = cudaMemsetAsync(next, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return cuda_error(e, "queue reset");
    int64_t blocks = (int64_t)sms * blocks_per_sm;
    if (!a.n_dev) blocks = std::min<int64_t>(blocks, (a.n_cells + threads - 1) / threads);
    if (blocks < 1) blocks = 1;
    k_burn_persistent<N, LT><<<(unsigned)blocks, threads, 0, st>>>(d, o, a, next);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_error(e, "burn kernel launch");
  count_launch(1);
  return MC_OK;
}

}  // namespace mc
