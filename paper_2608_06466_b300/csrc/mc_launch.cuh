// mc_launch.cuh -- launch of the burn kernels for one compiled ODE-count
// bucket N and matrix precision LT; instantiated once per bucket in
// mc_inst_<N>.cu so the buckets compile in parallel.
#pragma once

#include <algorithm>

#include "mc_internal.h"
#include "mc_warp.cuh"

namespace mc {

template <int N, typename LT>
mc_status launch_one(const DNet &d, const Opts &o, const CellArgs &a, int variant, int threads,
                     int blocks_per_sm, int strag_steps, unsigned long long *next, cudaStream_t st) {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaError_t e;
  if (variant == MC_VARIANT_WARP) {
    e = cudaMemsetAsync(next, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return cuda_error(e, "queue reset");
    const int per_warp = (int)wsh_bytes<N, LT>(d.R);
    const int wthreads = 128;
    const int smem = per_warp * (wthreads / 32);
    static thread_local int configured_w = 0;
    if (configured_w < smem) {
      e = cudaFuncSetAttribute(k_burn_warp<N, LT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
      if (e != cudaSuccess) return cuda_error(e, "warp kernel smem attribute");
      configured_w = smem;
    }
    int64_t blocks = (int64_t)sms * std::max(1, blocks_per_sm) * 2;
    const int64_t need = a.n_dev ? blocks : (a.n_cells + 3) / 4;
    blocks = std::max<int64_t>(1, std::min(blocks, need));
    k_burn_warp<N, LT><<<(unsigned)blocks, wthreads, smem, st>>>(d, o, a, next, per_warp);
  } else if (variant == MC_VARIANT_PLAIN) {
    if (a.n_cells <= 0) return MC_OK;
    const int64_t blocks = (a.n_cells + threads - 1) / threads;
    k_burn_plain<N, LT><<<(unsigned)blocks, threads, 0, st>>>(d, o, a);
  } else {
    e = cudaMemsetAsync(next, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return cuda_error(e, "queue reset");
    int64_t blocks = (int64_t)sms * blocks_per_sm;
    if (!a.n_dev) blocks = std::min<int64_t>(blocks, (a.n_cells + threads - 1) / threads);
    if (blocks < 1) blocks = 1;
    StragArgs sa{nullptr, nullptr, 0u, 0};
    // record list: room for every cell that may pass the threshold (a lane that
    // finds it full keeps its cell), bounded to 2 GB of records
    const int64_t rec_max = (int64_t)((2ull << 30) / sizeof(Lane<N, LT>));
    const int64_t ncap = a.n_dev ? 0 : std::min<int64_t>(rec_max, std::max<int64_t>(256, a.n_cells / 8));
    if (strag_steps > 0 && ncap > 0 && strag_steps < o.max_steps) {
      void *rec = nullptr;
      uint32_t *cnt = nullptr;
      mc_status s = straggler_scratch(sizeof(Lane<N, LT>) * (size_t)ncap, &rec, &cnt);
      if (s != MC_OK) return s;
      sa = StragArgs{rec, cnt, (uint32_t)ncap, strag_steps};
      e = cudaMemsetAsync(cnt, 0, sizeof(uint32_t), st);
      if (e != cudaSuccess) return cuda_error(e, "straggler counter reset");
    }
    k_burn_persistent<N, LT><<<(unsigned)blocks, threads, 0, st>>>(d, o, a, next, sa);
    if (sa.rec) {
      e = cudaGetLastError();
      if (e != cudaSuccess) return cuda_error(e, "burn kernel launch");
      count_launch(1);
      // warp-cooperative pass over the handed-off cells (count read on the device)
      // one-warp blocks, 16 per SM: four warps per SM sub-partition hide the
      // latency of each warp's dependent step logic
      const int per_warp = (int)wsh_bytes<N, LT>(d.R);
      const int wthreads = 32;
      const int smem = per_warp;
      static thread_local int configured = 0;
      if (configured < smem) {
        e = cudaFuncSetAttribute(k_burn_straggler<N, LT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return cuda_error(e, "straggler smem attribute");
        configured = smem;
      }
      e = cudaMemsetAsync(next + 1, 0, sizeof(unsigned long long), st);
      if (e != cudaSuccess) return cuda_error(e, "straggler queue reset");
      const int wblocks = std::max(1, std::min(sms * 16, (int)sa.cap));
      k_burn_straggler<N, LT><<<wblocks, wthreads, smem, st>>>(d, o, a, (const Lane<N, LT> *)sa.rec, sa.count,
                                                              sa.cap, next + 1, per_warp);
    }
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_error(e, "burn kernel launch");
  count_launch(1);
  return MC_OK;
}

}  // namespace mc
