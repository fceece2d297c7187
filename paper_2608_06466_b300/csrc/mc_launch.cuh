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
    int smem_max = 0;
    e = cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return cuda_error(e, "shared memory limit");
    // four warps a block unless their workspaces exceed a block's shared memory
    const int wthreads = std::max(32, std::min(128, 32 * (smem_max / per_warp)));
    const int smem = per_warp * (wthreads / 32);
    static thread_local DevAttrCache configured_w;
    if (configured_w.below(dev, smem)) {
      e = cudaFuncSetAttribute(k_burn_warp<N, LT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
      if (e != cudaSuccess) return cuda_error(e, "warp kernel smem attribute");
      configured_w.raise(dev, smem);
    }
    int64_t blocks = (int64_t)sms * std::max(1, blocks_per_sm) * 2 * (128 / wthreads);
    const int64_t need = a.n_dev ? blocks : (a.n_cells + wthreads / 32 - 1) / (wthreads / 32);
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
    StragArgs sa{nullptr, nullptr, 0u, 0, nullptr};
    // record list: room for every cell that may pass the threshold (a lane that
    // finds it full keeps its cell), bounded to 2 GB of records; a flag per
    // record follows the records
    const int64_t rec_max = (int64_t)((2ull << 30) / sizeof(Lane<N, LT>));
    const int64_t ncap = a.n_dev ? 0 : std::min<int64_t>(rec_max, std::max<int64_t>(256, a.n_cells / 8));
    if (strag_steps > 0 && ncap > 0 && strag_steps < o.max_steps) {
      void *rec = nullptr;
      uint32_t *cnt = nullptr;
      const size_t rbytes = (sizeof(Lane<N, LT>) * (size_t)ncap + 255) & ~(size_t)255;
      mc_status s = straggler_scratch(rbytes + sizeof(uint32_t) * (size_t)ncap, &rec, &cnt);
      if (s != MC_OK) return s;
      sa = StragArgs{rec, cnt, (uint32_t)ncap, strag_steps, (uint32_t *)((char *)rec + rbytes)};
      // cnt[0] records, cnt[1] fused claims, cnt[2] finished bulk warps
      e = cudaMemsetAsync(cnt, 0, 4 * sizeof(uint32_t), st);
      if (e == cudaSuccess) e = cudaMemsetAsync(sa.flag, 0, sizeof(uint32_t) * (size_t)ncap, st);
      if (e != cudaSuccess) return cuda_error(e, "straggler list reset");
    }
    // warp workspace of the cooperative matrix work; blocks shrink if the
    // workspaces of a full block would not fit the shared memory of a block
    const int per_warp_p = (int)wsh_bytes<N, LT>(d.R);
    int smem_max = 0;
    e = cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return cuda_error(e, "shared memory limit");
    const int pthreads = std::max(32, std::min(threads, 32 * (smem_max / per_warp_p)));
    const int psmem = per_warp_p * (pthreads / 32);
    static thread_local DevAttrCache configured_p;
    if (configured_p.below(dev, psmem)) {
      e = cudaFuncSetAttribute(k_burn_persistent<N, LT>, cudaFuncAttributeMaxDynamicSharedMemorySize, psmem);
      if (e != cudaSuccess) return cuda_error(e, "persistent kernel smem attribute");
      configured_p.raise(dev, psmem);
    }
    if (pthreads != threads) {
      blocks = (int64_t)sms * blocks_per_sm * (threads / pthreads);
      if (!a.n_dev) blocks = std::min<int64_t>(blocks, (a.n_cells + pthreads - 1) / pthreads);
      if (blocks < 1) blocks = 1;
    }
    if (!sa.rec) {
      k_burn_persistent<N, LT><<<(unsigned)blocks, pthreads, psmem, st>>>(d, o, a, next, sa, per_warp_p);
    } else {
      const int per_warp = (int)wsh_bytes<N, LT>(d.R);
      bool fused = false;
      if (threads == 128) {
        // one cooperative launch (every block resident): warps whose queue is
        // drained integrate the records while the rest of the bulk still runs
        const int fsmem = per_warp * 4;
        const int fsmem_sm = fsmem * std::max(1, blocks_per_sm);
        static thread_local DevAttrCache configured_f, carveout_f;
        e = cudaSuccess;
        if (configured_f.below(dev, fsmem) || carveout_f.below(dev, fsmem_sm)) {
          e = cudaFuncSetAttribute(k_burn_fused<N, LT>, cudaFuncAttributeMaxDynamicSharedMemorySize, fsmem);
          // shared-memory carveout just large enough for the resident blocks: the
          // rest stays L1, which caches the thread-form lanes' spilled state
          int smem_sm = 0;
          if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
          if (e == cudaSuccess && smem_sm > 0) {
            const int pct = std::min(100, (int)((100LL * fsmem_sm + smem_sm - 1) / smem_sm) + 1);
            e = cudaFuncSetAttribute(k_burn_fused<N, LT>, cudaFuncAttributePreferredSharedMemoryCarveout, pct);
          }
          if (e == cudaSuccess) {
            configured_f.raise(dev, fsmem);
            carveout_f.raise(dev, fsmem_sm);
          }
        }
        int per_sm = 0;
        if (e == cudaSuccess)
          e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_burn_fused<N, LT>, 128, fsmem);
        if (e != cudaSuccess) return cuda_error(e, "fused kernel set-up");
        if ((int64_t)per_sm * sms >= blocks) {
          DNet dd = d;
          Opts oo = o;
          CellArgs aa = a;
          unsigned long long *nx = next;
          FuseArgs fa{sa.count + 1, sa.count + 2, (uint32_t)(blocks * 4)};
          int pw = per_warp;
          void *args[] = {&dd, &oo, &aa, &nx, &sa, &fa, &pw};
          e = cudaLaunchCooperativeKernel((const void *)k_burn_fused<N, LT>, dim3((unsigned)blocks), dim3(128), args,
                                          (size_t)fsmem, st);
          if (e != cudaSuccess) return cuda_error(e, "fused burn launch");
          fused = true;
        }
      }
      if (!fused)
        k_burn_persistent<N, LT><<<(unsigned)blocks, pthreads, psmem, st>>>(d, o, a, next, sa, per_warp_p);
      e = cudaGetLastError();
      if (e != cudaSuccess) return cuda_error(e, "burn kernel launch");
      count_launch(1);
      // warp-cooperative pass over the handed-off cells not yet integrated
      // (count and flags read on the device); one-warp blocks, 16 per SM: four
      // warps per SM sub-partition hide the latency of each warp's dependent
      // step logic
      const int wthreads = 32;
      const int smem = per_warp;
      static thread_local DevAttrCache configured;
      if (configured.below(dev, smem)) {
        e = cudaFuncSetAttribute(k_burn_straggler<N, LT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return cuda_error(e, "straggler smem attribute");
        configured.raise(dev, smem);
      }
      e = cudaMemsetAsync(next + 1, 0, sizeof(unsigned long long), st);
      if (e != cudaSuccess) return cuda_error(e, "straggler queue reset");
      const int wblocks = std::max(1, std::min(sms * 16, (int)sa.cap));
      k_burn_straggler<N, LT><<<wblocks, wthreads, smem, st>>>(d, o, a, (const Lane<N, LT> *)sa.rec, sa.count,
                                                              sa.cap, sa.flag, next + 1, per_warp);
    }
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_error(e, "burn kernel launch");
  count_launch(1);
  return MC_OK;
}

}  // namespace mc
