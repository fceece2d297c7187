// mc_order.cu -- cost order of the persistent cell queue: per-cell key and
// bucket histogram (k_order_key, mc_kernels.cuh), an exclusive scan of the
// buckets, and a scatter that writes the queue's cell list, expensive first.
#include <algorithm>

#include "mc_internal.h"
#include "mc_kernels.cuh"

using namespace mc;

namespace {

// Exclusive prefix of the bucket counts, in place (256 entries: one thread).
__global__ void k_order_scan(uint32_t *hist) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  uint32_t s = 0;
  for (int b = 0; b < ORDER_BUCKETS; ++b) {
    const uint32_t v = hist[b];
    hist[b] = s;
    s += v;
  }
}

// Each block places the cells of its chunk: one reservation per (block,
// bucket) in offs, then positions inside the reserved range.
__global__ void __launch_bounds__(256) k_order_scatter(const uint8_t *bkt, int64_t n, uint32_t *offs,
                                                       int32_t *index) {
  __shared__ uint32_t cnt[ORDER_BUCKETS], base[ORDER_BUCKETS];
  const int64_t c0 = (int64_t)blockIdx.x * ORDER_CHUNK;
  const int64_t c1 = (c0 + ORDER_CHUNK < n) ? c0 + ORDER_CHUNK : n;
  for (int i = threadIdx.x; i < ORDER_BUCKETS; i += blockDim.x) cnt[i] = 0;
  __syncthreads();
  for (int64_t c = c0 + threadIdx.x; c < c1; c += blockDim.x) atomicAdd(&cnt[bkt[c]], 1u);
  __syncthreads();
  for (int i = threadIdx.x; i < ORDER_BUCKETS; i += blockDim.x) {
    base[i] = cnt[i] ? atomicAdd(&offs[i], cnt[i]) : 0u;
    cnt[i] = 0;
  }
  __syncthreads();
  for (int64_t c = c0 + threadIdx.x; c < c1; c += blockDim.x) {
    const int b = bkt[c];
    index[base[b] + atomicAdd(&cnt[b], 1u)] = (int32_t)c;
  }
}

template <int N>
void launch_key(const DNet &d, const Opts &o, const CellArgs &a, uint8_t *bkt, uint32_t *hist, int sms,
                cudaStream_t st) {
  const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((a.n_cells + 255) / 256, (int64_t)sms * 8));
  k_order_key<N><<<(unsigned)blocks, 256, 0, st>>>(d, o, a, bkt, hist);
}

}  // namespace

mc_status mc::order_cells(const mc_network *net, const Opts &o, const CellArgs &a, int32_t *index, uint8_t *bkt,
                          uint32_t *hist, cudaStream_t st) {
  if (a.n_cells <= 0) return MC_OK;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaError_t e = cudaMemsetAsync(hist, 0, sizeof(uint32_t) * ORDER_BUCKETS, st);
  if (e != cudaSuccess) return cuda_error(e, "order histogram reset");
  const DNet d = dnet_of(net);
  const int n = net->n;
  if (n <= 3) launch_key<3>(d, o, a, bkt, hist, sms, st);
  else if (n <= 8) launch_key<8>(d, o, a, bkt, hist, sms, st);
  else if (n <= 13) launch_key<13>(d, o, a, bkt, hist, sms, st);
  else if (n <= 16) launch_key<16>(d, o, a, bkt, hist, sms, st);
  else if (n <= 24) launch_key<24>(d, o, a, bkt, hist, sms, st);
  else if (n <= 33) launch_key<33>(d, o, a, bkt, hist, sms, st);
  else launch_key<NMAX_ODE>(d, o, a, bkt, hist, sms, st);
  k_order_scan<<<1, 32, 0, st>>>(hist);
  k_order_scatter<<<(unsigned)((a.n_cells + ORDER_CHUNK - 1) / ORDER_CHUNK), 256, 0, st>>>(bkt, a.n_cells, hist,
                                                                                          index);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_error(e, "order kernels");
  count_launch(3);
  return MC_OK;
}
