// mc_eval.cu -- pointwise evaluation of a network on the device with the same
// device functions the burn uses: rate coefficients at given temperatures, and
// the right-hand side (and Jacobian) at given states.
#include <cmath>

#include "mc_internal.h"
#include "mc_kernels.cuh"

using namespace mc;

namespace {

__global__ void k_rates(DNet net, int64_t n, const double *T, double *kf, double *kr, int64_t ld) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= n) return;
  const double t = T[c];
  const double lnT = log(t), invT = 1.0 / t;
  for (int r = 0; r < net.R; ++r) {
    const RxPar &p = net.par[r];
    kf[r * ld + c] = rexp(__ldg(&p.lnAf) + __ldg(&p.bf) * lnT - __ldg(&p.Cf) * invT, net.exptab);
    kr[r * ld + c] = (__ldg(&p.rev) != 0.0)
                         ? rexp(__ldg(&p.lnAr) + __ldg(&p.br) * lnT - __ldg(&p.Cr) * invT, net.exptab)
                         : 0.0;
  }
}

template <int N>
__global__ void k_rhs(DNet net, int64_t n, const double *y, int64_t ld, const double *T, const double *nd,
                      const double *ks, double *f, int32_t *ok) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= n) return;
  double yl[N], fl[N];
  for (int i = 0; i < N; ++i) yl[i] = (i < net.n) ? y[i * ld + c] : 0.0;
  CellIn ci;
  ci.nd = nd ? nd[c] : 1.0;
  const double t = T ? T[c] : 1.0;
  ci.lnT = log(t);
  ci.invT = 1.0 / t;
  ci.ks = ks ? ks + c : nullptr;
  ci.ks_ld = ld;
  ci.src = nullptr;
  const bool good = net_rhs<N>(net, ci, yl, fl);
  for (int i = 0; i < net.n; ++i) f[i * ld + c] = fl[i];
  ok[c] = good ? 1 : 0;
}

// The analytic Jacobian as the burn evaluates it: one warp per state, with
// the warp-cooperative routine of the persistent workers (w_jac). ok[c] is
// cleared where the Jacobian is not finite.
template <int N>
__global__ void __launch_bounds__(128) k_jac(DNet net, int64_t n, const double *y, int64_t ld, const double *T,
                                             const double *nd, const double *ks, double *jac, int32_t *ok,
                                             int smem_per_warp) {
  extern __shared__ __align__(16) unsigned char smem[];
  const WSh<double> sh = wsh_carve<N, double>(smem + (threadIdx.x >> 5) * (size_t)smem_per_warp, net.R);
  const int64_t c = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  if (c >= n) return;
  const int ln = wlane();
  for (int i = ln; i < net.n; i += 32) sh.yb[i] = y[i * ld + c];
  CellIn ci;
  ci.nd = nd ? nd[c] : 1.0;
  const double t = T ? T[c] : 1.0;
  ci.lnT = log(t);
  ci.invT = 1.0 / t;
  ci.ks = ks ? ks + c : nullptr;
  ci.ks_ld = ld;
  ci.src = nullptr;
  __syncwarp();
  const bool good = w_jac<N, double>(net, ci, sh);
  for (int idx = ln; idx < net.n * net.n; idx += 32) {
    const int i = idx / net.n, j = idx - i * net.n;
    jac[idx * ld + c] = good ? sh.J[i * N + j] : 0.0;
  }
  if (ln == 0 && !good) ok[c] = 0;
}

template <int N>
mc_status launch_rhs(const DNet &d, int64_t n, const double *y, int64_t ld, const double *T, const double *nd,
                     const double *ks, double *f, double *jac, int32_t *ok, cudaStream_t st) {
  k_rhs<N><<<(unsigned)((n + 63) / 64), 64, 0, st>>>(d, n, y, ld, T, nd, ks, f, ok);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_error(e, "rhs kernel");
  count_launch(1);
  if (!jac) return MC_OK;
  const int per_warp = (int)wsh_bytes<N, double>(d.R);
  const int smem = per_warp * 4;
  e = cudaFuncSetAttribute(k_jac<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return cuda_error(e, "jacobian kernel smem attribute");
  k_jac<N><<<(unsigned)((n + 3) / 4), 128, smem, st>>>(d, n, y, ld, T, nd, ks, jac, ok, per_warp);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_error(e, "jacobian kernel");
  count_launch(1);
  return MC_OK;
}

}  // namespace

extern "C" mc_status mc_network_rates(const mc_network *net, int64_t n, const double *T, double *kf, double *kr,
                                      int64_t ld, void *stream) {
  if (!net || n < 0 || ld < n || (n > 0 && (!T || !kf || !kr)))
    return set_error(MC_E_INVALID, "mc_network_rates: bad arguments");
  if (n == 0 || net->R == 0) return MC_OK;
  k_rates<<<(unsigned)((n + 127) / 128), 128, 0, (cudaStream_t)stream>>>(dnet_of(net), n, T, kf, kr, ld);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_error(e, "rates kernel");
  count_launch(1);
  return MC_OK;
}

extern "C" mc_status mc_network_rhs(const mc_network *net, int64_t n, const double *y, int64_t ld,
                                    const double *T, const double *ndens, const double *rate_scale, double *f,
                                    double *jac, int32_t *ok, void *stream) {
  if (!net || n < 0 || ld < n || (n > 0 && (!y || !f || !ok)))
    return set_error(MC_E_INVALID, "mc_network_rhs: bad arguments");
  if (n == 0) return MC_OK;
  const DNet d = dnet_of(net);
  cudaStream_t st = (cudaStream_t)stream;
  if (net->n <= 3) return launch_rhs<3>(d, n, y, ld, T, ndens, rate_scale, f, jac, ok, st);
  if (net->n <= 13) return launch_rhs<13>(d, n, y, ld, T, ndens, rate_scale, f, jac, ok, st);
  if (net->n <= 33) return launch_rhs<33>(d, n, y, ld, T, ndens, rate_scale, f, jac, ok, st);
  return launch_rhs<NMAX_ODE>(d, n, y, ld, T, ndens, rate_scale, f, jac, ok, st);
}
