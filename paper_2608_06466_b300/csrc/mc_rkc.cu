// mc_rkc.cu -- the explicit Runge-Kutta-Chebyshev integrator (order 2, damped;
// Sommeijer, Shampine & Verwer, J. Comput. Appl. Math. 88, 315-326, 1998) on
// the same network interface as the BDF burn: the paper's microphysics keeps
// the integrator separate from the network and offers RKC beside VODE
// (Software design section, paragraphs 2 and 4). Here it serves as a rung of
// the retry ladder and as a method on its own: one thread per cell.
//
// With s stages and damping eps = 2/13: w0 = 1 + eps/s^2, T_j, T_j', T_j'' the
// Chebyshev values at w0 by their three-term recurrences, w1 = T_s'/T_s'',
// b_j = T_j''/T_j'^2 (j >= 2, b_0 = b_1 = b_2),
//   Y_0 = y_n, Y_1 = Y_0 + b_1 w1 h F(Y_0),
//   Y_j = (1 - mu_j - nu_j) Y_0 + mu_j Y_{j-1} + nu_j Y_{j-2} + mt_j h F(Y_{j-1})
//         + gt_j h F(Y_0),
//   mu_j = 2 b_j w0 / b_{j-1}, nu_j = -b_j / b_{j-2}, mt_j = 2 b_j w1 / b_{j-1},
//   gt_j = -(1 - b_{j-1} T_{j-1}) mt_j, y_{n+1} = Y_s,
// stable for h rho <= beta_s = (1 + w0)/w1. Step control (the paper gives
// none): the fewest stages whose interval covers h rho, rho the Gershgorin
// bound of the Jacobian at the step's start (the step shrinks beyond 256
// stages); the error estimate (12 (y_n - y_{n+1}) + 6 h (F_n + F_{n+1}))/15 in
// the WRMS norm with weights rtol max(|y_n|, |y_{n+1}|) + atol; the next step
// h min(10, max(0.1, 0.8 err^(-1/3))), at most h after a rejection.
#include <cmath>
#include <mutex>
#include <vector>

#include "mc_internal.h"
#include "mc_kernels.cuh"

using namespace mc;

namespace {

constexpr double RKC_EPS = 2.0 / 13.0;
constexpr int RKC_SMAX = 256;

// w0 and w1 of the s-stage method
__device__ __forceinline__ void rkc_w(int s, double &w0, double &w1) {
  w0 = 1.0 + RKC_EPS / ((double)s * s);
  double T0 = 1.0, T1 = w0, d0 = 0.0, d1 = 1.0, e0 = 0.0, e1 = 0.0;
  for (int j = 2; j <= s; ++j) {
    const double T2 = 2.0 * w0 * T1 - T0;
    const double d2 = 2.0 * T1 + 2.0 * w0 * d1 - d0;
    const double e2 = 4.0 * d1 + 2.0 * w0 * e1 - e0;
    T0 = T1; T1 = T2; d0 = d1; d1 = d2; e0 = e1; e1 = e2;
  }
  w1 = d1 / e1;
}

// One s-stage step of size h from y0 with F(y0) = f0 into ys; false when a
// stage's right-hand side cannot be evaluated. Counts the stages' f.
template <int N>
__device__ bool rkc_step(const DNet &net, const CellIn &c, int s, double h, const double *y0, const double *f0,
                         double *ys, int *st) {
  const int n = net.n;
  double w0, w1;
  rkc_w(s, w0, w1);
  // recurrences rolled forward with the stages: index j-2, j-1 and j
  double Tm2 = 1.0, Tm1 = w0, dm2 = 0.0, dm1 = 1.0, em2 = 0.0, em1 = 0.0;
  // b_2 (and so b_0 = b_1 = b_2) from T_2'', T_2'
  const double T2 = 2.0 * w0 * Tm1 - Tm2, d2 = 2.0 * Tm1 + 2.0 * w0 * dm1 - dm2, e2 = 4.0 * dm1 + 2.0 * w0 * em1 - em2;
  (void)T2;
  const double b2 = e2 / (d2 * d2);
  double bm2 = b2, bm1 = b2;  // b_{j-2}, b_{j-1} entering stage j = 2
  double ym2[N], ym1[N], F[N];
  const double c2 = w1 * e2 / d2;
  double cprev = c2 / d2;  // c_1 (stage times: the network is autonomous, kept for the record)
  (void)cprev;
#pragma unroll
  for (int i = 0; i < N; ++i) {
    ym2[i] = (i < n) ? y0[i] : 0.0;
    ym1[i] = (i < n) ? y0[i] + bm1 * w1 * h * f0[i] : 0.0;
  }
  for (int j = 2; j <= s; ++j) {
    // T_j, T_j', T_j'' and b_j
    const double Tj = 2.0 * w0 * Tm1 - Tm2;
    const double dj = 2.0 * Tm1 + 2.0 * w0 * dm1 - dm2;
    const double ej = 4.0 * dm1 + 2.0 * w0 * em1 - em2;
    const double bj = (j == 2) ? b2 : ej / (dj * dj);
    if (!net_rhs<N>(net, c, ym1, F)) return false;
    st[ST_RHS] += 1;
    const double mu = 2.0 * bj * w0 / bm1;
    const double nu = -bj / bm2;
    const double mt = 2.0 * bj * w1 / bm1;
    const double gt = -(1.0 - bm1 * Tm1) * mt;
#pragma unroll
    for (int i = 0; i < N; ++i)
      if (i < n) {
        const double v = (1.0 - mu - nu) * y0[i] + mu * ym1[i] + nu * ym2[i] + mt * h * F[i] + gt * h * f0[i];
        ym2[i] = ym1[i];
        ym1[i] = v;
      }
    Tm2 = Tm1; Tm1 = Tj; dm2 = dm1; dm1 = dj; em2 = em1; em1 = ej;
    bm2 = bm1;
    bm1 = bj;
  }
#pragma unroll
  for (int i = 0; i < N; ++i)
    if (i < n) ys[i] = ym1[i];
  return true;
}

template <int N>
__device__ __forceinline__ double rkc_wrms(int n, const double *v, const double *w) {
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < N; ++i)
    if (i < n) {
      const double r = v[i] / w[i];
      s += r * r;
    }
  return sqrt(s / n);
}

// Adaptive RKC over [0, tend] from y (in/out); returns a cell status.
template <int N>
__device__ int rkc_integrate(const DNet &net, const CellIn &c, const Opts &o, const double *beta, double tend,
                             double *y, int *st) {
  const int n = net.n;
  double f0[N], w[N], yn[N], fn[N], est[N];
  if (!net_rhs<N>(net, c, y, f0)) return CELL_BAD_INPUT;
  st[ST_RHS] += 1;
#pragma unroll
  for (int i = 0; i < N; ++i) w[i] = (i < n) ? o.rtol * fabs(y[i]) + o.atol : 1.0;
  // starting step (Hairer, Norsett & Wanner, Solving ODEs I, II.4), p = 1
  double h;
  {
    const double d0 = rkc_wrms<N>(n, y, w), d1 = rkc_wrms<N>(n, f0, w);
    double h0 = (d0 < 1e-5 || d1 < 1e-5) ? 1e-6 : 0.01 * d0 / d1;
    h0 = fmin(h0, tend);
    double y1[N], f1[N];
#pragma unroll
    for (int i = 0; i < N; ++i) y1[i] = (i < n) ? y[i] + h0 * f0[i] : 0.0;
    st[ST_RHS] += 1;
    if (!net_rhs<N>(net, c, y1, f1)) {
      h = h0;
    } else {
#pragma unroll
      for (int i = 0; i < N; ++i) f1[i] -= f0[i];
      const double d2 = rkc_wrms<N>(n, f1, w) / h0;
      const double dm = fmax(d1, d2);
      const double h1 = (dm <= 1e-15) ? fmax(1e-6, h0 * 1e-3) : sqrt(0.01 / dm);
      h = fmin(fmin(100.0 * h0, h1), tend);
    }
  }
  double t = 0.0;
  int attempts = 0;
  bool rejected = false;
  const double beta_max = beta[RKC_SMAX];
  double J[N * N];
  while (t < tend) {
    if (attempts >= o.max_steps) return CELL_MAX_STEPS;
    bool last = false;
    if (t + h >= tend) {
      h = tend - t;
      last = true;
    }
    const bool jok = o.jac_fd ? net_fd_jac<N>(net, c, y, J, o.rtol, o.atol) : net_jac<N>(net, c, y, J);
    if (!jok) return CELL_NONFINITE;
    st[ST_JAC] += 1;
    double rho = 0.0;  // Gershgorin: largest absolute row sum
    for (int i = 0; i < n; ++i) {
      double r = 0.0;
      for (int j = 0; j < n; ++j) r += fabs(J[i * N + j]);
      if (r > rho) rho = r;
    }
    if (h * rho > beta_max) {
      h = 0.95 * beta_max / rho;
      last = false;
    }
    int s = 2;
    while (s < RKC_SMAX && beta[s] < h * rho) ++s;
    if (s > st[ST_ORDER]) st[ST_ORDER] = s;
    attempts += 1;
    double err = 2.0;
    bool ok = rkc_step<N>(net, c, s, h, y, f0, yn, st);
    if (ok) ok = net_rhs<N>(net, c, yn, fn);
    if (ok) {
      st[ST_RHS] += 1;
#pragma unroll
      for (int i = 0; i < N; ++i)
        if (i < n) {
          est[i] = (12.0 * (y[i] - yn[i]) + 6.0 * h * (f0[i] + fn[i])) / 15.0;
          w[i] = o.rtol * fmax(fabs(y[i]), fabs(yn[i])) + o.atol;
        }
      err = rkc_wrms<N>(n, est, w);
    }
    if (ok && err <= 1.0) {
      t = last ? tend : t + h;
#pragma unroll
      for (int i = 0; i < N; ++i)
        if (i < n) {
          y[i] = yn[i];
          f0[i] = fn[i];
        }
      st[ST_STEPS] += 1;
      double fac = err > 0.0 ? 0.8 * pow(err, -1.0 / 3.0) : 10.0;
      fac = fmin(10.0, fmax(0.1, fac));
      if (rejected) fac = fmin(fac, 1.0);
      rejected = false;
      h *= fac;
    } else {
      st[ST_ERR_FAILS] += 1;
      rejected = true;
      const double fac = ok ? fmin(1.0, fmax(0.1, 0.8 * pow(err, -1.0 / 3.0))) : 0.25;
      h *= fac;
    }
    if (t < tend && t + h == t) return CELL_H_UNDERFLOW;
  }
  return CELL_OK;
}

template <int N>
__global__ void __launch_bounds__(128) k_burn_rkc(DNet net, Opts o, CellArgs a, const double *beta) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= count_of(a)) return;
  const int64_t c = cell_of(a, k);
  if (!MC_IN(a, BC_RKC_CELL, c, MC_CELLS(a))) return;
  const int S = net.S, n = net.n;
  // inputs, checked as load_cell checks them
  double y[N];
  bool good = true;
  double X = 0.0;
#pragma unroll
  for (int i = 0; i < N; ++i) {
    const double v = (i < S) ? a.x[i * a.ld + c] : 0.0;
    y[i] = v;
    if (i < S) {
      X += v;
      if (!isfinite(v)) good = false;
    }
  }
  CellIn cin;
  cin.nd = a.nd ? a.nd[c] : 1.0;
  const double T = a.T ? a.T[c] : 1.0;
  if (!(cin.nd > 0.0) || !isfinite(cin.nd) || !(T > 0.0) || !isfinite(T)) good = false;
  cin.ks = a.ks ? a.ks + c : nullptr;
  cin.ks_ld = a.ld;
  cin.src = a.src ? a.src + c : nullptr;
  cin.lnT = 0.0;
  cin.invT = 0.0;
  if (net.energy) {
    if (!(X > 0.0) || !isfinite(X)) good = false;
    if (S < N) y[S] = X * KB_EV * T / net.gm1;
  } else {
    cin.lnT = log(T);
    cin.invT = 1.0 / T;
  }
  int st[NSTAT];
#pragma unroll
  for (int q = 0; q < NSTAT; ++q) st[q] = 0;
  int status = good ? rkc_integrate<N>(net, cin, o, beta, a.dt, y, st) : CELL_BAD_INPUT;
  if (good && status == CELL_OK) {
    for (int i = 0; i < n; ++i)
      if (!isfinite(y[i])) status = CELL_NONFINITE;
  }
  const int route = route_of(a, status);
  if (route == 1) { push_list(a, a.retry, a.retry_count, c); return; }
  if (route == 2) { push_list(a, a.lretry, a.lretry_count, c); return; }
  MC_STORED(a, c);
  if (good) {
    double Xo = 0.0;
    for (int i = 0; i < S; ++i) {
      a.x[i * a.ld + c] = y[i];
      Xo += y[i];
    }
    if (net.energy) a.T[c] = net.gm1 * y[S] / (KB_EV * Xo);
  }
  if (a.rung) a.rung[c] = a.rung_id;
  a.status[c] = status;
  if (a.stats)
    for (int q = 0; q < NSTAT; ++q) a.stats[q * a.ld + c] = st[q];
}

// beta_s = (1 + w0)/w1 for s = 0..RKC_SMAX (entries 0, 1 unused), computed on
// the host by the same recurrences, uploaded once per device.
std::mutex g_beta_mu;
double *g_beta[64] = {};

mc_status beta_table(int dev, double **out) {
  std::lock_guard<std::mutex> lk(g_beta_mu);
  if (dev < 0 || dev >= 64) return set_error(MC_E_INVALID, "device %d out of range", dev);
  if (!g_beta[dev]) {
    std::vector<double> b(RKC_SMAX + 1, 0.0);
    for (int s = 2; s <= RKC_SMAX; ++s) {
      const double w0 = 1.0 + RKC_EPS / ((double)s * s);
      double T0 = 1.0, T1 = w0, d0 = 0.0, d1 = 1.0, e0 = 0.0, e1 = 0.0;
      for (int j = 2; j <= s; ++j) {
        const double T2 = 2.0 * w0 * T1 - T0;
        const double d2 = 2.0 * T1 + 2.0 * w0 * d1 - d0;
        const double e2 = 4.0 * d1 + 2.0 * w0 * e1 - e0;
        T0 = T1; T1 = T2; d0 = d1; d1 = d2; e0 = e1; e1 = e2;
      }
      b[s] = (1.0 + w0) / (d1 / e1);
    }
    void *p = nullptr;
    cudaError_t e = dev_malloc(&p, sizeof(double) * b.size());
    if (e == cudaSuccess) e = cudaMemcpy(p, b.data(), sizeof(double) * b.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      cudaFree(p);
      return cuda_error(e, "RKC coefficient table");
    }
    g_beta[dev] = (double *)p;
  }
  *out = g_beta[dev];
  return MC_OK;
}

template <int N>
void launch_rkc(const DNet &d, const Opts &o, const CellArgs &a, const double *beta, cudaStream_t st) {
  // a list-driven launch (device count) covers the list's upper bound
  const int64_t blocks = (a.n_cells + 127) / 128;
  k_burn_rkc<N><<<(unsigned)blocks, 128, 0, st>>>(d, o, a, beta);
}

}  // namespace

mc_status mc::burn_rkc_device(const mc_network *net, const mc_burn_opts &ob, const CellArgs &a0, cudaStream_t st) {
  if (a0.n_cells <= 0) return MC_OK;
  CellArgs a = a0;
  bc_attach(a);
  int dev = 0;
  cudaGetDevice(&dev);
  double *beta;
  mc_status s = beta_table(dev, &beta);
  if (s != MC_OK) return s;
  const DNet d = dnet_of(net);
  const Opts o{ob.rtol, ob.atol, ob.max_order, ob.max_steps, ob.jacobian == MC_JAC_FD ? 1 : 0};
  if (net->n <= 3) launch_rkc<3>(d, o, a, beta, st);
  else if (net->n <= 13) launch_rkc<13>(d, o, a, beta, st);
  else if (net->n <= 33) launch_rkc<33>(d, o, a, beta, st);
  else launch_rkc<NMAX_ODE>(d, o, a, beta, st);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_error(e, "RKC launch");
  count_launch(1);
  return MC_OK;
}
