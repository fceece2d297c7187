// mc_warp.cuh -- warp-cooperative form of the same integrator, for cells that
// need far more steps than the rest (stragglers).
//
// On this GPU an FP64 warp instruction occupies the FP64 pipe for the whole
// warp whether 1 or 32 lanes are active, so a long cell left alone on one lane
// pays full-warp price for every operation of every step. Here the whole warp
// advances ONE cell: vector components live one per lane (component i on lane
// i mod 32, slot i / 32), the reaction rates of a right-hand side are spread
// over the lanes, per-species sums follow the network's occurrence lists, the
// iteration matrix sits in shared memory and is factored row-parallel, and
// scalars are replicated so every lane takes the same branch. The decisions
// are the thread form's (same rules, same constants); only the order of a few
// floating-point reductions differs.
#pragma once

#include "mc_kernels.cuh"

namespace mc {

// register state of the warp's cell (vector slots: component lane + 32 s)
template <int N>
struct WState {
  static constexpr int NS = WSlots<N>::NS;
  double z[QMAX + 2][NS];
  double e[NS], es[NS], iw[NS], y[NS], f[NS];
  double l[QMAX + 1];
  double hist[QMAX + 3];
  double t, h, tend, crate, gamma_p, gamma, cq, esave_h, delp, eta_max, h0;
  CellIn cin;
  int64_t cell;
  int q, qwait, nef, ncf, jage, page, attempts, m, phase, status;
  bool need_j, need_p, jcur, have_es, last;
  bool p64;  // FP32-matrix cell now factoring in FP64 (w_switches)
  int st[NSTAT];
};

// value of distributed component c (all lanes receive it)
template <int NS>
__device__ __forceinline__ double wget(const double (&v)[NS], int c) {
  double x = v[0];
  if (NS > 1 && c >= 32) x = v[NS - 1];
  return __shfl_sync(WFULL, x, c & 31);
}

template <int N>
__device__ __forceinline__ double w_wrms(int n, const double (&v)[WState<N>::NS], const double (&iw)[WState<N>::NS]) {
  constexpr int NS = WState<N>::NS;
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < NS; ++k) {
    const int i = wlane() + 32 * k;
    if (i < n) {
      const double r = v[k] * iw[k];
      s += r * r;
    }
  }
  return sqrt(wsum(s) / n);
}

template <int N, typename LT>
__device__ __forceinline__ void w_load(WState<N> &W, const Lane<N, LT> &L, const WSh<LT> &sh, const DNet &net) {
  constexpr int NS = WState<N>::NS;
  const int n = net.n, ln = wlane();
#pragma unroll
  for (int k = 0; k < NS; ++k) {
    const int i = ln + 32 * k;
    const bool in = i < n;
    for (int j = 0; j < QMAX + 1; ++j) W.z[j][k] = in ? L.z[j][in ? i : 0] : 0.0;
    W.z[QMAX + 1][k] = 0.0;
    W.e[k] = in ? L.e[in ? i : 0] : 0.0;
    W.es[k] = in ? L.es[in ? i : 0] : 0.0;
    W.iw[k] = in ? L.iw[in ? i : 0] : 0.0;
    W.y[k] = in ? L.y[in ? i : 0] : 0.0;
    W.f[k] = 0.0;
  }
  for (int idx = ln; idx < n * N; idx += 32) {
    sh.J[idx] = L.J[idx];
    sh.P[idx] = L.P[idx];
  }
  for (int i = ln; i < n; i += 32) sh.piv[i] = L.piv[i];
  for (int k = 0; k <= QMAX; ++k) W.l[k] = L.l[k];
  for (int k = 0; k < QMAX + 3; ++k) W.hist[k] = L.hist[k];
  W.t = L.t; W.h = L.h; W.tend = L.tend; W.crate = L.crate; W.gamma_p = L.gamma_p; W.gamma = L.gamma;
  W.cq = L.cq; W.esave_h = L.esave_h; W.delp = L.delp; W.eta_max = L.eta_max; W.h0 = L.h0;
  W.cin = L.cin; W.cell = L.cell;
  W.q = L.q; W.qwait = L.qwait; W.nef = L.nef; W.ncf = L.ncf; W.jage = L.jage; W.page = L.page;
  W.attempts = L.attempts; W.m = L.m; W.phase = L.phase; W.status = L.status;
  W.need_j = L.need_j; W.need_p = L.need_p; W.jcur = L.jcur; W.have_es = L.have_es; W.last = L.last;
  W.p64 = false;
  for (int k = 0; k < NSTAT; ++k) W.st[k] = L.st[k];
  __syncwarp();
}

// Load cell c straight from the cell arrays (warp form of load_cell): same
// input checks; sets PH_F0, or PH_DONE with CELL_BAD_INPUT (m = -1: outputs are
// then left untouched).
template <int N>
__device__ __forceinline__ void w_load_cell(WState<N> &W, const DNet &net, const CellArgs &a, int64_t c) {
  constexpr int NS = WState<N>::NS;
  const int S = net.S, n = net.n, ln = wlane();
  W.cell = c;
  W.status = CELL_OK;
  W.q = 0;
  W.p64 = false;
  for (int k = 0; k < NSTAT; ++k) W.st[k] = 0;
  if (!MC_IN(a, BC_WARP_LOAD, c, MC_CELLS(a))) {
    W.status = CELL_BAD_INPUT;
    W.phase = PH_DONE;
    W.m = -1;
    return;
  }
  bool bad = false;
  double xs = 0.0;
#pragma unroll
  for (int k = 0; k < NS; ++k) {
    const int i = ln + 32 * k;
    const double v = (i < S) ? a.x[i * a.ld + c] : 0.0;
#pragma unroll
    for (int j = 0; j < QMAX + 2; ++j) W.z[j][k] = 0.0;
    W.z[0][k] = v;
    W.e[k] = 0.0;
    W.es[k] = 0.0;
    W.f[k] = 0.0;
    if (i < S) {
      xs += v;
      if (!isfinite(v)) bad = true;
    }
  }
  const double X = wsum(xs);
  const double nd = a.nd ? a.nd[c] : 1.0;
  const double T = a.T ? a.T[c] : 1.0;
  bool good = !__any_sync(WFULL, bad) && nd > 0.0 && isfinite(nd) && T > 0.0 && isfinite(T);
  W.cin.nd = nd;
  W.cin.ks = a.ks ? a.ks + c : nullptr;
  W.cin.ks_ld = a.ld;
  W.cin.src = a.src ? a.src + c : nullptr;
  if (net.energy) {
    if (!(X > 0.0) || !isfinite(X)) good = false;
    const double u = X * KB_EV * T / net.gm1;
#pragma unroll
    for (int k = 0; k < NS; ++k)
      if (ln + 32 * k == S) W.z[0][k] = u;
    W.cin.lnT = 0.0;
    W.cin.invT = 0.0;
  } else {
    W.cin.lnT = log(T);
    W.cin.invT = 1.0 / T;
  }
  if (!good) {
    W.status = CELL_BAD_INPUT;
    W.phase = PH_DONE;
    W.m = -1;
    return;
  }
  W.m = 0;
  W.tend = a.dt;
#pragma unroll
  for (int k = 0; k < NS; ++k) W.y[k] = (ln + 32 * k < n) ? W.z[0][k] : 0.0;
  W.phase = PH_F0;
}

// Right-hand side at W.y into W.f; returns false (uniformly) when it cannot be evaluated.
template <int N, typename LT>
__device__ __forceinline__ bool w_rhs(WState<N> &W, const WSh<LT> &sh, const DNet &net) {
  constexpr int NS = WState<N>::NS;
  const int n = net.n, ln = wlane();
#pragma unroll
  for (int k = 0; k < NS; ++k) {
    const int i = ln + 32 * k;
    if (i < n) sh.yb[i] = W.y[k];
  }
  __syncwarp();
  return w_rhs_core<N, LT>(net, W.cin, sh, W.f);
}

// x = (LU)^-1 b for the distributed vector b (FP64 in), in precision LT.
template <int N, typename LT>
__device__ __forceinline__ void w_apply(const WSh<LT> &sh, int n, const double (&bd)[WState<N>::NS],
                                        LT (&b)[WState<N>::NS]) {
  constexpr int NS = WState<N>::NS;
  const int ln = wlane();
#pragma unroll
  for (int k = 0; k < NS; ++k) b[k] = (LT)bd[k];
  auto get = [&](int c) -> LT {
    LT x = b[0];
    if (NS > 1 && c >= 32) x = b[NS - 1];
    return __shfl_sync(WFULL, x, c & 31);
  };
  auto put = [&](int c, LT v) {
    if ((c & 31) == ln) {
      if (NS > 1 && c >= 32) b[NS - 1] = v;
      else b[0] = v;
    }
  };
  for (int k = 0; k < n; ++k) {
    const int p = sh.piv[k];
    if (p != k) {
      const LT vk = get(k), vp = get(p);
      put(k, vp);
      put(p, vk);
    }
  }
  for (int j = 0; j < n; ++j) {
    const LT bj = get(j);
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      const int i = ln + 32 * k;
      if (i > j && i < n) b[k] -= sh.P[i * N + j] * bj;
    }
  }
  for (int j = n - 1; j >= 0; --j) {
    LT bj = get(j);
    bj = bj * sh.P[j * N + j];
    put(j, bj);
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      const int i = ln + 32 * k;
      if (i < j) b[k] -= sh.P[i * N + j] * bj;
    }
  }
}

// Newton correction d <- (I - gamma_P J)^-1 d for the distributed d: the
// thread form's newton_solve (FP64 factors: one solve; FP32 factors: the same
// mixed-precision iterative refinement, rows of J on their lanes). Returns
// false (uniformly) when the refinement cannot reach the FP64 solve.
template <int N, typename LT>
__device__ __forceinline__ bool w_solve(const WSh<LT> &sh, int n, double gamma_p, const double (&iw)[WState<N>::NS],
                                        double (&d)[WState<N>::NS]) {
  constexpr int NS = WState<N>::NS;
  const int ln = wlane();
  LT b[NS];
  if constexpr (sizeof(LT) == sizeof(double)) {
    w_apply<N, LT>(sh, n, d, b);
#pragma unroll
    for (int k = 0; k < NS; ++k) d[k] = (double)b[k];
    return true;
  } else {
    double r[NS];
    float w[NS];
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      r[k] = d[k];
      w[k] = (float)iw[k];
    }
    w_apply<N, LT>(sh, n, r, b);
    float nl = 0.0f;
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      d[k] = (ln + 32 * k < n) ? (double)b[k] : 0.0;
      if (ln + 32 * k < n) nl = fmaxf(nl, fabsf(b[k]) * w[k]);
    }
    const float nd = wmaxf(nl);
    float np = nd;
    for (int it = 0; it < REFINE_MAX; ++it) {
      double acc[NS], s[NS];
#pragma unroll
      for (int k = 0; k < NS; ++k) acc[k] = 0.0;
      for (int j = 0; j < n; ++j) {
        double x = d[0];
        if (NS > 1 && j >= 32) x = d[NS - 1];
        const double dj = __shfl_sync(WFULL, x, j & 31);
#pragma unroll
        for (int k = 0; k < NS; ++k) {
          const int i = ln + 32 * k;
          if (i < n) acc[k] = fma(sh.J[i * N + j], dj, acc[k]);
        }
      }
#pragma unroll
      for (int k = 0; k < NS; ++k) s[k] = (ln + 32 * k < n) ? fma(gamma_p, acc[k], r[k] - d[k]) : 0.0;
      w_apply<N, LT>(sh, n, s, b);
      nl = 0.0f;
#pragma unroll
      for (int k = 0; k < NS; ++k)
        if (ln + 32 * k < n) nl = fmaxf(nl, fabsf(b[k]) * w[k]);
      const float nc = wmaxf(nl);
      const float tol = fmaxf(REFINE_TOL * nd, REFINE_ABS);
      const bool done = nc <= tol;
      if (!done && !(nc < np)) return false;  // no longer contracting
#pragma unroll
      for (int k = 0; k < NS; ++k)
        if (ln + 32 * k < n) d[k] += (double)b[k];
      if (done || nc * (nc / np) <= tol) return true;
      np = nc;
    }
    return false;
  }
}

// ---- step logic (mirrors the thread form in mc_device.cuh) -----------------
template <int N>
__device__ __forceinline__ void w_rescale(WState<N> &W, int n, double eta) {
  constexpr int NS = WState<N>::NS;
  double r = 1.0;
#pragma unroll
  for (int j = 1; j <= QMAX + 1; ++j) {
    if (j <= W.q) {
      r *= eta;
#pragma unroll
      for (int k = 0; k < NS; ++k) W.z[j][k] *= r;
    }
  }
}

template <int N>
__device__ __forceinline__ void w_predict(WState<N> &W) {
  constexpr int NS = WState<N>::NS;
  const int q = W.q;
#pragma unroll
  for (int k = 0; k < QMAX; ++k)
#pragma unroll
    for (int j = QMAX; j > k; --j)
      if (k < q && j <= q)
#pragma unroll
        for (int s = 0; s < NS; ++s) W.z[j - 1][s] += W.z[j][s];
}

template <int N>
__device__ __forceinline__ void w_retract(WState<N> &W) {
  constexpr int NS = WState<N>::NS;
  const int q = W.q;
#pragma unroll
  for (int k = QMAX - 1; k >= 0; --k)
#pragma unroll
    for (int j = k + 1; j <= QMAX; ++j)
      if (k < q && j <= q)
#pragma unroll
        for (int s = 0; s < NS; ++s) W.z[j - 1][s] -= W.z[j][s];
}

template <int N>
__device__ __forceinline__ void w_begin_step(WState<N> &W, const DNet &net, const Opts &o) {
  constexpr int NS = WState<N>::NS;
  const int n = net.n, ln = wlane();
  if (!(W.t < W.tend)) { W.status = CELL_OK; W.phase = PH_DONE; return; }
  if (W.attempts >= o.max_steps) { W.status = CELL_MAX_STEPS; W.phase = PH_DONE; return; }
  W.last = false;
  if (W.t + W.h >= W.tend) {
    const double hn = W.tend - W.t;
    w_rescale(W, n, hn / W.h);
    W.h = hn;
    W.last = true;
  }
  W.attempts += 1;
#pragma unroll
  for (int k = 0; k < NS; ++k) {
    const int i = ln + 32 * k;
    W.iw[k] = (i < n) ? 1.0 / (o.rtol * fabs(W.z[0][k]) + o.atol) : 0.0;
  }
  w_predict(W);
  const int q = W.q;
  double gaps[QMAX + 2], xi[QMAX + 2];
  gaps[0] = W.h;
#pragma unroll
  for (int k = 0; k < QMAX + 1; ++k) gaps[k + 1] = W.hist[k];
  xi_of(W.h, gaps, q + 1, xi);
#pragma unroll
  for (int k = 0; k <= QMAX; ++k) W.l[k] = 0.0;
  W.l[0] = 1.0;
#pragma unroll
  for (int j = 1; j <= QMAX; ++j)
    if (j <= q) {
      const double c = 1.0 / xi[j - 1];
#pragma unroll
      for (int k = QMAX; k >= 1; --k)
        if (k <= j) W.l[k] += c * W.l[k - 1];
    }
  double xq = xi[0];
#pragma unroll
  for (int j = 1; j <= QMAX; ++j)
    if (j == q) xq = xi[j];
  W.cq = (1.0 / xq) / W.l[1];
  W.gamma = W.h / W.l[1];
  W.jcur = false;
  W.m = 0;
#pragma unroll
  for (int k = 0; k < NS; ++k) {
    W.e[k] = 0.0;
    W.y[k] = W.z[0][k];
  }
  W.phase = PH_NEWTON;
}

template <int N>
__device__ __forceinline__ void w_conv_failure(WState<N> &W, const DNet &net, const Opts &o) {
  w_retract(W);
  W.ncf += 1;
  W.st[ST_CONV_FAILS] += 1;
  if (W.ncf >= MXNCF) { W.status = CELL_CONV_FAIL; W.phase = PH_DONE; return; }
  w_rescale(W, net.n, ETACF);
  W.h *= ETACF;
  W.need_p = true;
  W.qwait = W.q + 1;
  W.have_es = false;
  if (W.t + W.h == W.t) { W.status = CELL_H_UNDERFLOW; W.phase = PH_DONE; return; }
  w_begin_step(W, net, o);
}

template <int N>
__device__ __forceinline__ void w_lower_order(WState<N> &W, const double *xi) {
  constexpr int NS = WState<N>::NS;
  double c[QMAX + 2];
  const int q = W.q;
  shifted_product(q, xi, c);
  double zq[NS];
#pragma unroll
  for (int s = 0; s < NS; ++s) zq[s] = 0.0;
#pragma unroll
  for (int j = 2; j <= QMAX; ++j)
    if (j == q)
#pragma unroll
      for (int s = 0; s < NS; ++s) zq[s] = W.z[j][s];
#pragma unroll
  for (int j = 1; j < QMAX; ++j)
    if (j < q)
#pragma unroll
      for (int s = 0; s < NS; ++s) W.z[j][s] -= c[j] * zq[s];
  W.q = q - 1;
}

template <int N>
__device__ __forceinline__ void w_after_convergence(WState<N> &W, const DNet &net, const Opts &o) {
  constexpr int NS = WState<N>::NS;
  const int n = net.n;
  const int q = W.q;
  const double dsm = W.cq * w_wrms<N>(n, W.e, W.iw);
  double xi[QMAX + 2];
  if (dsm > 1.0) {
    w_retract(W);
    W.nef += 1;
    W.st[ST_ERR_FAILS] += 1;
    W.have_es = false;
    if (W.nef >= KFC) {
#pragma unroll
      for (int s = 0; s < NS; ++s) W.y[s] = W.z[0][s];
      W.phase = PH_RESTART;
      return;
    }
    double eta = 1.0 / (root_k(BIAS_Q * dsm, q + 1, net.exptab) + ADDON);
    int qn = q;
    if (q > 1) {
      xi_of(W.h, W.hist, q, xi);
      double prod = 1.0, l1 = 0.0;
#pragma unroll
      for (int j = 1; j <= QMAX; ++j)
        if (j <= q - 1) {
          prod *= xi[j - 1];
          l1 += 1.0 / xi[j - 1];
        }
      double zq[NS];
#pragma unroll
      for (int k = 0; k < NS; ++k) zq[k] = 0.0;
#pragma unroll
      for (int j = 2; j <= QMAX; ++j)
        if (j == q)
#pragma unroll
          for (int k = 0; k < NS; ++k) zq[k] = W.z[j][k];
      const double est = (prod / l1) * w_wrms<N>(n, zq, W.iw);
      const double eta_m = 1.0 / (root_k(BIAS_QM1 * est, q, net.exptab) + ADDON);
      if (eta_m > eta) { eta = eta_m; qn = q - 1; }
    }
    eta = fmax(ETAMIN, fmin(eta, 1.0));
    if (qn < q) w_lower_order(W, xi);
    w_rescale(W, n, eta);
    W.h *= eta;
    W.qwait = W.q + 1;
    if (W.t + W.h == W.t) { W.status = CELL_H_UNDERFLOW; W.phase = PH_DONE; return; }
    w_begin_step(W, net, o);
    return;
  }
#pragma unroll
  for (int j = 0; j <= QMAX; ++j)
    if (j <= q)
#pragma unroll
      for (int s = 0; s < NS; ++s) W.z[j][s] += W.l[j] * W.e[s];
  W.t = W.last ? W.tend : W.t + W.h;
  for (int k = QMAX + 2; k > 0; --k) W.hist[k] = W.hist[k - 1];
  W.hist[0] = W.h;
  W.st[ST_STEPS] += 1;
  W.nef = 0;
  W.ncf = 0;
  W.jage += 1;
  W.page += 1;
  W.qwait -= 1;
  if (W.qwait == 1 && q < o.qmax) {
#pragma unroll
    for (int s = 0; s < NS; ++s) W.es[s] = W.e[s];
    W.esave_h = W.h;
    W.have_es = true;
  }
  if (W.last) { W.status = CELL_OK; W.phase = PH_DONE; return; }
  if (W.qwait > 0) { w_begin_step(W, net, o); return; }
  double eta = 1.0 / (root_k(BIAS_Q * dsm, q + 1, net.exptab) + ADDON);
  int qn = q;
  xi_of(W.h, W.hist, q + 1, xi);
  if (q > 1) {
    double prod = 1.0, l1 = 0.0;
#pragma unroll
    for (int j = 1; j <= QMAX; ++j)
      if (j <= q - 1) {
        prod *= xi[j - 1];
        l1 += 1.0 / xi[j - 1];
      }
    double zq[NS];
#pragma unroll
    for (int k = 0; k < NS; ++k) zq[k] = 0.0;
#pragma unroll
    for (int j = 2; j <= QMAX; ++j)
      if (j == q)
#pragma unroll
        for (int k = 0; k < NS; ++k) zq[k] = W.z[j][k];
    const double est = (prod / l1) * w_wrms<N>(n, zq, W.iw);
    const double eta_m = 1.0 / (root_k(BIAS_QM1 * est, q, net.exptab) + ADDON);
    if (eta_m > eta) { eta = eta_m; qn = q - 1; }
  }
  if (q < o.qmax && W.have_es) {
    const double r = ipow(W.h / W.esave_h, q + 1);
    double dv[NS];
#pragma unroll
    for (int s = 0; s < NS; ++s) dv[s] = W.e[s] - r * W.es[s];
    const double est = w_wrms<N>(n, dv, W.iw) / ((double)(q + 2) * harmonic(q + 1));
    const double eta_p = 1.0 / (root_k(BIAS_QP1 * est, q + 2, net.exptab) + ADDON);
    if (eta_p > eta) { eta = eta_p; qn = q + 1; }
  }
  W.have_es = false;
  if (eta < THRESH) {
    W.qwait = 2;
    w_begin_step(W, net, o);
    return;
  }
  eta = fmin(eta, W.eta_max);
  W.eta_max = ETAMX;
  if (qn > q) {
    double prod = 1.0, c[QMAX + 2];
#pragma unroll
    for (int j = 1; j <= QMAX + 1; ++j)
      if (j <= q + 1) prod *= xi[j - 1];
    const double C = 1.0 / prod;
    shifted_product(q + 1, xi, c);
#pragma unroll
    for (int j = 2; j <= QMAX + 1; ++j)
      if (j == q + 1)
#pragma unroll
        for (int s = 0; s < NS; ++s) W.z[j][s] = 0.0;
#pragma unroll
    for (int j = 1; j <= QMAX + 1; ++j)
      if (j <= q + 1)
#pragma unroll
        for (int s = 0; s < NS; ++s) W.z[j][s] += c[j] * C * W.e[s];
    W.q = q + 1;
  } else if (qn < q) {
    w_lower_order(W, xi);
  }
  w_rescale(W, n, eta);
  W.h *= eta;
  W.qwait = W.q + 1;
  w_begin_step(W, net, o);
}

template <int N, typename LT>
__device__ __forceinline__ int w_newton_iter(WState<N> &W, const WSh<LT> &sh, const DNet &net, const Opts &o,
                                             bool ok) {
  constexpr int NS = WState<N>::NS;
  const int n = net.n, ln = wlane();
  if (!ok) return 3;
  W.st[ST_RHS] += 1;
  if (W.m == 0) {
    bool newp = false;
    if (W.need_j || W.jage >= MSBJ) {
      if (!(o.jac_fd ? w_fd_jac<N, LT>(net, W.cin, sh, o.rtol, o.atol) : w_jac<N, LT>(net, W.cin, sh))) return 3;
      W.st[ST_JAC] += 1;
      W.jcur = true;
      W.need_j = false;
      W.jage = 0;
      newp = true;
    }
    if (newp || W.need_p || W.page >= MSBP || fabs(W.gamma / W.gamma_p - 1.0) > CCMAX) {
      W.st[ST_LU] += 1;
      W.gamma_p = W.gamma;
      W.page = 0;
      W.need_p = false;
      W.crate = CRATE0;
      bool lu_ok;
      if (w_switches<N, LT>() && W.p64) {
        const WSh<double> v = wsh_fp64(sh);
        w_form_p<N, double>(v, n, W.gamma);
        lu_ok = w_lu<N, double>(v, n);
      } else {
        w_form_p<N, LT>(sh, n, W.gamma);
        lu_ok = w_lu<N, LT>(sh, n);
      }
      if (!lu_ok) {
        W.need_p = true;
        return 2;
      }
    }
  }
  double d[NS];
  const double rl1 = 1.0 / W.l[1];
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    const int i = ln + 32 * s;
    d[s] = (i < n) ? (W.h * W.f[s] - W.z[1][s]) * rl1 - W.e[s] : 0.0;
  }
  if constexpr (w_switches<N, LT>()) {
    const WSh<double> v = wsh_fp64(sh);
    if (W.p64) {
      w_solve<N, double>(v, n, W.gamma_p, W.iw, d);
    } else {
      double d0[NS];
#pragma unroll
      for (int s = 0; s < NS; ++s) d0[s] = d[s];
      if (!w_solve<N, LT>(sh, n, W.gamma_p, W.iw, d)) {
        // the FP32 factors of this matrix cannot reach the FP64 solve: factor
        // the same matrix (J and gamma_P unchanged) in FP64, solve with it,
        // and keep FP64 factors for the rest of this cell
        W.p64 = true;
        W.st[ST_LU] += 1;
        w_form_p<N, double>(v, n, W.gamma_p);
        if (!w_lu<N, double>(v, n)) {
          W.need_p = true;
          return 2;
        }
#pragma unroll
        for (int s = 0; s < NS; ++s) d[s] = d0[s];
        w_solve<N, double>(v, n, W.gamma_p, W.iw, d);
      }
    }
  } else {
    if (!w_solve<N, LT>(sh, n, W.gamma_p, W.iw, d)) return 4;
  }
  W.st[ST_NEWTON] += 1;
  if (W.gamma != W.gamma_p) {
    const double sc = 2.0 / (1.0 + W.gamma / W.gamma_p);
#pragma unroll
    for (int s = 0; s < NS; ++s) d[s] *= sc;
  }
  const double del = w_wrms<N>(n, d, W.iw);
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    W.e[s] += d[s];
    W.y[s] = W.z[0][s] + W.e[s];
  }
  if (W.m > 0) W.crate = fmax(CRDOWN * W.crate, del / W.delp);
  const double dcon = del * fmin(1.0, W.crate) * W.cq / CORTES;
  if (dcon <= 1.0) return 1;
  W.m += 1;
  if (W.m == MAXCOR || (W.m >= 2 && del > RDIV * W.delp)) return 2;
  W.delp = del;
  return 0;
}

// Consume f(y) according to the cell's phase.
template <int N, typename LT>
__device__ __forceinline__ void w_advance(WState<N> &W, const WSh<LT> &sh, const DNet &net, const Opts &o, bool ok) {
  constexpr int NS = WState<N>::NS;
  const int n = net.n, ln = wlane();
  if (W.phase == PH_F0) {
    if (!ok) { W.status = CELL_BAD_INPUT; W.phase = PH_DONE; return; }
    W.st[ST_RHS] += 1;
    // starting step (Hairer, Norsett & Wanner, Solving ODEs I, II.4), p = 1
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      const int i = ln + 32 * k;
      W.iw[k] = (i < n) ? 1.0 / (o.rtol * fabs(W.z[0][k]) + o.atol) : 0.0;
    }
    const double d0 = w_wrms<N>(n, W.z[0], W.iw), d1 = w_wrms<N>(n, W.f, W.iw);
    double h0 = (d0 < 1e-5 || d1 < 1e-5) ? 1e-6 : 0.01 * d0 / d1;
    h0 = fmin(h0, W.tend);
    W.h0 = h0;
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      W.e[k] = W.f[k];  // f0 parked in e
      W.y[k] = W.z[0][k] + h0 * W.f[k];
    }
    W.st[ST_RHS] += 1;
    W.phase = PH_HW;
    return;
  }
  if (W.phase == PH_HW) {
    double h = W.h0;
    if (ok) {
      double dv[NS];
#pragma unroll
      for (int k = 0; k < NS; ++k) dv[k] = W.f[k] - W.e[k];
      const double d1 = w_wrms<N>(n, W.e, W.iw);
      const double d2 = w_wrms<N>(n, dv, W.iw) / W.h0;
      const double dm = fmax(d1, d2);
      const double h1 = (dm <= 1e-15) ? fmax(1e-6, W.h0 * 1e-3) : sqrt(0.01 / dm);
      h = fmin(fmin(100.0 * W.h0, h1), W.tend);
    }
    W.h = h;
#pragma unroll
    for (int k = 0; k < NS; ++k) W.z[1][k] = h * W.e[k];
    W.t = 0.0;
    W.q = 1;
    W.qwait = 2;
#pragma unroll
    for (int k = 0; k < QMAX + 3; ++k) W.hist[k] = h;
    W.need_j = true;
    W.need_p = true;
    W.crate = CRATE0;
    W.gamma_p = 1.0;
    W.eta_max = ETAMX_FIRST;
    W.nef = W.ncf = 0;
    W.jage = W.page = 0;
    W.have_es = false;
    W.attempts = 0;
    w_begin_step(W, net, o);
    return;
  }
  if (W.phase == PH_NEWTON) {
    const int r = w_newton_iter<N, LT>(W, sh, net, o, ok);
    if (r == 0) return;
    if (r == 4) { W.status = CELL_RETRY64; W.phase = PH_DONE; return; }  // to the FP64 retry pass
    if (r == 1) { w_after_convergence(W, net, o); return; }
    if (r == 2 && !W.jcur) {
      W.need_j = true;
      W.m = 0;
#pragma unroll
      for (int s = 0; s < NS; ++s) {
        W.e[s] = 0.0;
        W.y[s] = W.z[0][s];
      }
      return;
    }
    w_conv_failure(W, net, o);
    return;
  }
  if (W.phase == PH_RESTART) {
    if (!ok) { W.status = CELL_NONFINITE; W.phase = PH_DONE; return; }
    W.st[ST_RHS] += 1;
    W.h *= ETAMIN;
    W.q = 1;
#pragma unroll
    for (int s = 0; s < NS; ++s) W.z[1][s] = W.h * W.f[s];
    W.qwait = 2;
    if (W.t + W.h == W.t) { W.status = CELL_H_UNDERFLOW; W.phase = PH_DONE; return; }
    w_begin_step(W, net, o);
  }
}

template <int N>
__device__ __forceinline__ void w_store(WState<N> &W, const DNet &net, const CellArgs &a) {
  constexpr int NS = WState<N>::NS;
  const int64_t c = W.cell;
  const int S = net.S, ln = wlane();
  const int route = route_of(a, W.status);
  if (route != 0) {
    if (ln == 0) {
      if (route == 1) push_list(a, a.retry, a.retry_count, c);
      else push_list(a, a.lretry, a.lretry_count, c);
    }
    __syncwarp();
    return;
  }
  if (!MC_IN(a, BC_CELL_STORE, c, MC_CELLS(a))) return;
  if (ln == 0) MC_STORED(a, c);
  if (a.rung && ln == 0) a.rung[c] = a.rung_id;
  if (!(W.status == CELL_BAD_INPUT && W.m < 0)) {
    double xs = 0.0;
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      const int i = ln + 32 * s;
      if (i < S) {
        a.x[i * a.ld + c] = W.z[0][s];
        xs += W.z[0][s];
      }
    }
    const double X = wsum(xs);
    if (net.energy) {
      const double u = wget<NS>(W.z[0], S);
      if (ln == 0) a.T[c] = net.gm1 * u / (KB_EV * X);
    }
  }
  if (ln == 0) a.status[c] = W.status;
  if (a.stats && ln < NSTAT) {
    int v = 0;
    for (int k = 0; k < NSTAT; ++k)
      if (k == ln) v = (k == ST_ORDER) ? ((W.status == CELL_BAD_INPUT) ? 0 : W.q) : W.st[k];
    a.stats[ln * a.ld + c] = v;
  }
  __syncwarp();
}

// Warp-per-cell persistent worker: the warp pulls cells one at a time from
// the queue and integrates each with the whole warp.
template <int N, typename LT>
__device__ __forceinline__ void warp_worker(const DNet &net, const Opts &o, const CellArgs &a,
                                            unsigned long long *next, const WSh<LT> &sh) {
  const int64_t total = count_of(a);
  for (;;) {
    unsigned long long k = 0;
    if (wlane() == 0) k = atomicAdd(next, 1ull);
    k = __shfl_sync(WFULL, k, 0);
    if ((int64_t)k >= total) break;
    WState<N> W;
    w_load_cell<N>(W, net, a, cell_of(a, (int64_t)k));
    while (W.phase != PH_DONE) {
      const bool ok = w_rhs<N, LT>(W, sh, net);
      w_advance<N, LT>(W, sh, net, o, ok);
    }
    w_store<N>(W, net, a);
  }
}

template <int N, typename LT>
__global__ void __launch_bounds__(128) k_burn_warp(DNet net, Opts o, CellArgs a, unsigned long long *next,
                                                   int smem_per_warp) {
  extern __shared__ __align__(16) unsigned char smem[];
  const WSh<LT> sh = wsh_carve<N, LT>(smem + (threadIdx.x >> 5) * (size_t)smem_per_warp, net.R);
  warp_worker<N, LT>(net, o, a, next, sh);
}

// One segment of a mixed launch: a network, its cells and its compiled bucket.
struct SegDev {
  DNet net;
  CellArgs a;
  int bucket;
};

constexpr int MIXED_MAX_SEGS = 8;

struct MixedArgs {
  SegDev seg[MIXED_MAX_SEGS];
  StragArgs sa[MIXED_MAX_SEGS];  // hand-off of the thread-per-cell segments (rec = nullptr: none)
  int nseg;
  int smem_per_warp;  // warp workspace (the largest segment's)
};

// Mixed persistent launch: every warp drains the segment queues starting at a
// segment chosen by its warp index, so all networks start at once and warps
// that finish one network move on to the next (one launch for all networks).
// Networks of up to 13 ODEs run thread-per-cell (a cell still running after
// the hand-off threshold goes to its segment's record list, finished after the
// launch by k_burn_straggler), larger ones warp-per-cell.
template <typename LT>
__global__ void __launch_bounds__(128) k_burn_mixed(MixedArgs m, Opts o, unsigned long long *next) {
  extern __shared__ __align__(16) unsigned char smem[];
  unsigned char *wsp = smem + (threadIdx.x >> 5) * (size_t)m.smem_per_warp;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  for (int s0 = 0; s0 < m.nseg; ++s0) {
    const int s = (s0 + warp) % m.nseg;
    const SegDev &g = m.seg[s];
    switch (g.bucket) {
      case 3: persistent_worker<3, LT>(g.net, o, g.a, next + s, m.sa[s], wsh_carve<3, LT>(wsp, g.net.R)); break;
      case 13: persistent_worker<13, LT>(g.net, o, g.a, next + s, m.sa[s], wsh_carve<13, LT>(wsp, g.net.R)); break;
      case 33: warp_worker<33, LT>(g.net, o, g.a, next + s, wsh_carve<33, LT>(wsp, g.net.R)); break;
      default: warp_worker<40, LT>(g.net, o, g.a, next + s, wsh_carve<40, LT>(wsp, g.net.R)); break;
    }
  }
}

// Straggler kernel: each warp takes handed-off cells (records of the thread
// form's state) until the list is done; count is read on the device. After a
// fused launch it integrates only the records that launch left (flag != 2).
template <int N, typename LT>
__global__ void __launch_bounds__(128) k_burn_straggler(DNet net, Opts o, CellArgs a, const Lane<N, LT> *rec,
                                                        const uint32_t *count, uint32_t cap, const uint32_t *flag,
                                                        unsigned long long *next, int smem_per_warp) {
  extern __shared__ __align__(16) unsigned char smem[];
  const WSh<LT> sh = wsh_carve<N, LT>(smem + (threadIdx.x >> 5) * (size_t)smem_per_warp, net.R);
  const uint32_t total = min(*count, cap);
  for (;;) {
    unsigned long long k = 0;
    int skip = 0;
    if (wlane() == 0) {
      k = atomicAdd(next, 1ull);
      skip = (k < total && flag && flag[k] == 2u) ? 1 : 0;
    }
    k = __shfl_sync(WFULL, k, 0);
    if (k >= total) break;
    if (__shfl_sync(WFULL, skip, 0)) continue;
    if (!MC_IN(a, BC_RECORD, k, cap)) continue;
    WState<N> W;
    w_load<N, LT>(W, rec[k], sh, net);
    while (W.phase != PH_DONE) {
      const bool ok = w_rhs<N, LT>(W, sh, net);
      w_advance<N, LT>(W, sh, net, o, ok);
    }
    w_store<N>(W, net, a);
  }
}

// ---- fused launch: bulk and hand-off in one grid -----------------------------
// Every warp first runs the thread-per-cell queue; once its queue is drained it
// integrates handed-off records warp-per-cell while other warps are still in
// the bulk, so the long cells start before the bulk has ended. Launched
// cooperatively (all blocks resident), because these warps wait for records
// that other blocks write.
struct FuseArgs {
  uint32_t *claim;       // records claimed by warp-form workers
  uint32_t *bulk_done;   // bulk warps whose queue loop has ended
  uint32_t n_bulk_warps;
};

// Polls without progress after which a waiting warp leaves (its record, and any
// record left, is then integrated by k_burn_straggler after the launch).
constexpr uint32_t FUSE_SPIN_LIMIT = 1u << 21;

// Lane 0 waits for record j: 1 once it is written; 0 once every bulk warp is
// done and record j will never be written; -1 after FUSE_SPIN_LIMIT polls in a
// row during which neither the cell queue nor the bulk-done count moved. Polls
// are relaxed loads with a sleep that doubles up to 8 us.
__device__ __forceinline__ int fuse_wait(const StragArgs &sa, const FuseArgs &fa, uint32_t j,
                                         const unsigned long long *next) {
  int r = -1;
  if (wlane() == 0) {
    unsigned long long q0 = ld_relaxed(next);
    uint32_t d0 = ld_relaxed(fa.bulk_done);
    unsigned ns = 256;
    for (uint32_t spins = 0; spins < FUSE_SPIN_LIMIT;) {
      if (ld_relaxed(&sa.flag[j]) != 0u) { r = 1; break; }
      const uint32_t d = ld_relaxed(fa.bulk_done);
      // all bulk warps done: the record count is final; a record below it is
      // written already and its flag shows on a later poll
      if (d >= fa.n_bulk_warps && j >= min(ld_relaxed(sa.count), sa.cap)) { r = 0; break; }
      const unsigned long long q = ld_relaxed(next);
      if (q != q0 || d != d0) {
        q0 = q;
        d0 = d;
        spins = 0;
      } else {
        ++spins;
      }
      __nanosleep(ns);
      if (ns < 8192) ns *= 2;
    }
  }
  return __shfl_sync(WFULL, r, 0);
}

template <int N, typename LT>
__device__ __forceinline__ void fused_records(const DNet &net, const Opts &o, const CellArgs &a,
                                              const StragArgs &sa, const FuseArgs &fa,
                                              const unsigned long long *next, const WSh<LT> &sh) {
  const Lane<N, LT> *rec = static_cast<const Lane<N, LT> *>(sa.rec);
  for (;;) {
    uint32_t j = 0;
    if (wlane() == 0) j = atomicAdd(fa.claim, 1u);
    j = __shfl_sync(WFULL, j, 0);
    if (j >= sa.cap) return;
    if (fuse_wait(sa, fa, j, next) != 1) return;
    if (!MC_IN(a, BC_RECORD, j, sa.cap)) return;
    // every lane observes the flag, then fences: it synchronises with the
    // release store of the record's writer before reading the record
    (void)ld_relaxed(&sa.flag[j]);
    __threadfence();
    WState<N> W;
    w_load<N, LT>(W, rec[j], sh, net);
    while (W.phase != PH_DONE) {
      const bool ok = w_rhs<N, LT>(W, sh, net);
      w_advance<N, LT>(W, sh, net, o, ok);
    }
    w_store<N>(W, net, a);
    __syncwarp();
    if (wlane() == 0) st_release(&sa.flag[j], 2u);
  }
}

template <int N, typename LT>
__global__ void __launch_bounds__(128, 3) k_burn_fused(DNet net, Opts o, CellArgs a, unsigned long long *next,
                                                       StragArgs sa, FuseArgs fa, int smem_per_warp) {
  extern __shared__ __align__(16) unsigned char smem[];
  const WSh<LT> sh = wsh_carve<N, LT>(smem + (threadIdx.x >> 5) * (size_t)smem_per_warp, net.R);
  persistent_worker<N, LT>(net, o, a, next, sa, sh);
  __syncwarp();
  if (wlane() == 0) {
    __threadfence();
    atomicAdd(fa.bulk_done, 1u);
  }
  fused_records<N, LT>(net, o, a, sa, fa, next, sh);
}

}  // namespace mc
