// mc_coop.cuh -- warp-cooperative pieces of the burn: the Jacobian and the
// factorisation of the iteration matrix of ONE cell computed by a whole warp
// in shared memory.
//
// On this GPU an FP64 warp instruction occupies the FP64 pipe for the whole
// warp whether 1 or 32 lanes are active. A thread-per-cell worker whose lanes
// each need a new Jacobian about once every 50 right-hand sides would, done
// lane by lane, run the Jacobian code in about every second loop trip for one
// or two lanes. Here the warp serves the waiting lanes one cell at a time
// instead: reaction rates and their derivatives spread over the lanes, matrix
// rows assembled row-parallel from the network's occurrence lists, and a
// row-parallel LU with partial pivoting. The same routines serve the
// warp-per-cell form (mc_warp.cuh).
#pragma once

#include "mc_device.cuh"

namespace mc {

constexpr unsigned WFULL = 0xffffffffu;

__device__ __forceinline__ int wlane() { return threadIdx.x & 31; }

__device__ __forceinline__ double wsum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(WFULL, v, o);
  return v;
}

__device__ __forceinline__ float wmaxf(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(WFULL, v, o));
  return v;
}

// vector slots of a distributed vector of N components (component i on lane
// i mod 32, slot i / 32)
template <int N>
struct WSlots {
  static constexpr int NS = (N + 31) / 32;
};

// what a lane hands the warp when it asks for matrix work
struct WReq {
  CellIn cin;
  double gamma;
  int want_j;
};

// per-warp shared workspace (carved from dynamic shared memory)
template <typename LT>
struct WSh {
  double *J;        // [N*N] Jacobian (FP64), row stride N
  LT *P;            // [N*N] iteration matrix, then its factors (see w_lu)
  unsigned char *piv;
  double *yb;       // [N]   point of evaluation, for broadcast
  double *wb;       // [R]   net reaction rates
  double *dw;       // [5R]  d w / d x per side slot, then d w / d T
  WReq *req;        // request of the lane being served
  double *P64;      // [N*N] FP64 factors of a warp-form cell whose FP32 solves
  unsigned char *piv64;  // could not be refined (see w_newton_iter), or nullptr
};

// Warp-form cells with an FP32 matrix switch to FP64 factors in place when the
// refinement of their FP32 solves stops converging (networks above 16 ODEs,
// which always run warp-per-cell); thread-form cells hand such cells to the
// FP64 retry pass instead.
template <int N, typename LT>
__host__ __device__ constexpr bool w_switches() {
  return sizeof(LT) == sizeof(float) && N > 16;
}

template <int N, typename LT>
__host__ __device__ inline size_t wsh_bytes(int R) {
  auto al = [](size_t b) { return (b + 15) & ~(size_t)15; };
  const size_t r = (size_t)(R > 0 ? R : 1);
  size_t b = al(sizeof(double) * N * N) + al(sizeof(LT) * N * N) + al(N) + al(sizeof(double) * N) +
             al(sizeof(double) * r) + al(sizeof(double) * 5 * r) + al(sizeof(WReq));
  if constexpr (w_switches<N, LT>()) b += al(sizeof(double) * N * N) + al(N);
  return b;
}

template <int N, typename LT>
__device__ __forceinline__ WSh<LT> wsh_carve(unsigned char *p, int R) {
  auto al = [](size_t b) { return (b + 15) & ~(size_t)15; };
  const size_t r = (size_t)(R > 0 ? R : 1);
  WSh<LT> s;
  s.J = (double *)p;
  p += al(sizeof(double) * N * N);
  s.P = (LT *)p;
  p += al(sizeof(LT) * N * N);
  s.piv = p;
  p += al(N);
  s.yb = (double *)p;
  p += al(sizeof(double) * N);
  s.wb = (double *)p;
  p += al(sizeof(double) * r);
  s.dw = (double *)p;
  p += al(sizeof(double) * 5 * r);
  s.req = (WReq *)p;
  p += al(sizeof(WReq));
  s.P64 = nullptr;
  s.piv64 = nullptr;
  if constexpr (w_switches<N, LT>()) {
    s.P64 = (double *)p;
    p += al(sizeof(double) * N * N);
    s.piv64 = p;
  }
  return s;
}

// the FP64 factor view of a workspace (the same J, point and rates)
template <typename LT>
__device__ __forceinline__ WSh<double> wsh_fp64(const WSh<LT> &s) {
  WSh<double> v;
  v.J = s.J;
  v.P = s.P64;
  v.piv = s.piv64;
  v.yb = s.yb;
  v.wb = s.wb;
  v.dw = s.dw;
  v.req = s.req;
  v.P64 = nullptr;
  v.piv64 = nullptr;
  return v;
}

// temperature quantities of the point in yb (energy form) or of the cell
__device__ __forceinline__ bool w_temperature(const DNet &net, const CellIn &c, const double *yb, double &T,
                                              double &X, double &lnT, double &invT) {
  lnT = c.lnT;
  invT = c.invT;
  T = 0.0;
  X = 0.0;
  if (!net.energy) return true;
  double xs = 0.0;
  for (int i = wlane(); i < net.S; i += 32) xs += yb[i];
  X = wsum(xs);
  T = net.gm1 * yb[net.S] / (KB_EV * X);
  if (!(T > 0.0) || !isfinite(T)) return false;
  lnT = log(T);
  invT = 1.0 / T;
  return true;
}

// Analytic Jacobian (the formulas of net_jac) at the point in sh.yb, into
// sh.J. Phases: reaction r on lane r mod 32 writes d w_r / d x per side slot
// and d w_r / d T; lane i < S assembles species row i and the energy row's
// column i from species i's occurrence list; then every row i < n adds the
// EOS chain-rule terms g_i dT/dx_j and g_i dT/du. Returns false (uniformly)
// when the point cannot be evaluated or an entry is not finite.
template <int N, typename LT>
__device__ __forceinline__ bool w_jac(const DNet &net, const CellIn &c, const WSh<LT> &sh) {
  const int n = net.n, S = net.S, ln = wlane();
  double T, X, lnT, invT;
  if (!w_temperature(net, c, sh.yb, T, X, lnT, invT)) return false;
  double gpart = 0.0;
  for (int r = ln; r < net.R; r += 32) {
    const int4 s = __ldg(&net.side[r]);
    const RxPar &p = net.par[r];
    const double bf = __ldg(&p.bf), Cf = __ldg(&p.Cf);
    double kf = rexp(__ldg(&p.lnAf) + bf * lnT - Cf * invT, net.exptab);
    double kr = 0.0, br = 0.0, Cr = 0.0;
    if (has_reverse(p)) {
      br = __ldg(&p.br);
      Cr = __ldg(&p.Cr);
      kr = rexp(__ldg(&p.lnAr) + br * lnT - Cr * invT, net.exptab);
    }
    if (c.ks) {
      const double sc = c.ks[r * c.ks_ld];
      kf *= sc;
      kr *= sc;
    }
    double *d = sh.dw + 5 * r;
    double pf, pr;
    if (s.y < 0) { pf = sh.yb[s.x]; d[0] = kf; d[1] = 0.0; }
    else { pf = c.nd * sh.yb[s.x] * sh.yb[s.y]; d[0] = kf * (c.nd * sh.yb[s.y]); d[1] = kf * (c.nd * sh.yb[s.x]); }
    if (s.w < 0) { pr = sh.yb[s.z]; d[2] = -kr; d[3] = 0.0; }
    else { pr = c.nd * sh.yb[s.z] * sh.yb[s.w]; d[2] = -kr * (c.nd * sh.yb[s.w]); d[3] = -kr * (c.nd * sh.yb[s.z]); }
    d[4] = kf * (bf + Cf * invT) * invT * pf - kr * (br + Cr * invT) * invT * pr;
    if (net.energy) gpart += __ldg(&p.dE) * d[4];
  }
  const double gS = net.energy ? wsum(gpart) : 0.0;
  for (int idx = ln; idx < n * N; idx += 32) sh.J[idx] = 0.0;
  __syncwarp();
  // species rows, and the energy row's column of each species
  constexpr int NS = WSlots<N>::NS;
  double g[NS];
#pragma unroll
  for (int k = 0; k < NS; ++k) {
    g[k] = 0.0;
    const int i = ln + 32 * k;
    if (i < S) {
      double acc = 0.0;
      for (int q = __ldg(&net.csr_ptr[i]); q < __ldg(&net.csr_ptr[i + 1]); ++q) {
        const int ent = __ldg(&net.csr_ent[q]);
        const int r = ent >> 2;
        const double sgn = ((ent & 3) < 2) ? -1.0 : 1.0;
        const int4 s = __ldg(&net.side[r]);
        const int col[4] = {s.x, s.y, s.z, s.w};
        const double *d = sh.dw + 5 * r;
        g[k] += sgn * d[4];
#pragma unroll
        for (int b = 0; b < 4; ++b)
          if (col[b] >= 0) sh.J[i * N + col[b]] += sgn * d[b];
        if (net.energy) acc += __ldg(&net.par[r].dE) * d[ent & 3];
      }
      if (net.energy) sh.J[S * N + i] = acc;
    }
  }
  __syncwarp();
  // chain rule through the EOS temperature, and the finite test
  bool bad = false;
  const double dTdx = net.energy ? -T / X : 0.0, dTdu = net.energy ? net.gm1 / (KB_EV * X) : 0.0;
#pragma unroll
  for (int k = 0; k < NS; ++k) {
    const int i = ln + 32 * k;
    if (i < n) {
      if (net.energy) {
        const double gi = (i < S) ? g[k] : gS;
        const double gx = gi * dTdx;
        for (int j = 0; j < S; ++j) sh.J[i * N + j] += gx;
        sh.J[i * N + S] += gi * dTdu;
      }
      for (int j = 0; j < n; ++j)
        if (!finite64(sh.J[i * N + j])) bad = true;
    }
  }
  __syncwarp();
  return !__any_sync(WFULL, bad);
}

// sh.P = I - gamma sh.J in the matrix precision
template <int N, typename LT>
__device__ __forceinline__ void w_form_p(const WSh<LT> &sh, int n, double gamma) {
  const LT g = (LT)gamma;
  for (int idx = wlane(); idx < n * N; idx += 32) {
    const int i = idx / N, j = idx - i * N;
    if (j < n) sh.P[idx] = (i == j ? (LT)1 : (LT)0) - g * (LT)sh.J[idx];
  }
  __syncwarp();
}

// Row-parallel LU with partial pivoting in shared memory (first maximal |a|).
// As lu_factor: L below the diagonal, U above, U's diagonal as reciprocals.
template <int N, typename LT>
__device__ __forceinline__ bool w_lu(const WSh<LT> &sh, int n) {
  const int ln = wlane();
  for (int k = 0; k < n; ++k) {
    LT best = (LT)-1;
    int bi = n;
    for (int i = k + ln; i < n; i += 32) {
      const LT v = fabs(sh.P[i * N + k]);
      if (v > best) { best = v; bi = i; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const LT ov = __shfl_xor_sync(WFULL, best, o);
      const int oi = __shfl_xor_sync(WFULL, bi, o);
      if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
    }
    if (ln == 0) sh.piv[k] = (unsigned char)bi;
    if (!(best > (LT)0)) { __syncwarp(); return false; }
    if (bi != k)
      for (int j = ln; j < n; j += 32) {
        const LT tmp = sh.P[k * N + j];
        sh.P[k * N + j] = sh.P[bi * N + j];
        sh.P[bi * N + j] = tmp;
      }
    __syncwarp();
    const LT inv = (LT)1 / sh.P[k * N + k];
    for (int i = k + 1 + ln; i < n; i += 32) {
      const LT m = sh.P[i * N + k] * inv;
      sh.P[i * N + k] = m;
      for (int j = k + 1; j < n; ++j) sh.P[i * N + j] -= m * sh.P[k * N + j];
    }
    __syncwarp();
    if (ln == 0) sh.P[k * N + k] = inv;
  }
  __syncwarp();
  return true;
}

// Right-hand side at the point in sh.yb by the whole warp: reaction r's net
// rate on lane r mod 32 (into sh.wb), then component i on lane i mod 32 (slot
// i / 32) summed from its occurrence list, the energy rate by a warp sum.
// Returns false (uniformly) when the point cannot be evaluated or f is not
// finite.
template <int N, typename LT>
__device__ __forceinline__ bool w_rhs_core(const DNet &net, const CellIn &c, const WSh<LT> &sh,
                                           double (&f)[WSlots<N>::NS]) {
  constexpr int NS = WSlots<N>::NS;
  const int n = net.n, S = net.S, ln = wlane();
  double T, X, lnT, invT;
  if (!w_temperature(net, c, sh.yb, T, X, lnT, invT)) return false;
  double epart = 0.0;
  for (int r = ln; r < net.R; r += 32) {
    const int4 s = __ldg(&net.side[r]);
    const RxPar &p = net.par[r];
    double kf = rexp(__ldg(&p.lnAf) + __ldg(&p.bf) * lnT - __ldg(&p.Cf) * invT, net.exptab);
    double kr = 0.0;
    if (has_reverse(p)) kr = rexp(__ldg(&p.lnAr) + __ldg(&p.br) * lnT - __ldg(&p.Cr) * invT, net.exptab);
    if (c.ks) {
      const double sc = c.ks[r * c.ks_ld];
      kf *= sc;
      kr *= sc;
    }
    const double pf = (s.y < 0) ? sh.yb[s.x] : c.nd * sh.yb[s.x] * sh.yb[s.y];
    const double pr = (s.w < 0) ? sh.yb[s.z] : c.nd * sh.yb[s.z] * sh.yb[s.w];
    const double w = kf * pf - kr * pr;
    sh.wb[r] = w;
    if (net.energy) epart += __ldg(&p.dE) * w;
  }
  __syncwarp();
  const double fu = net.energy ? wsum(epart) : 0.0;
  bool bad = false;
#pragma unroll
  for (int k = 0; k < NS; ++k) {
    const int i = ln + 32 * k;
    double v = 0.0;
    if (i < S) {
      for (int q = __ldg(&net.csr_ptr[i]); q < __ldg(&net.csr_ptr[i + 1]); ++q) {
        const int ent = __ldg(&net.csr_ent[q]);
        const double w = sh.wb[ent >> 2];
        v = ((ent & 3) < 2) ? v - w : v + w;
      }
    } else if (i == S && net.energy) {
      v = fu;
    }
    if (c.src && i < n) v += c.src[i * c.ks_ld];
    f[k] = v;
    if (i < n && !finite64(v)) bad = true;
  }
  __syncwarp();
  return !__any_sync(WFULL, bad);
}

// Forward-difference Jacobian (net_fd_jac's columns) at the point in sh.yb,
// into sh.J: one warp right-hand side per column, lane i writing row i.
template <int N, typename LT>
__device__ __forceinline__ bool w_fd_jac(const DNet &net, const CellIn &c, const WSh<LT> &sh, double rtol,
                                         double atol) {
  constexpr int NS = WSlots<N>::NS;
  const int n = net.n, ln = wlane();
  double f0[NS], f1[NS];
  if (!w_rhs_core<N, LT>(net, c, sh, f0)) return false;
  for (int j = 0; j < n; ++j) {
    const double yj = sh.yb[j];
    const double yp = yj + FD_SQRT_EPS * (fabs(yj) + atol / rtol);
    const double dj = yp - yj;
    if (!(dj != 0.0)) return false;
    __syncwarp();
    if (ln == 0) sh.yb[j] = yp;
    __syncwarp();
    const bool ok = w_rhs_core<N, LT>(net, c, sh, f1);
    if (ln == 0) sh.yb[j] = yj;
    __syncwarp();
    if (!ok) return false;
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      const int i = ln + 32 * k;
      if (i < n) sh.J[i * N + j] = (f1[k] - f0[k]) / dj;
    }
  }
  __syncwarp();
  return true;
}

// Matrix work of the lanes of a thread-per-cell worker whose Newton iteration
// waits for it (todo == TD_MATRIX), done by the whole warp one cell at a time:
// the waiting lane publishes its point, its cell inputs, gamma and (when only
// a refactorisation is due) its Jacobian in the warp's workspace; the warp
// evaluates the Jacobian (w_jac), forms P = I - gamma J (w_form_p) and factors
// it (w_lu); the lane copies J, the factors and the pivots into its own state.
// The lanes' corrections then run together in the TD_CORRECT stage. Called by
// all 32 lanes of the warp.
template <int N, typename LT>
__device__ __forceinline__ void coop_matrix(Lane<N, LT> &L, const DNet &net, const Opts &o, const WSh<LT> &sh) {
  const int n = net.n, ln = wlane();
  unsigned wait = __ballot_sync(WFULL, L.todo == TD_MATRIX);
  bool jok = true, pok = false;
  while (wait) {
    const int src = __ffs(wait) - 1;
    wait &= wait - 1;
    if (ln == src) {
      for (int i = 0; i < n; ++i) sh.yb[i] = L.y[i];
      if (!L.want_j)
        for (int idx = 0; idx < n * N; ++idx) sh.J[idx] = L.J[idx];
      sh.req->cin = L.cin;
      sh.req->gamma = L.gamma;
      sh.req->want_j = L.want_j ? 1 : 0;
    }
    __syncwarp();
    const CellIn c = sh.req->cin;
    const bool wj = sh.req->want_j != 0;
    const double gamma = sh.req->gamma;
    bool j_ok = true, p_ok = false;
    if (wj) j_ok = o.jac_fd ? w_fd_jac<N, LT>(net, c, sh, o.rtol, o.atol) : w_jac<N, LT>(net, c, sh);
    if (j_ok) {
      w_form_p<N, LT>(sh, n, gamma);
      p_ok = w_lu<N, LT>(sh, n);
    }
    if (ln == src) {
      jok = j_ok;
      pok = p_ok;
      if (wj && j_ok)
        for (int idx = 0; idx < n * N; ++idx) L.J[idx] = sh.J[idx];
      if (j_ok) {
        for (int idx = 0; idx < n * N; ++idx) L.P[idx] = sh.P[idx];
        for (int i = 0; i < n; ++i) L.piv[i] = sh.piv[i];
      }
    }
    __syncwarp();
  }
  if (L.todo == TD_MATRIX) newton_outcome(L, n, newton_after_matrix(L, jok, pok));
}

}  // namespace mc
