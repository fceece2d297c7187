// mc_device.cuh -- device side of the per-cell burn (sm_103a).
//
// One lane integrates one cell (thread-per-cell): the paper's single-zone
// routine applied to every zone on the GPU (Software design section,
// paragraph 3). The integrator is written as a per-lane state machine whose
// loop body performs exactly ONE right-hand-side evaluation for every active
// lane; what a lane does before and after it (Newton update, error test,
// step/order change, a new cell) is cheap, so lanes of a warp stay converged
// on the expensive part even when they sit in different cells, steps or
// Newton iterations. That is what lets a persistent worker refill a lane the
// moment its cell is done.
//
// Method (VODE-style BDF; the paper cites Brown, Byrne & Hindmarsh 1989 and
// gives no details, so this is the library's restatement, shared with nothing
// else in the tree):
//   Nordsieck array z_j = h^j y^(j)/j!, j <= q <= 5, holding the polynomial
//   through the last q+1 accepted values. Prediction is the Taylor shift
//   z <- z*Pascal. The corrector e solves h f(z_0 + e) = z_1 + l_1 e by
//   modified Newton with P = I - gamma J, gamma = h/l_1, where
//   l = coeffs of prod_{j<=q} (1 + x/xi_j), xi_j = (t_n - t_{n-j})/h.
//   Local error estimate e (1/xi_{q+1}) / l_1; step/order selection from the
//   q-1, q, q+1 estimates; Jacobian kept 50 steps, matrix 20 steps or until
//   gamma drifts 30 %.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace mc {

constexpr int QMAX = 5;
constexpr double KB_EV = 8.617333262e-5;  // Boltzmann constant, eV/K

// ---- policy constants of the integrator ------------------------------------
constexpr int MAXCOR = 3;          // Newton corrections per attempt
constexpr double RDIV = 2.0;       // divergence: del > RDIV * previous del
constexpr double CRDOWN = 0.3;     // memory of the convergence rate
constexpr double CORTES = 0.1;     // Newton error allowed, share of the local error
constexpr double CRATE0 = 0.7;     // rate estimate after a new matrix
constexpr double ETACF = 0.25;     // step factor after a Newton failure
constexpr int MXNCF = 10;          // consecutive Newton failures allowed
constexpr int KFC = 3;             // error failures before an order-1 restart
constexpr double ETAMIN = 0.1;     // smallest factor after an error failure
constexpr double BIAS_QM1 = 6.0, BIAS_Q = 6.0, BIAS_QP1 = 10.0, ADDON = 1.0e-6;
constexpr double THRESH = 1.5;     // smallest growth worth a step change
constexpr double ETAMX_FIRST = 1.0e4, ETAMX = 10.0;
constexpr int MSBJ = 50;           // accepted steps between Jacobians
constexpr int MSBP = 20;           // accepted steps between factorisations
constexpr double CCMAX = 0.3;      // refactor when |gamma/gamma_P - 1| > CCMAX

// CELL_RETRY64 is internal: an FP32-matrix cell whose refined solves cannot
// reach the FP64 solve goes to the FP64 retry pass (never stored as a status).
enum CellStatus : int { CELL_OK = 0, CELL_MAX_STEPS = 1, CELL_H_UNDERFLOW = 2, CELL_CONV_FAIL = 3,
                        CELL_BAD_INPUT = 4, CELL_NONFINITE = 5, CELL_RETRY64 = 6 };
enum Stat : int { ST_STEPS = 0, ST_ERR_FAILS, ST_CONV_FAILS, ST_RHS, ST_JAC, ST_LU, ST_NEWTON,
                  ST_ORDER, NSTAT };

// ---- network in device memory ----------------------------------------------
struct __align__(64) RxPar {
  double lnAf, bf, Cf;   // forward: k = exp(lnA + b ln T - C / T)
  double lnAr, br, Cr;   // reverse
  double dE;             // energy released by a forward event (eV)
  double rev;            // 1 if the reverse direction exists
};

struct DNet {
  int S, R, n, energy;   // species, reactions, ODEs, energy equation flag
  double gm1;            // gamma - 1
  double inv_n;          // 1 / n (the RMS norms' mean)
  const int4 *side;      // (reactant0, reactant1, product0, product1), -1 = empty
  const RxPar *par;
  const double *exptab;  // 2^(j/64), j = 0..63 (for rexp)
  // per-species occurrence lists: species i appears in slots csr_ent[csr_ptr[i]
  // .. csr_ptr[i+1]) with entry = 4 r + slot (slots 0,1 reactants, 2,3 products),
  // in the order the thread right-hand side applies them
  const int *csr_ptr;
  const int *csr_ent;
};

// Table-driven exponential for the rate coefficients (the dominant FP64 cost
// of the burn), after Tang's table-driven method (P. T. P. Tang, ACM TOMS 15,
// 144-157, 1989): x = (n/64) ln 2 + r with n = round(64 x / ln 2) (obtained by
// adding 1.5 * 2^52, which leaves n in the low mantissa bits), r reduced with
// a two-part ln2/64 in two FMAs, |r| <= ln2/128; exp(r) - 1 by its Taylor
// polynomial to degree 5 (truncation below 4e-17 relative on that interval);
// exp(x) = 2^(n >> 6) * (T + T (exp(r) - 1)), T = 2^((n & 63)/64) from a
// 64-entry table computed on the host, the power of two applied to the
// exponent field. About 10 FP64 instructions; the range test reads the high
// word of x in the integer unit, so it costs the FP64 pipe nothing. Within a
// few ulp of the correctly rounded value (checked against the CUDA exp in the
// tests).
__device__ __forceinline__ double rexp(double x, const double *tab) {
  if ((__double2hiint(x) & 0x7fffffff) >= 0x40862000) {  // |x| >= 708, infinite or NaN
    if (!(x > -745.2)) return (x != x) ? x : 0.0;         // NaN propagates; -inf and underflow give 0
    if (x > 709.78) return __longlong_as_double(0x7ff0000000000000ll);
  }
  const double SHIFT = 6755399441055744.0;           // 1.5 * 2^52
  const double INVL = 92.332482616893656768;        // 64 / ln 2
  const double L_HI = 0.010830424696249145;         // ln 2 / 64, leading part
  const double L_LO = 3.623510646634843e-19;         // ln 2 / 64 - L_HI
  const double kd = fma(x, INVL, SHIFT);
  const int n = __double2loint(kd);
  const double nd = kd - SHIFT;
  double r = fma(-nd, L_HI, x);
  r = fma(-nd, L_LO, r);
  double p = fma(r, 1.0 / 120.0, 1.0 / 24.0);
  p = fma(p, r, 1.0 / 6.0);
  p = fma(p, r, 0.5);
  p = fma(p, r, 1.0);
  p = p * r;
  const double t = __ldg(&tab[n & 63]);
  double v = fma(t, p, t);
  const int m = n >> 6;
  if (m >= -1021) {
    return __hiloint2double(__double2hiint(v) + (m << 20), __double2loint(v));
  }
  // result below the normal range: scale in two steps so the rounding happens once
  v = __hiloint2double(__double2hiint(v) + ((m + 600) << 20), __double2loint(v));
  return v * 2.409919865102884e-181;                 // 2^-600
}

// v^(1/k) for v >= 0, k = 1..8, as exp(log(v) / k) with the table exponential:
// the step-size factors' root (the library pow costs several times more FP64
// instructions for the same rounding-level result).
__device__ __forceinline__ double root_k(double v, int k, const double *tab) {
  const double inv = (k == 1) ? 1.0 : (k == 2) ? 0.5 : (k == 3) ? 1.0 / 3.0 : (k == 4) ? 0.25 : (k == 5) ? 0.2
                   : (k == 6) ? 1.0 / 6.0 : (k == 7) ? 1.0 / 7.0 : 0.125;
  return rexp(log(v) * inv, tab);
}

// x^k for k = 1..8 by repeated multiplication
__device__ __forceinline__ double ipow(double x, int k) {
  double r = x;
  for (int j = 1; j < k; ++j) r *= x;
  return r;
}

// Harmonic numbers G_k = sum_{j<=k} 1/j as the same sum in double gives them.
__device__ __forceinline__ double harmonic(int k) {
  return (k <= 1) ? 1.0 : (k == 2) ? 1.5 : (k == 3) ? 1.8333333333333333 : (k == 4) ? 2.083333333333333
       : (k == 5) ? 2.283333333333333 : (k == 6) ? 2.4499999999999997 : (k == 7) ? 2.5928571428571425
       : 2.7178571428571425;
}

// Finite test on the high word in the integer unit (no FP64 instruction).
__device__ __forceinline__ bool finite64(double v) {
  return (__double2hiint(v) & 0x7ff00000) != 0x7ff00000;
}

// Reverse-direction flag of a reaction record (0.0 or 1.0), read as an integer.
__device__ __forceinline__ bool has_reverse(const RxPar &p) { return __double2hiint(__ldg(&p.rev)) != 0; }

// per-cell inputs the right-hand side needs
struct CellIn {
  double nd;             // total density n
  double lnT, invT;      // isothermal networks: fixed temperature
  const double *ks;      // rate_scale + cell (stride ks_ld) or nullptr
  int64_t ks_ld;
  const double *src;     // constant source + cell (stride ks_ld, one per ODE) or nullptr
};

// Right-hand side f(y). Returns false when the state cannot be evaluated (the
// EOS gives T <= 0 or a non-finite value) or f is not finite.
template <int N>
__device__ __forceinline__ bool net_rhs(const DNet &net, const CellIn &c, const double *y,
                                        double *f) {
  const int S = net.S;
  double lnT = c.lnT, invT = c.invT;
  if (net.energy) {
    double X = 0.0;
    for (int i = 0; i < S; ++i) X += y[i];
    const double T = net.gm1 * y[S] / (KB_EV * X);
    if (!(T > 0.0) || !isfinite(T)) return false;
    lnT = log(T);
    invT = 1.0 / T;
  }
#pragma unroll
  for (int i = 0; i < N; ++i) f[i] = 0.0;
  double fu = 0.0;
  for (int r = 0; r < net.R; ++r) {
    const int4 s = __ldg(&net.side[r]);
    const RxPar &p = net.par[r];
    const double lnAf = __ldg(&p.lnAf), bf = __ldg(&p.bf), Cf = __ldg(&p.Cf);
    double kf = rexp(lnAf + bf * lnT - Cf * invT, net.exptab);
    double kr = 0.0;
    if (has_reverse(p)) kr = rexp(__ldg(&p.lnAr) + __ldg(&p.br) * lnT - __ldg(&p.Cr) * invT, net.exptab);
    if (c.ks) {
      const double sc = c.ks[r * c.ks_ld];
      kf *= sc;
      kr *= sc;
    }
    const double pf = (s.y < 0) ? y[s.x] : c.nd * y[s.x] * y[s.y];
    const double pr = (s.w < 0) ? y[s.z] : c.nd * y[s.z] * y[s.w];
    const double w = kf * pf - kr * pr;
    f[s.x] -= w;
    f[s.z] += w;
    if (s.y >= 0) f[s.y] -= w;
    if (s.w >= 0) f[s.w] += w;
    if (net.energy) fu += __ldg(&p.dE) * w;
  }
  if (net.energy) f[S] = fu;
  if (c.src) {
    // a constant source per component: the coupling term of a burn inside a
    // spectral-deferred-corrections step (Software design section, paragraph 4)
#pragma unroll
    for (int i = 0; i < N; ++i)
      if (i < net.n) f[i] += c.src[i * c.ks_ld];
  }
  bool ok = true;
#pragma unroll
  for (int i = 0; i < N; ++i)
    if (i < net.n && !finite64(f[i])) ok = false;
  return ok;
}

// Analytic Jacobian J[i*N + j] = d f_i / d y_j (row stride N), in FP64, one
// thread (the persistent workers evaluate it warp-cooperatively instead, see
// mc_coop.cuh). For the energy form T depends on the state through the EOS
// (dT/dx_j = -T / sum x, dT/du = (gamma-1) / (k_B sum x)); g_i = d f_i / dT at
// fixed x enters every column through that chain rule. dk/dT = k (b + C/T) / T.
template <int N>
__device__ __forceinline__ bool net_jac(const DNet &net, const CellIn &c, const double *y, double *J) {
  const int S = net.S, n = net.n;
  double lnT = c.lnT, invT = c.invT, T = 0.0, X = 0.0;
  if (net.energy) {
    for (int i = 0; i < S; ++i) X += y[i];
    T = net.gm1 * y[S] / (KB_EV * X);
    if (!(T > 0.0) || !isfinite(T)) return false;
    lnT = log(T);
    invT = 1.0 / T;
  }
  double g[N];
  for (int i = 0; i < n * N; ++i) J[i] = 0.0;
#pragma unroll
  for (int i = 0; i < N; ++i) g[i] = 0.0;
  for (int r = 0; r < net.R; ++r) {
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
    // column contributions d w / d x at fixed T, one per side slot
    const int col[4] = {s.x, s.y, s.z, s.w};
    double dw[4];
    double pf, pr;
    if (s.y < 0) { pf = y[s.x]; dw[0] = kf; dw[1] = 0.0; }
    else { pf = c.nd * y[s.x] * y[s.y]; dw[0] = kf * (c.nd * y[s.y]); dw[1] = kf * (c.nd * y[s.x]); }
    if (s.w < 0) { pr = y[s.z]; dw[2] = -kr; dw[3] = 0.0; }
    else { pr = c.nd * y[s.z] * y[s.w]; dw[2] = -kr * (c.nd * y[s.w]); dw[3] = -kr * (c.nd * y[s.z]); }
    const double dwdT = kf * (bf + Cf * invT) * invT * pf - kr * (br + Cr * invT) * invT * pr;
    const double sgn[4] = {-1.0, -1.0, 1.0, 1.0};
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      if (col[a] < 0) continue;
      const int row = col[a];
      g[row] += sgn[a] * dwdT;
#pragma unroll
      for (int b = 0; b < 4; ++b)
        if (col[b] >= 0) J[row * N + col[b]] += sgn[a] * dw[b];
    }
    if (net.energy) {
      const double dE = __ldg(&p.dE);
      g[S] += dE * dwdT;
#pragma unroll
      for (int b = 0; b < 4; ++b)
        if (col[b] >= 0) J[S * N + col[b]] += dE * dw[b];
    }
  }
  if (net.energy) {
    const double dTdx = -T / X, dTdu = net.gm1 / (KB_EV * X);
    for (int i = 0; i < n; ++i) {
      const double gx = g[i] * dTdx;
      for (int j = 0; j < S; ++j) J[i * N + j] += gx;
      J[i * N + S] += g[i] * dTdu;
    }
  }
  bool ok = true;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j)
      if (!finite64(J[i * N + j])) ok = false;
  return ok;
}

// Increment of the forward-difference Jacobian: d_j = sqrt(eps) (|y_j| + atol/rtol),
// eps the FP64 machine epsilon (sqrt(2^-52) = 2^-26 exactly).
constexpr double FD_SQRT_EPS = 1.4901161193847656e-08;

// Forward-difference Jacobian, column j = (f(y + d_j e_j) - f(y)) / d_j with
// d_j the representable step from y_j (the retry ladder's approximate
// Jacobian; one thread).
template <int N>
__device__ __forceinline__ bool net_fd_jac(const DNet &net, const CellIn &c, const double *y, double *J,
                                           double rtol, double atol) {
  const int n = net.n;
  double f0[N], f1[N], yp[N];
  if (!net_rhs<N>(net, c, y, f0)) return false;
  for (int j = 0; j < n; ++j) {
#pragma unroll
    for (int i = 0; i < N; ++i) yp[i] = (i < n) ? y[i] : 0.0;
    yp[j] = y[j] + FD_SQRT_EPS * (fabs(y[j]) + atol / rtol);
    const double dj = yp[j] - y[j];
    if (!(dj != 0.0)) return false;
    if (!net_rhs<N>(net, c, yp, f1)) return false;
    for (int i = 0; i < n; ++i) J[i * N + j] = (f1[i] - f0[i]) / dj;
  }
  return true;
}

// ---- dense LU with partial pivoting (first maximal |a| wins ties) ----------
// On return a holds L (unit diagonal, below) and U (above), with U's diagonal
// stored as its reciprocals so a solve multiplies instead of dividing.
template <int N, typename LT>
__device__ __forceinline__ bool lu_factor(int n, LT *a, unsigned char *piv) {
  for (int k = 0; k < n; ++k) {
    int p = k;
    LT best = fabs(a[k * N + k]);
    for (int i = k + 1; i < n; ++i) {
      const LT v = fabs(a[i * N + k]);
      if (v > best) { best = v; p = i; }
    }
    piv[k] = (unsigned char)p;
    if (best == (LT)0) return false;
    if (p != k)
      for (int j = 0; j < n; ++j) {
        const LT tmp = a[k * N + j];
        a[k * N + j] = a[p * N + j];
        a[p * N + j] = tmp;
      }
    const LT inv = (LT)1 / a[k * N + k];
    for (int i = k + 1; i < n; ++i) {
      const LT m = a[i * N + k] * inv;
      a[i * N + k] = m;
      for (int j = k + 1; j < n; ++j) a[i * N + j] -= m * a[k * N + j];
    }
    a[k * N + k] = inv;
  }
  return true;
}

// P = I - gamma J in the matrix precision (row stride N).
template <int N, typename LT>
__device__ __forceinline__ void form_p(int n, const double *J, double gamma, LT *P) {
  const LT g = (LT)gamma;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) P[i * N + j] = (i == j ? (LT)1 : (LT)0) - g * (LT)J[i * N + j];
}

// x = A^-1 b with the factors of lu_factor, in precision LT (b in FP64). The
// row interchanges go through a small indexed array; the triangular sweeps
// run on registers.
template <int N, typename LT>
__device__ __forceinline__ void lu_apply(int n, const LT *a, const unsigned char *piv, const double *bd, LT *x) {
  LT t[N];
#pragma unroll
  for (int i = 0; i < N; ++i) t[i] = (i < n) ? (LT)bd[i] : (LT)0;
  for (int k = 0; k < n; ++k) {
    const int p = piv[k];
    if (p != k) {
      const LT tmp = t[k];
      t[k] = t[p];
      t[p] = tmp;
    }
  }
  LT b[N];
#pragma unroll
  for (int i = 0; i < N; ++i) b[i] = t[i];
#pragma unroll
  for (int i = 1; i < N; ++i)
    if (i < n) {
      LT s = b[i];
#pragma unroll
      for (int j = 0; j < i; ++j) s -= a[i * N + j] * b[j];
      b[i] = s;
    }
#pragma unroll
  for (int i = N - 1; i >= 0; --i)
    if (i < n) {
      LT s = b[i];
#pragma unroll
      for (int j = i + 1; j < N; ++j)
        if (j < n) s -= a[i * N + j] * b[j];
      b[i] = s * a[i * N + i];
    }
#pragma unroll
  for (int i = 0; i < N; ++i) x[i] = b[i];
}

// ---- integrator state of one lane -------------------------------------------
enum Phase : int { PH_IDLE = 0, PH_F0, PH_HW, PH_NEWTON, PH_RESTART, PH_DONE };

struct Opts {
  double rtol, atol;
  int qmax, max_steps;
  int jac_fd;              // 1: forward-difference Jacobian instead of the analytic one
  int lane_matrix;         // 1: thread-per-cell lanes do their own matrix work (no warp cooperation)
};

template <int N, typename LT>
struct Lane {
  double z[QMAX + 1][N];   // Nordsieck array
  double e[N];             // accumulated correction
  double es[N];            // correction saved for the order-rise estimate
  double iw[N];            // 1 / error weight, from the start of the step
  double y[N];             // point at which f is wanted next
  double f[N];             // f(y)
  double J[N * N];         // Jacobian (FP64), kept between evaluations
  LT P[N * N];             // factored iteration matrix (see lu_factor)
  float iw32[N];           // iw in FP32, for the refinement's stopping test
  unsigned char piv[N];
  double l[QMAX + 1];
  double hist[QMAX + 3];   // accepted step sizes, most recent first
  double t, h, tend, crate, gamma_p, gamma, cq, esave_h, delp, eta_max, h0;
  double eta_pend;         // Nordsieck rescale factor the next begin_step applies
  double dsm;              // local-error norm of the last converged attempt
  CellIn cin;
  int64_t cell;
  int q, qwait, nef, ncf, jage, page, attempts, m, phase, status;
  int todo;                // next stage (Todo)
  bool need_j, need_p, jcur, have_es, last;
  bool want_j, want_p;     // matrix work the current Newton iteration waits for
  bool kept;               // hand-off refused (record list full): finish here
  int st[NSTAT];
};

// Mixed-precision iterative refinement of the FP32-matrix solve (Wilkinson
// 1963; C. B. Moler, J. ACM 14, 316-321, 1967): the FP32 factors act as a
// preconditioner, the residual r - (I - gamma_P J) d is formed in FP64 with the
// FP64 Jacobian, and the correction is added in FP64. Sweeps stop once the
// error-weighted max-norm of a correction is (or is predicted, from the
// contraction of the last two, to be) below REFINE_TOL of the solution's or
// below REFINE_ABS error-weight units outright, when the corrections stop
// shrinking, or after REFINE_MAX sweeps (late in a burn gamma J reaches 1e10
// and cond(P) 1e12, where a sweep contracts the error only by 0.05-0.2, so the
// cap leaves room for those). The Newton correction then equals the FP64
// solve's up to 1e-8 of a tolerance unit (Newton itself stops at about 0.1
// of one), so the FP32 form takes the FP64 form's Newton iterates and
// decisions.
constexpr int REFINE_MAX = 24;
constexpr float REFINE_TOL = 1e-10f;
constexpr float REFINE_ABS = 1e-8f;

// Newton correction: d <- (I - gamma_P J)^-1 d with the lane's factors.
// Returns false when the FP32 factors cannot reproduce the FP64 solve (the
// refinement stopped contracting or ran out of sweeps): the cell then goes to
// the FP64 retry pass.
template <int N, typename LT>
__device__ __forceinline__ bool newton_solve(const Lane<N, LT> &L, int n, double *d) {
  if constexpr (sizeof(LT) == sizeof(double)) {
    double x[N];
    lu_apply<N, double>(n, L.P, L.piv, d, x);
#pragma unroll
    for (int i = 0; i < N; ++i)
      if (i < n) d[i] = x[i];
    return true;
  } else {
    double r[N];
    float b[N];
#pragma unroll
    for (int i = 0; i < N; ++i) r[i] = (i < n) ? d[i] : 0.0;
    lu_apply<N, float>(n, L.P, L.piv, r, b);
    float nd = 0.0f;
#pragma unroll
    for (int i = 0; i < N; ++i)
      if (i < n) {
        d[i] = (double)b[i];
        nd = fmaxf(nd, fabsf(b[i]) * L.iw32[i]);
      }
    float np = nd;
    const double g = L.gamma_p;
    for (int k = 0; k < REFINE_MAX; ++k) {
      double s[N];
#pragma unroll
      for (int i = 0; i < N; ++i) {
        s[i] = 0.0;
        if (i < n) {
          double acc = 0.0;
#pragma unroll
          for (int j = 0; j < N; ++j)
            if (j < n) acc = fma(L.J[i * N + j], d[j], acc);
          s[i] = fma(g, acc, r[i] - d[i]);
        }
      }
      lu_apply<N, float>(n, L.P, L.piv, s, b);
      float nc = 0.0f;
#pragma unroll
      for (int i = 0; i < N; ++i)
        if (i < n) nc = fmaxf(nc, fabsf(b[i]) * L.iw32[i]);
      const float tol = fmaxf(REFINE_TOL * nd, REFINE_ABS);
      const bool done = nc <= tol;
      if (!done && !(nc < np)) return false;  // no longer contracting
#pragma unroll
      for (int i = 0; i < N; ++i)
        if (i < n) d[i] += (double)b[i];
      if (done || nc * (nc / np) <= tol) return true;
      np = nc;
    }
    return false;
  }
}

template <int N>
__device__ __forceinline__ double wrms(int n, const double *v, const double *iw) {
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < N; ++i)
    if (i < n) {
      const double r = v[i] * iw[i];
      s += r * r;
    }
  return sqrt(s / n);
}

template <int N, typename LT>
__device__ __forceinline__ void rescale(Lane<N, LT> &L, int n, double eta) {
  double r = 1.0;
  for (int j = 1; j <= L.q; ++j) {
    r *= eta;
#pragma unroll
    for (int i = 0; i < N; ++i)
      if (i < n) L.z[j][i] *= r;
  }
}

template <int N, typename LT>
__device__ __forceinline__ void predict(Lane<N, LT> &L, int n) {
  const int q = L.q;
  for (int k = 0; k < q; ++k)
    for (int j = q; j > k; --j)
#pragma unroll
      for (int i = 0; i < N; ++i)
        if (i < n) L.z[j - 1][i] += L.z[j][i];
}

template <int N, typename LT>
__device__ __forceinline__ void retract(Lane<N, LT> &L, int n) {
  const int q = L.q;
  for (int k = q - 1; k >= 0; --k)
    for (int j = k + 1; j <= q; ++j)
#pragma unroll
      for (int i = 0; i < N; ++i)
        if (i < n) L.z[j - 1][i] -= L.z[j][i];
}

// xi_j = (sum of the first j gaps)/h for j = 1..m (m <= QMAX + 2); loops are
// unrolled over the fixed maximum so the small arrays stay in registers
__device__ __forceinline__ void xi_of(double h, const double *gaps, int m, double *xi) {
  double s = 0.0;
  const double hinv = 1.0 / h;
#pragma unroll
  for (int j = 0; j < QMAX + 2; ++j)
    if (j < m) {
      s += gaps[j];
      xi[j] = s * hinv;
    }
}

// coefficients of x * prod_{i<k}(x + xi_i), k = number of factors (c[0..k], k <= QMAX + 1)
__device__ __forceinline__ void shifted_product(int k, const double *xi, double *c) {
#pragma unroll
  for (int j = 0; j < QMAX + 2; ++j) c[j] = 0.0;
  c[1] = 1.0;
#pragma unroll
  for (int i = 1; i <= QMAX; ++i) {
    if (i <= k - 1) {
      const double a = xi[i - 1];
#pragma unroll
      for (int j = QMAX + 1; j >= 1; --j)
        if (j <= i + 1) c[j] = c[j - 1] + a * c[j];
      c[0] = a * c[0];
    }
  }
}


// ---- step logic, staged ---------------------------------------------------
// advance() consumes f(y) and only records what the lane needs next (L.todo);
// run_stages() then runs each stage of the step logic from ONE call site, so
// lanes that reached the same stage by different paths execute it together
// once per loop trip instead of once per path. Factors that rescale the
// Nordsieck array are applied by begin_step (after the stage's own order
// change), in the same order the method defines: the stage's factor, then the
// final-step clip.
// TD_MATRIX: a Newton iteration waits for a Jacobian and/or factorisation;
// TD_CORRECT: it has f(y) and its matrix and takes the correction.
enum Todo : int { TD_NONE = 0, TD_BEGIN, TD_CONVERGED, TD_CONVFAIL, TD_REJECT, TD_ACCEPT, TD_SELECT,
                  TD_MATRIX, TD_CORRECT };

template <int N, typename LT>
__device__ __forceinline__ void finish(Lane<N, LT> &L, int status) {
  L.status = status;
  L.phase = PH_DONE;
  L.todo = TD_NONE;
}

// Start a step attempt (or finish the cell): pending rescale, clip the last
// step to t_end, weights from the accepted state, predict, variable-step
// coefficients.
template <int N, typename LT>
__device__ __forceinline__ void begin_step(Lane<N, LT> &L, const DNet &net, const Opts &o) {
  const int n = net.n;
  L.todo = TD_NONE;
  if (L.eta_pend != 1.0) {
    rescale(L, n, L.eta_pend);
    L.eta_pend = 1.0;
  }
  if (!(L.t < L.tend)) { finish(L, CELL_OK); return; }
  if (L.attempts >= o.max_steps) { finish(L, CELL_MAX_STEPS); return; }
  L.last = false;
  if (L.t + L.h >= L.tend) {
    const double hn = L.tend - L.t;
    rescale(L, n, hn / L.h);
    L.h = hn;
    L.last = true;
  }
  L.attempts += 1;
#pragma unroll
  for (int i = 0; i < N; ++i)
    if (i < n) {
      L.iw[i] = 1.0 / (o.rtol * fabs(L.z[0][i]) + o.atol);
      L.iw32[i] = (float)L.iw[i];
    }
  predict(L, n);
  const int q = L.q;
  double gaps[QMAX + 2], xi[QMAX + 2];
  gaps[0] = L.h;
#pragma unroll
  for (int k = 0; k < QMAX + 1; ++k) gaps[k + 1] = L.hist[k];
  xi_of(L.h, gaps, q + 1, xi);
  // l = coefficients of prod_{j<=q} (1 + x/xi_j)
  double l[QMAX + 1];
#pragma unroll
  for (int k = 0; k <= QMAX; ++k) l[k] = 0.0;
  l[0] = 1.0;
#pragma unroll
  for (int j = 1; j <= QMAX; ++j)
    if (j <= q) {
      const double c = 1.0 / xi[j - 1];
#pragma unroll
      for (int k = QMAX; k >= 1; --k)
        if (k <= j) l[k] += c * l[k - 1];
    }
  double xq = xi[0];
#pragma unroll
  for (int j = 1; j <= QMAX; ++j)
    if (j == q) xq = xi[j];
#pragma unroll
  for (int k = 0; k <= QMAX; ++k) L.l[k] = l[k];
  L.cq = (1.0 / xq) / l[1];
  L.gamma = L.h / l[1];
  L.jcur = false;
  L.m = 0;
#pragma unroll
  for (int i = 0; i < N; ++i)
    if (i < n) {
      L.e[i] = 0.0;
      L.y[i] = L.z[0][i];
    }
  L.phase = PH_NEWTON;
}

// Order drop q -> q-1 (z_j -= c_j z_q) with xi at the array's point.
template <int N, typename LT>
__device__ __forceinline__ void lower_order(Lane<N, LT> &L, int n, const double *xi) {
  double c[QMAX + 2];
  const int q = L.q;
  shifted_product(q, xi, c);
  for (int j = 1; j < q; ++j)
#pragma unroll
    for (int i = 0; i < N; ++i)
      if (i < n) L.z[j][i] -= c[j] * L.z[q][i];
  L.q = q - 1;
}

// est_{q-1} coefficient prod_{j<q} xi_j / sum_{j<q} 1/xi_j
__device__ __forceinline__ double qm1_coef(int q, const double *xi) {
  double prod = 1.0, l1 = 0.0;
#pragma unroll
  for (int j = 1; j <= QMAX; ++j)
    if (j <= q - 1) {
      prod *= xi[j - 1];
      l1 += 1.0 / xi[j - 1];
    }
  return prod / l1;
}

// Newton failure: undo the prediction, cut h by ETACF.
template <int N, typename LT>
__device__ __forceinline__ void stage_conv_failure(Lane<N, LT> &L, const DNet &net) {
  retract(L, net.n);
  L.ncf += 1;
  L.st[ST_CONV_FAILS] += 1;
  if (L.ncf >= MXNCF) { finish(L, CELL_CONV_FAIL); return; }
  L.eta_pend = ETACF;
  L.h *= ETACF;
  L.need_p = true;
  L.qwait = L.q + 1;
  L.have_es = false;
  if (L.t + L.h == L.t) { finish(L, CELL_H_UNDERFLOW); return; }
  L.todo = TD_BEGIN;
}

template <int N, typename LT>
__device__ __forceinline__ void stage_error_test(Lane<N, LT> &L, const DNet &net) {
  L.dsm = L.cq * wrms<N>(net.n, L.e, L.iw);
  L.todo = (L.dsm > 1.0) ? TD_REJECT : TD_ACCEPT;
}

// Local-error test failed: undo the prediction, then a smaller step (maybe
// one order lower), or after KFC failures a restart at order 1 (needs f(z_0)).
template <int N, typename LT>
__device__ __forceinline__ void stage_reject(Lane<N, LT> &L, const DNet &net) {
  const int n = net.n;
  const int q = L.q;
  retract(L, n);
  L.nef += 1;
  L.st[ST_ERR_FAILS] += 1;
  L.have_es = false;
  if (L.nef >= KFC) {
#pragma unroll
    for (int i = 0; i < N; ++i)
      if (i < n) L.y[i] = L.z[0][i];
    L.phase = PH_RESTART;
    L.todo = TD_NONE;
    return;
  }
  double eta = 1.0 / (root_k(BIAS_Q * L.dsm, q + 1, net.exptab) + ADDON);
  int qn = q;
  double xi[QMAX + 2];
  if (q > 1) {
    xi_of(L.h, L.hist, q, xi);
    const double est = qm1_coef(q, xi) * wrms<N>(n, L.z[q], L.iw);
    const double eta_m = 1.0 / (root_k(BIAS_QM1 * est, q, net.exptab) + ADDON);
    if (eta_m > eta) { eta = eta_m; qn = q - 1; }
  }
  eta = fmax(ETAMIN, fmin(eta, 1.0));
  if (qn < q) lower_order(L, n, xi);
  L.eta_pend = eta;
  L.h *= eta;
  L.qwait = L.q + 1;
  if (L.t + L.h == L.t) { finish(L, CELL_H_UNDERFLOW); return; }
  L.todo = TD_BEGIN;
}

template <int N, typename LT>
__device__ __forceinline__ void stage_accept(Lane<N, LT> &L, const DNet &net, const Opts &o) {
  const int n = net.n;
  const int q = L.q;
  for (int j = 0; j <= q; ++j)
#pragma unroll
    for (int i = 0; i < N; ++i)
      if (i < n) L.z[j][i] += L.l[j] * L.e[i];
  L.t = L.last ? L.tend : L.t + L.h;
#pragma unroll
  for (int k = QMAX + 2; k > 0; --k) L.hist[k] = L.hist[k - 1];
  L.hist[0] = L.h;
  L.st[ST_STEPS] += 1;
  L.nef = 0;
  L.ncf = 0;
  L.jage += 1;
  L.page += 1;
  L.qwait -= 1;
  if (L.qwait == 1 && q < o.qmax) {
#pragma unroll
    for (int i = 0; i < N; ++i)
      if (i < n) L.es[i] = L.e[i];
    L.esave_h = L.h;
    L.have_es = true;
  }
  if (L.last) { finish(L, CELL_OK); return; }
  L.todo = (L.qwait > 0) ? TD_BEGIN : TD_SELECT;
}

// Step size and order selection from the q-1, q, q+1 estimates.
template <int N, typename LT>
__device__ __forceinline__ void stage_select(Lane<N, LT> &L, const DNet &net, const Opts &o) {
  const int n = net.n;
  const int q = L.q;
  double xi[QMAX + 2];
  double eta = 1.0 / (root_k(BIAS_Q * L.dsm, q + 1, net.exptab) + ADDON);
  int qn = q;
  xi_of(L.h, L.hist, q + 1, xi);
  if (q > 1) {
    const double est = qm1_coef(q, xi) * wrms<N>(n, L.z[q], L.iw);
    const double eta_m = 1.0 / (root_k(BIAS_QM1 * est, q, net.exptab) + ADDON);
    if (eta_m > eta) { eta = eta_m; qn = q - 1; }
  }
  if (q < o.qmax && L.have_es) {
    const double r = ipow(L.h / L.esave_h, q + 1);
    double dv[N];
#pragma unroll
    for (int i = 0; i < N; ++i) dv[i] = (i < n) ? L.e[i] - r * L.es[i] : 0.0;
    const double est = wrms<N>(n, dv, L.iw) / ((double)(q + 2) * harmonic(q + 1));
    const double eta_p = 1.0 / (root_k(BIAS_QP1 * est, q + 2, net.exptab) + ADDON);
    if (eta_p > eta) { eta = eta_p; qn = q + 1; }
  }
  L.have_es = false;
  L.todo = TD_BEGIN;
  if (eta < THRESH) {
    L.qwait = 2;
    return;
  }
  eta = fmin(eta, L.eta_max);
  L.eta_max = ETAMX;
  if (qn > q) {
    double prod = 1.0, c[QMAX + 2];
#pragma unroll
    for (int j = 1; j <= QMAX + 1; ++j)
      if (j <= q + 1) prod *= xi[j - 1];
    const double C = 1.0 / prod;
    shifted_product(q + 1, xi, c);
#pragma unroll
    for (int i = 0; i < N; ++i)
      if (i < n) L.z[q + 1][i] = 0.0;
    for (int j = 1; j <= q + 1; ++j)
#pragma unroll
      for (int i = 0; i < N; ++i)
        if (i < n) L.z[j][i] += c[j] * C * L.e[i];
    L.q = q + 1;
  } else if (qn < q) {
    lower_order(L, n, xi);
  }
  L.eta_pend = eta;
  L.h *= eta;
  L.qwait = L.q + 1;
}

// One modified-Newton correction with f = f(y) just evaluated and the matrix
// work of the iteration done. 0 = continue, 1 = converged, 2 = failed,
// 3 = failed (could not evaluate), 7 = handed to the FP64 retry.
template <int N, typename LT>
__device__ __forceinline__ int newton_correct(Lane<N, LT> &L, const DNet &net) {
  const int n = net.n;
  double d[N];
  const double rl1 = 1.0 / L.l[1];
#pragma unroll
  for (int i = 0; i < N; ++i) d[i] = (i < n) ? (L.h * L.f[i] - L.z[1][i]) * rl1 - L.e[i] : 0.0;
  if (!newton_solve<N, LT>(L, n, d)) {
    finish(L, CELL_RETRY64);
    return 7;
  }
  L.st[ST_NEWTON] += 1;
  if (L.gamma != L.gamma_p) {
    const double sc = 2.0 / (1.0 + L.gamma / L.gamma_p);
#pragma unroll
    for (int i = 0; i < N; ++i) d[i] *= sc;
  }
  const double del = wrms<N>(n, d, L.iw);
#pragma unroll
  for (int i = 0; i < N; ++i)
    if (i < n) {
      L.e[i] += d[i];
      L.y[i] = L.z[0][i] + L.e[i];
    }
  if (L.m > 0) L.crate = fmax(CRDOWN * L.crate, del / L.delp);
  const double dcon = del * fmin(1.0, L.crate) * L.cq / CORTES;
  if (dcon <= 1.0) return 1;
  L.m += 1;
  if (L.m == MAXCOR || (L.m >= 2 && del > RDIV * L.delp)) return 2;
  L.delp = del;
  return 0;
}

// Consume f(y) of a Newton iteration. The first iteration of an attempt may
// need a new Jacobian (first step, every MSBJ steps, after a stale-Jacobian
// failure) and a new factorisation of P = I - gamma J (then, every MSBP steps,
// or when gamma drifted more than CCMAX from the factored one): it returns 4
// with want_j / want_p set, and the caller does that work (one thread:
// matrix_thread; a warp: coop_matrix) and continues with newton_after_matrix.
// Otherwise 5: the correction is next (newton_correct); 3: f could not be
// evaluated.
template <int N, typename LT>
__device__ __forceinline__ int newton_iter(Lane<N, LT> &L, bool ok) {
  if (!ok) return 3;
  L.st[ST_RHS] += 1;
  if (L.m == 0) {
    L.want_j = L.need_j || L.jage >= MSBJ;
    L.want_p = L.want_j || L.need_p || L.page >= MSBP || fabs(L.gamma / L.gamma_p - 1.0) > CCMAX;
    if (L.want_p) return 4;
  }
  return 5;
}

// Bookkeeping after the matrix work (jok: the Jacobian, if wanted, is finite;
// pok: P is factored): 5 (the correction is next), 2 (singular matrix) or 3.
template <int N, typename LT>
__device__ __forceinline__ int newton_after_matrix(Lane<N, LT> &L, bool jok, bool pok) {
  if (L.want_j) {
    if (!jok) return 3;
    L.st[ST_JAC] += 1;
    L.jcur = true;
    L.need_j = false;
    L.jage = 0;
  }
  L.st[ST_LU] += 1;
  L.gamma_p = L.gamma;
  L.page = 0;
  L.need_p = false;
  L.crate = CRATE0;
  if (!pok) {
    L.need_p = true;
    return 2;
  }
  return 5;
}

// What a Newton iteration's outcome r asks for next (sets L.todo).
template <int N, typename LT>
__device__ __forceinline__ void newton_outcome(Lane<N, LT> &L, int n, int r) {
  L.todo = TD_NONE;
  if (r == 0 || r == 7) return;  // 7: the cell went to the FP64 retry (finished here)
  if (r == 1) { L.todo = TD_CONVERGED; return; }
  if (r == 4) { L.todo = TD_MATRIX; return; }
  if (r == 5) { L.todo = TD_CORRECT; return; }
  if (r == 2 && !L.jcur) {
    // stale Jacobian: refresh it and redo the corrector from the prediction
    L.need_j = true;
    L.m = 0;
#pragma unroll
    for (int i = 0; i < N; ++i)
      if (i < n) {
        L.e[i] = 0.0;
        L.y[i] = L.z[0][i];
      }
    return;
  }
  L.todo = TD_CONVFAIL;
}

// The matrix work of a waiting Newton iteration done by the lane itself.
template <int N, typename LT>
__device__ __forceinline__ void matrix_thread(Lane<N, LT> &L, const DNet &net, const Opts &o) {
  bool jok = true, pok = false;
  if (L.want_j)
    jok = o.jac_fd ? net_fd_jac<N>(net, L.cin, L.y, L.J, o.rtol, o.atol) : net_jac<N>(net, L.cin, L.y, L.J);
  if (jok) {
    form_p<N, LT>(net.n, L.J, L.gamma, L.P);
    pok = lu_factor<N, LT>(net.n, L.P, L.piv);
  }
  newton_outcome(L, net.n, newton_after_matrix(L, jok, pok));
}

// Consume f(y) according to the lane's phase; record what comes next.
template <int N, typename LT>
__device__ __forceinline__ void advance(Lane<N, LT> &L, const DNet &net, const Opts &o, bool ok) {
  const int n = net.n;
  L.todo = TD_NONE;
  if (L.phase == PH_NEWTON) {
    newton_outcome(L, n, newton_iter<N, LT>(L, ok));
    return;
  }
  if (L.phase == PH_F0) {
    if (!ok) { finish(L, CELL_BAD_INPUT); return; }
    L.st[ST_RHS] += 1;
    // starting step (Hairer, Norsett & Wanner, Solving ODEs I, II.4), p = 1
#pragma unroll
    for (int i = 0; i < N; ++i)
      if (i < n) L.iw[i] = 1.0 / (o.rtol * fabs(L.z[0][i]) + o.atol);
    const double d0 = wrms<N>(n, L.z[0], L.iw), d1 = wrms<N>(n, L.f, L.iw);
    double h0 = (d0 < 1e-5 || d1 < 1e-5) ? 1e-6 : 0.01 * d0 / d1;
    h0 = fmin(h0, L.tend);
    L.h0 = h0;
#pragma unroll
    for (int i = 0; i < N; ++i)
      if (i < n) {
        L.e[i] = L.f[i];  // f0 parked in e
        L.y[i] = L.z[0][i] + h0 * L.f[i];
      }
    L.st[ST_RHS] += 1;
    L.phase = PH_HW;
    return;
  }
  if (L.phase == PH_HW) {
    double h = L.h0;
    if (ok) {
      double dv[N];
#pragma unroll
      for (int i = 0; i < N; ++i) dv[i] = (i < n) ? L.f[i] - L.e[i] : 0.0;
      const double d1 = wrms<N>(n, L.e, L.iw);
      const double d2 = wrms<N>(n, dv, L.iw) / L.h0;
      const double dm = fmax(d1, d2);
      const double h1 = (dm <= 1e-15) ? fmax(1e-6, L.h0 * 1e-3) : sqrt(0.01 / dm);
      h = fmin(fmin(100.0 * L.h0, h1), L.tend);
    }
    L.h = h;
#pragma unroll
    for (int i = 0; i < N; ++i)
      if (i < n) L.z[1][i] = h * L.e[i];
    L.t = 0.0;
    L.q = 1;
    L.qwait = 2;
#pragma unroll
    for (int k = 0; k < QMAX + 3; ++k) L.hist[k] = h;
    L.need_j = true;
    L.need_p = true;
    L.crate = CRATE0;
    L.gamma_p = 1.0;
    L.eta_max = ETAMX_FIRST;
    L.eta_pend = 1.0;
    L.nef = L.ncf = 0;
    L.jage = L.page = 0;
    L.have_es = false;
    L.attempts = 0;
    L.todo = TD_BEGIN;
    return;
  }
  if (L.phase == PH_RESTART) {
    if (!ok) { finish(L, CELL_NONFINITE); return; }
    L.st[ST_RHS] += 1;
    L.h *= ETAMIN;
    L.q = 1;
#pragma unroll
    for (int i = 0; i < N; ++i)
      if (i < n) L.z[1][i] = L.h * L.f[i];
    L.qwait = 2;
    if (L.t + L.h == L.t) { finish(L, CELL_H_UNDERFLOW); return; }
    L.todo = TD_BEGIN;
  }
}

// The stages, each from exactly one call site (TD_MATRIX is resolved before).
template <int N, typename LT>
__device__ __forceinline__ void run_stages(Lane<N, LT> &L, const DNet &net, const Opts &o) {
  if (L.todo == TD_CORRECT) newton_outcome(L, net.n, newton_correct(L, net));
  if (L.todo == TD_CONVFAIL) stage_conv_failure(L, net);
  if (L.todo == TD_CONVERGED) stage_error_test(L, net);
  if (L.todo == TD_REJECT) stage_reject(L, net);
  if (L.todo == TD_ACCEPT) stage_accept(L, net, o);
  if (L.todo == TD_SELECT) stage_select(L, net, o);
  if (L.todo == TD_BEGIN) begin_step(L, net, o);
}

}  // namespace mc
