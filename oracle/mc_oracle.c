/*
 * mc_oracle.c -- plain, slow FP64 CPU oracle for the per-cell burn.
 *
 * TEST INFRASTRUCTURE. Only tests/, the package smoke check and the
 * benchmark's CPU-baseline leg may load or call this file. It shares no code,
 * header, table or constant generator with the CUDA path, and the CUDA path
 * never calls it.
 *
 * What it computes. The paper's burn (Software design section, paragraphs 2-4)
 * integrates one zone's reaction network over an operator-split step dt with
 * a C++ port of VODE (Brown, Byrne & Hindmarsh 1989), caps the number of
 * steps and hands failures back to the caller. The paper gives no algorithmic
 * detail of VODE, so every integrator rule below is the builder's restatement
 * of the published variable-coefficient BDF method in Nordsieck form, derived
 * from the mathematics:
 *
 *   z_j = h^j y^(j) / j!              Nordsieck history, j = 0..q, q <= 5: the
 *                                     polynomial through the last q+1 values
 *   predict      z <- z * Pascal      (Taylor shift by h)
 *   correct      z <- z + e * l       l = coefficients of
 *                Lambda(x) = prod_{j=1}^{q} (1 + x/xi_j), xi_j = (t_n - t_{n-j}) / h
 *   corrector    G(e) = h f(z_0 + e) - z_1 - l_1 e = 0, modified Newton with
 *                P = I - gamma J, gamma = h / l_1
 *   error        est_q = e (1/xi_{q+1}) / l_1
 *
 * Each function below names what it follows. Pins (tests/test_oracle_*.py):
 * Robertson values at t = 40, the A->B->C closed form, element and energy
 * conservation, brute-force backward Euler, exactness of the step on
 * polynomials, exactness of the q and q-1 error estimates, the q+1 estimate's
 * limit, the order of convergence, the starting step's closed form on linear
 * problems, the modified Newton correction (one exact correction on a linear
 * problem with a current matrix; the contraction factor of the scaled
 * correction with a matrix formed at another gamma), the step-size rule's
 * target (after a step change at order 1 the error estimates settle at
 * 1/BIAS_q = 1/6; after an order raise at 1/BIAS_q+1 = 1/10), the Jacobian
 * against finite differences, and the LU against the definition.
 *
 * Failure retry (same paragraph 3: a failed zone may be integrated again under
 * other tolerances or with an approximate Jacobian): a forward-difference
 * Jacobian (pinned exact on a
 * linear chain up to rounding, to its closed-form error on Robertson, to the
 * analytic Jacobian, and through Robertson's published values) and a per-cell
 * retry ladder (pinned against the plain burn of each rung).
 *
 * Alternative integrator (paragraph 4's network/integrator separation): RKC,
 * explicit Runge-Kutta-Chebyshev of order 2 (pinned to its closed-form
 * stability polynomial, its order, closed forms and Robertson's values).
 *
 * Coupling by spectral deferred corrections (paragraph 4): an optional
 * constant source per cell and component added to the right-hand side
 * (pinned to straight lines, to a matrix exponential, to element totals).
 *
 * Parity unpinned: the rest of the step-control policy (the bounds of the
 * step-size factors, when h and q may change, the Newton convergence
 * constants, the Jacobian/matrix reuse ages, the failure ladders). These are
 * heuristics with no closed form; they are checked only through solution
 * accuracy and through parity with the independent CUDA implementation of the
 * same rules.
 */
#include <float.h>
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_NMAX 40   /* largest ODE count handled (32 species + energy = 33) */
#define OR_QMAX 5    /* highest BDF order */
#define OR_RMAX 512  /* largest reaction count */

/* ---- integrator policy constants (builder's readings; paper silent) ---- */
#define OR_MAXCOR 3        /* Newton corrections per attempt */
#define OR_RDIV 2.0        /* divergence: del > RDIV * previous del */
#define OR_CRDOWN 0.3      /* convergence-rate memory */
#define OR_CORTES 0.1      /* Newton error allowed, as a share of the local error */
#define OR_CRATE0 0.7      /* convergence-rate estimate after a new matrix */
#define OR_ETACF 0.25      /* step factor after a Newton failure */
#define OR_MXNCF 10        /* consecutive Newton failures before giving up */
#define OR_KFC 3           /* consecutive error failures before an order-1 restart */
#define OR_ETAMIN 0.1      /* smallest step factor after an error failure */
#define OR_BIAS_QM1 6.0
#define OR_BIAS_Q 6.0
#define OR_BIAS_QP1 10.0
#define OR_ADDON 1.0e-6
#define OR_THRESH 1.5      /* smallest step growth worth a change */
#define OR_ETAMX_FIRST 1.0e4
#define OR_ETAMX 10.0
#define OR_MSBJ 50         /* accepted steps between Jacobian evaluations */
#define OR_MSBP 20         /* accepted steps between matrix factorisations */
#define OR_CCMAX 0.3       /* refactor when |gamma/gamma_P - 1| exceeds this */

/* per-cell status codes */
enum { OR_OK = 0, OR_MAX_STEPS = 1, OR_H_UNDERFLOW = 2, OR_CONV_FAIL = 3,
       OR_BAD_INPUT = 4, OR_NONFINITE = 5 };

/* stats layout: one int32 per entry */
enum { ST_STEPS = 0, ST_ERR_FAILS, ST_CONV_FAILS, ST_RHS, ST_JAC, ST_LU,
       ST_NEWTON, ST_ORDER, OR_NSTAT };

/* ------------------------------------------------------------------------ */
/* Generic ODE interface: the network/integrator separation of the Software  */
/* design section (paragraph 4): any right-hand side with its Jacobian.      */
/* ------------------------------------------------------------------------ */
typedef struct {
    int n;
    int (*rhs)(void *ctx, double t, const double *y, double *f);  /* 0 = ok */
    int (*jac)(void *ctx, double t, const double *y, double *J);  /* row-major n x n */
    void *ctx;
} or_ode;

typedef struct {
    double rtol, atol;
    int max_order, max_steps;
    int jac_fd;        /* 1: forward-difference Jacobian instead of the analytic one */
    int method;        /* 0: BDF (the paper's VODE-style integrator), 1: RKC */
    double *steplog;   /* optional record of accepted steps (the pins' view):      */
    int steplog_cap;   /* (t after the step, h, q, error estimate) per step, at    */
    int *steplog_n;    /* most steplog_cap of them; *steplog_n counts them         */
} or_opts;

static double harmonic(int k)
{
    double s = 0.0;
    for (int j = 1; j <= k; ++j) s += 1.0 / j;
    return s;
}

/* Weighted root-mean-square norm sqrt(sum (v_i / w_i)^2 / n), summed in index
   order. */
static double wrms(int n, const double *v, const double *w)
{
    double s = 0.0;
    for (int i = 0; i < n; ++i) {
        double r = v[i] / w[i];
        s += r * r;
    }
    return sqrt(s / n);
}

/* Error weights w_i = rtol |y_i| + atol. */
static void weights(int n, const double *y, double rtol, double atol, double *w)
{
    for (int i = 0; i < n; ++i) w[i] = rtol * fabs(y[i]) + atol;
}

static int all_finite(int n, const double *v)
{
    for (int i = 0; i < n; ++i)
        if (!isfinite(v[i])) return 0;
    return 1;
}

/* ------------------------------------------------------------------------ */
/* Dense LU with partial pivoting (Doolittle, in place, row-major). The     */
/* pivot is the first entry of largest magnitude (lowest row on ties).      */
/* Returns 0, or 1 if a pivot is exactly zero.                              */
/* ------------------------------------------------------------------------ */
int or_lu_factor(int n, double *a, int *piv)
{
    for (int k = 0; k < n; ++k) {
        int p = k;
        double best = fabs(a[k * n + k]);
        for (int i = k + 1; i < n; ++i) {
            double v = fabs(a[i * n + k]);
            if (v > best) { best = v; p = i; }
        }
        piv[k] = p;
        if (best == 0.0) return 1;
        if (p != k)
            for (int j = 0; j < n; ++j) {
                double tmp = a[k * n + j];
                a[k * n + j] = a[p * n + j];
                a[p * n + j] = tmp;
            }
        for (int i = k + 1; i < n; ++i) {
            double m = a[i * n + k] / a[k * n + k];
            a[i * n + k] = m;
            for (int j = k + 1; j < n; ++j) a[i * n + j] -= m * a[k * n + j];
        }
    }
    return 0;
}

/* Solve (LU) x = P b in place: row swaps in factor order, then forward
   substitution with the unit lower factor, then back substitution. */
void or_lu_solve(int n, const double *lu, const int *piv, double *b)
{
    for (int k = 0; k < n; ++k)
        if (piv[k] != k) {
            double tmp = b[k];
            b[k] = b[piv[k]];
            b[piv[k]] = tmp;
        }
    for (int i = 1; i < n; ++i) {
        double s = b[i];
        for (int j = 0; j < i; ++j) s -= lu[i * n + j] * b[j];
        b[i] = s;
    }
    for (int i = n - 1; i >= 0; --i) {
        double s = b[i];
        for (int j = i + 1; j < n; ++j) s -= lu[i * n + j] * b[j];
        b[i] = s / lu[i * n + i];
    }
}

/* ------------------------------------------------------------------------ */
/* BDF coefficients (paper silent; restated from the BDF mathematics).      */
/* ------------------------------------------------------------------------ */

/* xi_j = (sum of the first j gaps) / h, j = 1..m, written to xi[0..m-1]. The
   gaps run backwards from the point the Nordsieck array is taken at. */
void or_xi_from_gaps(double h, const double *gaps, int m, double *xi)
{
    double s = 0.0;
    for (int j = 0; j < m; ++j) {
        s += gaps[j];
        xi[j] = s / h;
    }
}

/* Corrector vector l[0..q] of the variable-coefficient BDF of order q: the
   coefficients of Lambda(x) = prod_{j=1}^{q} (1 + x/xi_j), which vanishes at
   the q previous points, so that P_n = P_{n-1} + e Lambda keeps interpolating
   the last q+1 values; l_1 = sum_{j<=q} 1/xi_j.

   Also returns the local-error coefficient cq. For a solution that is a
   polynomial of degree q+1 with leading coefficient a, the predictor misses
   y(t_n) by d = a prod_{j=1}^{q+1}(t_n - t_{n-j}), and one step from exact back
   values has local error d (S/l_1 - 1) = d (1/xi_{q+1}) / l_1,
   S = sum_{i<=q+1} 1/xi_i. Once earlier local errors have settled into a smooth
   global error the correction e of a step equals that predictor miss, so the
   error estimate is cq e with cq = (1/xi_{q+1}) / l_1; at constant steps this is
   the textbook constant 1/((q+1) G_q). xi[0..q] holds xi_1..xi_{q+1}. */
void or_bdf_coeffs(int q, const double *xi, double *l, double *cq)
{
    double poly[OR_QMAX + 2];
    for (int k = 0; k <= q; ++k) poly[k] = 0.0;
    poly[0] = 1.0;
    for (int j = 1; j <= q; ++j) {
        double c = 1.0 / xi[j - 1];
        for (int k = j; k >= 1; --k) poly[k] += c * poly[k - 1];
    }
    for (int k = 0; k <= q; ++k) l[k] = poly[k];
    *cq = (1.0 / xi[q]) / l[1];
}

/* Coefficient c with est_{q-1} = c z_q: the local error an order q-1 step of
   the same size would have made, for a solution that is a polynomial of
   degree q with history on it. With a = z_q / h^q that error is
   a prod_{j<=q}(t_n - t_{n-j}) (1/xi_q) / l'_1, l'_1 = sum_{j<q} 1/xi_j, so
   c = prod_{j<q} xi_j / l'_1 (q >= 2). xi[0..q-1] = xi_1..xi_q at the
   Nordsieck point. */
double or_err_coef_qm1(int q, const double *xi)
{
    double prod = 1.0, l1 = 0.0;
    for (int j = 1; j <= q - 1; ++j) {
        prod *= xi[j - 1];
        l1 += 1.0 / xi[j - 1];
    }
    return prod / l1;
}

/* Coefficient c with est_{q+1} = c (e_n - (h_n/h_{n-1})^{q+1} e_{n-1}): with
   e_n ~ h^{q+1} y^(q+1) (the settled correction above), the difference of two
   corrections estimates h^{q+2} y^(q+2), and the order q+1 local error is
   h^{q+2} y^(q+2) / ((q+2) G_{q+1}). */
double or_err_coef_qp1(int q)
{
    return 1.0 / ((double)(q + 2) * harmonic(q + 1));
}

/* Order rise q -> q+1: the degree q+1 polynomial Q through the new value and
   the q+1 previous points differs from P_n by C x prod_{i=1}^{q} (x + xi_i),
   whose leading coefficient is C = e_n / prod_{j=1}^{q+1} xi_j. Returns
   1 / prod xi_j; the column update itself uses or_order_lower_coefs(q+1, xi). */
double or_order_raise_coef(int q, const double *xi)
{
    double prod = 1.0;
    for (int j = 1; j <= q + 1; ++j) prod *= xi[j - 1];
    return 1.0 / prod;
}

/* Order drop q -> q-1: z_j -= c_j z_q (j = 1..q), where c_j are the
   coefficients of x prod_{i=1}^{q-1} (x + xi_i); the result is the degree q-1
   polynomial through the current point and the q-1 previous points.
   c[0..q] is written (c[0] = 0, c[q] = 1). */
void or_order_lower_coefs(int q, const double *xi, double *c)
{
    double poly[OR_QMAX + 2];
    for (int k = 0; k <= q; ++k) poly[k] = 0.0;
    poly[1] = 1.0;          /* x */
    int deg = 1;
    for (int i = 1; i <= q - 1; ++i) {
        double a = xi[i - 1];
        /* multiply by (x + a) */
        for (int k = deg + 1; k >= 1; --k) poly[k] = poly[k - 1] + a * poly[k];
        poly[0] = a * poly[0];
        deg += 1;
    }
    for (int k = 0; k <= q; ++k) c[k] = poly[k];
}

/* Taylor shift of the Nordsieck array by one step: z <- z * Pascal. */
void or_predict(int n, int q, double *z /* [(q+1) * n] */)
{
    for (int k = 0; k < q; ++k)
        for (int j = q; j > k; --j)
            for (int i = 0; i < n; ++i) z[(j - 1) * n + i] += z[j * n + i];
}

/* Exact reverse of or_predict's additions (undo the prediction). */
void or_retract(int n, int q, double *z)
{
    for (int k = q - 1; k >= 0; --k)
        for (int j = k + 1; j <= q; ++j)
            for (int i = 0; i < n; ++i) z[(j - 1) * n + i] -= z[j * n + i];
}

/* z_j <- eta^j z_j, j = 1..q (new step h * eta). */
static void rescale(int n, int q, double *z, double eta)
{
    double r = 1.0;
    for (int j = 1; j <= q; ++j) {
        r *= eta;
        for (int i = 0; i < n; ++i) z[j * n + i] *= r;
    }
}

/* ------------------------------------------------------------------------ */
/* The integrator.                                                           */
/* ------------------------------------------------------------------------ */
typedef struct {
    int n, q, qwait, nef, ncf, jage, page, need_j, need_p, have_esave, jcur;
    double t, h, eta_max, crate, gamma_p;
    double z[(OR_QMAX + 2) * OR_NMAX];
    double hist[OR_QMAX + 3];
    double esave[OR_NMAX], esave_h;
    double J[OR_NMAX * OR_NMAX], P[OR_NMAX * OR_NMAX];
    int piv[OR_NMAX];
    int32_t *st;
    double *trace;     /* optional: e after each Newton correction (the pins' record) */
    int ntrace;
} or_bdf;

enum { NW_CONVERGED = 0, NW_FAIL = 1, NW_FAIL_RHS = 2 };

/* Modified Newton on G(e) = h f(z_0 + e) - z_1 - l_1 e = 0 (z predicted):
   delta = P^{-1} [(h f(y) - z_1)/l_1 - e], e += delta, where P = I - gamma J was
   formed at gamma_P; with gamma != gamma_P, delta is scaled by
   2 / (1 + gamma/gamma_P). Converged when del * min(1, rate) * cq / CORTES <= 1
   (the remaining Newton error, as a local-error estimate, is a tenth of the
   tolerance); fails after MAXCOR corrections or when del grows by more than
   RDIV. The Jacobian is refreshed at the first iteration when it is due and
   the matrix is refactored when gamma drifted or it is due. */
static int newton(or_bdf *s, const or_ode *ode, const double *w, const double *l,
                  double cq, double gamma, double *e, double *y)
{
    const int n = s->n;
    double f[OR_NMAX], d[OR_NMAX];
    double delp = 0.0;
    for (int i = 0; i < n; ++i) { e[i] = 0.0; y[i] = s->z[i]; }
    for (int m = 0;;) {
        if (ode->rhs(ode->ctx, s->t + s->h, y, f) != 0 || !all_finite(n, f)) return NW_FAIL_RHS;
        s->st[ST_RHS] += 1;
        if (m == 0) {
            int newp = 0;
            if (s->need_j || s->jage >= OR_MSBJ) {
                if (ode->jac(ode->ctx, s->t + s->h, y, s->J) != 0 || !all_finite(n * n, s->J))
                    return NW_FAIL_RHS;
                s->st[ST_JAC] += 1;
                s->jcur = 1;
                s->need_j = 0;
                s->jage = 0;
                newp = 1;
            }
            if (newp || s->need_p || s->page >= OR_MSBP || fabs(gamma / s->gamma_p - 1.0) > OR_CCMAX) {
                for (int i = 0; i < n; ++i)
                    for (int j = 0; j < n; ++j)
                        s->P[i * n + j] = (i == j ? 1.0 : 0.0) - gamma * s->J[i * n + j];
                s->st[ST_LU] += 1;
                s->gamma_p = gamma;
                s->page = 0;
                s->need_p = 0;
                s->crate = OR_CRATE0;
                if (or_lu_factor(n, s->P, s->piv) != 0) {
                    s->need_p = 1;
                    return NW_FAIL;
                }
            }
        }
        for (int i = 0; i < n; ++i) d[i] = (s->h * f[i] - s->z[n + i]) / l[1] - e[i];
        or_lu_solve(n, s->P, s->piv, d);
        s->st[ST_NEWTON] += 1;
        if (gamma != s->gamma_p) {
            double sc = 2.0 / (1.0 + gamma / s->gamma_p);
            for (int i = 0; i < n; ++i) d[i] *= sc;
        }
        double del = wrms(n, d, w);
        for (int i = 0; i < n; ++i) {
            e[i] += d[i];
            y[i] = s->z[i] + e[i];
        }
        if (s->trace && s->ntrace < OR_MAXCOR) {
            for (int i = 0; i < n; ++i) s->trace[s->ntrace * n + i] = e[i];
            s->ntrace += 1;
        }
        if (m > 0) s->crate = fmax(OR_CRDOWN * s->crate, del / delp);
        double dcon = del * fmin(1.0, s->crate) * cq / OR_CORTES;
        if (dcon <= 1.0) return NW_CONVERGED;
        m += 1;
        if (m == OR_MAXCOR || (m >= 2 && del > OR_RDIV * delp)) return NW_FAIL;
        delp = del;
    }
}

/* Starting step of Hairer, Norsett & Wanner (Solving ODEs I, sec. II.4) with
   p = 1: h0 from |y0| / |f0|, a trial Euler step for a second-derivative
   estimate, then min(100 h0, (0.01 / max(d1, d2))^(1/2), span). */
static double initial_step(const or_ode *ode, double t0, double span, const double *y0,
                           const double *f0, const double *w, int32_t *st)
{
    const int n = ode->n;
    double d0 = wrms(n, y0, w), d1 = wrms(n, f0, w);
    double h0 = (d0 < 1e-5 || d1 < 1e-5) ? 1e-6 : 0.01 * d0 / d1;
    h0 = fmin(h0, span);
    double y1[OR_NMAX] = {0.0}, f1[OR_NMAX];
    for (int i = 0; i < n; ++i) y1[i] = y0[i] + h0 * f0[i];
    st[ST_RHS] += 1;
    if (ode->rhs(ode->ctx, t0 + h0, y1, f1) != 0 || !all_finite(n, f1)) return h0;
    for (int i = 0; i < n; ++i) f1[i] -= f0[i];
    double d2 = wrms(n, f1, w) / h0;
    double dm = fmax(d1, d2);
    double h1 = (dm <= 1e-15) ? fmax(1e-6, h0 * 1e-3) : sqrt(0.01 / dm);
    return fmin(fmin(100.0 * h0, h1), span);
}

/* Integrate y' = f(t, y) from t0 to t1 (t1 > t0) with the BDF above; y holds
   y(t0) on entry and y(t1) on success. st[0..OR_NSTAT-1] receives counters.
   Returns a per-cell status code. The step cap and the hand-back of failures
   follow the Software design section (paragraph 3). */
int or_bdf_integrate(const or_ode *ode, const or_opts *o, double t0, double t1, double *y,
                     int32_t *st)
{
    or_bdf S, *s = &S;
    const int n = ode->n;
    const int qmax = o->max_order < 1 ? 1 : (o->max_order > OR_QMAX ? OR_QMAX : o->max_order);
    double w[OR_NMAX], f0[OR_NMAX], e[OR_NMAX], yv[OR_NMAX], l[OR_QMAX + 2], xi[OR_QMAX + 2];
    double gaps[OR_QMAX + 3];
    for (int k = 0; k < OR_NSTAT; ++k) st[k] = 0;
    if (n < 1 || n > OR_NMAX || !(t1 > t0) || !all_finite(n, y)) return OR_BAD_INPUT;
    memset(s, 0, sizeof(*s));
    s->n = n;
    s->st = st;
    if (ode->rhs(ode->ctx, t0, y, f0) != 0 || !all_finite(n, f0)) return OR_BAD_INPUT;
    st[ST_RHS] += 1;
    weights(n, y, o->rtol, o->atol, w);
    s->h = initial_step(ode, t0, t1 - t0, y, f0, w, st);
    s->t = t0;
    s->q = 1;
    s->qwait = 2;
    for (int i = 0; i < n; ++i) {
        s->z[i] = y[i];
        s->z[n + i] = s->h * f0[i];
    }
    for (int k = 0; k < OR_QMAX + 3; ++k) s->hist[k] = s->h;
    s->need_j = 1;
    s->need_p = 1;
    s->crate = OR_CRATE0;
    s->gamma_p = 1.0;
    s->eta_max = OR_ETAMX_FIRST;
    int status = OR_OK, attempts = 0;

    while (s->t < t1) {
        if (attempts >= o->max_steps) { status = OR_MAX_STEPS; break; }
        int last = 0;
        if (s->t + s->h >= t1) {
            double hn = t1 - s->t;
            rescale(n, s->q, s->z, hn / s->h);
            s->h = hn;
            last = 1;
        }
        attempts += 1;
        const int q = s->q;
        weights(n, s->z, o->rtol, o->atol, w);
        or_predict(n, q, s->z);
        gaps[0] = s->h;
        for (int k = 0; k < q; ++k) gaps[k + 1] = s->hist[k];
        or_xi_from_gaps(s->h, gaps, q + 1, xi);
        double cq;
        or_bdf_coeffs(q, xi, l, &cq);
        double gamma = s->h / l[1];
        s->jcur = 0;
        int nw;
        for (;;) {
            nw = newton(s, ode, w, l, cq, gamma, e, yv);
            if (nw == NW_FAIL && !s->jcur) { s->need_j = 1; continue; }
            break;
        }
        if (nw != NW_CONVERGED) {
            or_retract(n, q, s->z);
            s->ncf += 1;
            st[ST_CONV_FAILS] += 1;
            if (s->ncf >= OR_MXNCF) { status = OR_CONV_FAIL; break; }
            rescale(n, q, s->z, OR_ETACF);
            s->h *= OR_ETACF;
            s->need_p = 1;
            s->qwait = q + 1;
            s->have_esave = 0;
            if (s->t + s->h == s->t) { status = OR_H_UNDERFLOW; break; }
            continue;
        }
        double dsm = cq * wrms(n, e, w);
        if (dsm > 1.0) {
            or_retract(n, q, s->z);
            s->nef += 1;
            st[ST_ERR_FAILS] += 1;
            s->have_esave = 0;
            if (s->nef >= OR_KFC) {
                /* restart at order 1 from the last accepted state */
                double f[OR_NMAX];
                if (ode->rhs(ode->ctx, s->t, s->z, f) != 0 || !all_finite(n, f)) {
                    status = OR_NONFINITE;
                    break;
                }
                st[ST_RHS] += 1;
                s->h *= OR_ETAMIN;
                s->q = 1;
                for (int i = 0; i < n; ++i) s->z[n + i] = s->h * f[i];
            } else {
                double eta = 1.0 / (pow(OR_BIAS_Q * dsm, 1.0 / (q + 1)) + OR_ADDON);
                int qn = q;
                if (q > 1) {
                    or_xi_from_gaps(s->h, s->hist, q, xi);
                    double est = or_err_coef_qm1(q, xi) * wrms(n, s->z + q * n, w);
                    double eta_m = 1.0 / (pow(OR_BIAS_QM1 * est, 1.0 / q) + OR_ADDON);
                    if (eta_m > eta) { eta = eta_m; qn = q - 1; }
                }
                eta = fmax(OR_ETAMIN, fmin(eta, 1.0));
                if (qn < q) {
                    double c[OR_QMAX + 2];
                    or_order_lower_coefs(q, xi, c);
                    for (int j = 1; j < q; ++j)
                        for (int i = 0; i < n; ++i) s->z[j * n + i] -= c[j] * s->z[q * n + i];
                    s->q = qn;
                }
                rescale(n, s->q, s->z, eta);
                s->h *= eta;
            }
            s->qwait = s->q + 1;
            if (s->t + s->h == s->t) { status = OR_H_UNDERFLOW; break; }
            continue;
        }
        /* accept */
        for (int j = 0; j <= q; ++j)
            for (int i = 0; i < n; ++i) s->z[j * n + i] += l[j] * e[i];
        s->t = last ? t1 : s->t + s->h;
        if (o->steplog && o->steplog_n && *o->steplog_n < o->steplog_cap) {
            double *r = o->steplog + 4 * (*o->steplog_n);
            r[0] = s->t;
            r[1] = s->h;
            r[2] = q;
            r[3] = dsm;
            *o->steplog_n += 1;
        }
        for (int k = OR_QMAX + 2; k > 0; --k) s->hist[k] = s->hist[k - 1];
        s->hist[0] = s->h;
        st[ST_STEPS] += 1;
        s->nef = 0;
        s->ncf = 0;
        s->jage += 1;
        s->page += 1;
        s->qwait -= 1;
        if (s->qwait == 1 && q < qmax) {
            for (int i = 0; i < n; ++i) s->esave[i] = e[i];
            s->esave_h = s->h;
            s->have_esave = 1;
        }
        if (last) break;
        if (s->qwait > 0) continue;
        /* step size and order selection */
        double eta = 1.0 / (pow(OR_BIAS_Q * dsm, 1.0 / (q + 1)) + OR_ADDON);
        int qn = q;
        or_xi_from_gaps(s->h, s->hist, q + 1, xi);
        if (q > 1) {
            double est = or_err_coef_qm1(q, xi) * wrms(n, s->z + q * n, w);
            double eta_m = 1.0 / (pow(OR_BIAS_QM1 * est, 1.0 / q) + OR_ADDON);
            if (eta_m > eta) { eta = eta_m; qn = q - 1; }
        }
        if (q < qmax && s->have_esave) {
            double r = pow(s->h / s->esave_h, (double)(q + 1));
            double dv[OR_NMAX];
            for (int i = 0; i < n; ++i) dv[i] = e[i] - r * s->esave[i];
            double est = or_err_coef_qp1(q) * wrms(n, dv, w);
            double eta_p = 1.0 / (pow(OR_BIAS_QP1 * est, 1.0 / (q + 2)) + OR_ADDON);
            if (eta_p > eta) { eta = eta_p; qn = q + 1; }
        }
        s->have_esave = 0;
        if (eta < OR_THRESH) { s->qwait = 2; continue; }
        eta = fmin(eta, s->eta_max);
        s->eta_max = OR_ETAMX;
        if (qn > q) {
            double C = or_order_raise_coef(q, xi), c[OR_QMAX + 2];
            or_order_lower_coefs(q + 1, xi, c);
            for (int i = 0; i < n; ++i) s->z[(q + 1) * n + i] = 0.0;
            for (int j = 1; j <= q + 1; ++j)
                for (int i = 0; i < n; ++i) s->z[j * n + i] += c[j] * C * e[i];
        } else if (qn < q) {
            double c[OR_QMAX + 2];
            or_order_lower_coefs(q, xi, c);
            for (int j = 1; j < q; ++j)
                for (int i = 0; i < n; ++i) s->z[j * n + i] -= c[j] * s->z[q * n + i];
        }
        s->q = qn;
        rescale(n, s->q, s->z, eta);
        s->h *= eta;
        s->qwait = s->q + 1;
    }
    for (int i = 0; i < n; ++i) y[i] = s->z[i];
    st[ST_ORDER] = s->q;
    if (status == OR_OK && !all_finite(n, y)) status = OR_NONFINITE;
    return status;
}

/* ------------------------------------------------------------------------ */
/* Fixed-order, prescribed-step driver for the formula pins: each step is    */
/* predicted, corrected to full Newton convergence with the exact Jacobian   */
/* at order q (no error control), and accepted. Writes each step's           */
/* correction e and estimate cq*e; hist holds the past accepted steps and is */
/* updated. Returns 0, or 1 if Newton did not converge.                      */
/* ------------------------------------------------------------------------ */
int or_fixed_steps(const or_ode *ode, int q, int nsteps, const double *hs, double t0,
                   double *z /* [(q+1) n] */, double *hist /* [>= q+2] */,
                   double *e_out /* [nsteps n] */, double *est_out /* [nsteps n] */)
{
    const int n = ode->n;
    double t = t0;
    double l[OR_QMAX + 2], xi[OR_QMAX + 2], gaps[OR_QMAX + 3];
    double J[OR_NMAX * OR_NMAX], P[OR_NMAX * OR_NMAX], f[OR_NMAX], d[OR_NMAX], e[OR_NMAX],
        y[OR_NMAX];
    int piv[OR_NMAX];
    for (int s = 0; s < nsteps; ++s) {
        double h = hs[s];
        or_predict(n, q, z);
        gaps[0] = h;
        for (int k = 0; k < q; ++k) gaps[k + 1] = hist[k];
        or_xi_from_gaps(h, gaps, q + 1, xi);
        double cq;
        or_bdf_coeffs(q, xi, l, &cq);
        double gamma = h / l[1];
        for (int i = 0; i < n; ++i) { e[i] = 0.0; y[i] = z[i]; }
        int ok = 0;
        for (int it = 0; it < 50; ++it) {
            ode->rhs(ode->ctx, t + h, y, f);
            ode->jac(ode->ctx, t + h, y, J);
            for (int i = 0; i < n; ++i)
                for (int j = 0; j < n; ++j) P[i * n + j] = (i == j ? 1.0 : 0.0) - gamma * J[i * n + j];
            if (or_lu_factor(n, P, piv) != 0) return 1;
            double mx = 0.0, ms = 0.0;
            for (int i = 0; i < n; ++i) d[i] = (h * f[i] - z[n + i]) / l[1] - e[i];
            or_lu_solve(n, P, piv, d);
            for (int i = 0; i < n; ++i) {
                e[i] += d[i];
                y[i] = z[i] + e[i];
                mx = fmax(mx, fabs(d[i]));
                ms = fmax(ms, fabs(e[i]) + fabs(z[i]));
            }
            if (mx <= 1e-15 * ms || mx == 0.0) { ok = 1; break; }
        }
        if (!ok) return 1;
        for (int j = 0; j <= q; ++j)
            for (int i = 0; i < n; ++i) z[j * n + i] += l[j] * e[i];
        for (int i = 0; i < n; ++i) {
            e_out[s * n + i] = e[i];
            est_out[s * n + i] = cq * e[i];
        }
        for (int k = q + 1; k > 0; --k) hist[k] = hist[k - 1];
        hist[0] = h;
        t += h;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Linear test ODE y' = A y + sum_k c_k t^k (A dense, row-major).            */
/* ------------------------------------------------------------------------ */
typedef struct {
    int n, deg;
    double A[OR_NMAX * OR_NMAX];
    double c[8 * OR_NMAX];
} or_linear;

static int linear_rhs(void *ctx, double t, const double *y, double *f)
{
    const or_linear *p = (const or_linear *)ctx;
    for (int i = 0; i < p->n; ++i) {
        double s = 0.0;
        for (int j = 0; j < p->n; ++j) s += p->A[i * p->n + j] * y[j];
        double tk = 1.0;
        for (int k = 0; k <= p->deg; ++k) {
            s += p->c[k * p->n + i] * tk;
            tk *= t;
        }
        f[i] = s;
    }
    return 0;
}

static int linear_jac(void *ctx, double t, const double *y, double *J)
{
    (void)t;
    (void)y;
    const or_linear *p = (const or_linear *)ctx;
    memcpy(J, p->A, sizeof(double) * p->n * p->n);
    return 0;
}

static void linear_ode(or_linear *p, int n, const double *A, int deg, const double *c, or_ode *ode)
{
    p->n = n;
    p->deg = deg;
    memcpy(p->A, A, sizeof(double) * n * n);
    memcpy(p->c, c, sizeof(double) * (deg + 1) * n);
    ode->n = n;
    ode->rhs = linear_rhs;
    ode->jac = linear_jac;
    ode->ctx = p;
}

int or_linear_integrate(int n, const double *A, int deg, const double *c, double rtol,
                        double atol, int max_order, int max_steps, double t0, double t1,
                        double *y, int32_t *st)
{
    or_linear p;
    or_ode ode;
    if (n < 1 || n > OR_NMAX || deg < 0 || deg > 7) return OR_BAD_INPUT;
    linear_ode(&p, n, A, deg, c, &ode);
    or_opts o = {rtol, atol, max_order, max_steps};
    return or_bdf_integrate(&ode, &o, t0, t1, y, st);
}

/* or_linear_integrate with the record of accepted steps: steplog[4 k ..] =
   (t after step k, h, q, error estimate) for k < *nlog <= cap. */
int or_linear_integrate_steps(int n, const double *A, int deg, const double *c, double rtol,
                              double atol, int max_order, int max_steps, double t0, double t1,
                              double *y, int32_t *st, double *steplog, int cap, int *nlog)
{
    or_linear p;
    or_ode ode;
    if (n < 1 || n > OR_NMAX || deg < 0 || deg > 7) return OR_BAD_INPUT;
    linear_ode(&p, n, A, deg, c, &ode);
    or_opts o = {rtol, atol, max_order, max_steps};
    *nlog = 0;
    o.steplog = steplog;
    o.steplog_cap = cap;
    o.steplog_n = nlog;
    return or_bdf_integrate(&ode, &o, t0, t1, y, st);
}

int or_linear_fixed_steps(int n, const double *A, int deg, const double *c, int q, int nsteps,
                          const double *hs, double t0, double *z, double *hist, double *e_out,
                          double *est_out)
{
    or_linear p;
    or_ode ode;
    if (n < 1 || n > OR_NMAX || q < 1 || q > OR_QMAX || deg < 0 || deg > 7) return 1;
    linear_ode(&p, n, A, deg, c, &ode);
    return or_fixed_steps(&ode, q, nsteps, hs, t0, z, hist, e_out, est_out);
}

/* Starting step of initial_step for y' = A y at y0 (t0 = 0), weights from y0
   as the integrator takes them. For the pins: its closed form on scalar and
   diagonal linear problems. */
double or_linear_initial_step(int n, const double *A, const double *y0, double rtol, double atol,
                              double span)
{
    or_linear p;
    or_ode ode;
    double c[OR_NMAX] = {0.0}, f0[OR_NMAX], w[OR_NMAX];
    int32_t st[OR_NSTAT] = {0};
    if (n < 1 || n > OR_NMAX) return -1.0;
    linear_ode(&p, n, A, 0, c, &ode);
    linear_rhs(&p, 0.0, y0, f0);
    weights(n, y0, rtol, atol, w);
    return initial_step(&ode, 0.0, span, y0, f0, w, st);
}

/* One call of the integrator's modified Newton (newton) on y' = A y for the
   predicted Nordsieck columns z0 = z[0..n), z1 = z[n..2n) with corrector
   coefficient l1 and step h, weights w, error constant cq. The matrix is first
   formed and factored at gamma_P = gamma_p_ratio * h / l1 (by a Newton call at
   that gamma), then the recorded call runs at gamma = h / l1 and reuses it,
   scaling its corrections by 2 / (1 + gamma/gamma_P) when the two differ.
   trace[k n + i] receives e after correction k (at most OR_MAXCOR); returns the
   number recorded, and *result the newton() outcome (0 converged, 1 failed). */
int or_linear_newton(int n, const double *A, const double *z, double l1, double h,
                     double gamma_p_ratio, const double *w, double cq, double *trace, int *result)
{
    or_linear p;
    or_ode ode;
    double c[OR_NMAX] = {0.0}, l[OR_QMAX + 2] = {1.0, l1}, e[OR_NMAX], y[OR_NMAX];
    int32_t st[OR_NSTAT] = {0};
    if (n < 1 || n > OR_NMAX || !(fabs(gamma_p_ratio - 1.0) <= OR_CCMAX)) return -1;
    or_bdf *s = (or_bdf *)calloc(1, sizeof(or_bdf));
    if (!s) return -1;
    linear_ode(&p, n, A, 0, c, &ode);
    s->n = n;
    s->st = st;
    s->h = h;
    s->gamma_p = 1.0;
    s->crate = OR_CRATE0;
    memcpy(s->z, z, sizeof(double) * 2 * n);
    /* factor at gamma_P: a first call with need_j set */
    s->need_j = 1;
    (void)newton(s, &ode, w, l, cq, gamma_p_ratio * h / l1, e, y);
    /* the recorded call at gamma = h / l1 reuses that matrix */
    s->jage = 1;
    s->page = 1;
    s->trace = trace;
    s->ntrace = 0;
    *result = newton(s, &ode, w, l, cq, h / l1, e, y);
    const int k = s->ntrace;
    free(s);
    return k;
}

/* ------------------------------------------------------------------------ */
/* RKC: the explicit, stabilised Runge-Kutta-Chebyshev method of order 2     */
/* (Sommeijer, Shampine & Verwer 1998) -- the alternative integrator the     */
/* network/integrator separation admits (Software design section, ¶4). With  */
/* s stages and damping eps = 2/13:                                          */
/*   w0 = 1 + eps/s^2, w1 = T_s'(w0) / T_s''(w0),                             */
/*   b_j = T_j''(w0) / T_j'(w0)^2 (j >= 2), b_0 = b_1 = b_2,                  */
/*   Y_0 = y_n, Y_1 = Y_0 + b_1 w1 h F(Y_0),                                  */
/*   Y_j = (1 - mu_j - nu_j) Y_0 + mu_j Y_{j-1} + nu_j Y_{j-2}                */
/*         + mt_j h F(Y_{j-1}) + gt_j h F(Y_0),                               */
/*   mu_j = 2 b_j w0 / b_{j-1}, nu_j = -b_j / b_{j-2}, mt_j = 2 b_j w1 / b_{j-1}, */
/*   gt_j = -(1 - b_{j-1} T_{j-1}(w0)) mt_j,  y_{n+1} = Y_s.                  */
/* Stage j sits at time t_n + c_j h, c_j = w1 T_j''(w0) / T_j'(w0) (j >= 2),   */
/* c_1 = c_2 / T_2'(w0). On y' = lambda y a step multiplies y by             */
/*   P_s(z) = 1 - b_s T_s(w0) + b_s T_s(w0 + w1 z), z = h lambda,             */
/* bounded by 1 on [-beta_s, 0], beta_s = (1 + w0) / w1 (about 0.65 s^2).      */
/* Error estimate of the same paper: (12 (y_n - y_{n+1}) + 6 h (F_n + F_{n+1})) / 15. */
/* ------------------------------------------------------------------------ */
#define OR_RKC_EPS (2.0 / 13.0)
#define OR_RKC_SMAX 256

typedef struct {
    int s;
    double w0, w1;
    double T[OR_RKC_SMAX + 1], dT[OR_RKC_SMAX + 1], ddT[OR_RKC_SMAX + 1], b[OR_RKC_SMAX + 1];
} or_rkc_coef;

/* Chebyshev values and first two derivatives at w0 by their three-term
   recurrences, then w1 and the b_j. */
static void rkc_coef(int s, or_rkc_coef *k)
{
    const double w0 = 1.0 + OR_RKC_EPS / ((double)s * s);
    k->s = s;
    k->w0 = w0;
    k->T[0] = 1.0; k->dT[0] = 0.0; k->ddT[0] = 0.0;
    k->T[1] = w0;  k->dT[1] = 1.0; k->ddT[1] = 0.0;
    for (int j = 2; j <= s; ++j) {
        k->T[j] = 2.0 * w0 * k->T[j - 1] - k->T[j - 2];
        k->dT[j] = 2.0 * k->T[j - 1] + 2.0 * w0 * k->dT[j - 1] - k->dT[j - 2];
        k->ddT[j] = 4.0 * k->dT[j - 1] + 2.0 * w0 * k->ddT[j - 1] - k->ddT[j - 2];
    }
    k->w1 = k->dT[s] / k->ddT[s];
    for (int j = 2; j <= s; ++j) k->b[j] = k->ddT[j] / (k->dT[j] * k->dT[j]);
    k->b[0] = k->b[1] = k->b[2];
}

/* Left end of the real stability interval: w0 + w1 z = -1. */
static double rkc_beta(int s)
{
    or_rkc_coef k;
    rkc_coef(s, &k);
    return (1.0 + k.w0) / k.w1;
}

/* One RKC step of size h from (t, y0) with F(y0) = f0; result in ys. Returns 0,
   or 1 if a stage's right-hand side cannot be evaluated. */
static int rkc_step(const or_ode *ode, const or_rkc_coef *k, double t, double h, const double *y0,
                    const double *f0, double *ys, int32_t *st)
{
    const int n = ode->n, s = k->s;
    double a[OR_NMAX], b[OR_NMAX], F[OR_NMAX];
    double *ym2 = a, *ym1 = b;
    const double c2 = k->w1 * k->ddT[2] / k->dT[2];
    double cprev = c2 / k->dT[2];                       /* c_1 */
    for (int i = 0; i < n; ++i) {
        ym2[i] = y0[i];
        ym1[i] = y0[i] + k->b[1] * k->w1 * h * f0[i];
    }
    for (int j = 2; j <= s; ++j) {
        if (ode->rhs(ode->ctx, t + cprev * h, ym1, F) != 0) return 1;
        st[ST_RHS] += 1;
        const double mu = 2.0 * k->b[j] * k->w0 / k->b[j - 1];
        const double nu = -k->b[j] / k->b[j - 2];
        const double mt = 2.0 * k->b[j] * k->w1 / k->b[j - 1];
        const double gt = -(1.0 - k->b[j - 1] * k->T[j - 1]) * mt;
        for (int i = 0; i < n; ++i) {
            const double v = (1.0 - mu - nu) * y0[i] + mu * ym1[i] + nu * ym2[i] + mt * h * F[i] +
                             gt * h * f0[i];
            ym2[i] = v;                                   /* ym2 now holds Y_j */
        }
        double *tmp = ym2; ym2 = ym1; ym1 = tmp;         /* (Y_{j-1}, Y_j) */
        cprev = k->w1 * k->ddT[j] / k->dT[j];
    }
    for (int i = 0; i < n; ++i) ys[i] = ym1[i];
    return 0;
}

/* Upper bound on the spectral radius of J: the largest absolute row sum
   (Gershgorin). */
static double gershgorin(int n, const double *J)
{
    double r = 0.0;
    for (int i = 0; i < n; ++i) {
        double a = 0.0;
        for (int j = 0; j < n; ++j) a += fabs(J[i * n + j]);
        if (a > r) r = a;
    }
    return r;
}

/* Adaptive RKC from t0 to t1 (the builder's step control; the paper gives
   none): each step takes the fewest stages s >= 2 whose interval covers
   h rho, rho the Gershgorin bound of the Jacobian at the step's start; with
   more than OR_RKC_SMAX stages needed the step shrinks instead. A step is
   accepted when the WRMS norm of the estimate, with weights
   rtol max(|y_n|, |y_{n+1}|) + atol, is at most 1; the next step is
   h min(10, max(0.1, 0.8 err^(-1/3))), at most h after a rejection. Counters:
   accepted steps, rejections, right-hand sides, Jacobians (for rho), and the
   largest stage count in the order slot. */
int or_rkc_integrate(const or_ode *ode, const or_opts *o, double t0, double t1, double *y, int32_t *st)
{
    const int n = ode->n;
    double f0[OR_NMAX], w[OR_NMAX], yn[OR_NMAX], fn[OR_NMAX], J[OR_NMAX * OR_NMAX], est[OR_NMAX];
    for (int k = 0; k < OR_NSTAT; ++k) st[k] = 0;
    if (n < 1 || n > OR_NMAX || !(t1 > t0) || !all_finite(n, y)) return OR_BAD_INPUT;
    if (ode->rhs(ode->ctx, t0, y, f0) != 0 || !all_finite(n, f0)) return OR_BAD_INPUT;
    st[ST_RHS] += 1;
    weights(n, y, o->rtol, o->atol, w);
    double h = initial_step(ode, t0, t1 - t0, y, f0, w, st);
    double t = t0;
    int attempts = 0, rejected = 0;
    const double beta_max = rkc_beta(OR_RKC_SMAX);
    while (t < t1) {
        if (attempts >= o->max_steps) return OR_MAX_STEPS;
        int last = 0;
        if (t + h >= t1) { h = t1 - t; last = 1; }
        if (ode->jac(ode->ctx, t, y, J) != 0 || !all_finite(n * n, J)) return OR_NONFINITE;
        st[ST_JAC] += 1;
        const double rho = gershgorin(n, J);
        if (h * rho > beta_max) { h = 0.95 * beta_max / rho; last = 0; }
        int s = 2;
        while (s < OR_RKC_SMAX && rkc_beta(s) < h * rho) ++s;
        or_rkc_coef k;
        rkc_coef(s, &k);
        if (s > st[ST_ORDER]) st[ST_ORDER] = s;
        attempts += 1;
        double err = 2.0;
        int ok = rkc_step(ode, &k, t, h, y, f0, yn, st) == 0 && all_finite(n, yn);
        if (ok) ok = ode->rhs(ode->ctx, t + h, yn, fn) == 0 && all_finite(n, fn);
        if (ok) {
            st[ST_RHS] += 1;
            for (int i = 0; i < n; ++i) {
                est[i] = (12.0 * (y[i] - yn[i]) + 6.0 * h * (f0[i] + fn[i])) / 15.0;
                w[i] = o->rtol * fmax(fabs(y[i]), fabs(yn[i])) + o->atol;
            }
            err = wrms(n, est, w);
        }
        if (ok && err <= 1.0) {
            t = last ? t1 : t + h;
            for (int i = 0; i < n; ++i) { y[i] = yn[i]; f0[i] = fn[i]; }
            st[ST_STEPS] += 1;
            double fac = err > 0.0 ? 0.8 * pow(err, -1.0 / 3.0) : 10.0;
            fac = fmin(10.0, fmax(0.1, fac));
            if (rejected) fac = fmin(fac, 1.0);
            rejected = 0;
            h *= fac;
        } else {
            st[ST_ERR_FAILS] += 1;
            rejected = 1;
            const double fac = ok ? fmin(1.0, fmax(0.1, 0.8 * pow(err, -1.0 / 3.0))) : 0.25;
            h *= fac;
        }
        if (t < t1 && t + h == t) return OR_H_UNDERFLOW;
    }
    return OR_OK;
}

/* For the pins: one RKC step with s stages on y' = A y + sum_k c_k t^k, and
   the adaptive RKC on the same system. */
int or_rkc_linear_step(int n, const double *A, int deg, const double *c, int s, double t, double h,
                       double *y)
{
    or_linear p;
    or_ode ode;
    double f0[OR_NMAX], ys[OR_NMAX];
    int32_t st[OR_NSTAT] = {0};
    if (n < 1 || n > OR_NMAX || deg < 0 || deg > 7 || s < 2 || s > OR_RKC_SMAX) return 1;
    linear_ode(&p, n, A, deg, c, &ode);
    if (ode.rhs(ode.ctx, t, y, f0) != 0) return 1;
    or_rkc_coef k;
    rkc_coef(s, &k);
    if (rkc_step(&ode, &k, t, h, y, f0, ys, st) != 0) return 1;
    for (int i = 0; i < n; ++i) y[i] = ys[i];
    return 0;
}

int or_rkc_linear_integrate(int n, const double *A, int deg, const double *c, double rtol, double atol,
                            int max_steps, double t0, double t1, double *y, int32_t *st)
{
    or_linear p;
    or_ode ode;
    if (n < 1 || n > OR_NMAX || deg < 0 || deg > 7) return OR_BAD_INPUT;
    linear_ode(&p, n, A, deg, c, &ode);
    or_opts o = {rtol, atol, 2, max_steps, 0, 1};
    return or_rkc_integrate(&ode, &o, t0, t1, y, st);
}

/* ------------------------------------------------------------------------ */
/* Reaction network: rates, right-hand side, Jacobian.                       */
/*                                                                           */
/* State y = (x_1..x_S) for an isothermal network, or (x_1..x_S, u) with the  */
/* thermal energy per unit density u = (sum_i x_i) k_B T / (gamma - 1) in eV. */
/* The ideal-gas EOS inversion gives T = (gamma - 1) u / (k_B sum_i x_i).     */
/* Rate coefficient of a direction: k = s_r A T^b exp(-C/T) (s_r a per-cell   */
/* factor, 1 by default). Net rate per unit density of reaction r:            */
/*   w_r = k_f n^{m_f - 1} prod x(reactants) - k_r n^{m_r - 1} prod x(products) */
/* with m the number of species on that side; dx_i/dt = sum_r nu_ir w_r and   */
/* du/dt = sum_r dE_r w_r (energy released by forward events).               */
/* ------------------------------------------------------------------------ */
#define OR_KB_EV 8.617333262e-5

typedef struct {
    int S, E, R, energy;
    int react[OR_RMAX][2], prod[OR_RMAX][2];
    double Af[OR_RMAX], bf[OR_RMAX], Cf[OR_RMAX], Ar[OR_RMAX], br[OR_RMAX], Cr[OR_RMAX];
    double dE[OR_RMAX];
    double gamma;
} or_net;

typedef struct {
    const or_net *net;
    double ndens;      /* total density n, cm^-3 (1 for dimensionless systems) */
    double T_iso;      /* temperature of an isothermal network */
    const double *ks;  /* per-reaction factors s_r, NULL for all ones */
    const double *src; /* constant source per ODE component, NULL for none */
} or_cell;

or_net *or_net_create(int S, int E, int R, int energy, const int32_t *react,
                      const int32_t *prod, const double *Af, const double *bf,
                      const double *Cf, const double *Ar, const double *br,
                      const double *Cr, const double *dE, double gamma)
{
    if (S < 1 || S + (energy ? 1 : 0) > OR_NMAX || R < 0 || R > OR_RMAX) return NULL;
    or_net *net = (or_net *)calloc(1, sizeof(or_net));
    if (!net) return NULL;
    net->S = S;
    net->E = E;
    net->R = R;
    net->energy = energy ? 1 : 0;
    for (int r = 0; r < R; ++r) {
        net->react[r][0] = react[2 * r];
        net->react[r][1] = react[2 * r + 1];
        net->prod[r][0] = prod[2 * r];
        net->prod[r][1] = prod[2 * r + 1];
        net->Af[r] = Af[r];
        net->bf[r] = bf[r];
        net->Cf[r] = Cf[r];
        net->Ar[r] = Ar[r];
        net->br[r] = br[r];
        net->Cr[r] = Cr[r];
        net->dE[r] = dE[r];
    }
    net->gamma = gamma;
    return net;
}

void or_net_destroy(or_net *net) { free(net); }

static double arrhenius(double A, double b, double C, double T)
{
    if (A == 0.0) return 0.0;
    return A * pow(T, b) * exp(-C / T);
}

/* Temperature of the state (EOS inversion for the energy form). */
static double state_T(const or_cell *c, const double *y)
{
    const or_net *net = c->net;
    if (!net->energy) return c->T_iso;
    double X = 0.0;
    for (int i = 0; i < net->S; ++i) X += y[i];
    return (net->gamma - 1.0) * y[net->S] / (OR_KB_EV * X);
}

/* Product of a side's abundances times n^(m-1), and its partial derivatives
   with respect to the side's species (dp[0], dp[1] for slots 0 and 1). */
static double side_product(const int *side, const double *x, double n, double *dp)
{
    if (side[1] < 0) {
        dp[0] = 1.0;
        dp[1] = 0.0;
        return x[side[0]];
    }
    dp[0] = n * x[side[1]];
    dp[1] = n * x[side[0]];
    return n * x[side[0]] * x[side[1]];
}

int or_net_rhs(void *ctx, double t, const double *y, double *f)
{
    (void)t;
    const or_cell *c = (const or_cell *)ctx;
    const or_net *net = c->net;
    const int S = net->S;
    double T = state_T(c, y);
    if (!(T > 0.0) || !isfinite(T)) return 1;
    for (int i = 0; i < S + net->energy; ++i) f[i] = 0.0;
    for (int r = 0; r < net->R; ++r) {
        double s = c->ks ? c->ks[r] : 1.0;
        double kf = s * arrhenius(net->Af[r], net->bf[r], net->Cf[r], T);
        double kr = s * arrhenius(net->Ar[r], net->br[r], net->Cr[r], T);
        double dp[2];
        double pf = side_product(net->react[r], y, c->ndens, dp);
        double pr = side_product(net->prod[r], y, c->ndens, dp);
        double wr = kf * pf - kr * pr;
        for (int k = 0; k < 2; ++k) {
            if (net->react[r][k] >= 0) f[net->react[r][k]] -= wr;
            if (net->prod[r][k] >= 0) f[net->prod[r][k]] += wr;
        }
        if (net->energy) f[S] += net->dE[r] * wr;
    }
    /* a constant source (e.g. the advective term of an SDC-coupled burn,    */
    /* Software design section, paragraph 4) adds to every component         */
    if (c->src)
        for (int i = 0; i < S + net->energy; ++i) f[i] += c->src[i];
    return 0;
}

/* Analytic Jacobian. For the energy form, T depends on the state through the
   EOS: dT/dx_j = -T / sum x, dT/du = (gamma - 1) / (k_B sum x); with
   g_i = d f_i / dT at fixed x, J_ij = (d f_i / d x_j)|_T + g_i dT/dy_j.
   dk/dT = k (b + C/T) / T. */
int or_net_jac(void *ctx, double t, const double *y, double *J)
{
    (void)t;
    const or_cell *c = (const or_cell *)ctx;
    const or_net *net = c->net;
    const int S = net->S, N = S + net->energy;
    double T = state_T(c, y);
    if (!(T > 0.0) || !isfinite(T)) return 1;
    double g[OR_NMAX];
    for (int i = 0; i < N * N; ++i) J[i] = 0.0;
    for (int i = 0; i < N; ++i) g[i] = 0.0;
    for (int r = 0; r < net->R; ++r) {
        double s = c->ks ? c->ks[r] : 1.0;
        double kf = s * arrhenius(net->Af[r], net->bf[r], net->Cf[r], T);
        double kr = s * arrhenius(net->Ar[r], net->br[r], net->Cr[r], T);
        double dpf[2], dpr[2];
        double pf = side_product(net->react[r], y, c->ndens, dpf);
        double pr = side_product(net->prod[r], y, c->ndens, dpr);
        /* d w_r / d x_j at fixed T, accumulated per species slot */
        double dw[OR_NMAX];
        for (int j = 0; j < S; ++j) dw[j] = 0.0;
        for (int k = 0; k < 2; ++k) {
            if (net->react[r][k] >= 0) dw[net->react[r][k]] += kf * dpf[k];
            if (net->prod[r][k] >= 0) dw[net->prod[r][k]] -= kr * dpr[k];
        }
        double dkf = kf * (net->bf[r] + net->Cf[r] / T) / T;
        double dkr = kr * (net->br[r] + net->Cr[r] / T) / T;
        double dwdT = dkf * pf - dkr * pr;
        /* rows touched by reaction r: nu_ir */
        double nu[OR_NMAX];
        for (int i = 0; i < S; ++i) nu[i] = 0.0;
        for (int k = 0; k < 2; ++k) {
            if (net->react[r][k] >= 0) nu[net->react[r][k]] -= 1.0;
            if (net->prod[r][k] >= 0) nu[net->prod[r][k]] += 1.0;
        }
        for (int i = 0; i < S; ++i) {
            if (nu[i] == 0.0) continue;
            for (int j = 0; j < S; ++j) J[i * N + j] += nu[i] * dw[j];
            g[i] += nu[i] * dwdT;
        }
        if (net->energy) {
            for (int j = 0; j < S; ++j) J[S * N + j] += net->dE[r] * dw[j];
            g[S] += net->dE[r] * dwdT;
        }
    }
    if (net->energy) {
        double X = 0.0;
        for (int i = 0; i < S; ++i) X += y[i];
        double dTdx = -T / X, dTdu = (net->gamma - 1.0) / (OR_KB_EV * X);
        for (int i = 0; i < N; ++i) {
            for (int j = 0; j < S; ++j) J[i * N + j] += g[i] * dTdx;
            J[i * N + S] += g[i] * dTdu;
        }
    }
    return 0;
}

/* Single-state evaluation hooks for the pins. y has S (+1) entries. */
int or_net_eval(const or_net *net, double ndens, double T_iso, const double *ks, const double *y,
                double *f, double *J)
{
    or_cell c = {net, ndens, T_iso, ks};
    if (f && or_net_rhs(&c, 0.0, y, f) != 0) return 1;
    if (J && or_net_jac(&c, 0.0, y, J) != 0) return 1;
    return 0;
}

/* Forward-difference Jacobian: an approximate Jacobian of the kind the      */
/* paper's failure policy may retry with (Software design section, ¶3). The  */
/* paper gives no formula; this is the plain one-sided difference           */
/*   J[:, j] = (f(y + d_j e_j) - f(y)) / d_j,                                 */
/*   d_j = sqrt(eps) (|y_j| + atol / rtol),                                   */
/* the increment scaled like the error weight rtol |y_j| + atol, and d_j      */
/* taken as the difference actually represented, (y_j + d_j) - y_j.          */
typedef struct {
    const or_ode *inner;
    double rtol, atol;
} or_fd;

static int fd_rhs(void *ctx, double t, const double *y, double *f)
{
    const or_fd *p = (const or_fd *)ctx;
    return p->inner->rhs(p->inner->ctx, t, y, f);
}

static int fd_jac(void *ctx, double t, const double *y, double *J)
{
    const or_fd *p = (const or_fd *)ctx;
    const or_ode *in = p->inner;
    const int n = in->n;
    double f0[OR_NMAX], f1[OR_NMAX], yp[OR_NMAX];
    if (in->rhs(in->ctx, t, y, f0) != 0) return 1;
    for (int j = 0; j < n; ++j) {
        for (int i = 0; i < n; ++i) yp[i] = y[i];
        yp[j] = y[j] + sqrt(DBL_EPSILON) * (fabs(y[j]) + p->atol / p->rtol);
        const double dj = yp[j] - y[j];
        if (!(dj != 0.0)) return 1;
        if (in->rhs(in->ctx, t, yp, f1) != 0) return 1;
        for (int i = 0; i < n; ++i) J[i * n + j] = (f1[i] - f0[i]) / dj;
    }
    return 0;
}

/* The forward-difference Jacobian of a network's ODE system at y (for the   */
/* pins; the integrator uses the same function).                             */
int or_net_fd_jac(const or_net *net, double ndens, double T_iso, const double *ks, const double *y,
                  double rtol, double atol, double *J)
{
    or_cell c = {net, ndens, T_iso, ks};
    or_ode ode = {net->S + net->energy, or_net_rhs, or_net_jac, &c};
    or_fd fd = {&ode, rtol, atol};
    return fd_jac(&fd, 0.0, y, J);
}

/* Burn one cell: the operator-split reaction step of length dt (Software
   design section, paragraph 4) for the state (x, T). For the energy form the
   thermal energy u = sum x k_B T/(gamma-1) is integrated and T recovered by
   the EOS inversion at the end. x has S entries; T is in/out. */
int or_burn_cell(const or_net *net, const or_opts *o, double dt, double *x, double *T,
                 double ndens, const double *ks, const double *src, int32_t *st)
{
    const int S = net->S;
    double y[OR_NMAX];
    or_cell c = {net, ndens, T ? *T : 1.0, ks, src};
    or_ode exact = {S + net->energy, or_net_rhs, or_net_jac, &c};
    or_fd fd = {&exact, o->rtol, o->atol};
    or_ode approx = {S + net->energy, fd_rhs, fd_jac, &fd};
    const or_ode ode = o->jac_fd ? approx : exact;
    for (int i = 0; i < S; ++i) y[i] = x[i];
    if (net->energy) {
        double X = 0.0;
        for (int i = 0; i < S; ++i) X += x[i];
        if (!T || !(*T > 0.0) || !isfinite(*T) || !(X > 0.0) || !isfinite(X)) {
            for (int k = 0; k < OR_NSTAT; ++k) st[k] = 0;
            return OR_BAD_INPUT;
        }
        y[S] = X * OR_KB_EV * (*T) / (net->gamma - 1.0);
    }
    if (!(ndens > 0.0) || !isfinite(ndens)) {
        for (int k = 0; k < OR_NSTAT; ++k) st[k] = 0;
        return OR_BAD_INPUT;
    }
    int status = o->method == 1 ? or_rkc_integrate(&ode, o, 0.0, dt, y, st)
                                : or_bdf_integrate(&ode, o, 0.0, dt, y, st);
    for (int i = 0; i < S; ++i) x[i] = y[i];
    if (net->energy) {
        double X = 0.0;
        for (int i = 0; i < S; ++i) X += y[i];
        *T = (net->gamma - 1.0) * y[S] / (OR_KB_EV * X);
    }
    return status;
}

/* ------------------------------------------------------------------------ */
/* Batch driver over host threads (structure-of-arrays in and out, like the  */
/* device interface): x[i * ld + c], T[c], ndens[c], ks[r * ld + c].          */
/* ------------------------------------------------------------------------ */
typedef struct {
    const or_net *net;
    or_opts o;
    int64_t ncells, ld;
    double dt;
    double *x, *T;
    const double *ndens, *ks;
    int32_t *status, *stats;
    int64_t next;
    const double *src;  /* [n_ode][ld] constant sources, or NULL */
} or_batch;

static void *batch_worker(void *arg)
{
    or_batch *b = (or_batch *)arg;
    const int S = b->net->S, R = b->net->R;
    for (;;) {
        int64_t c0 = __atomic_fetch_add(&b->next, 16, __ATOMIC_RELAXED);
        if (c0 >= b->ncells) break;
        int64_t c1 = c0 + 16 < b->ncells ? c0 + 16 : b->ncells;
        for (int64_t c = c0; c < c1; ++c) {
            double x[OR_NMAX], ks[OR_RMAX], src[OR_NMAX], T = b->T ? b->T[c] : 1.0;
            int32_t st[OR_NSTAT];
            for (int i = 0; i < S; ++i) x[i] = b->x[i * b->ld + c];
            if (b->ks)
                for (int r = 0; r < R; ++r) ks[r] = b->ks[r * b->ld + c];
            if (b->src)
                for (int i = 0; i < S + b->net->energy; ++i) src[i] = b->src[i * b->ld + c];
            double nd = b->ndens ? b->ndens[c] : 1.0;
            int s = or_burn_cell(b->net, &b->o, b->dt, x, b->T ? &T : NULL, nd,
                                 b->ks ? ks : NULL, b->src ? src : NULL, st);
            for (int i = 0; i < S; ++i) b->x[i * b->ld + c] = x[i];
            if (b->T) b->T[c] = T;
            b->status[c] = s;
            if (b->stats)
                for (int k = 0; k < OR_NSTAT; ++k) b->stats[k * b->ld + c] = st[k];
        }
    }
    return NULL;
}

/* Burn with a constant source per cell and ODE component, src[i * ld + c]   */
/* (species rates in fraction/s, then the energy rate in eV/s per unit n).   */
int or_burn_batch_src(const or_net *net, double rtol, double atol, int max_order, int max_steps,
                      int64_t ncells, double dt, double *x, int64_t ld, double *T,
                      const double *ndens, const double *ks, const double *src, int32_t *status,
                      int32_t *stats, int nthreads)
{
    if (!net || ncells < 0 || ld < ncells || (net->energy && !T)) return 1;
    or_batch b = {net, {rtol, atol, max_order, max_steps}, ncells, ld, dt, x, T, ndens, ks,
                  status, stats, 0, src};
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    pthread_t th[256];
    int started = 0;
    for (int i = 1; i < nthreads; ++i)
        if (pthread_create(&th[started], NULL, batch_worker, &b) == 0) started++;
    batch_worker(&b);
    for (int i = 0; i < started; ++i) pthread_join(th[i], NULL);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Retry ladder (Software design section, ¶3: a zone whose integration fails */
/* may be integrated again on its own under other tolerances or with an      */
/* approximate Jacobian, or the failure handed back). Each cell is burned    */
/* from its inputs with rung 0; while it fails with a status a retry can     */
/* change (step cap, step-size underflow, Newton failures, non-finite      */
/* state) and rungs remain, it is burned again from the same inputs with    */
/* the next rung.                                                            */
/* The outputs are those of the last attempt, rung[c] says which rung gave   */
/* them. Rejected inputs are never retried.                                  */
/* ------------------------------------------------------------------------ */
typedef struct {
    const or_net *net;
    int n_rungs;
    const or_opts *rungs;
    int64_t ncells, ld;
    double dt;
    double *x, *T;
    const double *ndens, *ks;
    int32_t *status, *stats, *rung;
    int64_t next;
} or_ladder;

static void *ladder_worker(void *arg)
{
    or_ladder *b = (or_ladder *)arg;
    const int S = b->net->S, R = b->net->R;
    for (;;) {
        int64_t c = __atomic_fetch_add(&b->next, 1, __ATOMIC_RELAXED);
        if (c >= b->ncells) break;
        double x0[OR_NMAX], ks[OR_RMAX], x[OR_NMAX], T = 1.0;
        const double T0 = b->T ? b->T[c] : 1.0;
        int32_t st[OR_NSTAT];
        for (int i = 0; i < S; ++i) x0[i] = b->x[i * b->ld + c];
        if (b->ks)
            for (int r = 0; r < R; ++r) ks[r] = b->ks[r * b->ld + c];
        const double nd = b->ndens ? b->ndens[c] : 1.0;
        int s = OR_BAD_INPUT, k = 0;
        for (k = 0; k < b->n_rungs; ++k) {
            for (int i = 0; i < S; ++i) x[i] = x0[i];
            T = T0;
            s = or_burn_cell(b->net, &b->rungs[k], b->dt, x, b->T ? &T : NULL, nd, b->ks ? ks : NULL, NULL,
                             st);
            const int retry = (s == OR_MAX_STEPS || s == OR_H_UNDERFLOW || s == OR_CONV_FAIL ||
                               s == OR_NONFINITE);
            if (!retry || k + 1 == b->n_rungs) break;
        }
        if (s != OR_BAD_INPUT) {
            for (int i = 0; i < S; ++i) b->x[i * b->ld + c] = x[i];
            if (b->T) b->T[c] = T;
        }
        b->status[c] = s;
        b->rung[c] = k;
        if (b->stats)
            for (int q = 0; q < OR_NSTAT; ++q) b->stats[q * b->ld + c] = st[q];
    }
    return NULL;
}

int or_burn_batch_ladder(const or_net *net, int n_rungs, const double *rtol, const double *atol,
                         const int32_t *max_order, const int32_t *max_steps, const int32_t *jac_fd,
                         const int32_t *method, int64_t ncells, double dt, double *x, int64_t ld, double *T, const double *ndens,
                         const double *ks, int32_t *status, int32_t *stats, int32_t *rung, int nthreads)
{
    if (!net || n_rungs < 1 || n_rungs > 8 || ncells < 0 || ld < ncells || (net->energy && !T) || !rung)
        return 1;
    or_opts rungs[8];
    for (int k = 0; k < n_rungs; ++k) {
        if (!(rtol[k] > 0.0) || !(atol[k] > 0.0) || max_order[k] < 1 || max_order[k] > OR_QMAX ||
            max_steps[k] < 1)
            return 1;
        if (method[k] != 0 && method[k] != 1) return 1;
        rungs[k] = (or_opts){rtol[k], atol[k], max_order[k], max_steps[k], jac_fd[k] ? 1 : 0, method[k]};
    }
    or_ladder b = {net, n_rungs, rungs, ncells, ld, dt, x, T, ndens, ks, status, stats, rung, 0};
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    pthread_t th[256];
    int started = 0;
    for (int i = 1; i < nthreads; ++i)
        if (pthread_create(&th[started], NULL, ladder_worker, &b) == 0) started++;
    ladder_worker(&b);
    for (int i = 0; i < started; ++i) pthread_join(th[i], NULL);
    return 0;
}

int or_burn_batch(const or_net *net, double rtol, double atol, int max_order, int max_steps,
                  int64_t ncells, double dt, double *x, int64_t ld, double *T,
                  const double *ndens, const double *ks, int32_t *status, int32_t *stats,
                  int nthreads)
{
    return or_burn_batch_src(net, rtol, atol, max_order, max_steps, ncells, dt, x, ld, T, ndens, ks,
                             NULL, status, stats, nthreads);
}

int or_nstat(void) { return OR_NSTAT; }
