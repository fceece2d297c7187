"""ctypes binding of the C oracle (test infrastructure only; see package doc)."""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mc_oracle.c")
_OUT = os.path.join(_HERE, "_build", "libmc_oracle.so")
_lock = threading.Lock()
_lib = None

NSTAT = 8
STAT_NAMES = ["steps", "err_fails", "conv_fails", "rhs", "jac", "lu", "newton", "order"]
STATUS = {0: "ok", 1: "max_steps", 2: "h_underflow", 3: "conv_fail", 4: "bad_input", 5: "nonfinite"}

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int32)


def build(force: bool = False, fma: bool = False) -> str:
    """Compile mc_oracle.c into _build/libmc_oracle.so (plain IEEE double:
    -O2, no fast-math, no FMA contraction). fma=True builds the same source
    with FMA contraction into a separate library: a rounding twin used only to
    calibrate the parity rule."""
    out = _OUT.replace(".so", "_fma.so") if fma else _OUT
    os.makedirs(os.path.dirname(out), exist_ok=True)
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(_SRC):
        tmp = out + f".tmp{os.getpid()}"
        flags = ["-mfma", "-ffp-contract=fast"] if fma else ["-ffp-contract=off"]
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared",
                               "-fno-fast-math", "-Wall", "-o", tmp, _SRC, "-lm", "-lpthread"] + flags)
        os.replace(tmp, out)
    return out


def rounding_twin():
    """A second, independent instance of this module bound to the FMA-contracted
    build of the same oracle source (same algorithm, different rounding)."""
    import importlib.util
    spec = importlib.util.spec_from_file_location("oracle_fma_twin", __file__)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    path = build(fma=True)
    mod.build = lambda force=False, fma=False: path
    return mod


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            L.or_net_create.restype = C.c_void_p
            L.or_net_create.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, _ip, _ip] + [_dp] * 7 + [C.c_double]
            L.or_net_destroy.argtypes = [C.c_void_p]
            L.or_net_eval.argtypes = [C.c_void_p, C.c_double, C.c_double, _dp, _dp, _dp, _dp]
            L.or_burn_batch.argtypes = [C.c_void_p, C.c_double, C.c_double, C.c_int, C.c_int,
                                        C.c_int64, C.c_double, _dp, C.c_int64, _dp, _dp, _dp,
                                        _ip, _ip, C.c_int]
            L.or_burn_batch_src.argtypes = [C.c_void_p, C.c_double, C.c_double, C.c_int, C.c_int,
                                            C.c_int64, C.c_double, _dp, C.c_int64, _dp, _dp, _dp, _dp,
                                            _ip, _ip, C.c_int]
            L.or_net_fd_jac.argtypes = [C.c_void_p, C.c_double, C.c_double, _dp, _dp, C.c_double, C.c_double,
                                        _dp]
            L.or_rkc_linear_step.argtypes = [C.c_int, _dp, C.c_int, _dp, C.c_int, C.c_double, C.c_double, _dp]
            L.or_rkc_linear_integrate.argtypes = [C.c_int, _dp, C.c_int, _dp, C.c_double, C.c_double, C.c_int,
                                                  C.c_double, C.c_double, _dp, _ip]
            L.or_burn_batch_ladder.argtypes = [C.c_void_p, C.c_int, _dp, _dp, _ip, _ip, _ip, _ip, C.c_int64,
                                               C.c_double, _dp, C.c_int64, _dp, _dp, _dp, _ip, _ip, _ip,
                                               C.c_int]
            L.or_linear_integrate.argtypes = [C.c_int, _dp, C.c_int, _dp, C.c_double, C.c_double,
                                              C.c_int, C.c_int, C.c_double, C.c_double, _dp, _ip]
            L.or_linear_integrate_steps.argtypes = [C.c_int, _dp, C.c_int, _dp, C.c_double, C.c_double,
                                                    C.c_int, C.c_int, C.c_double, C.c_double, _dp, _ip, _dp,
                                                    C.c_int, _ip]
            L.or_linear_fixed_steps.argtypes = [C.c_int, _dp, C.c_int, _dp, C.c_int, C.c_int, _dp,
                                                C.c_double, _dp, _dp, _dp, _dp]
            L.or_linear_initial_step.argtypes = [C.c_int, _dp, _dp, C.c_double, C.c_double, C.c_double]
            L.or_linear_initial_step.restype = C.c_double
            L.or_linear_newton.argtypes = [C.c_int, _dp, _dp, C.c_double, C.c_double, C.c_double, _dp,
                                           C.c_double, _dp, _ip]
            L.or_bdf_coeffs.argtypes = [C.c_int, _dp, _dp, _dp]
            L.or_err_coef_qm1.argtypes = [C.c_int, _dp]
            L.or_err_coef_qm1.restype = C.c_double
            L.or_err_coef_qp1.argtypes = [C.c_int]
            L.or_err_coef_qp1.restype = C.c_double
            L.or_order_raise_coef.argtypes = [C.c_int, _dp]
            L.or_order_raise_coef.restype = C.c_double
            L.or_order_lower_coefs.argtypes = [C.c_int, _dp, _dp]
            L.or_lu_factor.argtypes = [C.c_int, _dp, _ip]
            L.or_lu_solve.argtypes = [C.c_int, _dp, _ip, _dp]
            L.or_predict.argtypes = [C.c_int, C.c_int, _dp]
            L.or_retract.argtypes = [C.c_int, C.c_int, _dp]
            _lib = L
    return _lib


def _d(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_dp)


def _i(a: np.ndarray):
    assert a.dtype == np.int32 and a.flags.c_contiguous
    return a.ctypes.data_as(_ip)


class OracleNetwork:
    """A network (``mc_inputs.Network``) loaded into the oracle."""

    def __init__(self, net):
        self.net = net
        L = lib()
        f = lambda a: np.ascontiguousarray(a, dtype=np.float64)
        self._keep = [np.ascontiguousarray(net.react, dtype=np.int32).ravel(),
                      np.ascontiguousarray(net.prod, dtype=np.int32).ravel(),
                      f(net.A_f), f(net.b_f), f(net.C_f), f(net.A_r), f(net.b_r), f(net.C_r),
                      f(net.dE_eV)]
        k = self._keep
        self.h = L.or_net_create(net.n_species, net.n_elements, net.n_reactions,
                                 1 if net.energy_eq else 0, _i(k[0]), _i(k[1]), *[_d(a) for a in k[2:]],
                                 float(net.gamma))
        if not self.h:
            raise ValueError("network too large for the oracle")

    def __del__(self):
        try:
            lib().or_net_destroy(self.h)
        except Exception:
            pass

    def eval(self, y, ndens=1.0, T_iso=1.0, rate_scale=None, jac=True):
        """Right-hand side (and Jacobian) of one state y."""
        y = np.ascontiguousarray(y, dtype=np.float64)
        n = y.size
        f = np.zeros(n)
        J = np.zeros((n, n)) if jac else None
        ks = None if rate_scale is None else np.ascontiguousarray(rate_scale, dtype=np.float64)
        rc = lib().or_net_eval(self.h, float(ndens), float(T_iso), _d(ks) if ks is not None else None,
                               _d(y), _d(f), _d(J) if jac else None)
        if rc != 0:
            raise ValueError("state cannot be evaluated (T <= 0)")
        return (f, J) if jac else f

    def fd_jac(self, y, ndens=1.0, T_iso=1.0, rate_scale=None, rtol=1e-6, atol=1e-10):
        """Forward-difference Jacobian of one state y (the integrator's
        alternative to the analytic one)."""
        y = np.ascontiguousarray(y, dtype=np.float64)
        J = np.zeros((y.size, y.size))
        ks = None if rate_scale is None else np.ascontiguousarray(rate_scale, dtype=np.float64)
        rc = lib().or_net_fd_jac(self.h, float(ndens), float(T_iso), _d(ks) if ks is not None else None,
                                 _d(y), float(rtol), float(atol), _d(J))
        if rc != 0:
            raise ValueError("state cannot be evaluated")
        return J


def burn(onet: OracleNetwork, cells: dict, dt: float, rtol=1e-6, atol=1e-10, max_order=5,
         max_steps=100000, nthreads=None, index=None, source=None):
    """Burn cells (SoA dict from mc_inputs) on host threads. ``index`` selects
    a subset of the cells. ``source`` [n_ode, n] is a constant source added to
    each cell's right-hand side (species rates, then the energy rate), as in a
    burn coupled by spectral deferred corrections. Returns (x [S, n], T [n] or
    None, status [n], stats [NSTAT, n])."""
    net = onet.net
    x = np.asarray(cells["x"], dtype=np.float64)
    sel = (lambda a: a[..., index]) if index is not None else (lambda a: a)
    x = np.array(sel(x), dtype=np.float64, order="C", copy=True)
    n = x.shape[1]
    T = None if cells.get("T") is None else np.array(sel(np.asarray(cells["T"], dtype=np.float64)), order="C", copy=True)
    nd = None if cells.get("ndens") is None else np.ascontiguousarray(sel(np.asarray(cells["ndens"], dtype=np.float64)))
    ks = None if cells.get("rate_scale") is None else np.ascontiguousarray(sel(np.asarray(cells["rate_scale"], dtype=np.float64)))
    status = np.zeros(n, dtype=np.int32)
    stats = np.zeros((NSTAT, n), dtype=np.int32)
    nthreads = nthreads or os.cpu_count() or 1
    if source is None:
        rc = lib().or_burn_batch(onet.h, rtol, atol, max_order, max_steps, n, dt, _d(x), n,
                                 _d(T) if T is not None else None, _d(nd) if nd is not None else None,
                                 _d(ks) if ks is not None else None, _i(status), _i(stats), int(nthreads))
    else:
        src = np.array(sel(np.asarray(source, dtype=np.float64)), dtype=np.float64, order="C", copy=True)
        if src.shape != (net.n_ode, n):
            raise ValueError(f"source must be [{net.n_ode}, {n}]")
        rc = lib().or_burn_batch_src(onet.h, rtol, atol, max_order, max_steps, n, dt, _d(x), n,
                                     _d(T) if T is not None else None, _d(nd) if nd is not None else None,
                                     _d(ks) if ks is not None else None, _d(src), _i(status), _i(stats),
                                     int(nthreads))
    if rc != 0:
        raise ValueError("oracle batch rejected its arguments")
    return x, T, status, stats


def burn_ladder(onet: OracleNetwork, cells: dict, dt: float, rungs, nthreads=None, index=None):
    """Burn cells with a retry ladder: ``rungs`` is a list (1 to 8) of dicts
    with keys rtol, atol, max_order, max_steps, jac ("analytic" or "fd") and
    method ("bdf" or "rkc", the explicit Runge-Kutta-Chebyshev integrator).
    A cell that fails with a retryable status is burned again from its inputs
    with the next rung. Returns (x, T, status, stats, rung), where rung [n]
    is the rung whose attempt gave the cell's outputs."""
    net = onet.net
    sel = (lambda a: a[..., index]) if index is not None else (lambda a: a)
    x = np.array(sel(np.asarray(cells["x"], dtype=np.float64)), dtype=np.float64, order="C", copy=True)
    n = x.shape[1]
    T = None if cells.get("T") is None else np.array(sel(np.asarray(cells["T"], dtype=np.float64)), order="C", copy=True)
    nd = None if cells.get("ndens") is None else np.ascontiguousarray(sel(np.asarray(cells["ndens"], dtype=np.float64)))
    ks = None if cells.get("rate_scale") is None else np.ascontiguousarray(sel(np.asarray(cells["rate_scale"], dtype=np.float64)))
    k = len(rungs)
    rt = np.array([r.get("rtol", 1e-6) for r in rungs], dtype=np.float64)
    at = np.array([r.get("atol", 1e-10) for r in rungs], dtype=np.float64)
    mo = np.array([r.get("max_order", 5) for r in rungs], dtype=np.int32)
    ms = np.array([r.get("max_steps", 100000) for r in rungs], dtype=np.int32)
    fd = np.array([1 if r.get("jac", "analytic") == "fd" else 0 for r in rungs], dtype=np.int32)
    meth = np.array([{"bdf": 0, "rkc": 1}[r.get("method", "bdf")] for r in rungs], dtype=np.int32)
    status = np.zeros(n, dtype=np.int32)
    stats = np.zeros((NSTAT, n), dtype=np.int32)
    rung = np.zeros(n, dtype=np.int32)
    nthreads = nthreads or os.cpu_count() or 1
    rc = lib().or_burn_batch_ladder(onet.h, k, _d(rt), _d(at), _i(mo), _i(ms), _i(fd), _i(meth), n, dt, _d(x), n,
                                    _d(T) if T is not None else None, _d(nd) if nd is not None else None,
                                    _d(ks) if ks is not None else None, _i(status), _i(stats), _i(rung),
                                    int(nthreads))
    if rc != 0:
        raise ValueError("oracle ladder rejected its arguments")
    return x, T, status, stats, rung


def rkc_linear_step(A, c, y, t, h, s):
    """One RKC step with s stages on y' = A y + sum_k c[k] t^k."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    c = np.ascontiguousarray(np.atleast_2d(c), dtype=np.float64)
    y = np.array(y, dtype=np.float64, copy=True)
    if lib().or_rkc_linear_step(y.size, _d(A), c.shape[0] - 1, _d(c), int(s), float(t), float(h), _d(y)) != 0:
        raise ValueError("rkc step rejected its arguments")
    return y


def rkc_linear_integrate(A, c, y0, t0, t1, rtol=1e-6, atol=1e-10, max_steps=100000):
    """Integrate y' = A y + sum_k c[k] t^k from t0 to t1 with the adaptive RKC.
    Returns (y, status, stats)."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    c = np.ascontiguousarray(np.atleast_2d(c), dtype=np.float64)
    y = np.array(y0, dtype=np.float64, copy=True)
    st = np.zeros(NSTAT, dtype=np.int32)
    s = lib().or_rkc_linear_integrate(y.size, _d(A), c.shape[0] - 1, _d(c), rtol, atol, max_steps, t0, t1,
                                      _d(y), _i(st))
    return y, s, st


def linear_integrate(A, c, y0, t0, t1, rtol=1e-6, atol=1e-10, max_order=5, max_steps=100000):
    """Integrate y' = A y + sum_k c[k] t^k from t0 to t1 with the adaptive BDF."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    c = np.ascontiguousarray(np.atleast_2d(c), dtype=np.float64)
    y = np.array(y0, dtype=np.float64)
    st = np.zeros(NSTAT, dtype=np.int32)
    s = lib().or_linear_integrate(y.size, _d(A), c.shape[0] - 1, _d(c), rtol, atol, max_order,
                                  max_steps, t0, t1, _d(y), _i(st))
    return y, s, dict(zip(STAT_NAMES, st.tolist()))


def linear_integrate_steps(A, c, y0, t0, t1, rtol=1e-6, atol=1e-10, max_order=5, max_steps=100000, cap=200000):
    """linear_integrate with the record of accepted steps: rows (t after the
    step, h, q, error estimate in the error-test norm)."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    c = np.ascontiguousarray(np.atleast_2d(c), dtype=np.float64)
    y = np.array(y0, dtype=np.float64)
    st = np.zeros(NSTAT, dtype=np.int32)
    log = np.zeros((cap, 4), dtype=np.float64)
    nlog = np.zeros(1, dtype=np.int32)
    s = lib().or_linear_integrate_steps(y.size, _d(A), c.shape[0] - 1, _d(c), rtol, atol, max_order,
                                        max_steps, t0, t1, _d(y), _i(st), _d(log), cap, _i(nlog))
    return y, s, dict(zip(STAT_NAMES, st.tolist())), log[:int(nlog[0])].copy()


def linear_fixed_steps(A, c, q, hs, t0, z, hist):
    """Fixed-order steps with prescribed sizes ``hs`` (full Newton, no error
    control). z: Nordsieck array [(q+1), n]; hist: past steps (most recent
    first). Returns (z, hist, e [steps, n], est [steps, n])."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    c = np.ascontiguousarray(np.atleast_2d(c), dtype=np.float64)
    z = np.ascontiguousarray(z, dtype=np.float64).copy()
    n = z.shape[1]
    hs = np.ascontiguousarray(hs, dtype=np.float64)
    h8 = np.zeros(8)
    h8[: len(hist)] = hist
    e = np.zeros((hs.size, n))
    est = np.zeros((hs.size, n))
    rc = lib().or_linear_fixed_steps(n, _d(A), c.shape[0] - 1, _d(c), q, hs.size, _d(hs), t0,
                                     _d(z), _d(h8), _d(e), _d(est))
    if rc != 0:
        raise RuntimeError("Newton did not converge")
    return z, h8, e, est


def linear_initial_step(A, y0, rtol=1e-6, atol=1e-10, span=1e30):
    """The integrator's starting step for y' = A y at y0."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    y0 = np.ascontiguousarray(y0, dtype=np.float64)
    return lib().or_linear_initial_step(y0.size, _d(A), _d(y0), rtol, atol, span)


def linear_newton(A, z0, z1, l1, h, gamma_p_ratio, w, cq=1.0):
    """The integrator's modified Newton on y' = A y: returns (iterates e_k as
    rows, outcome 0 converged / 1 failed); see or_linear_newton."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    n = A.shape[0]
    z = np.ascontiguousarray(np.concatenate([z0, z1]), dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.float64)
    tr = np.zeros(3 * n)
    res = np.zeros(1, dtype=np.int32)
    k = lib().or_linear_newton(n, _d(A), _d(z), l1, h, gamma_p_ratio, _d(w), cq, _d(tr), _i(res))
    if k < 0:
        raise ValueError("bad arguments")
    return tr[:k * n].reshape(k, n), int(res[0])


def bdf_coeffs(q, xi):
    xi = np.ascontiguousarray(xi, dtype=np.float64)
    l = np.zeros(q + 1)
    cq = np.zeros(1)
    lib().or_bdf_coeffs(q, _d(xi), _d(l), _d(cq))
    return l, float(cq[0])


def err_coef_qm1(q, xi):
    return lib().or_err_coef_qm1(q, _d(np.ascontiguousarray(xi, dtype=np.float64)))


def err_coef_qp1(q):
    return lib().or_err_coef_qp1(q)


def order_raise_coef(q, xi):
    return lib().or_order_raise_coef(q, _d(np.ascontiguousarray(xi, dtype=np.float64)))


def order_lower_coefs(q, xi):
    c = np.zeros(q + 1)
    lib().or_order_lower_coefs(q, _d(np.ascontiguousarray(xi, dtype=np.float64)), _d(c))
    return c


def lu_factor(a):
    a = np.ascontiguousarray(a, dtype=np.float64).copy()
    n = a.shape[0]
    piv = np.zeros(n, dtype=np.int32)
    rc = lib().or_lu_factor(n, _d(a), _i(piv))
    return a, piv, rc


def lu_solve(lu, piv, b):
    b = np.ascontiguousarray(b, dtype=np.float64).copy()
    lib().or_lu_solve(lu.shape[0], _d(np.ascontiguousarray(lu)), _i(piv), _d(b))
    return b


def predict(z):
    z = np.ascontiguousarray(z, dtype=np.float64).copy()
    lib().or_predict(z.shape[1], z.shape[0] - 1, _d(z))
    return z


def retract(z):
    z = np.ascontiguousarray(z, dtype=np.float64).copy()
    lib().or_retract(z.shape[1], z.shape[0] - 1, _d(z))
    return z
