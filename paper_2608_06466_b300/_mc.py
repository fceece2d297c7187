"""ctypes binding of libmc.so with the C ABI's names (include/mc.h).

Argument marshalling only: every step of the burn runs in the library's CUDA
kernels. Cell arrays may be torch CUDA tensors (device path, asynchronous on
the given stream) or numpy arrays / CPU tensors (host path, synchronous). If
libmc.so is missing or cannot be loaded, importing this module raises.
MC_LIBRARY, when set, names the library file to load instead (the
bounds-check build libmc_check.so, for instance).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("MC_LIBRARY") or os.path.join(_HERE, "libmc.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with `python paper_2608_06466_b300/build.py` "
                      "(there is no CPU fallback)")
lib = C.CDLL(LIB_PATH)

MC_OK, MC_PENDING = 0, 1
ERRORS = {-1: "MC_E_INVALID", -2: "MC_E_NOMEM", -3: "MC_E_CUDA", -4: "MC_E_BUSY", -5: "MC_E_TIMEOUT",
          -6: "MC_E_NOTFOUND", -7: "MC_E_BUDGET", -8: "MC_E_UNSUPPORTED"}
CELL_STATUS = {0: "ok", 1: "max_steps", 2: "h_underflow", 3: "conv_fail", 4: "bad_input", 5: "nonfinite"}
STAT_NAMES = ["steps", "err_fails", "conv_fails", "rhs", "jac", "lu", "newton", "order"]
MC_NSTAT = 8
MC_VARIANT_AUTO, MC_VARIANT_PLAIN, MC_VARIANT_PERSISTENT, MC_VARIANT_WARP = 0, 1, 2, 3

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int32)


class mc_network_desc(C.Structure):
    _fields_ = [("n_species", C.c_int32), ("n_elements", C.c_int32), ("n_reactions", C.c_int32),
                ("energy_eq", C.c_int32), ("react", _ip), ("prod", _ip),
                ("A_f", _dp), ("b_f", _dp), ("C_f", _dp), ("A_r", _dp), ("b_r", _dp), ("C_r", _dp),
                ("dE_eV", _dp), ("gamma", C.c_double)]


class mc_burn_opts(C.Structure):
    _fields_ = [("rtol", C.c_double), ("atol", C.c_double), ("max_order", C.c_int32),
                ("max_steps", C.c_int32), ("lu_precision", C.c_int32), ("variant", C.c_int32),
                ("block_threads", C.c_int32), ("blocks_per_sm", C.c_int32), ("straggler_steps", C.c_int32),
                ("jacobian", C.c_int32), ("staging", C.c_int32)]


class mc_rung(C.Structure):
    _fields_ = [("opts", mc_burn_opts), ("method", C.c_int32)]


class mc_segment(C.Structure):
    _fields_ = [("net", C.c_void_p), ("n_cells", C.c_int64), ("ld", C.c_int64), ("x", C.c_void_p),
                ("T", C.c_void_p), ("ndens", C.c_void_p), ("rate_scale", C.c_void_p),
                ("status", C.c_void_p), ("stats", C.c_void_p), ("dt", C.c_double)]


class mc_request_info(C.Structure):
    _fields_ = [("state", C.c_int32), ("n_failed", C.c_int32), ("n_cells", C.c_int64),
                ("t_submit", C.c_double), ("t_admit", C.c_double), ("t_done", C.c_double),
                ("gpu_start", C.c_double), ("gpu_end", C.c_double)]


class mc_bounds_info(C.Structure):
    _fields_ = [("enabled", C.c_int32), ("refused", C.c_uint32), ("first_site", C.c_int32), ("pad", C.c_int32),
                ("first_index", C.c_int64), ("first_bound", C.c_int64), ("calls_checked", C.c_int64),
                ("cells_checked", C.c_int64), ("cells_not_once", C.c_int64)]


def _sig(name, res, args):
    f = getattr(lib, name, None)
    if f is None:
        return None
    f.restype = res
    f.argtypes = args
    return f


_sig("mc_burn_opts_default", None, [C.POINTER(mc_burn_opts)])
_sig("mc_network_create", C.c_int32, [C.POINTER(mc_network_desc), C.POINTER(C.c_void_p)])
_sig("mc_network_destroy", C.c_int32, [C.c_void_p])
_sig("mc_network_n_ode", C.c_int32, [C.c_void_p])
_sig("mc_burn_batch", C.c_int32, [C.c_void_p, C.POINTER(mc_burn_opts), C.c_int64, C.c_double, C.c_void_p,
                                  C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                  C.c_void_p])
_sig("mc_burn_batch_sdc", C.c_int32, [C.c_void_p, C.POINTER(mc_burn_opts), C.c_int64, C.c_double, C.c_void_p,
                                      C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                      C.c_void_p, C.c_void_p])
_sig("mc_burn_ladder", C.c_int32, [C.c_void_p, C.POINTER(mc_rung), C.c_int32, C.c_int64, C.c_double, C.c_void_p,
                                   C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                   C.c_void_p, C.c_void_p])
_sig("mc_burn_batch_noalloc", C.c_int32, [C.c_void_p, C.POINTER(mc_burn_opts), C.c_int64, C.c_double, C.c_void_p,
                                          C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                          C.c_void_p])
_sig("mc_burn_mixed", C.c_int32, [C.POINTER(mc_segment), C.c_int32, C.POINTER(mc_burn_opts), C.c_double,
                                  C.c_void_p])
_sig("mc_graph_create", C.c_int32, [C.POINTER(mc_segment), C.c_int32, C.POINTER(mc_burn_opts), C.c_double,
                                    C.c_void_p, C.c_void_p, C.POINTER(C.c_void_p)])
_sig("mc_graph_launch", C.c_int32, [C.c_void_p, C.c_void_p])
_sig("mc_graph_destroy", C.c_int32, [C.c_void_p])
_sig("mc_server_create", C.c_int32, [C.c_int32, C.c_uint64, C.POINTER(mc_burn_opts), C.POINTER(C.c_void_p)])
_sig("mc_request_submit", C.c_int32, [C.c_void_p, C.c_void_p, C.POINTER(mc_burn_opts), C.c_int64, C.c_double,
                                      C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p,
                                      C.POINTER(C.c_uint64)])
_sig("mc_request_bytes", C.c_int32, [C.c_void_p, C.POINTER(mc_burn_opts), C.c_int64, C.POINTER(C.c_uint64),
                                     C.POINTER(C.c_uint64)])
_sig("mc_request_poll", C.c_int32, [C.c_void_p, C.c_uint64, C.POINTER(mc_request_info)])
_sig("mc_server_drain", C.c_int32, [C.c_void_p, C.c_double])
_sig("mc_server_destroy", C.c_int32, [C.c_void_p])
_sig("mc_last_error", C.c_char_p, [])
_sig("mc_version", C.c_int32, [])
_sig("mc_launch_count", C.c_int64, [C.c_int32])
_sig("mc_alloc_count", C.c_int64, [])
_sig("mc_network_rates", C.c_int32, [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64,
                                     C.c_void_p])
_sig("mc_network_rhs", C.c_int32, [C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p,
                                   C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p])
_sig("mc_autotune", C.c_int32, [C.c_void_p, C.POINTER(mc_burn_opts), C.c_int64, C.c_double, C.c_void_p, C.c_int64,
                                C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(mc_burn_opts)])
_sig("mc_probe_fma_rate", C.c_int32, [C.POINTER(C.c_double), C.POINTER(C.c_double)])
_sig("mc_bounds_report", C.c_int32, [C.c_int32, C.POINTER(mc_bounds_info)])
_sig("mc_bounds_reset", C.c_int32, [C.c_int32])


class MCError(RuntimeError):
    pass


def check(rc: int, what: str = "") -> int:
    if rc < 0:
        msg = lib.mc_last_error().decode(errors="replace")
        raise MCError(f"{what}: {ERRORS.get(rc, rc)}: {msg}")
    return rc


def mc_last_error() -> str:
    return lib.mc_last_error().decode(errors="replace")


def mc_burn_opts_default(**over) -> mc_burn_opts:
    o = mc_burn_opts()
    lib.mc_burn_opts_default(C.byref(o))
    for k, v in over.items():
        setattr(o, k, v)
    return o


def _ptr(a):
    """Raw address of a torch tensor, numpy array or None."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    raise TypeError(f"unsupported array type {type(a)}")


def _stream_ptr(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


class Network:
    """An uploaded network (handle owner). ``net`` is an object with the fields
    of mc_inputs.Network (n_species, react, prod, A_f, ...)."""

    def __init__(self, net):
        self.src = net
        f = lambda a: np.ascontiguousarray(a, dtype=np.float64)
        self._keep = [np.ascontiguousarray(net.react, dtype=np.int32).ravel(),
                      np.ascontiguousarray(net.prod, dtype=np.int32).ravel(),
                      f(net.A_f), f(net.b_f), f(net.C_f), f(net.A_r), f(net.b_r), f(net.C_r), f(net.dE_eV)]
        k = self._keep
        d = mc_network_desc(net.n_species, net.n_elements, int(k[2].size), 1 if net.energy_eq else 0,
                            k[0].ctypes.data_as(_ip), k[1].ctypes.data_as(_ip),
                            *[a.ctypes.data_as(_dp) for a in k[2:]], float(net.gamma))
        h = C.c_void_p()
        check(lib.mc_network_create(C.byref(d), C.byref(h)), "mc_network_create")
        self.handle = h
        self.n_species = net.n_species
        self.n_reactions = int(k[2].size)
        self.energy_eq = bool(net.energy_eq)
        self.n_ode = lib.mc_network_n_ode(h)

    def close(self):
        if self.handle:
            lib.mc_network_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mc_network_create(net) -> Network:
    return Network(net)


def mc_network_destroy(net: Network) -> None:
    net.close()


def mc_burn_batch(net: Network, opts: mc_burn_opts | None, n_cells: int, dt: float, x, ld: int, T, ndens,
                  rate_scale, status, stats, stream=None) -> int:
    """Same arguments as the C function; arrays are torch tensors or numpy
    arrays laid out as in mc.h ([rows][ld])."""
    o = opts if opts is not None else mc_burn_opts_default()
    return check(lib.mc_burn_batch(net.handle, C.byref(o), int(n_cells), float(dt), _ptr(x), int(ld), _ptr(T),
                                   _ptr(ndens), _ptr(rate_scale), _ptr(status), _ptr(stats),
                                   _stream_ptr(stream)), "mc_burn_batch")


def mc_burn_batch_sdc(net: Network, opts: mc_burn_opts | None, n_cells: int, dt: float, x, ld: int, T, ndens,
                      rate_scale, source, status, stats, stream=None) -> int:
    """mc_burn_batch with a constant source [n_ode][ld] added to the right-hand side."""
    o = opts if opts is not None else mc_burn_opts_default()
    return check(lib.mc_burn_batch_sdc(net.handle, C.byref(o), int(n_cells), float(dt), _ptr(x), int(ld), _ptr(T),
                                       _ptr(ndens), _ptr(rate_scale), _ptr(source), _ptr(status), _ptr(stats),
                                       _stream_ptr(stream)), "mc_burn_batch_sdc")


MC_JAC_ANALYTIC, MC_JAC_FD = 0, 1
MC_STAGING_AUTO, MC_STAGING_SHARED, MC_STAGING_LANE = 0, 1, 2
MC_METHOD_BDF, MC_METHOD_RKC = 0, 1


def rung(method=MC_METHOD_BDF, **opts) -> mc_rung:
    """One retry-ladder rung: mc_burn_opts fields as keywords, and the method."""
    return mc_rung(mc_burn_opts_default(**opts), int(method))


def mc_burn_ladder(net: Network, rungs, n_cells: int, dt: float, x, ld: int, T, ndens, rate_scale, status, stats,
                   rung_out=None, stream=None) -> int:
    """Burn with a retry ladder (device arrays); rung_out [n] int32 receives
    the rung that produced each cell's outputs."""
    arr = (mc_rung * len(rungs))(*rungs)
    return check(lib.mc_burn_ladder(net.handle, arr, len(rungs), int(n_cells), float(dt), _ptr(x), int(ld), _ptr(T),
                                    _ptr(ndens), _ptr(rate_scale), _ptr(status), _ptr(stats), _ptr(rung_out),
                                    _stream_ptr(stream)), "mc_burn_ladder")


MC_NOALLOC_MAX_CELLS = 1 << 20


def mc_burn_batch_noalloc(net: Network, opts: mc_burn_opts | None, n_cells: int, dt: float, x, ld: int, T, ndens,
                          rate_scale, status, stats, stream=None) -> int:
    """The allocation-free burn: device arrays only, n_cells <= MC_NOALLOC_MAX_CELLS,
    scratch in a fixed device array shared by all calls (overlapping calls race)."""
    o = opts if opts is not None else mc_burn_opts_default()
    return check(lib.mc_burn_batch_noalloc(net.handle, C.byref(o), int(n_cells), float(dt), _ptr(x), int(ld), _ptr(T),
                                           _ptr(ndens), _ptr(rate_scale), _ptr(status), _ptr(stats),
                                           _stream_ptr(stream)), "mc_burn_batch_noalloc")


def segment(net: Network, n_cells, ld, x, T, ndens, rate_scale, status, stats, dt=0.0) -> mc_segment:
    """One segment of a mixed burn; dt = 0 takes the call's dt."""
    return mc_segment(net.handle.value, int(n_cells), int(ld), _ptr(x), _ptr(T), _ptr(ndens), _ptr(rate_scale),
                      _ptr(status), _ptr(stats), float(dt))


def mc_burn_mixed(segs, opts: mc_burn_opts | None, dt: float, stream=None) -> int:
    arr = (mc_segment * len(segs))(*segs)
    o = opts if opts is not None else mc_burn_opts_default()
    return check(lib.mc_burn_mixed(arr, len(segs), C.byref(o), float(dt), _stream_ptr(stream)), "mc_burn_mixed")


class Graph:
    def __init__(self, segs, opts, dt, totals=None, stream=None):
        self._segs = (mc_segment * len(segs))(*segs)
        self._opts = opts if opts is not None else mc_burn_opts_default()
        h = C.c_void_p()
        check(lib.mc_graph_create(self._segs, len(segs), C.byref(self._opts), float(dt), _ptr(totals),
                                  _stream_ptr(stream), C.byref(h)), "mc_graph_create")
        self.handle = h

    def launch(self, stream=None):
        return check(lib.mc_graph_launch(self.handle, _stream_ptr(stream)), "mc_graph_launch")

    def close(self):
        if self.handle:
            lib.mc_graph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mc_graph_create(segs, opts, dt, totals=None, stream=None) -> Graph:
    return Graph(segs, opts, dt, totals, stream)


class Server:
    def __init__(self, device: int = 0, hbm_budget_bytes: int = 150 << 30, opts: mc_burn_opts | None = None):
        self._opts = opts if opts is not None else mc_burn_opts_default()
        h = C.c_void_p()
        check(lib.mc_server_create(int(device), int(hbm_budget_bytes), C.byref(self._opts), C.byref(h)),
              "mc_server_create")
        self.handle = h
        self._arrays = {}  # request id -> its arrays, held until the request is done

    def submit(self, net: Network, n_cells, dt, x, ld, T, ndens, status, opts: mc_burn_opts | None = None) -> int:
        """Queue a request. The library reads and writes the arrays until the
        request is done; the binding holds them until then."""
        rid = C.c_uint64()
        check(lib.mc_request_submit(self.handle, net.handle, C.byref(opts) if opts is not None else None,
                                    int(n_cells), float(dt), _ptr(x), int(ld), _ptr(T), _ptr(ndens), _ptr(status),
                                    C.byref(rid)), "mc_request_submit")
        self._arrays[rid.value] = (x, T, ndens, status)
        return rid.value

    @staticmethod
    def request_bytes(net: Network, n_cells, opts: mc_burn_opts | None = None):
        """(state bytes, stream scratch bytes) a request charges against the budget."""
        a, b = C.c_uint64(), C.c_uint64()
        check(lib.mc_request_bytes(net.handle, C.byref(opts) if opts is not None else None, int(n_cells),
                                   C.byref(a), C.byref(b)), "mc_request_bytes")
        return a.value, b.value

    def poll(self, req_id: int):
        info = mc_request_info()
        rc = check(lib.mc_request_poll(self.handle, C.c_uint64(req_id), C.byref(info)), "mc_request_poll")
        if rc == MC_OK:
            self._arrays.pop(req_id, None)
        return rc, info

    def drain(self, timeout_s: float = 600.0):
        rc = check(lib.mc_server_drain(self.handle, float(timeout_s)), "mc_server_drain")
        self._arrays.clear()  # every request is done
        return rc

    def close(self):
        if self.handle:
            check(lib.mc_server_destroy(self.handle), "mc_server_destroy")
            self.handle = None
            self._arrays.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mc_server_create(device=0, hbm_budget_bytes=150 << 30, opts=None) -> Server:
    return Server(device, hbm_budget_bytes, opts)


def mc_network_rates(net: Network, n, T, kf, kr, ld, stream=None) -> int:
    return check(lib.mc_network_rates(net.handle, int(n), _ptr(T), _ptr(kf), _ptr(kr), int(ld), _stream_ptr(stream)),
                 "mc_network_rates")


def mc_network_rhs(net: Network, n, y, ld, T, ndens, rate_scale, f, jac, ok, stream=None) -> int:
    return check(lib.mc_network_rhs(net.handle, int(n), _ptr(y), int(ld), _ptr(T), _ptr(ndens), _ptr(rate_scale),
                                    _ptr(f), _ptr(jac), _ptr(ok), _stream_ptr(stream)), "mc_network_rhs")


def mc_autotune(net: Network, opts, n_sample, dt, x, ld, T, ndens, stream=None) -> mc_burn_opts:
    o = opts if opts is not None else mc_burn_opts_default()
    best = mc_burn_opts()
    check(lib.mc_autotune(net.handle, C.byref(o), int(n_sample), float(dt), _ptr(x), int(ld), _ptr(T), _ptr(ndens),
                          _stream_ptr(stream), C.byref(best)), "mc_autotune")
    return best


def mc_probe_fma_rate():
    """(FP64, FP32) fused multiply-add rate of the current device in TFLOP/s."""
    a, b = C.c_double(), C.c_double()
    check(lib.mc_probe_fma_rate(C.byref(a), C.byref(b)), "mc_probe_fma_rate")
    return a.value, b.value


def mc_launch_count(reset: bool = False) -> int:
    return int(lib.mc_launch_count(1 if reset else 0))


def mc_bounds_report(device: int = 0) -> dict:
    """The bounds-check record of a device (enabled = 0 in the normal build)."""
    info = mc_bounds_info()
    check(lib.mc_bounds_report(device, C.byref(info)), "mc_bounds_report")
    return {f: getattr(info, f) for f, _ in mc_bounds_info._fields_ if f != "pad"}


def mc_bounds_reset(device: int = 0) -> None:
    check(lib.mc_bounds_reset(device), "mc_bounds_reset")


def mc_alloc_count() -> int:
    return int(lib.mc_alloc_count())
