// mc_kernels.cuh -- burn kernels: plain (one launch, one thread per cell) and
// persistent (workers pull cells from a queue; a lane whose cell is done takes
// the next one, so a warp never idles behind one stiff cell -- the thread
// divergence the paper's Software design section, paragraph 3, names).
#pragma once

#include "mc_check.cuh"
#include "mc_coop.cuh"

namespace mc {

// Cell arrays of one launch (structure-of-arrays, see mc.h).
struct CellArgs {
  int64_t n_cells;          // number of cells (or entries of index)
  int64_t ld;
  double dt;
  double *x;
  double *T;
  const double *nd;
  const double *ks;
  const double *src;        // optional constant source [n_ode][ld]
  int32_t *status;
  int32_t *stats;
  const int32_t *index;     // optional cell list: entry k is cell index[k]
  const uint32_t *n_dev;    // optional device-side count overriding n_cells
  int32_t *retry;           // FP32 pass: cells to redo in FP64 (nullptr = none)
  uint32_t *retry_count;
  uint32_t retry_mask;      // statuses (bit 1 << status) that go to retry
  int32_t *lretry;          // retry ladder: cells for the next rung (nullptr = none)
  uint32_t *lretry_count;
  uint32_t lretry_mask;     // statuses that go to lretry
  int32_t *rung;            // retry ladder: rung that wrote each cell's outputs, or nullptr
  int32_t rung_id;
#ifdef MC_BOUNDS_CHECK
  BoundsCheck *bc;          // the device's check record
  int64_t cells;            // cells of the call (bound of cell indices and list positions; 0: n_cells)
#endif
};

// statuses an FP32-matrix pass hands to its FP64 retry pass
constexpr uint32_t FP32_RETRY_MASK = (1u << CELL_CONV_FAIL) | (1u << CELL_H_UNDERFLOW) | (1u << CELL_RETRY64);
// statuses a retry-ladder rung hands to the next rung
constexpr uint32_t LADDER_MASK = (1u << CELL_MAX_STEPS) | (1u << CELL_H_UNDERFLOW) | (1u << CELL_CONV_FAIL) |
                                 (1u << CELL_NONFINITE) | (1u << CELL_RETRY64);

// Where a finished cell goes: 1 = the FP64 retry list, 2 = the next rung's
// list, 0 = its outputs are written (status adjusted when nothing takes it).
__device__ __forceinline__ int route_of(const CellArgs &a, int &status) {
  const uint32_t bit = 1u << status;
  if (a.retry && (a.retry_mask & bit)) return 1;
  if (a.lretry && (a.lretry_mask & bit)) return 2;
  if (status == CELL_RETRY64) status = CELL_CONV_FAIL;  // no retry pass to take it
  return 0;
}

__device__ __forceinline__ void push_list(const CellArgs &a, int32_t *list, uint32_t *count, int64_t c) {
  const uint32_t k = atomicAdd(count, 1u);
  if (MC_IN(a, BC_LIST_PUSH, k, MC_CELLS(a))) list[k] = (int32_t)c;
}

__device__ __forceinline__ int64_t cell_of(const CellArgs &a, int64_t k) {
  if (!a.index) return k;
  return MC_IN(a, BC_LIST_READ, k, MC_CELLS(a)) ? (int64_t)a.index[k] : -1;
}

__device__ __forceinline__ int64_t count_of(const CellArgs &a) {
  return a.n_dev ? (int64_t)(*a.n_dev) : a.n_cells;
}

// Load cell c: inputs checked the way the burn's definition needs them
// (finite abundances, T > 0, n > 0; for the energy form sum x > 0), the
// energy form's u = (sum x) k_B T / (gamma - 1). Sets PH_F0, or PH_DONE with
// CELL_BAD_INPUT (outputs then left untouched).
template <int N, typename LT>
__device__ void load_cell(Lane<N, LT> &L, const DNet &net, const CellArgs &a, int64_t c) {
  const int S = net.S, n = net.n;
  L.cell = c;
  if (!MC_IN(a, BC_CELL_LOAD, c, MC_CELLS(a))) {
    L.status = CELL_BAD_INPUT;
    L.phase = PH_DONE;
    L.m = -1;
    return;
  }
  L.status = CELL_OK;
  L.q = 0;
  L.kept = false;
  L.todo = TD_NONE;
  L.eta_pend = 1.0;
#pragma unroll
  for (int k = 0; k < NSTAT; ++k) L.st[k] = 0;
  bool good = true;
  double X = 0.0;
#pragma unroll
  for (int i = 0; i < N; ++i) {
    const double v = (i < S) ? a.x[i * a.ld + c] : 0.0;
    L.z[0][i] = v;
    if (i < S) {
      X += v;
      if (!isfinite(v)) good = false;
    }
  }
  const double nd = a.nd ? a.nd[c] : 1.0;
  if (!(nd > 0.0) || !isfinite(nd)) good = false;
  const double T = a.T ? a.T[c] : 1.0;
  if (!(T > 0.0) || !isfinite(T)) good = false;
  L.cin.nd = nd;
  L.cin.ks = a.ks ? a.ks + c : nullptr;
  L.cin.ks_ld = a.ld;
  L.cin.src = a.src ? a.src + c : nullptr;
  if (net.energy) {
    if (!(X > 0.0) || !isfinite(X)) good = false;
    L.z[0][S] = X * KB_EV * T / net.gm1;
    L.cin.lnT = 0.0;
    L.cin.invT = 0.0;
  } else {
    L.cin.lnT = log(T);
    L.cin.invT = 1.0 / T;
  }
  if (!good) {
    L.status = CELL_BAD_INPUT;
    L.phase = PH_DONE;
    L.m = -1;  // marks "inputs rejected": outputs are not written
    return;
  }
  L.m = 0;
  L.tend = a.dt;
#pragma unroll
  for (int i = 0; i < N; ++i) L.y[i] = (i < n) ? L.z[0][i] : 0.0;
  L.phase = PH_F0;
}

// Write cell results. FP32-matrix runs hand Newton and step-size failures, and
// cells whose refined FP32 solves could not reach the FP64 solve, to an FP64
// retry list instead of writing them, and a retry-ladder rung hands its
// retryable failures to the next rung's list (the inputs stay in place).
template <int N, typename LT>
__device__ void store_cell(Lane<N, LT> &L, const DNet &net, const CellArgs &a) {
  const int64_t c = L.cell;
  const int S = net.S;
  const int route = route_of(a, L.status);
  if (route == 1) { push_list(a, a.retry, a.retry_count, c); return; }
  if (route == 2) { push_list(a, a.lretry, a.lretry_count, c); return; }
  if (!MC_IN(a, BC_CELL_STORE, c, MC_CELLS(a))) return;
  MC_STORED(a, c);
  if (a.rung) a.rung[c] = a.rung_id;
  const bool rejected = (L.status == CELL_BAD_INPUT && L.m < 0);
  if (!rejected) {
    double X = 0.0;
#pragma unroll
    for (int i = 0; i < N; ++i)
      if (i < S) {
        a.x[i * a.ld + c] = L.z[0][i];
        X += L.z[0][i];
      }
    if (net.energy) a.T[c] = net.gm1 * L.z[0][S] / (KB_EV * X);
  }
  a.status[c] = L.status;
  if (a.stats) {
    L.st[ST_ORDER] = (L.status == CELL_BAD_INPUT) ? 0 : L.q;
#pragma unroll
    for (int k = 0; k < NSTAT; ++k) a.stats[k * a.ld + c] = L.st[k];
  }
}

template <int N, typename LT>
__global__ void __launch_bounds__(256) k_burn_plain(DNet net, Opts o, CellArgs a) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= count_of(a)) return;
  Lane<N, LT> L;
  load_cell(L, net, a, cell_of(a, k));
  while (L.phase != PH_DONE) {
    const bool ok = net_rhs<N>(net, L.cin, L.y, L.f);
    advance(L, net, o, ok);
    if (L.todo == TD_MATRIX) matrix_thread(L, net, o);
    run_stages(L, net, o);
  }
  store_cell(L, net, a);
}

// Straggler hand-off: a cell still running after `threshold` step attempts is
// written (whole lane state, at the start of an attempt) to record k of `rec`
// and finished later by the warp-cooperative kernel; the lane takes a new cell.
struct StragArgs {
  void *rec;           // nullptr: no hand-off
  uint32_t *count;     // records claimed (may exceed cap; only cap are written)
  uint32_t cap;
  int threshold;
  uint32_t *flag;      // per record: 0 not yet written, 1 written, 2 integrated
};

// Relaxed loads for polling: unlike an acquire they leave the SM's L1 (which
// holds the spilled lane state of the thread-form workers) untouched.
__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t *p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned long long ld_relaxed(const unsigned long long *p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release(uint32_t *p, uint32_t v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" : : "l"(p), "r"(v) : "memory");
}

// Persistent worker loop over one queue of cells. `next` counts cells handed
// out (reset to 0 before the launch). Every lane of the warp runs the loop, so
// the warp-wide votes are safe; the loop returns once the queue is drained and
// every lane's cell is stored or handed off. One loop trip: one right-hand
// side for every busy lane, the matrix work of the lanes that wait for it
// (warp-cooperative in the warp's workspace sh, coop_matrix; or, with
// o.lane_matrix, each lane alone, matrix_thread), then the step logic's
// stages.
template <int N, typename LT>
__device__ void persistent_worker(const DNet &net, const Opts &o, const CellArgs &a,
                                  unsigned long long *next, const StragArgs &sa, const WSh<LT> &sh) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int64_t total = count_of(a);
  Lane<N, LT> L;
  L.phase = PH_IDLE;
  L.todo = TD_NONE;
  bool active = true;
  for (;;) {
    if (L.phase == PH_DONE) {
      store_cell(L, net, a);
      L.phase = PH_IDLE;
    }
    const bool want = (L.phase == PH_IDLE) && active;
    const unsigned need = __ballot_sync(FULL, want);
    if (need) {
      const int leader = __ffs(need) - 1;
      unsigned long long base = 0;
      if (lane == leader) base = atomicAdd(next, (unsigned long long)__popc(need));
      base = __shfl_sync(FULL, base, leader);
      if (want) {
        const int64_t k = (int64_t)base + __popc(need & ((1u << lane) - 1u));
        if (k < total) load_cell(L, net, a, cell_of(a, k));
        else active = false;
      }
    }
    if (!__any_sync(FULL, L.phase != PH_IDLE)) break;
    const bool busy = L.phase != PH_IDLE && L.phase != PH_DONE;
    if (busy) {
      const bool ok = net_rhs<N>(net, L.cin, L.y, L.f);
      advance(L, net, o, ok);
    }
    if (o.lane_matrix) {
      if (L.todo == TD_MATRIX) matrix_thread(L, net, o);
    } else {
      coop_matrix<N, LT>(L, net, o, sh);
    }
    if (busy) {
      run_stages(L, net, o);
      if (sa.rec && L.phase == PH_NEWTON && L.m == 0 && L.attempts >= sa.threshold && !L.kept) {
        const uint32_t k = atomicAdd(sa.count, 1u);
        if (k < sa.cap) {
          static_cast<Lane<N, LT> *>(sa.rec)[k] = L;
          if (sa.flag) st_release(&sa.flag[k], 1u);  // record k is complete
          L.phase = PH_IDLE;
        } else {
          L.kept = true;
        }
      }
    }
  }
}

template <int N, typename LT>
__global__ void __launch_bounds__(256) k_burn_persistent(DNet net, Opts o, CellArgs a,
                                                         unsigned long long *next, StragArgs sa,
                                                         int smem_per_warp) {
  extern __shared__ __align__(16) unsigned char smem[];
  const WSh<LT> sh = wsh_carve<N, LT>(smem + (threadIdx.x >> 5) * (size_t)smem_per_warp, net.R);
  persistent_worker<N, LT>(net, o, a, next, sa, sh);
}

// ---- cost order of the cell queue -------------------------------------------
// A cell's result does not depend on where it sits in the queue (each cell is
// integrated on its own, and the hand-off happens at a fixed attempt count), so
// the queue may hand out expensive cells first: the drain at the end of a
// persistent launch then holds cheap cells only, and long cells reach the
// hand-off early. The cost key is dt times the weighted RMS norm of f(y0) with
// the error-test weights 1/(rtol |y0_i| + atol) -- the number of the cell's
// natural time scales in the step, the quantity the starting-step rule
// (Hairer, Norsett & Wanner, Solving ODEs I, II.4) begins from. Keys are
// grouped in half-octaves; bucket 0 is the most expensive.
constexpr int ORDER_BUCKETS = 256;
constexpr int ORDER_CHUNK = 4096;  // cells per block of the scatter kernel

template <int N>
__device__ int cost_bucket(const DNet &net, const Opts &o, const CellArgs &a, int64_t c) {
  const int S = net.S, n = net.n;
  double y[N], f[N];
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
  } else if (good) {
    cin.lnT = log(T);
    cin.invT = 1.0 / T;
  }
  if (!good || !net_rhs<N>(net, cin, y, f)) return ORDER_BUCKETS - 1;
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < N; ++i)
    if (i < n) {
      const double w = f[i] / (o.rtol * fabs(y[i]) + o.atol);
      s += w * w;
    }
  const double k = sqrt(s / n) * a.dt;
  if (!(k > 1.0)) return ORDER_BUCKETS - 2;  // less than one time scale (or not a number)
  const int lv = (int)(2.0f * log2f((float)fmin(k, 1e38)));
  return max(0, ORDER_BUCKETS - 3 - lv);
}

// Bucket of every cell (bkt[c]) and the bucket histogram (hist, zeroed first).
template <int N>
__global__ void __launch_bounds__(256) k_order_key(DNet net, Opts o, CellArgs a, uint8_t *bkt, uint32_t *hist) {
  __shared__ uint32_t h[ORDER_BUCKETS];
  for (int i = threadIdx.x; i < ORDER_BUCKETS; i += blockDim.x) h[i] = 0;
  __syncthreads();
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < a.n_cells;
       c += (int64_t)gridDim.x * blockDim.x) {
    const int b = cost_bucket<N>(net, o, a, c);
    bkt[c] = (uint8_t)b;
    atomicAdd(&h[b], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < ORDER_BUCKETS; i += blockDim.x)
    if (h[i]) atomicAdd(&hist[i], h[i]);
}

}  // namespace mc
