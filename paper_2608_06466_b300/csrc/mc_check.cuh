// mc_check.cuh -- the bounds-check build (the same sources compiled with
// -DMC_BOUNDS_CHECK into libmc_check.so).
//
// Every cell index, list position and record index a burn kernel computes is
// tested before the access it guards. A refused access is counted, the first
// one is recorded (site, index, bound) and the access is skipped, so a kernel
// with an index error returns with the evidence instead of faulting. Each
// cell's final store is counted as well, so that the host can check after a
// call that the queue handed out every cell once and that hand-off, retry
// lists and ladder rungs neither lost nor duplicated one: every cell of the
// call written exactly once. In the normal build the checks compile to
// nothing.
#pragma once

#include <cstdint>

namespace mc {

enum BoundsSite : int {
  BC_NONE = 0,
  BC_CELL_LOAD = 1,   // cell index read by a thread-per-cell load
  BC_CELL_STORE = 2,  // cell index of a final store
  BC_LIST_READ = 3,   // position in a cell list (cost order, retry list)
  BC_LIST_PUSH = 4,   // position of a push onto a retry or ladder list
  BC_RECORD = 5,      // straggler record index
  BC_WARP_LOAD = 6,   // cell index read by a warp-per-cell load
  BC_RKC_CELL = 7,    // cell index of the RKC kernel
};

// Device record of one GPU (the check build keeps one per device).
struct BoundsCheck {
  unsigned int refused;     // accesses refused since the last reset
  int site;                 // first refused access: its site,
  long long index;          // index
  long long bound;          // and bound
  unsigned int *stores;     // per cell of the call being verified: final stores (nullptr: none)
  long long cells;          // entries of stores
  long long calls;          // calls verified
  long long cells_checked;  // cells over those calls
  long long not_once;       // cells of those calls not stored exactly once
};

#ifdef MC_BOUNDS_CHECK
__device__ __forceinline__ bool bc_in(BoundsCheck *bc, int site, long long i, long long n) {
  if (i >= 0 && i < n) return true;
  if (bc && atomicAdd(&bc->refused, 1u) == 0u) {
    bc->site = site;
    bc->index = i;
    bc->bound = n;
  }
  return false;
}
// cells a launch may index: the call's cell count (lists hold at most as many)
#define MC_CELLS(a) ((a).cells > 0 ? (a).cells : (a).n_cells)
#define MC_IN(a, site, i, n) ::mc::bc_in((a).bc, (site), (long long)(i), (long long)(n))
#define MC_STORED(a, c)                                                            \
  do {                                                                             \
    ::mc::BoundsCheck *bc_ = (a).bc;                                               \
    if (bc_ && bc_->stores && ::mc::bc_in(bc_, ::mc::BC_CELL_STORE, (long long)(c), bc_->cells)) \
      atomicAdd(&bc_->stores[(c)], 1u);                                            \
  } while (0)
#else
#define MC_IN(a, site, i, n) true
#define MC_STORED(a, c) \
  do {                  \
  } while (0)
#endif

}  // namespace mc
