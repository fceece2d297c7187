// mc_autotune.cu -- launch-shape selection (variant, threads per block,
// persistent blocks per SM) per network size and matrix precision.
#include <mutex>

#include "mc_internal.h"

using namespace mc;

Tuned mc::autotune_pick(const mc_network *net, const mc_burn_opts &o) {
  (void)net;
  Tuned t;
  t.variant = o.variant == MC_VARIANT_AUTO ? MC_VARIANT_PERSISTENT : o.variant;
  t.threads = o.block_threads ? o.block_threads : 128;
  t.blocks_per_sm = o.blocks_per_sm ? o.blocks_per_sm : 2;
  return t;
}
