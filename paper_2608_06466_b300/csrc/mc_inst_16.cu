// mc_inst_16.cu -- burn kernels for networks of up to 16 ODEs.
#include "mc_launch.cuh"

namespace mc {
template mc_status launch_one<16, double>(const DNet &, const Opts &, const CellArgs &, int, int, int, int,
                                          unsigned long long *, cudaStream_t);
template mc_status launch_one<16, float>(const DNet &, const Opts &, const CellArgs &, int, int, int, int,
                                         unsigned long long *, cudaStream_t);
}  // namespace mc
