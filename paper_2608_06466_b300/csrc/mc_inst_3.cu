// mc_inst_3.cu -- burn kernels for networks of up to 3 ODEs.
#include "mc_launch.cuh"

namespace mc {
template mc_status launch_one<3, double>(const DNet &, const Opts &, const CellArgs &, int, int, int, int,
                                          unsigned long long *, cudaStream_t);
template mc_status launch_one<3, float>(const DNet &, const Opts &, const CellArgs &, int, int, int, int,
                                         unsigned long long *, cudaStream_t);
}  // namespace mc
