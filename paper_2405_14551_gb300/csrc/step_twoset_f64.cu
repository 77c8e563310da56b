// Step kernels instantiated for storage 3 (two population sets, FP64).
#include "step_launch.cuh"

namespace lbcg {

template cudaError_t launch_phi_acc_t<3>(const Geo&, const StateBuf&, unsigned long long*, cudaStream_t);
template cudaError_t launch_step_s<3>(int, bool, bool, int, const Geo&, const Phys&, const StateBuf&, const InitBuf&,
                                      PhiSrc, AccBufs, StateBuf, void*, unsigned*, cudaStream_t);
template cudaError_t launch_export_t<3>(int, const Geo&, const Phys&, const StateBuf&, const InitBuf&, int, int, int,
                                        int, int, int, double*, double*, cudaStream_t);

}  // namespace lbcg
