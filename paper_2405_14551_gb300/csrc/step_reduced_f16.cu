// Step kernels instantiated for storage 2 (reduced single set, FP16 deviations).
#include "step_launch.cuh"

namespace lbcg {

template cudaError_t launch_phi_acc_t<2>(const Geo&, const StateBuf&, unsigned long long*, cudaStream_t);
template cudaError_t launch_step_s<2>(int, bool, bool, int, const Geo&, const Phys&, const StateBuf&, const InitBuf&,
                                      PhiSrc, AccBufs, StateBuf, void*, unsigned*, cudaStream_t);
template cudaError_t launch_export_t<2>(int, const Geo&, const Phys&, const StateBuf&, const InitBuf&, int, int, int,
                                        int, int, int, double*, double*, cudaStream_t);

template cudaError_t launch_batched_t<2>(const RunDesc*, int, long long, int, int, long long, int, int, int,
                                         unsigned*, cudaStream_t);

}  // namespace lbcg
