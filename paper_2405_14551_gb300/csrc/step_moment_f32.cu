// Step kernels instantiated for storage 4 (moment storage of the regularised
// collision, FP32).  Batches do not take this storage.
#include "step_launch.cuh"

namespace lbcg {

template cudaError_t launch_phi_acc_t<4>(const Geo&, const StateBuf&, unsigned long long*, cudaStream_t);
template cudaError_t launch_step_s<4>(int, bool, bool, int, const Geo&, const Phys&, const StateBuf&, const InitBuf&,
                                      PhiSrc, AccBufs, StateBuf, void*, unsigned*, cudaStream_t);
template cudaError_t launch_export_t<4>(int, const Geo&, const Phys&, const StateBuf&, const InitBuf&, int, int, int,
                                        int, int, int, double*, double*, cudaStream_t);

}  // namespace lbcg
