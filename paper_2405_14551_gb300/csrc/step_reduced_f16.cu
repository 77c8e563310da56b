// Step kernels instantiated for storage 2 (reduced single set, FP16 deviations).
#include "step_launch.cuh"

namespace lbcg {

template cudaError_t launch_phi_t<2>(const Geo&, const StateBuf&, void*, cudaStream_t);
template cudaError_t launch_nc_t<2>(int, const Geo&, const Phys&, const void*, unsigned char*, cudaStream_t);
template cudaError_t launch_step_s<2>(int, bool, bool, int, const Geo&, const Phys&, const StateBuf&, const InitBuf&,
                                         const void*, const unsigned char*, StateBuf, void*, unsigned*, cudaStream_t);
template cudaError_t launch_export_t<2>(int, const Geo&, const Phys&, const StateBuf&, const InitBuf&, int, int, int,
                                          int, int, int, double*, double*, cudaStream_t);

template cudaError_t launch_batched_t<2>(const RunDesc*, int, long long, long long, int, int, long long, int, int,
                                           unsigned*, cudaStream_t);

}  // namespace lbcg
