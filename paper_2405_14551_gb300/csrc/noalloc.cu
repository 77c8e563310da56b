// Allocation-free variant of the FP64 field reduction.
//
// lb_reduce_f64 keeps its block partial sums in device memory that the handle
// allocated.  Some callers cannot allocate device memory when they need the
// sums: programs that hand out all device memory themselves up front and
// forbid allocations afterwards, or code paths where the implicit
// synchronisation of cudaMalloc/cudaFree is not acceptable.  For them,
// lb_reduce_fields_f64_static reduces a caller-provided fields array into a
// caller-provided output and keeps its partial sums in the file-scope device
// array below, which every GPU that loads this library holds until the
// process exits.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/lbcg.h"
#include "internal.h"

namespace {

// One partial sum of 8 doubles per reduction block; the reduction never uses
// more than LB_STATIC_REDUCE_MAX_BLOCKS blocks, so 64 KiB cover every grid
// the library accepts (up to 2^31 - 1 nodes).
constexpr int kPartialDoubles = LB_STATIC_REDUCE_MAX_BLOCKS * 8;
static __device__ __align__(256) double g_static_partials[kPartialDoubles];

constexpr int kMaxDevices = 64;
double* g_partials_ptr[kMaxDevices] = {};
std::mutex g_setup_mutex;

// Device address of the partials array on the current device.  Host code only
// sees a host-side stand-in under the array's name, so the address comes from
// cudaGetSymbolAddress, once per device, with that device current.  The
// cached address belongs to the device's primary context: after a
// cudaDeviceReset of that device it no longer refers to the array (see the
// declaration in lbcg.h).
int partials_for_current_device(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return lbcg::report_error(LB_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return lbcg::report_error(LB_EINVAL, "device ordinal above 63");
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_partials_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_partials);
    if (e != cudaSuccess || !p)
      return lbcg::report_error(LB_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_partials_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_partials_ptr[dev];
  return LB_OK;
}

}  // namespace

extern "C" int lb_reduce_fields_f64_static(const void* fields, int fields_are_f64, int32_t nx, int32_t ny,
                                           int32_t nz, uint32_t walls, double* out, void* stream) {
  if (!fields || !out) return lbcg::report_error(LB_EINVAL, "fields and out must be device pointers");
  if (nx < 1 || ny < 1 || nz < 1) return lbcg::report_error(LB_EINVAL, "grid extents must be >= 1");
  if (walls & ~7u) return lbcg::report_error(LB_EINVAL, "walls uses bits 0..2 only");
  const long long N = (long long)nx * ny * nz;
  if (N > 0x7fffffffLL) return lbcg::report_error(LB_EINVAL, "grid has more than 2^31-1 nodes");
  // defensive: reduce_blocks never exceeds RED_MAX_BLOCKS, which a
  // static_assert in aux_kernels.cu keeps within the static array
  if (lbcg::reduce_blocks(N) > LB_STATIC_REDUCE_MAX_BLOCKS)
    return lbcg::report_error(LB_EINVAL, "grid needs more partial sums than the static scratch holds");
  double* partials = nullptr;
  int rc = partials_for_current_device(&partials);
  if (rc) return rc;
  lbcg::Geo g;
  g.nx = nx;
  g.ny = ny;
  g.nz = nz;
  g.wx = (walls >> 0) & 1u;
  g.wy = (walls >> 1) & 1u;
  g.wz = (walls >> 2) & 1u;
  g.N = N;
  // every block overwrites its own partials and the final block writes all of
  // out, so nothing has to be cleared between calls
  cudaError_t e = lbcg::launch_reduce(fields_are_f64 ? LB_STORAGE_TWOSET_F64 : LB_STORAGE_TWOSET_F32, g, fields,
                                      partials, out, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return lbcg::report_error(LB_ECUDA, std::string("static reduction: ") + cudaGetErrorString(e));
  lbcg::count_launches(2);
  return LB_OK;
}
