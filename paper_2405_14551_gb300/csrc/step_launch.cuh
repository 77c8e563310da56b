// Launchers of the step kernels, instantiated once per storage format.
#pragma once
#include "step_impl.cuh"

namespace lbcg {

inline int sm_count() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

// CTAs of a kernel that fit on one SM at once (computed once per kernel).
template <typename K>
inline int resident_ctas(K kern, int threads, size_t smem) {
  int b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, threads, smem) != cudaSuccess || b < 1) {
    cudaGetLastError();
    b = 1;
  }
  return b;
}

template <int ST>
cudaError_t launch_phi_t(const Geo& g, const StateBuf& in, void* phi, cudaStream_t st) {
  using R = typename Store<ST>::R;
  if constexpr (!Store<ST>::TWOSET) {  // reduced storage: tiles with staged colour scalars
    constexpr int TX = 32, TY = 8, TZ = 4;
    const bool idx32r = (unsigned long long)(2 * Q) * (unsigned long long)g.N < (1ull << 32);
    const size_t smem = sizeof(float4) * (TX + 2) * (TY + 2) * (TZ + 2);
    const dim3 grid((g.nx + TX - 1) / TX, (g.ny + TY - 1) / TY, (g.nz + TZ - 1) / TZ);
    auto kern = idx32r ? k_phi_tiled<ST, TX, TY, TZ, true> : k_phi_tiled<ST, TX, TY, TZ, false>;
    trace_kernel("k_phi_tiled", kern, grid, dim3(TX, TY), smem);
    kern<<<grid, dim3(TX, TY), smem, st>>>(view<ST>(in), g, reinterpret_cast<R*>(phi));
    return cudaGetLastError();
  }
  static const int occ32 = resident_ctas(k_phi<ST, true>, 256, 0);
  static const int occ64 = resident_ctas(k_phi<ST, false>, 256, 0);
  const bool idx32 = (unsigned long long)(2 * Q) * (unsigned long long)g.N < (1ull << 32);
  // one wave of resident CTAs striding over the lattice: no second, partial wave
  const long long blocks_needed = (g.N + 255) / 256;
  const long long cap = (long long)sm_count() * (idx32 ? occ32 : occ64);
  const int blocks = (int)(blocks_needed < cap ? blocks_needed : cap);
  auto kern = idx32 ? k_phi<ST, true> : k_phi<ST, false>;
  trace_kernel("k_phi", kern, dim3(blocks), dim3(256), 0);
  kern<<<blocks, 256, 0, st>>>(view<ST>(in), g, reinterpret_cast<R*>(phi));
  return cudaGetLastError();
}

template <int ST, int TX, int TY, int TZ>
inline cudaError_t launch_nc_tt(const Geo& g, const Phys& p, const void* phi, unsigned char* hnc, cudaStream_t st) {
  using R = typename Store<ST>::R;
  if (p.halo != p.K + 1 || p.halo < 2 || p.halo > 7) return cudaErrorInvalidValue;
  const size_t smem = nc_smem_bytes<R>(TX, TY, TZ, p.halo);
  const dim3 grid((g.nx + TX - 1) / TX, (g.ny + TY - 1) / TY, (g.nz + TZ - 1) / TZ);
  cudaError_t e = cudaSuccess;
  with_halo(p.halo, [&](auto hc) {
    auto kern = k_nc<ST, TX, TY, TZ, decltype(hc)::value>;
    if (smem > 48 * 1024) e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return;
    trace_kernel("k_nc", kern, grid, dim3(TX, TY), smem);
    kern<<<grid, dim3(TX, TY), smem, st>>>(reinterpret_cast<const R*>(phi), g, p, hnc);
    e = cudaGetLastError();
  });
  return e;
}

// Near-contact tile shapes (x, y threads, z nodes per thread): 32x8x8,
// 32x8x4, 32x8x16, 32x4x16.  FP64 storage (parity runs) uses 32x8x4 only.
template <int ST>
cudaError_t launch_nc_t(int variant, const Geo& g, const Phys& p, const void* phi, unsigned char* hnc,
                        cudaStream_t st) {
  if (p.A_h == 0.0) return cudaSuccess;
  if constexpr (ST == 3) {
    return launch_nc_tt<ST, 32, 8, 4>(g, p, phi, hnc, st);
  } else {
    switch (variant) {
      case 1: return launch_nc_tt<ST, 32, 8, 4>(g, p, phi, hnc, st);
      case 2: return launch_nc_tt<ST, 32, 8, 16>(g, p, phi, hnc, st);
      case 3: return launch_nc_tt<ST, 32, 4, 16>(g, p, phi, hnc, st);
      default: return launch_nc_tt<ST, 32, 8, 8>(g, p, phi, hnc, st);
    }
  }
}

template <int ST, int LOADER, bool WS, bool WF, int TX, int TY, int TZ, int MINB = 2>
inline cudaError_t launch_step_t(const Geo& g, const Phys& p, const StateBuf& in, const InitBuf& init,
                                 const void* phi, const unsigned char* hnc, StateBuf out, void* fields,
                                 unsigned* status, cudaStream_t st) {
  using R = typename Store<ST>::R;
  const size_t smem = step_smem_bytes<R>(TX, TY, TZ);
  // 32-bit population offsets when every offset of the lattice fits
  const bool idx32 = (unsigned long long)(2 * Q) * (unsigned long long)g.N < (1ull << 32);
  auto kern = idx32 ? k_step<ST, LOADER, WS, WF, TX, TY, TZ, true, MINB> : k_step<ST, LOADER, WS, WF, TX, TY, TZ, false, MINB>;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  dim3 grid((g.nx + TX - 1) / TX, (g.ny + TY - 1) / TY, (g.nz + TZ - 1) / TZ);
  dim3 block(TX, TY, 1);
  trace_kernel("k_step", kern, grid, block, smem);
  kern<<<grid, block, smem, st>>>(view<ST>(in), view<ST>(out), init, reinterpret_cast<const R*>(phi), hnc, g, p,
                                  reinterpret_cast<R*>(fields), status);
  return cudaGetLastError();
}

template <int ST, int LOADER, bool WS, bool WF>
inline cudaError_t launch_step_tiles(int tile, const Geo& g, const Phys& p, const StateBuf& in, const InitBuf& init,
                                     const void* phi, const unsigned char* hnc, StateBuf out, void* fields,
                                     unsigned* status, cudaStream_t st) {
  if constexpr (LOADER == LOAD_PULL && WS && !WF) {
    switch (tile) {
      case 1: return launch_step_t<ST, LOADER, WS, WF, 32, 8, 8>(g, p, in, init, phi, hnc, out, fields, status, st);
      case 2: return launch_step_t<ST, LOADER, WS, WF, 32, 8, 4, 3>(g, p, in, init, phi, hnc, out, fields, status, st);
      case 3: return launch_step_t<ST, LOADER, WS, WF, 64, 4, 4>(g, p, in, init, phi, hnc, out, fields, status, st);
      case 4: return launch_step_t<ST, LOADER, WS, WF, 32, 8, 4, 4>(g, p, in, init, phi, hnc, out, fields, status, st);
      default: break;
    }
  }
  return launch_step_t<ST, LOADER, WS, WF, 32, 8, 4>(g, p, in, init, phi, hnc, out, fields, status, st);
}

template <int ST>
cudaError_t launch_step_s(int loader, bool ws, bool wf, int tile, const Geo& g, const Phys& p, const StateBuf& in,
                          const InitBuf& init, const void* phi, const unsigned char* hnc, StateBuf out, void* fields,
                          unsigned* status, cudaStream_t st) {
  if (loader == LOAD_PULL) {
    if (ws && !wf) return launch_step_tiles<ST, LOAD_PULL, true, false>(tile, g, p, in, init, phi, hnc, out, fields, status, st);
    if (ws && wf) return launch_step_tiles<ST, LOAD_PULL, true, true>(0, g, p, in, init, phi, hnc, out, fields, status, st);
    if (!ws && wf) return launch_step_tiles<ST, LOAD_PULL, false, true>(0, g, p, in, init, phi, hnc, out, fields, status, st);
  } else {
    if (ws && !wf) return launch_step_tiles<ST, LOAD_FIELDS, true, false>(0, g, p, in, init, phi, hnc, out, fields, status, st);
    if (ws && wf) return launch_step_tiles<ST, LOAD_FIELDS, true, true>(0, g, p, in, init, phi, hnc, out, fields, status, st);
    if (!ws && wf) return launch_step_tiles<ST, LOAD_FIELDS, false, true>(0, g, p, in, init, phi, hnc, out, fields, status, st);
  }
  return cudaErrorInvalidValue;
}

template <int ST>
cudaError_t launch_export_t(int loader, const Geo& g, const Phys& p, const StateBuf& in, const InitBuf& init,
                                   int x0, int y0, int z0, int bx, int by, int bz, double* outA, double* outB,
                                   cudaStream_t st) {
  const long long M = (long long)bx * by * bz;
  const long long need = (M + 127) / 128;
  const int blocks = (int)(need < 4096 ? need : 4096);
  if (loader == LOAD_PULL)
    k_export<ST, LOAD_PULL><<<blocks, 128, 0, st>>>(view<ST>(in), init, g, p, x0, y0, z0, bx, by, bz, outA, outB);
  else
    k_export<ST, LOAD_FIELDS><<<blocks, 128, 0, st>>>(view<ST>(in), init, g, p, x0, y0, z0, bx, by, bz, outA, outB);
  return cudaGetLastError();
}

template <int ST, int TX, int TY, int TZ, bool IDX32, int MINB = 2>
inline cudaError_t launch_batched_step_t(const RunDesc* d_runs, int nruns, long long ntiles, int halo_max,
                                         int parity, int blocks, unsigned* status, cudaStream_t st) {
  using R = typename Store<ST>::R;
  if (halo_max > 1) {  // some run has near contact
    const size_t nsmem = nc_smem_bytes<R>(TX, TY, TZ, halo_max);
    auto nk = k_nc_batched<ST, TX, TY, TZ>;
    if (nsmem > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(nk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)nsmem);
      if (e != cudaSuccess) return e;
    }
    trace_kernel("k_nc_batched", nk, dim3(blocks), dim3(TX, TY), nsmem);
    nk<<<blocks, dim3(TX, TY), nsmem, st>>>(d_runs, nruns, ntiles);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  const size_t smem = step_smem_bytes<R>(TX, TY, TZ);
  auto kern = k_step_batched<ST, TX, TY, TZ, IDX32, MINB>;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  trace_kernel("k_step_batched", kern, dim3(blocks), dim3(TX, TY), smem);
  kern<<<blocks, dim3(TX, TY), smem, st>>>(d_runs, nruns, ntiles, parity, status);
  return cudaGetLastError();
}

template <int ST, bool IDX32>
inline cudaError_t launch_batched_tiles(int tile, const RunDesc* d_runs, int nruns, long long ntiles, int halo_max,
                                        int parity, int blocks, unsigned* status, cudaStream_t st) {
  switch (tile) {
    case 1: return launch_batched_step_t<ST, 32, 8, 8, IDX32>(d_runs, nruns, ntiles, halo_max, parity, blocks, status, st);
    case 2: return launch_batched_step_t<ST, 32, 8, 4, IDX32, 3>(d_runs, nruns, ntiles, halo_max, parity, blocks, status, st);
    case 3: return launch_batched_step_t<ST, 64, 4, 4, IDX32>(d_runs, nruns, ntiles, halo_max, parity, blocks, status, st);
    case 4: return launch_batched_step_t<ST, 32, 8, 4, IDX32, 4>(d_runs, nruns, ntiles, halo_max, parity, blocks, status, st);
    default: return launch_batched_step_t<ST, 32, 8, 4, IDX32>(d_runs, nruns, ntiles, halo_max, parity, blocks, status, st);
  }
}

template <int ST>
cudaError_t launch_batched_t(const RunDesc* d_runs, int nruns, long long nchunks, long long ntiles, int tile,
                             int halo_max, long long max_nodes, int parity, int blocks_per_sm, unsigned* status,
                             cudaStream_t st) {
  const int blocks = sm_count() * (blocks_per_sm > 0 ? blocks_per_sm : 2);
  const bool idx32 = (unsigned long long)(2 * Q) * (unsigned long long)max_nodes < (1ull << 32);
  auto pk = idx32 ? k_phi_batched<ST, true> : k_phi_batched<ST, false>;
  static const int pocc32 = resident_ctas(k_phi_batched<ST, true>, 256, 0);
  static const int pocc64 = resident_ctas(k_phi_batched<ST, false>, 256, 0);
  const int pblocks = sm_count() * (idx32 ? pocc32 : pocc64);
  trace_kernel("k_phi_batched", pk, dim3(pblocks), dim3(256), 0);
  pk<<<pblocks, 256, 0, st>>>(d_runs, nruns, nchunks, parity);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (idx32) return launch_batched_tiles<ST, true>(tile, d_runs, nruns, ntiles, halo_max, parity, blocks, status, st);
  return launch_batched_tiles<ST, false>(tile, d_runs, nruns, ntiles, halo_max, parity, blocks, status, st);
}

}  // namespace lbcg
