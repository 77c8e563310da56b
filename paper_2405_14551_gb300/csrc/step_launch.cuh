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

// 32-bit population offsets when every offset of a lattice of N nodes fits
inline bool fits_idx32(long long N) { return (unsigned long long)(2 * Q) * (unsigned long long)N < (1ull << 32); }

// Calls f with the staging halo (1, 4 or 7) as a compile-time constant.
template <typename F>
inline cudaError_t with_stage_halo(int halo, F&& f) {
  switch (halo) {
    case 1: return f(std::integral_constant<int, 1>{});
    case 4: return f(std::integral_constant<int, 4>{});
    case 7: return f(std::integral_constant<int, 7>{});
  }
  return cudaErrorInvalidValue;
}

template <int ST>
cudaError_t launch_phi_acc_t(const Geo& g, const StateBuf& in, unsigned long long* acc, cudaStream_t st) {
  const bool idx32 = fits_idx32(g.N);
  static const int occ32 = resident_ctas(k_phi_acc<ST, true>, 256, 0);
  static const int occ64 = resident_ctas(k_phi_acc<ST, false>, 256, 0);
  const long long need = (g.N + 255) / 256;
  const long long cap = (long long)sm_count() * (idx32 ? occ32 : occ64);
  const int blocks = (int)(need < cap ? need : cap);
  auto kern = idx32 ? k_phi_acc<ST, true> : k_phi_acc<ST, false>;
  trace_kernel("k_phi_acc", kern, dim3(blocks), dim3(256), 0);
  kern<<<blocks, 256, 0, st>>>(view<ST>(in), g, acc);
  return cudaGetLastError();
}

// IX: the offset width the kernel is built for (1: 32-bit, 0: 64-bit, -1:
// either, chosen by the lattice size).
template <int ST, int LOADER, bool WS, bool WF, int TX, int TY, int TZ, int H, int MINB = 2, bool INL = false,
          int IX = -1>
inline cudaError_t launch_step_t(const Geo& g, const Phys& p, const StateBuf& in, const InitBuf& init, PhiSrc src,
                                 AccBufs ab, StateBuf out, void* fields, unsigned* status, cudaStream_t st) {
  using R = typename Store<ST>::R;
  const size_t smem = Layout<R, TX, TY, TZ, H, 1, !INL>::bytes;
  const bool i32 = fits_idx32(g.N);
  using K = decltype(&k_step<ST, LOADER, WS, WF, TX, TY, TZ, H, true, MINB, INL>);
  K kern = nullptr;
  if constexpr (IX != 0) {
    if (i32) kern = k_step<ST, LOADER, WS, WF, TX, TY, TZ, H, true, MINB, INL>;
  }
  if constexpr (IX != 1) {
    if (!i32) kern = k_step<ST, LOADER, WS, WF, TX, TY, TZ, H, false, MINB, INL>;
  }
  if (!kern) return cudaErrorInvalidValue;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  dim3 grid((g.nx + TX - 1) / TX, (g.ny + TY - 1) / TY, (g.nz + TZ - 1) / TZ);
  dim3 block(TX, TY, 1);
  trace_kernel("k_step", kern, grid, block, smem);
  kern<<<grid, block, smem, st>>>(view<ST>(in), view<ST>(out), init, src, ab, g, p, reinterpret_cast<R*>(fields),
                                  status);
  return cudaGetLastError();
}

// Tile shapes of the hot variant (pull, write state): 0..5 as kTiles; the
// widest halo (7) only with tile 0.  Other variants, FP64 and lattices that
// need 64-bit offsets use tile 0.
template <int ST, int LOADER, bool WS, bool WF>
inline cudaError_t launch_step_tiles(int tile, const Geo& g, const Phys& p, const StateBuf& in, const InitBuf& init,
                                     PhiSrc src, AccBufs ab, StateBuf out, void* fields, unsigned* status,
                                     cudaStream_t st) {
  return with_stage_halo(stage_halo(p), [&](auto hc) -> cudaError_t {
    constexpr int H = decltype(hc)::value;
    if constexpr (LOADER == LOAD_PULL && WS && !WF && ST != 3 && H < 7) {
      if (fits_idx32(g.N)) {
        switch (tile) {
          case 1: return launch_step_t<ST, LOADER, WS, WF, 32, 8, 8, H, 2, false, 1>(g, p, in, init, src, ab, out, fields, status, st);
          case 2: return launch_step_t<ST, LOADER, WS, WF, 32, 8, 4, H, 3, false, 1>(g, p, in, init, src, ab, out, fields, status, st);
          case 3: return launch_step_t<ST, LOADER, WS, WF, 32, 8, 6, H, 3, false, 1>(g, p, in, init, src, ab, out, fields, status, st);
          case 4: return launch_step_t<ST, LOADER, WS, WF, 32, 4, 4, H, 6, false, 1>(g, p, in, init, src, ab, out, fields, status, st);
          case 5: return launch_step_t<ST, LOADER, WS, WF, 32, 8, 8, H, 2, true, 1>(g, p, in, init, src, ab, out, fields, status, st);
          default: break;
        }
      }
    }
    return launch_step_t<ST, LOADER, WS, WF, 32, 8, 4, H>(g, p, in, init, src, ab, out, fields, status, st);
  });
}

// Shan-Chen step (two-set storages; one tile shape, one-node halo)
template <int ST, int LOADER, bool WS, bool WF>
inline cudaError_t launch_step_sc(const Geo& g, const Phys& p, const StateBuf& in, const InitBuf& init, PhiSrc src,
                                  AccBufs ab, StateBuf out, void* fields, unsigned* status, cudaStream_t st) {
  if constexpr (!Store<ST>::TWOSET) {
    return cudaErrorInvalidValue;
  } else {
    using R = typename Store<ST>::R;
    constexpr int TX = 32, TY = 8, TZ = 4;
    const size_t smem = Layout<R, TX, TY, TZ, 1, 3>::bytes;
    auto kern = fits_idx32(g.N) ? k_step_sc<ST, LOADER, WS, WF, TX, TY, TZ, true>
                                : k_step_sc<ST, LOADER, WS, WF, TX, TY, TZ, false>;
    if (smem > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
    }
    dim3 grid((g.nx + TX - 1) / TX, (g.ny + TY - 1) / TY, (g.nz + TZ - 1) / TZ);
    trace_kernel("k_step_sc", kern, grid, dim3(TX, TY), smem);
    kern<<<grid, dim3(TX, TY), smem, st>>>(view<ST>(in), view<ST>(out), init, src, ab, g, p,
                                           reinterpret_cast<R*>(fields), status);
    return cudaGetLastError();
  }
}

template <int ST>
cudaError_t launch_step_s(int loader, bool ws, bool wf, int tile, const Geo& g, const Phys& p, const StateBuf& in,
                          const InitBuf& init, PhiSrc src, AccBufs ab, StateBuf out, void* fields, unsigned* status,
                          cudaStream_t st) {
  if (p.model == 1) {
    if (loader == LOAD_PULL) {
      if (ws && !wf) return launch_step_sc<ST, LOAD_PULL, true, false>(g, p, in, init, src, ab, out, fields, status, st);
      if (!ws && wf) return launch_step_sc<ST, LOAD_PULL, false, true>(g, p, in, init, src, ab, out, fields, status, st);
    } else {
      if (ws && !wf) return launch_step_sc<ST, LOAD_FIELDS, true, false>(g, p, in, init, src, ab, out, fields, status, st);
      if (!ws && wf) return launch_step_sc<ST, LOAD_FIELDS, false, true>(g, p, in, init, src, ab, out, fields, status, st);
    }
    return cudaErrorInvalidValue;
  }
  if (loader == LOAD_PULL) {
    if (ws && !wf) return launch_step_tiles<ST, LOAD_PULL, true, false>(tile, g, p, in, init, src, ab, out, fields, status, st);
    if (!ws && wf) return launch_step_tiles<ST, LOAD_PULL, false, true>(0, g, p, in, init, src, ab, out, fields, status, st);
  } else {
    if (ws && !wf) return launch_step_tiles<ST, LOAD_FIELDS, true, false>(0, g, p, in, init, src, ab, out, fields, status, st);
    if (!ws && wf) return launch_step_tiles<ST, LOAD_FIELDS, false, true>(0, g, p, in, init, src, ab, out, fields, status, st);
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

template <int ST, int TX, int TY, int TZ, int H, bool IDX32, int MINB = 2, bool INL = false>
inline cudaError_t launch_batched_step_t(const RunDesc* d_runs, int nruns, long long ntiles, int parity, int k,
                                         int blocks, unsigned* status, cudaStream_t st) {
  using R = typename Store<ST>::R;
  const size_t smem = Layout<R, TX, TY, TZ, H, 1, !INL>::bytes;
  auto kern = k_step_batched<ST, TX, TY, TZ, H, IDX32, MINB, INL>;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  trace_kernel("k_step_batched", kern, dim3(blocks), dim3(TX, TY), smem);
  kern<<<blocks, dim3(TX, TY), smem, st>>>(d_runs, nruns, ntiles, parity, k, status);
  return cudaGetLastError();
}

template <int ST, bool IDX32>
inline cudaError_t launch_batched_tiles(int tile, int halo, const RunDesc* d_runs, int nruns, long long ntiles,
                                        int parity, int k, int blocks, unsigned* status, cudaStream_t st) {
  return with_stage_halo(halo, [&](auto hc) -> cudaError_t {
    constexpr int H = decltype(hc)::value;
    if constexpr (H < 7 && IDX32) {  // 64-bit offsets: tile 0
      switch (tile) {
        case 1: return launch_batched_step_t<ST, 32, 8, 8, H, IDX32>(d_runs, nruns, ntiles, parity, k, blocks, status, st);
        case 2: return launch_batched_step_t<ST, 32, 8, 4, H, IDX32, 3>(d_runs, nruns, ntiles, parity, k, blocks, status, st);
        case 3: return launch_batched_step_t<ST, 32, 8, 6, H, IDX32, 3>(d_runs, nruns, ntiles, parity, k, blocks, status, st);
        case 4: return launch_batched_step_t<ST, 32, 4, 4, H, IDX32, 6>(d_runs, nruns, ntiles, parity, k, blocks, status, st);
        case 5: return launch_batched_step_t<ST, 32, 8, 8, H, IDX32, 2, true>(d_runs, nruns, ntiles, parity, k, blocks, status, st);
        default: break;
      }
    }
    return launch_batched_step_t<ST, 32, 8, 4, H, IDX32>(d_runs, nruns, ntiles, parity, k, blocks, status, st);
  });
}

template <int ST>
cudaError_t launch_batched_t(const RunDesc* d_runs, int nruns, long long ntiles, int tile, int halo,
                             long long max_nodes, int parity, int k, int blocks_per_sm, unsigned* status,
                             cudaStream_t st) {
  const int blocks = sm_count() * (blocks_per_sm > 0 ? blocks_per_sm : 2);
  if (fits_idx32(max_nodes))
    return launch_batched_tiles<ST, true>(tile, halo, d_runs, nruns, ntiles, parity, k, blocks, status, st);
  return launch_batched_tiles<ST, false>(tile, halo, d_runs, nruns, ntiles, parity, k, blocks, status, st);
}

}  // namespace lbcg
