// Storage-format dispatch of the step launchers.
#include "internal.h"
#include "lattice.cuh"

namespace lbcg {

// tile 2: the 32x8x4 tile with registers capped for 3 CTAs per SM; tile 3: a
// 32x8x6 tile capped for 3 CTAs per SM; tile 4: 32x4x4 (128 threads) capped
// for 6 CTAs per SM; tile 5: 32x8x8 with the near-contact scan inside the
// node loop
const Tile kTiles[NUM_TILES] = {{32, 8, 4}, {32, 8, 8}, {32, 8, 4}, {32, 8, 6}, {32, 4, 4}, {32, 8, 8}};

template <int ST>
cudaError_t launch_phi_acc_t(const Geo& g, const StateBuf& in, unsigned long long* acc, cudaStream_t st);
template <int ST>
cudaError_t launch_step_s(int loader, bool ws, bool wf, int tile, const Geo& g, const Phys& p, const StateBuf& in,
                          const InitBuf& init, PhiSrc src, AccBufs ab, StateBuf out, void* fields, unsigned* status,
                          cudaStream_t st);
template <int ST>
cudaError_t launch_batched_t(const RunDesc* d_runs, int nruns, long long ntiles, int tile, int halo,
                             long long max_nodes, int parity, int k, int blocks_per_sm, unsigned* status,
                             cudaStream_t st);
template <int ST>
cudaError_t launch_export_t(int loader, const Geo& g, const Phys& p, const StateBuf& in, const InitBuf& init, int x0,
                            int y0, int z0, int bx, int by, int bz, double* outA, double* outB, cudaStream_t st);

cudaError_t launch_phi_acc(int storage, const Geo& g, const StateBuf& in, unsigned long long* acc, cudaStream_t st) {
  switch (storage) {
    case 0: return launch_phi_acc_t<0>(g, in, acc, st);
    case 1: return launch_phi_acc_t<1>(g, in, acc, st);
    case 2: return launch_phi_acc_t<2>(g, in, acc, st);
    case 3: return launch_phi_acc_t<3>(g, in, acc, st);
    case 4: return launch_phi_acc_t<4>(g, in, acc, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_step(int storage, int loader, bool write_state, bool write_fields, int tile, const Geo& g,
                        const Phys& p, const StateBuf& in, const InitBuf& init, PhiSrc src, AccBufs ab, StateBuf out,
                        void* fields, unsigned* status, cudaStream_t st) {
  switch (storage) {
    case 0: return launch_step_s<0>(loader, write_state, write_fields, tile, g, p, in, init, src, ab, out, fields, status, st);
    case 1: return launch_step_s<1>(loader, write_state, write_fields, tile, g, p, in, init, src, ab, out, fields, status, st);
    case 2: return launch_step_s<2>(loader, write_state, write_fields, tile, g, p, in, init, src, ab, out, fields, status, st);
    case 3: return launch_step_s<3>(loader, write_state, write_fields, tile, g, p, in, init, src, ab, out, fields, status, st);
    case 4: return launch_step_s<4>(loader, write_state, write_fields, tile, g, p, in, init, src, ab, out, fields, status, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_export(int storage, int loader, const Geo& g, const Phys& p, const StateBuf& in,
                          const InitBuf& init, int x0, int y0, int z0, int bx, int by, int bz, double* outA,
                          double* outB, cudaStream_t st) {
  switch (storage) {
    case 0: return launch_export_t<0>(loader, g, p, in, init, x0, y0, z0, bx, by, bz, outA, outB, st);
    case 1: return launch_export_t<1>(loader, g, p, in, init, x0, y0, z0, bx, by, bz, outA, outB, st);
    case 2: return launch_export_t<2>(loader, g, p, in, init, x0, y0, z0, bx, by, bz, outA, outB, st);
    case 3: return launch_export_t<3>(loader, g, p, in, init, x0, y0, z0, bx, by, bz, outA, outB, st);
    case 4: return launch_export_t<4>(loader, g, p, in, init, x0, y0, z0, bx, by, bz, outA, outB, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_batched(int storage, const RunDesc* d_runs, int nruns, long long ntiles, int tile, int halo,
                           long long max_nodes, int parity, int k, int blocks_per_sm, unsigned* status,
                           cudaStream_t st) {
  switch (storage) {
    case 0: return launch_batched_t<0>(d_runs, nruns, ntiles, tile, halo, max_nodes, parity, k, blocks_per_sm, status, st);
    case 1: return launch_batched_t<1>(d_runs, nruns, ntiles, tile, halo, max_nodes, parity, k, blocks_per_sm, status, st);
    case 2: return launch_batched_t<2>(d_runs, nruns, ntiles, tile, halo, max_nodes, parity, k, blocks_per_sm, status, st);
  }
  return cudaErrorInvalidValue;  // no batched FP64 or moment instantiation
}

int sm_count_host() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

size_t elem_bytes(int storage) { return storage == 3 ? 8 : (storage == 2 ? 2 : 4); }
int state_arrays(int storage) { return storage == 4 ? MOMENT_COEFS : (storage == 0 || storage == 3 ? 2 * Q : Q); }
bool storage_is_twoset(int storage) { return storage == 0 || storage == 3; }
bool storage_is_f64(int storage) { return storage == 3; }

}  // namespace lbcg
