// Internal interface between the C-ABI runtime and the kernel translation units.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <string>

namespace lbcg {

// Box geometry; w* = 1 makes layers 0 and n-1 of that axis solid.
struct Geo {
  int nx, ny, nz;
  int wx, wy, wz;
  long long N;
};

// Model parameters as seen by the kernels (converted to the compute type in
// the kernel prologue).
struct Phys {
  double tau_a, tau_b;
  int equal_tau;
  double A2;  // (A_a + A_b) / 2
  double beta;
  double A_h, h_min, h_max;
  int K;      // floor(h_max): scan length
  double phi_I;
  double g[3];
  int g_mode;
  int collision;  // 0 BGK, 1 regularised
  int model;      // 0 colour gradient, 1 Shan-Chen
  double G;       // Shan-Chen coupling
  double psi0;    // Shan-Chen pseudo-potential scale rho_0
};

// Device pointers of one population lattice.  Two-set storage: f holds
// f^A [27][N] followed by f^B [27][N].  Reduced storage: f holds f* [27][N]
// (FP32 or FP16 deviations) and sv holds the colour scalars (s, vx, vy, vz)
// of each node as one float4.
struct StateBuf {
  void* f;
  float4* sv;
};

// Initial fields (device, float): phi[N], rho[N] or null, u[3][N] or null.
struct InitBuf {
  const float* phi;
  const float* rho;
  const float* u;
  int regularised;
};

enum Loader { LOAD_PULL = 0, LOAD_FIELDS = 1 };

// Where a step reads phi(t): the accumulator of the previous step, or a
// plain array of the compute type (the initial fields' phi).  Exactly one is
// non-null.
struct PhiSrc {
  const void* phi;
  const unsigned long long* acc;
};

// Accumulators written by a step: out receives the component densities of
// the next time level (all zero before the step); the step zeroes its own
// nodes of zero (read by the step before, written by the step after).
struct AccBufs {
  unsigned long long* out;
  unsigned long long* zero;
};

// 64-bit words of one node's accumulator: 1 (FP32 storages, both component
// sums packed), 2 (FP64).
inline int acc_words(int storage) { return storage == 3 ? 2 : 1; }

// One run of a batch, as seen by the batched persistent kernel.
struct RunDesc {
  Geo g;
  Phys p;
  StateBuf S[2];
  unsigned long long* acc[3];  // accumulator rotation (see AccBufs)
  int tiles_x, tiles_y, tiles_z;
  long long tile_begin;  // first work item of this run
};

// Tile shapes of the fused step kernel (x, y extent of the thread block and z
// nodes per thread).  Tile 5 scans near contact inside the node loop.
struct Tile {
  int tx, ty, tz;
};
constexpr int NUM_TILES = 6;
extern const Tile kTiles[NUM_TILES];

size_t elem_bytes(int storage);
// population-like arrays of a state: 2 x 27 (two sets), 27 (single set) or
// the 10 quadratic-form coefficients of the moment storage
int state_arrays(int storage);
bool storage_is_twoset(int storage);
bool storage_is_f64(int storage);

// --- step_kernels.cu -------------------------------------------------------
// halo of the phi tile a step stages: 1 without near contact, else 4 (scan
// length K <= 3) or 7 (K <= 6)
inline int stage_halo(const Phys& p) { return p.A_h == 0.0 ? 1 : (p.K <= 3 ? 4 : 7); }
// rebuild the accumulator of the current time level from the populations of in
cudaError_t launch_phi_acc(int storage, const Geo& g, const StateBuf& in, unsigned long long* acc, cudaStream_t st);
// one step (write_state) and/or the fields of the current level (write_fields);
// tile indexes kTiles (only tile 0 for the variants that are not hot)
cudaError_t launch_step(int storage, int loader, bool write_state, bool write_fields, int tile, const Geo& g,
                        const Phys& p, const StateBuf& in, const InitBuf& init, PhiSrc src, AccBufs ab, StateBuf out,
                        void* fields, unsigned* status, cudaStream_t st);
// export pre-collision populations of a box, canonical order, as double
cudaError_t launch_export(int storage, int loader, const Geo& g, const Phys& p, const StateBuf& in,
                          const InitBuf& init, int x0, int y0, int z0, int bx, int by, int bz, double* outA,
                          double* outB, cudaStream_t st);

// batched step over runs[0..nruns): one persistent launch of blocks_per_sm x
// SMs CTAs; parity selects S[parity] as input, k the accumulator phase
// (runs read acc[k], add into acc[(k+1)%3], clear acc[(k+2)%3]); halo is the
// largest stage_halo of the runs
cudaError_t launch_batched(int storage, const RunDesc* d_runs, int nruns, long long ntiles, int tile, int halo,
                           long long max_nodes, int parity, int k, int blocks_per_sm, unsigned* status,
                           cudaStream_t st);
int sm_count_host();

// --- aux_kernels.cu ----------------------------------------------------------
cudaError_t launch_init_droplets(const Geo& g, int n, const double* d_centres, const double* d_radii, double width,
                                 float* phi0, float* rho0, float* u0, cudaStream_t st);
cudaError_t launch_phi_from_init(int storage, const Geo& g, const float* phi0, void* phi, cudaStream_t st);
// deterministic FP64 sums of the fields buffer; partials needs nblocks*8 doubles
int reduce_blocks(long long N);
cudaError_t launch_reduce(int storage, const Geo& g, const void* fields, double* partials, double* out8,
                          cudaStream_t st);
cudaError_t launch_laplace(int storage, const Geo& g, const void* fields, double cut, double* partials,
                           double* out4, cudaStream_t st);
cudaError_t launch_cc(int storage, const Geo& g, const void* fields, int* labels, int* count, unsigned* status,
                      cudaStream_t st);
// droplet count and dispersed volume of a float phase-field array [N]
cudaError_t launch_phi_monitor(const Geo& g, const float* phi, int* labels, int* count, double* partials,
                               double* volume, unsigned* status, cudaStream_t st);

// --- surrogate_rt.cu ---------------------------------------------------------
struct SurrogateState;
void destroy_surrogate(SurrogateState* s);

// --- runtime.cu --------------------------------------------------------------
// record code + message as the calling thread's last error; returns code
int report_error(int code, const std::string& msg);
}  // namespace lbcg
struct lb_handle;
namespace lbcg {
// handle internals for the surrogate runtime
cudaStream_t handle_stream(lb_handle* h);
void handle_dims(const lb_handle* h, int* nx, int* ny, int* nz, uint32_t* walls);
void* handle_alloc(lb_handle* h, size_t bytes);  // owned (freed) by the handle
SurrogateState*& handle_surrogate(lb_handle* h);
// add n to the library's kernel launch counter
void count_launches(int n);

}  // namespace lbcg
