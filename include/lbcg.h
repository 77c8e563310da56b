/*
 * lbcg.h -- C ABI of the GB300 colour-gradient lattice Boltzmann library.
 *
 * One time step of the two-component colour-gradient lattice Boltzmann scheme
 * on D3Q27 with the coarse-grained near-contact repulsion of arXiv 2405.14551:
 *   BGK collision on the total populations   (Sec. III.B Eq. eq:lbm,
 *                                             Sec. III.C.1 Eq. CGLBE),
 *   surface-tension perturbation             (Sec. III.C.1, Omega^(2), Eq. sigmaA),
 *   Latva-Kokko recolouring                  (Eqs. ome3_1, ome3_2),
 *   near-contact force F_rep = -A_h n delta_I (Eqs. stress_jump, near_cont_force),
 *   forcing term (Guo)                       (near-contact paragraph: "forcing contribution"),
 *   streaming with periodic wrap and halfway bounce-back walls (Sec. III.D).
 *
 * Every function returns LB_OK (0) or a negative LB_E* code; lb_strerror()
 * names it and lb_last_error() gives the detail of the last failure on the
 * calling thread.  Nothing falls back to the CPU: without a CUDA device the
 * calls fail with LB_ECUDA.
 *
 * Threading: a handle is not thread safe; distinct handles may be used from
 * distinct threads.  All device work of a handle is issued on its stream
 * (lb_set_stream, default: the legacy default stream).
 */
#ifndef LBCG_H
#define LBCG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ------------------------------------------------------ */
#define LB_OK 0
#define LB_EINVAL -1    /* an argument failed host-side validation; no GPU work was issued */
#define LB_ENOMEM -2    /* a device or host allocation failed */
#define LB_ECUDA -3     /* a CUDA runtime call failed (detail in lb_last_error) */
#define LB_EUNSTABLE -4 /* the device status word saw a density that is not finite, not positive or not below 4
                           (64 in FP64 storage), the range of the fixed-point density sums */
#define LB_ETIMEOUT -5  /* a bounded device wait gave up */
#define LB_ESTATE -6    /* the call is not valid in the handle's current state */
#define LB_EIO -7       /* file read/write failed or the file is not a checkpoint of this grid */

/* ---- population storage formats ---------------------------------------- */
/* Two population sets f^A, f^B in FP32, [comp][27][nz][ny][nx]; 432 B per node update. */
#define LB_STORAGE_TWOSET_F32 0
/* Exact single-set form: total post-collision f* (27 x FP32) plus the colour
 * scalars s = rhoA/rho and v = beta rhoA rhoB/rho n (one float4); the pulling
 * node rebuilds f^A_i = s f*_i + w_i c_i.v/|c_i| (recolouring, Eq. ome3_1). */
#define LB_STORAGE_REDUCED_F32 1
/* As REDUCED_F32 but f*_i stored as FP16 deviations (f*_i - w_i) * 4096 from
 * the rest equilibrium at rho_0 = 1, u_0 = 0 (Sec. IV.B, Eq. eq:shift_f); all
 * arithmetic in FP32. */
#define LB_STORAGE_REDUCED_F16 2
/* Two population sets in FP64, FP64 arithmetic (parity instantiation). */
#define LB_STORAGE_TWOSET_F64 3
/* Moment storage (population-free, Sec. IV.C, Eqs. distnoneq, LBpostmom,
 * eq:llb-pull): with the regularised collision every post-collision total
 * population is w_i times a quadratic form in c_i, so a node stores the ten
 * coefficients (alpha, beta, Gamma) of f*_i = w_i (alpha + beta.c_i +
 * c_i.Gamma.c_i) plus the colour scalars (s, v) of REDUCED_F32; the pulling
 * node evaluates them.  FP32 records (alpha, beta) [N] float4, (Gamma_xx,
 * Gamma_yy, Gamma_zz, 2 Gamma_xy) [N] float4, (2 Gamma_xz, 2 Gamma_yz) [N]
 * float2, then (s, v) [N] float4: 56 B per node per lattice (112 B per node
 * update).  Requires collision = 1 (LB_EINVAL otherwise). */
#define LB_STORAGE_MOMENT_F32 4

/* ---- field selection for lb_fields: bit k selects field k --------------- */
#define LB_F_PHI (1u << 0)  /* order parameter (rhoA-rhoB)/(rhoA+rhoB), Eq. order_param */
#define LB_F_RHO (1u << 1)  /* total density, Sec. III.C.1 */
#define LB_F_UX (1u << 2)   /* barycentric velocity u = (j + F/2)/rho */
#define LB_F_UY (1u << 3)
#define LB_F_UZ (1u << 4)
#define LB_F_RHOA (1u << 5)
#define LB_F_RHOB (1u << 6)
#define LB_F_FRX (1u << 7)  /* near-contact force F_rep, Eq. near_cont_force */
#define LB_F_FRY (1u << 8)
#define LB_F_FRZ (1u << 9)
#define LB_F_H (1u << 10)   /* near-contact distance h(x) in lattice units, 0 = inactive */
#define LB_F_GX (1u << 11)  /* colour gradient grad phi */
#define LB_F_GY (1u << 12)
#define LB_F_GZ (1u << 13)
#define LB_NFIELDS 14

typedef struct lb_handle lb_handle;

/* Lattice box.  x is fastest: node (x,y,z) has index x + nx*(y + ny*z).
 * walls bit a (a = 0,1,2 for x,y,z) makes layers 0 and n_a-1 of that axis
 * solid (halfway bounce-back); other axes are periodic (Sec. III.D). */
typedef struct {
  int32_t nx, ny, nz;
  uint32_t walls;
} lb_grid;

/* Model parameters, named after the paper's notation (Sec. III.C.1). */
typedef struct {
  double tau_a, tau_b;    /* relaxation times (> 0.5); nu_k = (tau_k - 1/2)/3, mixed harmonically (Eq. sigmaA) */
  double A_a, A_b;        /* perturbation amplitudes A_k; sigma = (2/9)(A_a + A_b) tau_bar */
  double beta;            /* recolouring parameter, [0, 1] */
  double A_h;             /* near-contact strength A_h (0 switches the force off) */
  double h_min, h_max;    /* A_h constant for h <= h_min, ~ h^-3 up to h_max, 0 beyond; 1 <= h_max <= 6 */
  double phi_I;           /* |phi| < phi_I marks interface nodes for the near-contact scan (0.9) */
  double g[3];            /* body-force vector */
  int32_t g_mode;         /* 0 none; 1 F = rho g; 2 F = s(z) rhoA g, s = +1 below nz/2, -1 above, 0 at z = 0, nz/2 */
  int32_t storage;        /* LB_STORAGE_* */
  int32_t collision;      /* 0: BGK on the total (Sec. III.B); 1: regularised colour-gradient collision (the
                             ghost-mode filtering Sec. III.C.1 cites): the non-equilibrium part of the total is
                             projected on Hermite orders 1 and 2 before relaxation; moments up to order 2 as BGK */
  int32_t model;          /* LB_MODEL_COLOUR_GRADIENT (0) or LB_MODEL_SHAN_CHEN (1) */
  double G;               /* Shan-Chen coupling G_AB = G_BA (G_AA = G_BB = 0); model 1 only */
  double psi0;            /* rho_0 of the pseudo-potential psi(rho) = rho_0 (1 - exp(-rho/rho_0)); model 1 only */
} lb_params;

/* Two-component models.  COLOUR_GRADIENT: the scheme above (A_a, A_b, beta,
 * near contact).  SHAN_CHEN: the lattice pseudo-potential model of Sec.
 * III.C.3: each component relaxes by BGK with its own tau_k towards
 * f^eq(rho_k, u'), u' = sum_k (j_k + F_k/2)/tau_k / sum_k rho_k/tau_k, with
 * the Guo source of its own force F_k(x) = -psi_k(x) G sum_i w_i
 * psi_k'(x + c_i) c_i (k' the other component; a solid neighbour
 * contributes the node's own psi), plus its share of the body force (rho_k g
 * for g_mode 1, all of it on A for g_mode 2).  Requires a two-set storage
 * (TWOSET_F32 or TWOSET_F64), A_h = 0, collision = 0 and psi0 > 0; A_a, A_b
 * and beta are ignored.  Fields: F_rep holds the total Shan-Chen force
 * F_A + F_B, h is 0. */
#define LB_MODEL_COLOUR_GRADIENT 0
#define LB_MODEL_SHAN_CHEN 1

/* Optional device allocator (for example PyTorch's caching allocator).  With
 * a NULL lb_alloc the library uses cudaMalloc/cudaFree.  alloc returns a
 * device pointer aligned to 256 bytes or NULL; free releases it.  The handle
 * calls free for every pointer it obtained, at lb_destroy at the latest. */
typedef struct {
  void* (*alloc)(void* ctx, size_t bytes);
  void (*free)(void* ctx, void* ptr);
  void* ctx;
} lb_alloc;

/* Create a handle on the current CUDA device.  Validates grid and params on
 * the host (LB_EINVAL, nothing allocated), then allocates two population
 * lattices in the chosen storage, three accumulators of the component
 * densities (8 bytes per node each, 16 in FP64 storage) that carry phi from
 * one step to the next, and the initial-field arrays.  *out receives the
 * handle (caller-owned; release with lb_destroy). */
int lb_create(const lb_grid* grid, const lb_params* params, const lb_alloc* alloc, lb_handle** out);

/* Release all device memory of the handle (after synchronising its stream). */
int lb_destroy(lb_handle* h);

/* Issue all further work of h on the given cudaStream_t (NULL: legacy stream).
 * Drops any captured step graph. */
int lb_set_stream(lb_handle* h, void* stream);

/* Droplet initial state: phi = +1 within distance R_j of centre j (periodic
 * distance on open axes, union over droplets), -1 elsewhere; with width > 0,
 * phi = max_j tanh((R_j - d_j)/width).  rho = 1, u = 0, populations at the
 * component equilibria f^k_i = f^eq_i(rho_k, u) (Eq. disteq).  centres (3n
 * doubles, x,y,z) and radii (n doubles) are host arrays; 0 <= n <= 1<<20.
 * Resets the step counter to 0.  Asynchronous on the handle's stream. */
int lb_init_droplets(lb_handle* h, int32_t n, const double* centres, const double* radii, double width);

/* Initial state from fields: phi[N], rho[N] (NULL: 1), u[3][N] (NULL: 0).
 * regularised = 0: component equilibria; 1: regularised reconstruction
 * f_i = f^eq_i + w_i/(2 c_s^4) Q_i : Pi^neq with Pi^neq = -rho c_s^2 tau_bar
 * (grad u + grad u^T) (Sec. IV.C, Eqs. distnoneq, eq:llb-pull), colour split
 * f^A = (rhoA/rho) f.  is_device selects device or host pointers (float).
 * Resets the step counter to 0. */
int lb_init_fields(lb_handle* h, const float* phi, const float* rho, const float* u, int regularised,
                   int is_device);

/* Advance nsteps >= 0 time steps, asynchronously on the handle's stream.
 * Each step is one kernel over tiles of nodes: it stages phi of the tile and
 * a halo, runs the near-contact scan of Eqs. stress_jump / near_cont_force
 * for the tile's interface nodes (with A_h != 0), pulls, collides, recolours
 * and stores every node (one read and one write of the population state),
 * and adds each stored component population to the density sums of the node
 * that pulls it next, which give phi at the next step (Eq. order_param).
 * Runs of 12 steps are replayed from a captured CUDA graph. */
int lb_step(lb_handle* h, int64_t nsteps);

/* Choose the tile shape of the step kernel (0..5: 32x8x4, 32x8x8, 32x8x4
 * with a register cap for 3 CTAs per SM, 32x8x6 capped for 3 CTAs per SM,
 * 32x4x4 capped for 6 CTAs per SM, nodes per CTA; 5: 32x8x8 with the
 * near-contact scan of each interface node inside the node loop instead of
 * a phase of its own); used by the autotuner.  Results do not depend on the
 * tile (bit for bit).  Lattices too large for 32-bit population offsets
 * (2 x 27 x nodes >= 2^32) step with tile 0 whatever the setting.
 * lb_get_tile returns the current index. */
int lb_set_tile(lb_handle* h, int tile);
int lb_get_tile(const lb_handle* h);

/* Advance nsteps >= 1 steps without graph replay, recording a CUDA event on
 * the handle's stream after every step kernel.  Synchronises the stream;
 * *ms receives the mean duration of one step kernel in milliseconds. */
int lb_step_timed(lb_handle* h, int64_t nsteps, double* ms);

/* Steps taken since the last initialisation. */
int64_t lb_time(const lb_handle* h);

/* Write the selected fields at the current time level, [k][nz][ny][nx] float
 * in increasing bit order of mask, to dst (device or host pointer of
 * popcount(mask)*N floats, caller-owned).  Synchronises the stream when dst is
 * on the host.  Solid nodes hold 0. */
int lb_fields(lb_handle* h, uint32_t mask, float* dst, int dst_is_device);
/* Same in double precision (fields of an FP64 handle keep full precision). */
int lb_fields_f64(lb_handle* h, uint32_t mask, double* dst, int dst_is_device);

/* Pre-collision populations of both components at the current time level for
 * the box [x0,x0+bx) x [y0,y0+by) x [z0,z0+bz) (inside the grid), written to
 * host arrays fA, fB of 27*bx*by*bz doubles, [dir][z][y][x] with the canonical
 * direction index (cx+1) + 3(cy+1) + 9(cz+1).  Synchronises the stream. */
int lb_get_populations(lb_handle* h, int32_t x0, int32_t y0, int32_t z0, int32_t bx, int32_t by, int32_t bz,
                       double* fA, double* fB);

/* FP64 sums over fluid nodes at the current time level (deterministic order):
 * out[0] mass A, [1] mass B, [2..4] momentum rho u, [5] A volume sum (1+phi)/2,
 * [6] near-contact active nodes, [7] kinetic energy sum rho |u|^2 / 2.
 * out is a host array of 8 doubles.  Synchronises the stream. */
int lb_reduce_f64(lb_handle* h, double* out);

/* Laplace readout in FP64 (extended Young-Laplace relation, pi = 0 for an
 * isolated droplet): dp = c_s^2 (<rho>_{phi > cut} - <rho>_{phi < -cut}).
 * Returns LB_ESTATE if either region is empty.  Synchronises the stream. */
int lb_laplace_f64(lb_handle* h, double cut, double* dp);

/* Number of droplets: connected components of fluid nodes with phi > 0,
 * 6-connected, periodic on open axes.  Synchronises the stream. */
int lb_droplet_count(lb_handle* h, int32_t* count);

/* Drift monitors of a phase field that is not (yet) the handle's state, for
 * example a surrogate's candidate: phi is a device array of nx*ny*nz floats
 * on the handle's grid (x fastest).  *count receives the number of
 * 6-connected phi > 0 components among fluid nodes (periodic on open axes,
 * as lb_droplet_count) and *volume the dispersed volume, the sum over fluid
 * nodes of (1 + phi)/2 in FP64 (the same sum, in the same order, as
 * lb_reduce_f64's out[5]).  Uses the handle's scratch, leaves its state
 * untouched and synchronises its stream.  LB_ETIMEOUT if the union-find gave
 * up.  These are the drift monitors of the surrogate controller. */
int lb_phi_monitor(lb_handle* h, const float* phi, int32_t* count, double* volume);

/* Learned surrogate (an extension of the method: a network that
 * advances (phi, rho, u) by K steps, with the plain LB as fallback and judge;
 * populations rebuilt by the regularised reconstruction of Sec. IV.C).
 *
 * lb_surrogate_load: read a U-Net weight file written by
 * paper_2405_14551_gb300.surrogate.UNet.save (4 levels, base 8..64 channels,
 * 16 input and head channels, FP32 weights stored as BF16 on the device) and
 * allocate its weights and activation buffers for the handle's grid through
 * the handle's allocator (released by lb_destroy).  Every extent must be a
 * multiple of 8.  LB_EIO for a missing or mismatched file, LB_ESTATE if a
 * network is already loaded, LB_EINVAL for unsuitable extents.
 *
 * lb_surrogate_predict: the candidate state K steps ahead, [5][N] float
 * (phi, rho, ux, uy, uz) into out (a device pointer, or NULL to keep it only
 * inside the handle); the handle's state is not changed.  Synchronises the
 * stream; LB_ETIMEOUT if a tensor-core kernel gave up a bounded wait.
 *
 * lb_surrogate_cycle: one jump of K steps on h.  The candidate is checked by
 * the drift monitors (droplet count unchanged, dispersed volume within
 * vol_tol relative, as lb_phi_monitor); with judge != NULL (a handle of the
 * same grid and storage) the plain LB also advances the exact same state by
 * K steps on judge and *phi_err receives mean |phi_candidate - phi_LB| over
 * all nodes, which must not exceed phi_tol (else *phi_err = -1).  Accepted
 * (*accepted = 1): h is re-initialised from the candidate by regularised
 * reconstruction (step counter reset).  Rejected: h takes the judge's state,
 * or steps K plain LB steps without a judge. */
int lb_surrogate_load(lb_handle* h, const char* path);
int lb_surrogate_predict(lb_handle* h, float* out);
int lb_surrogate_cycle(lb_handle* h, lb_handle* judge, int32_t K, double vol_tol, double phi_tol, int32_t* accepted,
                       double* phi_err);

/* Synchronise the stream and read the device status word: LB_OK or
 * LB_EUNSTABLE once any step met a density that is not finite, not positive
 * or not below 4 (64 in FP64 storage). */
int lb_check(lb_handle* h);

/* Checkpoint: raw population state, step counter, grid, parameters and a
 * format version.  lb_load requires a handle of the same grid and storage. */
int lb_save(lb_handle* h, const char* path);
int lb_load(lb_handle* h, const char* path);

/* Copy the state of src into dst (same grid, walls and storage; parameters
 * may differ): the population lattice, or the initial fields if src has not
 * stepped yet, and the step counter.  Waits for src's stream, then copies
 * device to device on dst's stream (asynchronous for dst).  LB_EINVAL if the
 * handles differ in grid or storage, LB_ESTATE if src is not initialised.
 * Used to start a plain-LB judge run from the exact state of a run. */
int lb_copy_state(lb_handle* dst, lb_handle* src);

/* Number of kernels this library has launched in this process (graph replays
 * count every kernel node). */
uint64_t lb_launch_count(void);

/* Bytes of device memory the handle holds. */
size_t lb_device_bytes(const lb_handle* h);

/* ---- batches of independent runs (uneven grids and parameters) ---------- */
typedef struct lb_batch lb_batch;

/* Create nruns runs (grids[r], params[r]; one storage format for all, FP32 or
 * FP16; FP64 is rejected) on the current device, sharing one stream.  Each run
 * is a full lb_handle reachable through lb_batch_run; the batch owns them. */
int lb_batch_create(int32_t nruns, const lb_grid* grids, const lb_params* params, const lb_alloc* alloc,
                    lb_batch** out);
int lb_batch_destroy(lb_batch* b);

/* Borrowed handle of run r (initialise it with lb_init_droplets/lb_init_fields,
 * read it with lb_fields/lb_reduce_f64/...; do not destroy it).  NULL when r
 * is out of range. */
lb_handle* lb_batch_run(lb_batch* b, int32_t run);
int32_t lb_batch_size(const lb_batch* b);
int64_t lb_batch_nodes(const lb_batch* b);
int lb_batch_set_stream(lb_batch* b, void* stream);

/* Advance every run by nsteps: per step one persistent launch over the work
 * list of all runs' (run, tile) items (the step of lb_step on each tile),
 * replayed from a captured CUDA graph.  All runs must be initialised and at
 * the same lattice parity; the first step of freshly initialised runs is
 * taken per run. */
int lb_batch_step(lb_batch* b, int64_t nsteps);

/* The one-run-at-a-time baseline: lb_step on each run in turn. */
int lb_batch_step_sequential(lb_batch* b, int64_t nsteps);

/* Tile shape (0..5, as lb_set_tile) and persistent CTAs per SM (1..16). */
int lb_batch_set_tile(lb_batch* b, int tile, int blocks_per_sm);

/* Autotuner: time `steps` batched steps for every tile shape and CTAs-per-SM
 * in {1, 2, 4}, keep the fastest.  Needs freshly initialised runs (step 0)
 * and returns every run to its initial state afterwards.  With use_cache, a result stored for the same
 * GPU, storage and set of run shapes is reused.  Results are appended to the
 * file named by LBCG_TUNE_CACHE (default $HOME/.cache/lbcg_tune.txt).
 * result (host, 4 doubles): tile, blocks_per_sm, ms per step, 1 if cached. */
int lb_batch_autotune(lb_batch* b, int32_t steps, int use_cache, double* result);

/* lb_check on every run. */
int lb_batch_check(lb_batch* b);

/* ---- allocation-free reduction (no counterpart in the paper) ------------- */
/* Same sums as lb_reduce_f64, for callers that cannot allocate device memory
 * (programs that hand out all device memory themselves and forbid later
 * allocations, or paths that must avoid the implicit synchronisation of
 * cudaMalloc/cudaFree).  Allocates nothing: the block partial sums live in a
 * static 64 KiB device array of the library (LB_STATIC_REDUCE_MAX_BLOCKS
 * blocks x 8 doubles), held by every GPU that loads the library until the
 * process exits.
 *   fields: device array [14][nz][ny][nx] as written by lb_fields with all 14
 *           fields selected (float, or double when fields_are_f64 != 0);
 *   out:    device array of 8 doubles (same meaning as lb_reduce_f64's),
 *           written asynchronously on `stream` (cudaStream_t, NULL = legacy);
 *   walls:  as lb_grid.walls (solid layers are excluded from the sums).
 * Grids above 2^31 - 1 nodes are rejected with LB_EINVAL.  The first call on
 * a device looks up the array's device address (cudaGetSymbolAddress) with
 * that device current; make that first call before any stream capture.
 * Every call shares the one array: calls that overlap on the GPU (concurrent
 * streams) race and must be serialised by the caller.  Nothing needs
 * clearing between calls: every partial and every output is overwritten.
 * The address found by the first call stays in use for the life of the
 * process; after a cudaDeviceReset of a device, do not call this entry point
 * on that device again. */
#define LB_STATIC_REDUCE_MAX_BLOCKS 1024
int lb_reduce_fields_f64_static(const void* fields, int fields_are_f64, int32_t nx, int32_t ny, int32_t nz,
                                uint32_t walls, double* out, void* stream);

const char* lb_strerror(int code);
const char* lb_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* LBCG_H */
