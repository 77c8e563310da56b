// 3-D convolutions of the surrogate network on the tcgen05 tensor cores.
//
// Activations are channels-last BF16, X[v][c] with v = x + nx (y + ny (z + nz b)).
// Forward (and, with flipped weights, the input gradient) is an implicit GEMM
//   D[M = voxels][N = Cout] = sum_K A[M][K] B[N][K],  K = taps x Cin,
// A[v][(t,ci)] = X[v + off_t][ci] gathered on the fly, B[co][(t,ci)] = W[co][t][ci].
// The weight gradient is the GEMM
//   dW^T[M = taps x Cin][N = Cout] = sum_v X[v + off_t][ci] dY[v][co]
// with K = voxels; its operands are MN-major (channels contiguous).
// Grids with nx % 8 == 0 and ny % 16 == 0 (every level of the network) take
// the spatially tiled, pipelined kernels k_conv_fwd_pipe and
// k_conv_wgrad_pipe: persistent CTAs with copy, UMMA-issue and epilogue
// warps handing shared-memory buffers and tensor-memory accumulators over
// through mbarriers, the input block of a tile staged once per channel
// chunk.  Other grids and the 1x1x1 head take k_conv_fwd / k_conv_wgrad: one
// CTA of 128 threads owns a 128-row accumulator in tensor memory (one lane
// per row, FP32), operands are gathered through two shared-memory buffers in
// the no-swizzle core-matrix layout, one thread issues the UMMAs and commits
// them to an mbarrier per buffer.  Every wait is bounded; a wait that gives
// up sets bit 4 of the status word.
#include <cuda_bf16.h>

#include <atomic>
#include <string>

#include "../../include/lbcg.h"
#include "../../include/lbnn.h"
#include "internal.h"
#include "tc_ptx.cuh"

namespace lbcg {

struct ConvGeo {
  int nx, ny, nz, nb;  // spatial extents and batch
  int px, py, pz;      // 1: periodic axis, 0: zero padding
};

constexpr int CONV_M = 128;
constexpr unsigned CONV_TIMEOUT = 16u;
// Polls of a drain wait (all committed UMMAs done before tensor memory is
// freed); the handshake waits take their limit from the launch.
constexpr uint32_t CONV_DRAIN_SPIN = 1u << 22;

__device__ __forceinline__ long long conv_nbr(const ConvGeo& g, int b, int x, int y, int z, int dx, int dy, int dz) {
  x += dx;
  y += dy;
  z += dz;
  if (x < 0 || x >= g.nx) {
    if (!g.px) return -1;
    x = x < 0 ? x + g.nx : x - g.nx;
  }
  if (y < 0 || y >= g.ny) {
    if (!g.py) return -1;
    y = y < 0 ? y + g.ny : y - g.ny;
  }
  if (z < 0 || z >= g.nz) {
    if (!g.pz) return -1;
    z = z < 0 ? z + g.nz : z - g.nz;
  }
  return (((long long)b * g.nz + z) * g.ny + y) * g.nx + x;
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&h);
}

// ---------------------------------------------------------------------------
// forward / input gradient
// ---------------------------------------------------------------------------
// smem: A[2][128 * KC] | B[2][Cout * KC] (BF16, core-matrix layout) | mbar[2] | tmem address
template <int NT>
__global__ void __launch_bounds__(128, 1)
    k_conv_fwd(const __nv_bfloat16* __restrict__ X, int Cin, const __nv_bfloat16* __restrict__ W,
               const float* __restrict__ bias, __nv_bfloat16* __restrict__ Y, float* __restrict__ Yf, int Cout, int ldy,
               int KC, ConvGeo g, int relu, unsigned spin, unsigned* __restrict__ status) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int t = threadIdx.x;
  const int warp = t >> 5;
  const size_t a_bytes = (size_t)CONV_M * KC * 2, b_bytes = (size_t)Cout * KC * 2;
  unsigned char* sA[2] = {smem, smem + a_bytes};
  unsigned char* sB[2] = {smem + 2 * a_bytes, smem + 2 * a_bytes + b_bytes};
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + 2 * a_bytes + 2 * b_bytes);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar + 2);
  uint32_t ncols = 32;
  while ((int)ncols < Cout) ncols <<= 1;

  if (warp == 0) {
    tc::tmem_alloc(tmem_slot, ncols);
    tc::tmem_relinquish();
  }
  if (t == 0) {
    tc::mbar_init(&bar[0], 1);
    tc::mbar_init(&bar[1], 1);
    tc::fence_mbar_init();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tmem_slot;

  const long long nvox = (long long)g.nb * g.nz * g.ny * g.nx;
  const long long v = (long long)blockIdx.x * CONV_M + t;
  const bool valid = v < nvox;
  int x = 0, y = 0, z = 0, b = 0;
  if (valid) {
    long long r = v;
    x = (int)(r % g.nx);
    r /= g.nx;
    y = (int)(r % g.ny);
    r /= g.ny;
    z = (int)(r % g.nz);
    b = (int)(r / g.nz);
  }
  const int cpt = Cin / KC;  // chunks per tap
  const int nchunks = NT * cpt;
  const uint32_t idesc = tc::idesc_bf16(CONV_M, Cout, false, false);
  const uint32_t a_lbo = CONV_M * 16, b_lbo = (uint32_t)Cout * 16;
  bool ok = true;
  int issued = 0;  // chunks whose UMMAs were issued and committed

  for (int ch = 0; ch < nchunks; ++ch) {
    const int buf = ch & 1;
    if (ch >= 2) {  // the UMMAs that read this buffer two chunks ago must be done
      bool w = tc::mbar_wait(&bar[buf], (uint32_t)(((ch >> 1) - 1) & 1), spin);
      ok = __syncthreads_and(w);
      if (!ok) break;
    }
    const int tap = ch / cpt;
    const int c0 = (ch % cpt) * KC;
    const int dx = NT == 1 ? 0 : tap % 3 - 1, dy = NT == 1 ? 0 : (tap / 3) % 3 - 1, dz = NT == 1 ? 0 : tap / 9 - 1;
    // A: this thread's row
    const long long src = valid ? conv_nbr(g, b, x, y, z, dx, dy, dz) : -1;
    const uint4* xs = reinterpret_cast<const uint4*>(X + (src >= 0 ? src : 0) * (long long)Cin + c0);
    for (int kg = 0; kg < KC / 8; ++kg) {
      uint4 val = make_uint4(0, 0, 0, 0);
      if (src >= 0) val = xs[kg];
      *reinterpret_cast<uint4*>(sA[buf] + (size_t)t * 16 + (size_t)kg * a_lbo) = val;
    }
    // B: rows co = t, t + 128, ...
    for (int co = t; co < Cout; co += CONV_M) {
      const uint4* ws = reinterpret_cast<const uint4*>(W + ((size_t)co * NT + tap) * Cin + c0);
      for (int kg = 0; kg < KC / 8; ++kg)
        *reinterpret_cast<uint4*>(sB[buf] + (size_t)co * 16 + (size_t)kg * b_lbo) = ws[kg];
    }
    tc::fence_proxy_async_smem();
    __syncthreads();
    if (t == 0) {
      tc::fence_after_sync();
      const uint32_t a0 = tc::smem_u32(sA[buf]), b0 = tc::smem_u32(sB[buf]);
      for (int j = 0; j < KC / 16; ++j) {
        const uint64_t ad = tc::smem_desc(a0 + (uint32_t)j * 2 * a_lbo, a_lbo, 128);
        const uint64_t bd = tc::smem_desc(b0 + (uint32_t)j * 2 * b_lbo, b_lbo, 128);
        tc::mma_bf16(tmem, ad, bd, idesc, (ch > 0 || j > 0) ? 1u : 0u);
      }
      tc::mma_commit(&bar[buf]);
    }
    issued = ch + 1;
  }
  // every committed UMMA, also after a give-up: the last commit covers every
  // earlier one of the issuing thread; the drain has its own fixed bound
  bool done = true;
  if (issued > 0) {
    const int last = issued - 1;
    done = tc::mbar_wait(&bar[last & 1], (uint32_t)((last >> 1) & 1), CONV_DRAIN_SPIN);
    if (!done) done = tc::mbar_wait(&bar[last & 1], (uint32_t)((last >> 1) & 1), CONV_DRAIN_SPIN);
  }
  ok = __syncthreads_and(ok && done);
  tc::fence_after_sync();
  if (ok) {
    const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
    for (int col = 0; col < Cout; col += 16) {
      float acc[16];
      tc::tmem_ld16(lane_base + (uint32_t)col, acc);
      if (valid) {
#pragma unroll
        for (int k = 0; k < 16; ++k) {
          float vv = acc[k] + (bias ? bias[col + k] : 0.0f);
          acc[k] = relu ? fmaxf(vv, 0.0f) : vv;
        }
        if (Y) {
          uint4* yp = reinterpret_cast<uint4*>(Y + v * ldy + col);
          yp[0] = make_uint4(pack_bf16(acc[0], acc[1]), pack_bf16(acc[2], acc[3]), pack_bf16(acc[4], acc[5]),
                             pack_bf16(acc[6], acc[7]));
          yp[1] = make_uint4(pack_bf16(acc[8], acc[9]), pack_bf16(acc[10], acc[11]), pack_bf16(acc[12], acc[13]),
                             pack_bf16(acc[14], acc[15]));
        }
        if (Yf) {
          float4* fp = reinterpret_cast<float4*>(Yf + v * ldy + col);
#pragma unroll
          for (int q = 0; q < 4; ++q) fp[q] = make_float4(acc[4 * q], acc[4 * q + 1], acc[4 * q + 2], acc[4 * q + 3]);
        }
      }
    }
  } else if (t == 0) {
    atomicOr(status, CONV_TIMEOUT);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, ncols);
}

// ---------------------------------------------------------------------------
// forward / input gradient, spatially tiled and pipelined (3x3x3 taps)
// ---------------------------------------------------------------------------
// Work item: an output block of 8 (x) x 16 (y) x TZ (z) voxels and CT output
// channels (CT = Cout, or a slice of it when Cout is large and the grid
// small).  Persistent CTAs walk the work items; warps have fixed roles:
//   warps 0-3  epilogue: tensor memory -> bias, ReLU -> BF16 / FP32 stores
//   warps 4-7  copies (cp.async, zero fill for padded voxels)
//   warp 8     tensor-memory allocation; lane 0 issues the UMMAs
// and hand buffers over through mbarriers only.
//
// Per chunk of KC input channels the input block with a one-voxel halo
// (10 x 18 x (TZ + 2) voxels) is staged once, in the layout
//   piece (cg, zz, yy, xx) of 8 channels at ((cg * SZH + zz) * 18 + yy) * 10 + xx,
// so that the 128 output rows of a z plane (8 x voxels = one core matrix,
// 16 y rows 160 bytes apart) read a tap's input as the same staged block at
// a shifted start address.
//
// MERGE (3 CT <= 256): the three z taps of one (dx, dy) share the A operand.
// The weights of (dx, dy) are staged as one B operand of 3 CT rows, block s
// holding the tap dz = s - 1, and the accumulator of output plane q sits at
// column (TZ - 1 - q) CT.  One UMMA with input plane zz and blocks
// [s_lo, s_hi] then adds W(dz = s - 1) X(zz) to plane q = zz - s for every
// block at once: 9 steps of TZ + 2 UMMAs of up to 3 CT columns per chunk
// instead of 27 steps of TZ UMMAs of CT columns.  The first k-step of a work
// item is issued block by block (block 1 first, without accumulation) so
// that every plane is initialised before it is accumulated.
//
// Without MERGE a step is one tap: TZ UMMAs of CT columns.
// Decoder layers read their input in place: channels [0, cs) from X, the
// rest from X2 at the parent voxel (nearest x2 upsampling), a chunk lying
// wholly in one source, so the concatenated tensor is never written.
// Accumulators are double buffered (2 TZ CT <= 512 columns), so the epilogue
// of one work item overlaps the UMMAs of the next.  Every wait is bounded; a
// wait that gives up sets bit 4 of the status word and the CTA winds down.
constexpr int PCONV_EPI = 128;     // epilogue threads (warps 0-3, one per tensor-memory lane quarter)
constexpr int PCONV_THREADS = 288;
constexpr int PCONV_PROD0 = 128;  // first copy thread
constexpr int PCONV_NPROD = 128;  // copy threads
constexpr int PCONV_MMA_WARP = 8;
constexpr int PCONV_MAXWP = 8;    // weight pieces per copy thread and step (3 CT or CT rows x KC / 8 <= 1024)
constexpr int PCONV_LAG = 5;      // steps a copy thread keeps in flight before it signals them
constexpr int PCONV_NSW_MAX = 8;  // weight ring slots (at most)

__device__ __forceinline__ int wrap_or_pad(int c, int n, int periodic) {
  if (c >= 0 && c < n) return c;
  if (!periodic) return -1;
  return c < 0 ? c + n : c - n;
}

// Bounded wait that also gives up once another role has given up.
// After a few polls the waiting warp backs off briefly, so that idle roles do
// not crowd the shared-memory pipe that the copies and the UMMAs use.
__device__ __forceinline__ bool pconv_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag, uint32_t limit) {
  for (uint32_t it = 0; it < limit; ++it) {
    if (tc::mbar_try_wait(bar, parity)) return true;
    if ((it & 255u) == 255u && *abort_flag) return false;
    if (it >= 16) __nanosleep(32);
  }
  return false;
}

struct PConvArgs {
  const __nv_bfloat16* X;   // input channels [0, cs): X[v][cs]
  const __nv_bfloat16* X2;  // input channels [cs, Cin), nearest x2 upsampled: X2[parent(v)][Cin - cs] (or null)
  int cs;
  const __nv_bfloat16* W;  // [Cout][27][Cin]
  const float* bias;
  __nv_bfloat16* Y;
  float* Yf;
  int Cin, Cout, ldy, KC, CT, nsw;
  ConvGeo g;
  int relu;
  unsigned spin;  // polls of a handshake wait before it gives up
  unsigned* status;
};

template <int TZ, bool MERGE>
__global__ void __launch_bounds__(PCONV_THREADS, 1) k_conv_fwd_pipe(PConvArgs P) {
  constexpr int SZH = TZ + 2;
  constexpr int HV = 10 * 18 * SZH;  // staged voxels
  constexpr int NBLK = MERGE ? 3 : 1;
  constexpr int SPC = MERGE ? 9 : 27;  // steps per chunk
  extern __shared__ __align__(1024) unsigned char smem[];
  const int t = threadIdx.x;
  const int warp = t >> 5;
  const int KC = P.KC, CT = P.CT, Cin = P.Cin, nsw = P.nsw;
  const int NB = NBLK * CT;  // rows of a staged B operand
  const int cgs = KC / 8;
  const size_t halo_bytes = (size_t)HV * KC * 2, w_bytes = (size_t)NB * KC * 2;
  unsigned char* sH = smem;                    // 2 input blocks
  unsigned char* sW = smem + 2 * halo_bytes;   // nsw weight slots
  uint64_t* bar = reinterpret_cast<uint64_t*>(sW + (size_t)nsw * w_bytes);
  uint64_t* w_full = bar;
  uint64_t* w_empty = bar + PCONV_NSW_MAX;
  uint64_t* h_full = bar + 2 * PCONV_NSW_MAX;
  uint64_t* h_empty = h_full + 2;
  uint64_t* a_full = h_full + 4;
  uint64_t* a_empty = h_full + 6;
  uint64_t* fin = h_full + 8;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(fin + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  float* sbias = reinterpret_cast<float*>(tmem_slot + 4);  // Cout values (0 without bias)
  uint32_t ncols = 32;
  while ((int)ncols < 2 * TZ * CT) ncols <<= 1;
  for (int c = t; c < P.Cout; c += PCONV_THREADS) sbias[c] = P.bias ? P.bias[c] : 0.0f;

  if (warp == PCONV_MMA_WARP) {
    tc::tmem_alloc(tmem_slot, ncols);
    tc::tmem_relinquish();
  }
  if (t == 0) {
    for (int k = 0; k < PCONV_NSW_MAX; ++k) {
      tc::mbar_init(&w_full[k], PCONV_NPROD);
      tc::mbar_init(&w_empty[k], 1);
    }
    for (int k = 0; k < 2; ++k) {
      tc::mbar_init(&h_full[k], PCONV_NPROD);
      tc::mbar_init(&h_empty[k], 1);
      tc::mbar_init(&a_full[k], 1);
      tc::mbar_init(&a_empty[k], PCONV_EPI);
    }
    tc::mbar_init(fin, 1);
    *abort_flag = 0;
    tc::fence_mbar_init();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tmem_slot;

  const ConvGeo& g = P.g;
  const int bxs = g.nx / 8, bys = g.ny / 16, bzs = g.nz / TZ;
  const int nsplit = P.Cout / CT;
  const int nitems = bxs * bys * bzs * g.nb * nsplit;
  const int nchunks = Cin / KC;
  const int my_items = blockIdx.x < nitems ? (nitems - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  auto item_of = [&](int k, int& x0, int& y0, int& z0, int& b, int& n0) {
    int it = blockIdx.x + k * gridDim.x;
    n0 = (it % nsplit) * CT;
    it /= nsplit;
    x0 = (it % bxs) * 8;
    it /= bxs;
    y0 = (it % bys) * 16;
    it /= bys;
    z0 = (it % bzs) * TZ;
    b = it / bzs;
  };

  if (t >= PCONV_PROD0 && t < PCONV_PROD0 + PCONV_NPROD) {
    // ------------------------------------------------------------ copies
    const int pt = t - PCONV_PROD0;
    const int nsteps = my_items * nchunks * SPC;
    // Weight pieces: a copy thread stages the same (k group, row) positions
    // of every step, so their offsets are set up once; a step only adds its
    // tap and channel chunk.
    int woff[PCONV_MAXWP];
    uint32_t wdo[PCONV_MAXWP];
#pragma unroll
    for (int i = 0; i < PCONV_MAXWP; ++i) {
      const int p = pt + i * PCONV_NPROD;
      const int kg = p % cgs, n = p / cgs;
      woff[i] = p < NB * cgs ? ((n % CT) * 27 + 9 * (n / CT)) * Cin + kg * 8 : -1;
      wdo[i] = (uint32_t)(kg * NB + n) * 16;
    }
    // Input pieces: one staged row (zz, yy) holds 10 x voxels x cgs groups;
    // a thread keeps its (xx, group) place in the row and walks the rows.
    const int hl = 10 * cgs, hr = PCONV_NPROD / hl;
    const bool hact = pt < hr * hl;
    const int hq = (pt % hl) % cgs, hxx = (pt % hl) / cgs, hy0 = pt / hl;
    bool ok = true;
    int gs = 0;
    for (int k = 0; k < my_items && ok; ++k) {
      int x0, y0, z0, b, n0;
      item_of(k, x0, y0, z0, b, n0);
      const int gx = wrap_or_pad(x0 - 1 + hxx, g.nx, g.px);
      const int cl = Cin - P.cs;
      const __nv_bfloat16* wbase = P.W + (size_t)n0 * 27 * Cin;
      for (int c = 0; c < nchunks && ok; ++c) {
        const int c0 = c * KC;
        for (int st = 0; st < SPC; ++st, ++gs) {
          const int slot = gs % nsw;
          if (gs >= nsw && !pconv_wait(&w_empty[slot], (uint32_t)(((gs / nsw) - 1) & 1), abort_flag, P.spin)) {
            ok = false;
            break;
          }
          unsigned char* wdst = sW + (size_t)slot * w_bytes;
          const __nv_bfloat16* wsrc = wbase + st * Cin + c0;
#pragma unroll
          for (int i = 0; i < PCONV_MAXWP; ++i)
            if (woff[i] >= 0) tc::cp_async16(wdst + wdo[i], wsrc + woff[i], true);
          if (st == 0) {
            const int cg = gs / SPC;
            if (cg >= 2 && !pconv_wait(&h_empty[cg & 1], (uint32_t)(((cg >> 1) - 1) & 1), abort_flag, P.spin)) {
              ok = false;
              break;
            }
            if (hact) {
              unsigned char* hdst = sH + (size_t)(cg & 1) * halo_bytes + ((size_t)hq * SZH * 180 + hxx) * 16;
              // a chunk lies wholly in one source (KC divides cs); the second is read at the parent voxel
              const bool up = c0 >= P.cs;
              const __nv_bfloat16* hsrc = up ? P.X2 + (c0 - P.cs) + hq * 8 : P.X + c0 + hq * 8;
              const int sh = up ? 1 : 0, ld = up ? cl : P.cs;
              const int nyv = g.ny >> sh, nxv = g.nx >> sh, nzv = g.nz >> sh, gxv = gx >> sh;
              for (int row = hy0; row < SZH * 18; row += hr) {
                const int zz = row / 18, yy = row - 18 * zz;
                const int gy = wrap_or_pad(y0 - 1 + yy, g.ny, g.py);
                const int gz = wrap_or_pad(z0 - 1 + zz, g.nz, g.pz);
                const bool in = gx >= 0 && gy >= 0 && gz >= 0;
                const int v = in ? ((b * nzv + (gz >> sh)) * nyv + (gy >> sh)) * nxv + gxv : 0;
                tc::cp_async16(hdst + (size_t)row * 160, hsrc + (long long)v * ld, in);
              }
            }
          }
          tc::cp_async_commit();
          if (gs >= PCONV_LAG) {  // step gs - LAG has landed: hand it over
            tc::cp_async_wait<PCONV_LAG>();
            tc::fence_proxy_async_smem();
            const int r = gs - PCONV_LAG;
            tc::mbar_arrive(&w_full[r % nsw]);
            if (r % SPC == 0) tc::mbar_arrive(&h_full[(r / SPC) & 1]);
          }
        }
      }
    }
    tc::cp_async_wait<0>();
    tc::fence_proxy_async_smem();
    if (ok) {
      for (int r = nsteps > PCONV_LAG ? nsteps - PCONV_LAG : 0; r < nsteps; ++r) {
        tc::mbar_arrive(&w_full[r % nsw]);
        if (r % SPC == 0) tc::mbar_arrive(&h_full[(r / SPC) & 1]);
      }
    } else {
      *abort_flag = 1;
      atomicOr(P.status, CONV_TIMEOUT);
    }
  } else if (warp == PCONV_MMA_WARP) {
    // ------------------------------------------------------------ UMMA issue
    if ((t & 31) == 0) {
      // descriptors: constant part + (shared address >> 4); every offset below is in 16-byte units
      const uint32_t a_lbo = (uint32_t)HV * 16, b_lbo = (uint32_t)NB * 16;
      const uint64_t adb = tc::smem_desc_base(a_lbo, 160), bdb = tc::smem_desc_base(b_lbo, 128);
      const uint32_t a_j = 2 * a_lbo >> 4, b_j = 2 * b_lbo >> 4;  // one k-step of 16 channels
      const uint32_t id1 = tc::idesc_bf16(CONV_M, CT, false, false);
      const uint32_t id2 = MERGE ? tc::idesc_bf16(CONV_M, 2 * CT, false, false) : id1;
      const uint32_t id3 = MERGE ? tc::idesc_bf16(CONV_M, 3 * CT, false, false) : id1;
      const int njs = KC / 16;
      bool ok = true;
      int gs = 0, slot = 0;
      uint32_t wphase = 0;
      for (int k = 0; k < my_items && ok; ++k) {
        const int ab = k & 1;
        if (k >= 2 && !pconv_wait(&a_empty[ab], (uint32_t)(((k >> 1) - 1) & 1), abort_flag, P.spin)) {
          ok = false;
          break;
        }
        tc::fence_after_sync();
        const uint32_t acc = tmem + (uint32_t)(ab * TZ * CT);
        for (int c = 0; c < nchunks && ok; ++c) {
          const int cg = gs / SPC;
          if (!pconv_wait(&h_full[cg & 1], (uint32_t)((cg >> 1) & 1), abort_flag, P.spin)) {
            ok = false;
            break;
          }
          const uint32_t hb = tc::smem_u32(sH + (size_t)(cg & 1) * halo_bytes);
          for (int st = 0; st < SPC; ++st, ++gs) {
            if (!pconv_wait(&w_full[slot], wphase, abort_flag, P.spin)) {
              ok = false;
              break;
            }
            tc::fence_after_sync();
            const uint64_t b0 = bdb + (tc::smem_u32(sW + (size_t)slot * w_bytes) >> 4);
            if (MERGE) {
              const int dxp = st % 3, dyp = st / 3;
              const uint64_t a0 = adb + ((hb + (uint32_t)(dyp * 10 + dxp) * 16) >> 4);
              for (int j = 0; j < njs; ++j) {
                const uint64_t aj = a0 + (uint64_t)j * a_j, bj = b0 + (uint64_t)j * b_j;
                if (c == 0 && st == 0 && j == 0) {
                  // block 1 (dz = 0) initialises every plane, then blocks 0 and 2 accumulate
#pragma unroll
                  for (int sb = 0; sb < 3; ++sb) {
                    const int s = sb == 0 ? 1 : (sb == 1 ? 0 : 2);
#pragma unroll
                    for (int q = 0; q < TZ; ++q)
                      tc::mma_bf16(acc + (uint32_t)((TZ - 1 - q) * CT), aj + (uint64_t)((q + s) * 180),
                                   bj + (uint64_t)(s * CT), id1, s == 1 ? 0u : 1u);
                  }
                } else {
#pragma unroll
                  for (int zz = 0; zz < SZH; ++zz) {
                    const int s_lo = zz - (TZ - 1) > 0 ? zz - (TZ - 1) : 0;
                    const int s_hi = zz < 2 ? zz : 2;
                    const uint32_t id = s_hi - s_lo == 0 ? id1 : (s_hi - s_lo == 1 ? id2 : id3);
                    tc::mma_bf16(acc + (uint32_t)((TZ - 1 - zz + s_lo) * CT), aj + (uint64_t)(zz * 180),
                                 bj + (uint64_t)(s_lo * CT), id, 1u);
                  }
                }
              }
            } else {
              const int dxp = st % 3, dyp = (st / 3) % 3, dzp = st / 9;
              const uint64_t a0 = adb + ((hb + (uint32_t)((dzp * 18 + dyp) * 10 + dxp) * 16) >> 4);
              for (int j = 0; j < njs; ++j) {
                const uint64_t aj = a0 + (uint64_t)j * a_j, bj = b0 + (uint64_t)j * b_j;
                const uint32_t accf = (c > 0 || st > 0 || j > 0) ? 1u : 0u;
#pragma unroll
                for (int q = 0; q < TZ; ++q)
                  tc::mma_bf16(acc + (uint32_t)(q * CT), aj + (uint64_t)(q * 180), bj, id1, accf);
              }
            }
            tc::mma_commit(&w_empty[slot]);
            if (++slot == nsw) {
              slot = 0;
              wphase ^= 1u;
            }
          }
          if (ok) tc::mma_commit(&h_empty[cg & 1]);
        }
        if (ok) tc::mma_commit(&a_full[ab]);
      }
      // every UMMA issued so far has completed before the CTA winds down
      tc::mma_commit(fin);
      if (!tc::mbar_wait(fin, 0u, CONV_DRAIN_SPIN)) ok = false;
      if (!ok) {
        *abort_flag = 1;
        atomicOr(P.status, CONV_TIMEOUT);
      }
    }
    __syncwarp();
  } else if (warp < PCONV_EPI / 32) {
    // ------------------------------------------------------------ epilogue
    const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
    const int r = t;  // accumulator row = output voxel (x0 + r % 8, y0 + r / 8)
    for (int k = 0; k < my_items; ++k) {
      const int ab = k & 1;
      // warp-uniform, so that the warp's tensor-memory loads stay converged
      if (!__all_sync(0xffffffffu, pconv_wait(&a_full[ab], (uint32_t)((k >> 1) & 1), abort_flag, P.spin))) {
        *abort_flag = 1;
        atomicOr(P.status, CONV_TIMEOUT);
        break;
      }
      tc::fence_after_sync();
      int x0, y0, z0, b, n0;
      item_of(k, x0, y0, z0, b, n0);
      const int x = x0 + (r & 7), y = y0 + (r >> 3);
      for (int q = 0; q < TZ; ++q) {
        const long long v = (((long long)b * g.nz + z0 + q) * g.ny + y) * g.nx + x;
        const uint32_t colq = (uint32_t)(ab * TZ * CT + (MERGE ? TZ - 1 - q : q) * CT);
        for (int col = 0; col < CT; col += 32) {
          const bool two = col + 16 < CT;
          uint32_t u[32];
          tc::tmem_ld16_nowait(lane_base + colq + (uint32_t)col, u);
          if (two) tc::tmem_ld16_nowait(lane_base + colq + (uint32_t)col + 16, u + 16);
          tc::tmem_wait_ld();
          const int ng = two ? 2 : 1;
          for (int h = 0; h < ng; ++h) {
            float a[16];
#pragma unroll
            for (int e = 0; e < 16; ++e) {
              const float vv = __uint_as_float(u[16 * h + e]) + sbias[n0 + col + 16 * h + e];
              a[e] = P.relu ? fmaxf(vv, 0.0f) : vv;
            }
            const int c0 = n0 + col + 16 * h;
            if (P.Y) {
              uint4* yp = reinterpret_cast<uint4*>(P.Y + v * P.ldy + c0);
              yp[0] = make_uint4(pack_bf16(a[0], a[1]), pack_bf16(a[2], a[3]), pack_bf16(a[4], a[5]),
                                 pack_bf16(a[6], a[7]));
              yp[1] = make_uint4(pack_bf16(a[8], a[9]), pack_bf16(a[10], a[11]), pack_bf16(a[12], a[13]),
                                 pack_bf16(a[14], a[15]));
            }
            if (P.Yf) {
              float4* fp = reinterpret_cast<float4*>(P.Yf + v * P.ldy + c0);
#pragma unroll
              for (int e = 0; e < 4; ++e) fp[e] = make_float4(a[4 * e], a[4 * e + 1], a[4 * e + 2], a[4 * e + 3]);
            }
          }
        }
      }
      tc::fence_before_sync();
      tc::mbar_arrive(&a_empty[ab]);
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == PCONV_MMA_WARP) tc::tmem_dealloc(tmem, ncols);
}

// ---------------------------------------------------------------------------
// weight gradient, spatially tiled and pipelined (3x3x3 taps)
// ---------------------------------------------------------------------------
// dW[co][t][ci] = sum_v dY[v][co] X[v + off_t][ci], summed over plane blocks
// of 8 (x) x 16 (y) voxels.  One operand, H (CH channels), is staged with a
// one-voxel halo, its planes ordered (channel group, z):
//   piece (plane lp = 3 hg + zz - 16 j, yy, xx) of 8 channels at (lp * 18 + yy) * 10 + xx,
// the other, P (CP channels), for the block alone:
//   piece (pg, y, x) at (pg * 16 + y) * 8 + x.
// Both are MN-major operands (8 channels contiguous, 8 x voxels 16 bytes
// apart).  One UMMA D[M = 128][N = CN] += H(dx, dy) P over K = 16 voxels
// (two y rows) then adds, for one (dx, dy), the three z taps of 16 / 3
// channel groups at once: M row (lp, e) is channel 8 hg + e at dz = zz - 1.
// O1: H = X, P = dY: D row (ci, dz), column co, tap offset +(dx, dy, dz).
// O2: H = dY, P = X: D row (co, dz), column ci, tap offset -(dx, dy, dz)
//     (sum_v dY[v] X[v + off] = sum_u dY[u - off] X[u]).
// A pass is (M block j, group of (dx, dy) taps, slice of P channels); every
// CTA accumulates its pass over its run of blocks in tensor memory and adds
// the result to dW with FP32 atomics once.  Warp roles and bounded waits as
// in the forward kernel; up to four staged blocks are in flight, and a copy
// thread signals a block nst - 2 blocks after issuing it (nst = staged
// slots: two with four, one with three, at once with two), so the slot it
// refills next was handed over earlier.
constexpr int WCONV_HPLANE = 180 * 16;           // bytes of one staged halo plane
constexpr int WCONV_HBYTES = 16 * WCONV_HPLANE;  // the 16 planes of an M block

struct WConvArgs {
  const __nv_bfloat16* H;  // [v][CH]
  const __nv_bfloat16* P;  // [v][CP]
  float* dW;               // [Cout][27][Cin]
  int CH, CP, Cin, o2;
  int CN, TG, ngroups, nchunks, blocks_per_cta, nst;  // nst: staged blocks in flight (2..4)
  ConvGeo g;
  unsigned spin;  // polls of a handshake wait before it gives up
  unsigned* status;
};

__global__ void __launch_bounds__(PCONV_THREADS, 1) k_conv_wgrad_pipe(WConvArgs P) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int t = threadIdx.x;
  const int warp = t >> 5;
  const int CN = P.CN;
  const size_t p_bytes = (size_t)128 * CN * 2, stage_bytes = WCONV_HBYTES + p_bytes;
  const int nst = P.nst;
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + (size_t)nst * stage_bytes);
  uint64_t* full = bar;
  uint64_t* empty = bar + 4;
  uint64_t* done = bar + 8;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar + 9);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  // this CTA's pass and run of blocks
  int pass = blockIdx.y;
  const int nc = pass % P.nchunks;
  pass /= P.nchunks;
  const int grp = pass % P.ngroups;
  const int mj = pass / P.ngroups;
  const int n0 = nc * CN;
  const int ntap = min(P.TG, 9 - grp * P.TG), tap0 = grp * P.TG;
  const ConvGeo& g = P.g;
  const int bxs = g.nx / 8, bys = g.ny / 16;
  const long long nblocks = (long long)bxs * bys * g.nz * g.nb;
  const long long b_begin = (long long)blockIdx.x * P.blocks_per_cta;
  const long long b_end = b_begin + P.blocks_per_cta < nblocks ? b_begin + P.blocks_per_cta : nblocks;
  const int nmine = b_end > b_begin ? (int)(b_end - b_begin) : 0;
  const int nplanes = 3 * (P.CH / 8);  // valid (hg, zz) planes over all M blocks
  uint32_t ncols = 32;
  while ((int)ncols < ntap * CN) ncols <<= 1;

  if (warp == PCONV_MMA_WARP) {
    tc::tmem_alloc(tmem_slot, ncols);
    tc::tmem_relinquish();
  }
  if (t == 0) {
    for (int k = 0; k < 4; ++k) {
      tc::mbar_init(&full[k], PCONV_NPROD);
      tc::mbar_init(&empty[k], 1);
    }
    tc::mbar_init(done, 1);
    *abort_flag = 0;
    tc::fence_mbar_init();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tmem_slot;
  auto block_of = [&](long long bi, int& x0, int& y0, int& z, int& b) {
    x0 = (int)(bi % bxs) * 8;
    bi /= bxs;
    y0 = (int)(bi % bys) * 16;
    bi /= bys;
    z = (int)(bi % g.nz);
    b = (int)(bi / g.nz);
  };

  if (t >= PCONV_PROD0 && t < PCONV_PROD0 + PCONV_NPROD) {
    // ------------------------------------------------------------ copies
    const int pt = t - PCONV_PROD0;
    const int hrow0 = pt / 10, hxx = pt % 10;  // 12 halo rows per pass (120 threads)
    const bool hact = pt < 120;
    // blocks a copy thread keeps in flight before it signals them; the slot it
    // refills next must belong to a block whose UMMAs were already issued
    const int lag = nst >= 3 ? nst - 2 : 0;
    bool ok = true;
    for (int i = 0; i < nmine && ok; ++i) {
      const int s = i % nst;
      if (i >= nst && !pconv_wait(&empty[s], (uint32_t)(((i / nst) - 1) & 1), abort_flag, P.spin)) {
        ok = false;
        break;
      }
      int x0, y0, z, b;
      block_of(b_begin + i, x0, y0, z, b);
      unsigned char* sH = smem + (size_t)s * stage_bytes;
      unsigned char* sP = sH + WCONV_HBYTES;
      if (hact) {
        const int gx = wrap_or_pad(x0 - 1 + hxx, g.nx, g.px);
        for (int row = hrow0; row < 16 * 18; row += 12) {
          const int lp = row / 18, yy = row - 18 * lp;
          const int p = 16 * mj + lp;
          if (p >= nplanes) break;  // rows of planes past the channels feed D rows nobody reads
          const int hg = p / 3, zz = p - 3 * hg;
          const int gy = wrap_or_pad(y0 - 1 + yy, g.ny, g.py);
          const int gz = wrap_or_pad(z - 1 + zz, g.nz, g.pz);
          const bool in = gx >= 0 && gy >= 0 && gz >= 0;
          const long long v = in ? (((long long)b * g.nz + gz) * g.ny + gy) * g.nx + gx : 0;
          tc::cp_async16(sH + (size_t)(row * 10 + hxx) * 16, P.H + v * P.CH + hg * 8, in);
        }
      }
      const long long vrow = (((long long)b * g.nz + z) * g.ny + y0) * g.nx + x0;
      for (int q = pt; q < 128 * (CN / 8); q += PCONV_NPROD) {
        const int x = q & 7, y = (q >> 3) & 15, pg = q >> 7;
        tc::cp_async16(sP + (size_t)q * 16, P.P + (vrow + (long long)y * g.nx + x) * P.CP + n0 + pg * 8, true);
      }
      tc::cp_async_commit();
      if (i >= lag) {
        if (lag == 2) tc::cp_async_wait<2>();
        else if (lag == 1) tc::cp_async_wait<1>();
        else tc::cp_async_wait<0>();
        tc::fence_proxy_async_smem();
        tc::mbar_arrive(&full[(i - lag) % nst]);
      }
    }
    tc::cp_async_wait<0>();
    tc::fence_proxy_async_smem();
    if (ok)
      for (int r = nmine > lag ? nmine - lag : 0; r < nmine; ++r) tc::mbar_arrive(&full[r % nst]);
    if (!ok) {
      *abort_flag = 1;
      atomicOr(P.status, CONV_TIMEOUT);
    }
  } else if (warp == PCONV_MMA_WARP) {
    // ------------------------------------------------------------ UMMA issue
    if ((t & 31) == 0) {
      const uint32_t idesc = tc::idesc_bf16(CONV_M, CN, true, true);
      bool ok = true;
      for (int i = 0; i < nmine; ++i) {
        const int s = i % nst;
        if (!pconv_wait(&full[s], (uint32_t)((i / nst) & 1), abort_flag, P.spin)) {
          ok = false;
          break;
        }
        tc::fence_after_sync();
        const uint32_t h0 = tc::smem_u32(smem + (size_t)s * stage_bytes);
        const uint64_t bd0 = tc::smem_desc_base(128, 2048) + ((h0 + WCONV_HBYTES) >> 4);
        const uint64_t ad0 = tc::smem_desc_base(160, WCONV_HPLANE) + (h0 >> 4);
        for (int tt = 0; tt < ntap; ++tt) {
          const int dxy = tap0 + tt, dxp = dxy % 3, dyp = dxy / 3;
          const uint64_t a0 = ad0 + (uint64_t)(dyp * 10 + dxp);
          const uint32_t d = tmem + (uint32_t)(tt * CN);
#pragma unroll
          for (int k = 0; k < 8; ++k)  // k-step: two rows of 8 voxels (320 and 256 bytes on)
            tc::mma_bf16(d, a0 + (uint64_t)(k * 20), bd0 + (uint64_t)(k * 16), idesc, (i > 0 || k > 0) ? 1u : 0u);
        }
        tc::mma_commit(&empty[s]);
      }
      tc::mma_commit(done);  // every UMMA of this CTA, or none
      // drained here too, so that tensor memory outlives every committed UMMA
      // even when the epilogue's wait gives up
      if (!tc::mbar_wait(done, 0u, CONV_DRAIN_SPIN)) ok = false;
      if (!ok) {
        *abort_flag = 1;
        atomicOr(P.status, CONV_TIMEOUT);
      }
    }
    __syncwarp();
  } else if (warp < PCONV_EPI / 32) {
    // ------------------------------------------------------------ epilogue
    bool ok = __all_sync(0xffffffffu, pconv_wait(done, 0u, abort_flag, P.spin));
    ok = __all_sync(0xffffffffu, ok && *abort_flag == 0);  // no partial sums after a give-up
    tc::fence_after_sync();
    const int m = t;
    const int lp = m >> 3, e = m & 7;
    const int p = 16 * mj + lp;
    const bool valid = ok && nmine > 0 && p < nplanes;
    const int hg = p / 3, zz = p - 3 * hg, hch = hg * 8 + e;
    if (ok && nmine > 0) {
      const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
      for (int tt = 0; tt < ntap; ++tt) {
        const int dxy = tap0 + tt, dxp = dxy % 3, dyp = dxy / 3;
        const int tap = P.o2 ? (2 - dxp) + 3 * (2 - dyp) + 9 * (2 - zz) : dxp + 3 * dyp + 9 * zz;
        for (int col = 0; col < CN; col += 16) {
          float a[16];
          tc::tmem_ld16(lane_base + (uint32_t)(tt * CN + col), a);
          if (valid) {
#pragma unroll
            for (int k = 0; k < 16; ++k) {
              const int pch = n0 + col + k;
              const int co = P.o2 ? hch : pch, ci = P.o2 ? pch : hch;
              atomicAdd(P.dW + ((size_t)co * 27 + tap) * P.Cin + ci, a[k]);
            }
          }
        }
      }
    } else if (!ok && t == 0) {
      *abort_flag = 1;
      atomicOr(P.status, CONV_TIMEOUT);
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == PCONV_MMA_WARP) tc::tmem_dealloc(tmem, ncols);
}

// ---------------------------------------------------------------------------
// weight gradient
// ---------------------------------------------------------------------------
// dW[co][(t,ci)] = sum_v X[v + off_t][ci] dY[v][co] as D[M = 128 (t,ci)
// columns][N = Cout] with K = voxels.  Both operands are MN-major: for one
// voxel, 8 consecutive channels are 16 contiguous bytes.  A CTA owns one block
// of 128 (t,ci) columns (blockIdx.y) and a slice of voxels (blockIdx.x) and
// adds its partial sums to the FP32 output with atomics.
// smem: A[2][128 * 64] | B[2][Cout * 64] (BF16, MN-major core matrices) | mbar[2] | tmem
template <int NT>
__global__ void __launch_bounds__(128, 1)
    k_conv_wgrad(const __nv_bfloat16* __restrict__ dY, int Cout, const __nv_bfloat16* __restrict__ X, int Cin,
                 float* __restrict__ dW, ConvGeo g, long long vox_per_cta, unsigned spin,
                 unsigned* __restrict__ status) {
  extern __shared__ __align__(1024) unsigned char smem[];
  constexpr int KV = 64;  // voxels per stage (the GEMM K)
  const int t = threadIdx.x;
  const int warp = t >> 5;
  const int ntot = NT * Cin;           // all (t,ci) columns
  const int col0 = blockIdx.y * CONV_M;
  const size_t a_bytes = (size_t)CONV_M * KV * 2, b_bytes = (size_t)Cout * KV * 2;
  unsigned char* sA[2] = {smem, smem + a_bytes};
  unsigned char* sB[2] = {smem + 2 * a_bytes, smem + 2 * a_bytes + b_bytes};
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + 2 * a_bytes + 2 * b_bytes);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar + 2);
  uint32_t ncols = 32;
  while ((int)ncols < Cout) ncols <<= 1;

  if (warp == 0) {
    tc::tmem_alloc(tmem_slot, ncols);
    tc::tmem_relinquish();
  }
  if (t == 0) {
    tc::mbar_init(&bar[0], 1);
    tc::mbar_init(&bar[1], 1);
    tc::fence_mbar_init();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tmem_slot;

  const long long nvox = (long long)g.nb * g.nz * g.ny * g.nx;
  const long long v_begin = (long long)blockIdx.x * vox_per_cta;
  const long long v_end = min(nvox, v_begin + vox_per_cta);
  const int nchunks = v_end > v_begin ? (int)((v_end - v_begin + KV - 1) / KV) : 0;
  // core matrix (mn group, k group) at mn * 128 + k * (rows / 8) * 128.  As
  // for the K-major operands, the descriptor's leading byte offset is the
  // stride between core matrices adjacent along K and the stride byte offset
  // the one along M/N.
  const uint32_t a_mn = 128, a_k = (uint32_t)(CONV_M / 8) * 128;
  const uint32_t b_mn = 128, b_k = (uint32_t)(Cout / 8) * 128;
  const uint32_t a_lbo = a_k, a_sbo = a_mn;
  const uint32_t b_lbo = b_k, b_sbo = b_mn;
  const uint32_t idesc = tc::idesc_bf16(CONV_M, Cout, true, true);
  bool ok = true;
  int issued = 0;  // chunks whose UMMAs were issued and committed

  for (int ch = 0; ch < nchunks; ++ch) {
    const int buf = ch & 1;
    if (ch >= 2) {
      bool w = tc::mbar_wait(&bar[buf], (uint32_t)(((ch >> 1) - 1) & 1), spin);
      ok = __syncthreads_and(w);
      if (!ok) break;
    }
    const long long vb = v_begin + (long long)ch * KV;
    // A[(t,ci)][kv] = X[vb + kv + off_t][ci], 8 columns per 16-byte piece
    for (int p = t; p < KV * (CONV_M / 8); p += CONV_M) {
      const int kv = p / (CONV_M / 8), mg = p % (CONV_M / 8);
      const int colg = col0 + mg * 8;
      const long long vv = vb + kv;
      uint4 val = make_uint4(0, 0, 0, 0);
      if (vv < v_end && colg < ntot) {
        const int tap = colg / Cin, ci = colg % Cin;
        long long r = vv;
        const int x = (int)(r % g.nx);
        r /= g.nx;
        const int y = (int)(r % g.ny);
        r /= g.ny;
        const int z = (int)(r % g.nz);
        const int bb = (int)(r / g.nz);
        const int dx = NT == 1 ? 0 : tap % 3 - 1, dy = NT == 1 ? 0 : (tap / 3) % 3 - 1,
                  dz = NT == 1 ? 0 : tap / 9 - 1;
        const long long src = conv_nbr(g, bb, x, y, z, dx, dy, dz);
        if (src >= 0) val = *reinterpret_cast<const uint4*>(X + src * Cin + ci);
      }
      *reinterpret_cast<uint4*>(sA[buf] + (size_t)mg * a_mn + (size_t)(kv >> 3) * a_k + (kv & 7) * 16) = val;
    }
    // B[co][kv] = dY[vb + kv][co]
    for (int p = t; p < KV * (Cout / 8); p += CONV_M) {
      const int kv = p / (Cout / 8), ng = p % (Cout / 8);
      const long long vv = vb + kv;
      uint4 val = make_uint4(0, 0, 0, 0);
      if (vv < v_end) val = *reinterpret_cast<const uint4*>(dY + vv * Cout + ng * 8);
      *reinterpret_cast<uint4*>(sB[buf] + (size_t)ng * b_mn + (size_t)(kv >> 3) * b_k + (kv & 7) * 16) = val;
    }
    tc::fence_proxy_async_smem();
    __syncthreads();
    if (t == 0) {
      tc::fence_after_sync();
      const uint32_t a0 = tc::smem_u32(sA[buf]), b0 = tc::smem_u32(sB[buf]);
      for (int j = 0; j < KV / 16; ++j) {  // K = 16 voxels = two core-matrix groups along K
        const uint64_t ad = tc::smem_desc(a0 + (uint32_t)j * 2 * a_k, a_lbo, a_sbo);
        const uint64_t bd = tc::smem_desc(b0 + (uint32_t)j * 2 * b_k, b_lbo, b_sbo);
        tc::mma_bf16(tmem, ad, bd, idesc, (ch > 0 || j > 0) ? 1u : 0u);
      }
      tc::mma_commit(&bar[buf]);
    }
    issued = ch + 1;
  }
  if (nchunks > 0) {  // every committed UMMA (fixed bound, also after a give-up)
    bool done = true;
    if (issued > 0) {
      const int last = issued - 1;
      done = tc::mbar_wait(&bar[last & 1], (uint32_t)((last >> 1) & 1), CONV_DRAIN_SPIN);
      if (!done) done = tc::mbar_wait(&bar[last & 1], (uint32_t)((last >> 1) & 1), CONV_DRAIN_SPIN);
    }
    ok = __syncthreads_and(ok && done);
  }
  tc::fence_after_sync();
  if (ok && nchunks > 0) {
    const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
    const int col = col0 + t;  // this thread's (t,ci) column
    for (int n0 = 0; n0 < Cout; n0 += 16) {
      float acc[16];
      tc::tmem_ld16(lane_base + (uint32_t)n0, acc);
      if (col < ntot) {
#pragma unroll
        for (int k = 0; k < 16; ++k) atomicAdd(dW + (size_t)(n0 + k) * ntot + col, acc[k]);
      }
    }
  } else if (!ok && t == 0) {
    atomicOr(status, CONV_TIMEOUT);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, ncols);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
// Poll limit of the handshake waits of the next launches (lbnn_set_wait_limit).
static std::atomic<uint32_t> g_wait_limit{LBNN_WAIT_LIMIT_DEFAULT};
static uint32_t wait_limit() { return g_wait_limit.load(std::memory_order_relaxed); }

// Dynamic shared memory of a conv CTA: the staged operands, raised where
// needed so that no more CTAs share an SM than their tensor-memory
// allocations (ncols columns each, 512 per SM) fit side by side; an
// allocation therefore never waits for another CTA's columns.
static size_t conv_smem(size_t need, int cout) {
  int ncols = 32;
  while (ncols < cout) ncols <<= 1;
  int dev = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  const int kmax = 512 / ncols;
  const size_t floor_bytes = (size_t)per_sm / (size_t)(kmax + 1) + 64;  // kmax + 1 CTAs exceed the SM
  return need > floor_bytes ? need : floor_bytes;
}
static size_t conv_fwd_smem(int Cout, int KC) {
  return conv_smem(2 * (size_t)CONV_M * KC * 2 + 2 * (size_t)Cout * KC * 2 + 64, Cout);
}
static size_t conv_wgrad_smem(int Cout) {
  return conv_smem(2 * (size_t)CONV_M * 64 * 2 + 2 * (size_t)Cout * 64 * 2 + 64, Cout);
}

// Shared memory of the pipelined forward kernel: two input blocks, the
// weight ring, barriers, the tensor-memory slot and the abort flag.
constexpr size_t CONV_TILED_SMEM_MAX = 225 * 1024;
static size_t pconv_smem_need(int tz, int KC, int CT, bool merge, int nsw) {
  const size_t halo = (size_t)10 * 18 * (tz + 2) * KC * 2;
  return 2 * halo + (size_t)nsw * (merge ? 3 : 1) * CT * KC * 2 + 256 + 1024;  // + barriers, flags, bias
}

struct PConvCfg {
  int tz = 0, kc = 0, ct = 0, nsw = 0;
  bool merge = false;
  long long items = 0;
};

// Choose the work item and staging of the pipelined forward kernel: enough
// work items for every SM if the grid allows (else the most), then the widest
// channel slice, the deepest z block (fewer halo voxels per output), the
// largest channel chunk and the deepest weight ring that fit shared memory.
static PConvCfg pconv_choose(int cin, int cs, int cout, int nx, int ny, int nz, int nb, int nsm) {
  PConvCfg best;
  auto better = [&](const PConvCfg& a, const PConvCfg& b) {  // a better than b
    if (!b.tz) return true;
    const bool fa = a.items >= nsm, fb = b.items >= nsm;
    if (fa != fb) return fa;
    if (!fa && a.items != b.items) return a.items > b.items;
    if (a.ct != b.ct) return a.ct > b.ct;
    if (a.tz != b.tz) return a.tz > b.tz;
    if (a.kc != b.kc) return a.kc > b.kc;
    return a.nsw > b.nsw;
  };
  const int cts[2] = {cout, cout / 2};
  for (int ci = 0; ci < 2; ++ci) {
    const int ct = cts[ci];
    if (ct < 16 || ct % 16 || cout % ct || (ci == 1 && cout < 128)) continue;
    const bool merge = 3 * ct <= 256;
    for (int tz = 8; tz >= 1; tz >>= 1) {
      if (2 * tz * ct > 512 || nz % tz) continue;
      const int kcs[4] = {64, 48, 32, 16};
      for (int k = 0; k < 4; ++k) {
        const int kc = kcs[k];
        if (kc > cin || cin % kc || cs % kc) continue;
        for (int nsw = PCONV_NSW_MAX; nsw >= PCONV_LAG + 2; --nsw) {
          if (pconv_smem_need(tz, kc, ct, merge, nsw) > CONV_TILED_SMEM_MAX) continue;
          if ((merge ? 3 : 1) * ct * (kc / 8) > PCONV_MAXWP * PCONV_NPROD || 10 * (kc / 8) > PCONV_NPROD) continue;
          PConvCfg c;
          c.tz = tz;
          c.kc = kc;
          c.ct = ct;
          c.nsw = nsw;
          c.merge = merge;
          c.items = (long long)(nx / 8) * (ny / 16) * (nz / tz) * nb * (cout / ct);
          if (better(c, best)) best = c;
          break;
        }
      }
    }
  }
  return best;
}

// Launch of the pipelined forward kernel; channels [cs, cin) of the input
// come from x2 upsampled (nearest x2) when x2 is not null.
static int conv_fwd_pipe(const void* x, int cs, const void* x2, int cin, const void* w, const float* bias, void* y,
                         float* yf, int cout, int ldy, const ConvGeo& g, int relu, unsigned* status, cudaStream_t st) {
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const PConvCfg c = pconv_choose(cin, cs, cout, g.nx, g.ny, g.nz, g.nb, nsm);
  if (!c.tz) return report_error(LB_EINVAL, "conv fwd: no tiled configuration fits shared memory");
  const size_t smem = conv_smem(pconv_smem_need(c.tz, c.kc, c.ct, c.merge, c.nsw), 2 * c.tz * c.ct);
  PConvArgs a{(const __nv_bfloat16*)x, (const __nv_bfloat16*)x2, cs, (const __nv_bfloat16*)w, bias,
              (__nv_bfloat16*)y, yf, cin, cout, ldy, c.kc, c.ct, c.nsw, g, relu, wait_limit(), status};
  cudaError_t e = cudaSuccess;
  auto launch = [&](auto kern) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return;
    int occ = 1;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, PCONV_THREADS, smem);
    if (e != cudaSuccess) return;
    const long long cap = (long long)nsm * (occ > 0 ? occ : 1);
    const unsigned blocks = (unsigned)(c.items < cap ? c.items : cap);
    kern<<<blocks, PCONV_THREADS, smem, st>>>(a);
    e = cudaGetLastError();
  };
  if (c.merge) {
    if (c.tz == 8) launch(k_conv_fwd_pipe<8, true>);
    else if (c.tz == 4) launch(k_conv_fwd_pipe<4, true>);
    else if (c.tz == 2) launch(k_conv_fwd_pipe<2, true>);
    else launch(k_conv_fwd_pipe<1, true>);
  } else {
    if (c.tz == 2) launch(k_conv_fwd_pipe<2, false>);
    else if (c.tz == 1) launch(k_conv_fwd_pipe<1, false>);
    else e = cudaErrorInvalidValue;
  }
  if (e != cudaSuccess) return report_error(LB_ECUDA, std::string("conv fwd (tiled): ") + cudaGetErrorString(e));
  count_launches(1);
  return LB_OK;
}

// Launch of the pipelined weight-gradient kernel: the orientation with fewer
// UMMAs (H = x or H = dy), the P channel slices and the tap groups that fit
// tensor memory, and enough voxel runs for every SM.
static int conv_wgrad_pipe(const void* dy, int cout, const void* x, int cin, float* dw, const ConvGeo& g,
                           unsigned* status, cudaStream_t st) {
  struct Or {
    int o2, CH, CP, mblocks, nchunks, CN, ngroups, TG;
    long long cost;
  };
  auto plan = [](int o2, int CH, int CP) {
    Or o{o2, CH, CP, (3 * (CH / 8) + 15) / 16, 1, CP, 0, 0, 0};
    while (o.CN > 256 || o.CP % o.nchunks || (o.CP / o.nchunks) % 16) {
      ++o.nchunks;
      o.CN = o.CP / o.nchunks;
    }
    o.CN = o.CP / o.nchunks;
    const int fit = 512 / o.CN;  // taps whose accumulators fit tensor memory together
    o.ngroups = (9 + fit - 1) / fit;
    o.TG = (9 + o.ngroups - 1) / o.ngroups;
    o.cost = (long long)o.mblocks * o.nchunks;
    return o;
  };
  const Or a = plan(0, cin, cout), b = plan(1, cout, cin);
  const Or o = b.cost < a.cost ? b : a;
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const long long nblocks = (long long)(g.nx / 8) * (g.ny / 16) * g.nz * g.nb;
  const int npass = o.mblocks * o.ngroups * o.nchunks;
  long long slices = (nsm + npass - 1) / npass;
  if (slices > nblocks) slices = nblocks;
  if (slices < 1) slices = 1;
  const long long per = (nblocks + slices - 1) / slices;
  slices = (nblocks + per - 1) / per;
  if (npass > 65535) return report_error(LB_EINVAL, "conv wgrad: too many passes");
  const size_t stage = (size_t)WCONV_HBYTES + (size_t)128 * o.CN * 2;
  int nst = (int)((CONV_TILED_SMEM_MAX - 128) / stage);
  nst = nst > 4 ? 4 : nst;
  if (nst < 2) return report_error(LB_EINVAL, "conv wgrad: staging does not fit shared memory");
  const size_t smem = conv_smem((size_t)nst * stage + 128, o.TG * o.CN);
  WConvArgs args{(const __nv_bfloat16*)(o.o2 ? dy : x), (const __nv_bfloat16*)(o.o2 ? x : dy), dw, o.CH, o.CP, cin,
                 o.o2, o.CN, o.TG, o.ngroups, o.nchunks, (int)per, nst, g, wait_limit(), status};
  cudaError_t e = cudaFuncSetAttribute(k_conv_wgrad_pipe, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) {
    k_conv_wgrad_pipe<<<dim3((unsigned)slices, (unsigned)npass), PCONV_THREADS, smem, st>>>(args);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return report_error(LB_ECUDA, std::string("conv wgrad (tiled): ") + cudaGetErrorString(e));
  count_launches(1);
  return LB_OK;
}

static int pick_kc(int Cin) {
  if (Cin % 64 == 0) return 64;
  if (Cin % 32 == 0) return 32;
  return 16;
}

}  // namespace lbcg

using namespace lbcg;

extern "C" {

int lbnn_set_wait_limit(uint32_t limit, uint32_t* previous) {
  const uint32_t old = g_wait_limit.exchange(limit);
  if (previous) *previous = old;
  return LB_OK;
}

int lbnn_check_status(unsigned* status, void* stream) {
  if (!status) return report_error(LB_EINVAL, "null pointer");
  cudaStream_t st = (cudaStream_t)stream;
  unsigned word = 0;
  cudaError_t e = cudaMemcpyAsync(&word, status, sizeof(word), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(status, 0, sizeof(word), st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return report_error(LB_ECUDA, std::string("conv status: ") + cudaGetErrorString(e));
  if (word & CONV_TIMEOUT) return report_error(LB_ETIMEOUT, "a convolution gave up a bounded wait");
  return LB_OK;
}

int lbnn_conv3d_fwd(const void* x, int32_t cin, const void* w, int32_t taps, const float* bias, void* y, float* yf,
                    int32_t cout, int32_t ldy, int32_t nx, int32_t ny, int32_t nz, int32_t nb, uint32_t periodic,
                    int32_t relu, unsigned* status, void* stream) {
  if (!x || !w || (!y && !yf) || !status) return report_error(LB_EINVAL, "null pointer");
  if (taps != 1 && taps != 27) return report_error(LB_EINVAL, "taps must be 1 or 27");
  if (cin < 16 || cin % 16 || cin > 1024) return report_error(LB_EINVAL, "cin must be a multiple of 16 in [16, 1024]");
  if (cout < 16 || cout % 16 || cout > 256) return report_error(LB_EINVAL, "cout must be a multiple of 16 in [16, 256]");
  if (nx < 1 || ny < 1 || nz < 1 || nb < 1) return report_error(LB_EINVAL, "extents must be >= 1");
  if (ldy == 0) ldy = cout;
  if (ldy < cout || ldy % 8) return report_error(LB_EINVAL, "ldy must be >= cout and a multiple of 8");
  const long long nvox = (long long)nx * ny * nz * nb;
  if (nvox > (1ll << 31)) return report_error(LB_EINVAL, "too many voxels");
  if (((uintptr_t)x | (uintptr_t)w | (uintptr_t)y | (uintptr_t)yf) & 15)
    return report_error(LB_EINVAL, "tensors must be 16-byte aligned");
  ConvGeo g{nx, ny, nz, nb, (int)(periodic & 1u), (int)((periodic >> 1) & 1u), (int)((periodic >> 2) & 1u)};
  cudaStream_t st = (cudaStream_t)stream;
  if (taps == 27 && nx % 8 == 0 && ny % 16 == 0)
    return conv_fwd_pipe(x, cin, nullptr, cin, w, bias, y, yf, cout, ldy, g, relu, status, st);
  const int KC = pick_kc(cin);
  const size_t smem = conv_fwd_smem(cout, KC);
  const unsigned blocks = (unsigned)((nvox + CONV_M - 1) / CONV_M);
  cudaError_t e;
  if (taps == 27) {
    e = cudaFuncSetAttribute(k_conv_fwd<27>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
      k_conv_fwd<27><<<blocks, CONV_M, smem, st>>>((const __nv_bfloat16*)x, cin, (const __nv_bfloat16*)w, bias,
                                                   (__nv_bfloat16*)y, yf, cout, ldy, KC, g, relu, wait_limit(), status);
  } else {
    e = cudaFuncSetAttribute(k_conv_fwd<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
      k_conv_fwd<1><<<blocks, CONV_M, smem, st>>>((const __nv_bfloat16*)x, cin, (const __nv_bfloat16*)w, bias,
                                                  (__nv_bfloat16*)y, yf, cout, ldy, KC, g, relu, wait_limit(), status);
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return report_error(LB_ECUDA, std::string("conv fwd: ") + cudaGetErrorString(e));
  count_launches(1);
  return LB_OK;
}

int lbnn_conv3d_fwd_upcat(const void* skip, int32_t cs, const void* low, int32_t cl, const void* w, const float* bias,
                          void* y, float* yf, int32_t cout, int32_t ldy, int32_t nx, int32_t ny, int32_t nz, int32_t nb,
                          uint32_t periodic, int32_t relu, unsigned* status, void* stream) {
  if (!skip || !low || !w || (!y && !yf) || !status) return report_error(LB_EINVAL, "null pointer");
  if (cs < 16 || cs % 16 || cl < 16 || cl % 16 || cs + cl > 1024)
    return report_error(LB_EINVAL, "cs, cl must be multiples of 16 with cs + cl <= 1024");
  if (cout < 16 || cout % 16 || cout > 256) return report_error(LB_EINVAL, "cout must be a multiple of 16 in [16, 256]");
  if (nx < 8 || nx % 8 || ny < 16 || ny % 16 || nz < 2 || nz % 2 || nb < 1)
    return report_error(LB_EINVAL, "needs nx % 8 == 0, ny % 16 == 0 and an even nz");
  if (ldy == 0) ldy = cout;
  if (ldy < cout || ldy % 8) return report_error(LB_EINVAL, "ldy must be >= cout and a multiple of 8");
  const long long nvox = (long long)nx * ny * nz * nb;
  if (nvox > (1ll << 31)) return report_error(LB_EINVAL, "too many voxels");
  if (((uintptr_t)skip | (uintptr_t)low | (uintptr_t)w | (uintptr_t)y | (uintptr_t)yf) & 15)
    return report_error(LB_EINVAL, "tensors must be 16-byte aligned");
  ConvGeo g{nx, ny, nz, nb, (int)(periodic & 1u), (int)((periodic >> 1) & 1u), (int)((periodic >> 2) & 1u)};
  return conv_fwd_pipe(skip, cs, low, cs + cl, w, bias, y, yf, cout, ldy, g, relu, status, (cudaStream_t)stream);
}

int lbnn_conv3d_wgrad(const void* dy, int32_t cout, const void* x, int32_t cin, int32_t taps, float* dw, int32_t nx,
                      int32_t ny, int32_t nz, int32_t nb, uint32_t periodic, int32_t vox_per_cta, unsigned* status,
                      void* stream) {
  if (!dy || !x || !dw || !status) return report_error(LB_EINVAL, "null pointer");
  if (taps != 1 && taps != 27) return report_error(LB_EINVAL, "taps must be 1 or 27");
  if (cin < 16 || cin % 16 || cin > 1024) return report_error(LB_EINVAL, "cin must be a multiple of 16 in [16, 1024]");
  if (cout < 16 || cout % 16 || cout > 256) return report_error(LB_EINVAL, "cout must be a multiple of 16 in [16, 256]");
  if (nx < 1 || ny < 1 || nz < 1 || nb < 1) return report_error(LB_EINVAL, "extents must be >= 1");
  if (vox_per_cta < 64 || vox_per_cta % 64) return report_error(LB_EINVAL, "vox_per_cta must be a multiple of 64");
  const long long nvox = (long long)nx * ny * nz * nb;
  if (nvox > (1ll << 31)) return report_error(LB_EINVAL, "too many voxels");
  if (((uintptr_t)x | (uintptr_t)dy) & 15) return report_error(LB_EINVAL, "tensors must be 16-byte aligned");
  ConvGeo g{nx, ny, nz, nb, (int)(periodic & 1u), (int)((periodic >> 1) & 1u), (int)((periodic >> 2) & 1u)};
  if (taps == 27 && nx % 8 == 0 && ny % 16 == 0) return conv_wgrad_pipe(dy, cout, x, cin, dw, g, status, (cudaStream_t)stream);
  const size_t smem = conv_wgrad_smem(cout);
  dim3 grid((unsigned)((nvox + vox_per_cta - 1) / vox_per_cta), (unsigned)((taps * cin + CONV_M - 1) / CONV_M));
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e;
  if (taps == 27) {
    e = cudaFuncSetAttribute(k_conv_wgrad<27>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
      k_conv_wgrad<27><<<grid, 128, smem, st>>>((const __nv_bfloat16*)dy, cout, (const __nv_bfloat16*)x, cin, dw, g,
                                                vox_per_cta, wait_limit(), status);
  } else {
    e = cudaFuncSetAttribute(k_conv_wgrad<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
      k_conv_wgrad<1><<<grid, 128, smem, st>>>((const __nv_bfloat16*)dy, cout, (const __nv_bfloat16*)x, cin, dw, g,
                                               vox_per_cta, wait_limit(), status);
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return report_error(LB_ECUDA, std::string("conv wgrad: ") + cudaGetErrorString(e));
  count_launches(1);
  return LB_OK;
}

}  // extern "C"
