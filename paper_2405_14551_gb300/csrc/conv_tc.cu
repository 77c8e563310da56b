// 3-D convolutions of the surrogate network on the tcgen05 tensor cores.
//
// Activations are channels-last BF16, X[v][c] with v = x + nx (y + ny (z + nz b)).
// Forward (and, with flipped weights, the input gradient) is an implicit GEMM
//   D[M = voxels][N = Cout] = sum_K A[M][K] B[N][K],  K = taps x Cin,
// A[v][(t,ci)] = X[v + off_t][ci] gathered on the fly, B[co][(t,ci)] = W[co][t][ci].
// The weight gradient is the GEMM
//   dW^T[M = taps x Cin][N = Cout] = sum_v X[v + off_t][ci] dY[v][co]
// with K = voxels; its operands are MN-major (channels contiguous).
// One CTA of 128 threads owns a 128-row accumulator in tensor memory (one
// lane per row, FP32), operands are staged through two shared-memory buffers
// in the no-swizzle core-matrix layout, one thread issues the UMMAs and
// commits them to an mbarrier per buffer.  Every wait is bounded; a wait that
// gives up sets bit 4 of the status word.
#include <cuda_bf16.h>

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
               int KC, ConvGeo g, int relu, unsigned* __restrict__ status) {
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

  for (int ch = 0; ch < nchunks; ++ch) {
    const int buf = ch & 1;
    if (ch >= 2) {  // the UMMAs that read this buffer two chunks ago must be done
      bool w = tc::mbar_wait(&bar[buf], (uint32_t)(((ch >> 1) - 1) & 1), 1u << 22);
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
  }
  // all UMMAs: the last commit covers every earlier one of the issuing thread
  const int last = nchunks - 1;
  bool done = tc::mbar_wait(&bar[last & 1], (uint32_t)((last >> 1) & 1), 1u << 22);
  if (!done) done = tc::mbar_wait(&bar[last & 1], (uint32_t)((last >> 1) & 1), 1u << 22);  // second bounded wait
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
// forward / input gradient, spatially tiled (3x3x3 taps)
// ---------------------------------------------------------------------------
// A CTA owns an output block of 8 (x) x 16 (y) x TZ (z) voxels and all Cout
// channels: TZ accumulators of 128 rows x Cout columns in tensor memory.  Per
// channel chunk of KC channels it stages the input block with a one-voxel halo
// (10 x 18 x (TZ + 2) voxels) once, in the layout
//   piece (cg, zz, yy, xx) of 8 channels at ((cg * SZH + zz) * 18 + yy) * 10 + xx,
// so that for every tap the 128 output rows of one z plane read 16 core
// matrices of 8 consecutive x voxels (128 contiguous bytes) 160 bytes apart:
// the A operand of a tap is the same staged block at a shifted start address,
// and the input is read once per chunk instead of once per tap.  Weights of
// one (chunk, tap) step (Cout x KC) stream through a ring of NS buffers.  All
// 128 threads copy with cp.async (zero fill for padded voxels); one thread
// issues the UMMAs of a step (TZ planes x KC/16) and commits them to the
// step's ring barrier, and after the last tap of a chunk to the halo buffer's
// barrier, before a buffer is refilled.  Every wait is bounded.
constexpr int TCONV_NS = 5;  // weight ring depth
constexpr int TCONV_D = 3;   // steps loaded ahead; the slot refilled was read two steps before

__device__ __forceinline__ int wrap_or_pad(int c, int n, int periodic) {
  if (c >= 0 && c < n) return c;
  if (!periodic) return -1;
  return c < 0 ? c + n : c - n;
}

template <int TZ>
__global__ void __launch_bounds__(128, 1)
    k_conv_fwd_tiled(const __nv_bfloat16* __restrict__ X, int Cin, const __nv_bfloat16* __restrict__ W,
                     const float* __restrict__ bias, __nv_bfloat16* __restrict__ Y, float* __restrict__ Yf, int Cout,
                     int ldy, int KC, ConvGeo g, int relu, unsigned* __restrict__ status) {
  constexpr int SZH = TZ + 2;
  constexpr int HV = 10 * 18 * SZH;  // staged voxels
  extern __shared__ __align__(1024) unsigned char smem[];
  const int t = threadIdx.x;
  const int warp = t >> 5;
  const size_t halo_bytes = (size_t)HV * KC * 2, w_bytes = (size_t)Cout * KC * 2;
  const int nhalo = Cin > KC ? 2 : 1;  // one chunk needs one input buffer
  unsigned char* sH[2] = {smem, smem + (nhalo - 1) * halo_bytes};
  unsigned char* sW = smem + nhalo * halo_bytes;
  uint64_t* bar_w = reinterpret_cast<uint64_t*>(sW + TCONV_NS * w_bytes);
  uint64_t* bar_h = bar_w + TCONV_NS;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar_h + 2);
  uint32_t ncols = 32;
  while ((int)ncols < TZ * Cout) ncols <<= 1;

  if (warp == 0) {
    tc::tmem_alloc(tmem_slot, ncols);
    tc::tmem_relinquish();
  }
  if (t == 0) {
    for (int k = 0; k < TCONV_NS; ++k) tc::mbar_init(&bar_w[k], 1);
    tc::mbar_init(&bar_h[0], 1);
    tc::mbar_init(&bar_h[1], 1);
    tc::fence_mbar_init();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tmem_slot;

  const int bxs = g.nx / 8, bys = g.ny / 16, bzs = g.nz / TZ;
  int blk = blockIdx.x;
  const int x0 = (blk % bxs) * 8;
  blk /= bxs;
  const int y0 = (blk % bys) * 16;
  blk /= bys;
  const int z0 = (blk % bzs) * TZ;
  const int b = blk / bzs;

  const int nchunks = Cin / KC;
  const int nks = nchunks * 27;  // (chunk, tap) steps
  const int cgs = KC / 8;
  const uint32_t a_lbo = (uint32_t)HV * 16, a_sbo = 160;
  const uint32_t b_lbo = (uint32_t)Cout * 16, b_sbo = 128;
  const uint32_t idesc = tc::idesc_bf16(CONV_M, Cout, false, false);

  // issue the copies of step s (weights; the input block too at a chunk's first tap)
  auto load_step = [&](int s) {
    const int c = s / 27, tap = s % 27, c0 = c * KC;
    unsigned char* wdst = sW + (size_t)(s % TCONV_NS) * w_bytes;
    for (int p = t; p < Cout * cgs; p += 128) {
      const int co = p % Cout, kg = p / Cout;
      tc::cp_async16(wdst + ((size_t)kg * Cout + co) * 16, W + ((size_t)co * 27 + tap) * Cin + c0 + kg * 8, true);
    }
    if (tap == 0) {
      unsigned char* hdst = sH[c & 1];
      for (int p = t; p < HV * cgs; p += 128) {
        const int xx = p % 10, r = p / 10;
        const int yy = r % 18, r2 = r / 18;
        const int zz = r2 % SZH, cg = r2 / SZH;
        const int gx = wrap_or_pad(x0 - 1 + xx, g.nx, g.px);
        const int gy = wrap_or_pad(y0 - 1 + yy, g.ny, g.py);
        const int gz = wrap_or_pad(z0 - 1 + zz, g.nz, g.pz);
        const bool ok = gx >= 0 && gy >= 0 && gz >= 0;
        const long long v = ok ? (((long long)b * g.nz + gz) * g.ny + gy) * g.nx + gx : 0;
        tc::cp_async16(hdst + (size_t)p * 16, X + v * Cin + c0 + cg * 8, ok);
      }
    }
  };

  bool ok = true;
  for (int s = 0; s < TCONV_D && s < nks; ++s) {
    load_step(s);
    tc::cp_async_commit();
  }
  for (int s = 0; s < nks; ++s) {
    // refill: step s + D goes into the ring slot of step s + D - NS = s - 2 (and,
    // at a chunk's first tap, into the input buffer of chunk c - 2), so the
    // UMMAs that read it were issued two iterations ago
    const int pf = s + TCONV_D;
    bool wok = true;
    if (pf < nks) {
      if (pf >= TCONV_NS) wok = tc::mbar_wait(&bar_w[pf % TCONV_NS], (uint32_t)(((pf / TCONV_NS) - 1) & 1), 1u << 22);
      const int pc = pf / 27;
      if (wok && pf % 27 == 0 && pc >= 2) wok = tc::mbar_wait(&bar_h[pc & 1], (uint32_t)(((pc / 2) - 1) & 1), 1u << 22);
    }
    ok = __syncthreads_and(ok && wok);
    if (!ok) break;
    if (pf < nks) load_step(pf);
    tc::cp_async_commit();
    tc::cp_async_wait<TCONV_D>();  // step s has landed (this thread's copies)
    tc::fence_proxy_async_smem();
    __syncthreads();
    if (t == 0) {
      tc::fence_after_sync();
      const int c = s / 27, tap = s % 27;
      const int dx = tap % 3, dy = (tap / 3) % 3, dz = tap / 9;  // offsets + 1
      const uint32_t h0 = tc::smem_u32(sH[c & 1]) + (uint32_t)((dz * 18 + dy) * 10 + dx) * 16;
      const uint32_t w0 = tc::smem_u32(sW + (size_t)(s % TCONV_NS) * w_bytes);
      for (int z = 0; z < TZ; ++z) {
        for (int j = 0; j < KC / 16; ++j) {
          const uint64_t ad = tc::smem_desc(h0 + (uint32_t)z * 180 * 16 + (uint32_t)j * 2 * a_lbo, a_lbo, a_sbo);
          const uint64_t bd = tc::smem_desc(w0 + (uint32_t)j * 2 * b_lbo, b_lbo, b_sbo);
          tc::mma_bf16(tmem + (uint32_t)(z * Cout), ad, bd, idesc, (s > 0 || j > 0) ? 1u : 0u);
        }
      }
      tc::mma_commit(&bar_w[s % TCONV_NS]);
      if (tap == 26) tc::mma_commit(&bar_h[c & 1]);
    }
  }
  tc::cp_async_wait<0>();
  // the last commit covers every UMMA issued before it
  const int last = nks - 1;
  bool done = tc::mbar_wait(&bar_w[last % TCONV_NS], (uint32_t)((last / TCONV_NS) & 1), 1u << 22);
  if (!done) done = tc::mbar_wait(&bar_w[last % TCONV_NS], (uint32_t)((last / TCONV_NS) & 1), 1u << 22);
  ok = __syncthreads_and(ok && done);
  tc::fence_after_sync();
  if (ok) {
    const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
    const int x = x0 + (t & 7), y = y0 + (t >> 3);
    for (int z = 0; z < TZ; ++z) {
      const long long v = (((long long)b * g.nz + z0 + z) * g.ny + y) * g.nx + x;
      for (int col = 0; col < Cout; col += 16) {
        float acc[16];
        tc::tmem_ld16(lane_base + (uint32_t)(z * Cout + col), acc);
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
                 float* __restrict__ dW, ConvGeo g, long long vox_per_cta, unsigned* __restrict__ status) {
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

  for (int ch = 0; ch < nchunks; ++ch) {
    const int buf = ch & 1;
    if (ch >= 2) {
      bool w = tc::mbar_wait(&bar[buf], (uint32_t)(((ch >> 1) - 1) & 1), 1u << 22);
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
  }
  if (nchunks > 0) {
    const int last = nchunks - 1;
    bool done = tc::mbar_wait(&bar[last & 1], (uint32_t)((last >> 1) & 1), 1u << 22);
    if (!done) done = tc::mbar_wait(&bar[last & 1], (uint32_t)((last >> 1) & 1), 1u << 22);
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

// Shared memory of the tiled forward kernel: two input blocks, the weight
// ring, barriers and the tensor-memory slot, raised where needed so that the
// CTAs sharing an SM never ask for more than its 512 tensor-memory columns.
constexpr size_t CONV_TILED_SMEM_MAX = 225 * 1024;
static size_t conv_tiled_smem_need(int tz, int Cin, int Cout, int KC) {
  const size_t halo = (size_t)10 * 18 * (tz + 2) * KC * 2;
  const size_t nhalo = Cin > KC ? 2 : 1;
  return nhalo * halo + (size_t)TCONV_NS * Cout * KC * 2 + 8 * (TCONV_NS + 2) + 16;
}
static size_t conv_tiled_smem(int tz, int Cin, int Cout, int KC) {
  return conv_smem(conv_tiled_smem_need(tz, Cin, Cout, KC), Cout * tz);
}

static int pick_kc(int Cin) {
  if (Cin % 64 == 0) return 64;
  if (Cin % 32 == 0) return 32;
  return 16;
}

}  // namespace lbcg

using namespace lbcg;

extern "C" {

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
  if (taps == 27 && nx % 8 == 0 && ny % 16 == 0) {
    // spatially tiled kernel: TZ planes per CTA with TZ x Cout accumulator
    // columns <= 512 and KC input channels per chunk; every (chunk, tap) step
    // has a fixed cost, so take the fitting pair with the most work per step
    // (largest KC x TZ, then the larger TZ)
    int KCt = 0, tz = 0;
    {
      const int cands[7] = {128, 96, 64, 48, 32, 16, 0};
      int best = 0;
      for (int k = 0; cands[k]; ++k) {
        const int kc = cands[k];
        if (kc > cin || cin % kc) continue;
        for (int t = 4; t >= 1; t >>= 1) {
          if (t * cout > 512 || nz % t) continue;
          if (conv_tiled_smem_need(t, cin, cout, kc) > CONV_TILED_SMEM_MAX) continue;
          if (kc * t > best) {
            best = kc * t;
            KCt = kc;
            tz = t;
          }
        }
      }
    }
    if (!KCt) return report_error(LB_EINVAL, "conv fwd: no tiled configuration fits shared memory");
    const size_t smem = conv_tiled_smem(tz, cin, cout, KCt);
    cudaError_t e = cudaSuccess;
    auto launch = [&](auto kern) {
      e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return;
      const unsigned blocks = (unsigned)((nx / 8) * (ny / 16) * (nz / tz) * nb);
      kern<<<blocks, CONV_M, smem, st>>>((const __nv_bfloat16*)x, cin, (const __nv_bfloat16*)w, bias,
                                         (__nv_bfloat16*)y, yf, cout, ldy, KCt, g, relu, status);
      e = cudaGetLastError();
    };
    if (tz == 4) launch(k_conv_fwd_tiled<4>);
    else if (tz == 2) launch(k_conv_fwd_tiled<2>);
    else launch(k_conv_fwd_tiled<1>);
    if (e != cudaSuccess) return report_error(LB_ECUDA, std::string("conv fwd (tiled): ") + cudaGetErrorString(e));
    count_launches(1);
    return LB_OK;
  }
  const int KC = pick_kc(cin);
  const size_t smem = conv_fwd_smem(cout, KC);
  const unsigned blocks = (unsigned)((nvox + CONV_M - 1) / CONV_M);
  cudaError_t e;
  if (taps == 27) {
    e = cudaFuncSetAttribute(k_conv_fwd<27>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
      k_conv_fwd<27><<<blocks, CONV_M, smem, st>>>((const __nv_bfloat16*)x, cin, (const __nv_bfloat16*)w, bias,
                                                   (__nv_bfloat16*)y, yf, cout, ldy, KC, g, relu, status);
  } else {
    e = cudaFuncSetAttribute(k_conv_fwd<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
      k_conv_fwd<1><<<blocks, CONV_M, smem, st>>>((const __nv_bfloat16*)x, cin, (const __nv_bfloat16*)w, bias,
                                                  (__nv_bfloat16*)y, yf, cout, ldy, KC, g, relu, status);
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return report_error(LB_ECUDA, std::string("conv fwd: ") + cudaGetErrorString(e));
  count_launches(1);
  return LB_OK;
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
  const size_t smem = conv_wgrad_smem(cout);
  dim3 grid((unsigned)((nvox + vox_per_cta - 1) / vox_per_cta), (unsigned)((taps * cin + CONV_M - 1) / CONV_M));
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e;
  if (taps == 27) {
    e = cudaFuncSetAttribute(k_conv_wgrad<27>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
      k_conv_wgrad<27><<<grid, 128, smem, st>>>((const __nv_bfloat16*)dy, cout, (const __nv_bfloat16*)x, cin, dw, g,
                                                vox_per_cta, status);
  } else {
    e = cudaFuncSetAttribute(k_conv_wgrad<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
      k_conv_wgrad<1><<<grid, 128, smem, st>>>((const __nv_bfloat16*)dy, cout, (const __nv_bfloat16*)x, cin, dw, g,
                                               vox_per_cta, status);
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return report_error(LB_ECUDA, std::string("conv wgrad: ") + cudaGetErrorString(e));
  count_launches(1);
  return LB_OK;
}

}  // extern "C"
