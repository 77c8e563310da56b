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
  const int KC = pick_kc(cin);
  const size_t smem = conv_fwd_smem(cout, KC);
  const unsigned blocks = (unsigned)((nvox + CONV_M - 1) / CONV_M);
  cudaStream_t st = (cudaStream_t)stream;
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
