// Element-wise and data-movement kernels of the surrogate network (channels-
// last BF16 activations, FP32 gradients, FP32 master weights).  The
// convolutions themselves live in conv_tc.cu.
#include <cuda_bf16.h>

#include <string>

#include "../../include/lbcg.h"
#include "../../include/lbnn.h"
#include "internal.h"

namespace lbcg {

using bf16 = __nv_bfloat16;

__device__ __forceinline__ long long grid_stride_begin() { return (long long)blockIdx.x * blockDim.x + threadIdx.x; }
__device__ __forceinline__ long long grid_stride() { return (long long)gridDim.x * blockDim.x; }

static unsigned blocks_for(long long n) {
  long long b = (n + 255) / 256;
  return (unsigned)(b < 8192 ? (b < 1 ? 1 : b) : 8192);
}

// fields [5][N] (phi, rho, ux, uy, uz; FP32) -> x[N][C] BF16 with
// (phi, s_rho (rho - 1), s_u ux, s_u uy, s_u uz, 0, ...)
__global__ void k_pack_input(long long N, const float* __restrict__ f, int C, float s_rho, float s_u,
                             bf16* __restrict__ x) {
  for (long long v = grid_stride_begin(); v < N; v += grid_stride()) {
    const float vals[5] = {f[v], s_rho * (f[N + v] - 1.0f), s_u * f[2 * N + v], s_u * f[3 * N + v],
                           s_u * f[4 * N + v]};
    for (int c = 0; c < C; ++c) x[v * C + c] = __float2bfloat16(c < 5 ? vals[c] : 0.0f);
  }
}

// network output y[N][C] (FP32, first 5 channels = scaled increments) added to
// the input fields: out[5][N] = fields + (dphi, drho/s_rho, du/s_u); phi is
// clamped to [-1, 1], rho kept above rho_min.
__global__ void k_unpack_output(long long N, const float* __restrict__ f, const float* __restrict__ y, int C,
                                float s_rho, float s_u, float rho_min, float* __restrict__ out) {
  for (long long v = grid_stride_begin(); v < N; v += grid_stride()) {
    const float* yy = y + v * C;
    out[v] = fminf(1.0f, fmaxf(-1.0f, f[v] + yy[0]));
    out[N + v] = fmaxf(rho_min, f[N + v] + yy[1] / s_rho);
    out[2 * N + v] = f[2 * N + v] + yy[2] / s_u;
    out[3 * N + v] = f[3 * N + v] + yy[3] / s_u;
    out[4 * N + v] = f[4 * N + v] + yy[4] / s_u;
  }
}

// training target t[N][C] (FP32): scaled increments between two field sets
__global__ void k_pack_target(long long N, const float* __restrict__ f0, const float* __restrict__ f1, int C,
                              float s_rho, float s_u, float* __restrict__ t) {
  for (long long v = grid_stride_begin(); v < N; v += grid_stride()) {
    const float d[5] = {f1[v] - f0[v], s_rho * (f1[N + v] - f0[N + v]), s_u * (f1[2 * N + v] - f0[2 * N + v]),
                        s_u * (f1[3 * N + v] - f0[3 * N + v]), s_u * (f1[4 * N + v] - f0[4 * N + v])};
    for (int c = 0; c < C; ++c) t[v * C + c] = c < 5 ? d[c] : 0.0f;
  }
}

// 2x2x2 average pooling, channels last; output extents (nx/2, ny/2, nz/2)
__global__ void k_avgpool2(const bf16* __restrict__ x, int C, int nx, int ny, int nz, int nb, bf16* __restrict__ y) {
  const int ox = nx / 2, oy = ny / 2, oz = nz / 2;
  const long long n = (long long)nb * oz * oy * ox * C;
  for (long long e = grid_stride_begin(); e < n; e += grid_stride()) {
    const int c = (int)(e % C);
    long long r = e / C;
    const int x0 = (int)(r % ox) * 2;
    r /= ox;
    const int y0 = (int)(r % oy) * 2;
    r /= oy;
    const int z0 = (int)(r % oz) * 2;
    const int b = (int)(r / oz);
    float s = 0.0f;
    for (int dz = 0; dz < 2; ++dz)
      for (int dy = 0; dy < 2; ++dy)
        for (int dx = 0; dx < 2; ++dx)
          s += __bfloat162float(x[((((long long)b * nz + z0 + dz) * ny + y0 + dy) * nx + x0 + dx) * C + c]);
    y[e] = __float2bfloat16(0.125f * s);
  }
}

// The same pooling eight channels (16 bytes) at a time, for C % 8 == 0; the
// sum runs in the same order, so the results are identical.
__device__ __forceinline__ void bf16x8_to_f32(const uint4& v, float f[8]) {
  const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&v);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float2 t = __bfloat1622float2(h[k]);
    f[2 * k] = t.x;
    f[2 * k + 1] = t.y;
  }
}
__global__ void k_avgpool2_v8(const bf16* __restrict__ x, int C, int nx, int ny, int nz, int nb,
                              bf16* __restrict__ y) {
  const int ox = nx / 2, oy = ny / 2, oz = nz / 2, G = C / 8;
  const long long n = (long long)nb * oz * oy * ox * G;
  for (long long e = grid_stride_begin(); e < n; e += grid_stride()) {
    const int g = (int)(e % G);
    long long r = e / G;
    const int x0 = (int)(r % ox) * 2;
    r /= ox;
    const int y0 = (int)(r % oy) * 2;
    r /= oy;
    const int z0 = (int)(r % oz) * 2;
    const int b = (int)(r / oz);
    float s[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int dz = 0; dz < 2; ++dz)
      for (int dy = 0; dy < 2; ++dy)
        for (int dx = 0; dx < 2; ++dx) {
          const uint4 v = *reinterpret_cast<const uint4*>(
              x + ((((long long)b * nz + z0 + dz) * ny + y0 + dy) * nx + x0 + dx) * C + g * 8);
          float f[8];
          bf16x8_to_f32(v, f);
#pragma unroll
          for (int k = 0; k < 8; ++k) s[k] += f[k];
        }
    __align__(16) bf16 o[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) o[k] = __float2bfloat16(0.125f * s[k]);
    *reinterpret_cast<uint4*>(y + e * 8) = *reinterpret_cast<const uint4*>(o);
  }
}

// gradient of the pooling: dx[child] += dy[parent] / 8 (FP32, accumulate)
__global__ void k_avgpool2_bwd(const float* __restrict__ dy, int C, int nx, int ny, int nz, int nb,
                               float* __restrict__ dx) {
  const long long n = (long long)nb * nz * ny * nx * C;
  const int ox = nx / 2, oy = ny / 2, oz = nz / 2;
  for (long long e = grid_stride_begin(); e < n; e += grid_stride()) {
    const int c = (int)(e % C);
    long long r = e / C;
    const int x = (int)(r % nx);
    r /= nx;
    const int y = (int)(r % ny);
    r /= ny;
    const int z = (int)(r % nz);
    const int b = (int)(r / nz);
    dx[e] += 0.125f * dy[((((long long)b * oz + z / 2) * oy + y / 2) * ox + x / 2) * C + c];
  }
}

// The same copy eight channels (16 bytes) at a time, for Cs % 8 == Cl % 8 == 0.
__global__ void k_up_concat_v8(const bf16* __restrict__ skip, int Cs, const bf16* __restrict__ low, int Cl, int nx,
                               int ny, int nz, int nb, bf16* __restrict__ out) {
  const int Gs = Cs / 8, G = (Cs + Cl) / 8;
  const long long n = (long long)nb * nz * ny * nx * G;
  const int ox = nx / 2, oy = ny / 2, oz = nz / 2;
  for (long long e = grid_stride_begin(); e < n; e += grid_stride()) {
    const int g = (int)(e % G);
    const long long v = e / G;
    uint4 val;
    if (g < Gs) {
      val = *reinterpret_cast<const uint4*>(skip + v * Cs + g * 8);
    } else {
      long long r = v;
      const int x = (int)(r % nx);
      r /= nx;
      const int y = (int)(r % ny);
      r /= ny;
      const int z = (int)(r % nz);
      const int b = (int)(r / nz);
      val = *reinterpret_cast<const uint4*>(low + ((((long long)b * oz + z / 2) * oy + y / 2) * ox + x / 2) * Cl +
                                            (g - Gs) * 8);
    }
    *reinterpret_cast<uint4*>(out + e * 8) = val;
  }
}

// out[v][0:Cs) = skip[v], out[v][Cs:Cs+Cl) = low[parent(v)] (nearest x2)
__global__ void k_up_concat(const bf16* __restrict__ skip, int Cs, const bf16* __restrict__ low, int Cl, int nx,
                            int ny, int nz, int nb, bf16* __restrict__ out) {
  const int C = Cs + Cl;
  const long long n = (long long)nb * nz * ny * nx * C;
  const int ox = nx / 2, oy = ny / 2, oz = nz / 2;
  for (long long e = grid_stride_begin(); e < n; e += grid_stride()) {
    const int c = (int)(e % C);
    const long long v = e / C;
    if (c < Cs) {
      out[e] = skip[v * Cs + c];
    } else {
      long long r = v;
      const int x = (int)(r % nx);
      r /= nx;
      const int y = (int)(r % ny);
      r /= ny;
      const int z = (int)(r % nz);
      const int b = (int)(r / nz);
      out[e] = low[((((long long)b * oz + z / 2) * oy + y / 2) * ox + x / 2) * Cl + (c - Cs)];
    }
  }
}

// gradient of up_concat: dskip[v] += dout[v][0:Cs), dlow[parent] += sum over 8 children
__global__ void k_up_concat_bwd(const float* __restrict__ dout, int Cs, int Cl, int nx, int ny, int nz, int nb,
                                float* __restrict__ dskip, float* __restrict__ dlow) {
  const int C = Cs + Cl;
  const int ox = nx / 2, oy = ny / 2, oz = nz / 2;
  // one thread per (parent voxel, low channel): sum of the 8 children
  const long long nl = (long long)nb * oz * oy * ox * Cl;
  for (long long e = grid_stride_begin(); e < nl; e += grid_stride()) {
    const int c = (int)(e % Cl);
    long long r = e / Cl;
    const int px = (int)(r % ox);
    r /= ox;
    const int py = (int)(r % oy);
    r /= oy;
    const int pz = (int)(r % oz);
    const int b = (int)(r / oz);
    float s = 0.0f;
    for (int dz = 0; dz < 2; ++dz)
      for (int dy = 0; dy < 2; ++dy)
        for (int dx = 0; dx < 2; ++dx) {
          const long long v = (((long long)b * nz + 2 * pz + dz) * ny + 2 * py + dy) * nx + 2 * px + dx;
          s += dout[v * C + Cs + c];
        }
    dlow[e] += s;
  }
  const long long ns = (long long)nb * nz * ny * nx * Cs;
  for (long long e = grid_stride_begin(); e < ns; e += grid_stride()) {
    const int c = (int)(e % Cs);
    const long long v = e / Cs;
    dskip[e] += dout[v * C + c];
  }
}

// g_pre = g_post * (y > 0) (ReLU), as BF16 operand plus optional FP32 copy
__global__ void k_relu_bwd(long long n, const float* __restrict__ g, const bf16* __restrict__ y, int relu,
                           bf16* __restrict__ gb, float* __restrict__ gf) {
  for (long long e = grid_stride_begin(); e < n; e += grid_stride()) {
    float v = g[e];
    if (relu && !(__bfloat162float(y[e]) > 0.0f)) v = 0.0f;
    if (gb) gb[e] = __float2bfloat16(v);
    if (gf) gf[e] = v;
  }
}

// db[c] += sum_v g[v][c]
__global__ void __launch_bounds__(256) k_bias_grad(long long nvox, int C, const float* __restrict__ g,
                                                   float* __restrict__ db) {
  // thread layout: 256 threads = (256 / C) voxel lanes x C channels (C <= 256, power-of-two friendly)
  const int lanes = 256 / C;
  const int c = threadIdx.x % C, lane = threadIdx.x / C;
  if (lane >= lanes) return;
  float s = 0.0f;
  for (long long v = (long long)blockIdx.x * lanes + lane; v < nvox; v += (long long)gridDim.x * lanes) s += g[v * C + c];
  atomicAdd(db + c, s);
}

// dgrad weights: wt[ci][t][co] = w[co][taps-1-t][ci]
__global__ void k_flip_weights(const bf16* __restrict__ w, int cout, int taps, int cin, bf16* __restrict__ wt) {
  const long long n = (long long)cout * taps * cin;
  for (long long e = grid_stride_begin(); e < n; e += grid_stride()) {
    const int ci = (int)(e % cin);
    long long r = e / cin;
    const int t = (int)(r % taps);
    const int co = (int)(r / taps);
    wt[((long long)ci * taps + (taps - 1 - t)) * cout + co] = w[e];
  }
}

// MSE over the first nch channels of [N][C]: grad = 2 (p - t) w_c / count; loss sums in FP64
__global__ void __launch_bounds__(256) k_mse(long long N, int C, int nch, const float* __restrict__ p,
                                             const float* __restrict__ t, const float* __restrict__ wch,
                                             float inv_count, float* __restrict__ grad, double* __restrict__ loss) {
  __shared__ double red[256];
  double s = 0.0;
  for (long long e = grid_stride_begin(); e < N * C; e += grid_stride()) {
    const int c = (int)(e % C);
    float gv = 0.0f;
    if (c < nch) {
      const float d = p[e] - t[e];
      s += (double)wch[c] * d * d;
      gv = 2.0f * wch[c] * d * inv_count;
    }
    grad[e] = gv;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(loss, red[0] * inv_count);
}

// Adam on FP32 master weights, BF16 copy for the kernels (bf may be null)
__global__ void k_adam(long long n, float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2, float wd,
                       bf16* __restrict__ bf) {
  for (long long e = grid_stride_begin(); e < n; e += grid_stride()) {
    const float gg = g[e] + wd * p[e];
    const float mm = b1 * m[e] + (1.0f - b1) * gg;
    const float vv = b2 * v[e] + (1.0f - b2) * gg * gg;
    m[e] = mm;
    v[e] = vv;
    const float pe = p[e] - lr * (mm * c1) / (sqrtf(vv * c2) + eps);
    p[e] = pe;
    if (bf) bf[e] = __float2bfloat16(pe);
  }
}

__global__ void k_f32_to_bf16(long long n, const float* __restrict__ a, bf16* __restrict__ b) {
  for (long long e = grid_stride_begin(); e < n; e += grid_stride()) b[e] = __float2bfloat16(a[e]);
}

}  // namespace lbcg

using namespace lbcg;

namespace {
int launch_result(const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return report_error(LB_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
  count_launches(1);
  return LB_OK;
}
}  // namespace

extern "C" {

int lbnn_pack_input(const float* fields, int64_t n, int32_t c, float s_rho, float s_u, void* x, void* stream) {
  if (!fields || !x || n < 1 || c < 5) return report_error(LB_EINVAL, "pack_input arguments");
  k_pack_input<<<blocks_for(n), 256, 0, (cudaStream_t)stream>>>(n, fields, c, s_rho, s_u, (bf16*)x);
  return launch_result("pack_input");
}

int lbnn_unpack_output(const float* fields, const float* y, int64_t n, int32_t c, float s_rho, float s_u,
                       float rho_min, float* out, void* stream) {
  if (!fields || !y || !out || n < 1 || c < 5) return report_error(LB_EINVAL, "unpack_output arguments");
  k_unpack_output<<<blocks_for(n), 256, 0, (cudaStream_t)stream>>>(n, fields, y, c, s_rho, s_u, rho_min, out);
  return launch_result("unpack_output");
}

int lbnn_pack_target(const float* f0, const float* f1, int64_t n, int32_t c, float s_rho, float s_u, float* t,
                     void* stream) {
  if (!f0 || !f1 || !t || n < 1 || c < 5) return report_error(LB_EINVAL, "pack_target arguments");
  k_pack_target<<<blocks_for(n), 256, 0, (cudaStream_t)stream>>>(n, f0, f1, c, s_rho, s_u, t);
  return launch_result("pack_target");
}

int lbnn_avgpool2(const void* x, int32_t c, int32_t nx, int32_t ny, int32_t nz, int32_t nb, void* y, void* stream) {
  if (!x || !y || c < 1 || nx % 2 || ny % 2 || nz % 2 || nx < 2 || ny < 2 || nz < 2 || nb < 1)
    return report_error(LB_EINVAL, "avgpool2 needs even extents");
  if (c % 8 == 0 && !(((uintptr_t)x | (uintptr_t)y) & 15))
    k_avgpool2_v8<<<blocks_for((long long)nb * nz * ny * nx * c / 64), 256, 0, (cudaStream_t)stream>>>(
        (const bf16*)x, c, nx, ny, nz, nb, (bf16*)y);
  else
    k_avgpool2<<<blocks_for((long long)nb * nz * ny * nx * c / 8), 256, 0, (cudaStream_t)stream>>>(
        (const bf16*)x, c, nx, ny, nz, nb, (bf16*)y);
  return launch_result("avgpool2");
}

int lbnn_avgpool2_bwd(const float* dy, int32_t c, int32_t nx, int32_t ny, int32_t nz, int32_t nb, float* dx,
                      void* stream) {
  if (!dy || !dx || c < 1 || nx % 2 || ny % 2 || nz % 2 || nb < 1) return report_error(LB_EINVAL, "avgpool2_bwd");
  k_avgpool2_bwd<<<blocks_for((long long)nb * nz * ny * nx * c), 256, 0, (cudaStream_t)stream>>>(dy, c, nx, ny, nz,
                                                                                                 nb, dx);
  return launch_result("avgpool2_bwd");
}

int lbnn_up_concat(const void* skip, int32_t cs, const void* low, int32_t cl, int32_t nx, int32_t ny, int32_t nz,
                   int32_t nb, void* out, void* stream) {
  if (!skip || !low || !out || cs < 1 || cl < 1 || nx % 2 || ny % 2 || nz % 2 || nb < 1)
    return report_error(LB_EINVAL, "up_concat arguments");
  if (cs % 8 == 0 && cl % 8 == 0 && !(((uintptr_t)skip | (uintptr_t)low | (uintptr_t)out) & 15))
    k_up_concat_v8<<<blocks_for((long long)nb * nz * ny * nx * (cs + cl) / 8), 256, 0, (cudaStream_t)stream>>>(
        (const bf16*)skip, cs, (const bf16*)low, cl, nx, ny, nz, nb, (bf16*)out);
  else
    k_up_concat<<<blocks_for((long long)nb * nz * ny * nx * (cs + cl)), 256, 0, (cudaStream_t)stream>>>(
        (const bf16*)skip, cs, (const bf16*)low, cl, nx, ny, nz, nb, (bf16*)out);
  return launch_result("up_concat");
}

int lbnn_up_concat_bwd(const float* dout, int32_t cs, int32_t cl, int32_t nx, int32_t ny, int32_t nz, int32_t nb,
                       float* dskip, float* dlow, void* stream) {
  if (!dout || !dskip || !dlow || cs < 1 || cl < 1 || nx % 2 || ny % 2 || nz % 2 || nb < 1)
    return report_error(LB_EINVAL, "up_concat_bwd arguments");
  k_up_concat_bwd<<<blocks_for((long long)nb * nz * ny * nx * (cs + cl)), 256, 0, (cudaStream_t)stream>>>(
      dout, cs, cl, nx, ny, nz, nb, dskip, dlow);
  return launch_result("up_concat_bwd");
}

int lbnn_relu_bwd(const float* g, const void* y, int64_t n, int32_t relu, void* gb, float* gf, void* stream) {
  if (!g || n < 1 || (relu && !y) || (!gb && !gf)) return report_error(LB_EINVAL, "relu_bwd arguments");
  k_relu_bwd<<<blocks_for(n), 256, 0, (cudaStream_t)stream>>>(n, g, (const bf16*)y, relu, (bf16*)gb, gf);
  return launch_result("relu_bwd");
}

int lbnn_bias_grad(const float* g, int64_t nvox, int32_t c, float* db, void* stream) {
  if (!g || !db || nvox < 1 || c < 1 || c > 256 || 256 % c) return report_error(LB_EINVAL, "bias_grad arguments");
  k_bias_grad<<<512, 256, 0, (cudaStream_t)stream>>>(nvox, c, g, db);
  return launch_result("bias_grad");
}

int lbnn_flip_weights(const void* w, int32_t cout, int32_t taps, int32_t cin, void* wt, void* stream) {
  if (!w || !wt || cout < 1 || cin < 1 || (taps != 1 && taps != 27)) return report_error(LB_EINVAL, "flip_weights");
  k_flip_weights<<<blocks_for((long long)cout * taps * cin), 256, 0, (cudaStream_t)stream>>>((const bf16*)w, cout, taps,
                                                                                             cin, (bf16*)wt);
  return launch_result("flip_weights");
}

int lbnn_mse(const float* p, const float* t, int64_t n, int32_t c, int32_t nch, const float* wch, float* grad,
             double* loss, void* stream) {
  if (!p || !t || !wch || !grad || !loss || n < 1 || nch < 1 || nch > c) return report_error(LB_EINVAL, "mse");
  k_mse<<<blocks_for(n * c), 256, 0, (cudaStream_t)stream>>>(n, c, nch, p, t, wch, 1.0f / (float)(n * nch), grad,
                                                             loss);
  return launch_result("mse");
}

int lbnn_adam(float* p, const float* g, float* m, float* v, int64_t n, float lr, float b1, float b2, float eps,
              int32_t step, float wd, void* bf, void* stream) {
  if (!p || !g || !m || !v || n < 1 || step < 1) return report_error(LB_EINVAL, "adam arguments");
  const float c1 = 1.0f / (1.0f - powf(b1, (float)step)), c2 = 1.0f / (1.0f - powf(b2, (float)step));
  k_adam<<<blocks_for(n), 256, 0, (cudaStream_t)stream>>>(n, p, g, m, v, lr, b1, b2, eps, c1, c2, wd, (bf16*)bf);
  return launch_result("adam");
}

int lbnn_f32_to_bf16(const float* a, int64_t n, void* b, void* stream) {
  if (!a || !b || n < 1) return report_error(LB_EINVAL, "f32_to_bf16 arguments");
  k_f32_to_bf16<<<blocks_for(n), 256, 0, (cudaStream_t)stream>>>(n, a, (bf16*)b);
  return launch_result("f32_to_bf16");
}

}  // extern "C"
