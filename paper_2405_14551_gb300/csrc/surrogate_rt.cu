// Native surrogate runtime: the trained U-Net of a handle (weights loaded from
// a file) and one surrogate jump of K steps on the handle's state, built from
// the library's own kernels (include/lbnn.h) and C ABI calls.
//
// A jump: fields (phi, rho, u) of the current state -> network input ->
// U-Net forward (tcgen05 convolutions) -> candidate fields (the increments
// added, phi clamped, rho floored) -> drift monitors (droplet count and
// dispersed volume of the candidate against the current state) -> optional
// judgement by the plain LB (K steps on a second handle from the exact same
// state, mean |phi_candidate - phi_LB|) -> acceptance (regularised
// reconstruction of the candidate, Sec. IV.C) or the LB result.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/lbcg.h"
#include "../../include/lbnn.h"
#include "internal.h"

namespace lbcg {

constexpr uint32_t UNET_MAGIC = 0x4e4e424cu;  // "LBNN"
constexpr int32_t UNET_VERSION = 1;
constexpr int UNET_LAYERS = 15;
constexpr int RED_T = 256;
constexpr int RED_B = 1024;

struct UnetLayer {
  int ci, co, taps, relu;
  __nv_bfloat16* w;  // [co][taps][ci]
  float* b;          // [co]
};

struct SurrogateState {
  int base = 0, cin = 0, cout = 0;
  float s_rho = 0.f, s_u = 0.f;
  uint32_t periodic = 0;
  std::vector<UnetLayer> layers;  // c1a c1b c2a c2b c3a c3b c4a c4b c5a c5b c6a c6b c7a c7b head
  float* fields = nullptr;        // [5][N] current phi, rho, ux, uy, uz
  float* cand = nullptr;          // [5][N] candidate
  float* judge_phi = nullptr;     // [N]
  __nv_bfloat16* x = nullptr;     // [N][cin]
  std::vector<__nv_bfloat16*> act;  // per convolution output
  __nv_bfloat16 *p1 = nullptr, *p2 = nullptr, *p3 = nullptr, *u1 = nullptr, *u2 = nullptr, *u3 = nullptr;
  float* head = nullptr;          // [N][cout]
  unsigned* status = nullptr;
  double* partials = nullptr;     // RED_B + 1 doubles
};

void destroy_surrogate(SurrogateState* s) { delete s; }  // device buffers belong to the handle

// mean |a - b| over the fluid nodes: FP64 block partials in a fixed
// partition and a fixed tree order, then one block over the partials
__global__ void __launch_bounds__(RED_T) k_absdiff_partial(Geo g, const float* __restrict__ a,
                                                           const float* __restrict__ b, double* partials) {
  __shared__ double s[RED_T];
  const long long chunk = (g.N + gridDim.x - 1) / gridDim.x;
  const long long beg = (long long)blockIdx.x * chunk;
  const long long end = beg + chunk < g.N ? beg + chunk : g.N;
  double v = 0.0;
  for (long long i = beg + threadIdx.x; i < end; i += RED_T) v += fabs((double)a[i] - (double)b[i]);
  s[threadIdx.x] = v;
  __syncthreads();
  for (int w = RED_T / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) partials[blockIdx.x] = s[0];
}

__global__ void __launch_bounds__(RED_T) k_sum_partials(int nb, const double* __restrict__ partials, double* out) {
  __shared__ double s[RED_T];
  double v = 0.0;
  for (int i = threadIdx.x; i < nb; i += RED_T) v += partials[i];
  s[threadIdx.x] = v;
  __syncthreads();
  for (int w = RED_T / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = s[0];
}

namespace {

int fail(int code, const std::string& msg) { return report_error(code, msg); }

// (ci, co, taps, relu) of every convolution, in forward order
std::vector<std::vector<int>> unet_table(int base, int cin, int cout) {
  const int c1 = base, c2 = 2 * base, c3 = 4 * base, c4 = 8 * base;
  return {{cin, c1, 27, 1}, {c1, c1, 27, 1}, {c1, c2, 27, 1}, {c2, c2, 27, 1}, {c2, c3, 27, 1},
          {c3, c3, 27, 1},  {c3, c4, 27, 1}, {c4, c4, 27, 1}, {c3 + c4, c3, 27, 1}, {c3, c3, 27, 1},
          {c2 + c3, c2, 27, 1}, {c2, c2, 27, 1}, {c1 + c2, c1, 27, 1}, {c1, c1, 27, 1}, {c1, cout, 1, 0}};
}

int conv(SurrogateState* S, int li, const void* in, void* out_bf, float* out_f, int nx, int ny, int nz,
         cudaStream_t st) {
  const UnetLayer& L = S->layers[li];
  return lbnn_conv3d_fwd(in, L.ci, L.w, L.taps, L.b, out_bf, out_f, L.co, 0, nx, ny, nz, 1, S->periodic, L.relu,
                         S->status, st);
}

// Grids on which lbnn_conv3d_fwd_upcat reads the skip tensor and the
// upsampled coarse tensor directly (no concatenated copy).
bool upcat_fused(int nx, int ny, int nz) { return nx % 8 == 0 && ny % 16 == 0 && nz % 2 == 0; }

// conv(li) of concat(skip, up2(low)) at extents (nx, ny, nz)
int conv_cat(SurrogateState* S, int li, const void* skip, int cs, const void* low, int cl, void* ubuf, void* out,
             int nx, int ny, int nz, cudaStream_t st) {
  const UnetLayer& L = S->layers[li];
  if (upcat_fused(nx, ny, nz))
    return lbnn_conv3d_fwd_upcat(skip, cs, low, cl, L.w, L.b, out, nullptr, L.co, 0, nx, ny, nz, 1, S->periodic, L.relu,
                                 S->status, st);
  const int rc = lbnn_up_concat(skip, cs, low, cl, nx, ny, nz, 1, ubuf, st);
  return rc ? rc : conv(S, li, ubuf, out, nullptr, nx, ny, nz, st);
}

// U-Net forward on x (the handle's grid) into S->head
int forward(SurrogateState* S, int nx, int ny, int nz, cudaStream_t st) {
  const int c1 = S->base, c2 = 2 * c1, c3 = 4 * c1, c4 = 8 * c1;
  auto& a = S->act;
  int rc;
#define LBNN_TRY(expr) \
  if ((rc = (expr)) != LB_OK) return rc
  LBNN_TRY(conv(S, 0, S->x, a[0], nullptr, nx, ny, nz, st));
  LBNN_TRY(conv(S, 1, a[0], a[1], nullptr, nx, ny, nz, st));  // s1
  LBNN_TRY(lbnn_avgpool2(a[1], c1, nx, ny, nz, 1, S->p1, st));
  LBNN_TRY(conv(S, 2, S->p1, a[2], nullptr, nx / 2, ny / 2, nz / 2, st));
  LBNN_TRY(conv(S, 3, a[2], a[3], nullptr, nx / 2, ny / 2, nz / 2, st));  // s2
  LBNN_TRY(lbnn_avgpool2(a[3], c2, nx / 2, ny / 2, nz / 2, 1, S->p2, st));
  LBNN_TRY(conv(S, 4, S->p2, a[4], nullptr, nx / 4, ny / 4, nz / 4, st));
  LBNN_TRY(conv(S, 5, a[4], a[5], nullptr, nx / 4, ny / 4, nz / 4, st));  // s3
  LBNN_TRY(lbnn_avgpool2(a[5], c3, nx / 4, ny / 4, nz / 4, 1, S->p3, st));
  LBNN_TRY(conv(S, 6, S->p3, a[6], nullptr, nx / 8, ny / 8, nz / 8, st));
  LBNN_TRY(conv(S, 7, a[6], a[7], nullptr, nx / 8, ny / 8, nz / 8, st));  // b4
  LBNN_TRY(conv_cat(S, 8, a[5], c3, a[7], c4, S->u3, a[8], nx / 4, ny / 4, nz / 4, st));
  LBNN_TRY(conv(S, 9, a[8], a[9], nullptr, nx / 4, ny / 4, nz / 4, st));  // d3
  LBNN_TRY(conv_cat(S, 10, a[3], c2, a[9], c3, S->u2, a[10], nx / 2, ny / 2, nz / 2, st));
  LBNN_TRY(conv(S, 11, a[10], a[11], nullptr, nx / 2, ny / 2, nz / 2, st));  // d2
  LBNN_TRY(conv_cat(S, 12, a[1], c1, a[11], c2, S->u1, a[12], nx, ny, nz, st));
  LBNN_TRY(conv(S, 13, a[12], a[13], nullptr, nx, ny, nz, st));  // d1
  LBNN_TRY(conv(S, 14, a[13], nullptr, S->head, nx, ny, nz, st));
#undef LBNN_TRY
  return LB_OK;
}

}  // namespace
}  // namespace lbcg

using namespace lbcg;

extern "C" {

int lb_surrogate_load(lb_handle* h, const char* path) {
  if (!h || !path) return fail(LB_EINVAL, "null argument");
  int nx, ny, nz;
  uint32_t walls;
  handle_dims(h, &nx, &ny, &nz, &walls);
  if (nx % 8 || ny % 8 || nz % 8) return fail(LB_EINVAL, "the surrogate needs every extent a multiple of 8");
  if (handle_surrogate(h)) return fail(LB_ESTATE, "a surrogate is already loaded on this handle");
  FILE* fp = std::fopen(path, "rb");
  if (!fp) return fail(LB_EIO, std::string("cannot open ") + path);
  uint32_t magic = 0;
  int32_t ver = 0, hdr[3] = {0, 0, 0}, nl = 0;
  float sc[2] = {0, 0};
  uint32_t per = 0;
  bool ok = std::fread(&magic, 4, 1, fp) == 1 && std::fread(&ver, 4, 1, fp) == 1 && std::fread(hdr, 4, 3, fp) == 3 &&
            std::fread(sc, 4, 2, fp) == 2 && std::fread(&per, 4, 1, fp) == 1 && std::fread(&nl, 4, 1, fp) == 1;
  if (!ok || magic != UNET_MAGIC || ver != UNET_VERSION || nl != UNET_LAYERS || hdr[0] < 8 || hdr[0] > 64 ||
      hdr[0] % 8 || hdr[1] != 16 || hdr[2] != 16) {
    std::fclose(fp);
    return fail(LB_EIO, "not a U-Net weight file of this library (base 8..64, 16 input and head channels)");
  }
  auto* S = new SurrogateState();
  S->base = hdr[0];
  S->cin = hdr[1];
  S->cout = hdr[2];
  S->s_rho = sc[0];
  S->s_u = sc[1];
  S->periodic = per;
  const auto table = unet_table(S->base, S->cin, S->cout);
  cudaStream_t st = handle_stream(h);
  const size_t N = (size_t)nx * ny * nz;
  auto dalloc = [&](size_t bytes) -> void* { return handle_alloc(h, bytes); };
  std::vector<float> wbuf;
  for (int l = 0; l < UNET_LAYERS && ok; ++l) {
    int32_t d[4];
    ok = std::fread(d, 4, 4, fp) == 4 && d[0] == table[l][0] && d[1] == table[l][1] && d[2] == table[l][2] &&
         d[3] == table[l][3];
    if (!ok) break;
    UnetLayer L{d[0], d[1], d[2], d[3], nullptr, nullptr};
    const size_t nw = (size_t)L.co * L.taps * L.ci;
    wbuf.resize(nw + L.co);
    ok = std::fread(wbuf.data(), 4, nw + L.co, fp) == nw + L.co;
    if (!ok) break;
    std::vector<__nv_bfloat16> wb(nw);
    for (size_t i = 0; i < nw; ++i) wb[i] = __float2bfloat16_rn(wbuf[i]);
    L.w = (__nv_bfloat16*)dalloc(nw * sizeof(__nv_bfloat16));
    L.b = (float*)dalloc(L.co * sizeof(float));
    ok = L.w && L.b && cudaMemcpyAsync(L.w, wb.data(), nw * 2, cudaMemcpyHostToDevice, st) == cudaSuccess &&
         cudaMemcpyAsync(L.b, wbuf.data() + nw, L.co * 4, cudaMemcpyHostToDevice, st) == cudaSuccess &&
         cudaStreamSynchronize(st) == cudaSuccess;
    S->layers.push_back(L);
  }
  std::fclose(fp);
  if (!ok) {
    delete S;
    return fail(LB_EIO, "truncated or mismatched U-Net weight file");
  }
  // activation buffers for the handle's grid
  const int c1 = S->base, c2 = 2 * c1, c3 = 4 * c1, c4 = 8 * c1;
  const size_t lv[4] = {N, N / 8, N / 64, N / 512};
  const int lvl[14] = {0, 0, 1, 1, 2, 2, 3, 3, 2, 2, 1, 1, 0, 0};
  S->fields = (float*)dalloc(5 * N * 4);
  S->cand = (float*)dalloc(5 * N * 4);
  S->judge_phi = (float*)dalloc(N * 4);
  S->x = (__nv_bfloat16*)dalloc(N * S->cin * 2);
  S->head = (float*)dalloc(N * S->cout * 4);
  S->status = (unsigned*)dalloc(256);
  S->partials = (double*)dalloc((RED_B + 8) * sizeof(double));
  for (int l = 0; l < 14; ++l) S->act.push_back((__nv_bfloat16*)dalloc(lv[lvl[l]] * S->layers[l].co * 2));
  S->p1 = (__nv_bfloat16*)dalloc(lv[1] * c1 * 2);
  S->p2 = (__nv_bfloat16*)dalloc(lv[2] * c2 * 2);
  S->p3 = (__nv_bfloat16*)dalloc(lv[3] * c3 * 2);
  // concatenated decoder inputs, only for levels the fused up-concat convolution cannot take
  const bool f3 = upcat_fused(nx / 4, ny / 4, nz / 4), f2 = upcat_fused(nx / 2, ny / 2, nz / 2),
             f1 = upcat_fused(nx, ny, nz);
  S->u3 = f3 ? nullptr : (__nv_bfloat16*)dalloc(lv[2] * (c3 + c4) * 2);
  S->u2 = f2 ? nullptr : (__nv_bfloat16*)dalloc(lv[1] * (c2 + c3) * 2);
  S->u1 = f1 ? nullptr : (__nv_bfloat16*)dalloc(lv[0] * (c1 + c2) * 2);
  bool all = S->fields && S->cand && S->judge_phi && S->x && S->head && S->status && S->partials && S->p1 && S->p2 &&
             S->p3 && (f1 || S->u1) && (f2 || S->u2) && (f3 || S->u3);
  for (auto* p : S->act) all = all && p;
  if (!all) {
    delete S;
    return fail(LB_ENOMEM, "surrogate buffer allocation failed");
  }
  if (cudaMemsetAsync(S->status, 0, 256, st) != cudaSuccess) {
    delete S;
    return fail(LB_ECUDA, "surrogate status reset failed");
  }
  handle_surrogate(h) = S;
  return LB_OK;
}

int lb_surrogate_predict(lb_handle* h, float* out) {
  if (!h) return fail(LB_EINVAL, "null handle");
  SurrogateState* S = handle_surrogate(h);
  if (!S) return fail(LB_ESTATE, "no surrogate loaded on this handle");
  int nx, ny, nz;
  uint32_t walls;
  handle_dims(h, &nx, &ny, &nz, &walls);
  const int64_t N = (int64_t)nx * ny * nz;
  cudaStream_t st = handle_stream(h);
  int rc = lb_fields(h, 0x1Fu, S->fields, 1);  // phi, rho, ux, uy, uz
  if (rc) return rc;
  if ((rc = lbnn_pack_input(S->fields, N, S->cin, S->s_rho, S->s_u, S->x, st))) return rc;
  if ((rc = forward(S, nx, ny, nz, st))) return rc;
  if ((rc = lbnn_unpack_output(S->fields, S->head, N, S->cout, S->s_rho, S->s_u, 0.5f, S->cand, st))) return rc;
  unsigned stat = 0;
  if (cudaMemcpyAsync(&stat, S->status, sizeof(unsigned), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return fail(LB_ECUDA, "surrogate status read failed");
  if (stat) return fail(LB_ETIMEOUT, "a tensor-core kernel of the surrogate gave up a bounded wait");
  if (out && cudaMemcpyAsync(out, S->cand, 5 * N * sizeof(float), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return fail(LB_ECUDA, "candidate copy failed");
  return LB_OK;
}

int lb_surrogate_cycle(lb_handle* h, lb_handle* judge, int32_t K, double vol_tol, double phi_tol,
                       int32_t* accepted, double* phi_err) {
  if (!h || !accepted || !phi_err) return fail(LB_EINVAL, "null argument");
  if (K < 1) return fail(LB_EINVAL, "K must be >= 1");
  if (judge == h) return fail(LB_EINVAL, "the judge must be a second handle");
  SurrogateState* S = handle_surrogate(h);
  if (!S) return fail(LB_ESTATE, "no surrogate loaded on this handle");
  int nx, ny, nz;
  uint32_t walls;
  handle_dims(h, &nx, &ny, &nz, &walls);
  const int64_t N = (int64_t)nx * ny * nz;
  cudaStream_t st = handle_stream(h);
  int rc;
  if (judge) {  // the plain LB from the exact same state
    if ((rc = lb_copy_state(judge, h))) return rc;
    if ((rc = lb_step(judge, K))) return rc;
  }
  if ((rc = lb_surrogate_predict(h, nullptr))) return rc;
  int32_t c0 = 0, c1 = 0;
  double v0 = 0, v1 = 0;
  if ((rc = lb_phi_monitor(h, S->fields, &c0, &v0))) return rc;
  if ((rc = lb_phi_monitor(h, S->cand, &c1, &v1))) return rc;
  bool ok = c0 == c1 && std::fabs(v1 - v0) <= vol_tol * std::max(v0, 1.0);
  *phi_err = -1.0;
  if (judge) {
    if ((rc = lb_fields(judge, 1u, S->judge_phi, 1))) return rc;
    Geo g{nx, ny, nz, 0, 0, 0, (long long)N};
    const int nb = (int)std::min<int64_t>(RED_B, (N + RED_T * 8 - 1) / (RED_T * 8));
    cudaStream_t js = handle_stream(judge);
    cudaEvent_t ev;
    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) return fail(LB_ECUDA, "event");
    cudaEventRecord(ev, js);
    cudaStreamWaitEvent(st, ev, 0);
    cudaEventDestroy(ev);
    k_absdiff_partial<<<nb, RED_T, 0, st>>>(g, S->cand, S->judge_phi, S->partials);
    k_sum_partials<<<1, RED_T, 0, st>>>(nb, S->partials, S->partials + RED_B);
    double sum = 0;
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(&sum, S->partials + RED_B, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return fail(LB_ECUDA, "judgement reduction failed");
    count_launches(2);
    *phi_err = sum / (double)N;
    if (*phi_err > phi_tol) ok = false;
  }
  if (ok) {
    rc = lb_init_fields(h, S->cand, S->cand + N, S->cand + 2 * N, 1, 1);
  } else if (judge) {
    rc = lb_copy_state(h, judge);
  } else {
    rc = lb_step(h, K);
  }
  if (rc) return rc;
  *accepted = ok ? 1 : 0;
  return LB_OK;
}

}  // extern "C"
