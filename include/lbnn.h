/*
 * lbnn.h -- C ABI of the surrogate network's kernels (the learned part that
 * advances (phi, rho, u) by K lattice Boltzmann steps; its populations are
 * then rebuilt by the regularised reconstruction of lbcg.h, Sec. IV.C).
 *
 * Activations are channels-last BF16 tensors X[v][c], v = x + nx (y + ny (z +
 * nz b)), 16-byte aligned device pointers.  Convolutions run on the tcgen05
 * tensor cores (BF16 operands, FP32 accumulation in tensor memory).
 * periodic: bit a (a = 0,1,2 for x,y,z) wraps that axis, otherwise the
 * convolution pads with zeros.  status: device word; bit 4 is set when a
 * bounded wait inside a kernel gave up (the output is then not written).
 * All calls are asynchronous on `stream` (cudaStream_t, NULL = legacy stream)
 * and return LB_OK or an LB_E* code (lbcg.h) after host-side validation.
 */
#ifndef LBNN_H
#define LBNN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Poll limit of the bounded handshake waits (copies -> UMMAs -> epilogue)
 * inside the convolution kernels launched after this call (a kernel takes the
 * value at launch; a captured CUDA graph keeps the value of its capture).  A
 * wait that runs out makes the kernel give up: it still waits, with a fixed
 * bound of its own, for every UMMA it has committed, frees its tensor memory,
 * sets bit 4 of the status word and leaves its output unwritten or partial.
 * limit = 0 gives up at the first wait (exercises that path).  The default is
 * LBNN_WAIT_LIMIT_DEFAULT.  previous (may be NULL) receives the limit in force
 * before the call.  Process-wide; returns LB_OK. */
#define LBNN_WAIT_LIMIT_DEFAULT (1u << 22)
int lbnn_set_wait_limit(uint32_t limit, uint32_t* previous);

/* Reads the status word of the calls above (device pointer) after
 * synchronising `stream`, clears it, and returns LB_ETIMEOUT if bit 4 was set
 * (a bounded wait gave up), LB_ECUDA on a CUDA error, else LB_OK. */
int lbnn_check_status(unsigned* status, void* stream);

/* y[v][co] = act(bias[co] + sum_{t<taps, ci} w[co][t][ci] x[v + off_t][ci]),
 * taps = 27 (3x3x3, tap t = (dx+1) + 3(dy+1) + 9(dz+1)) or 1 (1x1x1).
 * cin, cout: multiples of 16 (cin <= 1024, cout <= 256).  bias may be NULL;
 * relu != 0 applies max(0, .).  y (BF16) and/or yf (FP32) receive the result
 * with row stride ldy elements (0: cout; otherwise a multiple of 8 >= cout),
 * so that several calls can fill disjoint channel ranges of one tensor. */
int lbnn_conv3d_fwd(const void* x, int32_t cin, const void* w, int32_t taps, const float* bias, void* y, float* yf,
                    int32_t cout, int32_t ldy, int32_t nx, int32_t ny, int32_t nz, int32_t nb, uint32_t periodic,
                    int32_t relu, unsigned* status, void* stream);

/* The 3x3x3 convolution above of the decoder input concat(skip, up2(low)):
 * channels [0, cs) are skip[v][cs] at full resolution, channels [cs, cs + cl)
 * are low[parent(v)][cl] of the half-resolution tensor (nearest x2
 * upsampling, parent(v) = (x/2, y/2, z/2)), read in place without the
 * concatenated copy; w is [cout][27][cs + cl].  Same outputs, ldy and
 * status word as lbnn_conv3d_fwd.  Needs nx % 8 == 0, ny % 16 == 0 and an
 * even nz (LB_EINVAL otherwise; concatenate with lbnn_up_concat then). */
int lbnn_conv3d_fwd_upcat(const void* skip, int32_t cs, const void* low, int32_t cl, const void* w, const float* bias,
                          void* y, float* yf, int32_t cout, int32_t ldy, int32_t nx, int32_t ny, int32_t nz, int32_t nb,
                          uint32_t periodic, int32_t relu, unsigned* status, void* stream);

/* dw[co][t][ci] += sum_v dy[v][co] x[v + off_t][ci] (FP32, accumulated with
 * atomics; clear dw first); cout a multiple of 16 up to 256.  With taps = 27,
 * nx % 8 == 0 and ny % 16 == 0 the sum runs over 8 x 16 plane blocks, each
 * CTA adding its partial sums once; otherwise voxels are split into slices
 * of vox_per_cta per CTA.  vox_per_cta: a multiple of 64 in either case. */
int lbnn_conv3d_wgrad(const void* dy, int32_t cout, const void* x, int32_t cin, int32_t taps, float* dw, int32_t nx,
                      int32_t ny, int32_t nz, int32_t nb, uint32_t periodic, int32_t vox_per_cta, unsigned* status,
                      void* stream);

/* ---- data movement and element-wise kernels ----------------------------- */
/* fields [5][n] FP32 (phi, rho, ux, uy, uz) -> x[n][c] BF16 channels
 * (phi, s_rho (rho - 1), s_u ux, s_u uy, s_u uz, 0 ...); c >= 5. */
int lbnn_pack_input(const float* fields, int64_t n, int32_t c, float s_rho, float s_u, void* x, void* stream);
/* out[5][n] = fields + (y0, y1/s_rho, y2/s_u, y3/s_u, y4/s_u), phi clamped to
 * [-1, 1] and rho to >= rho_min; y[n][c] FP32 network output. */
int lbnn_unpack_output(const float* fields, const float* y, int64_t n, int32_t c, float s_rho, float s_u,
                       float rho_min, float* out, void* stream);
/* t[n][c] FP32 = scaled increments (f1 - f0) in the channel order of pack_input. */
int lbnn_pack_target(const float* f0, const float* f1, int64_t n, int32_t c, float s_rho, float s_u, float* t,
                     void* stream);
/* 2x2x2 average pooling (even extents) and its gradient (dx += dy/8, FP32). */
int lbnn_avgpool2(const void* x, int32_t c, int32_t nx, int32_t ny, int32_t nz, int32_t nb, void* y, void* stream);
int lbnn_avgpool2_bwd(const float* dy, int32_t c, int32_t nx, int32_t ny, int32_t nz, int32_t nb, float* dx,
                      void* stream);
/* out[v] = (skip[v] (cs channels), low[parent(v)] (cl channels)), nearest
 * x2 upsampling of the half-resolution low; and its gradient (accumulating
 * into dskip and dlow). nx, ny, nz: full-resolution extents. */
int lbnn_up_concat(const void* skip, int32_t cs, const void* low, int32_t cl, int32_t nx, int32_t ny, int32_t nz,
                   int32_t nb, void* out, void* stream);
int lbnn_up_concat_bwd(const float* dout, int32_t cs, int32_t cl, int32_t nx, int32_t ny, int32_t nz, int32_t nb,
                       float* dskip, float* dlow, void* stream);
/* gradient through ReLU: g * (y > 0) (relu = 0: copy), to BF16 gb and/or FP32 gf. */
int lbnn_relu_bwd(const float* g, const void* y, int64_t n, int32_t relu, void* gb, float* gf, void* stream);
/* db[c] += sum_v g[v][c] (c divides 256). */
int lbnn_bias_grad(const float* g, int64_t nvox, int32_t c, float* db, void* stream);
/* weights of the input gradient: wt[ci][t][co] = w[co][taps-1-t][ci]. */
int lbnn_flip_weights(const void* w, int32_t cout, int32_t taps, int32_t cin, void* wt, void* stream);
/* weighted MSE over the first nch of c channels: grad = 2 w_c (p - t)/(n nch),
 * *loss += sum w_c (p - t)^2/(n nch) (FP64). */
int lbnn_mse(const float* p, const float* t, int64_t n, int32_t c, int32_t nch, const float* wch, float* grad,
             double* loss, void* stream);
/* Adam step (bias-corrected, step >= 1, decoupled weight decay wd) on FP32
 * master weights p; bf (nullable) receives a BF16 copy. */
int lbnn_adam(float* p, const float* g, float* m, float* v, int64_t n, float lr, float b1, float b2, float eps,
              int32_t step, float wd, void* bf, void* stream);
int lbnn_f32_to_bf16(const float* a, int64_t n, void* b, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* LBNN_H */
