#pragma once
// Device code of the time step of the two-component colour-gradient LB scheme on D3Q27
// (arXiv 2405.14551, Sec. III.B-III.D) for sm_103a.
//
// A step is one kernel, k_step, over CTA tiles of TX x TY x TZ nodes (TX x TY
// threads, TZ nodes per thread):
//   1. stage phi(t) of the tile plus a halo of H nodes in shared memory.  phi
//      is not stored between steps as an array of its own: the step before
//      accumulated the component densities rhoA, rhoB of every node on the
//      write side (item 4), and the staging decodes
//      phi = (rhoA - rhoB)/(rhoA + rhoB) (Eq. order_param) from them;
//   2. with near contact (A_h != 0, halo H > K): every interface node of the
//      tile scans along its outward normal (Eqs. stress_jump,
//      near_cont_force); the distance h stays in shared memory.  The
//      in-loop tile (INL) scans each interface node in item 3 instead,
//      while the node's population loads are in flight;
//   3. every thread pulls the 27 (x2) populations of its nodes (periodic
//      wrap, halfway bounce-back at solid neighbours, Sec. III.D), takes the
//      moments, the colour gradient from the staged tile, the repulsion from
//      h, the Guo-shifted velocity, relaxes the total populations (BGK), adds
//      the perturbation Omega^(2) and the forcing source, recolours (Eqs.
//      ome3_1/2) and stores the post-collision state once;
//   4. each post-collision component population f*^k_i(x) is also what the
//      node x + c_i pulls at the next step (x itself, as direction opp(i),
//      when x + c_i is solid), so it is x's contribution to rho_k there.  The
//      CTA sums the contributions over its tile plus a one-node ring in
//      shared memory as fixed-point integers and adds the sums to a global
//      accumulator with 64-bit integer atomics.  Integer sums are exact, so
//      phi(t+1) does not depend on the order of the additions (tile shape,
//      CTA schedule, batching), and it equals what a pull of the stored
//      populations gives (k_phi_acc rebuilds it that way after a load).
// The accumulators rotate over three buffers: a step reads phi(t) from one,
// adds phi(t+1) into the next (zeroed by the step before) and zeroes its own
// nodes of the third (read by the step before and not read again).  The
// populations are read and written once per step; the accumulators add 8 B
// read, 16 B atomically updated and 8 B zeroed per node (FP32 storages).
// Populations are structure-of-arrays [dir][z][y][x]: for a fixed direction
// consecutive threads read consecutive addresses (coalesced).
#include <cstdio>
#include <cstdlib>
#include <type_traits>

#include "internal.h"
#include "lattice.cuh"

namespace lbcg {

// LBCG_TRACE=1 prints every launch of this file with the kernel's attributes.
inline bool trace_on() {
  static int on = -1;
  if (on < 0) {
    const char* v = std::getenv("LBCG_TRACE");
    on = (v && v[0] == '1') ? 1 : 0;
  }
  return on == 1;
}

template <typename K>
inline void trace_kernel(const char* what, K kern, dim3 grid, dim3 block, size_t smem) {
  if (!trace_on()) return;
  cudaFuncAttributes a{};
  cudaError_t e = cudaFuncGetAttributes(&a, kern);
  std::fprintf(stderr, "[lbcg] %s grid=(%u,%u,%u) block=(%u,%u,%u) smem=%zu attr=%s regs=%d maxthreads=%d local=%zu\n",
               what, grid.x, grid.y, grid.z, block.x, block.y, block.z, smem, cudaGetErrorString(e), a.numRegs,
               a.maxThreadsPerBlock, (size_t)a.localSizeBytes);
  std::fflush(stderr);
}


// ---------------------------------------------------------------------------
// storage traits
// ---------------------------------------------------------------------------
template <int ST>
struct Store;
template <>
struct Store<0> {  // LB_STORAGE_TWOSET_F32
  using R = float;
  using E = float;
  static constexpr bool TWOSET = true;
  static constexpr bool MOMENT = false;
};
template <>
struct Store<1> {  // LB_STORAGE_REDUCED_F32
  using R = float;
  using E = float;
  static constexpr bool TWOSET = false;
  static constexpr bool MOMENT = false;
};
template <>
struct Store<2> {  // LB_STORAGE_REDUCED_F16
  using R = float;
  using E = __half;
  static constexpr bool TWOSET = false;
  static constexpr bool MOMENT = false;
};
template <>
struct Store<3> {  // LB_STORAGE_TWOSET_F64
  using R = double;
  using E = double;
  static constexpr bool TWOSET = true;
  static constexpr bool MOMENT = false;
};
// LB_STORAGE_MOMENT_F32: the coefficients of f*_i = w_i (alpha + beta.c_i +
// c_i.Gamma.c_i) in three arrays of 16- and 8-byte records, so that a
// direction reads at most three vectors: qa[N] = (alpha, beta_x, beta_y,
// beta_z), qb[N] = (Gamma_xx, Gamma_yy, Gamma_zz, 2 Gamma_xy) from float 4N
// on, qc[N] = (2 Gamma_xz, 2 Gamma_yz) from float 8N on; the colour scalars
// as in the reduced storage.
template <>
struct Store<4> {
  using R = float;
  using E = float;
  static constexpr bool TWOSET = false;
  static constexpr bool MOMENT = true;
};

template <int ST>
__device__ __forceinline__ typename Store<ST>::R decode(typename Store<ST>::E v, int i) {
  if constexpr (ST == 2) {
    return wgt<float>(i) + __half2float(v) * F16_INV_SCALE;
  } else {
    return v;
  }
}
template <int ST>
__device__ __forceinline__ typename Store<ST>::E encode(typename Store<ST>::R v, int i) {
  if constexpr (ST == 2) {
    return __float2half_rn((v - wgt<float>(i)) * F16_SCALE);
  } else {
    return v;
  }
}

// Rounded products without contraction: the sending and the pulling node
// must form the same component populations bit for bit (see colour_split).
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }

// Moment storage (Sec. IV.C, Eq. eq:llb-pull): f*_i = w_i (alpha + beta.c +
// c.Gamma.c) of a node's coefficients at c = c_i, or at c = -c_i when bb
// (bounce-back from the node itself, dir = opp(i)).  Only the coefficients
// that c_i touches enter; the products with c components are exact (+-1).
template <typename R>
__device__ __forceinline__ R eval_moment(const float4& qa, const float4& qb, const float2& qc, int i, bool bb) {
  R lin = R(0), quad = R(0);
  if (cx(i)) lin += R(cx(i)) * qa.y;
  if (cy(i)) lin += R(cy(i)) * qa.z;
  if (cz(i)) lin += R(cz(i)) * qa.w;
  if (cx(i)) quad += qb.x;
  if (cy(i)) quad += qb.y;
  if (cz(i)) quad += qb.z;
  if (cx(i) && cy(i)) quad += R(cx(i) * cy(i)) * qb.w;
  if (cx(i) && cz(i)) quad += R(cx(i) * cz(i)) * qc.x;
  if (cy(i) && cz(i)) quad += R(cy(i) * cz(i)) * qc.y;
  return mul_rn(wgt<R>(i), qa.x + quad + (bb ? -lin : lin));
}

// Stored post-collision total population f*_dir of node src (single set
// storages).  Reduced: the stored value.  Moment storage: the node's
// quadratic form (eval_moment); only the records that c_i touches are read.
template <int ST, typename I>
__device__ __forceinline__ typename Store<ST>::R load_fs(const typename Store<ST>::E* __restrict__ f, I N, I dir, I src,
                                                         int i, bool bb) {
  using R = typename Store<ST>::R;
  if constexpr (Store<ST>::MOMENT) {
    const float4 qa = reinterpret_cast<const float4*>(f)[src];
    float4 qb = make_float4(0.f, 0.f, 0.f, 0.f);
    float2 qc = make_float2(0.f, 0.f);
    if (cx(i) || cy(i) || cz(i)) qb = reinterpret_cast<const float4*>(f + (I)4 * N)[src];
    if ((cx(i) && cz(i)) || (cy(i) && cz(i))) qc = reinterpret_cast<const float2*>(f + (I)8 * N)[src];
    return eval_moment<R>(qa, qb, qc, i, bb);
  } else {
    return decode<ST>(f[dir * N + src], i);
  }
}

__device__ __forceinline__ float sqrt_(float v) { return sqrtf(v); }
__device__ __forceinline__ double sqrt_(double v) { return sqrt(v); }
__device__ __forceinline__ float round_(float v) { return roundf(v); }  // half away from zero
__device__ __forceinline__ double round_(double v) { return round(v); }
__device__ __forceinline__ bool finite_(float v) { return isfinite(v); }
__device__ __forceinline__ bool finite_(double v) { return isfinite(v); }

// Wrapped neighbour coordinates of a node: c[d+1] = coordinate + d on periodic
// axes (mod n); raw on wall axes.  solid[d+1] marks a solid layer.
struct Nbr {
  int xs[3], ys[3], zs[3];
  bool sx[3], sy[3], sz[3];
};

__device__ __forceinline__ void make_nbr(const Geo& g, int x, int y, int z, Nbr& n) {
#pragma unroll
  for (int d = -1; d <= 1; ++d) {
    int a = x + d, b = y + d, c = z + d;
    if (!g.wx) a = a < 0 ? a + g.nx : (a >= g.nx ? a - g.nx : a);
    if (!g.wy) b = b < 0 ? b + g.ny : (b >= g.ny ? b - g.ny : b);
    if (!g.wz) c = c < 0 ? c + g.nz : (c >= g.nz ? c - g.nz : c);
    n.xs[d + 1] = a;
    n.ys[d + 1] = b;
    n.zs[d + 1] = c;
    n.sx[d + 1] = g.wx && (a <= 0 || a >= g.nx - 1);
    n.sy[d + 1] = g.wy && (b <= 0 || b >= g.ny - 1);
    n.sz[d + 1] = g.wz && (c <= 0 || c >= g.nz - 1);
  }
}

__device__ __forceinline__ bool is_solid(const Geo& g, int x, int y, int z) {
  return (g.wx && (x == 0 || x == g.nx - 1)) || (g.wy && (y == 0 || y == g.ny - 1)) ||
         (g.wz && (z == 0 || z == g.nz - 1));
}

__device__ __forceinline__ bool near_wall(const Geo& g, int x, int y, int z) {
  return (g.wx && (x <= 1 || x >= g.nx - 2)) || (g.wy && (y <= 1 || y >= g.ny - 2)) ||
         (g.wz && (z <= 1 || z >= g.nz - 2));
}

// Whether the box [x0 - d, x0 + TX - 1 + d] x ... (a tile and its halo of d
// nodes) holds a solid layer or leaves the box on a walled axis.
__device__ __forceinline__ bool region_walled(const Geo& g, int x0, int y0, int z0, int tx, int ty, int tz, int d) {
  return (g.wx && (x0 - d <= 0 || x0 + tx - 1 + d >= g.nx - 1)) ||
         (g.wy && (y0 - d <= 0 || y0 + ty - 1 + d >= g.ny - 1)) ||
         (g.wz && (z0 - d <= 0 || z0 + tz - 1 + d >= g.nz - 1));
}

template <int ST>
struct View {
  using E = typename Store<ST>::E;
  E* f;
  float4* sv;
};

template <int ST>
__host__ __device__ __forceinline__ View<ST> view(const StateBuf& b) {
  View<ST> v;
  v.f = reinterpret_cast<typename Store<ST>::E*>(b.f);
  v.sv = b.sv;
  return v;
}

// Component split of a single-set population as the pulling node rebuilds it
// (recolouring, Eq. ome3_1, evaluated one step later): f^A_i = s f*_i +
// w_i c_i.v/|c_i|, f^B_i = f*_i - f^A_i, with (s, v) the colour scalars of the
// node that stored f*_i.  bb: bounce-back, the node's own f*_opp(i) pulled as
// direction i, whose segregation term is the negative of direction i's.  The
// rounding is explicit, so the sender of a value (step_nodes) and its puller
// form the same f^A_i, f^B_i bit for bit.
template <typename R, bool MAYBB>
__device__ __forceinline__ void colour_split(R fs, const float4& sv, int i, bool bb, R& va, R& vb) {
  R cv = R(0);
  if (cx(i)) cv += R(cx(i)) * R(sv.y);
  if (cy(i)) cv += R(cy(i)) * R(sv.z);
  if (cz(i)) cv += R(cz(i)) * R(sv.w);
  const R k = wgt<R>(i) * inv_norm<R>(i);  // folded to one constant per direction
  R seg = mul_rn(k, cv);
  if constexpr (MAYBB) seg = bb ? -seg : seg;
  va = fma_rn(R(sv.x), fs, seg);
  vb = fs - va;
}

// Pull the pre-collision populations of node `self` (streaming, Eq. eq:lbm):
// f_i(x) = f*_i(x - c_i), or f*_{opp(i)}(x) when x - c_i is solid (halfway
// bounce-back).  Returns the totals f_i and the component densities.  With
// per-component output (fa, fb non-null) also the component populations.
template <int ST, bool COMP>
__device__ __forceinline__ void pull_node(const View<ST>& S, const Geo& g, const Nbr& n, long long self,
                                          typename Store<ST>::R f[Q], typename Store<ST>::R& rA,
                                          typename Store<ST>::R& rB, typename Store<ST>::R* fa,
                                          typename Store<ST>::R* fb) {
  using R = typename Store<ST>::R;
  const size_t N = (size_t)g.N;
  rA = R(0);
  rB = R(0);
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const int a = 1 - cx(i), b = 1 - cy(i), c = 1 - cz(i);
    const bool bb = n.sx[a] | n.sy[b] | n.sz[c];
    const long long src = bb ? self : (long long)n.xs[a] + (long long)g.nx * ((long long)n.ys[b] + (long long)g.ny * n.zs[c]);
    const int dir = bb ? opp(i) : i;
    R va, vb;
    if constexpr (Store<ST>::TWOSET) {
      va = decode<ST>(S.f[(size_t)dir * N + src], i);
      vb = decode<ST>(S.f[(size_t)(Q + dir) * N + src], i);
      f[i] = va + vb;
    } else {
      const R fs = load_fs<ST, size_t>(S.f, N, (size_t)dir, (size_t)src, i, bb);
      colour_split<R, true>(fs, S.sv[src], i, bb, va, vb);
      f[i] = fs;
    }
    rA += va;
    rB += vb;
    if constexpr (COMP) {
      fa[i] = va;
      fb[i] = vb;
    }
  }
}

// Pre-collision populations from fields (initial state or reconstruction):
// f_i = f^eq_i(rho, u) (Eq. disteq) [+ w_i/(2 cs^4) Q_i:Pi^neq], f^A = (rhoA/rho) f.
template <typename R, bool COMP>
__device__ __forceinline__ void fields_node(const InitBuf& I, const Geo& g, const Phys& P, const Nbr& n,
                                            long long self, R f[Q], R& rA, R& rB, R* fa, R* fb) {
  const R ph = I.phi[self];
  const R rho = I.rho ? R(I.rho[self]) : R(1);
  R u[3] = {R(0), R(0), R(0)};
  if (I.u) {
    u[0] = I.u[self];
    u[1] = I.u[(size_t)g.N + self];
    u[2] = I.u[2 * (size_t)g.N + self];
  }
  rA = rho * (R(1) + ph) * R(0.5);
  rB = rho * (R(1) - ph) * R(0.5);
  R Pi[6] = {R(0), R(0), R(0), R(0), R(0), R(0)};  // xx yy zz xy xz yz
  if (I.regularised && I.u) {
    // isotropic stencil gradient du[b][a] = d_a u_b; solid neighbour -> own value
    R du[3][3] = {{R(0), R(0), R(0)}, {R(0), R(0), R(0)}, {R(0), R(0), R(0)}};
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      if (i == REST) continue;
      const int a = 1 + cx(i), b = 1 + cy(i), c = 1 + cz(i);
      const bool sol = n.sx[a] | n.sy[b] | n.sz[c];
      const long long m =
          sol ? self : (long long)n.xs[a] + (long long)g.nx * ((long long)n.ys[b] + (long long)g.ny * n.zs[c]);
      const R w3 = R(3) * wgt<R>(i);
#pragma unroll
      for (int bcomp = 0; bcomp < 3; ++bcomp) {
        const R ub = I.u[(size_t)bcomp * g.N + m];
        du[bcomp][0] += w3 * R(cx(i)) * ub;
        du[bcomp][1] += w3 * R(cy(i)) * ub;
        du[bcomp][2] += w3 * R(cz(i)) * ub;
      }
    }
    R tau;
    if (P.equal_tau) {
      tau = R(P.tau_a);
    } else {
      const R nu_a = (R(P.tau_a) - R(0.5)) / R(3), nu_b = (R(P.tau_b) - R(0.5)) / R(3);
      const R nu = R(1) / ((rA / rho) / nu_a + (rB / rho) / nu_b);
      tau = R(3) * nu + R(0.5);
    }
    const R pref = -rho * tau / R(3);  // Pi^neq = -rho cs2 tau (grad u + grad u^T)
    Pi[0] = pref * R(2) * du[0][0];
    Pi[1] = pref * R(2) * du[1][1];
    Pi[2] = pref * R(2) * du[2][2];
    Pi[3] = pref * (du[0][1] + du[1][0]);
    Pi[4] = pref * (du[0][2] + du[2][0]);
    Pi[5] = pref * (du[1][2] + du[2][1]);
  }
  const R uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  const R trPi = Pi[0] + Pi[1] + Pi[2];
  const R sA = rA / rho;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const R cu = R(cx(i)) * u[0] + R(cy(i)) * u[1] + R(cz(i)) * u[2];
    R fi = wgt<R>(i) * rho * (R(1) + R(3) * cu + R(4.5) * cu * cu - R(1.5) * uu);
    // (c c - cs2 I):Pi with symmetric Pi
    const R qpi = R(cx(i) * cx(i)) * Pi[0] + R(cy(i) * cy(i)) * Pi[1] + R(cz(i) * cz(i)) * Pi[2] +
                  R(2 * cx(i) * cy(i)) * Pi[3] + R(2 * cx(i) * cz(i)) * Pi[4] + R(2 * cy(i) * cz(i)) * Pi[5] -
                  trPi / R(3);
    fi += wgt<R>(i) * R(4.5) * qpi;
    f[i] = fi;
    if constexpr (COMP) {
      fa[i] = sA * fi;
      fb[i] = fi - sA * fi;
    }
  }
}

// Pull for the hot path: totals f_i and component densities.  WALLFREE: no
// neighbour of the node is solid (no bounce-back test).  IDX32: every
// population offset fits in 32 bits.  TOTALS (single-set storages): only the
// totals f_i; the neighbours' colour scalars are not read and rA, rB are left
// to the caller.
template <int ST, bool WALLFREE, bool IDX32, bool TOTALS>
__device__ __forceinline__ void pull_fast(const View<ST>& S, const Geo& g, const Nbr& n, int self,
                                          typename Store<ST>::R f[Q], typename Store<ST>::R& rA,
                                          typename Store<ST>::R& rB) {
  using R = typename Store<ST>::R;
  using I = typename std::conditional<IDX32, unsigned, size_t>::type;
  const I N = (I)g.N;
  int rb[3][3];
#pragma unroll
  for (int b = 0; b < 3; ++b)
#pragma unroll
    for (int c = 0; c < 3; ++c) rb[b][c] = g.nx * (n.ys[b] + g.ny * n.zs[c]);
  rA = R(0);
  rB = R(0);
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const int a = 1 - cx(i), b = 1 - cy(i), c = 1 - cz(i);
    int src = n.xs[a] + rb[b][c];
    I dir = (I)i;
    bool bb = false;
    if constexpr (!WALLFREE) {
      bb = n.sx[a] | n.sy[b] | n.sz[c];
      src = bb ? self : src;
      dir = bb ? (I)opp(i) : dir;
    }
    if constexpr (Store<ST>::TWOSET) {
      const R va = decode<ST>(S.f[dir * N + (I)src], i);
      const R vb = decode<ST>(S.f[((I)Q + dir) * N + (I)src], i);
      f[i] = va + vb;
      rA += va;
      rB += vb;
    } else if constexpr (TOTALS) {
      f[i] = load_fs<ST, I>(S.f, N, dir, (I)src, i, bb);
    } else {
      const R fs = load_fs<ST, I>(S.f, N, dir, (I)src, i, bb);
      R va, vb;
      colour_split<R, !WALLFREE>(fs, S.sv[src], i, bb, va, vb);
      f[i] = fs;
      rA += va;
      rB += vb;
    }
  }
}

// The pull of pull_fast split in two: the raw stored values (both sets, or
// the single set's totals) are loaded first and decoded and summed later, so
// that independent work (the near-contact scan) runs while the loads are in
// flight.  Same values and the same order of additions as pull_fast.
template <int ST, bool WALLFREE, bool IDX32>
__device__ __forceinline__ void pull_raw(const View<ST>& S, const Geo& g, const Nbr& n, int self,
                                         typename Store<ST>::E ra[Q], typename Store<ST>::E rb[Q]) {
  using I = typename std::conditional<IDX32, unsigned, size_t>::type;
  const I N = (I)g.N;
  int rbo[3][3];
#pragma unroll
  for (int b = 0; b < 3; ++b)
#pragma unroll
    for (int c = 0; c < 3; ++c) rbo[b][c] = g.nx * (n.ys[b] + g.ny * n.zs[c]);
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const int a = 1 - cx(i), b = 1 - cy(i), c = 1 - cz(i);
    int src = n.xs[a] + rbo[b][c];
    I dir = (I)i;
    if constexpr (!WALLFREE) {
      const bool bb = n.sx[a] | n.sy[b] | n.sz[c];
      src = bb ? self : src;
      dir = bb ? (I)opp(i) : dir;
    }
    ra[i] = S.f[dir * N + (I)src];
    if constexpr (Store<ST>::TWOSET) rb[i] = S.f[((I)Q + dir) * N + (I)src];
  }
}
template <int ST>
__device__ __forceinline__ void pull_raw_finish(const typename Store<ST>::E ra[Q], const typename Store<ST>::E rb[Q],
                                                typename Store<ST>::R f[Q], typename Store<ST>::R& rA,
                                                typename Store<ST>::R& rB) {
  using R = typename Store<ST>::R;
  rA = R(0);
  rB = R(0);
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    if constexpr (Store<ST>::TWOSET) {
      const R va = decode<ST>(ra[i], i), vb = decode<ST>(rb[i], i);
      f[i] = va + vb;
      rA += va;
      rB += vb;
    } else {
      f[i] = decode<ST>(ra[i], i);
    }
  }
}

// ---------------------------------------------------------------------------
// write-side accumulation of the next time level's component densities
// ---------------------------------------------------------------------------
// Each contribution f*^k_i is rounded to a multiple of 2^-SHIFT and summed as
// an integer.  FP32 storages: SHIFT = 28 (component sums within +-8, step
// 3.7e-9, below the FP32 rounding of a density near 1), the two sums of a
// node packed in one 64-bit word (rhoA in the high half, rhoB in the low
// half, two's complement), so one atomic adds both.  FP64: SHIFT = 56 (sums
// within +-128, step 1.4e-17), two 64-bit words per node.  RHO_MAX bounds the
// density that the status check accepts, so that no sum leaves its range.
// The accumulator words are staged, zeroed and updated by every step while
// the population state streams through L2; their loads, stores and
// reductions carry an evict-last L2 policy, so that more of them are still
// in L2 when the next access comes (measured: 3.24 -> 3.17 ms per step on
// the 256x256x512 emulsion).
__device__ __forceinline__ unsigned long long acc_policy() {
  unsigned long long pol;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ void acc_red(unsigned long long* p, unsigned long long v) {
  asm volatile("red.global.add.L2::cache_hint.u64 [%0], %1, %2;" ::"l"(__cvta_generic_to_global(p)), "l"(v),
               "l"(acc_policy())
               : "memory");
}
__device__ __forceinline__ void acc_st(unsigned long long* p, unsigned long long v) {
  asm volatile("st.global.L2::cache_hint.u64 [%0], %1, %2;" ::"l"(__cvta_generic_to_global(p)), "l"(v),
               "l"(acc_policy())
               : "memory");
}
__device__ __forceinline__ ulonglong2 acc_ld2(const unsigned long long* p) {
  ulonglong2 v;
  asm volatile("ld.global.L2::cache_hint.v2.u64 {%0, %1}, [%2], %3;"
               : "=l"(v.x), "=l"(v.y)
               : "l"(__cvta_generic_to_global(p)), "l"(acc_policy()));
  return v;
}

template <typename R>
struct Acc;
template <>
struct Acc<float> {
  static constexpr int W = 1;  // 64-bit words per node, in global and in shared memory
  using S = int;               // sum of one component
  static constexpr float RHO_MAX = 4.0f;
  __device__ static __forceinline__ S q(float v) { return __float2int_rn(v * 268435456.0f); }
  // add one node's contributions (a, b) to the shared partial sums of node e:
  // two planes of E 32-bit words (rhoA, then rhoB) in the E 64-bit words of
  // sw; 32-bit shared atomics (one packed 64-bit shared atomic per direction
  // measured slower)
  __device__ static __forceinline__ void send_shared(unsigned long long* sw, int E, int e, float a, float b) {
    int* p = reinterpret_cast<int*>(sw);
    atomicAdd(p + e, q(a));
    atomicAdd(p + E + e, q(b));
  }
  __device__ static __forceinline__ void flush_shared(unsigned long long* acc, size_t node,
                                                      const unsigned long long* sw, int E, int e) {
    const int* p = reinterpret_cast<const int*>(sw);
    const unsigned long long w = pack(p[e], p[E + e]);
    if (w) acc_red(acc + node, w);
  }
  __device__ static __forceinline__ bool shared_zero(const unsigned long long* sw, int E, int e) {
    const int* p = reinterpret_cast<const int*>(sw);
    return (p[e] | p[E + e]) == 0;
  }
  __device__ static __forceinline__ unsigned long long pack(S a, S b) {
    return ((unsigned long long)(unsigned)a << 32) + (unsigned long long)(long long)b;
  }
  __device__ static __forceinline__ void store(unsigned long long* acc, size_t node, S a, S b) {
    acc[node] = pack(a, b);
  }
  __device__ static __forceinline__ void zero(unsigned long long* acc, size_t node) { acc_st(acc + node, 0ull); }
  // phi = (rhoA - rhoB)/(rhoA + rhoB) of one packed word.  The halves are
  // rhoA and rhoB in units of 2^-28; with densities below RHO_MAX (< 2^30
  // units) the difference and the sum are exact 32-bit integers, each rounded
  // once to FP32, and the quotient is taken with the fast reciprocal (about 2
  // ulp; every stage of phi uses this one function, so results are
  // reproducible).  phi feeds the colour gradient and the near-contact scan
  // only; the component densities come from the sums themselves (densities).
  __device__ static __forceinline__ float phi_word(unsigned long long w) {
    const int lo = (int)(unsigned)w;
    const int hi = (int)(unsigned)(w >> 32) + (int)((unsigned)lo >> 31);  // undo the borrow of a negative low half
    return __fdividef((float)(hi - lo), (float)(hi + lo));
  }
  __device__ static __forceinline__ float phi(const unsigned long long* acc, size_t node) {
    return phi_word(acc[node]);
  }
  // rhoA and rhoB of a node, each rounded once
  __device__ static __forceinline__ void densities(const unsigned long long* acc, size_t node, float& a, float& b) {
    const unsigned long long w = acc[node];
    const int lo = (int)(unsigned)w;
    const int hi = (int)(unsigned)(w >> 32) + (int)((unsigned)lo >> 31);
    a = (float)hi * (1.0f / 268435456.0f);
    b = (float)lo * (1.0f / 268435456.0f);
  }
};
template <>
struct Acc<double> {
  static constexpr int W = 2;
  using S = long long;
  static constexpr double RHO_MAX = 64.0;
  __device__ static __forceinline__ S q(double v) { return __double2ll_rn(v * 72057594037927936.0); }
  // two planes of E shared words: rhoA at sw[e], rhoB at sw[E + e]
  __device__ static __forceinline__ void send_shared(unsigned long long* sw, int E, int e, double a, double b) {
    atomicAdd(sw + e, (unsigned long long)q(a));
    atomicAdd(sw + E + e, (unsigned long long)q(b));
  }
  __device__ static __forceinline__ void flush_shared(unsigned long long* acc, size_t node,
                                                      const unsigned long long* sw, int E, int e) {
    if (sw[e]) acc_red(acc + 2 * node, sw[e]);
    if (sw[E + e]) acc_red(acc + 2 * node + 1, sw[E + e]);
  }
  __device__ static __forceinline__ bool shared_zero(const unsigned long long* sw, int E, int e) {
    return (sw[e] | sw[E + e]) == 0ull;
  }
  __device__ static __forceinline__ void store(unsigned long long* acc, size_t node, S a, S b) {
    acc[2 * node] = (unsigned long long)a;
    acc[2 * node + 1] = (unsigned long long)b;
  }
  __device__ static __forceinline__ void zero(unsigned long long* acc, size_t node) {
    acc_st(acc + 2 * node, 0ull);
    acc_st(acc + 2 * node + 1, 0ull);
  }
  __device__ static __forceinline__ double phi_words(unsigned long long wa, unsigned long long wb) {
    const long long a = (long long)wa, b = (long long)wb;
    return (double)(a - b) / (double)(a + b);
  }
  __device__ static __forceinline__ double phi(const unsigned long long* acc, size_t node) {
    return phi_words(acc[2 * node], acc[2 * node + 1]);
  }
  __device__ static __forceinline__ void densities(const unsigned long long* acc, size_t node, double& a, double& b) {
    a = (double)(long long)acc[2 * node] * (1.0 / 72057594037927936.0);
    b = (double)(long long)acc[2 * node + 1] * (1.0 / 72057594037927936.0);
  }
};

// The integer sums of the component populations a node pulls (the same
// values, hence the same sums, as the senders accumulated).
template <int ST, bool WALLFREE, bool IDX32>
__device__ __forceinline__ void pull_acc(const View<ST>& S, const Geo& g, const Nbr& n, int self,
                                         typename Acc<typename Store<ST>::R>::S& sa,
                                         typename Acc<typename Store<ST>::R>::S& sb) {
  using R = typename Store<ST>::R;
  using A = Acc<R>;
  using I = typename std::conditional<IDX32, unsigned, size_t>::type;
  const I N = (I)g.N;
  sa = 0;
  sb = 0;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const int a = 1 - cx(i), b = 1 - cy(i), c = 1 - cz(i);
    const bool bb = WALLFREE ? false : (n.sx[a] | n.sy[b] | n.sz[c]);
    const I src = bb ? (I)self : (I)n.xs[a] + (I)g.nx * ((I)n.ys[b] + (I)g.ny * (I)n.zs[c]);
    const I dir = bb ? (I)opp(i) : (I)i;
    R va, vb;
    if constexpr (Store<ST>::TWOSET) {
      va = decode<ST>(S.f[dir * N + src], i);
      vb = decode<ST>(S.f[((I)Q + dir) * N + src], i);
    } else {
      const R fs = load_fs<ST, I>(S.f, N, dir, src, i, bb);
      colour_split<R, !WALLFREE>(fs, S.sv[src], i, bb, va, vb);
    }
    sa += A::q(va);
    sb += A::q(vb);
  }
}

// Rebuild the accumulator of the current time level from stored populations
// (after a checkpoint load or a state copy): one node per thread.
template <int ST, bool IDX32>
__global__ void __launch_bounds__(256) k_phi_acc(View<ST> S, Geo g, unsigned long long* __restrict__ acc) {
  using A = Acc<typename Store<ST>::R>;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < g.N; idx += stride) {
    const int x = (int)(idx % g.nx);
    const long long yz = idx / g.nx;
    const int y = (int)(yz % g.ny);
    const int z = (int)(yz / g.ny);
    if (is_solid(g, x, y, z)) {
      A::zero(acc, (size_t)idx);
      continue;
    }
    Nbr n;
    make_nbr(g, x, y, z, n);
    typename A::S sa, sb;
    if (near_wall(g, x, y, z))
      pull_acc<ST, false, IDX32>(S, g, n, (int)idx, sa, sb);
    else
      pull_acc<ST, true, IDX32>(S, g, n, (int)idx, sa, sb);
    A::store(acc, (size_t)idx, sa, sb);
  }
}

// ---------------------------------------------------------------------------
// shared-memory layout of a tile
// ---------------------------------------------------------------------------
// phi of the tile plus a halo of H nodes (HX along x: 1 without near
// contact, else H rounded up to a multiple of 4 so that rows start on 16-byte
// vectors), the component partial sums over the tile plus a one-node ring,
// and with near contact the scan queue, the distance h of each tile node and
// the queue counter.
constexpr size_t align16(size_t b) { return (b + 15) / 16 * 16; }

template <typename R, int TX, int TY, int TZ, int H, int NPH = 1, bool QH = true>
struct Layout {
  static constexpr int HX = H == 1 ? 1 : (H + 3) / 4 * 4;
  static constexpr int SX = TX + 2 * HX, SY = TY + 2 * H, SZ = TZ + 2 * H, SXY = SX * SY, NS = SXY * SZ;
  static constexpr int EX = TX + 2, EY = TY + 2, EZ = TZ + 2, EXY = EX * EY, E = EXY * EZ;
  static constexpr int NT = TX * TY * TZ;
  // NPH staged scalar fields of NS values each (phi; the Shan-Chen model
  // adds psi_A and psi_B)
  static constexpr size_t off_acc = align16(sizeof(R) * (size_t)NS * NPH);
  // the scan's queue and h (QH: a tile that scans in its own phase)
  static constexpr size_t off_queue = off_acc + align16(8 * (size_t)Acc<R>::W * (size_t)E);
  static constexpr size_t off_h = off_queue + (H > 1 && QH ? align16(2 * (size_t)NT) : 0);
  static constexpr size_t off_count = off_h + (H > 1 && QH ? align16((size_t)NT) : 0);
  static constexpr size_t bytes = off_count + 16;
};

template <typename R, bool FROM_ACC>
struct PhiLoad {
  // nodes per 16-byte vector
  static constexpr int V = FROM_ACC ? 16 / (8 * Acc<R>::W) : 16 / (int)sizeof(R);
  using Raw = typename std::conditional<FROM_ACC, ulonglong2,
                                        typename std::conditional<sizeof(R) == 4, float4, double2>::type>::type;
  __device__ static __forceinline__ R one(const PhiSrc& s, size_t node) {
    if constexpr (FROM_ACC) return Acc<R>::phi(s.acc, node);
    else return reinterpret_cast<const R*>(s.phi)[node];
  }
  // the V consecutive nodes from `node` (a multiple of V) as one load ...
  __device__ static __forceinline__ Raw ld(const PhiSrc& s, size_t node) {
    if constexpr (FROM_ACC) return acc_ld2(s.acc + Acc<R>::W * node);
    else return *reinterpret_cast<const Raw*>(reinterpret_cast<const R*>(s.phi) + node);
  }
  // ... and their phi
  __device__ static __forceinline__ void dec(const Raw& w, R* out) {
    if constexpr (FROM_ACC) {
      if constexpr (Acc<R>::W == 1) {
        out[0] = Acc<float>::phi_word(w.x);
        out[1] = Acc<float>::phi_word(w.y);
      } else {
        out[0] = Acc<double>::phi_words(w.x, w.y);
      }
    } else {
      const R* r = reinterpret_cast<const R*>(&w);
#pragma unroll
      for (int j = 0; j < V; ++j) out[j] = r[j];
    }
  }
};

// Stage phi of the tile plus its halo (Layout) in shared memory; solid and
// beyond-wall nodes get the marker PHI_SOLID, periodic axes wrap.  The block
// is walked as one flat list (of 16-byte vectors when the rows allow it), so
// no lane idles on a short row.  No barrier.
template <typename R, bool FROM_ACC, int TX, int TY, int TZ, int H>
__device__ __forceinline__ void stage_phi(const PhiSrc& src, const Geo& g, R* sp, int x0, int y0, int z0) {
  using L = Layout<R, TX, TY, TZ, H>;
  using PL = PhiLoad<R, FROM_ACC>;
  constexpr int V = PL::V;
  const int tid = threadIdx.y * TX + threadIdx.x;
  if constexpr (H > 1) {
    static_assert(L::HX % V == 0 && TX % V == 0, "vector staging needs whole vectors per row");
  }
  if (H > 1 && g.nx % V == 0) {
    // every vector lies wholly inside or wholly outside the box along x; NB
    // vectors per thread are loaded before any is decoded, so their latencies
    // overlap
    constexpr int QR = (H > 1 ? L::SX : V) / V, NQ = QR * L::SY * L::SZ, NB = 4;
    using Raw = typename PL::Raw;
    for (int q0 = tid; q0 < NQ; q0 += NB * TX * TY) {
      Raw raw[NB];
      int meta[NB];  // row * QR + qx, or -1 beyond the block
      unsigned fill = 0;  // bit b: vector b is solid or beyond a wall (no load)
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        const int q = q0 + b * TX * TY;
        meta[b] = -1;
        if (q >= NQ) continue;
        meta[b] = q;
        const int qx = q % QR, row = q / QR;
        const int ly = row % L::SY, lz = row / L::SY;
        int gy = y0 - H + ly, gz = z0 - H + lz;
        bool rsolid = false;
        if (g.wy) rsolid |= (gy <= 0 || gy >= g.ny - 1);
        else if ((unsigned)gy >= (unsigned)g.ny) gy = ((gy % g.ny) + g.ny) % g.ny;
        if (g.wz) rsolid |= (gz <= 0 || gz >= g.nz - 1);
        else if ((unsigned)gz >= (unsigned)g.nz) gz = ((gz % g.nz) + g.nz) % g.nz;
        const int gx0 = x0 - L::HX + qx * V;
        bool inside = gx0 >= 0 && gx0 < g.nx;
        int gxl = gx0;
        if (!inside && !g.wx) {
          gxl = ((gx0 % g.nx) + g.nx) % g.nx;
          inside = true;
        }
        if (inside && !rsolid) raw[b] = PL::ld(src, (size_t)gxl + (size_t)g.nx * ((size_t)gy + (size_t)g.ny * gz));
        else fill |= 1u << b;
        if (rsolid) fill |= 1u << (NB + b);
      }
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        if (meta[b] < 0) continue;
        const int qx = meta[b] % QR, row = meta[b] / QR;
        R v[V];
        if ((fill >> b) & 1u) {
#pragma unroll
          for (int j = 0; j < V; ++j) v[j] = R(PHI_SOLID);
        } else {
          PL::dec(raw[b], v);
        }
        const bool rsolid = (fill >> (NB + b)) & 1u;
        const int gx0 = x0 - L::HX + qx * V;
        R* dst = sp + (size_t)row * L::SX + qx * V;
#pragma unroll
        for (int j = 0; j < V; ++j) {
          const int xj = gx0 + j;
          const bool solid = rsolid || (g.wx && (xj <= 0 || xj >= g.nx - 1));
          dst[j] = solid ? R(PHI_SOLID) : v[j];
        }
      }
    }
  } else {
    for (int q = tid; q < L::NS; q += TX * TY) {
      const int lx = q % L::SX, row = q / L::SX;
      const int ly = row % L::SY, lz = row / L::SY;
      int gx = x0 - L::HX + lx, gy = y0 - H + ly, gz = z0 - H + lz;
      bool solid = false;
      if (g.wx) solid |= (gx <= 0 || gx >= g.nx - 1);
      else if ((unsigned)gx >= (unsigned)g.nx) gx = ((gx % g.nx) + g.nx) % g.nx;
      if (g.wy) solid |= (gy <= 0 || gy >= g.ny - 1);
      else if ((unsigned)gy >= (unsigned)g.ny) gy = ((gy % g.ny) + g.ny) % g.ny;
      if (g.wz) solid |= (gz <= 0 || gz >= g.nz - 1);
      else if ((unsigned)gz >= (unsigned)g.nz) gz = ((gz % g.nz) + g.nz) % g.nz;
      sp[q] = solid ? R(PHI_SOLID) : PL::one(src, (size_t)gx + (size_t)g.nx * ((size_t)gy + (size_t)g.ny * gz));
    }
  }
}

// ---------------------------------------------------------------------------
// colour gradient and near-contact scan on the staged tile
// ---------------------------------------------------------------------------
// Colour gradient grad phi(p) = (1/cs2) sum_i w_i c_i phi(p + c_i) on the
// shared tile; a solid neighbour contributes phi(p) (neutral wetting).  Tiles
// whose halo holds no solid node skip the solid test (WALLFREE).  The D3Q27
// weights factor: for c_a = +-1, w(c) = v(c_b) v(c_c) / 216 with v(0) = 4,
// v(+-1) = 1 on the two other axes, so each component is the central
// difference along its axis smoothed by (1, 4, 1) x (1, 4, 1) across the
// others, times 3/216 = 1/72.  Evaluated one z plane of the 3x3x3 block at a
// time.
template <typename R, bool WALLFREE>
__device__ __forceinline__ void tile_grad(const R* sp, int c, int SX, int SXY, R gr[3]) {
  const R p0 = sp[c];
  R gx = R(0), gy = R(0), gz = R(0);
#pragma unroll
  for (int dz = -1; dz <= 1; ++dz) {
    R p[3][3];
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy) {
#pragma unroll
      for (int dx = -1; dx <= 1; ++dx) {
        if (dz == 0 && dy == 0 && dx == 0) {
          p[1][1] = p0;
          continue;
        }
        R v = sp[c + dx + SX * dy + SXY * dz];
        if constexpr (!WALLFREE) v = (v > R(0.5) * R(PHI_SOLID)) ? p0 : v;
        p[dy + 1][dx + 1] = v;
      }
    }
    // x differences smoothed over y, y differences smoothed over x
    const R ex = (p[0][2] - p[0][0]) + (p[2][2] - p[2][0]) + R(4) * (p[1][2] - p[1][0]);
    const R ey = (p[2][0] - p[0][0]) + (p[2][2] - p[0][2]) + R(4) * (p[2][1] - p[0][1]);
    if (dz == 0) {
      gx += R(4) * ex;
      gy += R(4) * ey;
    } else {
      gx += ex;
      gy += ey;
      // the plane smoothed over x and y enters the z difference
      const R sm = (p[0][0] + p[0][2] + R(4) * p[0][1]) + (p[2][0] + p[2][2] + R(4) * p[2][1]) +
                   R(4) * (p[1][0] + p[1][2] + R(4) * p[1][1]);
      gz += dz > 0 ? sm : -sm;
    }
  }
  constexpr R k72 = R(1) / R(72);
  gr[0] = gx * k72;
  gr[1] = gy * k72;
  gr[2] = gz * k72;
}

// Near-contact scan of one interface node (Eqs. stress_jump, near_cont_force):
// step along the outward normal n_out = -grad phi/|grad phi| by round(k n_out),
// k = 1..K; the first target that is an interface node (|phi| < phi_I,
// |grad phi| >= NC_GRAD_MIN) with a normal antiparallel to the node's own
// gives h = k; 0 when there is none.  The scan stops at a wall layer.  sp is
// the phi tile with a halo of at least K + 1, c the node's tile index, gr and
// gg = |gr| its gradient.
template <typename R, bool WALLFREE>
__device__ __forceinline__ int nc_scan(const R* sp, int c, int SX, int SXY, int K, int x, int y, int z, const Geo& g,
                                       const Phys& P, const R gr[3], R gg) {
  const R phi_I = R(P.phi_I);
  const R inv = R(-1) / gg;
  const R no0 = gr[0] * inv, no1 = gr[1] * inv, no2 = gr[2] * inv;
#pragma unroll 1
  for (int k = 1; k <= K; ++k) {
    // |n_out| = 1, so |d| <= k <= K; the clamp also covers non-finite normals
    const int dx = max(-k, min(k, (int)round_(R(k) * no0)));
    const int dy = max(-k, min(k, (int)round_(R(k) * no1)));
    const int dz = max(-k, min(k, (int)round_(R(k) * no2)));
    if constexpr (!WALLFREE) {
      if (g.wx && (x + dx <= 0 || x + dx >= g.nx - 1)) break;
      if (g.wy && (y + dy <= 0 || y + dy >= g.ny - 1)) break;
      if (g.wz && (z + dz <= 0 || z + dz >= g.nz - 1)) break;
    }
    const int ct = c + dx + SX * dy + SXY * dz;
    if (!(fabs(sp[ct]) < phi_I)) continue;
    R gt[3];
    tile_grad<R, WALLFREE>(sp, ct, SX, SXY, gt);
    const R gm2 = gt[0] * gt[0] + gt[1] * gt[1] + gt[2] * gt[2];
    if (gm2 < R(NC_GRAD_MIN) * R(NC_GRAD_MIN)) continue;
    const R dot = gr[0] * gt[0] + gr[1] * gt[1] + gr[2] * gt[2];
    if (dot < -R(NC_COS_TOL) * gg * sqrt_(gm2)) return k;
  }
  return 0;
}

// Near-contact distance of every node of the tile into hs (Layout::NT bytes,
// 0 for nodes without a partner): queue the tile's interface nodes (|phi| <
// phi_I; solid nodes hold PHI_SOLID and are never queued) by warp-aggregated
// appends, then all threads take queue entries in turn, so no lane idles on a
// bulk node.  The counter was cleared before the staging barrier.  Ends with
// a barrier.
template <typename R, int TX, int TY, int TZ, int H, bool WALLFREE>
__device__ __forceinline__ void nc_tile(const R* sp, const Geo& g, const Phys& P, unsigned char* hs,
                                        unsigned short* queue, int* count, int x0, int y0, int z0) {
  using L = Layout<R, TX, TY, TZ, H>;
  const int tid = threadIdx.y * TX + threadIdx.x;
  const int lane = tid & 31;
  const R phi_I = R(P.phi_I);
  for (int lz = 0; lz < TZ; ++lz) {
    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y, z = z0 + lz;
    const bool in = x < g.nx && y < g.ny && z < g.nz;
    const int o = (lz * TY + threadIdx.y) * TX + threadIdx.x;
    const int c = (lz + H) * L::SXY + (threadIdx.y + H) * L::SX + (threadIdx.x + L::HX);
    const bool iface = in && fabs(sp[c]) < phi_I;
    hs[o] = 0;
    const unsigned m = __ballot_sync(0xffffffffu, iface);
    if (m) {
      const int leader = __ffs(m) - 1;
      int base = 0;
      if (lane == leader) base = atomicAdd(count, __popc(m));
      base = __shfl_sync(0xffffffffu, base, leader);
      if (iface) queue[base + __popc(m & ((1u << lane) - 1u))] = (unsigned short)o;
    }
  }
  __syncthreads();
  const int n = *count;
  for (int q = tid; q < n; q += TX * TY) {
    const int o = queue[q];
    const int lx = o % TX, ly = (o / TX) % TY, lz = o / (TX * TY);
    const int c = (lz + H) * L::SXY + (ly + H) * L::SX + (lx + L::HX);
    R gr[3];
    tile_grad<R, WALLFREE>(sp, c, L::SX, L::SXY, gr);
    const R gg = sqrt_(gr[0] * gr[0] + gr[1] * gr[1] + gr[2] * gr[2]);
    int h = 0;
    if (gg >= R(NC_GRAD_MIN))
      h = nc_scan<R, WALLFREE>(sp, c, L::SX, L::SXY, P.K, x0 + lx, y0 + ly, z0 + lz, g, P, gr, gg);
    hs[o] = (unsigned char)h;
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// the nodes of one tile
// ---------------------------------------------------------------------------
// Send the component populations (a, b) of direction i of the node at
// accumulator index e0 to the node that pulls them: x + c_i, or the node
// itself when x + c_i is solid (halfway bounce-back).
template <typename R, bool WALLFREE, int EX, int EXY, int E>
__device__ __forceinline__ void send(unsigned long long* sw, int e0, const Nbr& n, int i, R a, R b) {
  int e = e0 + cx(i) + EX * cy(i) + EXY * cz(i);
  if constexpr (!WALLFREE) {
    if (n.sx[1 + cx(i)] | n.sy[1 + cy(i)] | n.sz[1 + cz(i)]) e = e0;
  }
  Acc<R>::send_shared(sw, E, e, a, b);
}

// Pull, collide, recolour and store every node of the tile; with WS also
// send the post-collision component populations to the tile's partial sums.
// sp holds phi of the tile and its halo (Layout), hs the near-contact
// distance of each tile node (read when A_h != 0).
// INL: the near-contact scan of an interface node runs here, between the
// loads and the sums of its pull, instead of in a separate phase of the tile
// (same h: the same scan from the same gradient).  zero_acc (non-null): the
// accumulator two steps ahead, zeroed here node by node.
template <int ST, int LOADER, bool WS, bool WF, int TX, int TY, int TZ, int H, bool WALLFREE, bool IDX32, bool REG,
          bool INL = false>
__device__ __forceinline__ void step_nodes(const View<ST>& S, const View<ST>& O, const InitBuf& init, const Geo& g,
                                           const Phys& P, const unsigned char* hs,
                                           typename Store<ST>::R* __restrict__ fields,
                                           unsigned* __restrict__ status, const typename Store<ST>::R* sp,
                                           unsigned long long* sw, const unsigned long long* __restrict__ accin,
                                           int x0, int y0, int z0, unsigned long long* __restrict__ zero_acc = nullptr) {
  using R = typename Store<ST>::R;
  using L = Layout<R, TX, TY, TZ, H>;
  using I = typename std::conditional<IDX32, unsigned, size_t>::type;
  const R tau_a = R(P.tau_a), tau_b = R(P.tau_b);
  const R A2 = R(P.A2), beta = R(P.beta), A_h = R(P.A_h);
  const I N = (I)g.N;
  const size_t NF = (size_t)g.N;

  for (int lz = 0; lz < TZ; ++lz) {
    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y, z = z0 + lz;
    if (x >= g.nx || y >= g.ny || z >= g.nz) continue;
    const int self = x + g.nx * (y + g.ny * z);
    if (zero_acc) Acc<R>::zero(zero_acc, (size_t)self);  // the accumulator two steps ahead
    if (!WALLFREE && is_solid(g, x, y, z)) {
      if constexpr (WF) {
        for (int k = 0; k < NFIELDS; ++k) fields[(size_t)k * NF + self] = R(0);
      }
      continue;
    }
    Nbr n;
    make_nbr(g, x, y, z, n);
    R f[Q], rA, rB;
    const int c = (lz + H) * L::SXY + (threadIdx.y + H) * L::SX + (threadIdx.x + L::HX);
    const int e0 = (lz + 1) * L::EXY + (threadIdx.y + 1) * L::EX + (threadIdx.x + 1);
    const R phx = sp[c];
    // colour gradient from the tile; near-contact distance from the scan
    R gr[3], gg;
    int h = 0;
    constexpr bool SPLIT = INL && LOADER == LOAD_PULL && !Store<ST>::MOMENT;
    if constexpr (SPLIT) {
      typename Store<ST>::E ra[Q], rb[Q];
      pull_raw<ST, WALLFREE, IDX32>(S, g, n, self, ra, rb);
      tile_grad<R, WALLFREE>(sp, c, L::SX, L::SXY, gr);
      gg = sqrt_(gr[0] * gr[0] + gr[1] * gr[1] + gr[2] * gr[2]);
      if (H > 1 && A_h != R(0) && fabs(phx) < R(P.phi_I) && gg >= R(NC_GRAD_MIN))
        h = nc_scan<R, WALLFREE>(sp, c, L::SX, L::SXY, P.K, x, y, z, g, P, gr, gg);
      pull_raw_finish<ST>(ra, rb, f, rA, rB);
    }
    if constexpr (SPLIT && Store<ST>::TWOSET) {
      // pulled and summed above
    } else if constexpr (LOADER == LOAD_PULL) {
      if constexpr (Store<ST>::TWOSET) {
        pull_fast<ST, WALLFREE, IDX32, false>(S, g, n, self, f, rA, rB);
      } else {
        // single set: rhoA of the node is the sum the senders accumulated
        // (what a pull of the rebuilt f^A_i gives), so the neighbours' colour
        // scalars need not be read
        if constexpr (!SPLIT) pull_fast<ST, WALLFREE, IDX32, true>(S, g, n, self, f, rA, rB);
        R rt = R(0);
#pragma unroll
        for (int i = 0; i < Q; ++i) rt += f[i];
        if (accin) {
          Acc<R>::densities(accin, (size_t)self, rA, rB);
        } else {  // phi given as an array: split the pulled total by it
          rA = R(0.5) * rt * (R(1) + phx);
        }
        rB = rt - rA;  // rho is the sum of the pulled totals, as for the momentum
      }
    } else {
      fields_node<R, false>(init, g, P, n, (long long)self, f, rA, rB, nullptr, nullptr);
    }

    // moments (Sec. III.C.1): rho = rhoA + rhoB, j = sum_i f_i c_i taken over
    // opposite pairs (p, 26-p), p = 0..12
    const R rho = rA + rB;
    R j0 = R(0), j1 = R(0), j2 = R(0);
#pragma unroll
    for (int p = 0; p < REST; ++p) {
      const R d = f[p] - f[opp(p)];
      if (cx(p)) j0 += R(cx(p)) * d;
      if (cy(p)) j1 += R(cy(p)) * d;
      if (cz(p)) j2 += R(cz(p)) * d;
    }

    if constexpr (!SPLIT) {
      tile_grad<R, WALLFREE>(sp, c, L::SX, L::SXY, gr);
      gg = sqrt_(gr[0] * gr[0] + gr[1] * gr[1] + gr[2] * gr[2]);
      if (H > 1 && A_h != R(0)) {
        if constexpr (INL) {
          if (fabs(phx) < R(P.phi_I) && gg >= R(NC_GRAD_MIN))
            h = nc_scan<R, WALLFREE>(sp, c, L::SX, L::SXY, P.K, x, y, z, g, P, gr, gg);
        } else {
          h = hs[(lz * TY + threadIdx.y) * TX + threadIdx.x];
        }
      }
    }
    R Ahh = R(0);
    if (H > 1 && A_h != R(0)) {
      if (h > 0) {
        const R hk = R(h);
        if (hk <= R(P.h_min)) Ahh = A_h;
        else if (hk <= R(P.h_max)) {
          const R q = R(P.h_min) / hk;
          Ahh = A_h * q * q * q;
        }
      }
    }
    // F_rep = -A_h n_out delta_I, delta_I = |grad phi|/2  ->  (A_h/2) grad phi
    const R Fr0 = R(0.5) * Ahh * gr[0], Fr1 = R(0.5) * Ahh * gr[1], Fr2 = R(0.5) * Ahh * gr[2];
    R F0 = Fr0, F1 = Fr1, F2 = Fr2;
    if (P.g_mode == 1) {
      F0 += rho * R(P.g[0]);
      F1 += rho * R(P.g[1]);
      F2 += rho * R(P.g[2]);
    } else if (P.g_mode == 2) {
      const R sg = (z == 0 || 2 * z == g.nz) ? R(0) : (2 * z < g.nz ? R(1) : R(-1));
      F0 += sg * rA * R(P.g[0]);
      F1 += sg * rA * R(P.g[1]);
      F2 += sg * rA * R(P.g[2]);
    }

    // Guo-shifted velocity
    const R irho = R(1) / rho;
    const R u0 = (j0 + R(0.5) * F0) * irho, u1 = (j1 + R(0.5) * F1) * irho, u2 = (j2 + R(0.5) * F2) * irho;
    // a density outside (0, RHO_MAX), or not finite, marks the run unstable
    if (!(rho > R(0) && rho < R(Acc<R>::RHO_MAX))) atomicOr(status, 1u);

    if constexpr (WF) {
      fields[(size_t)F_PHI * NF + self] = phx;
      fields[(size_t)F_RHO * NF + self] = rho;
      fields[(size_t)F_UX * NF + self] = u0;
      fields[(size_t)F_UY * NF + self] = u1;
      fields[(size_t)F_UZ * NF + self] = u2;
      fields[(size_t)F_RHOA * NF + self] = rA;
      fields[(size_t)F_RHOB * NF + self] = rB;
      fields[(size_t)F_FRX * NF + self] = Fr0;
      fields[(size_t)F_FRY * NF + self] = Fr1;
      fields[(size_t)F_FRZ * NF + self] = Fr2;
      fields[(size_t)F_H * NF + self] = R(h);
      fields[(size_t)F_GX * NF + self] = gr[0];
      fields[(size_t)F_GY * NF + self] = gr[1];
      fields[(size_t)F_GZ * NF + self] = gr[2];
    }
    if constexpr (!WS) continue;

    // mixture relaxation time (harmonic nu_bar, Eq. sigmaA)
    R tau;
    if (P.equal_tau) {
      tau = tau_a;
    } else {
      const R nu_a = (tau_a - R(0.5)) / R(3), nu_b = (tau_b - R(0.5)) / R(3);
      const R nu = R(1) / ((rA * irho) / nu_a + (rB * irho) / nu_b);
      tau = R(3) * nu + R(0.5);
    }
    const R omega = R(1) / tau;
    const R keep = R(1) - omega;
    const R guo = R(1) - R(0.5) * omega;
    const R uu = u0 * u0 + u1 * u1 + u2 * u2;
    const R uF = u0 * F0 + u1 * F1 + u2 * F2;
    // perturbation: (A_a+A_b)/2 |g| [w (c.n)^2 - B] = A2 [w (c.grad)^2/|g| - |g| B]
    const bool pert = gg >= R(GRAD_EPS);
    const R A2g = pert ? A2 * gg : R(0);
    const R A2ig = pert ? A2 / gg : R(0);
    // recolouring segregation amplitude beta rhoA rhoB / rho with the normal
    // grad phi / max(|grad phi|, floor)
    const R gn = gg > R(NORMAL_FLOOR) ? gg : R(NORMAL_FLOOR);
    const R segamp = beta * rA * rB * irho / gn;
    const R sA = rA * irho;
    // equilibrium (Eq. disteq) and Guo source split into parts even and odd
    // under c -> -c: feq = w [rho(1 - 1.5 uu) + 4.5 rho (c.u)^2] + 3 w rho (c.u),
    // S = guo w [9 (c.u)(c.F) - 3 u.F] + 3 guo w (c.F)
    const R r0 = rho * (R(1) - R(1.5) * uu);
    const R r45 = R(4.5) * rho;
    const R r3 = R(3) * rho;
    const R g9 = R(9) * guo, g3 = R(3) * guo, gm3uF = -R(3) * guo * uF;
    // BGK relaxes f towards feq: keep f + omega feq.  The regularised
    // collision (collision == 1) keeps feq and relaxes the non-equilibrium
    // part projected on Hermite orders 1 and 2:
    //   feq + keep w [3 c.J + 4.5 (c.Pi.c - tr(Pi)/3)],
    //   J = j - rho u = -F/2,  Pi = sum_i c c f_i - rho (u u + I/3).
    constexpr bool reg = REG;
    const R wf = reg ? R(1) : omega;
    R Pxx = R(0), Pyy = R(0), Pzz = R(0), Pxy = R(0), Pxz = R(0), Pyz = R(0), trP = R(0);
    if constexpr (reg) {
#pragma unroll
      for (int p = 0; p < REST; ++p) {
        const R sp2 = f[p] + f[opp(p)];
        if (cx(p)) Pxx += sp2;
        if (cy(p)) Pyy += sp2;
        if (cz(p)) Pzz += sp2;
        if (cx(p) && cy(p)) Pxy += R(cx(p) * cy(p)) * sp2;
        if (cx(p) && cz(p)) Pxz += R(cx(p) * cz(p)) * sp2;
        if (cy(p) && cz(p)) Pyz += R(cy(p) * cz(p)) * sp2;
      }
      const R r3rd = rho * (R(1) / R(3));
      Pxx -= rho * u0 * u0 + r3rd;
      Pyy -= rho * u1 * u1 + r3rd;
      Pzz -= rho * u2 * u2 + r3rd;
      Pxy -= rho * u0 * u1;
      Pxz -= rho * u0 * u2;
      Pyz -= rho * u1 * u2;
      trP = Pxx + Pyy + Pzz;
    }
    // colour scalars of the single-set storages, as stored
    float4 svo = make_float4(0.f, 0.f, 0.f, 0.f);
    if constexpr (!Store<ST>::TWOSET) {
      svo = make_float4(sA, segamp * gr[0], segamp * gr[1], segamp * gr[2]);
      O.sv[self] = svo;
    }
    if constexpr (Store<ST>::MOMENT) {
      // f*_i = w_i (alpha + beta.c_i + c_i.Gamma.c_i): the equilibrium, the
      // relaxed Hermite orders 1-2, the perturbation (B_i = w_i (|c_i|^2 - 2/3))
      // and the Guo source below are each w_i times a quadratic form in c_i
      // (Eqs. disteq, distnoneq, LBpostmom; the host admits this storage with
      // the regularised collision only)
      const R kP = keep * R(4.5), hg9 = R(0.5) * g9;
      const R bF = g3 - R(1.5) * keep;  // beta = 3 rho u + (3 guo - 1.5 keep) F
      const float4 qa = make_float4(r0 + gm3uF - R(1.5) * keep * trP + (R(2) / R(3)) * A2g, r3 * u0 + bF * F0,
                                    r3 * u1 + bF * F1, r3 * u2 + bF * F2);
      const float4 qb = make_float4(r45 * u0 * u0 + g9 * u0 * F0 + A2ig * gr[0] * gr[0] - A2g + kP * Pxx,
                                    r45 * u1 * u1 + g9 * u1 * F1 + A2ig * gr[1] * gr[1] - A2g + kP * Pyy,
                                    r45 * u2 * u2 + g9 * u2 * F2 + A2ig * gr[2] * gr[2] - A2g + kP * Pzz,
                                    R(2) * (r45 * u0 * u1 + hg9 * (u0 * F1 + F0 * u1) + A2ig * gr[0] * gr[1] + kP * Pxy));
      const float2 qc =
          make_float2(R(2) * (r45 * u0 * u2 + hg9 * (u0 * F2 + F0 * u2) + A2ig * gr[0] * gr[2] + kP * Pxz),
                      R(2) * (r45 * u1 * u2 + hg9 * (u1 * F2 + F1 * u2) + A2ig * gr[1] * gr[2] + kP * Pyz));
      reinterpret_cast<float4*>(O.f)[self] = qa;
      reinterpret_cast<float4*>(O.f + (I)4 * N)[self] = qb;
      reinterpret_cast<float2*>(O.f + (I)8 * N)[self] = qc;
      // what the neighbours will pull: the quadratic form at each c_i
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        R va, vb;
        colour_split<R, false>(eval_moment<R>(qa, qb, qc, i, false), svo, i, false, va, vb);
        send<R, WALLFREE, L::EX, L::EXY, L::E>(sw, e0, n, i, va, vb);
      }
      continue;
    }
    {  // rest direction
      const R W = wgt<R>(REST);
      const R rel = reg ? R(-1.5) * W * trP : f[REST];
      const R fs = keep * rel + wf * W * r0 - bweight<R>(REST) * A2g + W * gm3uF;
      if constexpr (Store<ST>::TWOSET) {
        const R fa = sA * fs;
        const R fb = fs - fa;
        O.f[(I)REST * N + (I)self] = encode<ST>(fa, REST);
        O.f[(I)(Q + REST) * N + (I)self] = encode<ST>(fb, REST);
        send<R, WALLFREE, L::EX, L::EXY, L::E>(sw, e0, n, REST, fa, fb);
      } else {
        const typename Store<ST>::E enc = encode<ST>(fs, REST);
        O.f[(I)REST * N + (I)self] = enc;
        R va, vb;
        colour_split<R, false>(decode<ST>(enc, REST), svo, REST, false, va, vb);
        send<R, WALLFREE, L::EX, L::EXY, L::E>(sw, e0, n, REST, va, vb);
      }
    }
#pragma unroll
    for (int p = 0; p < REST; ++p) {
      const int q = opp(p);
      const R W = wgt<R>(p);
      R cu = R(0), cF = R(0), cg = R(0);
      if (cx(p)) { cu += R(cx(p)) * u0; cF += R(cx(p)) * F0; cg += R(cx(p)) * gr[0]; }
      if (cy(p)) { cu += R(cy(p)) * u1; cF += R(cy(p)) * F1; cg += R(cy(p)) * gr[1]; }
      if (cz(p)) { cu += R(cz(p)) * u2; cF += R(cz(p)) * F2; cg += R(cz(p)) * gr[2]; }
      R even = W * (wf * (r0 + r45 * cu * cu) + g9 * cu * cF + gm3uF + A2ig * cg * cg) - bweight<R>(p) * A2g;
      R odd = W * (wf * r3 * cu + g3 * cF);
      R bp = f[p], bq = f[q];
      if constexpr (reg) {
        // c.Pi.c and c.J = -(c.F)/2 for this pair's velocity
        R cpc = R(0);
        if (cx(p)) cpc += Pxx;
        if (cy(p)) cpc += Pyy;
        if (cz(p)) cpc += Pzz;
        if (cx(p) && cy(p)) cpc += R(2 * cx(p) * cy(p)) * Pxy;
        if (cx(p) && cz(p)) cpc += R(2 * cx(p) * cz(p)) * Pxz;
        if (cy(p) && cz(p)) cpc += R(2 * cy(p) * cz(p)) * Pyz;
        even += keep * W * R(4.5) * (cpc - trP * (R(1) / R(3)));
        odd += keep * W * R(-1.5) * cF;
        bp = R(0);
        bq = R(0);
      }
      const R fsp = keep * bp + even + odd;
      const R fsq = keep * bq + even - odd;
      if constexpr (Store<ST>::TWOSET) {
        const R seg = segamp * W * inv_norm<R>(p) * cg;
        const R fap = sA * fsp + seg;
        const R faq = sA * fsq - seg;
        const R fbp = fsp - fap, fbq = fsq - faq;
        O.f[(I)p * N + (I)self] = encode<ST>(fap, p);
        O.f[(I)q * N + (I)self] = encode<ST>(faq, q);
        O.f[(I)(Q + p) * N + (I)self] = encode<ST>(fbp, p);
        O.f[(I)(Q + q) * N + (I)self] = encode<ST>(fbq, q);
        send<R, WALLFREE, L::EX, L::EXY, L::E>(sw, e0, n, p, fap, fbp);
        send<R, WALLFREE, L::EX, L::EXY, L::E>(sw, e0, n, q, faq, fbq);
      } else {
        const typename Store<ST>::E ep = encode<ST>(fsp, p), eq = encode<ST>(fsq, q);
        O.f[(I)p * N + (I)self] = ep;
        O.f[(I)q * N + (I)self] = eq;
        // colour_split of p and of its opposite q: c_q.v = -(c_p.v) exactly,
        // so the segregation term is formed once and negated (bit for bit
        // what colour_split gives for q)
        R cv = R(0);
        if (cx(p)) cv += R(cx(p)) * R(svo.y);
        if (cy(p)) cv += R(cy(p)) * R(svo.z);
        if (cz(p)) cv += R(cz(p)) * R(svo.w);
        const R seg = mul_rn(W * inv_norm<R>(p), cv);
        const R dp = decode<ST>(ep, p), dq = decode<ST>(eq, q);
        const R vap = fma_rn(R(svo.x), dp, seg), vaq = fma_rn(R(svo.x), dq, -seg);
        send<R, WALLFREE, L::EX, L::EXY, L::E>(sw, e0, n, p, vap, dp - vap);
        send<R, WALLFREE, L::EX, L::EXY, L::E>(sw, e0, n, q, vaq, dq - vaq);
      }
    }
  }
}

// Add the tile's partial sums (tile plus a one-node ring) to the global
// accumulator; entries beyond a wall are never sent to, periodic axes wrap.
template <typename R, int TX, int TY, int TZ, int H>
__device__ __forceinline__ void flush_partials(const unsigned long long* sw, unsigned long long* __restrict__ acc,
                                               const Geo& g, int x0, int y0, int z0) {
  using L = Layout<R, TX, TY, TZ, H>;
  for (int e = threadIdx.y * TX + threadIdx.x; e < L::E; e += TX * TY) {
    if (Acc<R>::shared_zero(sw, L::E, e)) continue;
    const int ex = e % L::EX, ey = (e / L::EX) % L::EY, ez = e / L::EXY;
    int gx = x0 - 1 + ex, gy = y0 - 1 + ey, gz = z0 - 1 + ez;
    if ((unsigned)gx >= (unsigned)g.nx) {
      if (g.wx) continue;
      gx = ((gx % g.nx) + g.nx) % g.nx;
    }
    if ((unsigned)gy >= (unsigned)g.ny) {
      if (g.wy) continue;
      gy = ((gy % g.ny) + g.ny) % g.ny;
    }
    if ((unsigned)gz >= (unsigned)g.nz) {
      if (g.wz) continue;
      gz = ((gz % g.nz) + g.nz) % g.nz;
    }
    Acc<R>::flush_shared(acc, (size_t)gx + (size_t)g.nx * ((size_t)gy + (size_t)g.ny * gz), sw, L::E, e);
  }
}

// ---------------------------------------------------------------------------
// Shan-Chen multicomponent model (Sec. III.C.3, lattice pseudo-potential)
// ---------------------------------------------------------------------------
__device__ __forceinline__ float sc_psi(float r, float psi0) { return psi0 * (1.0f - expf(-r / psi0)); }
__device__ __forceinline__ double sc_psi(double r, double psi0) { return psi0 * (1.0 - exp(-r / psi0)); }

// Stage phi, psi_A and psi_B (pseudo-potential psi(rho) = rho_0 (1 -
// exp(-rho/rho_0)) of each component) of the tile plus a one-node halo; solid
// and beyond-wall nodes get the marker.  The component densities come from
// the accumulator of the step before, or (first step) from the initial
// fields: rho_k = rho (1 +- phi)/2.  No barrier.
template <typename R, bool FROM_ACC, int TX, int TY, int TZ>
__device__ __forceinline__ void stage_sc(const PhiSrc& src, const InitBuf& init, const Geo& g, R psi0, R* sp,
                                         R* spa, R* spb, int x0, int y0, int z0) {
  using L = Layout<R, TX, TY, TZ, 1, 3>;
  for (int q = threadIdx.y * TX + threadIdx.x; q < L::NS; q += TX * TY) {
    const int lx = q % L::SX, row = q / L::SX;
    const int ly = row % L::SY, lz = row / L::SY;
    int gx = x0 - 1 + lx, gy = y0 - 1 + ly, gz = z0 - 1 + lz;
    bool solid = false;
    if (g.wx) solid |= (gx <= 0 || gx >= g.nx - 1);
    else if ((unsigned)gx >= (unsigned)g.nx) gx = ((gx % g.nx) + g.nx) % g.nx;
    if (g.wy) solid |= (gy <= 0 || gy >= g.ny - 1);
    else if ((unsigned)gy >= (unsigned)g.ny) gy = ((gy % g.ny) + g.ny) % g.ny;
    if (g.wz) solid |= (gz <= 0 || gz >= g.nz - 1);
    else if ((unsigned)gz >= (unsigned)g.nz) gz = ((gz % g.nz) + g.nz) % g.nz;
    if (solid) {
      sp[q] = spa[q] = spb[q] = R(PHI_SOLID);
      continue;
    }
    const size_t node = (size_t)gx + (size_t)g.nx * ((size_t)gy + (size_t)g.ny * gz);
    R ra, rb;
    if constexpr (FROM_ACC) {
      Acc<R>::densities(src.acc, node, ra, rb);
    } else {
      const R ph = reinterpret_cast<const R*>(src.phi)[node];
      const R rho = init.rho ? R(init.rho[node]) : R(1);
      ra = rho * (R(1) + ph) * R(0.5);
      rb = rho * (R(1) - ph) * R(0.5);
    }
    sp[q] = (ra - rb) / (ra + rb);
    spa[q] = sc_psi(ra, psi0);
    spb[q] = sc_psi(rb, psi0);
  }
}

// Pull of both component sets (two-set storages): f^A_i, f^B_i and their sums.
template <int ST, bool WALLFREE, bool IDX32>
__device__ __forceinline__ void pull_comp(const View<ST>& S, const Geo& g, const Nbr& n, int self,
                                          typename Store<ST>::R fa[Q], typename Store<ST>::R fb[Q],
                                          typename Store<ST>::R& rA, typename Store<ST>::R& rB) {
  using R = typename Store<ST>::R;
  using I = typename std::conditional<IDX32, unsigned, size_t>::type;
  const I N = (I)g.N;
  rA = R(0);
  rB = R(0);
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const int a = 1 - cx(i), b = 1 - cy(i), c = 1 - cz(i);
    const bool bb = WALLFREE ? false : (n.sx[a] | n.sy[b] | n.sz[c]);
    const I src = bb ? (I)self : (I)n.xs[a] + (I)g.nx * ((I)n.ys[b] + (I)g.ny * (I)n.zs[c]);
    const I dir = bb ? (I)opp(i) : (I)i;
    fa[i] = decode<ST>(S.f[dir * N + src], i);
    fb[i] = decode<ST>(S.f[((I)Q + dir) * N + src], i);
    rA += fa[i];
    rB += fb[i];
  }
}

// The nodes of one tile in the Shan-Chen model: pull both components, the
// pseudo-potential forces F_A = -psi_A G sum_i w_i psi_B(x + c_i) c_i (= -psi_A
// (G/3) times the stencil gradient of psi_B; a solid neighbour contributes the
// node's own psi) and F_B alike, the body force, the common velocity
// u' = sum_k (j_k + F_k/2)/tau_k / sum_k rho_k/tau_k, then per component BGK
// towards f^eq(rho_k, u') with the Guo source of F_k, store and send.
template <int ST, int LOADER, bool WS, bool WF, int TX, int TY, int TZ, bool WALLFREE, bool IDX32>
__device__ __forceinline__ void step_nodes_sc(const View<ST>& S, const View<ST>& O, const InitBuf& init,
                                              const Geo& g, const Phys& P, typename Store<ST>::R* __restrict__ fields,
                                              unsigned* __restrict__ status, const typename Store<ST>::R* sp,
                                              const typename Store<ST>::R* spa, const typename Store<ST>::R* spb,
                                              unsigned long long* sw, int x0, int y0, int z0) {
  using R = typename Store<ST>::R;
  using L = Layout<R, TX, TY, TZ, 1, 3>;
  using I = typename std::conditional<IDX32, unsigned, size_t>::type;
  const I N = (I)g.N;
  const size_t NF = (size_t)g.N;
  const R wa = R(1) / R(P.tau_a), wb = R(1) / R(P.tau_b);
  const R G3 = R(P.G) / R(3);
  for (int lz = 0; lz < TZ; ++lz) {
    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y, z = z0 + lz;
    if (x >= g.nx || y >= g.ny || z >= g.nz) continue;
    const int self = x + g.nx * (y + g.ny * z);
    if (!WALLFREE && is_solid(g, x, y, z)) {
      if constexpr (WF) {
        for (int k = 0; k < NFIELDS; ++k) fields[(size_t)k * NF + self] = R(0);
      }
      continue;
    }
    Nbr n;
    make_nbr(g, x, y, z, n);
    R fa[Q], fb[Q], rA, rB;
    if constexpr (LOADER == LOAD_PULL) {
      pull_comp<ST, WALLFREE, IDX32>(S, g, n, self, fa, fb, rA, rB);
    } else {
      R f[Q];
      fields_node<R, true>(init, g, P, n, (long long)self, f, rA, rB, fa, fb);
    }
    const int c = (lz + 1) * L::SXY + (threadIdx.y + 1) * L::SX + (threadIdx.x + 1);
    const int e0 = (lz + 1) * L::EXY + (threadIdx.y + 1) * L::EX + (threadIdx.x + 1);
    R jA[3] = {R(0), R(0), R(0)}, jB[3] = {R(0), R(0), R(0)};
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      if (cx(i)) { jA[0] += R(cx(i)) * fa[i]; jB[0] += R(cx(i)) * fb[i]; }
      if (cy(i)) { jA[1] += R(cy(i)) * fa[i]; jB[1] += R(cy(i)) * fb[i]; }
      if (cz(i)) { jA[2] += R(cz(i)) * fa[i]; jB[2] += R(cz(i)) * fb[i]; }
    }
    R gA[3], gB[3], gphi[3];
    tile_grad<R, WALLFREE>(spa, c, L::SX, L::SXY, gA);
    tile_grad<R, WALLFREE>(spb, c, L::SX, L::SXY, gB);
    R FA[3], FB[3], Fs[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      FA[a] = -spa[c] * G3 * gB[a];
      FB[a] = -spb[c] * G3 * gA[a];
      Fs[a] = FA[a] + FB[a];
    }
    if (P.g_mode == 1) {
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        FA[a] += rA * R(P.g[a]);
        FB[a] += rB * R(P.g[a]);
      }
    } else if (P.g_mode == 2) {
      const R sg = (z == 0 || 2 * z == g.nz) ? R(0) : (2 * z < g.nz ? R(1) : R(-1));
#pragma unroll
      for (int a = 0; a < 3; ++a) FA[a] += sg * rA * R(P.g[a]);
    }
    const R rho = rA + rB;
    if (!(rho > R(0) && rho < R(Acc<R>::RHO_MAX))) atomicOr(status, 1u);
    const R iw = R(1) / (wa * rA + wb * rB);
    R u[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) u[a] = (wa * (jA[a] + R(0.5) * FA[a]) + wb * (jB[a] + R(0.5) * FB[a])) * iw;
    if constexpr (WF) {
      tile_grad<R, WALLFREE>(sp, c, L::SX, L::SXY, gphi);
      const R irho = R(1) / rho;
      fields[(size_t)F_PHI * NF + self] = sp[c];
      fields[(size_t)F_RHO * NF + self] = rho;
      fields[(size_t)F_UX * NF + self] = (jA[0] + jB[0] + R(0.5) * (FA[0] + FB[0])) * irho;
      fields[(size_t)F_UY * NF + self] = (jA[1] + jB[1] + R(0.5) * (FA[1] + FB[1])) * irho;
      fields[(size_t)F_UZ * NF + self] = (jA[2] + jB[2] + R(0.5) * (FA[2] + FB[2])) * irho;
      fields[(size_t)F_RHOA * NF + self] = rA;
      fields[(size_t)F_RHOB * NF + self] = rB;
      fields[(size_t)F_FRX * NF + self] = Fs[0];
      fields[(size_t)F_FRY * NF + self] = Fs[1];
      fields[(size_t)F_FRZ * NF + self] = Fs[2];
      fields[(size_t)F_H * NF + self] = R(0);
      fields[(size_t)F_GX * NF + self] = gphi[0];
      fields[(size_t)F_GY * NF + self] = gphi[1];
      fields[(size_t)F_GZ * NF + self] = gphi[2];
    }
    if constexpr (!WS) continue;
    const R uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    const R ga = R(1) - R(0.5) * wa, gb = R(1) - R(0.5) * wb;
    const R uFA = u[0] * FA[0] + u[1] * FA[1] + u[2] * FA[2], uFB = u[0] * FB[0] + u[1] * FB[1] + u[2] * FB[2];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const R W = wgt<R>(i);
      R cu = R(0), cFA = R(0), cFB = R(0);
      if (cx(i)) { cu += R(cx(i)) * u[0]; cFA += R(cx(i)) * FA[0]; cFB += R(cx(i)) * FB[0]; }
      if (cy(i)) { cu += R(cy(i)) * u[1]; cFA += R(cy(i)) * FA[1]; cFB += R(cy(i)) * FB[1]; }
      if (cz(i)) { cu += R(cz(i)) * u[2]; cFA += R(cz(i)) * FA[2]; cFB += R(cz(i)) * FB[2]; }
      const R e = R(1) + R(3) * cu + R(4.5) * cu * cu - R(1.5) * uu;  // f^eq_i / (w_i rho_k)
      // Guo: (1 - 1/(2 tau_k)) w_i [3 (c_i - u) + 9 (c_i.u) c_i] . F_k
      const R sA = ga * W * (R(3) * (cFA - uFA) + R(9) * cu * cFA);
      const R sB = gb * W * (R(3) * (cFB - uFB) + R(9) * cu * cFB);
      const R oa = fa[i] + wa * (W * rA * e - fa[i]) + sA;
      const R ob = fb[i] + wb * (W * rB * e - fb[i]) + sB;
      O.f[(I)i * N + (I)self] = encode<ST>(oa, i);
      O.f[(I)(Q + i) * N + (I)self] = encode<ST>(ob, i);
      send<R, WALLFREE, L::EX, L::EXY, L::E>(sw, e0, n, i, oa, ob);
    }
  }
}

// One tile of the Shan-Chen step: clear, stage, step, flush.  Ends with a
// barrier.
template <int ST, int LOADER, bool WS, bool WF, int TX, int TY, int TZ, bool IDX32>
__device__ __forceinline__ void step_tile_sc(const View<ST>& S, const View<ST>& O, const InitBuf& init,
                                             const PhiSrc& src, const AccBufs& ab, const Geo& g, const Phys& P,
                                             typename Store<ST>::R* __restrict__ fields,
                                             unsigned* __restrict__ status, unsigned char* smem, int x0, int y0,
                                             int z0) {
  using R = typename Store<ST>::R;
  using L = Layout<R, TX, TY, TZ, 1, 3>;
  R* sp = reinterpret_cast<R*>(smem);
  R* spa = sp + L::NS;
  R* spb = spa + L::NS;
  unsigned long long* sw = reinterpret_cast<unsigned long long*>(smem + L::off_acc);
  const int tid = threadIdx.y * TX + threadIdx.x;
  if constexpr (WS) {
    for (int lz = 0; lz < TZ; ++lz) {
      const int x = x0 + threadIdx.x, y = y0 + threadIdx.y, z = z0 + lz;
      if (x < g.nx && y < g.ny && z < g.nz) Acc<R>::zero(ab.zero, (size_t)x + (size_t)g.nx * ((size_t)y + (size_t)g.ny * z));
    }
    for (int e = tid; e < Acc<R>::W * L::E; e += TX * TY) sw[e] = 0ull;
  }
  if (src.acc) stage_sc<R, true, TX, TY, TZ>(src, init, g, R(P.psi0), sp, spa, spb, x0, y0, z0);
  else stage_sc<R, false, TX, TY, TZ>(src, init, g, R(P.psi0), sp, spa, spb, x0, y0, z0);
  __syncthreads();
  if (!region_walled(g, x0, y0, z0, TX, TY, TZ, 1))
    step_nodes_sc<ST, LOADER, WS, WF, TX, TY, TZ, true, IDX32>(S, O, init, g, P, fields, status, sp, spa, spb, sw, x0,
                                                               y0, z0);
  else
    step_nodes_sc<ST, LOADER, WS, WF, TX, TY, TZ, false, IDX32>(S, O, init, g, P, fields, status, sp, spa, spb, sw,
                                                                x0, y0, z0);
  __syncthreads();
  if constexpr (WS) {
    flush_partials<R, TX, TY, TZ, 1>(sw, ab.out, g, x0, y0, z0);
    __syncthreads();
  }
}

template <int ST, int LOADER, bool WS, bool WF, int TX, int TY, int TZ, bool IDX32>
__global__ void __launch_bounds__(TX* TY, (ST == 3) ? 1 : 2)
    k_step_sc(View<ST> S, View<ST> O, InitBuf init, PhiSrc src, AccBufs ab, Geo g, Phys P,
              typename Store<ST>::R* __restrict__ fields, unsigned* __restrict__ status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  step_tile_sc<ST, LOADER, WS, WF, TX, TY, TZ, IDX32>(S, O, init, src, ab, g, P, fields, status, smem_raw,
                                                      blockIdx.x * TX, blockIdx.y * TY, blockIdx.z * TZ);
}

// One tile of the step: clear, stage, scan, step, flush.  Ends with a
// barrier, so the caller may reuse the shared memory.
template <int ST, int LOADER, bool WS, bool WF, int TX, int TY, int TZ, int H, bool IDX32, bool INL = false>
__device__ __forceinline__ void step_tile(const View<ST>& S, const View<ST>& O, const InitBuf& init, const PhiSrc& src,
                                          const AccBufs& ab, const Geo& g, const Phys& P,
                                          typename Store<ST>::R* __restrict__ fields, unsigned* __restrict__ status,
                                          unsigned char* smem, int x0, int y0, int z0) {
  using R = typename Store<ST>::R;
  using L = Layout<R, TX, TY, TZ, H, 1, !INL>;
  R* sp = reinterpret_cast<R*>(smem);
  unsigned long long* sw = reinterpret_cast<unsigned long long*>(smem + L::off_acc);
  unsigned short* queue = reinterpret_cast<unsigned short*>(smem + L::off_queue);
  unsigned char* hs = smem + L::off_h;
  int* count = reinterpret_cast<int*>(smem + L::off_count);
  const int tid = threadIdx.y * TX + threadIdx.x;
  if constexpr (WS) {
    // this tile's nodes of the accumulator two steps ahead (INL: in the node loop)
    if constexpr (!INL) {
      for (int lz = 0; lz < TZ; ++lz) {
        const int x = x0 + threadIdx.x, y = y0 + threadIdx.y, z = z0 + lz;
        if (x < g.nx && y < g.ny && z < g.nz)
          Acc<R>::zero(ab.zero, (size_t)x + (size_t)g.nx * ((size_t)y + (size_t)g.ny * z));
      }
    }
    for (int e = tid; e < Acc<R>::W * L::E; e += TX * TY) sw[e] = 0ull;
  }
  if (H > 1 && tid == 0) *count = 0;
  if (src.acc) stage_phi<R, true, TX, TY, TZ, H>(src, g, sp, x0, y0, z0);
  else stage_phi<R, false, TX, TY, TZ, H>(src, g, sp, x0, y0, z0);
  __syncthreads();
  const bool nc = H > 1 && P.A_h != 0.0;
  if constexpr (H > 1 && !INL) {
    if (nc) {
      if (region_walled(g, x0, y0, z0, TX, TY, TZ, P.K + 1))
        nc_tile<R, TX, TY, TZ, H, false>(sp, g, P, hs, queue, count, x0, y0, z0);
      else
        nc_tile<R, TX, TY, TZ, H, true>(sp, g, P, hs, queue, count, x0, y0, z0);
    }
  }
  // a tile whose one-node halo holds no solid node needs no bounce-back or
  // wall tests (INL: nor the scan's halo of K + 1 nodes)
  const bool wallfree = !region_walled(g, x0, y0, z0, TX, TY, TZ, (INL && nc) ? P.K + 1 : 1);
  unsigned long long* zacc = INL ? ab.zero : nullptr;
  if (P.collision == 1) {  // regularised collision
    if (wallfree)
      step_nodes<ST, LOADER, WS, WF, TX, TY, TZ, H, true, IDX32, true, INL>(S, O, init, g, P, hs, fields, status, sp,
                                                                            sw, src.acc, x0, y0, z0, zacc);
    else
      step_nodes<ST, LOADER, WS, WF, TX, TY, TZ, H, false, IDX32, true, INL>(S, O, init, g, P, hs, fields, status, sp,
                                                                             sw, src.acc, x0, y0, z0, zacc);
  } else {
    if (wallfree)
      step_nodes<ST, LOADER, WS, WF, TX, TY, TZ, H, true, IDX32, false, INL>(S, O, init, g, P, hs, fields, status, sp,
                                                                             sw, src.acc, x0, y0, z0, zacc);
    else
      step_nodes<ST, LOADER, WS, WF, TX, TY, TZ, H, false, IDX32, false, INL>(S, O, init, g, P, hs, fields, status,
                                                                              sp, sw, src.acc, x0, y0, z0, zacc);
  }
  __syncthreads();
  if constexpr (WS) {
    flush_partials<R, TX, TY, TZ, H>(sw, ab.out, g, x0, y0, z0);
    __syncthreads();
  }
}

template <int ST, int LOADER, bool WS, bool WF, int TX, int TY, int TZ, int H, bool IDX32, int MINB = 2,
          bool INL = false>
__global__ void __launch_bounds__(TX* TY, (ST == 3) ? 1 : MINB)
    k_step(View<ST> S, View<ST> O, InitBuf init, PhiSrc src, AccBufs ab, Geo g, Phys P,
           typename Store<ST>::R* __restrict__ fields, unsigned* __restrict__ status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  step_tile<ST, LOADER, WS, WF, TX, TY, TZ, H, IDX32, INL>(S, O, init, src, ab, g, P, fields, status, smem_raw,
                                                           blockIdx.x * TX, blockIdx.y * TY, blockIdx.z * TZ);
}

// ---------------------------------------------------------------------------
// batched persistent kernel: many independent runs of uneven sizes and
// parameters, one launch per step.  Work items are (run, tile); persistent
// CTAs stride over the item list and find the run of an item by binary
// search over the runs' prefix offsets.  Every run's accumulators are at the
// same phase k of their rotation.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int find_run(const RunDesc* runs, int nruns, long long item) {
  int lo = 0, hi = nruns - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (runs[mid].tile_begin <= item) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

template <int ST, int TX, int TY, int TZ, int H, bool IDX32, int MINB = 2, bool INL = false>
__global__ void __launch_bounds__(TX* TY, MINB)
    k_step_batched(const RunDesc* __restrict__ runs, int nruns, long long ntiles, int parity, int k,
                   unsigned* __restrict__ status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  InitBuf none{nullptr, nullptr, nullptr, 0};
  for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int r = find_run(runs, nruns, t);
    const RunDesc& d = runs[r];
    const long long lt = t - d.tile_begin;
    const int bx = (int)(lt % d.tiles_x);
    const int by = (int)((lt / d.tiles_x) % d.tiles_y);
    const int bz = (int)(lt / ((long long)d.tiles_x * d.tiles_y));
    const Geo g = d.g;
    const Phys P = d.p;
    const PhiSrc src{nullptr, d.acc[k]};
    const AccBufs ab{d.acc[(k + 1) % 3], d.acc[(k + 2) % 3]};
    step_tile<ST, LOAD_PULL, true, false, TX, TY, TZ, H, IDX32, INL>(view<ST>(d.S[parity]),
                                                                     view<ST>(d.S[parity ^ 1]), none, src, ab, g, P,
                                                                     nullptr, status, smem_raw, bx * TX, by * TY,
                                                                     bz * TZ);
  }
}

// ---------------------------------------------------------------------------
// population export (pre-collision, both components, canonical order, double)
// ---------------------------------------------------------------------------
template <int ST, int LOADER>
__global__ void __launch_bounds__(128) k_export(View<ST> S, InitBuf init, Geo g, Phys P, int x0, int y0, int z0,
                                                int bx, int by, int bz, double* outA, double* outB) {
  using R = typename Store<ST>::R;
  const long long M = (long long)bx * by * bz;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < M;
       e += (long long)gridDim.x * blockDim.x) {
    const int lx = (int)(e % bx);
    const int ly = (int)((e / bx) % by);
    const int lz = (int)(e / ((long long)bx * by));
    const int x = x0 + lx, y = y0 + ly, z = z0 + lz;
    const long long self = (long long)x + (long long)g.nx * ((long long)y + (long long)g.ny * z);
    if (is_solid(g, x, y, z)) {
      for (int i = 0; i < Q; ++i) {
        outA[(size_t)i * M + e] = 0.0;
        outB[(size_t)i * M + e] = 0.0;
      }
      continue;
    }
    Nbr n;
    make_nbr(g, x, y, z, n);
    R f[Q], fa[Q], fb[Q], rA, rB;
    if constexpr (LOADER == LOAD_PULL) {
      pull_node<ST, true>(S, g, n, self, f, rA, rB, fa, fb);
    } else {
      fields_node<R, true>(init, g, P, n, self, f, rA, rB, fa, fb);
    }
    for (int i = 0; i < Q; ++i) {
      outA[(size_t)i * M + e] = (double)fa[i];
      outB[(size_t)i * M + e] = (double)fb[i];
    }
  }
}

}  // namespace lbcg
