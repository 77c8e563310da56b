#pragma once
// Device code of the fused time step of the two-component colour-gradient LB scheme on D3Q27
// (arXiv 2405.14551, Sec. III.B-III.D) for sm_103a.
//
// A step is three passes over the lattice:
//   1. k_phi: pull the populations of every node and write its phase field
//      phi = (rhoA - rhoB)/(rhoA + rhoB) (Eq. order_param) to a side array.
//      The colour gradient and the near-contact scan of a node need phi of
//      the current time level up to h_max + 1 nodes away, which exists only
//      after every neighbour has been pulled; this pass provides it.
//   2. k_nc (only with near contact, A_h != 0): per CTA a tile of phi plus a
//      halo of K + 1 nodes in shared memory; every interface node scans along
//      its outward normal (Eqs. stress_jump, near_cont_force) and the found
//      distance h (0: none) is written as one byte per node.
//   3. k_step: per CTA a tile of (TX x TY x TZ) nodes stages phi of the tile
//      plus a one-node halo in shared memory; every thread then pulls the 27
//      (x2) populations of its node (periodic wrap, halfway bounce-back at
//      solid neighbours, Sec. III.D), takes the moments, the colour gradient
//      from the tile, the repulsion from h, forms the Guo-shifted velocity,
//      relaxes the total populations (BGK), adds the perturbation Omega^(2)
//      and the forcing source, recolours (Eqs. ome3_1/2) and stores the
//      post-collision state once.
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

// Stored post-collision total population f*_dir of node src (single set
// storages).  Reduced: the stored value.  Moment storage (Sec. IV.C, Eq.
// eq:llb-pull): w_i (alpha + beta.c + c.Gamma.c) of the node's coefficients at
// c = c_i, or at c = -c_i = c_opp(i) when bb (bounce-back from the node
// itself, dir = opp(i)); only the coefficients that c_i touches are read.
template <int ST, typename I>
__device__ __forceinline__ typename Store<ST>::R load_fs(const typename Store<ST>::E* __restrict__ f, I N, I dir, I src,
                                                         int i, bool bb) {
  using R = typename Store<ST>::R;
  if constexpr (Store<ST>::MOMENT) {
    const float4 qa = reinterpret_cast<const float4*>(f)[src];
    R lin = R(0), quad = R(0);
    if (cx(i)) lin += R(cx(i)) * qa.y;
    if (cy(i)) lin += R(cy(i)) * qa.z;
    if (cz(i)) lin += R(cz(i)) * qa.w;
    if (cx(i) || cy(i) || cz(i)) {
      const float4 qb = reinterpret_cast<const float4*>(f + (I)4 * N)[src];
      if (cx(i)) quad += qb.x;
      if (cy(i)) quad += qb.y;
      if (cz(i)) quad += qb.z;
      if (cx(i) && cy(i)) quad += R(cx(i) * cy(i)) * qb.w;
    }
    if ((cx(i) && cz(i)) || (cy(i) && cz(i))) {
      const float2 qc = reinterpret_cast<const float2*>(f + (I)8 * N)[src];
      if (cx(i) && cz(i)) quad += R(cx(i) * cz(i)) * qc.x;
      if (cy(i) && cz(i)) quad += R(cy(i) * cz(i)) * qc.y;
    }
    return wgt<R>(i) * (qa.x + quad + (bb ? -lin : lin));
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
    if constexpr (Store<ST>::TWOSET) {
      const R va = decode<ST>(S.f[(size_t)dir * N + src], i);
      const R vb = decode<ST>(S.f[(size_t)(Q + dir) * N + src], i);
      f[i] = va + vb;
      rA += va;
      rB += vb;
      if constexpr (COMP) {
        fa[i] = va;
        fb[i] = vb;
      }
    } else {
      // single set: f^A_dir(src) = s f*_dir + w c_dir.v/|c_dir| (recolouring, Eq. ome3_1)
      const R fs = load_fs<ST, size_t>(S.f, N, (size_t)dir, (size_t)src, i, bb);
      const float4 sv = S.sv[src];
      const R s = sv.x;
      const R cv = R(cx(i)) * R(sv.y) + R(cy(i)) * R(sv.z) + R(cz(i)) * R(sv.w);
      const R seg = (bb ? R(-1) : R(1)) * wgt<R>(i) * inv_norm<R>(i) * cv;
      const R va = s * fs + seg;
      const R vb = (R(1) - s) * fs - seg;
      f[i] = fs;
      rA += va;
      rB += vb;
      if constexpr (COMP) {
        fa[i] = va;
        fb[i] = vb;
      }
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

// ---------------------------------------------------------------------------
// pass 1: phase field
// ---------------------------------------------------------------------------
// pull_fast is defined with the fused step below
template <int ST, bool WALLFREE, bool IDX32, bool TOTALS>
__device__ __forceinline__ void pull_fast(const View<ST>& S, const Geo& g, const Nbr& n, int self,
                                          typename Store<ST>::R f[Q], typename Store<ST>::R& rA,
                                          typename Store<ST>::R& rB);

__device__ __forceinline__ bool near_wall(const Geo& g, int x, int y, int z) {
  return (g.wx && (x <= 1 || x >= g.nx - 2)) || (g.wy && (y <= 1 || y >= g.ny - 2)) ||
         (g.wz && (z <= 1 || z >= g.nz - 2));
}

// phase field of one node from its pulled populations
template <int ST, bool IDX32>
__device__ __forceinline__ void phi_node(const View<ST>& S, const Geo& g, long long idx,
                                         typename Store<ST>::R* __restrict__ phi) {
  using R = typename Store<ST>::R;
  const int x = (int)(idx % g.nx);
  const long long yz = idx / g.nx;
  const int y = (int)(yz % g.ny);
  const int z = (int)(yz / g.ny);
  if (is_solid(g, x, y, z)) {
    phi[idx] = R(0);
    return;
  }
  Nbr n;
  make_nbr(g, x, y, z, n);
  R f[Q], rA, rB;
  if (near_wall(g, x, y, z))
    pull_fast<ST, false, IDX32, false>(S, g, n, (int)idx, f, rA, rB);
  else
    pull_fast<ST, true, IDX32, false>(S, g, n, (int)idx, f, rA, rB);
  phi[idx] = (rA - rB) / (rA + rB);
}

template <int ST, bool IDX32>
__global__ void __launch_bounds__(256) k_phi(View<ST> S, Geo g, typename Store<ST>::R* __restrict__ phi) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < g.N; idx += stride)
    phi_node<ST, IDX32>(S, g, idx, phi);
}

// Reduced storage: the same pass over CTA tiles.  Every node combines the
// colour scalars (s, v) of its 27 source nodes; the tile's scalars plus a
// one-node halo are staged in shared memory once, so those reads leave the
// L1/L2 path.  Same arithmetic in the same order as phi_node.
template <int ST, bool WALLFREE, bool IDX32>
__device__ __forceinline__ void pull_reduced_tile(const View<ST>& S, const Geo& g, const Nbr& n, int self,
                                                  const float4* svt, int cl, int SX, int SXY,
                                                  typename Store<ST>::R& rA, typename Store<ST>::R& rB) {
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
    int sl = cl - cx(i) - SX * cy(i) - SXY * cz(i);
    I dir = (I)i;
    bool bb = false;
    if constexpr (!WALLFREE) {
      bb = n.sx[a] | n.sy[b] | n.sz[c];
      src = bb ? self : src;
      sl = bb ? cl : sl;
      dir = bb ? (I)opp(i) : dir;
    }
    const R fs = load_fs<ST, I>(S.f, N, dir, (I)src, i, bb);
    const float4 sv = svt[sl];
    const R s = sv.x;
    R cv = R(0);
    if (cx(i)) cv += R(cx(i)) * R(sv.y);
    if (cy(i)) cv += R(cy(i)) * R(sv.z);
    if (cz(i)) cv += R(cz(i)) * R(sv.w);
    R seg = wgt<R>(i) * inv_norm<R>(i) * cv;
    if constexpr (!WALLFREE) seg = bb ? -seg : seg;
    const R va = s * fs + seg;
    rA += va;
    rB += (fs - va);
  }
}

template <int ST, int TX, int TY, int TZ, bool IDX32>
__global__ void __launch_bounds__(TX* TY) k_phi_tiled(View<ST> S, Geo g, typename Store<ST>::R* __restrict__ phi) {
  using R = typename Store<ST>::R;
  extern __shared__ __align__(16) float4 svt[];
  constexpr int SX = TX + 2, SY = TY + 2, SZ = TZ + 2, SXY = SX * SY;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, z0 = blockIdx.z * TZ;
  // stage (s, v) of the tile + halo: periodic axes wrap; beyond a wall the
  // entry is never read (a solid source is replaced by the node itself)
  for (int row = threadIdx.y; row < SY * SZ; row += TY) {
    const int ly = row % SY, lz = row / SY;
    int gy = y0 - 1 + ly, gz = z0 - 1 + lz;
    bool out = false;
    if ((unsigned)gy >= (unsigned)g.ny) {
      if (g.wy) out = true;
      else gy = ((gy % g.ny) + g.ny) % g.ny;
    }
    if ((unsigned)gz >= (unsigned)g.nz) {
      if (g.wz) out = true;
      else gz = ((gz % g.nz) + g.nz) % g.nz;
    }
    for (int lx = threadIdx.x; lx < SX; lx += TX) {
      int gx = x0 - 1 + lx;
      bool o = out;
      if ((unsigned)gx >= (unsigned)g.nx) {
        if (g.wx) o = true;
        else gx = ((gx % g.nx) + g.nx) % g.nx;
      }
      svt[row * SX + lx] = o ? make_float4(0.f, 0.f, 0.f, 0.f)
                             : S.sv[(size_t)gx + (size_t)g.nx * ((size_t)gy + (size_t)g.ny * gz)];
    }
  }
  __syncthreads();
  for (int lz = 0; lz < TZ; ++lz) {
    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y, z = z0 + lz;
    if (x >= g.nx || y >= g.ny || z >= g.nz) continue;
    const int self = x + g.nx * (y + g.ny * z);
    if (is_solid(g, x, y, z)) {
      phi[self] = R(0);
      continue;
    }
    Nbr n;
    make_nbr(g, x, y, z, n);
    const int cl = (lz + 1) * SXY + (threadIdx.y + 1) * SX + (threadIdx.x + 1);
    R rA, rB;
    if (near_wall(g, x, y, z))
      pull_reduced_tile<ST, false, IDX32>(S, g, n, self, svt, cl, SX, SXY, rA, rB);
    else
      pull_reduced_tile<ST, true, IDX32>(S, g, n, self, svt, cl, SX, SXY, rA, rB);
    phi[self] = (rA - rB) / (rA + rB);
  }
}

// ---------------------------------------------------------------------------
// passes 2 and 3: near-contact scan and fused step
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

// Pull for the hot path: totals f_i and component densities.  WALLFREE: no
// neighbour of the node is solid (no bounce-back test).  IDX32: every
// population offset fits in 32 bits.  TOTALS (reduced storage): only the
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
      const float4 sv = S.sv[src];
      const R s = sv.x;
      R cv = R(0);
      if (cx(i)) cv += R(cx(i)) * R(sv.y);
      if (cy(i)) cv += R(cy(i)) * R(sv.z);
      if (cz(i)) cv += R(cz(i)) * R(sv.w);
      R seg = wgt<R>(i) * inv_norm<R>(i) * cv;
      if constexpr (!WALLFREE) seg = bb ? -seg : seg;
      const R va = s * fs + seg;
      f[i] = fs;
      rA += va;
      rB += (fs - va);
    }
  }
}

// Stage phi of a tile (TX x TY x SZ - 2H own nodes) plus a halo of HX nodes
// along x and H along y and z in shared memory (row length TX + 2 HX), one
// (y, z) row per thread row: solid and beyond-wall nodes get the marker
// PHI_SOLID; periodic axes wrap.  Returns (to every thread) whether the
// staged block holds no solid node.
template <typename R, int TX, int TY>
__device__ __forceinline__ bool stage_phi(const R* __restrict__ phi, const Geo& g, int HX, int H, int SZ, R* sp,
                                          int x0, int y0, int z0) {
  const int SX = TX + 2 * HX, SY = TY + 2 * H;
  const int SXY = SX * SY;
  bool any_solid = false;
  for (int row = threadIdx.y; row < SY * SZ; row += TY) {
    const int ly = row % SY, lz = row / SY;
    int gy = y0 - H + ly, gz = z0 - H + lz;
    bool rsolid = false;
    if (g.wy) rsolid |= (gy <= 0 || gy >= g.ny - 1);
    else if ((unsigned)gy >= (unsigned)g.ny) gy = ((gy % g.ny) + g.ny) % g.ny;
    if (g.wz) rsolid |= (gz <= 0 || gz >= g.nz - 1);
    else if ((unsigned)gz >= (unsigned)g.nz) gz = ((gz % g.nz) + g.nz) % g.nz;
    const long long rbase = (long long)g.nx * ((long long)gy + (long long)g.ny * gz);
    R* srow = sp + (size_t)lz * SXY + (size_t)ly * SX;
    for (int lx = threadIdx.x; lx < SX; lx += TX) {
      int gx = x0 - HX + lx;
      bool solid = rsolid;
      if (g.wx) solid |= (gx <= 0 || gx >= g.nx - 1);
      else if ((unsigned)gx >= (unsigned)g.nx) gx = ((gx % g.nx) + g.nx) % g.nx;
      any_solid |= solid;
      srow[lx] = solid ? R(PHI_SOLID) : phi[rbase + gx];
    }
  }
  return !__syncthreads_or(any_solid);
}

// The same staging with 16-byte loads and stores, for a lattice whose rows
// are whole 16-byte vectors (nx a multiple of V = 16 / sizeof(R)) and a tile
// whose x halo HX and start x0 are multiples of V: every vector then lies
// wholly inside or wholly outside the box along x.  The block is walked as
// one flat list of vectors, so no lane idles on a short row remainder.
template <typename R, int TX, int TY, int HX, int H, int SZ>
__device__ __forceinline__ bool stage_phi_vec(const R* __restrict__ phi, const Geo& g, R* sp, int x0, int y0,
                                              int z0) {
  constexpr int V = 16 / sizeof(R);
  static_assert(HX % V == 0 && TX % V == 0, "vector staging needs aligned rows");
  constexpr int SX = TX + 2 * HX, SY = TY + 2 * H, QR = SX / V, NQ = QR * SY * SZ;
  using VT = typename std::conditional<sizeof(R) == 4, float4, double2>::type;
  bool any_solid = false;
  for (int q = threadIdx.y * TX + threadIdx.x; q < NQ; q += TX * TY) {
    const int qx = q % QR, row = q / QR;
    const int ly = row % SY, lz = row / SY;
    int gy = y0 - H + ly, gz = z0 - H + lz;
    bool rsolid = false;
    if (g.wy) rsolid |= (gy <= 0 || gy >= g.ny - 1);
    else if ((unsigned)gy >= (unsigned)g.ny) gy = ((gy % g.ny) + g.ny) % g.ny;
    if (g.wz) rsolid |= (gz <= 0 || gz >= g.nz - 1);
    else if ((unsigned)gz >= (unsigned)g.nz) gz = ((gz % g.nz) + g.nz) % g.nz;
    const int gx0 = x0 - HX + qx * V;  // first x of the vector
    R v[V];
    bool vsolid[V];
    bool inside = gx0 >= 0 && gx0 < g.nx;
    int gxl = gx0;
    if (!inside && !g.wx) {  // periodic wrap of a whole vector
      gxl = ((gx0 % g.nx) + g.nx) % g.nx;
      inside = true;
    }
#pragma unroll
    for (int j = 0; j < V; ++j) {
      const int xj = gx0 + j;
      vsolid[j] = rsolid || (g.wx && (xj <= 0 || xj >= g.nx - 1));
    }
    if (inside && !rsolid) {
      const long long rbase = (long long)g.nx * ((long long)gy + (long long)g.ny * gz);
      const VT w = *reinterpret_cast<const VT*>(phi + rbase + gxl);
      const R* wr = reinterpret_cast<const R*>(&w);
#pragma unroll
      for (int j = 0; j < V; ++j) v[j] = wr[j];
    }
    VT o;
    R* orr = reinterpret_cast<R*>(&o);
#pragma unroll
    for (int j = 0; j < V; ++j) {
      orr[j] = vsolid[j] ? R(PHI_SOLID) : v[j];
      any_solid |= vsolid[j];
    }
    *reinterpret_cast<VT*>(sp + (size_t)row * SX + qx * V) = o;
  }
  return !__syncthreads_or(any_solid);
}

// Near-contact scan of one interface node (Eqs. stress_jump, near_cont_force):
// step along the outward normal n_out = -grad phi/|grad phi| by round(k n_out),
// k = 1..K (K = H - 1); the first target that is an interface node
// (|phi| < phi_I, |grad phi| >= NC_GRAD_MIN) with a normal antiparallel to
// the node's own gives h = k; 0 when there is none.  The scan stops at a
// wall layer.  sp is the phi tile with halo H, c the node's tile index, gr
// and gg = |gr| its gradient.
template <typename R, bool WALLFREE, int H, int SX, int SXY>
__device__ __forceinline__ int nc_scan(const R* sp, int c, int x, int y, int z, const Geo& g, const Phys& P,
                                       const R gr[3], R gg) {
  const R phi_I = R(P.phi_I);
  const R inv = R(-1) / gg;
  const R no0 = gr[0] * inv, no1 = gr[1] * inv, no2 = gr[2] * inv;
#pragma unroll 1
  for (int k = 1; k < H; ++k) {
    // |n_out| = 1, so |d| <= k <= K < H; the clamp also covers non-finite normals
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

// Scan every queued interface node of the tile; threads take queue entries
// in turn, so no lane idles on a bulk-phase node.
template <typename R, int TX, int TY, int TZ, int H, int HX, bool WALLFREE>
__device__ __forceinline__ void nc_queue(const R* sp, const unsigned short* queue, int n, const Geo& g, const Phys& P,
                                         unsigned char* __restrict__ hout, int x0, int y0, int z0) {
  constexpr int SX = TX + 2 * HX, SXY = SX * (TY + 2 * H);
  for (int q = threadIdx.y * TX + threadIdx.x; q < n; q += TX * TY) {
    const int o = queue[q];
    const int lx = o % TX, ly = (o / TX) % TY, lz = o / (TX * TY);
    const int x = x0 + lx, y = y0 + ly, z = z0 + lz;
    const int c = (lz + H) * SXY + (ly + H) * SX + (lx + HX);
    R gr[3];
    tile_grad<R, WALLFREE>(sp, c, SX, SXY, gr);
    const R gg = sqrt_(gr[0] * gr[0] + gr[1] * gr[1] + gr[2] * gr[2]);
    int h = 0;
    if (gg >= R(NC_GRAD_MIN)) h = nc_scan<R, WALLFREE, H, SX, SXY>(sp, c, x, y, z, g, P, gr, gg);
    hout[x + g.nx * (y + g.ny * z)] = (unsigned char)h;
  }
}

// x halo of the near-contact tile: H rounded up to whole 16-byte vectors.
template <typename R, int H>
__host__ __device__ constexpr int nc_halo_x() {
  constexpr int V = 16 / (int)sizeof(R);
  return (H + V - 1) / V * V;
}

// One tile of the near-contact pass (halo H = K + 1; HX along x): stage phi,
// queue the tile's interface nodes (|phi| < phi_I; solid nodes hold PHI_SOLID
// and are never queued) by warp-aggregated appends, write h = 0 for the
// others, then scan the queue.  Ends with a barrier, so the caller may reuse
// the shared memory.  Shared memory: phi tile, a 16-byte counter, TX*TY*TZ
// queue slots.
template <typename R, int TX, int TY, int TZ, int H>
__device__ __forceinline__ void nc_tile(const R* __restrict__ phi, const Geo& g, const Phys& P,
                                        unsigned char* __restrict__ hout, R* sp, int x0, int y0, int z0) {
  constexpr int HX = nc_halo_x<R, H>();
  constexpr int SX = TX + 2 * HX, SY = TY + 2 * H, SZ = TZ + 2 * H, SXY = SX * SY;
  int* count = reinterpret_cast<int*>(sp + (size_t)SXY * SZ);
  unsigned short* queue = reinterpret_cast<unsigned short*>(count + 4);
  const int tid = threadIdx.y * TX + threadIdx.x;
  if (tid == 0) *count = 0;
  // both stagings end with a barrier
  const bool wallfree = (g.nx % (16 / (int)sizeof(R)) == 0)
                            ? stage_phi_vec<R, TX, TY, HX, H, SZ>(phi, g, sp, x0, y0, z0)
                            : stage_phi<R, TX, TY>(phi, g, HX, H, SZ, sp, x0, y0, z0);
  const int lane = tid & 31;
  const R phi_I = R(P.phi_I);
  for (int lz = 0; lz < TZ; ++lz) {
    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y, z = z0 + lz;
    const bool in = x < g.nx && y < g.ny && z < g.nz;
    const int c = (lz + H) * SXY + (threadIdx.y + H) * SX + (threadIdx.x + HX);
    const bool iface = in && fabs(sp[c]) < phi_I;
    if (in && !iface) hout[x + g.nx * (y + g.ny * z)] = 0;
    const unsigned m = __ballot_sync(0xffffffffu, iface);
    if (m) {
      const int leader = __ffs(m) - 1;
      int base = 0;
      if (lane == leader) base = atomicAdd(count, __popc(m));
      base = __shfl_sync(0xffffffffu, base, leader);
      if (iface) queue[base + __popc(m & ((1u << lane) - 1u))] = (unsigned short)((lz * TY + threadIdx.y) * TX + threadIdx.x);
    }
  }
  __syncthreads();
  const int n = *count;
  if (wallfree) nc_queue<R, TX, TY, TZ, H, HX, true>(sp, queue, n, g, P, hout, x0, y0, z0);
  else nc_queue<R, TX, TY, TZ, H, HX, false>(sp, queue, n, g, P, hout, x0, y0, z0);
  __syncthreads();
}

// Shared memory of one near-contact tile with halo H (x halo rounded up to
// whole 16-byte vectors).
template <typename R>
inline size_t nc_smem_bytes(int TX, int TY, int TZ, int H) {
  const int V = 16 / (int)sizeof(R);
  const int HX = (H + V - 1) / V * V;
  return sizeof(R) * (size_t)(TX + 2 * HX) * (TY + 2 * H) * (TZ + 2 * H) + 16 + 2 * (size_t)TX * TY * TZ;
}

// Calls f with the near-contact halo H = K + 1 (2..7) as a compile-time
// constant.
template <typename F>
__host__ __device__ __forceinline__ void with_halo(int halo, F&& f) {
  switch (halo) {
    case 2: f(std::integral_constant<int, 2>{}); break;
    case 3: f(std::integral_constant<int, 3>{}); break;
    case 4: f(std::integral_constant<int, 4>{}); break;
    case 5: f(std::integral_constant<int, 5>{}); break;
    case 6: f(std::integral_constant<int, 6>{}); break;
    case 7: f(std::integral_constant<int, 7>{}); break;
    default: break;
  }
}

// (templated on the storage format, not only on R, so that every translation
// unit instantiates kernels of its own)
template <int ST, int TX, int TY, int TZ, int H>
__global__ void __launch_bounds__(TX* TY) k_nc(const typename Store<ST>::R* __restrict__ phi, Geo g, Phys P,
                                               unsigned char* __restrict__ hout) {
  using R = typename Store<ST>::R;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  nc_tile<R, TX, TY, TZ, H>(phi, g, P, hout, reinterpret_cast<R*>(smem_raw), blockIdx.x * TX, blockIdx.y * TY,
                            blockIdx.z * TZ);
}

// The nodes of one fused-step tile; sp holds phi of the tile with a one-node
// halo, hnc the near-contact distance of every node (read when A_h != 0).
template <int ST, int LOADER, bool WS, bool WF, int TX, int TY, int TZ, bool WALLFREE, bool IDX32, bool REG>
__device__ __forceinline__ void step_nodes(const View<ST>& S, const View<ST>& O, const InitBuf& init, const Geo& g,
                                           const Phys& P, const unsigned char* __restrict__ hnc,
                                           typename Store<ST>::R* __restrict__ fields,
                                           unsigned* __restrict__ status, const typename Store<ST>::R* sp, int x0,
                                           int y0, int z0) {
  constexpr int SX = TX + 2, SXY = SX * (TY + 2);
  using R = typename Store<ST>::R;
  using I = typename std::conditional<IDX32, unsigned, size_t>::type;
  const R tau_a = R(P.tau_a), tau_b = R(P.tau_b);
  const R A2 = R(P.A2), beta = R(P.beta), A_h = R(P.A_h);
  const I N = (I)g.N;
  const size_t NF = (size_t)g.N;

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
    R f[Q], rA, rB;
    const int c = (lz + 1) * SXY + (threadIdx.y + 1) * SX + (threadIdx.x + 1);
    const R phx = sp[c];
    if constexpr (LOADER == LOAD_PULL) {
      if constexpr (Store<ST>::TWOSET) {
        pull_fast<ST, WALLFREE, IDX32, false>(S, g, n, self, f, rA, rB);
      } else {
        // reduced state: the component densities follow from the total and
        // this time level's phase field phi = (rhoA - rhoB)/rho (the tile),
        // so the neighbours' colour scalars need not be read again
        pull_fast<ST, WALLFREE, IDX32, true>(S, g, n, self, f, rA, rB);
        R rt = R(0);
#pragma unroll
        for (int i = 0; i < Q; ++i) rt += f[i];
        rA = R(0.5) * rt * (R(1) + phx);
        rB = rt - rA;
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

    // colour gradient from the tile; near-contact distance from the scan pass
    R gr[3];
    tile_grad<R, WALLFREE>(sp, c, SX, SXY, gr);
    const R gg = sqrt_(gr[0] * gr[0] + gr[1] * gr[1] + gr[2] * gr[2]);
    int h = 0;
    R Ahh = R(0);
    if (A_h != R(0)) {
      h = hnc[self];
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
    if (!(rho > R(0)) || !finite_(rho)) atomicOr(status, 1u);

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
    if constexpr (Store<ST>::MOMENT) {
      // f*_i = w_i (alpha + beta.c_i + c_i.Gamma.c_i): the equilibrium, the
      // relaxed Hermite orders 1-2, the perturbation (B_i = w_i (|c_i|^2 - 2/3))
      // and the Guo source below are each w_i times a quadratic form in c_i
      // (Eqs. disteq, distnoneq, LBpostmom; the host admits this storage with
      // the regularised collision only)
      const R kP = keep * R(4.5), hg9 = R(0.5) * g9;
      const R bF = g3 - R(1.5) * keep;  // beta = 3 rho u + (3 guo - 1.5 keep) F
      reinterpret_cast<float4*>(O.f)[self] =
          make_float4(r0 + gm3uF - R(1.5) * keep * trP + (R(2) / R(3)) * A2g, r3 * u0 + bF * F0, r3 * u1 + bF * F1,
                      r3 * u2 + bF * F2);
      reinterpret_cast<float4*>(O.f + (I)4 * N)[self] =
          make_float4(r45 * u0 * u0 + g9 * u0 * F0 + A2ig * gr[0] * gr[0] - A2g + kP * Pxx,
                      r45 * u1 * u1 + g9 * u1 * F1 + A2ig * gr[1] * gr[1] - A2g + kP * Pyy,
                      r45 * u2 * u2 + g9 * u2 * F2 + A2ig * gr[2] * gr[2] - A2g + kP * Pzz,
                      R(2) * (r45 * u0 * u1 + hg9 * (u0 * F1 + F0 * u1) + A2ig * gr[0] * gr[1] + kP * Pxy));
      reinterpret_cast<float2*>(O.f + (I)8 * N)[self] =
          make_float2(R(2) * (r45 * u0 * u2 + hg9 * (u0 * F2 + F0 * u2) + A2ig * gr[0] * gr[2] + kP * Pxz),
                      R(2) * (r45 * u1 * u2 + hg9 * (u1 * F2 + F1 * u2) + A2ig * gr[1] * gr[2] + kP * Pyz));
      O.sv[self] = make_float4(sA, segamp * gr[0], segamp * gr[1], segamp * gr[2]);
      continue;
    }
    {  // rest direction
      const R W = wgt<R>(REST);
      const R rel = reg ? R(-1.5) * W * trP : f[REST];
      const R fs = keep * rel + wf * W * r0 - bweight<R>(REST) * A2g + W * gm3uF;
      if constexpr (Store<ST>::TWOSET) {
        const R fa = sA * fs;
        O.f[(I)REST * N + (I)self] = encode<ST>(fa, REST);
        O.f[(I)(Q + REST) * N + (I)self] = encode<ST>(fs - fa, REST);
      } else {
        O.f[(I)REST * N + (I)self] = encode<ST>(fs, REST);
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
        O.f[(I)p * N + (I)self] = encode<ST>(fap, p);
        O.f[(I)q * N + (I)self] = encode<ST>(faq, q);
        O.f[(I)(Q + p) * N + (I)self] = encode<ST>(fsp - fap, p);
        O.f[(I)(Q + q) * N + (I)self] = encode<ST>(fsq - faq, q);
      } else {
        O.f[(I)p * N + (I)self] = encode<ST>(fsp, p);
        O.f[(I)q * N + (I)self] = encode<ST>(fsq, q);
      }
    }
    if constexpr (!Store<ST>::TWOSET) {
      O.sv[self] = make_float4(sA, segamp * gr[0], segamp * gr[1], segamp * gr[2]);
    }
  }
}

// One tile of the fused step: stage phi of the tile + a one-node halo, then
// update the tile's nodes.  Ends with a barrier, so the caller may reuse the
// shared tile.
template <int ST, int LOADER, bool WS, bool WF, int TX, int TY, int TZ, bool IDX32>
__device__ __forceinline__ void step_tile(const View<ST>& S, const View<ST>& O, const InitBuf& init,
                                          const typename Store<ST>::R* __restrict__ phi,
                                          const unsigned char* __restrict__ hnc, const Geo& g, const Phys& P,
                                          typename Store<ST>::R* __restrict__ fields, unsigned* __restrict__ status,
                                          typename Store<ST>::R* sp, int x0, int y0, int z0) {
  using R = typename Store<ST>::R;
  // a tile whose halo holds no solid node needs no bounce-back or wall tests
  const bool wallfree = stage_phi<R, TX, TY>(phi, g, 1, 1, TZ + 2, sp, x0, y0, z0);
  if (P.collision == 1) {  // regularised collision
    if (wallfree)
      step_nodes<ST, LOADER, WS, WF, TX, TY, TZ, true, IDX32, true>(S, O, init, g, P, hnc, fields, status, sp, x0,
                                                                    y0, z0);
    else
      step_nodes<ST, LOADER, WS, WF, TX, TY, TZ, false, IDX32, true>(S, O, init, g, P, hnc, fields, status, sp, x0,
                                                                     y0, z0);
  } else {
    if (wallfree)
      step_nodes<ST, LOADER, WS, WF, TX, TY, TZ, true, IDX32, false>(S, O, init, g, P, hnc, fields, status, sp, x0,
                                                                     y0, z0);
    else
      step_nodes<ST, LOADER, WS, WF, TX, TY, TZ, false, IDX32, false>(S, O, init, g, P, hnc, fields, status, sp, x0,
                                                                      y0, z0);
  }
  __syncthreads();
}

// Shared memory of one fused-step tile: phi with a one-node halo.
template <typename R>
inline size_t step_smem_bytes(int TX, int TY, int TZ) {
  return sizeof(R) * (size_t)(TX + 2) * (TY + 2) * (TZ + 2);
}

template <int ST, int LOADER, bool WS, bool WF, int TX, int TY, int TZ, bool IDX32, int MINB = 2>
__global__ void __launch_bounds__(TX* TY, (ST == 3) ? 1 : MINB)
    k_step(View<ST> S, View<ST> O, InitBuf init, const typename Store<ST>::R* __restrict__ phi,
           const unsigned char* __restrict__ hnc, Geo g, Phys P, typename Store<ST>::R* __restrict__ fields,
           unsigned* __restrict__ status) {
  using R = typename Store<ST>::R;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  step_tile<ST, LOADER, WS, WF, TX, TY, TZ, IDX32>(S, O, init, phi, hnc, g, P, fields, status,
                                                   reinterpret_cast<R*>(smem_raw), blockIdx.x * TX, blockIdx.y * TY,
                                                   blockIdx.z * TZ);
}

// ---------------------------------------------------------------------------
// batched persistent kernels: many independent runs of uneven sizes and
// parameters.  Work items are (run, tile) for the step and (run, 256-node
// chunk) for the phase field; persistent CTAs stride over the item list and
// find the run of an item by binary search over the runs' prefix offsets.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int find_run(const RunDesc* runs, int nruns, long long item, bool by_tile) {
  int lo = 0, hi = nruns - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    const long long b = by_tile ? runs[mid].tile_begin : runs[mid].chunk_begin;
    if (b <= item) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

template <int ST, bool IDX32>
__global__ void __launch_bounds__(256) k_phi_batched(const RunDesc* __restrict__ runs, int nruns, long long nchunks,
                                                     int parity) {
  using R = typename Store<ST>::R;
  for (long long c = blockIdx.x; c < nchunks; c += gridDim.x) {
    const int r = find_run(runs, nruns, c, false);
    const Geo g = runs[r].g;
    const long long idx = (c - runs[r].chunk_begin) * 256 + threadIdx.x;
    if (idx >= g.N) continue;
    phi_node<ST, IDX32>(view<ST>(runs[r].S[parity]), g, idx, reinterpret_cast<R*>(runs[r].phi));
  }
}

template <int ST, int TX, int TY, int TZ, bool IDX32, int MINB = 2>
__global__ void __launch_bounds__(TX* TY, MINB)
    k_step_batched(const RunDesc* __restrict__ runs, int nruns, long long ntiles, int parity,
                   unsigned* __restrict__ status) {
  using R = typename Store<ST>::R;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R* sp = reinterpret_cast<R*>(smem_raw);
  InitBuf none{nullptr, nullptr, nullptr, 0};
  for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int r = find_run(runs, nruns, t, true);
    const RunDesc& d = runs[r];
    const long long lt = t - d.tile_begin;
    const int bx = (int)(lt % d.tiles_x);
    const int by = (int)((lt / d.tiles_x) % d.tiles_y);
    const int bz = (int)(lt / ((long long)d.tiles_x * d.tiles_y));
    const Geo g = d.g;
    const Phys P = d.p;
    step_tile<ST, LOAD_PULL, true, false, TX, TY, TZ, IDX32>(
        view<ST>(d.S[parity]), view<ST>(d.S[parity ^ 1]), none, reinterpret_cast<const R*>(d.phi), d.hnc, g, P,
        nullptr, status, sp, bx * TX, by * TY, bz * TZ);
  }
}

// Near-contact pass of a batch over the same (run, tile) items; runs without
// near contact are skipped (their step never reads h).
template <int ST, int TX, int TY, int TZ>
__global__ void __launch_bounds__(TX* TY) k_nc_batched(const RunDesc* __restrict__ runs, int nruns, long long ntiles) {
  using R = typename Store<ST>::R;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R* sp = reinterpret_cast<R*>(smem_raw);
  for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int r = find_run(runs, nruns, t, true);
    const RunDesc& d = runs[r];
    if (d.p.A_h == 0.0) continue;
    const long long lt = t - d.tile_begin;
    const int bx = (int)(lt % d.tiles_x);
    const int by = (int)((lt / d.tiles_x) % d.tiles_y);
    const int bz = (int)(lt / ((long long)d.tiles_x * d.tiles_y));
    with_halo(d.p.halo, [&](auto hc) {
      nc_tile<R, TX, TY, TZ, decltype(hc)::value>(reinterpret_cast<const R*>(d.phi), d.g, d.p, d.hnc, sp, bx * TX,
                                                  by * TY, bz * TZ);
    });
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
