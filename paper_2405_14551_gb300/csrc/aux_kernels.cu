// Initial state, FP64 global reductions, Laplace readout and droplet count.
//
// The reductions are the only FP64 arithmetic of the FP32 path: per-block
// partial sums in a fixed partition and a fixed tree order, then one block
// sums the partials in a fixed order, so results are bitwise reproducible.
#include "../../include/lbcg.h"
#include "internal.h"
#include "lattice.cuh"

namespace lbcg {

// ---------------------------------------------------------------------------
// droplet initial condition (reading of the initial state): phi = +1 within
// distance R_j of centre j (periodic distance on open axes, union over
// droplets), -1 elsewhere; with width > 0 phi = max_j tanh((R_j - d_j)/width).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_init_droplets(Geo g, int n, const double* __restrict__ cen,
                                                       const double* __restrict__ rad, double width,
                                                       float* __restrict__ phi0) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < g.N; idx += stride) {
    const int x = (int)(idx % g.nx);
    const long long yz = idx / g.nx;
    const int y = (int)(yz % g.ny);
    const int z = (int)(yz / g.ny);
    const int v[3] = {x, y, z};
    const int nn[3] = {g.nx, g.ny, g.nz};
    const int wall[3] = {g.wx, g.wy, g.wz};
    double best = -1.0;
    for (int d = 0; d < n; ++d) {
      double d2 = 0.0;
      for (int a = 0; a < 3; ++a) {
        double dx = (double)v[a] - cen[3 * d + a];
        if (!wall[a]) {
          dx = fmod(dx, (double)nn[a]);
          if (dx > 0.5 * nn[a]) dx -= nn[a];
          if (dx < -0.5 * nn[a]) dx += nn[a];
        }
        d2 += dx * dx;
      }
      const double dist = sqrt(d2);
      const double ph = width > 0.0 ? tanh((rad[d] - dist) / width) : (dist <= rad[d] ? 1.0 : -1.0);
      best = ph > best ? ph : best;
    }
    phi0[idx] = (float)best;
  }
}

cudaError_t launch_init_droplets(const Geo& g, int n, const double* d_centres, const double* d_radii, double width,
                                 float* phi0, float* rho0, float* u0, cudaStream_t st) {
  (void)rho0;
  (void)u0;
  const long long need = (g.N + 255) / 256;
  const int blocks = (int)(need < 65535 ? need : 65535);
  k_init_droplets<<<blocks, 256, 0, st>>>(g, n, d_centres, d_radii, width, phi0);
  return cudaGetLastError();
}

// phi side array for the first step, taken from the initial phi field
template <typename R>
__global__ void __launch_bounds__(256) k_phi_from_init(long long N, const float* __restrict__ phi0, R* __restrict__ phi) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
    phi[i] = (R)phi0[i];
}

cudaError_t launch_phi_from_init(int storage, const Geo& g, const float* phi0, void* phi, cudaStream_t st) {
  const long long need = (g.N + 255) / 256;
  const int blocks = (int)(need < 65535 ? need : 65535);
  if (storage_is_f64(storage))
    k_phi_from_init<double><<<blocks, 256, 0, st>>>(g.N, phi0, reinterpret_cast<double*>(phi));
  else
    k_phi_from_init<float><<<blocks, 256, 0, st>>>(g.N, phi0, reinterpret_cast<float*>(phi));
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// deterministic FP64 reductions over the fields buffer
// ---------------------------------------------------------------------------
constexpr int RED_THREADS = 256;
constexpr int RED_MAX_BLOCKS = 1024;
// the allocation-free reduction keeps one partial per block in a static array
// of LB_STATIC_REDUCE_MAX_BLOCKS entries
static_assert(RED_MAX_BLOCKS <= LB_STATIC_REDUCE_MAX_BLOCKS, "static partials too small for the reduction");

int reduce_blocks(long long N) {
  long long b = (N + RED_THREADS * 8 - 1) / (RED_THREADS * 8);
  if (b < 1) b = 1;
  if (b > RED_MAX_BLOCKS) b = RED_MAX_BLOCKS;
  return (int)b;
}

__device__ __forceinline__ bool node_solid(const Geo& g, long long idx) {
  const int x = (int)(idx % g.nx);
  const long long yz = idx / g.nx;
  const int y = (int)(yz % g.ny);
  const int z = (int)(yz / g.ny);
  return (g.wx && (x == 0 || x == g.nx - 1)) || (g.wy && (y == 0 || y == g.ny - 1)) ||
         (g.wz && (z == 0 || z == g.nz - 1));
}

// fixed-order tree sum of NV values per thread into s[0..NV)
template <int NV>
__device__ void block_tree(double (*s)[RED_THREADS], double v[NV]) {
  for (int k = 0; k < NV; ++k) s[k][threadIdx.x] = v[k];
  __syncthreads();
  for (int w = RED_THREADS / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
      for (int k = 0; k < NV; ++k) s[k][threadIdx.x] += s[k][threadIdx.x + w];
    __syncthreads();
  }
}

template <typename R>
__global__ void __launch_bounds__(RED_THREADS) k_reduce_partial(Geo g, const R* __restrict__ fl, double* partials) {
  __shared__ double s[8][RED_THREADS];
  const size_t N = (size_t)g.N;
  const long long chunk = (g.N + gridDim.x - 1) / gridDim.x;
  const long long beg = (long long)blockIdx.x * chunk;
  const long long end = beg + chunk < g.N ? beg + chunk : g.N;
  double v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (long long i = beg + threadIdx.x; i < end; i += RED_THREADS) {
    if (node_solid(g, i)) continue;
    const double rho = fl[F_RHO * N + i];
    const double ux = fl[F_UX * N + i], uy = fl[F_UY * N + i], uz = fl[F_UZ * N + i];
    v[0] += fl[F_RHOA * N + i];
    v[1] += fl[F_RHOB * N + i];
    v[2] += rho * ux;
    v[3] += rho * uy;
    v[4] += rho * uz;
    v[5] += 0.5 * (1.0 + (double)fl[F_PHI * N + i]);
    v[6] += fl[F_H * N + i] > R(0) ? 1.0 : 0.0;
    v[7] += 0.5 * rho * (ux * ux + uy * uy + uz * uz);
  }
  block_tree<8>(s, v);
  if (threadIdx.x == 0)
    for (int k = 0; k < 8; ++k) partials[(size_t)blockIdx.x * 8 + k] = s[k][0];
}

template <int NV>
__global__ void __launch_bounds__(RED_THREADS) k_reduce_final(int nblocks, const double* __restrict__ partials,
                                                              double* out) {
  __shared__ double s[NV][RED_THREADS];
  double v[NV];
  for (int k = 0; k < NV; ++k) v[k] = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += RED_THREADS)
    for (int k = 0; k < NV; ++k) v[k] += partials[(size_t)b * NV + k];
  block_tree<NV>(s, v);
  if (threadIdx.x == 0)
    for (int k = 0; k < NV; ++k) out[k] = s[k][0];
}

cudaError_t launch_reduce(int storage, const Geo& g, const void* fields, double* partials, double* out8,
                          cudaStream_t st) {
  const int nb = reduce_blocks(g.N);
  if (storage_is_f64(storage))
    k_reduce_partial<double><<<nb, RED_THREADS, 0, st>>>(g, reinterpret_cast<const double*>(fields), partials);
  else
    k_reduce_partial<float><<<nb, RED_THREADS, 0, st>>>(g, reinterpret_cast<const float*>(fields), partials);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_reduce_final<8><<<1, RED_THREADS, 0, st>>>(nb, partials, out8);
  return cudaGetLastError();
}

// dispersed volume sum over fluid nodes of (1 + phi)/2 of a phase-field array,
// in the partition and order of k_reduce_partial (same value as its v[5])
__global__ void __launch_bounds__(RED_THREADS) k_phi_volume_partial(Geo g, const float* __restrict__ phi,
                                                                    double* partials) {
  __shared__ double s[1][RED_THREADS];
  const long long chunk = (g.N + gridDim.x - 1) / gridDim.x;
  const long long beg = (long long)blockIdx.x * chunk;
  const long long end = beg + chunk < g.N ? beg + chunk : g.N;
  double v[1] = {0};
  for (long long i = beg + threadIdx.x; i < end; i += RED_THREADS) {
    if (node_solid(g, i)) continue;
    v[0] += 0.5 * (1.0 + (double)phi[i]);
  }
  block_tree<1>(s, v);
  if (threadIdx.x == 0) partials[blockIdx.x] = s[0][0];
}

template <typename R>
__global__ void __launch_bounds__(RED_THREADS) k_laplace_partial(Geo g, const R* __restrict__ fl, double cut,
                                                                 double* partials) {
  __shared__ double s[4][RED_THREADS];
  const size_t N = (size_t)g.N;
  const long long chunk = (g.N + gridDim.x - 1) / gridDim.x;
  const long long beg = (long long)blockIdx.x * chunk;
  const long long end = beg + chunk < g.N ? beg + chunk : g.N;
  double v[4] = {0, 0, 0, 0};
  for (long long i = beg + threadIdx.x; i < end; i += RED_THREADS) {
    if (node_solid(g, i)) continue;
    const double ph = fl[F_PHI * N + i], r = fl[F_RHO * N + i];
    if (ph > cut) {
      v[0] += r;
      v[1] += 1.0;
    } else if (ph < -cut) {
      v[2] += r;
      v[3] += 1.0;
    }
  }
  block_tree<4>(s, v);
  if (threadIdx.x == 0)
    for (int k = 0; k < 4; ++k) partials[(size_t)blockIdx.x * 4 + k] = s[k][0];
}

cudaError_t launch_laplace(int storage, const Geo& g, const void* fields, double cut, double* partials,
                           double* out4, cudaStream_t st) {
  const int nb = reduce_blocks(g.N);
  if (storage_is_f64(storage))
    k_laplace_partial<double><<<nb, RED_THREADS, 0, st>>>(g, reinterpret_cast<const double*>(fields), cut, partials);
  else
    k_laplace_partial<float><<<nb, RED_THREADS, 0, st>>>(g, reinterpret_cast<const float*>(fields), cut, partials);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_reduce_final<4><<<1, RED_THREADS, 0, st>>>(nb, partials, out4);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// droplet count: union-find over fluid nodes with phi > 0, 6-connected,
// periodic on open axes.  Roots hook the larger label under the smaller with
// atomicCAS; every loop is bounded and reports through the status word.
// A first pass joins the links inside 32 x 8 x 8 tiles in shared memory and
// writes, per node, the global index of its tile-local root (the smallest
// index of its tile-local component); the global pass then joins only the
// links that cross tile faces.
// ---------------------------------------------------------------------------
constexpr int CC_TX = 32, CC_TY = 8, CC_TZ = 8, CC_TN = CC_TX * CC_TY * CC_TZ;

__device__ __forceinline__ int cc_find_local(int* L, int i) {
  for (int it = 0; it < CC_TN; ++it) {
    const int p = L[i];
    if (p == i) return i;
    const int gp = L[p];
    if (gp != p) L[i] = gp;  // path halving; parents only move to ancestors
    i = p;
  }
  return -1;
}

template <typename R>
__global__ void __launch_bounds__(256) k_cc_local(Geo g, const R* __restrict__ phi, int* __restrict__ Lg,
                                                  unsigned* status) {
  __shared__ int L[CC_TN];
  const int x0 = blockIdx.x * CC_TX, y0 = blockIdx.y * CC_TY, z0 = blockIdx.z * CC_TZ;
  for (int k = threadIdx.x; k < CC_TN; k += blockDim.x) {
    const int x = x0 + k % CC_TX, y = y0 + (k / CC_TX) % CC_TY, z = z0 + k / (CC_TX * CC_TY);
    bool on = false;
    if (x < g.nx && y < g.ny && z < g.nz) {
      const long long i = (long long)x + (long long)g.nx * ((long long)y + (long long)g.ny * z);
      on = !node_solid(g, i) && phi[i] > R(0);
    }
    L[k] = on ? k : -1;
  }
  __syncthreads();
  bool ok = true;
  for (int k = threadIdx.x; k < CC_TN; k += blockDim.x) {
    if (L[k] < 0) continue;
    const int lx = k % CC_TX, ly = (k / CC_TX) % CC_TY, lz = k / (CC_TX * CC_TY);
    const int nb[3] = {lx + 1 < CC_TX ? k + 1 : -1, ly + 1 < CC_TY ? k + CC_TX : -1,
                       lz + 1 < CC_TZ ? k + CC_TX * CC_TY : -1};
    for (int a = 0; a < 3; ++a) {
      if (nb[a] < 0 || L[nb[a]] < 0) continue;
      int ra = k, rb = nb[a];
      bool done = false;
      for (int it = 0; it < CC_TN && !done; ++it) {
        ra = cc_find_local(L, ra);
        rb = cc_find_local(L, rb);
        if (ra < 0 || rb < 0) break;
        if (ra == rb) {
          done = true;
          break;
        }
        if (ra < rb) {
          const int t = ra;
          ra = rb;
          rb = t;
        }
        const int old = atomicCAS(&L[ra], ra, rb);
        if (old == ra) done = true;
        else ra = old;
      }
      ok = ok && done;
    }
  }
  if (!ok) atomicOr(status, 2u);
  __syncthreads();
  for (int k = threadIdx.x; k < CC_TN; k += blockDim.x) {
    const int x = x0 + k % CC_TX, y = y0 + (k / CC_TX) % CC_TY, z = z0 + k / (CC_TX * CC_TY);
    if (x >= g.nx || y >= g.ny || z >= g.nz) continue;
    const long long i = (long long)x + (long long)g.nx * ((long long)y + (long long)g.ny * z);
    int r = L[k] < 0 ? -1 : cc_find_local(L, k);
    if (L[k] >= 0 && r < 0) {
      atomicOr(status, 2u);
      r = k;
    }
    Lg[i] = r < 0 ? -1
                  : (int)((long long)(x0 + r % CC_TX) +
                          (long long)g.nx * ((long long)(y0 + (r / CC_TX) % CC_TY) +
                                             (long long)g.ny * (z0 + r / (CC_TX * CC_TY))));
  }
}

// Root of i.  Every parent label is smaller than its child's (the tile pass
// points every node at the smallest index of its tile component;
// a root is only ever hooked under a smaller root), so each node met on the
// way may be pointed at its grandparent (path halving, as in intermediate
// pointer jumping): the writes only shorten paths and keep the forest valid
// under concurrent unions.  -1 if the walk exceeded its limit.
__device__ __forceinline__ int cc_find(volatile int* L, int i, long long limit) {
  int curr = L[i];
  if (curr == i) return i;
  int prev = i;
  for (long long it = 0; it < limit; ++it) {
    const int next = L[curr];
    if (next >= curr) return curr;  // a root (next == curr)
    L[prev] = next;
    prev = curr;
    curr = next;
  }
  return -1;
}

__global__ void k_cc_union(Geo g, int* __restrict__ Lp, unsigned* status) {
  volatile int* L = Lp;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < g.N; i += (long long)gridDim.x * blockDim.x) {
    if (L[i] < 0) continue;
    const int x = (int)(i % g.nx);
    const long long yz = i / g.nx;
    const int y = (int)(yz % g.ny);
    const int z = (int)(yz / g.ny);
    for (int a = 0; a < 3; ++a) {
      int v[3] = {x, y, z};
      const int nn[3] = {g.nx, g.ny, g.nz};
      const int wall[3] = {g.wx, g.wy, g.wz};
      const int tile[3] = {CC_TX, CC_TY, CC_TZ};
      if ((v[a] + 1) % tile[a] != 0 && v[a] + 1 < nn[a]) continue;  // joined by the tile pass
      v[a] += 1;
      if (v[a] >= nn[a]) {
        if (wall[a]) continue;
        v[a] -= nn[a];
      }
      const long long j = (long long)v[0] + (long long)g.nx * ((long long)v[1] + (long long)g.ny * v[2]);
      if (L[j] < 0) continue;
      int ra = (int)i, rb = (int)j;
      bool done = false;
      for (int it = 0; it < (1 << 22) && !done; ++it) {
        ra = cc_find(L, ra, g.N);
        rb = cc_find(L, rb, g.N);
        if (ra < 0 || rb < 0) break;
        if (ra == rb) {
          done = true;
          break;
        }
        if (ra < rb) {
          const int t = ra;
          ra = rb;
          rb = t;
        }
        const int old = atomicCAS(Lp + ra, ra, rb);
        if (old == ra) done = true;
        else ra = old;
      }
      if (!done) atomicOr(status, 2u);
    }
  }
}

__global__ void k_cc_count(Geo g, int* __restrict__ Lp, int* count) {
  volatile int* L = Lp;
  int local = 0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < g.N; i += (long long)gridDim.x * blockDim.x)
    if (L[i] == (int)i) ++local;
  if (local) atomicAdd(count, local);
}

cudaError_t launch_cc(int storage, const Geo& g, const void* fields, int* labels, int* count, unsigned* status,
                      cudaStream_t st) {
  const long long need = (g.N + 255) / 256;
  const int blocks = (int)(need < 8192 ? need : 8192);
  const dim3 tiles((g.nx + CC_TX - 1) / CC_TX, (g.ny + CC_TY - 1) / CC_TY, (g.nz + CC_TZ - 1) / CC_TZ);
  if (storage_is_f64(storage))
    k_cc_local<double><<<tiles, 256, 0, st>>>(g, reinterpret_cast<const double*>(fields), labels, status);
  else
    k_cc_local<float><<<tiles, 256, 0, st>>>(g, reinterpret_cast<const float*>(fields), labels, status);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_cc_union<<<blocks, 256, 0, st>>>(g, labels, status);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(count, 0, sizeof(int), st)) != cudaSuccess) return e;
  k_cc_count<<<blocks, 256, 0, st>>>(g, labels, count);
  return cudaGetLastError();
}

cudaError_t launch_phi_monitor(const Geo& g, const float* phi, int* labels, int* count, double* partials,
                               double* volume, unsigned* status, cudaStream_t st) {
  cudaError_t e = launch_cc(0, g, phi, labels, count, status, st);  // phi is the first (only) field
  if (e != cudaSuccess) return e;
  const int nb = reduce_blocks(g.N);
  k_phi_volume_partial<<<nb, RED_THREADS, 0, st>>>(g, phi, partials);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_reduce_final<1><<<1, RED_THREADS, 0, st>>>(nb, partials, volume);
  return cudaGetLastError();
}

}  // namespace lbcg
