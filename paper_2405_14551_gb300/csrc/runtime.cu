// C-ABI runtime of the colour-gradient LB library (declared in include/lbcg.h).
//
// A handle owns two population lattices (ping-pong), three accumulators of
// the component densities that carry phi from one step to the next (see
// step_impl.cuh), the initial-field arrays and small scratch buffers.  Steps
// are issued asynchronously on the handle's stream, one kernel per step; runs
// of steps replay a captured CUDA graph of STEPS_PER_GRAPH steps, one graph
// per (lattice parity, accumulator phase).
#include <cuda_runtime.h>
#include <sys/stat.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <sstream>
#include <string>
#include <vector>

#include "../../include/lbcg.h"
#include "internal.h"
#include "lattice.cuh"

using namespace lbcg;

namespace {

// a multiple of 2 (lattice parity) and 3 (accumulator phase): a replay
// leaves both where they were
constexpr int STEPS_PER_GRAPH = 12;
constexpr uint32_t CKPT_MAGIC = 0x4742434cu;  // "LCBG"
constexpr uint32_t CKPT_VERSION = 3;  // 2: lb_params carries the collision model; 3: and the Shan-Chen model

std::atomic<uint64_t> g_launches{0};
thread_local std::string g_last_error;

int set_err(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

int cuda_err(cudaError_t e, const char* where) {
  if (e == cudaSuccess) return LB_OK;
  return set_err(LB_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define LB_CUDA(call)                                   \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return cuda_err(e_, #call);  \
  } while (0)

template <typename T>
__global__ void k_convert(long long n, const T* __restrict__ src, float* __restrict__ dst) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    dst[i] = (float)src[i];
}
template <typename T>
__global__ void k_convert_d(long long n, const T* __restrict__ src, double* __restrict__ dst) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    dst[i] = (double)src[i];
}

}  // namespace

namespace lbcg {
int report_error(int code, const std::string& msg) { return set_err(code, msg); }
void count_launches(int n) { g_launches += (uint64_t)n; }
}  // namespace lbcg

struct lb_handle {
  lb_grid grid;
  lb_params params;
  Geo g;
  Phys p;
  int storage;
  cudaStream_t stream = nullptr;   // stream all work is issued on
  cudaStream_t own_stream = nullptr;
  lb_alloc alloc{};
  bool have_alloc = false;
  std::vector<std::pair<void*, size_t>> owned;
  size_t bytes = 0;

  StateBuf S[2]{};
  int cur = 0;
  void* phi = nullptr;      // R[N]: phi of the initial fields
  // accumulators of the component densities: acc[phi_acc] holds phi of the
  // current time level, acc[(phi_acc + 1) % 3] is all zero; phi_acc = -1:
  // phi is in the phi array (initial state) and all three are zero
  unsigned long long* acc[3] = {nullptr, nullptr, nullptr};
  int phi_acc = -1;
  float* init_phi = nullptr;
  float* init_rho = nullptr;
  float* init_u = nullptr;
  bool use_rho = false, use_u = false;
  int regularised = 0;
  void* fields = nullptr;   // R[NFIELDS][N], lazily allocated
  double* red = nullptr;    // reduction partials, then 8 result doubles
  int* labels = nullptr;    // lazily allocated
  int* count = nullptr;
  unsigned* status = nullptr;
  int mode = 0;             // 0: state given by the initial fields, 1: by populations
  bool initialised = false;
  int64_t t = 0;
  int tile = 0;
  cudaGraphExec_t graph[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};  // [cur * 3 + phi_acc]
  uint64_t graph_launches = 0;  // kernel launches in one replay
  lbcg::SurrogateState* surrogate = nullptr;  // its device buffers are owned like the rest
};

namespace {
void* dev_alloc(lb_handle* h, size_t bytes);
}

namespace lbcg {
cudaStream_t handle_stream(lb_handle* h) { return h->stream; }
void handle_dims(const lb_handle* h, int* nx, int* ny, int* nz, uint32_t* walls) {
  *nx = h->grid.nx;
  *ny = h->grid.ny;
  *nz = h->grid.nz;
  *walls = h->grid.walls;
}
void* handle_alloc(lb_handle* h, size_t bytes) { return dev_alloc(h, bytes); }
SurrogateState*& handle_surrogate(lb_handle* h) { return h->surrogate; }
}  // namespace lbcg


namespace {

void* dev_alloc(lb_handle* h, size_t bytes) {
  void* p = nullptr;
  if (bytes == 0) bytes = 256;
  if (h->have_alloc) {
    p = h->alloc.alloc(h->alloc.ctx, bytes);
  } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  if (p) {
    h->owned.emplace_back(p, bytes);
    h->bytes += bytes;
  }
  return p;
}

void dev_free(lb_handle* h, void* p) {
  if (!p) return;
  for (size_t k = 0; k < h->owned.size(); ++k) {
    if (h->owned[k].first == p) {
      h->bytes -= h->owned[k].second;
      h->owned.erase(h->owned.begin() + (long)k);
      break;
    }
  }
  if (h->have_alloc) h->alloc.free(h->alloc.ctx, p);
  else cudaFree(p);
}

size_t real_bytes(int storage) { return storage_is_f64(storage) ? 8 : 4; }

size_t state_bytes(const lb_handle* h) {
  const size_t N = (size_t)h->g.N;
  const size_t fbytes = (size_t)state_arrays(h->storage) * N * elem_bytes(h->storage);
  if (storage_is_twoset(h->storage)) return fbytes;
  return fbytes + 4 * N * sizeof(float);
}

bool alloc_state(lb_handle* h, StateBuf& s) {
  const size_t N = (size_t)h->g.N;
  if (storage_is_twoset(h->storage)) {
    s.f = dev_alloc(h, (size_t)state_arrays(h->storage) * N * elem_bytes(h->storage));
    return s.f != nullptr;
  }
  // one allocation: f* (or the moment coefficients) then the float4 colour
  // scalars (256-byte aligned)
  const size_t fb = ((size_t)state_arrays(h->storage) * N * elem_bytes(h->storage) + 255) & ~(size_t)255;
  char* base = (char*)dev_alloc(h, fb + N * sizeof(float4));
  if (!base) return false;
  s.f = base;
  s.sv = (float4*)(base + fb);
  return true;
}

InitBuf init_buf(const lb_handle* h) {
  InitBuf b;
  b.phi = h->init_phi;
  b.rho = h->use_rho ? h->init_rho : nullptr;
  b.u = h->use_u ? h->init_u : nullptr;
  b.regularised = h->regularised;
  return b;
}

void drop_graphs(lb_handle* h) {
  for (int k = 0; k < 6; ++k) {
    if (h->graph[k]) cudaGraphExecDestroy(h->graph[k]);
    h->graph[k] = nullptr;
  }
}

int validate(const lb_grid* gr, const lb_params* p) {
  if (!gr || !p) return set_err(LB_EINVAL, "null grid or params");
  if (gr->nx < 1 || gr->ny < 1 || gr->nz < 1) return set_err(LB_EINVAL, "grid extents must be >= 1");
  if (gr->walls & ~7u) return set_err(LB_EINVAL, "walls uses bits 0..2 only");
  const int n[3] = {gr->nx, gr->ny, gr->nz};
  for (int a = 0; a < 3; ++a)
    if (((gr->walls >> a) & 1u) && n[a] < 3) return set_err(LB_EINVAL, "a walled axis needs at least 3 layers");
  const long long N = (long long)gr->nx * gr->ny * gr->nz;
  if (N > 0x7fffffffLL) return set_err(LB_EINVAL, "grid has more than 2^31-1 nodes");
  auto fin = [](double v) { return std::isfinite(v); };
  if (!(p->tau_a > 0.5) || !(p->tau_b > 0.5) || !fin(p->tau_a) || !fin(p->tau_b))
    return set_err(LB_EINVAL, "tau_a and tau_b must be finite and > 0.5");
  if (!fin(p->A_a) || !fin(p->A_b) || !fin(p->A_h)) return set_err(LB_EINVAL, "A_a, A_b, A_h must be finite");
  if (!(p->beta >= 0.0 && p->beta <= 1.0)) return set_err(LB_EINVAL, "beta must lie in [0, 1]");
  if (p->A_h != 0.0) {
    if (!(p->h_max >= 1.0 && p->h_max < 7.0)) return set_err(LB_EINVAL, "h_max must lie in [1, 7)");
    if (!(p->h_min > 0.0 && p->h_min <= p->h_max)) return set_err(LB_EINVAL, "h_min must lie in (0, h_max]");
    if (!(p->phi_I > 0.0 && p->phi_I <= 1.0)) return set_err(LB_EINVAL, "phi_I must lie in (0, 1]");
  }
  if (!fin(p->g[0]) || !fin(p->g[1]) || !fin(p->g[2])) return set_err(LB_EINVAL, "g must be finite");
  if (p->g_mode < 0 || p->g_mode > 2) return set_err(LB_EINVAL, "g_mode must be 0, 1 or 2");
  if (p->storage < 0 || p->storage > 4) return set_err(LB_EINVAL, "unknown storage format");
  if (p->collision < 0 || p->collision > 1) return set_err(LB_EINVAL, "collision must be 0 (BGK) or 1 (regularised)");
  if (p->storage == LB_STORAGE_MOMENT_F32 && p->collision != 1)
    return set_err(LB_EINVAL, "the moment storage holds the regularised collision only (collision = 1)");
  if (p->model < 0 || p->model > 1) return set_err(LB_EINVAL, "model must be 0 (colour gradient) or 1 (Shan-Chen)");
  if (p->model == LB_MODEL_SHAN_CHEN) {
    if (p->storage != LB_STORAGE_TWOSET_F32 && p->storage != LB_STORAGE_TWOSET_F64)
      return set_err(LB_EINVAL, "the Shan-Chen model needs a two-set storage");
    if (p->A_h != 0.0 || p->collision != 0) return set_err(LB_EINVAL, "the Shan-Chen model takes A_h = 0 and collision = 0");
    if (!fin(p->G) || !(p->psi0 > 0.0) || !fin(p->psi0)) return set_err(LB_EINVAL, "Shan-Chen needs a finite G and psi0 > 0");
  }
  return LB_OK;
}

size_t acc_bytes(const lb_handle* h) { return (size_t)h->g.N * (size_t)acc_words(h->storage) * 8; }

// Clear the three accumulators (phi then lives in the phi array).
cudaError_t reset_acc(lb_handle* h) {
  cudaError_t e = cudaSuccess;
  for (int k = 0; k < 3 && e == cudaSuccess; ++k) e = cudaMemsetAsync(h->acc[k], 0, acc_bytes(h), h->stream);
  h->phi_acc = -1;
  return e;
}

// Rebuild phi of the current population state into acc[0] (after populations
// were loaded or copied in), acc[1] and acc[2] zero.
cudaError_t rebuild_acc(lb_handle* h) {
  cudaError_t e = reset_acc(h);
  if (e == cudaSuccess) e = launch_phi_acc(h->storage, h->g, h->S[h->cur], h->acc[0], h->stream);
  g_launches += 1;
  h->phi_acc = 0;
  return e;
}

// Where the current phi is read from, and the accumulators a step writes.
PhiSrc phi_src(const lb_handle* h) {
  if (h->phi_acc < 0) return PhiSrc{h->phi, nullptr};
  return PhiSrc{nullptr, h->acc[h->phi_acc]};
}
AccBufs acc_bufs(const lb_handle* h) {
  const int k = h->phi_acc < 0 ? 2 : h->phi_acc;  // from the phi array: every accumulator is zero
  return AccBufs{h->acc[(k + 1) % 3], h->acc[(k + 2) % 3]};
}

// Issue one step (no graph).
int issue_step(lb_handle* h) {
  const int nxt = h->cur ^ 1;
  const bool fresh = h->mode == 0;
  LB_CUDA(launch_step(h->storage, fresh ? LOAD_FIELDS : LOAD_PULL, true, false, fresh ? 0 : h->tile, h->g, h->p,
                      h->S[h->cur], init_buf(h), phi_src(h), acc_bufs(h), h->S[nxt], nullptr, h->status, h->stream));
  g_launches += 1;
  h->phi_acc = ((h->phi_acc < 0 ? 2 : h->phi_acc) + 1) % 3;
  h->cur = nxt;
  h->mode = 1;
  h->t += 1;
  return LB_OK;
}

int graph_key(const lb_handle* h) { return h->cur * 3 + h->phi_acc; }

int build_graph(lb_handle* h) {
  cudaGraph_t graph = nullptr;
  const int save_cur = h->cur, save_acc = h->phi_acc, key = graph_key(h);
  const int64_t save_t = h->t;
  const uint64_t save_l = g_launches.load();
  LB_CUDA(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
  int rc = LB_OK;
  for (int k = 0; k < STEPS_PER_GRAPH && rc == LB_OK; ++k) rc = issue_step(h);
  cudaError_t e = cudaStreamEndCapture(h->stream, &graph);
  h->cur = save_cur;
  h->phi_acc = save_acc;
  h->t = save_t;
  h->graph_launches = g_launches.load() - save_l;
  g_launches = save_l;
  if (rc != LB_OK) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  if (e != cudaSuccess) return cuda_err(e, "cudaStreamEndCapture");
  e = cudaGraphInstantiate(&h->graph[key], graph, 0);
  cudaGraphDestroy(graph);
  return cuda_err(e, "cudaGraphInstantiate");
}

int ensure_fields(lb_handle* h) {
  if (!h->fields) {
    h->fields = dev_alloc(h, (size_t)NFIELDS * h->g.N * real_bytes(h->storage));
    if (!h->fields) return set_err(LB_ENOMEM, "fields buffer allocation failed");
  }
  return LB_OK;
}

// Fill the fields buffer at the current time level.
int compute_fields(lb_handle* h) {
  if (!h->initialised) return set_err(LB_ESTATE, "handle not initialised");
  int rc = ensure_fields(h);
  if (rc) return rc;
  LB_CUDA(launch_step(h->storage, h->mode == 0 ? LOAD_FIELDS : LOAD_PULL, false, true, 0, h->g, h->p, h->S[h->cur],
                      init_buf(h), phi_src(h), AccBufs{nullptr, nullptr}, h->S[h->cur ^ 1], h->fields, h->status,
                      h->stream));
  g_launches += 1;
  return LB_OK;
}

}  // namespace

extern "C" {

const char* lb_strerror(int code) {
  switch (code) {
    case LB_OK: return "ok";
    case LB_EINVAL: return "invalid argument";
    case LB_ENOMEM: return "out of memory";
    case LB_ECUDA: return "CUDA error";
    case LB_EUNSTABLE: return "unstable: non-finite or non-positive density";
    case LB_ETIMEOUT: return "bounded device wait gave up";
    case LB_ESTATE: return "invalid state for this call";
    case LB_EIO: return "file error or incompatible checkpoint";
  }
  return "unknown error";
}

const char* lb_last_error(void) { return g_last_error.c_str(); }

uint64_t lb_launch_count(void) { return g_launches.load(); }

size_t lb_device_bytes(const lb_handle* h) { return h ? h->bytes : 0; }

int64_t lb_time(const lb_handle* h) { return h ? h->t : -1; }

int lb_create(const lb_grid* grid, const lb_params* params, const lb_alloc* alloc, lb_handle** out) {
  if (!out) return set_err(LB_EINVAL, "out is null");
  *out = nullptr;
  int rc = validate(grid, params);
  if (rc) return rc;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return set_err(LB_ECUDA, "no CUDA device");
  }
  lb_handle* h = new lb_handle();
  h->grid = *grid;
  h->params = *params;
  h->storage = params->storage;
  h->g.nx = grid->nx;
  h->g.ny = grid->ny;
  h->g.nz = grid->nz;
  h->g.wx = (grid->walls >> 0) & 1u;
  h->g.wy = (grid->walls >> 1) & 1u;
  h->g.wz = (grid->walls >> 2) & 1u;
  h->g.N = (long long)grid->nx * grid->ny * grid->nz;
  Phys& p = h->p;
  p.tau_a = params->tau_a;
  p.tau_b = params->tau_b;
  p.equal_tau = params->tau_a == params->tau_b;
  p.A2 = 0.5 * (params->A_a + params->A_b);
  p.beta = params->beta;
  p.A_h = params->A_h;
  p.h_min = params->h_min;
  p.h_max = params->h_max;
  p.K = params->A_h != 0.0 ? (int)std::floor(params->h_max) : 0;
  p.phi_I = params->phi_I;
  for (int a = 0; a < 3; ++a) p.g[a] = params->g[a];
  p.g_mode = params->g_mode;
  p.collision = params->collision;
  p.model = params->model;
  p.G = params->G;
  p.psi0 = params->psi0;
  if (alloc && alloc->alloc && alloc->free) {
    h->alloc = *alloc;
    h->have_alloc = true;
  }
  cudaError_t e = cudaStreamCreate(&h->own_stream);
  if (e != cudaSuccess) {
    delete h;
    return cuda_err(e, "cudaStreamCreate");
  }
  h->stream = h->own_stream;
  const size_t N = (size_t)h->g.N;
  bool ok = alloc_state(h, h->S[0]) && alloc_state(h, h->S[1]);
  ok = ok && (h->phi = dev_alloc(h, N * real_bytes(h->storage))) != nullptr;
  for (int k = 0; k < 3; ++k) ok = ok && (h->acc[k] = (unsigned long long*)dev_alloc(h, acc_bytes(h))) != nullptr;
  ok = ok && (h->init_phi = (float*)dev_alloc(h, N * sizeof(float))) != nullptr;
  ok = ok && (h->red = (double*)dev_alloc(h, ((size_t)reduce_blocks(h->g.N) * 8 + 16) * sizeof(double))) != nullptr;
  ok = ok && (h->status = (unsigned*)dev_alloc(h, 256)) != nullptr;
  ok = ok && (h->count = (int*)dev_alloc(h, 256)) != nullptr;
  if (!ok) {
    lb_destroy(h);
    return set_err(LB_ENOMEM, "device allocation failed");
  }
  if ((e = cudaMemsetAsync(h->status, 0, sizeof(unsigned), h->stream)) != cudaSuccess ||
      (e = reset_acc(h)) != cudaSuccess) {
    lb_destroy(h);
    return cuda_err(e, "cudaMemsetAsync");
  }
  *out = h;
  return LB_OK;
}

int lb_destroy(lb_handle* h) {
  if (!h) return LB_OK;
  if (h->stream) cudaStreamSynchronize(h->stream);
  drop_graphs(h);
  if (h->surrogate) destroy_surrogate(h->surrogate);
  while (!h->owned.empty()) dev_free(h, h->owned.back().first);
  if (h->own_stream) cudaStreamDestroy(h->own_stream);
  delete h;
  return LB_OK;
}

int lb_set_stream(lb_handle* h, void* stream) {
  if (!h) return set_err(LB_EINVAL, "null handle");
  cudaStream_t s = (cudaStream_t)stream;
  cudaStream_t next = s ? s : h->own_stream;
  if (next != h->stream) {
    // order the switch: the new stream waits for work already on the old one
    cudaEvent_t ev;
    LB_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    cudaEventRecord(ev, h->stream);
    cudaStreamWaitEvent(next, ev, 0);
    cudaEventDestroy(ev);
    h->stream = next;
  }
  drop_graphs(h);
  return LB_OK;
}

int lb_init_droplets(lb_handle* h, int32_t n, const double* centres, const double* radii, double width) {
  if (!h) return set_err(LB_EINVAL, "null handle");
  if (n < 0 || n > (1 << 20)) return set_err(LB_EINVAL, "droplet count out of range");
  if (n > 0 && (!centres || !radii)) return set_err(LB_EINVAL, "null droplet arrays");
  if (!(width >= 0.0) || !std::isfinite(width)) return set_err(LB_EINVAL, "width must be finite and >= 0");
  for (int d = 0; d < n; ++d)
    if (!std::isfinite(radii[d]) || !std::isfinite(centres[3 * d]) || !std::isfinite(centres[3 * d + 1]) ||
        !std::isfinite(centres[3 * d + 2]))
      return set_err(LB_EINVAL, "non-finite droplet");
  double* dbuf = nullptr;
  if (n > 0) {
    dbuf = (double*)dev_alloc(h, sizeof(double) * 4 * (size_t)n);
    if (!dbuf) return set_err(LB_ENOMEM, "droplet buffer allocation failed");
    cudaError_t e = cudaMemcpyAsync(dbuf, centres, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(dbuf + 3 * n, radii, sizeof(double) * n, cudaMemcpyHostToDevice, h->stream);
    if (e != cudaSuccess) {
      dev_free(h, dbuf);
      return cuda_err(e, "droplet copy");
    }
  }
  cudaError_t e = launch_init_droplets(h->g, n, dbuf, dbuf ? dbuf + 3 * n : nullptr, width, h->init_phi, nullptr,
                                       nullptr, h->stream);
  if (e == cudaSuccess) e = launch_phi_from_init(h->storage, h->g, h->init_phi, h->phi, h->stream);
  if (e == cudaSuccess) e = reset_acc(h);
  g_launches += 2;
  if (dbuf) {
    cudaStreamSynchronize(h->stream);
    dev_free(h, dbuf);
  }
  if (e != cudaSuccess) return cuda_err(e, "init droplets");
  h->use_rho = h->use_u = false;
  h->regularised = 0;
  h->mode = 0;
  h->t = 0;
  h->initialised = true;
  return LB_OK;
}

int lb_init_fields(lb_handle* h, const float* phi, const float* rho, const float* u, int regularised, int is_device) {
  if (!h) return set_err(LB_EINVAL, "null handle");
  if (!phi) return set_err(LB_EINVAL, "phi is required");
  if (regularised && !u) return set_err(LB_EINVAL, "regularised reconstruction needs u");
  const size_t N = (size_t)h->g.N;
  const cudaMemcpyKind kind = is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  LB_CUDA(cudaMemcpyAsync(h->init_phi, phi, N * sizeof(float), kind, h->stream));
  if (rho) {
    if (!h->init_rho && !(h->init_rho = (float*)dev_alloc(h, N * sizeof(float))))
      return set_err(LB_ENOMEM, "rho buffer allocation failed");
    LB_CUDA(cudaMemcpyAsync(h->init_rho, rho, N * sizeof(float), kind, h->stream));
  }
  if (u) {
    if (!h->init_u && !(h->init_u = (float*)dev_alloc(h, 3 * N * sizeof(float))))
      return set_err(LB_ENOMEM, "u buffer allocation failed");
    LB_CUDA(cudaMemcpyAsync(h->init_u, u, 3 * N * sizeof(float), kind, h->stream));
  }
  LB_CUDA(launch_phi_from_init(h->storage, h->g, h->init_phi, h->phi, h->stream));
  LB_CUDA(reset_acc(h));
  g_launches += 1;
  if (!is_device) LB_CUDA(cudaStreamSynchronize(h->stream));
  h->use_rho = rho != nullptr;
  h->use_u = u != nullptr;
  h->regularised = regularised ? 1 : 0;
  h->mode = 0;
  h->t = 0;
  h->initialised = true;
  return LB_OK;
}

int lb_step(lb_handle* h, int64_t nsteps) {
  if (!h) return set_err(LB_EINVAL, "null handle");
  if (nsteps < 0) return set_err(LB_EINVAL, "nsteps must be >= 0");
  if (!h->initialised) return set_err(LB_ESTATE, "handle not initialised");
  int rc;
  if (nsteps > 0 && h->mode == 0) {
    if ((rc = issue_step(h))) return rc;
    --nsteps;
  }
  while (nsteps >= STEPS_PER_GRAPH) {
    const int key = graph_key(h);
    if (!h->graph[key] && (rc = build_graph(h))) return rc;
    LB_CUDA(cudaGraphLaunch(h->graph[key], h->stream));
    g_launches += h->graph_launches;
    h->t += STEPS_PER_GRAPH;  // parity and accumulator phase unchanged
    nsteps -= STEPS_PER_GRAPH;
  }
  while (nsteps-- > 0)
    if ((rc = issue_step(h))) return rc;
  return LB_OK;
}

int lb_step_timed(lb_handle* h, int64_t nsteps, double* ms) {
  if (!h || !ms) return set_err(LB_EINVAL, "null argument");
  if (nsteps < 1 || nsteps > 100000) return set_err(LB_EINVAL, "nsteps must lie in [1, 100000]");
  if (!h->initialised) return set_err(LB_ESTATE, "handle not initialised");
  int rc;
  if (h->mode == 0 && (rc = issue_step(h))) return rc;
  std::vector<cudaEvent_t> ev((size_t)(nsteps + 1));
  for (auto& e : ev) LB_CUDA(cudaEventCreate(&e));
  cudaError_t err = cudaEventRecord(ev[0], h->stream);
  for (int64_t k = 0; k < nsteps && err == cudaSuccess; ++k) {
    if ((rc = issue_step(h))) {
      for (auto& e : ev) cudaEventDestroy(e);
      return rc;
    }
    err = cudaEventRecord(ev[(size_t)k + 1], h->stream);
  }
  if (err == cudaSuccess) err = cudaStreamSynchronize(h->stream);
  double s = 0.0;
  for (int64_t k = 0; k < nsteps && err == cudaSuccess; ++k) {
    float a = 0;
    err = cudaEventElapsedTime(&a, ev[(size_t)k], ev[(size_t)k + 1]);
    s += a;
  }
  for (auto& e : ev) cudaEventDestroy(e);
  if (err != cudaSuccess) return cuda_err(err, "lb_step_timed");
  *ms = s / (double)nsteps;
  return LB_OK;
}

int lb_set_tile(lb_handle* h, int tile) {
  if (!h) return set_err(LB_EINVAL, "null handle");
  if (tile < 0 || tile >= NUM_TILES) return set_err(LB_EINVAL, "tile index out of range");
  if (tile != h->tile) drop_graphs(h);
  h->tile = tile;
  return LB_OK;
}

int lb_get_tile(const lb_handle* h) { return h ? h->tile : -1; }

static int fields_out(lb_handle* h, uint32_t mask, void* dst, int dst_is_device, bool dbl) {
  if (!h) return set_err(LB_EINVAL, "null handle");
  if (!dst) return set_err(LB_EINVAL, "dst is null");
  if (mask == 0 || (mask >> NFIELDS)) return set_err(LB_EINVAL, "field mask must select fields 0..13");
  int rc = compute_fields(h);
  if (rc) return rc;
  const size_t N = (size_t)h->g.N;
  const bool f64 = storage_is_f64(h->storage);
  const size_t ob = dbl ? sizeof(double) : sizeof(float);
  void* tmp = nullptr;
  if (f64 != dbl) {  // need a converted copy
    tmp = dev_alloc(h, N * ob);
    if (!tmp) return set_err(LB_ENOMEM, "conversion buffer allocation failed");
  }
  int slot = 0;
  for (int k = 0; k < NFIELDS; ++k) {
    if (!((mask >> k) & 1u)) continue;
    const char* src = (const char*)h->fields + (size_t)k * N * real_bytes(h->storage);
    char* d = (char*)dst + (size_t)slot * N * ob;
    const void* from = src;
    if (tmp) {
      const int blocks = (int)std::min<long long>((N + 255) / 256, 4096);
      if (dbl) k_convert_d<float><<<blocks, 256, 0, h->stream>>>((long long)N, (const float*)src, (double*)tmp);
      else k_convert<double><<<blocks, 256, 0, h->stream>>>((long long)N, (const double*)src, (float*)tmp);
      g_launches += 1;
      from = tmp;
    }
    cudaError_t e = cudaMemcpyAsync(d, from, N * ob, dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                    h->stream);
    if (e != cudaSuccess) {
      if (tmp) dev_free(h, tmp);
      return cuda_err(e, "fields copy");
    }
    ++slot;
  }
  if (!dst_is_device || tmp) {
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (tmp) dev_free(h, tmp);
    if (e != cudaSuccess) return cuda_err(e, "fields sync");
  }
  return LB_OK;
}

int lb_fields(lb_handle* h, uint32_t mask, float* dst, int dst_is_device) {
  return fields_out(h, mask, dst, dst_is_device, false);
}

int lb_fields_f64(lb_handle* h, uint32_t mask, double* dst, int dst_is_device) {
  return fields_out(h, mask, dst, dst_is_device, true);
}

int lb_get_populations(lb_handle* h, int32_t x0, int32_t y0, int32_t z0, int32_t bx, int32_t by, int32_t bz,
                       double* fA, double* fB) {
  if (!h) return set_err(LB_EINVAL, "null handle");
  if (!h->initialised) return set_err(LB_ESTATE, "handle not initialised");
  if (!fA || !fB) return set_err(LB_EINVAL, "null output");
  if (bx < 1 || by < 1 || bz < 1 || x0 < 0 || y0 < 0 || z0 < 0 || x0 + bx > h->g.nx || y0 + by > h->g.ny ||
      z0 + bz > h->g.nz)
    return set_err(LB_EINVAL, "box outside the grid");
  const size_t M = (size_t)bx * by * bz;
  double* d = (double*)dev_alloc(h, 2 * (size_t)Q * M * sizeof(double));
  if (!d) return set_err(LB_ENOMEM, "export buffer allocation failed");
  cudaError_t e = launch_export(h->storage, h->mode == 0 ? LOAD_FIELDS : LOAD_PULL, h->g, h->p, h->S[h->cur], init_buf(h), x0,
                      y0, z0, bx, by, bz, d, d + (size_t)Q * M, h->stream);
  g_launches += 1;
  if (e == cudaSuccess) e = cudaMemcpyAsync(fA, d, (size_t)Q * M * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(fB, d + (size_t)Q * M, (size_t)Q * M * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  dev_free(h, d);
  return cuda_err(e, "get populations");
}

int lb_reduce_f64(lb_handle* h, double* out) {
  if (!h || !out) return set_err(LB_EINVAL, "null argument");
  int rc = compute_fields(h);
  if (rc) return rc;
  const int nb = reduce_blocks(h->g.N);
  double* res = h->red + (size_t)nb * 8;
  LB_CUDA(launch_reduce(h->storage, h->g, h->fields, h->red, res, h->stream));
  g_launches += 2;
  LB_CUDA(cudaMemcpyAsync(out, res, 8 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  LB_CUDA(cudaStreamSynchronize(h->stream));
  return LB_OK;
}

int lb_laplace_f64(lb_handle* h, double cut, double* dp) {
  if (!h || !dp) return set_err(LB_EINVAL, "null argument");
  if (!(cut >= 0.0 && cut < 1.0)) return set_err(LB_EINVAL, "cut must lie in [0, 1)");
  int rc = compute_fields(h);
  if (rc) return rc;
  const int nb = reduce_blocks(h->g.N);
  double* res = h->red + (size_t)nb * 8;
  LB_CUDA(launch_laplace(h->storage, h->g, h->fields, cut, h->red, res, h->stream));
  g_launches += 2;
  double r[4];
  LB_CUDA(cudaMemcpyAsync(r, res, 4 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  LB_CUDA(cudaStreamSynchronize(h->stream));
  if (r[1] == 0.0 || r[3] == 0.0) return set_err(LB_ESTATE, "inside or outside region is empty");
  *dp = (r[0] / r[1] - r[2] / r[3]) / 3.0;
  return LB_OK;
}

int lb_droplet_count(lb_handle* h, int32_t* count) {
  if (!h || !count) return set_err(LB_EINVAL, "null argument");
  int rc = compute_fields(h);
  if (rc) return rc;
  if (!h->labels && !(h->labels = (int*)dev_alloc(h, (size_t)h->g.N * sizeof(int))))
    return set_err(LB_ENOMEM, "label buffer allocation failed");
  LB_CUDA(launch_cc(h->storage, h->g, h->fields, h->labels, h->count, h->status, h->stream));
  g_launches += 3;
  int c = 0;
  unsigned st = 0;
  LB_CUDA(cudaMemcpyAsync(&c, h->count, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  LB_CUDA(cudaMemcpyAsync(&st, h->status, sizeof(unsigned), cudaMemcpyDeviceToHost, h->stream));
  LB_CUDA(cudaStreamSynchronize(h->stream));
  if (st & 2u) return set_err(LB_ETIMEOUT, "union-find gave up after its iteration limit");
  *count = c;
  return LB_OK;
}

int lb_phi_monitor(lb_handle* h, const float* phi, int32_t* count, double* volume) {
  if (!h || !phi || !count || !volume) return set_err(LB_EINVAL, "null argument");
  if (!h->labels && !(h->labels = (int*)dev_alloc(h, (size_t)h->g.N * sizeof(int))))
    return set_err(LB_ENOMEM, "label buffer allocation failed");
  double* vol_dev = h->red + (size_t)reduce_blocks(h->g.N) * 8;  // past the partials
  LB_CUDA(launch_phi_monitor(h->g, phi, h->labels, h->count, h->red, vol_dev, h->status, h->stream));
  g_launches += 5;
  int c = 0;
  unsigned st = 0;
  double v = 0.0;
  LB_CUDA(cudaMemcpyAsync(&c, h->count, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  LB_CUDA(cudaMemcpyAsync(&v, vol_dev, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  LB_CUDA(cudaMemcpyAsync(&st, h->status, sizeof(unsigned), cudaMemcpyDeviceToHost, h->stream));
  LB_CUDA(cudaStreamSynchronize(h->stream));
  if (st & 2u) return set_err(LB_ETIMEOUT, "union-find gave up after its iteration limit");
  *count = c;
  *volume = v;
  return LB_OK;
}

int lb_check(lb_handle* h) {
  if (!h) return set_err(LB_EINVAL, "null handle");
  unsigned st = 0;
  LB_CUDA(cudaMemcpyAsync(&st, h->status, sizeof(unsigned), cudaMemcpyDeviceToHost, h->stream));
  LB_CUDA(cudaStreamSynchronize(h->stream));
  if (st & 1u) return set_err(LB_EUNSTABLE, "non-finite or non-positive density met");
  if (st & 2u) return set_err(LB_ETIMEOUT, "a bounded device loop gave up");
  return LB_OK;
}

int lb_save(lb_handle* h, const char* path) {
  if (!h || !path) return set_err(LB_EINVAL, "null argument");
  if (!h->initialised) return set_err(LB_ESTATE, "handle not initialised");
  FILE* fp = std::fopen(path, "wb");
  if (!fp) return set_err(LB_EIO, std::string("cannot open ") + path);
  const size_t N = (size_t)h->g.N;
  const size_t sb = state_bytes(h);
  std::vector<char> buf(h->mode == 1 ? sb : N * sizeof(float) * 5);
  cudaError_t e = cudaSuccess;
  int32_t hdr[4] = {(int32_t)CKPT_MAGIC, (int32_t)CKPT_VERSION, h->mode, h->regularised};
  bool ok = std::fwrite(hdr, sizeof(hdr), 1, fp) == 1 && std::fwrite(&h->grid, sizeof(lb_grid), 1, fp) == 1 &&
            std::fwrite(&h->params, sizeof(lb_params), 1, fp) == 1 && std::fwrite(&h->t, sizeof(int64_t), 1, fp) == 1;
  if (ok && h->mode == 1) {
    const StateBuf& s = h->S[h->cur];
    if (storage_is_twoset(h->storage)) {
      e = cudaMemcpyAsync(buf.data(), s.f, sb, cudaMemcpyDeviceToHost, h->stream);
    } else {
      const size_t fb = (size_t)state_arrays(h->storage) * N * elem_bytes(h->storage);
      e = cudaMemcpyAsync(buf.data(), s.f, fb, cudaMemcpyDeviceToHost, h->stream);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(buf.data() + fb, s.sv, N * sizeof(float4), cudaMemcpyDeviceToHost, h->stream);
    }
  } else if (ok) {
    int32_t flags[2] = {h->use_rho, h->use_u};
    ok = std::fwrite(flags, sizeof(flags), 1, fp) == 1;
    e = cudaMemcpyAsync(buf.data(), h->init_phi, N * sizeof(float), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess && h->use_rho)
      e = cudaMemcpyAsync(buf.data() + N * 4, h->init_rho, N * 4, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess && h->use_u)
      e = cudaMemcpyAsync(buf.data() + 2 * N * 4, h->init_u, 3 * N * 4, cudaMemcpyDeviceToHost, h->stream);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) {
    std::fclose(fp);
    return cuda_err(e, "checkpoint copy");
  }
  ok = ok && std::fwrite(buf.data(), 1, buf.size(), fp) == buf.size();
  ok = (std::fclose(fp) == 0) && ok;
  return ok ? LB_OK : set_err(LB_EIO, "checkpoint write failed");
}

int lb_load(lb_handle* h, const char* path) {
  if (!h || !path) return set_err(LB_EINVAL, "null argument");
  FILE* fp = std::fopen(path, "rb");
  if (!fp) return set_err(LB_EIO, std::string("cannot open ") + path);
  int32_t hdr[4];
  lb_grid gr;
  lb_params pr;
  int64_t t;
  bool ok = std::fread(hdr, sizeof(hdr), 1, fp) == 1 && std::fread(&gr, sizeof(gr), 1, fp) == 1 &&
            std::fread(&pr, sizeof(pr), 1, fp) == 1 && std::fread(&t, sizeof(t), 1, fp) == 1;
  if (!ok || hdr[0] != (int32_t)CKPT_MAGIC || hdr[1] != (int32_t)CKPT_VERSION || gr.nx != h->grid.nx ||
      gr.ny != h->grid.ny || gr.nz != h->grid.nz || gr.walls != h->grid.walls || pr.storage != h->storage) {
    std::fclose(fp);
    return set_err(LB_EIO, "not a checkpoint of this grid and storage");
  }
  const size_t N = (size_t)h->g.N;
  cudaError_t e = cudaSuccess;
  if (hdr[2] == 1) {
    const size_t sb = state_bytes(h);
    std::vector<char> buf(sb);
    ok = std::fread(buf.data(), 1, sb, fp) == sb;
    std::fclose(fp);
    if (!ok) return set_err(LB_EIO, "truncated checkpoint");
    const StateBuf& s = h->S[h->cur];
    if (storage_is_twoset(h->storage)) {
      e = cudaMemcpyAsync(s.f, buf.data(), sb, cudaMemcpyHostToDevice, h->stream);
    } else {
      const size_t fb = (size_t)state_arrays(h->storage) * N * elem_bytes(h->storage);
      e = cudaMemcpyAsync(s.f, buf.data(), fb, cudaMemcpyHostToDevice, h->stream);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(s.sv, buf.data() + fb, N * sizeof(float4), cudaMemcpyHostToDevice, h->stream);
    }
    if (e == cudaSuccess) e = rebuild_acc(h);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_err(e, "checkpoint upload");
    drop_graphs(h);
    h->mode = 1;
  } else {
    int32_t flags[2];
    ok = std::fread(flags, sizeof(flags), 1, fp) == 1;
    std::vector<char> buf(N * sizeof(float) * 5);
    ok = ok && std::fread(buf.data(), 1, buf.size(), fp) == buf.size();
    std::fclose(fp);
    if (!ok) return set_err(LB_EIO, "truncated checkpoint");
    const float* fl = (const float*)buf.data();
    int rc = lb_init_fields(h, fl, flags[0] ? fl + N : nullptr, flags[1] ? fl + 2 * N : nullptr, hdr[3], 0);
    if (rc) return rc;
  }
  h->t = t;
  h->initialised = true;
  return LB_OK;
}

int lb_copy_state(lb_handle* dst, lb_handle* src) {
  if (!dst || !src) return set_err(LB_EINVAL, "null handle");
  if (dst == src) return LB_OK;
  if (!src->initialised) return set_err(LB_ESTATE, "source handle not initialised");
  if (src->grid.nx != dst->grid.nx || src->grid.ny != dst->grid.ny || src->grid.nz != dst->grid.nz ||
      src->grid.walls != dst->grid.walls || src->storage != dst->storage)
    return set_err(LB_EINVAL, "handles differ in grid or storage");
  const size_t N = (size_t)src->g.N;
  cudaError_t e = cudaStreamSynchronize(src->stream);
  if (e == cudaSuccess && src->mode == 1) {
    const StateBuf& a = src->S[src->cur];
    const StateBuf& b = dst->S[dst->cur];
    if (storage_is_twoset(src->storage)) {
      e = cudaMemcpyAsync(b.f, a.f, state_bytes(src), cudaMemcpyDeviceToDevice, dst->stream);
    } else {
      const size_t fb = (size_t)state_arrays(src->storage) * N * elem_bytes(src->storage);
      e = cudaMemcpyAsync(b.f, a.f, fb, cudaMemcpyDeviceToDevice, dst->stream);
      if (e == cudaSuccess) e = cudaMemcpyAsync(b.sv, a.sv, N * sizeof(float4), cudaMemcpyDeviceToDevice, dst->stream);
    }
    if (e == cudaSuccess) e = rebuild_acc(dst);
  } else if (e == cudaSuccess) {
    e = cudaMemcpyAsync(dst->init_phi, src->init_phi, N * sizeof(float), cudaMemcpyDeviceToDevice, dst->stream);
    if (e == cudaSuccess && src->use_rho) {
      if (!dst->init_rho && !(dst->init_rho = (float*)dev_alloc(dst, N * sizeof(float))))
        return set_err(LB_ENOMEM, "field buffer allocation failed");
      e = cudaMemcpyAsync(dst->init_rho, src->init_rho, N * sizeof(float), cudaMemcpyDeviceToDevice, dst->stream);
    }
    if (e == cudaSuccess && src->use_u) {
      if (!dst->init_u && !(dst->init_u = (float*)dev_alloc(dst, 3 * N * sizeof(float))))
        return set_err(LB_ENOMEM, "field buffer allocation failed");
      e = cudaMemcpyAsync(dst->init_u, src->init_u, 3 * N * sizeof(float), cudaMemcpyDeviceToDevice, dst->stream);
    }
    if (e == cudaSuccess) e = launch_phi_from_init(dst->storage, dst->g, dst->init_phi, dst->phi, dst->stream);
    if (e == cudaSuccess) e = reset_acc(dst);
  }
  if (e != cudaSuccess) return cuda_err(e, "copy state");
  drop_graphs(dst);
  dst->mode = src->mode;
  dst->use_rho = src->use_rho;
  dst->use_u = src->use_u;
  dst->regularised = src->regularised;
  dst->t = src->t;
  dst->initialised = true;
  return LB_OK;
}

}  // extern "C"

// ===========================================================================
// batches of independent runs
// ===========================================================================
struct lb_batch {
  std::vector<lb_handle*> runs;
  int storage = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t own_stream = nullptr;
  RunDesc* d_runs = nullptr;
  std::vector<RunDesc> h_runs;
  long long ntiles = 0, max_nodes = 0, total_nodes = 0;
  int halo = 1;  // largest staging halo of the runs
  int tile = 0;
  int blocks_per_sm = 2;
  bool dirty = true;
  uint64_t graph_launches = 0;  // kernel launches in one replay
  cudaGraphExec_t graph[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};  // [parity * 3 + phase]
};

namespace {

constexpr int BATCH_STEPS_PER_GRAPH = 12;  // a multiple of 2 and 3, as STEPS_PER_GRAPH

void batch_drop_graphs(lb_batch* b) {
  for (int k = 0; k < 6; ++k) {
    if (b->graph[k]) cudaGraphExecDestroy(b->graph[k]);
    b->graph[k] = nullptr;
  }
}

int batch_descriptors(lb_batch* b) {
  const Tile& T = kTiles[b->tile];
  long long tb = 0;
  b->halo = 1;
  b->max_nodes = 0;
  b->h_runs.resize(b->runs.size());
  for (size_t r = 0; r < b->runs.size(); ++r) {
    lb_handle* h = b->runs[r];
    RunDesc& d = b->h_runs[r];
    d.g = h->g;
    d.p = h->p;
    d.S[0] = h->S[0];
    d.S[1] = h->S[1];
    for (int k = 0; k < 3; ++k) d.acc[k] = h->acc[k];
    d.tiles_x = (h->g.nx + T.tx - 1) / T.tx;
    d.tiles_y = (h->g.ny + T.ty - 1) / T.ty;
    d.tiles_z = (h->g.nz + T.tz - 1) / T.tz;
    d.tile_begin = tb;
    tb += (long long)d.tiles_x * d.tiles_y * d.tiles_z;
    b->halo = std::max(b->halo, stage_halo(h->p));
    b->max_nodes = std::max(b->max_nodes, h->g.N);
  }
  b->ntiles = tb;
  LB_CUDA(cudaMemcpyAsync(b->d_runs, b->h_runs.data(), sizeof(RunDesc) * b->h_runs.size(), cudaMemcpyHostToDevice,
                          b->stream));
  LB_CUDA(cudaStreamSynchronize(b->stream));
  b->dirty = false;
  return LB_OK;
}

// one batched step from lattice parity `parity` and accumulator phase k
int batch_issue(lb_batch* b, int parity, int k) {
  LB_CUDA(launch_batched(b->storage, b->d_runs, (int)b->runs.size(), b->ntiles, b->tile, b->halo, b->max_nodes,
                         parity, k, b->blocks_per_sm, b->runs[0]->status, b->stream));
  g_launches += 1;
  return LB_OK;
}

int batch_build_graph(lb_batch* b, int parity, int phase) {
  cudaGraph_t graph = nullptr;
  const uint64_t save_l = g_launches.load();
  LB_CUDA(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
  int rc = LB_OK;
  for (int k = 0; k < BATCH_STEPS_PER_GRAPH && rc == LB_OK; ++k) rc = batch_issue(b, parity ^ (k & 1), (phase + k) % 3);
  cudaError_t e = cudaStreamEndCapture(b->stream, &graph);
  b->graph_launches = g_launches.load() - save_l;
  g_launches = save_l;
  if (rc != LB_OK) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  if (e != cudaSuccess) return cuda_err(e, "cudaStreamEndCapture");
  e = cudaGraphInstantiate(&b->graph[parity * 3 + phase], graph, 0);
  cudaGraphDestroy(graph);
  return cuda_err(e, "cudaGraphInstantiate");
}

// bring every run to the population state, a common parity and a common
// accumulator phase (the accumulators of a run are renamed, not copied)
int batch_prepare(lb_batch* b) {
  for (lb_handle* h : b->runs) {
    if (!h->initialised) return set_err(LB_ESTATE, "a run of the batch is not initialised");
    if (h->mode == 0) {
      int rc = issue_step(h);
      if (rc) return rc;
    }
  }
  const int par = b->runs[0]->cur, k0 = b->runs[0]->phi_acc;
  for (lb_handle* h : b->runs) {
    if (h->cur != par) return set_err(LB_ESTATE, "runs of the batch are at different parities");
    if (h->phi_acc != k0) {
      unsigned long long* old[3] = {h->acc[0], h->acc[1], h->acc[2]};
      for (int j = 0; j < 3; ++j) h->acc[j] = old[(j - k0 + h->phi_acc + 3) % 3];
      h->phi_acc = k0;
      drop_graphs(h);
      b->dirty = true;
      batch_drop_graphs(b);
    }
  }
  if (b->dirty) return batch_descriptors(b);
  return LB_OK;
}

void batch_advance(lb_batch* b, int64_t n) {
  for (lb_handle* h : b->runs) {
    h->t += n;
    h->cur ^= (int)(n & 1);
    h->phi_acc = (int)((h->phi_acc + n) % 3);
  }
}

std::string tune_cache_path() {
  const char* p = std::getenv("LBCG_TUNE_CACHE");
  if (p && p[0]) return p;
  const char* home = std::getenv("HOME");
  return std::string(home ? home : "/tmp") + "/.cache/lbcg_tune.txt";
}

std::string batch_key(const lb_batch* b) {
  cudaDeviceProp prop{};
  int dev = 0;
  cudaGetDevice(&dev);
  cudaGetDeviceProperties(&prop, dev);
  std::vector<std::string> shapes;
  for (lb_handle* h : b->runs) {
    std::ostringstream os;
    os << h->g.nx << "x" << h->g.ny << "x" << h->g.nz << "w" << h->grid.walls << "h" << stage_halo(h->p);
    shapes.push_back(os.str());
  }
  std::sort(shapes.begin(), shapes.end());
  std::ostringstream key;
  std::string name = prop.name;
  for (char& c : name)
    if (c == ' ') c = '_';
  key << name << "|st" << b->storage << "|";
  for (auto& sh : shapes) key << sh << ",";
  return key.str();
}

int batch_tune(lb_batch* b, int32_t steps, int use_cache, double* result);

}  // namespace

extern "C" {

int lb_batch_create(int32_t nruns, const lb_grid* grids, const lb_params* params, const lb_alloc* alloc,
                    lb_batch** out) {
  if (!out) return set_err(LB_EINVAL, "out is null");
  *out = nullptr;
  if (nruns < 1 || nruns > 65536 || !grids || !params) return set_err(LB_EINVAL, "need 1..65536 runs with grids and params");
  for (int r = 0; r < nruns; ++r) {
    int rc = validate(&grids[r], &params[r]);
    if (rc) return rc;
    if (params[r].storage != params[0].storage) return set_err(LB_EINVAL, "all runs of a batch share one storage");
    if (params[r].model != LB_MODEL_COLOUR_GRADIENT) return set_err(LB_EINVAL, "batches run the colour-gradient model");
  }
  if (params[0].storage == LB_STORAGE_TWOSET_F64 || params[0].storage == LB_STORAGE_MOMENT_F32)
    return set_err(LB_EINVAL, "batches support the two-set and reduced FP32/FP16 storages only");
  lb_batch* b = new lb_batch();
  b->storage = params[0].storage;
  cudaError_t e = cudaStreamCreate(&b->own_stream);
  if (e != cudaSuccess) {
    delete b;
    return cuda_err(e, "cudaStreamCreate");
  }
  b->stream = b->own_stream;
  for (int r = 0; r < nruns; ++r) {
    lb_handle* h = nullptr;
    int rc = lb_create(&grids[r], &params[r], alloc, &h);
    if (rc) {
      lb_batch_destroy(b);
      return rc;
    }
    lb_set_stream(h, b->stream);
    b->runs.push_back(h);
    b->total_nodes += h->g.N;
  }
  b->d_runs = (RunDesc*)dev_alloc(b->runs[0], sizeof(RunDesc) * (size_t)nruns);
  if (!b->d_runs) {
    lb_batch_destroy(b);
    return set_err(LB_ENOMEM, "descriptor allocation failed");
  }
  *out = b;
  return LB_OK;
}

int lb_batch_destroy(lb_batch* b) {
  if (!b) return LB_OK;
  if (b->stream) cudaStreamSynchronize(b->stream);
  batch_drop_graphs(b);
  for (size_t r = b->runs.size(); r-- > 0;) lb_destroy(b->runs[r]);  // run 0 owns the descriptors
  if (b->own_stream) cudaStreamDestroy(b->own_stream);
  delete b;
  return LB_OK;
}

lb_handle* lb_batch_run(lb_batch* b, int32_t run) {
  if (!b || run < 0 || run >= (int)b->runs.size()) {
    set_err(LB_EINVAL, "run index out of range");
    return nullptr;
  }
  b->dirty = true;  // the caller may re-initialise the run
  batch_drop_graphs(b);
  return b->runs[(size_t)run];
}

int32_t lb_batch_size(const lb_batch* b) { return b ? (int32_t)b->runs.size() : -1; }

int64_t lb_batch_nodes(const lb_batch* b) { return b ? b->total_nodes : -1; }

int lb_batch_set_stream(lb_batch* b, void* stream) {
  if (!b) return set_err(LB_EINVAL, "null batch");
  cudaStream_t next = stream ? (cudaStream_t)stream : b->own_stream;
  for (lb_handle* h : b->runs) {
    int rc = lb_set_stream(h, next);
    if (rc) return rc;
  }
  b->stream = next;
  batch_drop_graphs(b);
  return LB_OK;
}

int lb_batch_set_tile(lb_batch* b, int tile, int blocks_per_sm) {
  if (!b) return set_err(LB_EINVAL, "null batch");
  if (tile < 0 || tile >= NUM_TILES || blocks_per_sm < 1 || blocks_per_sm > 16)
    return set_err(LB_EINVAL, "tile in 0..5 and blocks_per_sm in 1..16");
  if (tile != b->tile || blocks_per_sm != b->blocks_per_sm) {
    b->tile = tile;
    b->blocks_per_sm = blocks_per_sm;
    b->dirty = true;
    batch_drop_graphs(b);
  }
  return LB_OK;
}

int lb_batch_step(lb_batch* b, int64_t nsteps) {
  if (!b) return set_err(LB_EINVAL, "null batch");
  if (nsteps < 0) return set_err(LB_EINVAL, "nsteps must be >= 0");
  if (nsteps == 0) return LB_OK;
  int rc;
  bool first_done = false;
  for (lb_handle* h : b->runs)
    if (h->mode == 0) first_done = true;
  if ((rc = batch_prepare(b))) return rc;
  if (first_done) {  // the first step of freshly initialised runs was taken per run
    for (lb_handle* h : b->runs)
      if (h->t == 0) return set_err(LB_ESTATE, "internal: run not advanced");
    --nsteps;
  }
  while (nsteps >= BATCH_STEPS_PER_GRAPH) {
    const int par = b->runs[0]->cur, ph = b->runs[0]->phi_acc, key = par * 3 + ph;
    if (!b->graph[key] && (rc = batch_build_graph(b, par, ph))) return rc;
    LB_CUDA(cudaGraphLaunch(b->graph[key], b->stream));
    g_launches += b->graph_launches;
    batch_advance(b, BATCH_STEPS_PER_GRAPH);
    nsteps -= BATCH_STEPS_PER_GRAPH;
  }
  while (nsteps-- > 0) {
    if ((rc = batch_issue(b, b->runs[0]->cur, b->runs[0]->phi_acc))) return rc;
    batch_advance(b, 1);
  }
  return LB_OK;
}

int lb_batch_step_sequential(lb_batch* b, int64_t nsteps) {
  if (!b) return set_err(LB_EINVAL, "null batch");
  for (lb_handle* h : b->runs) {
    int rc = lb_step(h, nsteps);
    if (rc) return rc;
  }
  return LB_OK;
}

int lb_batch_check(lb_batch* b) {
  if (!b) return set_err(LB_EINVAL, "null batch");
  for (lb_handle* h : b->runs) {
    int rc = lb_check(h);
    if (rc) return rc;
  }
  return LB_OK;
}

int lb_batch_autotune(lb_batch* b, int32_t steps, int use_cache, double* result) {
  if (!b || !result) return set_err(LB_EINVAL, "null argument");
  if (steps < 1 || steps > 1000) return set_err(LB_EINVAL, "steps must lie in [1, 1000]");
  for (lb_handle* h : b->runs)
    if (!h->initialised || h->t != 0) return set_err(LB_ESTATE, "autotune needs freshly initialised runs");
  int rc = batch_tune(b, steps, use_cache, result);
  // the timed steps advanced the runs: return every run to its initial state
  for (lb_handle* h : b->runs) {
    cudaError_t e = launch_phi_from_init(h->storage, h->g, h->init_phi, h->phi, h->stream);
    if (e == cudaSuccess) e = reset_acc(h);
    g_launches += 1;
    if (e != cudaSuccess && rc == LB_OK) rc = cuda_err(e, "autotune reset");
    h->mode = 0;
    h->t = 0;
    h->cur = 0;
  }
  batch_drop_graphs(b);
  return rc;
}

}  // extern "C"

namespace {

int batch_tune(lb_batch* b, int32_t steps, int use_cache, double* result) {
  int rc = batch_prepare(b);
  if (rc) return rc;
  const std::string key = batch_key(b);
  const std::string path = tune_cache_path();
  if (use_cache) {
    std::ifstream in(path);
    std::string k;
    int tile, bps;
    double ms;
    while (in >> k >> tile >> bps >> ms) {
      if (k == key && tile >= 0 && tile < NUM_TILES && bps >= 1 && bps <= 16) {
        if ((rc = lb_batch_set_tile(b, tile, bps))) return rc;
        result[0] = tile;
        result[1] = bps;
        result[2] = ms;
        result[3] = 1;  // from the cache
        return LB_OK;
      }
    }
  }
  const int bps_opts[3] = {1, 2, 4};
  double best = 1e30;
  int best_tile = 0, best_bps = 2;
  cudaEvent_t e0, e1;
  LB_CUDA(cudaEventCreate(&e0));
  LB_CUDA(cudaEventCreate(&e1));
  for (int tile = 0; tile < NUM_TILES; ++tile) {
    for (int bps : bps_opts) {
      if ((rc = lb_batch_set_tile(b, tile, bps)) || (rc = batch_prepare(b))) break;
      for (int k = 0; k < 2 && rc == LB_OK; ++k) {
        rc = batch_issue(b, b->runs[0]->cur, b->runs[0]->phi_acc);
        batch_advance(b, 1);
      }
      cudaEventRecord(e0, b->stream);
      for (int k = 0; k < steps && rc == LB_OK; ++k) {
        rc = batch_issue(b, b->runs[0]->cur, b->runs[0]->phi_acc);
        batch_advance(b, 1);
      }
      cudaEventRecord(e1, b->stream);
      cudaError_t e = cudaEventSynchronize(e1);
      float ms = 0;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (rc == LB_OK && e != cudaSuccess) rc = cuda_err(e, "autotune timing");
      if (rc) break;
      const double per = ms / steps;
      if (per < best) {
        best = per;
        best_tile = tile;
        best_bps = bps;
      }
    }
    if (rc) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  if ((rc = lb_batch_set_tile(b, best_tile, best_bps))) return rc;
  result[0] = best_tile;
  result[1] = best_bps;
  result[2] = best;
  result[3] = 0;
  // append to the cache (best effort; creates the cache directory one level deep)
  const size_t slash = path.find_last_of('/');
  if (slash != std::string::npos) mkdir(path.substr(0, slash).c_str(), 0755);
  if (FILE* fp = std::fopen(path.c_str(), "a")) {
    std::fprintf(fp, "%s %d %d %.6f\n", key.c_str(), best_tile, best_bps, best);
    std::fclose(fp);
  }
  return LB_OK;
}

}  // namespace
