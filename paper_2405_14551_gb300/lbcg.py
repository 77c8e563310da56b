"""ctypes binding of liblbcg.so (the C ABI in include/lbcg.h).

Functions keep the C names (lb_create, lb_step, ...) and only marshal
arguments; every step of the computation runs in the library's CUDA kernels.
PyTorch provides device memory (through the lb_alloc callbacks) and streams.
Importing this module fails loudly when the library has not been built:
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblbcg.so")

LB_OK, LB_EINVAL, LB_ENOMEM, LB_ECUDA, LB_EUNSTABLE, LB_ETIMEOUT, LB_ESTATE, LB_EIO = 0, -1, -2, -3, -4, -5, -6, -7
STORAGE = {"twoset_f32": 0, "reduced_f32": 1, "reduced_f16": 2, "twoset_f64": 3, "moment_f32": 4}
FIELD_NAMES = ("phi", "rho", "ux", "uy", "uz", "rhoA", "rhoB", "Frx", "Fry", "Frz", "h", "gx", "gy", "gz")
FIELD_BIT = {n: 1 << k for k, n in enumerate(FIELD_NAMES)}
ALL_FIELDS = (1 << len(FIELD_NAMES)) - 1
# algorithmic bytes per node update (one read + one write of the stored state)
BYTES_PER_NODE = {0: 2 * 27 * 4 * 2, 1: (27 + 4) * 4 * 2, 2: (27 * 2 + 4 * 4) * 2, 3: 2 * 27 * 8 * 2,
                  4: (10 + 4) * 4 * 2}


class LBError(RuntimeError):
    def __init__(self, code: int, where: str, detail: str):
        super().__init__(f"{where} failed: {code} ({detail})")
        self.code = code


class lb_grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32), ("walls", ctypes.c_uint32)]


class lb_params(ctypes.Structure):
    _fields_ = [
        ("tau_a", ctypes.c_double), ("tau_b", ctypes.c_double),
        ("A_a", ctypes.c_double), ("A_b", ctypes.c_double),
        ("beta", ctypes.c_double),
        ("A_h", ctypes.c_double), ("h_min", ctypes.c_double), ("h_max", ctypes.c_double),
        ("phi_I", ctypes.c_double),
        ("g", ctypes.c_double * 3),
        ("g_mode", ctypes.c_int32),
        ("storage", ctypes.c_int32),
        ("collision", ctypes.c_int32),
        ("model", ctypes.c_int32),
        ("G", ctypes.c_double),
        ("psi0", ctypes.c_double),
    ]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class lb_alloc(ctypes.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("ctx", ctypes.c_void_p)]


# exported symbols and their signatures
_SIGS = {
    "lb_create": (ctypes.c_int, [ctypes.POINTER(lb_grid), ctypes.POINTER(lb_params), ctypes.POINTER(lb_alloc),
                                 ctypes.POINTER(ctypes.c_void_p)]),
    "lb_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "lb_set_stream": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "lb_init_droplets": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_double]),
    "lb_init_fields": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_int, ctypes.c_int]),
    "lb_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64]),
    "lb_set_tile": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "lb_copy_state": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "lb_surrogate_load": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_char_p]),
    "lb_surrogate_predict": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "lb_surrogate_cycle": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_double,
                                          ctypes.c_double, ctypes.POINTER(ctypes.c_int32),
                                          ctypes.POINTER(ctypes.c_double)]),
    "lb_phi_monitor": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32),
                                      ctypes.POINTER(ctypes.c_double)]),
    "lb_step_timed": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]),
    "lb_get_tile": (ctypes.c_int, [ctypes.c_void_p]),
    "lb_time": (ctypes.c_int64, [ctypes.c_void_p]),
    "lb_fields": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_int]),
    "lb_fields_f64": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_int]),
    "lb_get_populations": (ctypes.c_int, [ctypes.c_void_p] + [ctypes.c_int32] * 6 + [ctypes.c_void_p] * 2),
    "lb_reduce_f64": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "lb_laplace_f64": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.POINTER(ctypes.c_double)]),
    "lb_droplet_count": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32)]),
    "lb_check": (ctypes.c_int, [ctypes.c_void_p]),
    "lb_save": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_char_p]),
    "lb_load": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_char_p]),
    "lb_launch_count": (ctypes.c_uint64, []),
    "lb_device_bytes": (ctypes.c_size_t, [ctypes.c_void_p]),
    "lb_batch_create": (ctypes.c_int, [ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(lb_alloc),
                                       ctypes.POINTER(ctypes.c_void_p)]),
    "lb_batch_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "lb_batch_run": (ctypes.c_void_p, [ctypes.c_void_p, ctypes.c_int32]),
    "lb_batch_size": (ctypes.c_int32, [ctypes.c_void_p]),
    "lb_batch_nodes": (ctypes.c_int64, [ctypes.c_void_p]),
    "lb_batch_set_stream": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "lb_batch_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64]),
    "lb_batch_step_sequential": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64]),
    "lb_batch_set_tile": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int]),
    "lb_batch_autotune": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int, ctypes.c_void_p]),
    "lb_batch_check": (ctypes.c_int, [ctypes.c_void_p]),
    "lb_reduce_fields_f64_static": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int32, ctypes.c_int32,
                                                   ctypes.c_int32, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_void_p]),
    "lbnn_set_wait_limit": (ctypes.c_int, [ctypes.c_uint32, ctypes.POINTER(ctypes.c_uint32)]),
    "lbnn_check_status": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "lbnn_conv3d_fwd": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int32,
                                       ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                                       ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_uint32,
                                       ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]),
    "lbnn_conv3d_fwd_upcat": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int32,
                                             ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                             ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                             ctypes.c_int32, ctypes.c_int32, ctypes.c_uint32, ctypes.c_int32,
                                             ctypes.c_void_p, ctypes.c_void_p]),
    "lbnn_conv3d_wgrad": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int32,
                                         ctypes.c_int32, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                                         ctypes.c_int32, ctypes.c_int32, ctypes.c_uint32, ctypes.c_int32,
                                         ctypes.c_void_p, ctypes.c_void_p]),
    "lbnn_pack_input": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_float, ctypes.c_float, ctypes.c_void_p, ctypes.c_void_p]),
    "lbnn_unpack_output": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_void_p, ctypes.c_void_p]),
    "lbnn_pack_target": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_float, ctypes.c_float, ctypes.c_void_p, ctypes.c_void_p]),
    "lbnn_avgpool2": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]),
    "lbnn_avgpool2_bwd": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]),
    "lbnn_up_concat": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]),
    "lbnn_up_concat_bwd": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "lbnn_relu_bwd": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "lbnn_bias_grad": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]),
    "lbnn_flip_weights": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]),
    "lbnn_mse": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "lbnn_adam": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_int32, ctypes.c_float, ctypes.c_void_p, ctypes.c_void_p]),
    "lbnn_f32_to_bf16": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]),
    "lb_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "lb_last_error": (ctypes.c_char_p, []),
}

_lib = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load liblbcg.so; raises when it is missing (no fallback exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with paper_2405_14551_gb300.build.build() "
                          "(there is no CPU fallback)")
    L = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _check(rc: int, where: str):
    if rc != LB_OK:
        L = load_library()
        raise LBError(rc, where, f"{L.lb_strerror(rc).decode()}: {L.lb_last_error().decode()}")


class TorchAllocator:
    """lb_alloc backed by PyTorch's caching allocator on one device."""

    def __init__(self, device):
        import torch
        self._torch = torch
        self.device = torch.device(device)
        self.live = {}
        self._a = ALLOC_FN(self._alloc)
        self._f = FREE_FN(self._free)
        self.struct = lb_alloc(self._a, self._f, None)

    def _alloc(self, ctx, nbytes):
        try:
            t = self._torch.empty(int(nbytes), dtype=self._torch.uint8, device=self.device)
        except RuntimeError:
            return None
        p = t.data_ptr()
        self.live[p] = t
        return p

    def _free(self, ctx, ptr):
        self.live.pop(ptr, None)


# ---------------------------------------------------------------------------
# thin wrappers with the C names
# ---------------------------------------------------------------------------
def make_grid(nx, ny, nz, walls=0) -> lb_grid:
    return lb_grid(int(nx), int(ny), int(nz), int(walls))


def make_params(tau_a=1.0, tau_b=1.0, A_a=0.01, A_b=0.01, beta=0.7, A_h=0.0, h_min=3.0, h_max=3.0, phi_I=0.9,
                g=(0.0, 0.0, 0.0), g_mode=0, storage="twoset_f32", collision=0, model=0, G=0.0,
                psi0=1.0) -> lb_params:
    """model 0: colour gradient; model 1: Shan-Chen (G, psi0; two-set storages only)."""
    st = STORAGE[storage] if isinstance(storage, str) else int(storage)
    p = lb_params()
    p.tau_a, p.tau_b, p.A_a, p.A_b, p.beta = tau_a, tau_b, A_a, A_b, beta
    p.A_h, p.h_min, p.h_max, p.phi_I = A_h, h_min, h_max, phi_I
    p.g[0], p.g[1], p.g[2] = g
    p.g_mode = int(g_mode)
    p.storage = st
    p.collision = int(collision)
    p.model, p.G, p.psi0 = int(model), float(G), float(psi0)
    return p


def lb_create(grid: lb_grid, params: lb_params, alloc: TorchAllocator | None = None) -> ctypes.c_void_p:
    L = load_library()
    h = ctypes.c_void_p()
    _check(L.lb_create(ctypes.byref(grid), ctypes.byref(params), ctypes.byref(alloc.struct) if alloc else None,
                       ctypes.byref(h)), "lb_create")
    return h


def lb_destroy(h):
    _check(load_library().lb_destroy(h), "lb_destroy")


def lb_set_stream(h, stream_ptr: int):
    _check(load_library().lb_set_stream(h, ctypes.c_void_p(stream_ptr)), "lb_set_stream")


def lb_init_droplets(h, centres, radii, width=0.0):
    c = np.ascontiguousarray(np.asarray(centres, dtype=np.float64).reshape(-1, 3))
    r = np.ascontiguousarray(np.asarray(radii, dtype=np.float64).reshape(-1))
    if c.shape[0] != r.shape[0]:
        raise ValueError("centres and radii disagree in length")
    _check(load_library().lb_init_droplets(h, int(r.shape[0]), c.ctypes.data, r.ctypes.data, float(width)),
           "lb_init_droplets")


def lb_init_fields(h, phi, rho=None, u=None, regularised=False):
    """phi, rho, u: float32 numpy arrays (host) or CUDA tensors (device)."""
    is_dev = hasattr(phi, "is_cuda") and phi.is_cuda
    keep = []

    def ptr(a):
        if a is None:
            return None
        if is_dev:
            a = a.contiguous().float()
            keep.append(a)
            return a.data_ptr()
        a = np.ascontiguousarray(a, dtype=np.float32)
        keep.append(a)
        return a.ctypes.data

    _check(load_library().lb_init_fields(h, ptr(phi), ptr(rho), ptr(u), int(bool(regularised)), int(is_dev)),
           "lb_init_fields")


def lb_step(h, nsteps: int):
    _check(load_library().lb_step(h, int(nsteps)), "lb_step")


def lb_step_timed(h, nsteps: int) -> float:
    """Mean ms of one step kernel over nsteps steps (CUDA events on the
    handle's stream, no graph replay)."""
    ms = np.zeros(1)
    _check(load_library().lb_step_timed(h, int(nsteps), ms.ctypes.data), "lb_step_timed")
    return float(ms[0])


def lb_phi_monitor(h, phi):
    """(droplet count, dispersed volume) of a device float32 phase field of the
    handle's grid."""
    c, v = ctypes.c_int32(), ctypes.c_double()
    _check(load_library().lb_phi_monitor(h, ctypes.c_void_p(phi.data_ptr()), ctypes.byref(c), ctypes.byref(v)),
           "lb_phi_monitor")
    return int(c.value), float(v.value)


def lb_surrogate_load(h, path: str):
    _check(load_library().lb_surrogate_load(h, str(path).encode()), "lb_surrogate_load")


def lb_surrogate_predict(h, out=None):
    _check(load_library().lb_surrogate_predict(h, ctypes.c_void_p(out.data_ptr()) if out is not None else None),
           "lb_surrogate_predict")


def lb_surrogate_cycle(h, judge, K: int, vol_tol: float, phi_tol: float):
    """(accepted, judged phi error or -1)."""
    a, e = ctypes.c_int32(), ctypes.c_double()
    _check(load_library().lb_surrogate_cycle(h, judge, int(K), float(vol_tol), float(phi_tol), ctypes.byref(a),
                                             ctypes.byref(e)), "lb_surrogate_cycle")
    return bool(a.value), float(e.value)


def lb_copy_state(dst, src):
    _check(load_library().lb_copy_state(dst, src), "lb_copy_state")


NUM_TILES = 6  # tile shapes of lb_set_tile and lb_batch_set_tile


def lb_set_tile(h, tile: int):
    _check(load_library().lb_set_tile(h, int(tile)), "lb_set_tile")


def lb_get_tile(h) -> int:
    return int(load_library().lb_get_tile(h))


def lb_time(h) -> int:
    return int(load_library().lb_time(h))


def lb_fields(h, mask: int, dst, dst_is_device: bool, f64: bool = False):
    L = load_library()
    p = dst.data_ptr() if dst_is_device else dst.ctypes.data
    fn = L.lb_fields_f64 if f64 else L.lb_fields
    _check(fn(h, int(mask), p, int(bool(dst_is_device))), "lb_fields")


def lb_get_populations(h, box):
    x0, y0, z0, bx, by, bz = (int(v) for v in box)
    a = np.zeros((27, bz, by, bx))
    b = np.zeros((27, bz, by, bx))
    _check(load_library().lb_get_populations(h, x0, y0, z0, bx, by, bz, a.ctypes.data, b.ctypes.data),
           "lb_get_populations")
    return a, b


def lb_reduce_f64(h) -> np.ndarray:
    out = np.zeros(8)
    _check(load_library().lb_reduce_f64(h, out.ctypes.data), "lb_reduce_f64")
    return out


def lb_laplace_f64(h, cut=0.9) -> float:
    dp = ctypes.c_double()
    _check(load_library().lb_laplace_f64(h, float(cut), ctypes.byref(dp)), "lb_laplace_f64")
    return dp.value


def lb_droplet_count(h) -> int:
    c = ctypes.c_int32()
    _check(load_library().lb_droplet_count(h, ctypes.byref(c)), "lb_droplet_count")
    return c.value


def lb_check(h):
    _check(load_library().lb_check(h), "lb_check")


def lb_save(h, path: str):
    _check(load_library().lb_save(h, path.encode()), "lb_save")


def lb_load(h, path: str):
    _check(load_library().lb_load(h, path.encode()), "lb_load")


def lb_reduce_fields_f64_static(fields_ptr: int, fields_are_f64: bool, nx: int, ny: int, nz: int, walls: int,
                                out_ptr: int, stream_ptr: int = 0):
    """Allocation-free FP64 sums of a device fields array into 8 device doubles."""
    _check(load_library().lb_reduce_fields_f64_static(ctypes.c_void_p(fields_ptr), int(bool(fields_are_f64)), int(nx),
                                                      int(ny), int(nz), int(walls), ctypes.c_void_p(out_ptr),
                                                      ctypes.c_void_p(stream_ptr)),
           "lb_reduce_fields_f64_static")


LBNN_WAIT_LIMIT_DEFAULT = 1 << 22


def lbnn_set_wait_limit(limit: int) -> int:
    """Poll limit of the convolutions' handshake waits; returns the previous one."""
    prev = ctypes.c_uint32(0)
    _check(load_library().lbnn_set_wait_limit(int(limit), ctypes.byref(prev)), "lbnn_set_wait_limit")
    return int(prev.value)


def lbnn_check_status(status_ptr: int, stream_ptr: int = 0):
    """Reads and clears a convolution status word; LBError(LB_ETIMEOUT) after a give-up."""
    _check(load_library().lbnn_check_status(ctypes.c_void_p(status_ptr), ctypes.c_void_p(stream_ptr)),
           "lbnn_check_status")


def lb_launch_count() -> int:
    return int(load_library().lb_launch_count())


def lb_device_bytes(h) -> int:
    return int(load_library().lb_device_bytes(h))


# ---------------------------------------------------------------------------
# convenience object
# ---------------------------------------------------------------------------
class Sim:
    """One lattice on the current CUDA device, memory from PyTorch."""

    def __init__(self, nx, ny, nz, walls=0, use_torch_alloc=True, stream=None, **params):
        import torch
        self.shape = (nz, ny, nx)
        self.N = nx * ny * nz
        self.grid = make_grid(nx, ny, nz, walls)
        self.params = make_params(**params)
        self.storage = self.params.storage
        self._alloc = TorchAllocator(torch.device("cuda", torch.cuda.current_device())) if use_torch_alloc else None
        self.h = lb_create(self.grid, self.params, self._alloc)
        s = stream if stream is not None else torch.cuda.current_stream()
        lb_set_stream(self.h, s.cuda_stream)

    def close(self):
        if getattr(self, "h", None):
            lb_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init_droplets(self, centres, radii, width=0.0):
        lb_init_droplets(self.h, centres, radii, width)

    def init_fields(self, phi, rho=None, u=None, regularised=False):
        lb_init_fields(self.h, phi, rho, u, regularised)

    def step(self, n=1):
        lb_step(self.h, n)

    @property
    def t(self):
        return lb_time(self.h)

    def fields(self, names=FIELD_NAMES, f64=False) -> dict:
        mask = 0
        for n in names:
            mask |= FIELD_BIT[n]
        sel = [n for n in FIELD_NAMES if mask & FIELD_BIT[n]]
        out = np.zeros((len(sel),) + self.shape, dtype=np.float64 if f64 else np.float32)
        lb_fields(self.h, mask, out, False, f64=f64)
        return {n: out[k] for k, n in enumerate(sel)}

    def fields_device(self, mask=ALL_FIELDS):
        import torch
        k = bin(mask).count("1")
        out = torch.empty((k,) + self.shape, dtype=torch.float32, device="cuda")
        lb_fields(self.h, mask, out, True)
        return out

    def populations(self, box=None):
        if box is None:
            box = (0, 0, 0, self.shape[2], self.shape[1], self.shape[0])
        return lb_get_populations(self.h, box)

    def reduce(self):
        return lb_reduce_f64(self.h)

    def laplace(self, cut=0.9):
        return lb_laplace_f64(self.h, cut)

    def droplet_count(self):
        return lb_droplet_count(self.h)

    def check(self):
        lb_check(self.h)

    def save(self, path):
        lb_save(self.h, path)

    def load(self, path):
        lb_load(self.h, path)


# ---------------------------------------------------------------------------
# batches of independent runs
# ---------------------------------------------------------------------------
def lb_batch_create(grids, params, alloc: TorchAllocator | None = None):
    L = load_library()
    n = len(grids)
    ga = (lb_grid * n)(*grids)
    pa = (lb_params * n)(*params)
    b = ctypes.c_void_p()
    _check(L.lb_batch_create(n, ga, pa, ctypes.byref(alloc.struct) if alloc else None, ctypes.byref(b)),
           "lb_batch_create")
    return b


def lb_batch_destroy(b):
    _check(load_library().lb_batch_destroy(b), "lb_batch_destroy")


def lb_batch_run(b, r: int):
    h = load_library().lb_batch_run(b, int(r))
    if not h:
        _check(LB_EINVAL, "lb_batch_run")
    return ctypes.c_void_p(h)


def lb_batch_step(b, nsteps: int):
    _check(load_library().lb_batch_step(b, int(nsteps)), "lb_batch_step")


def lb_batch_step_sequential(b, nsteps: int):
    _check(load_library().lb_batch_step_sequential(b, int(nsteps)), "lb_batch_step_sequential")


def lb_batch_set_tile(b, tile: int, blocks_per_sm: int = 2):
    _check(load_library().lb_batch_set_tile(b, int(tile), int(blocks_per_sm)), "lb_batch_set_tile")


def lb_batch_autotune(b, steps: int = 4, use_cache: bool = True):
    """(tile, blocks_per_sm, ms per step, from_cache)."""
    out = np.zeros(4)
    _check(load_library().lb_batch_autotune(b, int(steps), int(bool(use_cache)), out.ctypes.data), "lb_batch_autotune")
    return int(out[0]), int(out[1]), float(out[2]), bool(out[3])


def lb_batch_check(b):
    _check(load_library().lb_batch_check(b), "lb_batch_check")


def lb_batch_nodes(b) -> int:
    return int(load_library().lb_batch_nodes(b))


def lb_batch_set_stream(b, stream_ptr: int):
    _check(load_library().lb_batch_set_stream(b, ctypes.c_void_p(stream_ptr)), "lb_batch_set_stream")


class Batch:
    """Many independent runs advanced together (memory from PyTorch)."""

    def __init__(self, workloads, storage="twoset_f32", stream=None, use_torch_alloc=True):
        import torch
        self.workloads = list(workloads)
        grids = [make_grid(*w.shape, walls=w.walls) for w in self.workloads]
        params = [make_params(storage=storage, **w.params) for w in self.workloads]
        self._alloc = TorchAllocator(torch.device("cuda", torch.cuda.current_device())) if use_torch_alloc else None
        self.b = lb_batch_create(grids, params, self._alloc)
        s = stream if stream is not None else torch.cuda.current_stream()
        lb_batch_set_stream(self.b, s.cuda_stream)
        self.nodes = lb_batch_nodes(self.b)
        for r, w in enumerate(self.workloads):
            h = lb_batch_run(self.b, r)
            if w.phi is not None:
                lb_init_fields(h, w.phi)
            else:
                lb_init_droplets(h, w.centres, w.radii)

    def run(self, r):
        return lb_batch_run(self.b, r)

    def step(self, n=1):
        lb_batch_step(self.b, n)

    def step_sequential(self, n=1):
        lb_batch_step_sequential(self.b, n)

    def autotune(self, steps=4, use_cache=True):
        return lb_batch_autotune(self.b, steps, use_cache)

    def check(self):
        lb_batch_check(self.b)

    def fields(self, r, names=FIELD_NAMES):
        w = self.workloads[r]
        mask = 0
        for n in names:
            mask |= FIELD_BIT[n]
        sel = [n for n in FIELD_NAMES if mask & FIELD_BIT[n]]
        out = np.zeros((len(sel),) + (w.shape[2], w.shape[1], w.shape[0]), dtype=np.float32)
        lb_fields(self.run(r), mask, out, False)
        return {n: out[k] for k, n in enumerate(sel)}

    def close(self):
        if getattr(self, "b", None):
            lb_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
