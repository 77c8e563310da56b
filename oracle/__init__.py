"""FP64 CPU oracle for the colour-gradient LB step (test infrastructure only).

The oracle is a plain double-precision C implementation (``cglb_oracle.c``)
of one time step of the two-component colour-gradient lattice Boltzmann
scheme with near-contact repulsion (arXiv 2405.14551, Sec. III.B-III.D), plus
a numpy FP64 reference for the surrogate's convolutions (``unet_ref.py``).
It shares no code with the CUDA library.  Only ``tests/``, the smoke check and
the bench's CPU-baseline / reference arm may import it; the product path never
does.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cglb_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libcglb_oracle.so")
_lock = threading.Lock()
_lib = None

Q = 27
NFIELD = 14
FIELD_NAMES = ("phi", "rho", "ux", "uy", "uz", "rhoA", "rhoB", "Frx", "Fry", "Frz", "h", "gx", "gy", "gz")


class OrcParams(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
        ("walls", ctypes.c_uint32),
        ("tau_a", ctypes.c_double), ("tau_b", ctypes.c_double),
        ("A_a", ctypes.c_double), ("A_b", ctypes.c_double),
        ("beta", ctypes.c_double),
        ("A_h", ctypes.c_double), ("h_min", ctypes.c_double), ("h_max", ctypes.c_double),
        ("phi_I", ctypes.c_double),
        ("g", ctypes.c_double * 3),
        ("g_mode", ctypes.c_int32),
        ("collision", ctypes.c_int32),
        ("model", ctypes.c_int32),
        ("G", ctypes.c_double),
        ("psi0", ctypes.c_double),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C11, OpenMP, no target-specific flags)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c11", "-O2", "-fopenmp", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            dp = ctypes.POINTER(ctypes.c_double)
            L.orc_create.restype = ctypes.c_void_p
            L.orc_create.argtypes = [ctypes.POINTER(OrcParams)]
            L.orc_destroy.argtypes = [ctypes.c_void_p]
            L.orc_init_droplets.argtypes = [ctypes.c_void_p, ctypes.c_int32, dp, dp, ctypes.c_double]
            L.orc_init_fields.argtypes = [ctypes.c_void_p, dp, dp, dp]
            L.orc_set_populations.argtypes = [ctypes.c_void_p, dp, dp]
            L.orc_get_populations.argtypes = [ctypes.c_void_p, dp, dp]
            L.orc_set_time.argtypes = [ctypes.c_void_p, ctypes.c_int64]
            L.orc_time.restype = ctypes.c_int64
            L.orc_time.argtypes = [ctypes.c_void_p]
            L.orc_step.argtypes = [ctypes.c_void_p, ctypes.c_int64]
            L.orc_sc_psi.restype = ctypes.c_double
            L.orc_sc_psi.argtypes = [ctypes.c_double, ctypes.c_double]
            L.orc_node_collide_sc.argtypes = [ctypes.POINTER(OrcParams), dp, dp, dp, dp, dp, dp, dp]
            L.orc_fields.argtypes = [ctypes.c_void_p, dp]
            L.orc_reduce.argtypes = [ctypes.c_void_p, dp]
            L.orc_laplace.restype = ctypes.c_double
            L.orc_laplace.argtypes = [ctypes.c_void_p, ctypes.c_double]
            L.orc_droplet_count.restype = ctypes.c_int32
            L.orc_droplet_count.argtypes = [ctypes.c_void_p]
            L.orc_reconstruct.argtypes = [ctypes.c_void_p, dp, dp, dp]
            L.orc_lattice.argtypes = [ctypes.c_void_p, dp, ctypes.c_void_p, dp]
            L.orc_feq.argtypes = [ctypes.c_double, dp, dp]
            L.orc_omega2.argtypes = [ctypes.c_double, ctypes.c_double, dp, dp]
            L.orc_guo.argtypes = [ctypes.c_double, dp, dp, dp]
            L.orc_tau_bar.restype = ctypes.c_double
            L.orc_tau_bar.argtypes = [ctypes.c_double] * 4
            L.orc_recolour.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double, dp, dp, dp, dp]
            L.orc_node_collide.argtypes = [ctypes.POINTER(OrcParams), dp, dp, dp, dp, dp, dp, dp]
            L.orc_regularise.argtypes = [dp, dp, dp]
            _lib = L
        return _lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def make_params(nx, ny, nz, walls=0, tau_a=1.0, tau_b=1.0, A_a=0.01, A_b=0.01, beta=0.7,
                A_h=0.0, h_min=3.0, h_max=3.0, phi_I=0.9, g=(0.0, 0.0, 0.0), g_mode=0, collision=0,
                model=0, G=0.0, psi0=1.0) -> OrcParams:
    """model 0: colour gradient (A_a, A_b, beta, near contact); model 1:
    Shan-Chen pseudo-potential (G, psi0; Sec. III.C.3)."""
    p = OrcParams()
    p.nx, p.ny, p.nz, p.walls = int(nx), int(ny), int(nz), int(walls)
    p.tau_a, p.tau_b, p.A_a, p.A_b, p.beta = tau_a, tau_b, A_a, A_b, beta
    p.A_h, p.h_min, p.h_max, p.phi_I = A_h, h_min, h_max, phi_I
    p.g[0], p.g[1], p.g[2] = g
    p.g_mode = int(g_mode)
    p.collision = int(collision)
    p.model, p.G, p.psi0 = int(model), float(G), float(psi0)
    return p


# ---------------------------------------------------------------------------
# per-node building blocks
# ---------------------------------------------------------------------------
def lattice():
    """(c[27,3] int, w[27], opp[27], B[27]) in the oracle's own order."""
    c = np.zeros((Q, 3), dtype=np.int32)
    w = np.zeros(Q)
    opp = np.zeros(Q, dtype=np.int32)
    B = np.zeros(Q)
    lib().orc_lattice(c.ctypes.data, _dp(w), opp.ctypes.data, _dp(B))
    return c, w, opp, B


def feq(rho, u):
    out = np.zeros(Q)
    lib().orc_feq(float(rho), _dp(np.ascontiguousarray(u, dtype=np.float64)), _dp(out))
    return out


def omega2(A_a, A_b, grad):
    out = np.zeros(Q)
    lib().orc_omega2(float(A_a), float(A_b), _dp(np.ascontiguousarray(grad, dtype=np.float64)), _dp(out))
    return out


def guo(tau, u, F):
    out = np.zeros(Q)
    lib().orc_guo(float(tau), _dp(np.ascontiguousarray(u, dtype=np.float64)),
                  _dp(np.ascontiguousarray(F, dtype=np.float64)), _dp(out))
    return out


def tau_bar(tau_a, tau_b, rhoA, rhoB):
    return lib().orc_tau_bar(float(tau_a), float(tau_b), float(rhoA), float(rhoB))


def recolour(beta, rhoA, rhoB, fstar, grad):
    oa, ob = np.zeros(Q), np.zeros(Q)
    lib().orc_recolour(float(beta), float(rhoA), float(rhoB),
                       _dp(np.ascontiguousarray(fstar, dtype=np.float64)),
                       _dp(np.ascontiguousarray(grad, dtype=np.float64)), _dp(oa), _dp(ob))
    return oa, ob


def regularise(f, feq):
    """Non-equilibrium part of f projected on Hermite orders 1 and 2."""
    out = np.zeros(Q)
    lib().orc_regularise(_dp(np.ascontiguousarray(f, dtype=np.float64)),
                         _dp(np.ascontiguousarray(feq, dtype=np.float64)), _dp(out))
    return out


def node_collide(params: OrcParams, fA, fB, grad, F):
    oa, ob, u = np.zeros(Q), np.zeros(Q), np.zeros(3)
    lib().orc_node_collide(ctypes.byref(params),
                           _dp(np.ascontiguousarray(fA, dtype=np.float64)),
                           _dp(np.ascontiguousarray(fB, dtype=np.float64)),
                           _dp(np.ascontiguousarray(grad, dtype=np.float64)),
                           _dp(np.ascontiguousarray(F, dtype=np.float64)), _dp(oa), _dp(ob), _dp(u))
    return oa, ob, u


def sc_psi(rho, psi0=1.0):
    """Shan-Chen pseudo-potential psi(rho) = rho_0 (1 - exp(-rho/rho_0))."""
    return float(lib().orc_sc_psi(float(rho), float(psi0)))


def node_collide_sc(params: OrcParams, fA, fB, FA, FB):
    """One node's Shan-Chen collision (forces include the body forces)."""
    oa, ob, u = np.zeros(Q), np.zeros(Q), np.zeros(3)
    lib().orc_node_collide_sc(ctypes.byref(params),
                              _dp(np.ascontiguousarray(fA, dtype=np.float64)),
                              _dp(np.ascontiguousarray(fB, dtype=np.float64)),
                              _dp(np.ascontiguousarray(FA, dtype=np.float64)),
                              _dp(np.ascontiguousarray(FB, dtype=np.float64)), _dp(oa), _dp(ob), _dp(u))
    return oa, ob, u


# ---------------------------------------------------------------------------
# whole-lattice simulation
# ---------------------------------------------------------------------------
class OracleSim:
    """FP64 two-set colour-gradient LB on an nx*ny*nz box (x fastest)."""

    def __init__(self, params: OrcParams):
        self.p = params
        self.shape = (params.nz, params.ny, params.nx)
        self.N = params.nx * params.ny * params.nz
        self._h = lib().orc_create(ctypes.byref(params))
        if not self._h:
            raise ValueError("oracle rejected the parameters")

    def close(self):
        if self._h:
            lib().orc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def t(self) -> int:
        return lib().orc_time(self._h)

    def init_droplets(self, centres, radii, width=0.0):
        c = np.ascontiguousarray(np.asarray(centres, dtype=np.float64).reshape(-1, 3))
        r = np.ascontiguousarray(np.asarray(radii, dtype=np.float64).reshape(-1))
        assert c.shape[0] == r.shape[0]
        lib().orc_init_droplets(self._h, int(r.shape[0]), _dp(c), _dp(r), float(width))

    def init_fields(self, phi, rho=None, u=None):
        phi = np.ascontiguousarray(phi, dtype=np.float64).reshape(-1)
        rho_p = _dp(np.ascontiguousarray(rho, dtype=np.float64).reshape(-1)) if rho is not None else None
        keep = []
        if u is not None:
            uu = np.ascontiguousarray(u, dtype=np.float64).reshape(3, -1)
            keep.append(uu)
            u_p = _dp(uu)
        else:
            u_p = None
        lib().orc_init_fields(self._h, _dp(phi), rho_p, u_p)

    def set_populations(self, fA, fB):
        """fA, fB: [27 canonical dirs][N], canonical dir = (cx+1)+3(cy+1)+9(cz+1)."""
        a = np.ascontiguousarray(fA, dtype=np.float64).reshape(Q, -1)
        b = np.ascontiguousarray(fB, dtype=np.float64).reshape(Q, -1)
        lib().orc_set_populations(self._h, _dp(a), _dp(b))

    def get_populations(self):
        a = np.zeros((Q, self.N))
        b = np.zeros((Q, self.N))
        lib().orc_get_populations(self._h, _dp(a), _dp(b))
        return a, b

    def set_time(self, t):
        lib().orc_set_time(self._h, int(t))

    def step(self, n=1):
        lib().orc_step(self._h, int(n))

    def fields(self) -> dict:
        out = np.zeros((NFIELD, self.N))
        lib().orc_fields(self._h, _dp(out))
        return {k: out[i].reshape(self.shape) for i, k in enumerate(FIELD_NAMES)}

    def reduce(self) -> np.ndarray:
        out = np.zeros(8)
        lib().orc_reduce(self._h, _dp(out))
        return out

    def laplace(self, cut=0.9) -> float:
        return lib().orc_laplace(self._h, float(cut))

    def droplet_count(self) -> int:
        return int(lib().orc_droplet_count(self._h))

    def reconstruct(self, phi, rho, u):
        phi = np.ascontiguousarray(phi, dtype=np.float64).reshape(-1)
        rho = np.ascontiguousarray(rho, dtype=np.float64).reshape(-1)
        u = np.ascontiguousarray(u, dtype=np.float64).reshape(3, -1)
        lib().orc_reconstruct(self._h, _dp(phi), _dp(rho), _dp(u))
