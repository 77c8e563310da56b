"""Seeded synthetic workloads (inputs only: geometry and parameters).

This module holds none of the lattice Boltzmann arithmetic.  It produces the
grids, parameters and initial droplet geometry of the five workloads, and is
the only code shared by the CUDA path's tests/bench and the oracle:

  small_droplet   32^3 periodic, one droplet R=8 at the centre, tau=1, A=0.01,
                  beta=0.7, no near-contact force, 200 steps.
  droplet_pair    64x64x128 periodic, droplets R=10 centred at z=52 and z=76
                  (24 apart), opposite body forces +-1e-5 on the A component,
                  A_h=0.1, h_min=h_max=3, 4000 steps.
  dense_emulsion  256x256x512 channel, walls y=0/255, periodic x,z; seeded
                  non-overlapping droplets with radii U[8,12] packed by random
                  sequential addition, grown into power-diagram cells and
                  eroded by a uniform film of DENSE_FILM = 6 nodes (dispersed
                  fraction below the 0.7 bound; the recipe can instead erode
                  to a target fraction); body force 1e-6 along z, A_h=0.1.
  batch_sweep     64 periodic runs with cubic grids drawn from {48,64,96,128},
                  A~U[0.005,0.02], A_h~U[0.05,0.2], 1..20 droplets with radii
                  U[6, min(12, L/6)] and gaps >= 2, 1000 steps.
  surrogate       dense_emulsion-style trajectories at 128x128x256.

Droplet fields are returned as phi arrays [nz][ny][nx] (float32, +1 inside,
-1 outside) or as (centres, radii) lists.
"""
from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass
class Workload:
    name: str
    shape: tuple            # (nx, ny, nz)
    walls: int              # bit0 x, bit1 y, bit2 z
    params: dict            # model parameters (lb_params names, without storage)
    steps: int
    centres: np.ndarray | None = None
    radii: np.ndarray | None = None
    phi: np.ndarray | None = None   # initial phi [nz][ny][nx] when not given by droplets
    info: dict = dataclasses.field(default_factory=dict)

    @property
    def nodes(self) -> int:
        return int(self.shape[0]) * int(self.shape[1]) * int(self.shape[2])


BASE = dict(tau_a=1.0, tau_b=1.0, A_a=0.01, A_b=0.01, beta=0.7, A_h=0.0, h_min=3.0, h_max=3.0, phi_I=0.9,
            g=(0.0, 0.0, 0.0), g_mode=0)


def small_droplet() -> Workload:
    return Workload("small_droplet_32^3", (32, 32, 32), 0, dict(BASE), 200,
                    centres=np.array([[16.0, 16.0, 16.0]]), radii=np.array([8.0]))


def droplet_pair(nx=64, ny=64, nz=128, R=10.0, sep=24.0, g=1e-5) -> Workload:
    p = dict(BASE, A_h=0.1, h_min=3.0, h_max=3.0, g=(0.0, 0.0, g), g_mode=2)
    zc = nz / 2.0
    c = np.array([[nx / 2.0, ny / 2.0, zc - sep / 2.0], [nx / 2.0, ny / 2.0, zc + sep / 2.0]])
    return Workload(f"droplet_pair_{nx}x{ny}x{nz}", (nx, ny, nz), 0, p, 4000, centres=c, radii=np.array([R, R]))


# ---------------------------------------------------------------------------
# random sequential addition of spheres with a minimum gap
# ---------------------------------------------------------------------------
def rsa_spheres(shape, walls, rng, rmin, rmax, gap=2.0, wall_gap=2.0, max_fail=3000, max_count=None):
    """Centres/radii of non-overlapping spheres (surface gap >= gap, periodic
    minimum image on open axes, >= wall_gap from solid layers)."""
    L = np.asarray(shape, dtype=np.float64)
    wall = [(walls >> a) & 1 for a in range(3)]
    cell = 2.0 * rmax + gap
    ncell = np.maximum(1, np.floor(L / cell).astype(int))
    buckets = {}
    cen, rad = [], []
    fails = 0
    while fails < max_fail and (max_count is None or len(cen) < max_count):
        r = rng.uniform(rmin, rmax)
        c = np.empty(3)
        ok = True
        for a in range(3):
            if wall[a]:
                lo, hi = 1.0 + wall_gap + r - 0.5, L[a] - 2.0 - wall_gap - r + 0.5
                if hi <= lo:
                    ok = False
                    break
                c[a] = rng.uniform(lo, hi)
            else:
                c[a] = rng.uniform(0.0, L[a])
        if not ok:
            fails += 1
            continue
        key = tuple((c // cell).astype(int) % ncell)
        hit = False
        for dx in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dz in (-1, 0, 1):
                    kk = ((key[0] + dx) % ncell[0], (key[1] + dy) % ncell[1], (key[2] + dz) % ncell[2])
                    for j in buckets.get(kk, ()):
                        d = c - cen[j]
                        for a in range(3):
                            if not wall[a]:
                                d[a] -= L[a] * np.round(d[a] / L[a])
                        if np.sqrt((d * d).sum()) < r + rad[j] + gap:
                            hit = True
                            break
                    if hit:
                        break
                if hit:
                    break
            if hit:
                break
        if hit:
            fails += 1
            continue
        fails = 0
        buckets.setdefault(key, []).append(len(cen))
        cen.append(c)
        rad.append(r)
    return np.array(cen).reshape(-1, 3), np.array(rad)


def _cell_candidates(shape, walls, centres, cell):
    """Seeds bucketed on a grid of cells at least `cell` wide (periodic on open
    axes).  Returns (ncell[3], table[ncells, maxc] of seed ids, -1 padded)."""
    L = np.asarray(shape, dtype=np.float64)
    ncell = np.maximum(1, np.floor(L / cell).astype(int))
    width = L / ncell
    cid = np.floor(np.mod(centres, L) / width).astype(int)
    cid = np.minimum(cid, ncell - 1)
    flat = cid[:, 0] + ncell[0] * (cid[:, 1] + ncell[1] * cid[:, 2])
    counts = np.bincount(flat, minlength=int(ncell.prod()))
    maxc = max(1, int(counts.max()))
    table = -np.ones((int(ncell.prod()), maxc), dtype=np.int64)
    fill = np.zeros(int(ncell.prod()), dtype=np.int64)
    for j, c in enumerate(flat):
        table[c, fill[c]] = j
        fill[c] += 1
    return ncell, width, table


def power_cell_margin(shape, walls, centres, radii, rmax, gap=2.0, chunk_z=16, device=None):
    """For every node: the power-diagram cell it belongs to (seeds weighted by
    radius^2) and its distance to the nearest cell face or solid wall plane.
    Candidates are the seeds of the 27 surrounding bucket cells.  Runs with
    numpy, or with torch on `device` (same formulas, float64)."""
    nx, ny, nz = shape
    wall = [(walls >> a) & 1 for a in range(3)]
    ncell, width, table = _cell_candidates(shape, walls, centres, 2.0 * rmax + gap)
    if device is not None:
        import torch
        xp = torch
        T = lambda a: torch.as_tensor(a, device=device)
    else:
        xp = np
        T = lambda a: a
    cen_t, r2_t, tab_t = T(centres.astype(np.float64)), T(radii.astype(np.float64) ** 2), T(table)
    ncell_t = T(ncell.astype(np.int64))
    margin = np.empty((nz, ny, nx), dtype=np.float32)
    owner = np.empty((nz, ny, nx), dtype=np.int32)
    offs = np.array([(a, b, c) for c in (-1, 0, 1) for b in (-1, 0, 1) for a in (-1, 0, 1)], dtype=np.int64)
    offs_t = T(offs)
    shape_t = T(np.array(shape, dtype=np.float64))
    width_t = T(width)
    for z0 in range(0, nz, chunk_z):
        z1 = min(nz, z0 + chunk_z)
        if device is not None:
            zz, yy, xx = torch.meshgrid(torch.arange(z0, z1, device=device, dtype=torch.float64),
                                        torch.arange(ny, device=device, dtype=torch.float64),
                                        torch.arange(nx, device=device, dtype=torch.float64), indexing="ij")
            P = torch.stack([xx.reshape(-1), yy.reshape(-1), zz.reshape(-1)], dim=1)
        else:
            zz, yy, xx = np.meshgrid(np.arange(z0, z1, dtype=np.float64), np.arange(ny, dtype=np.float64),
                                     np.arange(nx, dtype=np.float64), indexing="ij")
            P = np.stack([xx.reshape(-1), yy.reshape(-1), zz.reshape(-1)], axis=1)
        cid = xp.floor(P / width_t).long() if device is not None else np.floor(P / width).astype(np.int64)
        nb = cid[:, None, :] + offs_t[None, :, :]
        nb = (nb % ncell_t) if device is not None else np.mod(nb, ncell)
        flat = nb[..., 0] + ncell_t[0] * (nb[..., 1] + ncell_t[1] * nb[..., 2])
        cand = tab_t[flat].reshape(P.shape[0], -1)           # [n, 27*maxc]
        valid = cand >= 0
        candc = xp.where(valid, cand, xp.zeros_like(cand)) if device is not None else np.where(valid, cand, 0)
        d = P[:, None, :] - cen_t[candc]
        for a in range(3):
            if not wall[a]:
                d[..., a] -= shape_t[a] * xp.round(d[..., a] / shape_t[a])
        powd = (d * d).sum(-1) - r2_t[candc]
        big = 1e30
        powd = xp.where(valid, powd, xp.full_like(powd, big)) if device is not None else np.where(valid, powd, big)
        best = xp.argmin(powd, 1) if device is not None else np.argmin(powd, axis=1)
        rows = xp.arange(P.shape[0], device=device) if device is not None else np.arange(P.shape[0])
        own = candc[rows, best]
        pb = powd[rows, best]
        cd = cen_t[candc] - cen_t[own][:, None, :]
        for a in range(3):
            if not wall[a]:
                cd[..., a] -= shape_t[a] * xp.round(cd[..., a] / shape_t[a])
        sep = xp.sqrt((cd * cd).sum(-1))
        same = (candc == own[:, None]) | (~valid) | (sep == 0)
        sep_safe = xp.where(same, xp.ones_like(sep), sep) if device is not None else np.where(same, 1.0, sep)
        m = (powd - pb[:, None]) / (2.0 * sep_safe)
        m = xp.where(same, xp.full_like(m, big), m) if device is not None else np.where(same, big, m)
        mm = m.min(1).values if device is not None else m.min(axis=1)
        for a in range(3):
            if wall[a]:
                c = P[:, a]
                wd = xp.minimum(c - 0.5, shape[a] - 1.5 - c)
                mm = xp.minimum(mm, wd)
        if device is not None:
            mm = mm.float().cpu().numpy()
            own = own.int().cpu().numpy()
        margin[z0:z1] = mm.reshape(z1 - z0, ny, nx)
        owner[z0:z1] = own.reshape(z1 - z0, ny, nx)
    return owner, margin


def fluid_mask(shape, walls):
    nx, ny, nz = shape
    m = np.ones((nz, ny, nx), dtype=bool)
    if walls & 1:
        m[:, :, 0] = m[:, :, -1] = False
    if walls & 2:
        m[:, 0, :] = m[:, -1, :] = False
    if walls & 4:
        m[0, :, :] = m[-1, :, :] = False
    return m


# Film between neighbouring droplets of the dense emulsion, in lattice units:
# twice h_min, so that the near-contact force (active within h_min of an
# interface) reaches across a film from both sides once the sharp initial
# interfaces have relaxed.  Thinner films close before the force acts: the
# FP64 oracle on a 64^3 box (walls y, 10 seeds) merges every droplet within
# 200 steps with 3.2-node films, with or without near contact; with 6-node
# films near contact keeps all 10 apart over 2000 steps and without it they
# merge by step 600.
DENSE_FILM = 6.0


def dense_emulsion_phi(shape, walls, seed, phi_d=0.7, rmin=8.0, rmax=12.0, device=None, film=None):
    """Power-cell emulsion: RSA seeds grown into power-diagram cells, eroded by
    a uniform film: of the given thickness, or (film None) so that the
    dispersed fraction of fluid nodes is phi_d.
    device: optional torch device for the per-node geometry (same result)."""
    rng = np.random.default_rng(seed)
    cen, rad = rsa_spheres(shape, walls, rng, rmin, rmax, max_fail=400)
    if device is None:
        try:
            import torch  # noqa: F401  (same formulas, several times faster than numpy here)
            device = "cpu"
        except ImportError:
            device = None
    owner, margin = power_cell_margin(shape, walls, cen, rad, rmax, device=device)
    fl = fluid_mask(shape, walls)
    if film is None:
        vals = np.sort(margin[fl].ravel())
        half_film = float(vals[int(round((1.0 - phi_d) * (len(vals) - 1)))])
    else:
        half_film = 0.5 * float(film)
    phi = np.where(fl & (margin >= half_film), 1.0, -1.0).astype(np.float32)
    achieved = float((phi[fl] > 0).mean())
    return phi, dict(droplets=int(len(rad)), film=2.0 * half_film, phi_d=achieved,
                     rsa_fraction=float((4.0 / 3.0 * np.pi * (rad ** 3)).sum() / fl.sum()))


def dense_emulsion(shape=(256, 256, 512), seed=1234, film=DENSE_FILM, device=None) -> Workload:
    p = dict(BASE, A_h=0.1, h_min=3.0, h_max=3.0, g=(0.0, 0.0, 1e-6), g_mode=1)
    phi, info = dense_emulsion_phi(shape, 0b010, seed, device=device, film=film)
    return Workload(f"dense_emulsion_{shape[0]}x{shape[1]}x{shape[2]}", tuple(shape), 0b010, p, 20000, phi=phi,
                    info=info)


def batch_sweep(seed=2024, nruns=64, sizes=(48, 64, 96, 128)):
    rng = np.random.default_rng(seed)
    runs = []
    for r in range(nruns):
        L = int(rng.choice(sizes))
        A = float(rng.uniform(0.005, 0.02))
        Ah = float(rng.uniform(0.05, 0.2))
        nd = int(rng.integers(1, 21))
        rmax = min(12.0, L / 6.0)
        cen, rad = rsa_spheres((L, L, L), 0, rng, 6.0, rmax, gap=2.0, max_count=nd, max_fail=500)
        p = dict(BASE, A_a=A, A_b=A, A_h=Ah, h_min=3.0, h_max=3.0)
        runs.append(Workload(f"batch_run{r}_{L}^3", (L, L, L), 0, p, 1000, centres=cen, radii=rad))
    return runs


def surrogate_trajectory_phi(seed, shape=(128, 128, 256), film=DENSE_FILM, device=None):
    return dense_emulsion_phi(shape, 0b010, seed, device=device, film=film)
