#!/usr/bin/env python
"""Benchmark of the colour-gradient LB step on GB300.

Default workload: the confined dense emulsion, 256x256x512 nodes, walls at
y=0/255, 70 % dispersed phase, near-contact force on, FP32 two population
sets.  A "step" is one full LB time step over the whole box: one kernel
that stages phi, runs the near-contact scan, pulls, collides, recolours,
stores and accumulates the next step's component densities; the state
(14.5 GB) is far larger than L2 (129 MB), so no flush is needed between
steps.

Prints one JSON line (rank 0).  With torchrun and N > 1 every rank advances
its own replica (weak scaling, no data-path collective); the time is the max
over ranks.  --impl reference times the FP64 CPU oracle instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "D3Q27 two-fluid MLUPS, % of HBM roofline; surrogate speedup at fixed φ error"
SHAPE = (256, 256, 512)
SEED = 1234


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--storage", default="twoset_f32")
    ap.add_argument("--collision", type=int, default=None,
                    help="0 BGK, 1 regularised (default: 1 for the moment storage, else 0)")
    ap.add_argument("--no-extra", action="store_true", help="skip the other storage formats")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-sweep measurement")
    ap.add_argument("--no-surrogate", action="store_true", help="skip the surrogate training and controller run")
    ap.add_argument("--shape", default=None, help="nx,ny,nz of a smaller emulsion (profiling captures)")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end measurement")
    ap.add_argument("--no-tune", action="store_true", help="use --tile without autotuning")
    ap.add_argument("--tile", type=int, default=0, help="tile of the step kernel when --no-tune is given")
    ap.add_argument("--long-run", action="store_true",
                    help="error-vs-time table of the FP32 and FP16 storages against the FP64 oracle on the 64^3 "
                         "dense-emulsion analogue (20000 steps; prints one JSON line)")
    ap.add_argument("--long-steps", type=int, default=20000, help="last checkpoint of --long-run")
    ap.add_argument("--full-box", action="store_true",
                    help="the dense emulsion at full size, 200 steps in the FP64 oracle and on the GPU (FP32 two-set, "
                         "FP16-deviation): per-field errors over a fixed 64^3 crop and the whole box (prints one JSON line)")
    ap.add_argument("--conv", nargs="+", default=None, metavar="ARG",
                    help="MODE NX NY NZ CIN COUT [REPS]: time one surrogate convolution call instead "
                         "(MODE fwd, upcat or wgrad; used by the convolution profiles)")
    return ap.parse_args()


class Ranks:
    """The ranks of a torchrun launch (one replica per GPU, no data-path
    collective): a barrier around the timed region and the maximum of the
    ranks' times.  backend None: a single process."""

    def __init__(self, backend=None, device=None):
        import torch
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.dist = None
        self.device = device if device is not None else torch.device("cpu")
        if self.world > 1 and backend is not None:
            import torch.distributed as dist
            kw = {"device_id": device} if backend == "nccl" else {}
            dist.init_process_group(backend, **kw)
            self.dist = dist

    def barrier(self):
        if self.dist is not None:
            self.dist.barrier()

    def maxall(self, v):
        if self.dist is None:
            return v
        import torch
        t = torch.tensor([v], dtype=torch.float64, device=self.device)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.dist is not None:
            self.dist.destroy_process_group()
            self.dist = None


def weak_scaling_value(nodes_per_rank, steps, ms_max, world):
    """Whole-job MLUPS: every rank's node updates over the slowest rank's time."""
    return world * nodes_per_rank * steps / (ms_max / 1e3) / 1e6


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def fp32_alu_peak():
    """FP32 arithmetic roof of this GPU, measured: cuBLAS SGEMM 8192^3 with
    TF32 disabled (FMA pipes only), best of 5 back to back, CUDA events.  The
    FP16-deviation storage moves so few bytes that its fused kernel is judged
    against this roof as well as against the copy bandwidth."""
    import torch
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        n = 8192
        g = torch.Generator(device="cuda").manual_seed(0)
        a = torch.randn(n, n, device="cuda", generator=g)
        b = torch.randn(n, n, device="cuda", generator=g)
        for _ in range(2):
            torch.matmul(a, b)
        best = None
        for _ in range(5):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            torch.matmul(a, b)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            best = ms if best is None else min(best, ms)
        del a, b
        torch.cuda.empty_cache()
        return round(2.0 * n ** 3 / (best / 1e3) / 1e12, 1)
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "100", "-i", str(self.gpu), "-f", self.path],
                                         stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                self.proc.wait(5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            with open(self.path) as fh:
                for ln in fh:
                    parts = [p.strip() for p in ln.split(",")]
                    if len(parts) >= 9:
                        rows.append(parts)
        except OSError:
            pass
        finally:
            if self.path and os.path.exists(self.path):
                os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for r in rows:
            for k, n in enumerate(names):
                if r[5 + k].lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows),
                "power_w_max": max((float(r[3]) for r in rows if r[3].replace(".", "").isdigit()), default=None)}


# DRAM bytes per node of one step launch, read from an ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum of k_step on the dense emulsion
# 128x128x256 with the given tile, divided by its nodes; the kernel's traffic
# grows with the node count) together with a digest of the kernel sources it
# was taken on: a changed kernel reports null until it is captured again.
K_STEP_TRAFFIC = {  # storage -> (bytes per node, source digest, tile)
    "twoset_f32": (451.8, "437add262738ef64", 5),  # mean of 2 launches: 1892.1 / 1897.8 MB per 4194304 nodes
}


def kernel_digest():
    """Digest of the step kernel's sources with comments and blank lines
    removed (a comment edit does not invalidate a capture; any code edit
    does)."""
    import hashlib
    import re
    h = hashlib.sha256()
    base = os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_2405_14551_gb300", "csrc")
    for f in ("step_impl.cuh", "lattice.cuh", "step_launch.cuh"):
        with open(os.path.join(base, f), encoding="utf-8") as fh:
            src = re.sub(r"/\*.*?\*/", "", fh.read(), flags=re.S)
        lines = [re.sub(r"//.*$", "", ln).rstrip() for ln in src.splitlines()]
        h.update("\n".join(ln for ln in lines if ln).encode())
    return h.hexdigest()[:16]


def cpu_sample_phi(phi, max_nodes):
    """A crop of the workload's initial phi with the full wall-to-wall extent."""
    nz, ny, nx = phi.shape
    nzc = max(8, min(nz, max_nodes // (ny * nx)))
    return phi[:nzc].copy(), f"crop x 0..{nx - 1}, y 0..{ny - 1} (walls), z 0..{nzc - 1} (periodic in the crop)"


def oracle_rate(phi_crop, params, steps, warmup=1):
    """FP64 oracle MLUPS on a crop (time of `steps` steps after `warmup`)."""
    import numpy as np
    import oracle
    nz, ny, nx = phi_crop.shape
    p = dict(params)
    o = oracle.OracleSim(oracle.make_params(nx, ny, nz, walls=0b010, **p))
    o.init_fields(phi_crop.astype(np.float64))
    o.step(warmup)
    t = time.perf_counter()
    o.step(steps)
    dt = time.perf_counter() - t
    o.close()
    return nx * ny * nz * steps / dt / 1e6, dt


def reference_arm(args, wl_params, phi):
    cores = os.cpu_count() or 1
    os.environ.setdefault("OMP_NUM_THREADS", str(cores))
    import numpy as np
    # size the crop so that warmup + steps take about 90 s of CPU time
    probe, _ = cpu_sample_phi(phi, 256 * 256 * 8)
    rate, _ = oracle_rate(probe, wl_params, 1, 0)
    budget_nodes = int(90.0 * rate * 1e6 / max(1, args.steps + args.warmup))
    crop, desc = cpu_sample_phi(phi, max(256 * 256 * 8, budget_nodes))
    nodes = crop.size
    import oracle
    nz, ny, nx = crop.shape
    o = oracle.OracleSim(oracle.make_params(nx, ny, nz, walls=0b010, **wl_params))
    o.init_fields(crop.astype(np.float64))
    o.step(args.warmup)
    t = time.perf_counter()
    o.step(args.steps)
    dt = time.perf_counter() - t
    val = nodes * args.steps / dt / 1e6
    line = {
        "impl": "reference", "metric": METRIC, "value": round(val, 3), "unit": "MLUPS", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * dt / args.steps, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"dense_emulsion_{SHAPE[0]}x{SHAPE[1]}x{SHAPE[2]}", "seed": SEED,
                   "sample": desc, "nodes_per_step": int(nodes)},
        "cpu_baseline": {"value": round(val, 3), "unit": "MLUPS", "cores": int(os.environ["OMP_NUM_THREADS"]),
                         "kind": "oracle", "sample": desc},
        "e2e": {"value": round(val, 3), "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def end_to_end(args, L, sim, wl, nodes, world, barrier, maxall):
    """Same metric through the public API with pinned host buffers: upload the
    initial phi, K steps, download phi, rho and u."""
    import torch
    host_phi = torch.from_numpy(wl.phi).pin_memory()
    host_out = torch.empty((5,) + wl.phi.shape, dtype=torch.float32).pin_memory()
    mask = L.FIELD_BIT["phi"] | L.FIELD_BIT["rho"] | L.FIELD_BIT["ux"] | L.FIELD_BIT["uy"] | L.FIELD_BIT["uz"]
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    L.lb_init_fields(sim.h, host_phi.numpy())
    sim.step(args.steps)
    L.lb_fields(sim.h, mask, host_out.numpy(), False)
    t1 = time.perf_counter()
    e2e_s = maxall(t1 - t0)
    return {"value": round(world * nodes * args.steps / e2e_s / 1e6, 1), "unit": "MLUPS",
            "h2d_bytes_per_step": int(host_phi.numel() * 4 // args.steps),
            "d2h_bytes_per_step": int(host_out.numel() * 4 // args.steps),
            "region": "lb_init_fields(host phi) + lb_step(K) + lb_fields(phi,rho,u -> host)"}


def other_storages(args, L, make, stream, tile, world, nodes, maxall, peak):
    """The reduced FP32 and FP16-deviation formats on the same workload, the
    regularised collision in the bench's own storage, and the moment storage
    of the regularised collision (ten coefficients + colour scalars per node)."""
    import torch
    extra = {}
    for other, coll in (("reduced_f32", 0), ("reduced_f16", 0), (args.storage, 1), ("moment_f32", 1)):
        if other == args.storage and coll == 0:
            continue
        if other == "moment_f32" and args.storage == "moment_f32" and coll == 1 and f"{other}_regularised" in extra:
            continue
        s2 = make(other, collision=coll)
        s2.step(3)
        best, t2ms = tile, None
        if not args.no_tune:  # the tile of each storage tuned on its own
            for tl in range(L.NUM_TILES):
                L.lb_set_tile(s2.h, tl)
                s2.step(2)
                km = L.lb_step_timed(s2.h, 4)
                if t2ms is None or km < t2ms:
                    best, t2ms = tl, km
        L.lb_set_tile(s2.h, best)
        s2.step(args.warmup)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        s2.step(args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
        s2.check()
        m2 = maxall(e0.elapsed_time(e1))
        v2 = world * nodes * args.steps / (m2 / 1e3) / 1e6
        sm = L.lb_step_timed(s2.h, 20)
        b2 = L.BYTES_PER_NODE[L.STORAGE[other]]
        extra[other if coll == 0 else f"{other}_regularised"] = {"MLUPS": round(v2, 1), "bytes_per_node": b2, "tile": best,
                        "whole_step_frac": round(b2 * v2 * 1e6 / world / 1e9 / peak, 4),
                        "step_kernel_ms": round(sm, 4),
                        "step_kernel_GBps": round(b2 * nodes / (sm / 1e3) / 1e9, 1)}
        s2.close()
        del s2
        torch.cuda.empty_cache()
    return extra


def shan_chen_extra(args, L, wl, stream, world, nodes, maxall, peak):
    """The Shan-Chen model (Sec. III.C.3; G = 7.5, psi_0 = 1, tau = 1, the
    emulsion's phi and body force) on the same grid in FP32 two-set storage:
    one kernel per step, 432 B per node update like the colour-gradient
    step."""
    import torch
    nx, ny, nz = wl.shape
    p = dict(wl.params, A_h=0.0, A_a=0.0, A_b=0.0, beta=0.0, model=1, G=7.5, psi0=1.0)
    s = L.Sim(nx, ny, nz, walls=wl.walls, stream=stream, storage="twoset_f32", **p)
    s.init_fields(wl.phi)
    s.step(max(3, args.warmup))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    s.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    s.check()
    m = maxall(e0.elapsed_time(e1))
    v = world * nodes * args.steps / (m / 1e3) / 1e6
    km = L.lb_step_timed(s.h, 20)
    s.close()
    del s
    torch.cuda.empty_cache()
    return {"MLUPS": round(v, 1), "bytes_per_node": 432, "whole_step_frac": round(432 * v * 1e6 / world / 1e9 / peak, 4),
            "step_kernel_ms": round(km, 4), "step_kernel_GBps": round(432 * nodes / (km / 1e3) / 1e9, 1),
            "params": {"G": 7.5, "psi0": 1.0, "tau": 1.0}}


def batch_extra(args, L, W, stream):
    """The batched sweep: 64 independent runs (grids 48^3..128^3, seeded
    parameters and droplets) stepped together by the persistent kernels under a
    CUDA graph with the autotuned tile, against the same runs one at a time."""
    import torch
    runs = W.batch_sweep()
    b = L.Batch(runs, stream=stream)
    tile, bps, tune_ms, _ = b.autotune(steps=4, use_cache=False)
    steps = 64
    b.step(16)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    b.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    mb = e0.elapsed_time(e1)
    e0.record(stream)
    b.step_sequential(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_seq = e0.elapsed_time(e1)
    b.check()
    nodes = b.nodes
    b.close()
    del b
    torch.cuda.empty_cache()
    return {"workload": f"batch_sweep_{len(runs)}_runs", "nodes": int(nodes), "steps": steps,
            "tile": int(tile), "ctas_per_sm": int(bps),
            "MLUPS_batched": round(nodes * steps / (mb / 1e3) / 1e6, 1),
            "MLUPS_one_at_a_time": round(nodes * steps / (ms_seq / 1e3) / 1e6, 1),
            "speedup": round(ms_seq / mb, 3)}


def surrogate_extra(L, stream, ntraj=24, iters=4000, cycles=100, spinup=2000):
    """The learned surrogate on the 128x128x256 dense emulsion: trajectories
    from the LB itself (seeded emulsions, 2000 spin-up steps, snapshots 50
    steps apart: the slow, late-time regime of a long run), a training run of
    the BF16 U-Net on the library's tcgen05 kernels, its per-jump phi error on
    held-out pairs against the persistence forecast, and the controller (50 LB
    steps + one jump, plain-LB judge until a jump passes, then every 4th, the
    interval doubling up to every 16th after passes with margin; phi
    tolerance 1e-2) timed against plain LB from the same state over 10000
    steps (100 cycles), with the final phi difference and droplet counts."""
    import time
    import torch
    from paper_2405_14551_gb300 import surrogate as S
    from paper_2405_14551_gb300 import workloads as W
    shape = (128, 128, 256)
    nx, ny, nz = shape
    n = nx * ny * nz
    t0 = time.time()
    with torch.cuda.stream(stream):
        trajs = S.generate_pairs(range(ntraj), shape=shape, spinup=spinup, snaps=8, stream=stream)
        test = S.generate_pairs([1000], shape=shape, spinup=spinup, snaps=8, stream=stream)
        net = S.UNet(base=32, seed=0, stream=stream)
        t1 = time.time()
        S.train(net, trajs, shape, iters=iters, lr=1e-3, stream=stream, log_every=iters)
        torch.cuda.synchronize()
        t_train = time.time() - t1
        x = torch.empty((n, S.CIN), dtype=torch.bfloat16, device="cuda")
        out = torch.empty((5, n), dtype=torch.float32, device="cuda")
        err, pers, err_max = [], [], []
        for f0, f1 in zip(test[0][:-1], test[0][1:]):
            S.pack_input(f0, x, stream)
            y = net.forward(x, (nx, ny, nz, 1))
            S.unpack_output(f0, y, out, stream)
            err.append(float((out[0] - f1[0]).abs().mean()))
            err_max.append(float((out[0] - f1[0]).abs().max()))
            pers.append(float((f0[0] - f1[0]).abs().mean()))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for _ in range(2):
            net.forward(x, (nx, ny, nz, 1))
        e0.record(stream)
        for _ in range(5):
            net.forward(x, (nx, ny, nz, 1))
        e1.record(stream)
        torch.cuda.synchronize()
        fwd_ms = e0.elapsed_time(e1) / 5
        del trajs, test
        p = S.workload_params()
        phi, _ = W.dense_emulsion_phi(shape, 0b010, 1001, device=torch.device("cuda"), film=W.DENSE_FILM)
        a = L.Sim(nx, ny, nz, walls=0b010, stream=stream, **p)
        b = L.Sim(nx, ny, nz, walls=0b010, stream=stream, **p)
        for s_ in (a, b):
            s_.init_fields(phi)
            s_.step(spinup)
        ctl = S.Controller(a, net, shape, stream=stream)
        # one untimed cycle allocates the monitor and judge lattices and
        # captures their graphs; then the plain run restarts from the same state
        ctl.run(1)
        L.lb_copy_state(b.h, a.h)
        b.step(100)
        L.lb_copy_state(b.h, a.h)
        # noise floor: the plain LB against itself from a start one ulp away
        # (the last mantissa bit of one population of one node, through a
        # checkpoint), over the same steps
        c = L.Sim(nx, ny, nz, walls=0b010, stream=stream, **p)
        fd, ck = tempfile.mkstemp(suffix=".lbck")
        os.close(fd)
        try:
            b.save(ck)
            raw = bytearray(open(ck, "rb").read())
            node = n // 2 + nx * (ny // 2)
            off = len(raw) - 2 * 27 * n * 4 + (13 * n + node) * 4  # f^A, rest direction
            raw[off] ^= 1
            open(ck, "wb").write(bytes(raw))
            c.load(ck)
        finally:
            os.remove(ck)
        ctl.reset()
        torch.cuda.synchronize()
        t2 = time.time()
        ctl.run(cycles)
        torch.cuda.synchronize()
        t_ctl = time.time() - t2
        t3 = time.time()
        b.step(cycles * 100)
        torch.cuda.synchronize()
        t_lb = time.time() - t3
        c.step(cycles * 100)
        fa, fb = a.fields_device(1).reshape(-1), b.fields_device(1).reshape(-1)
        final_err = float((fa - fb).abs().mean())
        noise = float((c.fields_device(1).reshape(-1) - fb).abs().mean())
        c.close()
        counts = (a.droplet_count(), b.droplet_count())
        judged = [(c, round(e, 4)) for c, e in ctl.judged]
        acc, rej = ctl.accepted, ctl.rejected
        ctl.close()
        a.close()
        b.close()
    torch.cuda.empty_cache()
    return {"workload": "dense_emulsion_128x128x256 surrogate, K = 50", "spinup_steps": spinup,
            "train_trajectories": ntraj, "train_pairs": ntraj * 7, "train_iters": iters, "train_s": round(t_train, 1),
            "unet_forward_ms": round(fwd_ms, 2), "lb_50_steps_ms": round(t_lb / (cycles * 2) * 1e3, 2),
            "phi_err_per_jump": round(sum(err) / len(err), 4), "phi_err_per_jump_max": round(max(err_max), 4),
            "persistence_err": round(sum(pers) / len(pers), 4),
            "phi_tol": 1e-2, "controller_cycles": cycles, "accepted": acc, "rejected": rej, "judged": judged,
            "speedup_vs_plain_lb": round(t_lb / t_ctl, 3), "final_phi_err_vs_plain": round(final_err, 5),
            "noise_floor_plain_vs_plain_one_ulp": round(noise, 5),
            "droplet_count_ctrl_plain": list(counts), "total_s": round(time.time() - t0, 1)}


def cpu_baseline(wl):
    cores = os.cpu_count() or 1
    os.environ.setdefault("OMP_NUM_THREADS", str(cores))
    crop, desc = cpu_sample_phi(wl.phi, 256 * 256 * 64)
    rate, dt = oracle_rate(crop, wl.params, 4)
    return {"value": round(rate, 3), "unit": "MLUPS", "cores": int(os.environ["OMP_NUM_THREADS"]),
            "kind": "oracle", "sample": f"{desc}, 4 FP64 steps after 1 warm-up ({dt:.1f} s)"}


def conv_call(argv):
    """Time one call of a surrogate convolution kernel on random BF16 data.

    MODE fwd (lbnn_conv3d_fwd), upcat (lbnn_conv3d_fwd_upcat with a third of
    CIN at full resolution and the rest at half resolution) or wgrad
    (lbnn_conv3d_wgrad); 3x3x3 taps, x and z periodic, y zero-padded.  Prints
    the CUDA-event time of the last of REPS launches (default 3) and the FLOP
    rate of the implicit GEMM (2 x 27 x CIN x COUT per voxel)."""
    import ctypes
    import torch
    import paper_2405_14551_gb300.lbcg as L
    mode = argv[0]
    nx, ny, nz, cin, cout = (int(v) for v in argv[1:6])
    reps = int(argv[6]) if len(argv) > 6 else 3
    lib = L.load_library()
    dev = torch.device("cuda", 0)
    st = torch.cuda.Stream()
    sp = ctypes.c_void_p(st.cuda_stream)
    status = torch.zeros(4, dtype=torch.int32, device=dev)

    def P(t):
        return ctypes.c_void_p(t.data_ptr())

    nv = nx * ny * nz
    g = torch.Generator(device=dev).manual_seed(0)
    with torch.cuda.stream(st):
        w = (torch.randn(cout, 27, cin, device=dev, generator=g) * 0.05).to(torch.bfloat16)
        b = torch.zeros(cout, device=dev)
        cs = cin // 3 if mode == "upcat" else cin
        x = torch.randn(nv, cs, device=dev, generator=g).to(torch.bfloat16)
        x2 = torch.randn(nv // 8, cin - cs, device=dev, generator=g).to(torch.bfloat16) if mode == "upcat" else None
        y = torch.empty(nv, cout, device=dev, dtype=torch.bfloat16)
        gy = torch.randn(nv, cout, device=dev, generator=g).to(torch.bfloat16) if mode == "wgrad" else None
        dw = torch.zeros(cout, 27, cin, device=dev) if mode == "wgrad" else None
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for i in range(reps):
            if i == reps - 1:
                e0.record(st)
            if mode == "fwd":
                rc = lib.lbnn_conv3d_fwd(P(x), cin, P(w), 27, P(b), P(y), None, cout, 0, nx, ny, nz, 1, 5, 1,
                                         P(status), sp)
            elif mode == "upcat":
                rc = lib.lbnn_conv3d_fwd_upcat(P(x), cs, P(x2), cin - cs, P(w), P(b), P(y), None, cout, 0, nx, ny, nz,
                                               1, 5, 1, P(status), sp)
            elif mode == "wgrad":
                rc = lib.lbnn_conv3d_wgrad(P(gy), cout, P(x), cin, 27, P(dw), nx, ny, nz, 1, 5, 64, P(status), sp)
            else:
                raise SystemExit(f"unknown mode {mode}")
            if rc:
                raise SystemExit(f"{mode}: {lib.lb_last_error().decode()}")
        e1.record(st)
        st.synchronize()
    ms = e0.elapsed_time(e1)
    if int(status.sum().item()):
        raise SystemExit(f"{mode}: a kernel gave up a bounded wait (status {status.tolist()})")
    flop = 2.0 * nv * 27 * cin * cout
    print(f"{mode} {nx}x{ny}x{nz} {cin}->{cout}: {ms * 1e3:.1f} us, {flop / ms / 1e9:.1f} TFLOP/s")


def long_run(args):
    """The dense-emulsion analogue on 64^3 (walls y = 0, 63, seeded power-cell
    droplets eroded by 6-node films, near contact on, body force 1e-6 along
    z) from the same initial phi in the FP64 oracle (host cores) and on the
    GPU in the FP32 two-set, FP32 reduced, FP16-deviation reduced and FP64
    two-set storages.  At steps 1, 10, 100, 1000, 5000, 10000, 20000: max and
    mean |field - oracle| over fluid nodes per field (phi, rho, ux, uy, uz,
    rhoA, rhoB), and the statistics (droplet count, dispersed fraction, mean
    u_z over fluid nodes) of every run.  Pointwise agreement of the FP32
    forms is expected to be lost to the chaotic dynamics; the statistics are
    what the runs should share."""
    import numpy as np
    import torch
    import oracle
    import paper_2405_14551_gb300.lbcg as L
    from paper_2405_14551_gb300 import workloads as W
    cores = os.cpu_count() or 1
    os.environ.setdefault("OMP_NUM_THREADS", str(cores))
    shape, walls, seed = (64, 64, 64), 0b010, 1234
    phi, info = W.dense_emulsion_phi(shape, walls, seed, film=W.DENSE_FILM)
    params = dict(W.BASE, A_h=0.1, h_min=3.0, h_max=3.0, g=(0.0, 0.0, 1e-6), g_mode=1)
    nx, ny, nz = shape
    o = oracle.OracleSim(oracle.make_params(nx, ny, nz, walls=walls, **params))
    o.init_fields(phi.astype(np.float64))
    L.load_library()
    sims = {}
    for st in ("twoset_f32", "reduced_f32", "reduced_f16", "twoset_f64"):
        sims[st] = L.Sim(nx, ny, nz, walls=walls, storage=st, **params)
        sims[st].init_fields(phi)
    fl = W.fluid_mask(shape, walls)
    names = ("phi", "rho", "ux", "uy", "uz", "rhoA", "rhoB")

    def stats(f, count):
        return {"droplets": int(count), "phi_d": round(float((f["phi"][fl] > 0).mean()), 5),
                "mean_uz": float(f["uz"][fl].mean())}

    rows, t, t_orc = [], 0, 0.0
    for cp in [c for c in (1, 10, 100, 1000, 5000, 10000, 20000) if c <= args.long_steps]:
        t0 = time.perf_counter()
        o.step(cp - t)
        t_orc += time.perf_counter() - t0
        for sm in sims.values():
            sm.step(cp - t)
        t = cp
        fo = o.fields()
        row = {"step": cp, "oracle": stats(fo, o.droplet_count())}
        for st, sm in sims.items():
            fg = sm.fields(f64=True)
            err = {}
            for k in names:
                d = np.abs(fg[k][fl] - fo[k][fl])
                err[k] = [float(d.max()), float(d.mean())]
            row[st] = {"max_mean": err, **stats(fg, sm.droplet_count())}
        rows.append(row)
        print(json.dumps({"long_run_checkpoint": cp, "oracle_s": round(t_orc, 1)}), file=sys.stderr, flush=True)
    for sm in sims.values():
        sm.check()
        sm.close()
    o.close()
    print(json.dumps({"long_run": "dense_emulsion_64x64x64 analogue", "seed": seed, "film": W.DENSE_FILM,
                      "droplets0": info["droplets"], "phi_d0": round(info["phi_d"], 5),
                      "oracle_cores": int(os.environ["OMP_NUM_THREADS"]), "oracle_s": round(t_orc, 1),
                      "rows": rows}), flush=True)


def full_box(args):
    """The dense emulsion at its full size (256x256x512, walls y, seed 1234,
    6-node films, near contact on, body force 1e-6 along z) from the same
    initial phi in the FP64 oracle (host cores) and on the GPU in FP32 two-set
    and FP16-deviation storage (the bench's step kernel, tile 5).  At steps 1,
    10, 100 and 200: max and mean |field - oracle| per field over the fluid
    nodes of a fixed 64^3 crop (x 96..159, y 96..159, z 224..287) and of the
    whole box."""
    import numpy as np
    import torch
    import oracle
    import paper_2405_14551_gb300.lbcg as L
    from paper_2405_14551_gb300 import workloads as W
    cores = os.cpu_count() or 1
    os.environ.setdefault("OMP_NUM_THREADS", str(cores))
    wl = W.dense_emulsion((256, 256, 512), seed=SEED, device=torch.device("cuda"))
    nx, ny, nz = wl.shape
    o = oracle.OracleSim(oracle.make_params(nx, ny, nz, walls=wl.walls, **wl.params))
    o.init_fields(wl.phi.astype(np.float64))
    L.load_library()
    sims = {}
    for st in ("twoset_f32", "reduced_f16"):
        sims[st] = L.Sim(nx, ny, nz, walls=wl.walls, storage=st, **wl.params)
        sims[st].init_fields(wl.phi)
        L.lb_set_tile(sims[st].h, 5)
    fl = W.fluid_mask(wl.shape, wl.walls)
    crop = (slice(224, 288), slice(96, 160), slice(96, 160))  # [z][y][x]
    flc = fl[crop]
    names = ("phi", "rho", "ux", "uy", "uz", "rhoA", "rhoB")
    rows, t, t_orc = [], 0, 0.0
    for cp in (1, 10, 100, 200):
        t0 = time.perf_counter()
        o.step(cp - t)
        t_orc += time.perf_counter() - t0
        for sm in sims.values():
            sm.step(cp - t)
        t = cp
        fo = o.fields()
        row = {"step": cp}
        for st, sm in sims.items():
            fg = sm.fields(names, f64=True)
            err = {}
            for k in names:
                dc = np.abs(fg[k][crop][flc] - fo[k][crop][flc])
                db = np.abs(fg[k][fl] - fo[k][fl])
                err[k] = {"crop": [float(dc.max()), float(dc.mean())], "box": [float(db.max()), float(db.mean())]}
            row[st] = err
        rows.append(row)
        print(json.dumps({"full_box_checkpoint": cp, "oracle_s": round(t_orc, 1)}), file=sys.stderr, flush=True)
    for sm in sims.values():
        sm.check()
        sm.close()
    o.close()
    print(json.dumps({"full_box": wl.name, "seed": SEED, "droplets": wl.info.get("droplets"),
                      "crop": "x 96..159, y 96..159, z 224..287", "oracle_cores": int(os.environ["OMP_NUM_THREADS"]),
                      "oracle_s": round(t_orc, 1), "rows": rows}), flush=True)


def main():
    args = parse()
    if args.conv:
        conv_call(args.conv)
        return
    if args.long_run:
        long_run(args)
        return
    if args.full_box:
        full_box(args)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    from paper_2405_14551_gb300 import workloads as W

    if args.impl == "reference":
        if rank != 0:
            return
        dev = None
        try:
            import torch
            if torch.cuda.is_available():
                dev = torch.device("cuda", 0)  # input geometry only; the timed arm is the CPU oracle
        except ImportError:
            pass
        wl_phi, _ = W.dense_emulsion_phi(SHAPE, 0b010, SEED, device=dev, film=W.DENSE_FILM)
        params = dict(W.BASE, A_h=0.1, h_min=3.0, h_max=3.0, g=(0.0, 0.0, 1e-6), g_mode=1)
        reference_arm(args, params, wl_phi)
        return

    import numpy as np
    import torch
    import paper_2405_14551_gb300.lbcg as L

    torch.cuda.set_device(local)
    ranks = Ranks("nccl", torch.device("cuda", local))

    L.load_library()
    dev = torch.device("cuda", local)
    shape = tuple(int(v) for v in args.shape.split(",")) if args.shape else SHAPE
    wl = W.dense_emulsion(shape, seed=SEED, device=dev)
    nodes = wl.nodes
    stream = torch.cuda.Stream()
    storage = args.storage
    stid = L.STORAGE[storage]

    def make(storage_name, collision=0):
        nx, ny, nz = wl.shape
        s = L.Sim(nx, ny, nz, walls=wl.walls, stream=stream, storage=storage_name, collision=collision, **wl.params)
        s.init_fields(wl.phi)
        return s

    barrier, maxall = ranks.barrier, ranks.maxall

    collision = args.collision if args.collision is not None else (1 if storage == "moment_f32" else 0)
    sim = make(storage, collision)
    # autotune the tile of the step kernel: time every shape, keep the fastest
    tile_ms = []
    sim.step(max(3, args.warmup))
    for tile in range(0 if args.no_tune else L.NUM_TILES):
        L.lb_set_tile(sim.h, tile)
        sim.step(12)
        tile_ms.append(L.lb_step_timed(sim.h, 6))
    best_tile = int(np.argmin(tile_ms)) if tile_ms else args.tile
    L.lb_set_tile(sim.h, best_tile)
    sim.step(args.warmup)
    sim.check()

    gpu_index = os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[local if world > 1 else 0]
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches0 = L.lb_launch_count()
    with ClockSampler(gpu_index) as clk:
        barrier()
        torch.cuda.synchronize()
        ev0.record(stream)
        sim.step(args.steps)
        ev1.record(stream)
        torch.cuda.synchronize()
        barrier()
    launches = L.lb_launch_count() - launches0
    ms_max = maxall(ev0.elapsed_time(ev1))
    sim.check()
    value = weak_scaling_value(nodes, args.steps, ms_max, world)
    clocks = clk.summary()

    # live per-kernel timing (CUDA events on the library's stream)
    step_ms = L.lb_step_timed(sim.h, 20)
    peak, peak_kind = peaks()
    bpn = L.BYTES_PER_NODE[stid]
    achieved = bpn * nodes / (step_ms / 1e3) / 1e9
    tr = K_STEP_TRAFFIC.get(storage)
    traffic = round(tr[0] * nodes) if (tr and tr[1] == kernel_digest() and best_tile == tr[2]) else None
    step_frac = bpn * value * 1e6 / world / 1e9 / peak

    e2e = None if args.no_e2e else end_to_end(args, L, sim, wl, nodes, world, barrier, maxall)
    sim.close()
    del sim
    torch.cuda.empty_cache()
    extra = {} if args.no_extra else other_storages(args, L, make, stream, best_tile, world, nodes, maxall, peak)
    if not args.no_extra:
        extra["shan_chen_twoset_f32"] = shan_chen_extra(args, L, wl, stream, world, nodes, maxall, peak)
    if not args.no_extra:
        extra["fp32_alu"] = {"sgemm_tflops": fp32_alu_peak(),
                             "how": "cuBLAS SGEMM 8192^3 with TF32 off, best of 5 (FMA pipes only)"}
    if not args.no_batch and not args.shape:
        extra["batch"] = batch_extra(args, L, W, stream)
    if not args.no_surrogate and not args.shape and world == 1:
        extra["surrogate"] = surrogate_extra(L, stream)
    cpu = cpu_baseline(wl) if (rank == 0 and world == 1 and not args.no_cpu) else None

    if rank == 0:
        line = {
            "metric": METRIC,
            "value": round(value, 1),
            "unit": "MLUPS",
            "n_gpus": world,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": round(ms_max / args.steps, 4),
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f64" if storage == "twoset_f64" else "f32",
            "data": "synthetic",
            "config": {"workload": wl.name, "storage": storage, "collision": "regularised" if collision else "bgk",
                       "walls": "y", "seed": SEED,
                       "dispersed_fraction": round(wl.info.get("phi_d", 0.0), 4), "droplets": wl.info.get("droplets"),
                       "A_h": wl.params["A_h"], "h_min": wl.params["h_min"], "tile": best_tile,
                       "tile_ms": [round(v, 4) for v in tile_ms],
                       "l2": "state far larger than L2, no flush", "parallelism": f"replicas x{world}"},
            "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                         "frac": round(achieved / peak, 4), "traffic": traffic,
                         "kernel": "k_step (the whole step: one launch)",
                         "peak_kind": peak_kind, "kernel_ms": round(step_ms, 4),
                         "bytes_per_node": bpn, "whole_step_frac": round(step_frac, 4)},
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": int(launches),
            "clocks": clocks,
            "extra": extra,
        }
        print(json.dumps(line), flush=True)
    ranks.close()


if __name__ == "__main__":
    main()
