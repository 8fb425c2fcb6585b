"""Benchmark of the MDF-LBM fused MRT collide-and-stream step on GB300.

Workload (the 4096^2 periodic 2D case): Taylor-Green vortex (U0 = 0.01) plus
8 seeded divergence-free Fourier modes (seed 2108), D2Q5 x 3 distribution
sets (alpha = 0, 1, 2), FP32 rest-shifted population storage, FP32 collision
arithmetic, nu = 0.01 (s1 = 1/0.53), s2 from the paper's rule.

One benchmark step = one epilogue period: 100 lattice updates, the first of
which also writes the derived fields (P, u, du/dx, div, S, sigma, omega) of
Eq. 2-7, 3-15 .. 3-19 in FP64.  value = lattice updates per second of the
whole job in millions (MLUPS).  The populations (2 x 1.0 GB) are far larger
than the 129 MB L2, so no flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl mdf|reference]

Under torchrun each rank advances its own lattice (replicas; the method
needs no exchange between independent lattices): value = sum over ranks of
node updates / max over ranks of the timed region.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "MLUPS and % HBM roofline vs FP64 oracle error; time-to-steady (warm vs cold)"
N_GRID = 4096  # --grid overrides it (small cases for profiling)
EPI_EVERY = 100
NU = 0.01
S1 = 1.0 / (3 * NU + 0.5)
WORKLOAD = ("2D Taylor-Green + 8 seeded divergence-free modes (seed 2108), periodic "
            "4096x4096, D2Q5 x 3 sets, FP32 rest-shifted storage, FP32 arithmetic, "
            "epilogue every 100 steps")
# the 3D case (--workload tg3d): Taylor-Green vortex, 512^3, D3Q7 x 4 sets,
# U0 = 0.05, Re = 1600 on U0 and k = 2 pi / 512, epilogue every 200 steps
TG3D_U0, TG3D_RE = 0.05, 1600.0
# s2 of the 3D case: the paper's rule 8(2 - s1)/(8 - s1) (Sec. 4.1) gives
# 0.053 at that s1 = 1.960, which leaves D3Q7 linearly unstable at the flow's
# speeds (the run blows up within 400 steps); s2 = 1 is stable and leaves the
# viscosity (set by s1, Eq. 3-13a) unchanged.  The 2D case keeps the rule.
TG3D_S2 = 1.0
S2 = -1.0  # the workload's s2 (negative: the paper's rule); set in main()
KERNEL_SOURCES = ("paper_2108_08591_gb300/csrc/mdf_kernels.cuh",
                  "paper_2108_08591_gb300/csrc/mdf_lattice.cuh")
# sources of the equilibrium-shifted update (its recorded traffic is keyed
# by their hash)
EQ_SOURCES = KERNEL_SOURCES + ("paper_2108_08591_gb300/csrc/mdf_eq.cuh",
                               "paper_2108_08591_gb300/csrc/mdf_pack16.cuh")


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def _config(n_gpus: int, storage: str, d: int = 2, q: int = 0, inplace: bool = False):
    grid = [N_GRID] * d
    q = q or (5 if d == 2 else 7)
    pop_gb = N_GRID ** d * q * (d + 1) * {"f32": 4, "f16": 2, "bf16": 2,
                                          "f16eq": 2, "bf16eq": 2}.get(storage, 8) / 1e9
    return {"workload": WORKLOAD, "grid": grid, "lattice": f"D{d}Q{q}",
            "sets": d + 1, "storage": storage, "steps_per_bench_step": EPI_EVERY,
            "global_batch": n_gpus, "parallelism": f"replicas x{n_gpus}",
            "l2": f"inputs larger than L2 ({1 if inplace else 2} x {pop_gb:.2f} GB populations), no flush"}


def aggregate(local_updates: float, local_ms: float, dist=None, device="cpu"):
    """Whole-job throughput of replicas: every rank's timed region is reduced
    to the maximum (the job takes as long as its slowest rank) and the node
    updates of all ranks are summed.  Returns (MLUPS, max ms, world)."""
    world = 1
    t_max, total = float(local_ms), float(local_updates)
    if dist is not None and dist.is_initialized():
        import torch
        world = dist.get_world_size()
        t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        u = torch.tensor([float(local_updates)], dtype=torch.float64, device=device)
        dist.all_reduce(u, op=dist.ReduceOp.SUM)
        t_max, total = float(t.item()), float(u.item())
    return total / (t_max / 1e3) / 1e6, t_max, world


def _kernel_sha(sources=KERNEL_SOURCES) -> str:
    h = hashlib.sha256()
    for p in sources:
        with open(os.path.join(ROOT, p), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _traffic(kernel_sha: str, leg: str = ""):
    """DRAM bytes per launch of the step kernel (or of a storage leg's
    kernel) from the committed ncu summary, or None when the kernel changed
    since it was captured."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as fh:
            t = json.load(fh)
    except (OSError, ValueError):
        return None
    if leg:
        t = t.get(leg) or {}
    if t.get("kernel_sha") != kernel_sha:
        return None
    return t.get("dram_bytes_per_launch_4096")


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "measured"
    except (OSError, ValueError, KeyError):
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    rows.append((float(parts[1]), float(parts[2]), float(parts[3]), parts[5:9]))
                except ValueError:
                    continue
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i, v in enumerate(r[3]) if v == "Active"})
        loaded = [r for r in rows if r[2] > 200.0] or rows
        return {"sm_mhz": statistics.median(r[0] for r in loaded),
                "sm_max_mhz": max(r[1] for r in rows), "reasons": reasons,
                "samples": len(rows), "power_w_max": max(r[2] for r in rows)}


def cpu_oracle_sample(steps: int = 40, warmup: int = 1, single_thread: bool = True):
    """Time the FP64 CPU oracle, as it stands, on the benchmark workload:
    the full 4096^2 lattice, `steps` timed updates after `warmup` (about 16 s
    of work on 16 host cores)."""
    import oracle
    import synth
    P, u = synth.tg_plus_modes(N_GRID, U0=0.01, seed=2108)
    pb = oracle.Problem(d=2, n=(N_GRID, N_GRID), s1=S1)
    f = oracle.init(pb, P, u)
    del P, u
    oracle.run(pb, f, warmup)
    t0 = time.perf_counter()
    oracle.run(pb, f, steps)
    dt = time.perf_counter() - t0
    out = {"value": N_GRID * N_GRID * steps / dt / 1e6, "unit": "MLUPS",
           "cores": oracle.threads(), "kind": "oracle",
           "sample": f"{steps} FP64 oracle updates of the full {N_GRID}^2 D2Q5x3 lattice "
                     f"after {warmup} warm-up, OpenMP threads = {oracle.threads()}",
           "seconds": dt}
    if single_thread and oracle.threads() > 1:
        # the same oracle on one host thread (a fresh process: OpenMP reads
        # its thread count at start-up), one full-lattice update
        code = ("import json, bench; "
                "print(json.dumps(bench.cpu_oracle_sample(steps=1, warmup=0, single_thread=False)))")
        r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True,
                           env=dict(os.environ, OMP_NUM_THREADS="1"), timeout=600)
        lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
        if r.returncode == 0 and lines:
            one = json.loads(lines[-1])
            out["single_thread"] = {"value": one["value"], "unit": "MLUPS", "cores": one["cores"],
                                    "sample": one["sample"]}
    return out


def run_reference(args):
    rank, world, _ = _dist()
    if rank != 0:
        return 0
    import oracle
    import synth
    oracle.build()
    P, u = synth.tg_plus_modes(N_GRID, U0=0.01, seed=2108)
    pb = oracle.Problem(d=2, n=(N_GRID, N_GRID), s1=S1)
    f = oracle.init(pb, P, u)
    del P, u
    for _ in range(args.warmup):
        oracle.run(pb, f, 1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.run(pb, f, 1)
    dt = time.perf_counter() - t0
    mlups = N_GRID * N_GRID * args.steps / dt / 1e6
    cores = oracle.threads()
    line = {
        "impl": "reference", "metric": METRIC, "value": mlups, "unit": "MLUPS",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": _config(args.gpus, "f64 (oracle)"),
        "cpu_baseline": {"value": mlups, "unit": "MLUPS", "cores": cores, "kind": "oracle",
                         "sample": "each step: one FP64 oracle update of the full 4096^2 "
                                   "D2Q5x3 lattice on the host cores"},
        "e2e": {"value": mlups, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }
    print(json.dumps(line), flush=True)
    return 0


def _cs2(d: int, q: int) -> float:
    """c_s^2 of the lattice (Sec. 2.2), lattice units."""
    return {(2, 5): 1 / 3, (2, 4): 1 / 2, (3, 7): 1 / 4, (3, 6): 1 / 3}[(d, q or (5 if d == 2 else 7))]


def _workload(args):
    """(shape, s1, P, u) of the benchmark workload, FP64 host arrays.  The
    viscosity is the workload's; s1 follows from the lattice's c_s^2."""
    import synth
    if args.workload == "tg2d":
        P, u = synth.tg_plus_modes(N_GRID, U0=0.01, seed=2108)
        return (N_GRID, N_GRID), 1.0 / (NU / _cs2(2, args.q) + 0.5), P, u
    k = 2 * math.pi / N_GRID
    nu = TG3D_U0 / (k * TG3D_RE)
    P, u = synth.taylor_green_3d(N_GRID, U0=TG3D_U0)
    return (N_GRID,) * 3, 1.0 / (nu / _cs2(3, args.q) + 0.5), P, u


def sampled_oracle_error(shape, s1, P, u, storage, steps, samples=8, seed=77, q=0):
    s2 = S2
    """FP64 oracle error of the GPU fields at full size, on sampled nodes.

    After `steps` updates a node depends only on nodes within that many
    links, so the oracle advances a periodic (2 steps + 1)^d window around
    each sampled node; the GPU runs the whole lattice as the benchmark does
    (fused epilogue update first, then plain updates)."""
    import numpy as np
    import oracle
    import synth
    from paper_2108_08591_gb300 import Lattice
    d = len(shape)
    lat = Lattice(shape, s1=s1, s2=s2, storage=storage, q=q)
    lat.init(P, u)
    fl = lat.alloc_fields(("P",))
    lat.step_fields(steps, fl)
    names = ("u", "P", "G", "S", "omega")
    got = {k: v.cpu().numpy() for k, v in lat.fields(names).items()}
    lat.close()
    rng = synth.SplitMix64(seed)
    n = shape[0]
    W = 2 * steps + 1
    ref, num = {k: [] for k in names}, {k: [] for k in names}
    for _ in range(samples):
        c = [rng.randint(0, n - 1) for _ in range(d)]
        offs = np.arange(-steps, steps + 1)
        axes = [(c[b] + offs) % n for b in range(d)]
        if d == 2:
            sel = (axes[1][:, None] * n + axes[0][None, :]).ravel()
            g = c[1] * n + c[0]
        else:
            sel = ((axes[2][:, None, None] * n + axes[1][None, :, None]) * n
                   + axes[0][None, None, :]).ravel()
            g = (c[2] * n + c[1]) * n + c[0]
        pb = oracle.Problem(d=d, n=(W,) * d, s1=s1, s2=None if s2 < 0 else s2, nq=q)
        f = oracle.init(pb, P[sel], u[:, sel])
        oracle.run(pb, f, steps)
        Pr, ur, _ = oracle.macro(pb, f)
        D = oracle.derived(pb, f)
        mid = (W ** d) // 2
        ref["u"].append(ur[:, mid]); num["u"].append(got["u"][:, g])
        ref["P"].append(Pr[mid] - 1.0); num["P"].append(got["P"][g] - 1.0)
        for k in ("G", "S", "omega"):
            ref[k].append(D[k][..., mid]); num[k].append(got[k][..., g])
    err = {k: oracle.rel_l2(np.array(ref[k]), np.array(num[k])) for k in ref}
    err["case"] = (f"{samples} seeded nodes of the full lattice after {steps} updates, "
                   f"FP64 oracle on periodic {W}^{d} windows; P compared as P - 1; "
                   "G = du_a/dx_b (Eq. 3-16), S (Eq. 3-17), omega (Eq. 3-18)")
    return err


def storage_leg(shape, s1, P, u, storage, steps=5, warmup=3, q=0, oracle_check=True):
    """A second storage type on the same workload, outside the main timed
    region: device-timed throughput (fused epilogue update + plain updates per
    bench step, as the main line), the plain update's roofline fraction at
    that storage's algorithmic bytes per node, and its sampled FP64 oracle
    error per field."""
    import numpy as np
    import torch
    from paper_2108_08591_gb300 import Lattice
    N = int(np.prod(shape))
    stream = torch.cuda.current_stream()
    lat = Lattice(shape, s1=s1, s2=S2, storage=storage, stream=stream, q=q)
    lat.init(P, u)
    info = lat.info
    fields = lat.alloc_fields(("P", "u", "G", "div", "S", "sigma", "omega"))
    for _ in range(warmup):
        lat.step_fields(1, fields)
        lat.step(EPI_EVERY - 1)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    plain = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
             for _ in range(steps)]
    e0.record(stream)
    for a, b in plain:
        lat.step_fields(1, fields)
        a.record(stream)
        lat.step(EPI_EVERY - 1)
        b.record(stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    plain_ms = sum(a.elapsed_time(b) for a, b in plain) / (steps * (EPI_EVERY - 1))
    lat.close()
    del fields
    peak, kind = _peaks()
    achieved = info.bytes_per_update * N / (plain_ms / 1e3) / 1e9
    sha = _kernel_sha(EQ_SOURCES) if storage.endswith("eq") else _kernel_sha()
    traffic = _traffic(sha, storage) if (N_GRID == 4096 and len(shape) == 2) else None
    out = {"storage": storage, "value": steps * EPI_EVERY * N / (ms / 1e3) / 1e6, "unit": "MLUPS",
           "steps": steps, "warmup": warmup,
           "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                        "frac": achieved / peak, "traffic": traffic, "kernel_sha": sha,
                        "bytes_per_node": info.bytes_per_update,
                        "avg_launch_ms": plain_ms, "vx": info.vx, "block": info.block,
                        "peak_source": f"{kind} hbm_gbs (MEASURED_PEAKS.json)"}}
    if oracle_check:
        out["fp64_oracle_error"] = sampled_oracle_error(shape, s1, P, u, storage,
                                                        steps=64 if len(shape) == 2 else 16, q=q)
    return out


def tg3d_leg(oracle_check=True):
    """The 512^3 D3Q7 x 4 Taylor-Green workload (FP32 rest-shifted storage,
    s2 = TG3D_S2, epilogue every 200 updates) as a short extra leg of the
    default line: two bench steps after one warm-up step, through
    storage_leg, with its sampled FP64 oracle error after 16 updates."""
    import synth
    global S2, EPI_EVERY
    saved = (S2, EPI_EVERY)
    S2, EPI_EVERY = TG3D_S2, 200
    try:
        n = 512
        nu = TG3D_U0 / (2 * math.pi / n * TG3D_RE)
        P, u = synth.taylor_green_3d(n, U0=TG3D_U0)
        out = storage_leg((n,) * 3, 1.0 / (nu / _cs2(3, 0) + 0.5), P, u, "f32", steps=2, warmup=1,
                          oracle_check=oracle_check)
        out["workload"] = (f"3D Taylor-Green vortex, periodic 512^3, D3Q7 x 4 sets, U0 = {TG3D_U0}, "
                           f"Re = {TG3D_RE:.0f}, s2 = {TG3D_S2:g}, FP32 rest-shifted storage, "
                           "epilogue every 200 steps")
        out["kernel"] = "k_update<D3Q7,float,MODE_STEP,periodic>"
        return out
    finally:
        S2, EPI_EVERY = saved


def run_mdf(args):
    import numpy as np
    import torch

    from paper_2108_08591_gb300 import Lattice, _build

    rank, world, local = _dist()
    if not torch.cuda.is_available():
        raise RuntimeError("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0 or world == 1:
        _build.build()
    if dist is not None:
        dist.barrier()

    shape, s1, P, u = _workload(args)
    d = len(shape)
    N = int(np.prod(shape))
    stream = torch.cuda.current_stream()
    lat = Lattice(shape, s1=s1, s2=S2, storage=args.storage, stream=stream, vx=args.vx or 0,
                  block=args.block or 0, q=args.q, inplace=args.inplace)
    lat.init(P, u)
    info = lat.info
    fields = lat.alloc_fields(("P", "u", "G", "div", "S", "sigma", "omega"))

    def bench_step(ev_a=None, ev_b=None):
        lat.step_fields(1, fields)  # fused epilogue update
        if ev_a is not None:
            ev_a.record(stream)
        lat.step(EPI_EVERY - 1)  # plain updates
        if ev_b is not None:
            ev_b.record(stream)

    for _ in range(args.warmup):
        bench_step()
    torch.cuda.synchronize()

    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sampler = ClockSampler(local)
    with sampler:
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        start.record(stream)
        for k in range(args.steps):
            bench_step(*evs[k])
        stop.record(stream)
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
    elapsed_ms = start.elapsed_time(stop)
    plain_ms = sum(a.elapsed_time(b) for a, b in evs) / (args.steps * (EPI_EVERY - 1))
    clocks = sampler.summary()

    updates_local = args.steps * EPI_EVERY * N
    value, t_max, _ = aggregate(updates_local, elapsed_ms, dist, device="cuda")

    # end to end through the C-ABI's host-buffer path: every step hands the
    # library its inputs (P, u) in pinned host memory (mdf_init with
    # MDF_HOST: the host-to-device copy and the initialisation happen inside
    # the call), runs the step (fused epilogue + plain updates) and reads
    # (P, u) of the final state back into pinned host memory (mdf_fields
    # with MDF_HOST outputs: the kernel, the device-to-host copy and a
    # synchronisation inside the call).  Timed on the host clock.
    e2e_steps = max(2, min(args.steps, 20))
    Pn = torch.from_numpy(P).pin_memory().numpy()
    un = torch.from_numpy(np.ascontiguousarray(u)).pin_memory().numpy()
    outP = torch.empty(N, dtype=torch.float64).pin_memory().numpy()
    outu = torch.empty((d, N), dtype=torch.float64).pin_memory().numpy()
    lat.init(Pn, un)  # first host-path call: sizes the library's staging buffer
    lat.fields_host(("P", "u"), out={"P": outP, "u": outu})
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    t0 = time.perf_counter()
    for k in range(e2e_steps):
        lat.init(Pn, un)
        bench_step()
        lat.fields_host(("P", "u"), out={"P": outP, "u": outu})
    e2e_s = time.perf_counter() - t0
    assert np.isfinite(outP).all() and np.isfinite(outu).all()
    e2e_value, _, _ = aggregate(e2e_steps * EPI_EVERY * N, e2e_s * 1e3, dist, device="cuda")
    lat.close()
    del fields
    torch.cuda.empty_cache()

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0

    peak, peak_kind = _peaks()
    bytes_per_launch = info.bytes_per_update * N
    achieved = bytes_per_launch / (plain_ms / 1e3) / 1e9
    sha = _kernel_sha()
    default_lattice = args.q in (0, 5 if d == 2 else 7) and not args.inplace
    traffic = _traffic(sha) if (args.workload == "tg2d" and N_GRID == 4096
                                and args.storage == "f32" and default_lattice) else None
    oerr = None
    if not args.no_oracle_check:
        oerr = sampled_oracle_error(shape, s1, P, u, args.storage, steps=64 if d == 2 else 16, q=args.q)
    extra = None
    if args.storage == "f32" and default_lattice and not args.no_extra_storage:
        # the 16-bit arm of the same workload: equilibrium-shifted FP16
        # populations with FP32 node moments
        extra = storage_leg(shape, s1, P, u, "f16eq", oracle_check=not args.no_oracle_check)
    leg3d = None
    if (args.workload == "tg2d" and N_GRID == 4096 and args.storage == "f32" and default_lattice
            and not args.no_extra_storage):
        leg3d = tg3d_leg(oracle_check=not args.no_oracle_check)
    cpu = None
    if world == 1 and not args.no_cpu_baseline and args.workload == "tg2d" and default_lattice:
        cpu = cpu_oracle_sample()
    kname = f"D{d}Q{info.q}"
    tname = {"f32": "float", "f16": "__half", "bf16": "__nv_bfloat16", "f16eq": "__half",
             "bf16eq": "__nv_bfloat16"}[args.storage]
    if args.inplace:
        kernel = (f"k_update_aa_vec<{kname},{tname},VX={info.vx},even+odd,periodic>" if info.vx > 1
                  else f"k_update_aa<{kname},{tname},even+odd,MODE_STEP,periodic>")
    elif args.storage.endswith("eq"):
        kernel = f"k_update_eq<{kname},{tname},VX={info.vx},MODE_STEP,periodic>"
    elif info.vx == 4 and args.storage == "f32":
        kernel = f"k_update_vec_f32x4<{kname},MODE_STEP,periodic>"
    elif info.vx > 1 and d == 3 and args.storage in ("f16", "bf16"):
        kernel = f"k_update_vec16p<{kname},{tname},VX={info.vx},periodic>"
    elif info.vx > 1:
        kernel = f"k_update_vec<{kname},{tname},VX={info.vx},MODE_STEP,periodic>"
    else:
        kernel = f"k_update<{kname},{tname},MODE_STEP,periodic>"
    line = {
        "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"f32": "f32", "f16": "f16 storage / f32", "bf16": "bf16 storage / f32",
                  "f16eq": "f16 equilibrium-shifted storage + f32 moments / f32",
                  "bf16eq": "bf16 equilibrium-shifted storage + f32 moments / f32"}[args.storage],
        "data": "synthetic", "config": _config(world, args.storage, d, args.q, args.inplace),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "peak_source": f"{peak_kind} hbm_gbs (MEASURED_PEAKS.json)",
                     "kernel": kernel, "block": info.block,
                     "algorithmic_bytes_per_launch": bytes_per_launch,
                     "avg_launch_ms": plain_ms, "kernel_sha": sha},
        "fp64_oracle_error": oerr,
        "storage_f16eq": extra,
        "workload_tg3d": leg3d,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": "MLUPS", "steps": e2e_steps,
                "h2d_bytes_per_step": int(P.nbytes + u.nbytes),
                "d2h_bytes_per_step": int(outP.nbytes + outu.nbytes),
                "path": "C-ABI host buffers: mdf_init(MDF_HOST) from pinned memory, the step, "
                        "mdf_fields(MDF_HOST) into pinned memory; serial, host clock"},
        "gpu_launches": args.steps * EPI_EVERY,
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def run_cavities(args):
    """Batched lid-driven cavities (64 seeded boxes, sides from {65, 129, 257,
    513}, Re ~ U[100, 3200], lid 0.1, D2Q5 x 3 FP32): plain-step throughput of
    the persistent kernel, then every cavity to its residual tolerance."""
    import collections
    import numpy as np
    import torch
    import synth
    from paper_2108_08591_gb300 import CavityBatch, _build
    _build.build()
    if args.cavity_side:  # a uniform batch (profiling case), Re spread over [400, 1150]
        sides = [args.cavity_side] * args.cavity_count
        Res = [400.0 + 750.0 * k / max(1, args.cavity_count - 1) for k in range(args.cavity_count)]
    else:
        draw = synth.cavity_batch(64, seed=2108)
        sides = [s for s, _ in draw]
        Res = [r for _, r in draw]
    nodes = np.array(sides, dtype=np.int64) ** 2
    stream = torch.cuda.Stream()
    b = CavityBatch(sides, Res, lid_speed=0.1, stream=stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed():
        b.step(args.warmup * 100)
        torch.cuda.synchronize()
        e0.record(stream)
        b.step(args.steps * 100)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / (args.steps * 100)

    sched_default = b.schedule()
    ms_default = timed()
    t0 = time.perf_counter()
    sched = b.autotune(reps=60)  # untimed: chooses the persistent kernel's launch shape
    tune_s = time.perf_counter() - t0
    ms = timed()
    mlups = nodes.sum() / (ms / 1e3) / 1e6
    peak, kind = _peaks()
    b.init()
    t0 = time.perf_counter()
    if args.max_steps > 0:
        steps, status, res = b.run(tol=1e-8, max_steps=args.max_steps, check_every=100)
    else:  # throughput only
        steps, status, res = np.zeros(len(sides), np.int64), np.full(len(sides), 6, np.int32), np.zeros(len(sides))
    run_s = time.perf_counter() - t0
    names = {0: "converged", 4: "diverged", 6: "not_converged"}
    line = {
        "metric": METRIC, "workload": "cavities", "value": mlups, "unit": "MLUPS",
        "ms_per_step": ms, "nodes": int(nodes.sum()), "cavities": len(sides),
        "roofline": {"bound": "hbm", "achieved": mlups * 120 / 1e3, "peak": peak, "unit": "GB/s",
                     "frac": mlups * 120 / 1e3 / peak, "peak_source": f"{kind} hbm_gbs",
                     "kernel": f"k_batch_chunk<D2Q5,{sched['threads']},{sched['sched']}> "
                               "(persistent, cooperative)"},
        "schedule": {"tuned": sched, "default": sched_default, "autotune_s": tune_s,
                     "default_mlups": float(nodes.sum() / (ms_default / 1e3) / 1e6)},
        "to_steady": {"tol": 1e-8, "max_steps": args.max_steps, "seconds": run_s,
                      "aggregate_mlups": float((steps * nodes).sum()) / run_s / 1e6 if run_s > 0 else None,
                      "status": {names[k]: v for k, v in collections.Counter(status.tolist()).items()}},
        "per_cavity": [[int(sides[c]), round(Res[c], 1), int(steps[c]), int(status[c])]
                       for c in np.argsort(sides, kind="stable")],
    }
    print(json.dumps(line), flush=True)
    b.close()
    return 0


def run_conv(args):
    """Throughput of the network's tensor-core convolution kernels: each op
    repeated --steps times inside one CUDA graph (host launch cost excluded),
    inputs L2-resident (the network's working set), CUDA-event timed."""
    import torch
    from paper_2108_08591_gb300 import (_build, conv3x3_bf16, conv3x3_bf16_backward, conv3x3_bf16_wgrad,
                                        set_conv_kernel, set_wgrad_kernel)
    _build.build()
    rows = []
    shapes = [(8, 256, 32, 32), (8, 128, 64, 64), (8, 64, 128, 128), (8, 32, 256, 256),
              (8, 256, 96, 32), (8, 64, 384, 128), (8, 256, 16, 32), (8, 256, 64, 16)]
    # backward = dgrad (the forward kernel on flipped weights) + the default
    # tcgen05 weight gradient; with the halo kernel also + the mma.sync one
    for kern, wgrad in (("tcgen05-halo", "tcgen05"), ("tcgen05-halo", "mma.sync"), ("tcgen05", "tcgen05"),
                        ("mma.sync", "tcgen05")):
        set_conv_kernel(kern)
        set_wgrad_kernel(wgrad)
        for (B, H, Cin, Cout) in shapes:
            g = torch.Generator(device="cuda").manual_seed(1)
            x = torch.randn(B, H, H, Cin, device="cuda", generator=g).to(torch.bfloat16)
            w = (0.05 * torch.randn(Cout, 3, 3, Cin, device="cuda", generator=g)).to(torch.bfloat16)
            dz = torch.randn(B, H, H, Cout, device="cuda", generator=g).to(torch.bfloat16)
            flops = 2.0 * B * H * H * Cout * 9 * Cin
            ops = (("bwd", lambda: conv3x3_bf16_backward(x, w, dz), 2),)
            if kern == "tcgen05-halo":  # the weight gradient alone, once per weight-gradient kernel
                ops = (("wgrad", lambda: conv3x3_bf16_wgrad(x, dz), 1),) + ops
            if wgrad == "tcgen05":
                ops = (("fwd", lambda: conv3x3_bf16(x, w, out_fp32=False), 1),) + ops
            for name, fn, mult in ops:
                for _ in range(max(3, args.warmup)):
                    fn()
                torch.cuda.synchronize()
                graph = torch.cuda.CUDAGraph()
                with torch.cuda.graph(graph):
                    for _ in range(args.steps):
                        fn()
                graph.replay()
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                graph.replay()
                e1.record()
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1) / args.steps
                rows.append({"kernel": kern, "wgrad": wgrad if name != "fwd" else None, "B": B, "H": H,
                             "Cin": Cin, "Cout": Cout, "op": name, "ms": ms, "tflops": mult * flops / ms / 1e9})
                del graph
    set_conv_kernel("tcgen05-halo")
    set_wgrad_kernel("tcgen05")
    print(json.dumps({"workload": "conv", "unit": "TFLOP/s", "timing": "CUDA graph of --steps calls",
                      "rows": rows}), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("mdf", "reference"), default="mdf")
    ap.add_argument("--storage", choices=("f32", "f16", "bf16", "f16eq", "bf16eq"), default="f32")
    ap.add_argument("--vx", type=int, default=None,
                    help="x-nodes per thread of the step kernel (default: the library's choice)")
    ap.add_argument("--block", type=int, default=None, help="threads per block of the step kernel")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-oracle-check", action="store_true")
    ap.add_argument("--no-extra-storage", action="store_true",
                    help="skip the extra legs of the default line (FP16 equilibrium-shifted, 512^3 3D)")
    ap.add_argument("--workload", choices=("tg2d", "tg3d", "cavities", "conv", "warmstart"),
                    default="tg2d",
                    help="tg2d: the 4096^2 D2Q5 x 3 line (default); tg3d: 512^3 D3Q7 x 4; "
                         "cavities: 64 batched cavities; conv: network kernels; warmstart: "
                         "learned warm start vs cold start at 256^2")
    ap.add_argument("--max-steps", type=int, default=2_000_000,
                    help="cavities: step cap of the run to steady state (0 skips it)")
    ap.add_argument("--cavity-side", type=int, default=0,
                    help="cavities workload: a uniform batch of this side instead of the 64 seeded boxes")
    ap.add_argument("--cavity-count", type=int, default=16, help="cavities in the uniform batch")
    ap.add_argument("--q", type=int, default=0, choices=(0, 4, 5, 6, 7),
                    help="directions per set: 0 = D2Q5 / D3Q7 (default); 4 = D2Q4, 6 = D3Q6 "
                         "(no rest direction, rest-shifted storage only)")
    ap.add_argument("--inplace", action="store_true",
                    help="one population buffer, streamed in place by the AA pattern")
    ap.add_argument("--grid", type=int, default=4096,
                    help="lattice side (default 4096; smaller sides are profiling cases)")
    args = ap.parse_args()
    global N_GRID, WORKLOAD, EPI_EVERY, S2
    if args.workload == "tg3d":
        N_GRID, EPI_EVERY, S2 = 512, 200, TG3D_S2
        WORKLOAD = (f"3D Taylor-Green vortex, periodic 512^3, D3Q7 x 4 sets, U0 = {TG3D_U0}, "
                    f"Re = {TG3D_RE:.0f}, s2 = {TG3D_S2:g}, FP32 rest-shifted storage, FP32 "
                    "arithmetic, epilogue every 200 steps")
    if args.grid != 4096:
        WORKLOAD = WORKLOAD.replace(f"{N_GRID}x{N_GRID}", f"{args.grid}x{args.grid}").replace(
            f"{N_GRID}^3", f"{args.grid}^3")
        N_GRID = args.grid
    if args.inplace:
        WORKLOAD += ", in-place AA-pattern stream (one population buffer)"
    if args.q in (4, 6):
        WORKLOAD = WORKLOAD.replace("D2Q5", "D2Q4").replace("D3Q7", "D3Q6") + (
            ", same viscosity (s1 from the lattice's c_s^2)")
    if args.impl == "mdf" and args.storage != "f32":
        name = {"f16": "FP16 rest-shifted", "bf16": "BF16 rest-shifted",
                "f16eq": "FP16 equilibrium-shifted (+FP32 moments)",
                "bf16eq": "BF16 equilibrium-shifted (+FP32 moments)"}[args.storage]
        WORKLOAD = WORKLOAD.replace("FP32 rest-shifted", name).replace("F32 rest-shifted", name)
    if args.warmup < 3 and args.impl == "mdf":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "cavities":
        return run_cavities(args)
    if args.workload == "conv":
        return run_conv(args)
    if args.workload == "warmstart":
        from paper_2108_08591_gb300 import _build, warmstart
        _build.build()
        return warmstart.main([])
    return run_mdf(args)


if __name__ == "__main__":
    sys.exit(main())
