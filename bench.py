#!/usr/bin/env python3
"""Throughput benchmark of the fused D3Q27 central-moment LBM step on GB300.

Default workload: the decaying Taylor-Green vortex at 512^3 (periodic, U0 = 0.05, nu = 1e-4, FP32
storage: 134 M nodes, a 14.5 GB population store), the largest configuration that fits one GPU.
One step is one launch of the fused stream-collide kernel; MLUPS = nodes * steps / s.
--workload droplet128 is the forced path: the Shan-Chen static droplet at 128^3 (psi = 1 - exp(-rho),
G = -5.5, R = 24, rho_l = 2.4, rho_g = 0.13, tanh width 2, nu = 1/6), one step = the psi pass plus
the fused stream-collide kernel with the 26-neighbour force stencil.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload ...]

Under torchrun each rank runs its own independent replica (weak scaling, no data-path collective);
the time is the max over ranks and value is the sum of all ranks' node updates per second.
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
sys.path.insert(0, ROOT)

METRIC = "D3Q27 CM-LBM MLUPS & HBM roofline fraction; time-to-steady warm vs plain"
PROFILE_EVERY = 32  # kernel times of the step pairs t = 0, 1 (mod 32) are recorded inside the timed region


def profile_every(steps):
    """Sampling interval of the kernel-time events: every 32nd step pair on long runs, every pair
    on runs too short to contain eight sampled pairs."""
    return PROFILE_EVERY if steps >= 8 * PROFILE_EVERY else 2
BYTES_PER_NODE = {"fp32": 216, "fp16": 108, "bf16": 108}  # AA in place: 27 reads + 27 writes

WORKLOADS = {
    "droplet128": dict(n=128, kind="droplet", nu=1.0 / 6.0, G=-5.5, radius=24, rho_l=2.4, rho_g=0.13, width=2.0,
                       text="Shan-Chen static droplet 128^3 periodic, psi=1-exp(-rho), G=-5.5, R=24, "
                            "rho_l=2.4, rho_g=0.13, tanh width 2, nu=1/6"),
    "tgv512": dict(n=512, kind="tgv", nu=1e-4, u0=0.05,
                   text="decaying Taylor-Green vortex 512^3 periodic, U0=0.05, nu=1e-4"),
    "porous512": dict(n=0, kind="porous", count=512,
                      text="512 forced porous channels (nx,nz~U{32..96}, ny~U{32..48}, walls in y, sphere packs "
                           "of solid fraction U[0,0.2], nu~U[0.01,0.1], F_x~U[1e-6,1e-5]) in one batch"),
    "kolmogorov256": dict(n=256, kind="kolmogorov", nu=0.05, F0=1e-5,
                          text="Kolmogorov flow 256^3 periodic, nu=0.05, F_x=1e-5 sin(2 pi y/256)"),
    "orszag_tang128": dict(n=128, kind="mhd", nu=0.005, eta=0.005, u0=0.0203, b0=0.0203,
                           text="3D Orszag-Tang vortex 128^3 periodic (magnetic field on D3Q7, Lorentz force "
                                "j x b), u0=b0=0.0203, nu=eta=0.005"),
    "rayleigh_taylor64": dict(n=64, kind="cg", nu=0.005, rho_h=3.0, rho_l=1.0, A=1e-4, beta=0.7,
                              text="Rayleigh-Taylor instability, colour-gradient two-phase model, 64x256x64 "
                                   "(W=64, walls in y), At=0.5, Re=512, sqrt(gW)=0.04"),
}
# two-phase step, algorithmic bytes: both colours read and written once (432 + 432 B) and the
# phase fields written and read back (8 + 8 B).  The field pass reads the colours a second time
# (432 B), a cost of this two-pass design that is not counted.
CG_BYTES_PER_NODE = 880


def grid_shape(wl):
    n = wl["n"]
    return (n, 4 * n, n) if wl["kind"] == "cg" else (n, n, n)


def cg_params(wl):
    g = 0.04 ** 2 / wl["n"]
    return dict(rho_r0=wl["rho_h"], rho_b0=wl["rho_l"], nu_r=wl["nu"], nu_b=wl["nu"], A=wl["A"], beta=wl["beta"],
                g=(0.0, -g, 0.0))
# bytes per node of one step, AA in place: 27 populations read + written (+ 21 magnetic ones)
MHD_BYTES_PER_NODE = 216 + 168


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="tgv512")
    ap.add_argument("--storage", choices=["fp32", "fp16", "bf16"], default="fp32")
    ap.add_argument("--n", type=int, default=None, help="override the cube edge (profiling of smaller cases)")
    ap.add_argument("--count", type=int, default=None, help="override the number of batched domains")
    ap.add_argument("--shape", default=None,
                    help="batched launch shape tile,blocks_per_sm,schedule (e.g. 128,16,strided) instead of autotuning")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--budget-s", type=float, default=60.0,
                    help="reference arm: wall-time budget of warm-up plus timed oracle steps")
    return ap.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# --------------------------------------------------------------------------- inputs
def initial_fields(wl):
    import numpy as np

    from paper_1905_10182_gb300 import inputs
    n = wl["n"]
    if wl["kind"] == "droplet":
        rho = inputs.droplet_density(n, wl["radius"], wl["rho_l"], wl["rho_g"], wl["width"])
        z = np.zeros_like(rho)
        return rho, z, z, z
    if wl["kind"] == "tgv":
        return inputs.taylor_green(n, wl["u0"])
    if wl["kind"] == "mhd":
        u, _ = inputs.orszag_tang(n, wl["u0"], wl["b0"])
        return np.ones((n, n, n), dtype=np.float32), u[0], u[1], u[2]
    one = np.ones((n, n, n), dtype=np.float32)
    z = np.zeros_like(one)
    return one, z, z, z


def configure_force(s, wl):
    if wl["kind"] == "droplet":
        s.set_force("shan_chen", (wl["G"],))
    elif wl["kind"] == "kolmogorov":
        s.set_force("kolmogorov", (wl["F0"],))


def initial_magnetic(wl):
    from paper_1905_10182_gb300 import inputs
    return inputs.orszag_tang(wl["n"], wl["u0"], wl["b0"])[1]


def oracle_grid(wl, m, threads):
    """Oracle grid, initial state and step function for an m^3 sample of the workload."""
    import numpy as np

    import oracle
    sub = dict(wl, n=m)
    if wl["kind"] == "droplet":
        sub["radius"] = max(3.0, wl["radius"] * m / wl["n"])
    rho, ux, uy, uz = initial_fields(sub)
    u = np.stack([ux, uy, uz]).astype(np.float64)
    kw = dict(nu=wl["nu"], collision=oracle.COLL_PAPER, threads=threads)
    if wl["kind"] == "droplet":
        kw.update(force_kind=oracle.FORCE_SHAN_CHEN, G=wl["G"])
    elif wl["kind"] == "kolmogorov":
        kw.update(force_kind=oracle.FORCE_KOLMOGOROV, force=(wl["F0"], 0, 0))
    if wl["kind"] == "cg":
        from paper_1905_10182_gb300 import rayleigh_taylor
        rr, rb = rayleigh_taylor.initial_densities(m, wl["rho_h"], wl["rho_l"])
        prm = cg_params(sub)
        cg = oracle.CgGrid(m, 4 * m, m, rho_r0=prm["rho_r0"], rho_b0=prm["rho_b0"], nu_r=prm["nu_r"],
                           nu_b=prm["nu_b"], A=prm["A"], beta=prm["beta"], gvec=prm["g"], walls_y=True,
                           threads=threads)
        state = list(cg.cg_init(rr.astype(np.float64), rb.astype(np.float64)))

        def step(k):
            state[0], state[1] = cg.cg_step(state[0], state[1], k)
        return step
    if wl["kind"] == "mhd":
        g = oracle.MhdGrid(m, m, m, eta=wl["eta"], **kw)
        f = g.init_equilibrium(rho.astype(np.float64), u)
        h = g.mhd_init(initial_magnetic(sub).astype(np.float64), u)
        state = [f, h]

        def step(k):
            state[0], state[1] = g.mhd_step(state[0], state[1], k)
        return step
    g = oracle.Grid(m, m, m, **kw)
    state = [g.init_equilibrium(rho.astype(np.float64), u)]

    def step(k):
        state[0] = g.step(state[0], k)
    return step


# --------------------------------------------------------------------------- clocks
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(v):
            try:
                return float(v)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1])]
        smax = [num(r[2]) for r in rows if num(r[2])]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows),
                "power_w_max": max((num(r[3]) or 0.0) for r in rows)}


# --------------------------------------------------------------------------- oracle timing
def oracle_mlups(wl, target_s=12.0, threads=None):
    """The FP64 oracle (five-step algorithm of Sec. II) timed on the host cores on a bounded sample:
    the same initial state, as many steps as fit in about target_s seconds (at least one)."""
    import numpy as np

    import oracle
    threads = threads or os.cpu_count() or 1
    n = wl["n"]
    # a 512^3 FP64 oracle state (29 GB x 2) does not fit a bounded sample: use a 128^3 box
    sample_n = min(n, 128)
    if wl["kind"] == "cg":
        sample_n = min(n, 16)
    step = oracle_grid(wl, sample_n, threads)
    t0 = time.perf_counter()
    step(1)
    t1 = time.perf_counter() - t0
    steps = max(1, min(200, int(target_s / max(t1, 1e-6))))
    t0 = time.perf_counter()
    step(steps)
    dt = time.perf_counter() - t0
    shape = grid_shape(dict(wl, n=sample_n))
    nodes = shape[0] * shape[1] * shape[2]
    return {"value": nodes * steps / dt / 1e6, "unit": "MLUPS", "cores": threads, "kind": "oracle",
            "sample": f"{steps} oracle steps (FP64, five-step algorithm of Sec. II) on a "
                      f"{'x'.join(map(str, shape))} {'box of the ' if sample_n != n else ''}{wl['kind']} state, "
                      f"{dt:.1f} s"}


# --------------------------------------------------------------------------- reference arm
def run_reference(args, wl):
    world, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    oracle.build()
    threads = os.cpu_count() or 1
    # each step is a bounded sample: one oracle step on an m^3 box of the workload, m chosen so
    # that warm-up + timed steps take about a minute in total
    per_node = None
    m = 16
    probe = oracle_mlups(dict(wl, n=min(wl["n"], 32)), target_s=1.0, threads=threads)
    per_node = 1.0 / (probe["value"] * 1e6)
    budget = args.budget_s / max(1, args.steps + args.warmup)
    m = int(max(8, min(wl["n"], (budget / per_node) ** (1.0 / 3.0))))
    if wl["kind"] == "cg":
        m = max(8, int(m / 4 ** (1.0 / 3.0)))  # the box is m x 4m x m
    step = oracle_grid(wl, m, threads)
    step(args.warmup)
    t0 = time.perf_counter()
    step(args.steps)
    dt = time.perf_counter() - t0
    shape = grid_shape(dict(wl, n=m))
    val = shape[0] * shape[1] * shape[2] * args.steps / dt / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "MLUPS", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / max(1, args.steps),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl["text"] + f"; oracle sample box {'x'.join(map(str, shape))} per step",
                       "nodes_per_step": shape[0] * shape[1] * shape[2]},
            "cpu_baseline": {"value": val, "unit": "MLUPS", "cores": threads, "kind": "oracle",
                             "sample": f"{args.steps} timed oracle steps on a {'x'.join(map(str, shape))} box of the workload"},
            "e2e": {"value": val, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "gpu_launches": 0}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------- our arm
def kernel_source_hash(batch=False):
    """Hash of the code the single-domain stream-collide kernels (or, batch=True, the batched step)
    are built from (device building blocks, kernel templates and their instantiation units), with
    comments and blank space removed so that an edit of a comment does not void a traffic
    measurement."""
    import re
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1905_10182_gb300", "csrc")
    for name in sorted(os.listdir(csrc)):
        if (batch and name in ("lbm_device.cuh", "lbm_batch.cu")) or (not batch and (
                name in ("lbm_device.cuh", "lbm_kernels.cuh", "lbm_x2.cuh") or
                (name.startswith("lbm_k_") and name.endswith(".cu")))):
            text = open(os.path.join(csrc, name), encoding="utf-8").read()
            text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
            text = re.sub(r"//[^\n]*", " ", text)
            h.update(name.encode() + b"\0" + " ".join(text.split()).encode())
    return h.hexdigest()[:16]


def committed_traffic(workload, storage):
    """Per-launch DRAM bytes of the stream-collide kernel from the committed ncu summary, if it was
    taken on the current kernel sources; otherwise None."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        tab = json.load(open(path))
    except (OSError, ValueError):
        return None
    ent = tab.get(f"{workload}/{storage}")
    if not ent or ent.get("kernel_source_hash") != kernel_source_hash(batch=workload == "porous512"):
        return None
    return ent.get("dram_bytes_per_launch")


def run_batch(args, wl):
    """Batched porous channels: one persistent launch per step over all domains, graph-replayed."""
    import numpy as np
    import torch

    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    from paper_1905_10182_gb300 import BatchSolver, inputs
    from paper_1905_10182_gb300.buildlib import build
    build()
    # each rank takes its own seeds: independent problems, no data-path collective
    seeds = range(rank * wl["count"], (rank + 1) * wl["count"])
    doms = []
    for sd in seeds:
        c = inputs.porous_channel(sd)
        doms.append(dict(nx=c["nx"], ny=c["ny"], nz=c["nz"], nu=c["nu"], force=(c["fx"], 0.0, 0.0), walls_y=True,
                         mask=c["mask"]))
    fluid = int(sum(int((d["mask"] == 0).sum()) for d in doms))
    nodes = int(sum(d["nx"] * d["ny"] * d["nz"] for d in doms))
    b = BatchSolver(doms)
    if args.shape:
        tile, bps, sch = args.shape.split(",")
        b.set_shape(int(tile), int(bps), sch)
        tune = {"fixed": args.shape}
    else:
        tune = b.autotune(trial_steps=10)
    b.step(args.warmup)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    time.sleep(0.3)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    b.step(args.steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    if world > 1:
        t = torch.tensor([ms], device="cuda", dtype=torch.float64)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
    b.close()
    # end to end: masks and parameters from the host, the run, every domain's fields back to the host
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e = BatchSolver(doms)
    e.step(args.steps)
    outs = [e.macroscopic(k) for k in range(len(doms))]
    torch.cuda.synchronize()
    t_e2e = time.perf_counter() - t0
    e.close()
    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    peak = peaks.get("hbm_gbs") or 6800.0
    kernel_ms = ms / args.steps  # the timed region holds only the step kernels (one per step)
    achieved = 216 * fluid / (kernel_ms * 1e-3) / 1e9
    line = {
        "metric": METRIC, "value": world * fluid * args.steps / (ms * 1e-3) / 1e6, "unit": "MLUPS (fluid nodes)",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": wl["text"], "domains": len(doms), "nodes": nodes, "fluid_nodes": fluid,
                   "autotuned": tune, "l2": f"inputs larger than L2: population pool {27 * 4 * nodes / 1e9:.1f} GB"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": committed_traffic("porous512", "fp32") if args.count in (None, 512) else None,
                     "kernel": "k_batch_step", "algorithmic_bytes_per_launch": 216 * fluid,
                     "avg_launch_ms": kernel_ms,
                     "note": "algorithmic bytes count fluid nodes only; the 32-byte sectors that mix fluid and solid "
                             "nodes and the 4-byte link words are read too (traffic)"},
        "e2e": {"value": world * fluid * args.steps / t_e2e / 1e6, "unit": "MLUPS (fluid nodes)",
                "h2d_bytes_per_step": (nodes + 64 * len(doms)) / args.steps, "d2h_bytes_per_step": 16 * nodes / args.steps},
        "gpu_launches": args.steps, "clocks": clk,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def run_ours(args, wl):
    import numpy as np
    import torch

    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    from paper_1905_10182_gb300 import Solver
    from paper_1905_10182_gb300.buildlib import build
    build()

    n = wl["n"]
    shape = grid_shape(wl)
    nodes = shape[0] * shape[1] * shape[2]
    cg = wl["kind"] == "cg"
    if cg:
        from paper_1905_10182_gb300 import rayleigh_taylor
        rho_r, rho_b = rayleigh_taylor.initial_densities(n, wl["rho_h"], wl["rho_l"])
        rho = rho_r + rho_b
        ux = uy = uz = np.zeros_like(rho)
    else:
        rho, ux, uy, uz = initial_fields(wl)

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    # ---- device-resident run (value, roofline)
    s = Solver(*shape, nu=wl["nu"], storage=args.storage, walls_y=cg)
    configure_force(s, wl)
    if cg:
        s.set_colour_gradient(torch.from_numpy(rho_r).cuda(), torch.from_numpy(rho_b).cuda(), **cg_params(wl))
    else:
        s.set_state(torch.from_numpy(rho).cuda(), torch.from_numpy(ux).cuda(), torch.from_numpy(uy).cuda(),
                    torch.from_numpy(uz).cuda())
    mhd = wl["kind"] == "mhd"
    if mhd:
        bmag = initial_magnetic(wl)
        s.set_magnetic(wl["eta"], b=[torch.from_numpy(a).cuda() for a in bmag])
    s.step(args.warmup)
    s.synchronize()
    stream = torch.cuda.current_stream()
    clocks = ClockSampler(dev)
    clocks.start()
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize()
    s.profile(profile_every(args.steps))
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    s.step(args.steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    prof = s.profile_read()
    s.profile(0)
    st = s.stats()  # also raises if any node diverged
    ms_max = ms
    if world > 1:
        t = torch.tensor([ms], device="cuda", dtype=torch.float64)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms_max = float(t.item())
    value = world * nodes * args.steps / (ms_max * 1e-3) / 1e6
    s.close()
    del s

    # ---- end to end through the C ABI with host buffers (pinned), copies inside the timed region
    pin = [torch.from_numpy(a).pin_memory() for a in ((rho_r, rho_b) if cg else (rho, ux, uy, uz))]
    pin_b = [torch.from_numpy(a).pin_memory() for a in bmag] if mhd else None
    out = [torch.empty(a.shape, dtype=torch.float32).pin_memory() for a in (rho, ux, uy, uz)]
    e = Solver(*shape, nu=wl["nu"], storage=args.storage, walls_y=cg)
    configure_force(e, wl)
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    if cg:
        e.set_colour_gradient(*pin, **cg_params(wl))
    else:
        e.set_state(*pin)
    if mhd:
        e.set_magnetic(wl["eta"], b=pin_b)
    e.step(args.steps)
    e.macroscopic(*out)
    torch.cuda.synchronize()
    t_e2e = time.perf_counter() - t0
    barrier()
    if world > 1:
        t = torch.tensor([t_e2e], device="cuda", dtype=torch.float64)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        t_e2e = float(t.item())
    e.close()
    e2e = {"value": world * nodes * args.steps / t_e2e / 1e6, "unit": "MLUPS",
           "h2d_bytes_per_step": (8 if cg else (28 if mhd else 16)) * nodes / args.steps,
           "d2h_bytes_per_step": 16 * nodes / args.steps,
           "note": ("set_colour_gradient from pinned host rho_r, rho_b (8 B/node)" if cg else
                    "set_state from pinned host rho,u (16 B/node)" + (" and set_magnetic from pinned host b (12 B/node)"
                                                                      if mhd else "")) +
                   " + K steps + macroscopic to pinned host (16 B/node); bytes per step are the job's totals / K"}

    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return

    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    peak = peaks.get("hbm_gbs")
    peak_src = "measured" if peak else "fallback"
    peak = peak or 6800.0
    bpn = CG_BYTES_PER_NODE if cg else (MHD_BYTES_PER_NODE if mhd else BYTES_PER_NODE[args.storage])
    if not prof["collide_launches"]:
        raise RuntimeError("no stream-collide launch was timed inside the timed region")
    coll_avg_ms = prof["collide_ms"] / prof["collide_launches"]
    achieved = bpn * nodes / (coll_avg_ms * 1e-3) / 1e9
    traffic = committed_traffic(args.workload, args.storage) if args.n in (None, WORKLOADS[args.workload]["n"]) else None
    # every kernel launched in the timed region: one stream-collide per step, plus psi (Shan-Chen)
    launches = args.steps * (2 if prof["psi_launches"] else 1)

    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        try:
            cpu = oracle_mlups(wl)
        except Exception as exc:  # reported, not hidden
            cpu = {"value": None, "unit": "MLUPS", "cores": os.cpu_count(), "kind": "oracle",
                   "sample": f"failed: {exc}"}

    line = {
        "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": wl["text"] + f", {args.storage} storage", "nodes": nodes, "storage": args.storage,
                   "parallelism": f"{world} independent replicas" if world > 1 else "single GPU",
                   "l2": f"inputs larger than L2: population store {(54 if cg else 27) * nodes * (4 if args.storage == 'fp32' else 2) / 1e6:.0f} MB"
                         " > 129 MB, swept in full every step"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": traffic,
                     "kernel": "k_cg_fields + k_cg_step" if cg else ("k_mhd_step" if mhd else "k_stream_collide"),
                     "algorithmic_bytes_per_launch": bpn * nodes, "avg_launch_ms": coll_avg_ms,
                     "peak_source": f"{peak_src} hbm_gbs (MEASURED_PEAKS.json)" if peak_src == "measured" else "fallback 6.8 TB/s"},
        "kernel_ms_per_step": {"stream_collide": coll_avg_ms,
                               "psi": prof["psi_ms"] / max(1, prof["psi_launches"]) if prof["psi_launches"] else 0.0},
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clk,
        "final_stats": {k: st[k] for k in ("mass", "kinetic_energy", "umax", "step")},
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    args = parse()
    wl = dict(WORKLOADS[args.workload])
    if args.count and wl["kind"] == "porous":
        wl["count"] = args.count
        wl["text"] = wl["text"].replace("512 forced", f"{args.count} forced")
    if args.n:
        if wl["kind"] == "droplet":
            wl["radius"] = wl["radius"] * args.n / wl["n"]
        wl["text"] = wl["text"].replace(f"{wl['n']}^3", f"{args.n}^3")
        if wl["kind"] == "cg":
            wl["text"] = wl["text"].replace(f"{wl['n']}x{4 * wl['n']}x{wl['n']} (W={wl['n']}",
                                            f"{args.n}x{4 * args.n}x{args.n} (W={args.n}")
        wl["n"] = args.n
    if args.impl == "reference":
        run_reference(args, wl)
    elif wl["kind"] == "porous":
        run_batch(args, wl)
    else:
        run_ours(args, wl)


if __name__ == "__main__":
    main()
