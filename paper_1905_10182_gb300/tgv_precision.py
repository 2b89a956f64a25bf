"""Decaying Taylor-Green vortex at low viscosity with FP32, FP16 and BF16 deviation storage (the
arithmetic is FP32 in all three): kinetic-energy and enstrophy curves (FP64 diagnostics of
lbm_stats) at N^3.

    python -m paper_1905_10182_gb300.tgv_precision --n 512 --steps 5000 --every 250

Reported per storage: the curves, and the largest relative deviation of each from the FP32 curve.
The time unit L / U0 (L = N / (2 pi)) is given in steps.
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np


def gpu_curve(n, u0, nu, steps, every, storage):
    from . import Solver, inputs
    rho, ux, uy, uz = inputs.taylor_green(n, u0)
    s = Solver(n, n, n, nu=nu, storage=storage)
    s.set_state(rho, ux, uy, uz)
    t, ke, ens = [0], [], []
    st = s.stats()
    ke.append(st["kinetic_energy"])
    ens.append(st["enstrophy"])
    t0 = time.perf_counter()
    for k in range(every, steps + 1, every):
        s.step(every)
        st = s.stats()
        t.append(k)
        ke.append(st["kinetic_energy"])
        ens.append(st["enstrophy"])
    wall = time.perf_counter() - t0
    s.close()
    return {"t": t, "ke": ke, "enstrophy": ens, "wall_s": wall}


def rel_dev(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.max(np.abs(a - b) / np.abs(b)))


def main():
    import torch
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=512)
    ap.add_argument("--u0", type=float, default=0.05)
    ap.add_argument("--nu", type=float, default=1e-4)
    ap.add_argument("--steps", type=int, default=5000)
    ap.add_argument("--every", type=int, default=250)
    args = ap.parse_args()
    torch.cuda.set_device(0)
    L = args.n / (2 * math.pi)
    out = {"config": vars(args), "time_unit_steps": L / args.u0}
    curves = {st: gpu_curve(args.n, args.u0, args.nu, args.steps, args.every, st) for st in ("fp32", "fp16", "bf16")}
    for st in ("fp16", "bf16"):
        curves[st]["ke_rel_dev_vs_fp32"] = rel_dev(curves[st]["ke"], curves["fp32"]["ke"])
        curves[st]["enstrophy_rel_dev_vs_fp32"] = rel_dev(curves[st]["enstrophy"], curves["fp32"]["enstrophy"])
    out["gpu"] = curves
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
