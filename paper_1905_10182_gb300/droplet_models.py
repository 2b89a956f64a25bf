"""Static droplet with the Shan-Chen force under the complete and the second-order Hermite
expansions (Sec. III, static droplet: models M1, M4 and M5 compared by the time history of the
mean kinetic energy).

A periodic n^3 box holds a droplet of density rho_l = rho0 centred at node (n/2, n/2, n/2) in a
vapour of density rho0/8, G = -6 (the values of Sec. III).  The paper gives neither the radius,
nor the viscosity, nor the interface width: they are parameters here (default: a sharp step,
width 0).  For every model and viscosity the run records the mean kinetic energy (FP64
diagnostics of lbm_stats) every `every` steps and the first check at which the divergence flag
(rho <= 0, |u| >= 1 or NaN) was seen.

    python -m paper_1905_10182_gb300.droplet_models --n 200 --steps 2000 --nu 0.1667 0.05 0.01
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np


def initial_density(n, radius, rho_l, rho_g, width):
    if width > 0:
        from .inputs import droplet_density
        return droplet_density(n, radius, rho_l=rho_l, rho_g=rho_g, width=width)
    c = n / 2
    ax = np.arange(n, dtype=np.float64)
    z, y, x = np.meshgrid(ax, ax, ax, indexing="ij")
    r2 = (x - c) ** 2 + (y - c) ** 2 + (z - c) ** 2
    return np.where(r2 < radius * radius, rho_l, rho_g).astype(np.float32)


def run(model, n, nu, radius, G=-6.0, rho_l=1.0, rho_g=0.125, width=0.0, steps=2000, every=10,
        storage="fp32"):
    """Mean kinetic energy history of one droplet run; diverged_at is the first check that saw
    the divergence flag (None if the run stayed in range)."""
    from . import Solver
    from ._native import LBM_ERR_DIVERGED, LbmError
    s = Solver(n, n, n, nu=nu, storage=storage)
    s.set_force("shan_chen", (G,))
    s.set_model(model)
    rho = initial_density(n, radius, rho_l, rho_g, width)
    z = np.zeros_like(rho)
    s.set_state(rho, z, z, z)
    ke, t, diverged_at = [], [], None
    t0 = time.perf_counter()
    for k in range(0, steps, every):
        try:
            s.step(every)
            st = s.stats()
        except LbmError as e:
            if e.status != LBM_ERR_DIVERGED:
                raise
            diverged_at = k + every
            break
        ke.append(st["kinetic_energy"])
        t.append(k + every)
    wall = time.perf_counter() - t0
    s.close()
    out = {"model": model, "nu": nu, "radius": radius, "steps_run": t[-1] if t else 0,
           "diverged_at": diverged_at, "ke_max": max(ke) if ke else None,
           "ke_last": ke[-1] if ke else None, "wall_s": wall, "t": t, "ke": ke}
    return out


def main():
    import torch
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=200)
    ap.add_argument("--radius", type=float, default=None, help="default n/5")
    ap.add_argument("--nu", type=float, nargs="+", default=[1.0 / 6.0, 0.05, 0.01])
    ap.add_argument("--models", nargs="+", default=["M1", "M4", "M5"])
    ap.add_argument("--G", type=float, default=-6.0)
    ap.add_argument("--rho-l", type=float, default=1.0)
    ap.add_argument("--rho-g", type=float, default=0.125)
    ap.add_argument("--width", type=float, default=0.0)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--every", type=int, default=10)
    ap.add_argument("--storage", default="fp32")
    args = ap.parse_args()
    torch.cuda.set_device(0)
    R = args.radius if args.radius is not None else args.n / 5
    for nu in args.nu:
        for m in args.models:
            r = run(m, args.n, nu, R, G=args.G, rho_l=args.rho_l, rho_g=args.rho_g, width=args.width,
                    steps=args.steps, every=args.every, storage=args.storage)
            print(json.dumps(r), flush=True)


if __name__ == "__main__":
    main()
