"""Rayleigh-Taylor instability with the colour-gradient model (Sec. III and App. D).

A heavy fluid (red, rho_h) lies over a light one (blue, rho_l = 1) in a W x 4W x W box with
no-slip walls at the bottom and top and periodic sides; the interface starts at
y = 2W + 0.05 W [cos(2 pi x / W) + cos(2 pi z / W)] and a body force F = (rho - (rho_h + rho_l)/2) g,
g = (0, -g, 0), with sqrt(g W) = 0.04, drives it.  Re = W sqrt(g W) / nu, At = (rho_h - rho_l) /
(rho_h + rho_l); times in t0 = sqrt(W / g) steps.  Reported: the spike (the lowest point of the
heavy fluid, column x = z = W/2) and the bubble (the highest point of the light fluid, column
x = z = 0), in units of W, where the order parameter changes sign along the column (linear
interpolation, node j at height j + 1/2 above the bottom wall).

    python -m paper_1905_10182_gb300.rayleigh_taylor --W 64 --times 0 0.5 1 1.5 2 2.5 3 3.5 4
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np


def initial_densities(W, rho_h, rho_l):
    nx, ny, nz = W, 4 * W, W
    x = np.arange(nx)[None, None, :]
    z = np.arange(nz)[:, None, None]
    y = np.arange(ny)[None, :, None] + 0.5
    heavy = y > 2 * W + 0.05 * W * (np.cos(2 * math.pi * x / W) + np.cos(2 * math.pi * z / W))
    heavy = np.broadcast_to(heavy, (nz, ny, nx))
    rho_r = np.where(heavy, rho_h, 0.0).astype(np.float32)
    rho_b = np.where(heavy, 0.0, rho_l).astype(np.float32)
    return rho_r, rho_b


def crossing(profile):
    """Height (in nodes, j + 1/2) of the first sign change of the order parameter from below."""
    for j in range(len(profile) - 1):
        a, b = float(profile[j]), float(profile[j + 1])
        if a < 0.0 <= b:
            return j + 0.5 + a / (a - b)
    return float("nan")


def positions(s, W, rho_h, rho_l):
    rr, rb = s.colour_densities()
    phi = (rr / rho_h - rb / rho_l) / (rr / rho_h + rb / rho_l)
    spike = crossing(phi[W // 2, :, W // 2]) / W
    bubble = crossing(phi[0, :, 0]) / W
    return spike, bubble


def run(W=64, At=0.5, Re=512.0, A=1e-4, beta=0.7, times=(0, 0.5, 1, 1.5, 2, 2.5, 3, 3.5, 4)):
    from . import Solver
    rho_l = 1.0
    rho_h = rho_l * (1 + At) / (1 - At)
    g = 0.04 ** 2 / W
    nu = W * 0.04 / Re
    t0 = math.sqrt(W / g)
    s = Solver(W, 4 * W, W, nu=nu, walls_y=True)
    rr, rb = initial_densities(W, rho_h, rho_l)
    s.set_colour_gradient(rr, rb, rho_r0=rho_h, rho_b0=rho_l, nu_r=nu, nu_b=nu, A=A, beta=beta, g=(0.0, -g, 0.0))
    out, done = [], 0
    t_start = time.perf_counter()
    for tt in times:
        target = int(round(tt * t0))
        s.step(target - done)
        done = target
        sp, bu = positions(s, W, rho_h, rho_l)
        out.append({"t_over_t0": float(tt), "step": done, "spike": float(sp), "bubble": float(bu)})
    wall = time.perf_counter() - t_start
    stats = s.stats()
    s.close()
    return {"W": W, "At": At, "Re": Re, "A": A, "beta": beta, "t0_steps": t0, "wall_s": wall,
            "mass": float(stats["mass"]), "history": out}


def main():
    import torch
    ap = argparse.ArgumentParser()
    ap.add_argument("--W", type=int, default=64)
    ap.add_argument("--A", type=float, default=1e-4)
    ap.add_argument("--beta", type=float, default=0.7)
    ap.add_argument("--times", type=float, nargs="+", default=[0, 0.5, 1, 1.5, 2, 2.5, 3, 3.5, 4])
    args = ap.parse_args()
    torch.cuda.set_device(0)
    print(json.dumps(run(W=args.W, A=args.A, beta=args.beta, times=args.times)), flush=True)


if __name__ == "__main__":
    main()
