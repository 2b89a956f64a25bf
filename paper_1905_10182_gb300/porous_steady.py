"""The batched forced porous channels run to steady state, with a per-domain record.

512 channels (inputs.porous_channel, seeds 0..511: nx, nz ~ U{32..96}, ny ~ U{32..48}, walls in y,
sphere packs of solid fraction up to 0.2, nu ~ U[0.01, 0.1], F_x ~ U[1e-6, 1e-5]) advance in one
batch (one persistent launch per step, CUDA-graph replay, autotuned shape) until each is steady,
diverges, or max_steps elapse.  Per domain the record holds the steps, the status, the final
residual both per step (the stopping rule: r = ||u^n - u^(n - D)|| / (D ||u^n||), D = 100) and
over the window (D r), and the Mach number predicted by the clean-channel Poiseuille maximum
u_max = F_x H^2 / (8 nu) (H = ny) against the measured max |u| / c_s.  A domain that is not steady
or that diverged is a reported failure.

The windowed residual of 1e-8 (per step 1e-10) is then tried on the first floor_count domains
with a step cap: the final residuals show where FP32 storage stops improving.

    python -m paper_1905_10182_gb300.porous_steady --json porous512_steady.json
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

CS = 1.0 / math.sqrt(3.0)
STATUS = {0: "steady", 1: "not steady", 2: "diverged"}


def domains(count, seed0=0):
    from . import inputs
    doms, meta = [], []
    for sd in range(seed0, seed0 + count):
        c = inputs.porous_channel(sd)
        doms.append(dict(nx=c["nx"], ny=c["ny"], nz=c["nz"], nu=c["nu"], force=(c["fx"], 0.0, 0.0), walls_y=True,
                         mask=c["mask"]))
        meta.append(c)
    return doms, meta


def run(doms, tol, max_steps, check_every, shape=None):
    import torch

    from . import BatchSolver
    b = BatchSolver(doms)
    tune = b.autotune(trial_steps=10) if shape is None else (b.set_shape(*shape) or {"fixed": list(shape)})
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    steps, res, status = b.run(tol=tol, max_steps=max_steps, check_every=check_every)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    umax = []
    for k, d in enumerate(doms):
        _, ux, uy, uz = b.macroscopic(k)
        fluid = d["mask"] == 0
        sp = np.sqrt(ux.astype(np.float64) ** 2 + uy ** 2 + uz ** 2)[fluid]
        umax.append(float(sp.max()) if sp.size and np.isfinite(sp).all() else float("nan"))
    b.close()
    return steps, res, status, wall, umax, tune


def main():
    import torch
    ap = argparse.ArgumentParser()
    ap.add_argument("--count", type=int, default=512)
    ap.add_argument("--tol", type=float, default=1e-8, help="per-step residual tolerance")
    ap.add_argument("--max-steps", type=int, default=600000)
    ap.add_argument("--check-every", type=int, default=100)
    ap.add_argument("--floor-count", type=int, default=32)
    ap.add_argument("--floor-tol", type=float, default=1e-10)
    ap.add_argument("--floor-max-steps", type=int, default=200000)
    ap.add_argument("--json", default=None)
    args = ap.parse_args()
    torch.cuda.set_device(0)
    doms, meta = domains(args.count)
    nodes = sum(d["nx"] * d["ny"] * d["nz"] for d in doms)
    fluid = sum(int((d["mask"] == 0).sum()) for d in doms)
    steps, res, status, wall, umax, tune = run(doms, args.tol, args.max_steps, args.check_every)
    per = []
    for k, (d, c) in enumerate(zip(doms, meta)):
        pred = c["fx"] * c["ny"] ** 2 / (8.0 * c["nu"])
        per.append({"seed": c["seed"], "nx": d["nx"], "ny": d["ny"], "nz": d["nz"], "nu": c["nu"], "fx": c["fx"],
                    "solid_fraction": float(d["mask"].mean()), "steps": int(steps[k]),
                    "status": STATUS[int(status[k])], "residual_per_step": float(res[k]),
                    "residual_windowed": float(res[k] * args.check_every),
                    "mach_predicted": pred / CS, "mach_measured": umax[k] / CS})
    ok = [p for p in per if p["status"] == "steady"]
    summary = {
        "domains": len(doms), "nodes": nodes, "fluid_nodes": fluid, "autotuned": tune,
        "tol_per_step": args.tol, "tol_windowed": args.tol * args.check_every, "max_steps": args.max_steps,
        "steady": len(ok), "not_steady": sum(p["status"] == "not steady" for p in per),
        "diverged": sum(p["status"] == "diverged" for p in per), "wall_s": wall,
        "steps_mean": float(np.mean([p["steps"] for p in per])), "steps_max": int(max(p["steps"] for p in per)),
        "fluid_node_updates": int(sum(int((d["mask"] == 0).sum()) * p["steps"] for d, p in zip(doms, per))),
        "mach_predicted_max": max(p["mach_predicted"] for p in per),
        "mach_measured_max": float(np.nanmax([p["mach_measured"] for p in per])),
        "domains_mach_predicted_over_0.3": sum(p["mach_predicted"] > 0.3 for p in per),
    }
    summary["fluid_mlups_over_run"] = summary["fluid_node_updates"] / wall / 1e6
    print(json.dumps(summary), flush=True)

    # windowed 1e-8 on the first floor_count domains, capped
    fl = list(range(min(args.floor_count, len(doms))))
    fs, fr, fst, fwall, _, _ = run([doms[k] for k in fl], args.floor_tol, args.floor_max_steps, args.check_every,
                                   shape=(64, 8, "strided_prefetch"))
    floor = {"domains": [meta[k]["seed"] for k in fl], "tol_per_step": args.floor_tol,
             "tol_windowed": args.floor_tol * args.check_every, "max_steps": args.floor_max_steps,
             "reached": int((fst == 0).sum()), "steps": fs.tolist(), "status": [STATUS[int(s)] for s in fst],
             "final_residual_windowed": (fr * args.check_every).tolist(), "wall_s": fwall}
    print(json.dumps({k: v for k, v in floor.items() if not isinstance(v, list)} |
                     {"final_residual_windowed_median": float(np.median(fr) * args.check_every)}), flush=True)
    if args.json:
        with open(args.json, "w") as fh:
            json.dump({"summary": summary, "per_domain": per, "windowed_1e-8": floor}, fh, indent=1)


if __name__ == "__main__":
    main()
