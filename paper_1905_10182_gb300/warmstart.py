"""Learned warm start for steady solves of forced porous channels.

1. The batched solver (lbm_batch_*) runs a set of training channels to steady state.
2. The neural operator (lbm_no_*) is trained on the GPU to map (mask, F_x, nu, y) to the steady
   (u, rho), velocities scaled by the clean-channel Poiseuille maximum u_ref = F_x H^2 / (8 nu).
3. For held-out channels, the plain solver starts once from rest (cold) and once from
   f^eq(rho_hat, u_hat) of the prediction (warm); both run to the same residual tolerance.
   The cold run is the judge: reported are steps and wall time for both, and the field
   difference between the warm and the cold steady state.

    python -m paper_1905_10182_gb300.warmstart --train 512 --test 64 --epochs 60
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np


def make_domains(seeds, n):
    from . import inputs
    doms, meta = [], []
    for sd in seeds:
        c = inputs.porous_cube(sd, n)
        doms.append(dict(nx=n, ny=n, nz=n, nu=c["nu"], force=(c["fx"], 0.0, 0.0), walls_y=True, mask=c["mask"]))
        meta.append(c)
    return doms, meta


def u_ref(c):
    return c["fx"] * c["ny"] ** 2 / (8.0 * c["nu"])


def features(c):
    """Input channels of the operator: solid mask, F_x / 1e-5, nu / 0.1, (y + 1/2) / ny."""
    n = c["nx"]
    a = np.empty((4, n, n, n), np.float32)
    a[0] = c["mask"]
    a[1] = c["fx"] / 1e-5
    a[2] = c["nu"] / 0.1
    a[3] = ((np.arange(n) + 0.5) / n)[None, :, None]
    return a


def solve(doms, init=None, tol=1e-8, max_steps=400000, check_every=100):
    """Runs a batch to steady; init: optional list of (rho, ux, uy, uz) per domain."""
    import torch

    from . import BatchSolver
    b = BatchSolver(doms)
    b.autotune(trial_steps=4)
    if init is not None:
        for k, (r, ux, uy, uz) in enumerate(init):
            b.set_state(k, r, ux, uy, uz)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    steps, res, status = b.run(tol=tol, max_steps=max_steps, check_every=check_every)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    fields = [b.macroscopic(k) for k in range(len(doms))]
    b.close()
    return steps, res, status, wall, fields


def main():
    import torch

    from .neural import NeuralOperator
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=64)
    ap.add_argument("--train", type=int, default=512)
    ap.add_argument("--test", type=int, default=64)
    ap.add_argument("--epochs", type=int, default=60)
    ap.add_argument("--batch", type=int, default=4)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--width", type=int, default=32)
    ap.add_argument("--modes", type=int, default=12)
    ap.add_argument("--layers", type=int, default=4)
    ap.add_argument("--tol", type=float, default=1e-8)
    ap.add_argument("--max-steps", type=int, default=400000)
    ap.add_argument("--test-seed0", type=int, default=10000)
    args = ap.parse_args()
    torch.cuda.set_device(0)
    n = args.n
    report = {"config": vars(args)}

    # 1. training data from the batched solver
    tdoms, tmeta = make_domains(range(args.train), n)
    t0 = time.perf_counter()
    steps, res, status, wall, fields = solve(tdoms, tol=args.tol, max_steps=args.max_steps)
    print(json.dumps({"stage": "data done", "wall_s": time.perf_counter() - t0}), flush=True)
    report["data"] = {"wall_s": time.perf_counter() - t0, "solve_wall_s": wall, "steady": int((status == 0).sum()),
                      "diverged": int((status == 2).sum()), "mean_steps": float(steps.mean()),
                      "max_steps": int(steps.max())}
    keep = [k for k in range(args.train) if status[k] == 0]
    X = torch.empty((len(keep), 4, n, n, n), dtype=torch.float32, device="cuda")
    Y = torch.empty_like(X)
    for j, k in enumerate(keep):
        c = tmeta[k]
        X[j] = torch.from_numpy(features(c))
        r, ux, uy, uz = fields[k]
        ur = u_ref(c)
        Y[j] = torch.from_numpy(np.stack([ux / ur, uy / ur, uz / ur, (r - 1.0) / ur]).astype(np.float32))
    del fields

    # 2. training on the GPU with the operator's own kernels
    net = NeuralOperator(D=n, width=args.width, modes=args.modes, layers=args.layers, in_ch=4, out_ch=4,
                         max_batch=args.batch, seed=1)
    nb = len(keep) // args.batch
    rng = np.random.default_rng(0)
    t0 = time.perf_counter()
    hist = []
    total = args.epochs * nb
    it = 0
    for ep in range(args.epochs):
        perm = rng.permutation(len(keep))
        el = 0.0
        for i in range(nb):
            idx = torch.from_numpy(perm[i * args.batch:(i + 1) * args.batch]).cuda()
            lr = args.lr * 0.5 * (1.0 + math.cos(math.pi * it / total))
            el += net.train_step(X[idx].contiguous(), Y[idx].contiguous(), lr)
            it += 1
        hist.append(el / max(nb, 1))
        print(json.dumps({"epoch": ep, "loss": hist[-1], "t": time.perf_counter() - t0}), flush=True)
    torch.cuda.synchronize()
    report["train"] = {"samples": len(keep), "epochs": args.epochs, "wall_s": time.perf_counter() - t0,
                       "loss_first": hist[0] if hist else None, "loss_last": hist[-1] if hist else None,
                       "params": net.param_count, "loss_history": hist}

    # 3. held-out seeds: cold (rest) vs warm (prediction) to the same residual
    vdoms, vmeta = make_domains(range(args.test_seed0, args.test_seed0 + args.test), n)
    t0 = time.perf_counter()
    init, rel_pred = [], []
    out = torch.empty((1, 4, n, n, n), device="cuda")
    for c in vmeta:
        net.forward(torch.from_numpy(features(c)[None]).cuda(), out)
        p = out[0].cpu().numpy().astype(np.float64)
        ur = u_ref(c)
        fluid = c["mask"] == 0
        u = [np.where(fluid, p[k] * ur, 0.0).astype(np.float32) for k in range(3)]
        rho = np.where(fluid, 1.0 + p[3] * ur, 1.0).astype(np.float32)
        init.append((rho, u[0], u[1], u[2]))
    infer_wall = time.perf_counter() - t0
    cs, cr, cst, cwall, cf = solve(vdoms, tol=args.tol, max_steps=args.max_steps)
    ws, wr, wst, wwall, wf = solve(vdoms, init=init, tol=args.tol, max_steps=args.max_steps)
    errs, pred_errs, gain = [], [], []
    for k in range(args.test):
        uc = np.stack(cf[k][1:4]).astype(np.float64)
        uw = np.stack(wf[k][1:4]).astype(np.float64)
        up = np.stack(init[k][1:4]).astype(np.float64)
        nrm = np.linalg.norm(uc)
        errs.append(float(np.linalg.norm(uw - uc) / nrm))
        pred_errs.append(float(np.linalg.norm(up - uc) / nrm))
        if cst[k] == 0 and wst[k] == 0:
            gain.append(1.0 - ws[k] / cs[k])
    report["eval"] = {
        "domains": args.test, "cold_steady": int((cst == 0).sum()), "warm_steady": int((wst == 0).sum()),
        "cold_steps_mean": float(cs.mean()), "warm_steps_mean": float(ws.mean()),
        "cold_wall_s": cwall, "warm_wall_s": wwall, "warm_inference_s": infer_wall,
        "warm_total_wall_s": wwall + infer_wall,
        "wall_speedup": cwall / (wwall + infer_wall),
        "steps_saved_mean": float(np.mean(gain)) if gain else None,
        "prediction_rel_error_mean": float(np.mean(pred_errs)), "prediction_rel_error_median": float(np.median(pred_errs)),
        "final_field_rel_diff_max": float(np.max(errs)), "final_field_rel_diff_mean": float(np.mean(errs)),
        "bound_steps_saved_at_pred_error": float(math.log(1.0 / max(np.median(pred_errs), 1e-12)) / math.log(1.0 / args.tol)),
    }
    print(json.dumps(report), flush=True)


if __name__ == "__main__":
    main()
