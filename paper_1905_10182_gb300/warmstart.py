"""Learned warm start for steady solves of forced porous channels.

1. The batched solver (lbm_batch_*) runs a set of training channels to steady state.
2. The neural operator (lbm_no_*) is trained on the GPU to map (mask, F_x, nu, y) to the steady
   (u, rho), velocities scaled by the clean-channel Poiseuille maximum u_ref = F_x H^2 / (8 nu).
3. For held-out channels, the plain solver starts once from rest (cold) and once from
   f^eq(rho_hat, u_hat) of the prediction (warm); both run to the same residual tolerance.
   The cold run is the judge: reported are steps and wall time for both, and the field
   difference between the warm and the cold steady state.  A warm solve that does not reach the
   tolerance (not steady within max_steps, or diverged) is replaced by a cold solve of the same
   domain, whose steps and wall time are charged to the warm side.

Steady criterion: r = ||u^n - u^(n - Delta)||_2 / (Delta ||u^n||_2) over fluid nodes, FP64,
checked every Delta = check_every = 100 steps, r <= tol (1e-8): the mean relative change per
step.  The windowed change ||u^n - u^(n - Delta)|| / ||u^n|| is Delta r, 1e-6 at that tolerance;
both are reported.

    python -m paper_1905_10182_gb300.warmstart --train 2000 --test 256 --epochs 30 --json out.json
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

CHECK_EVERY = 100


def make_domains(seeds, n, nu_range=(0.01, 0.1)):
    from . import inputs
    doms, meta = [], []
    for sd in seeds:
        c = inputs.porous_cube(sd, n, nu_range)
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


def solve(doms, init=None, tol=1e-8, max_steps=400000, check_every=CHECK_EVERY, shape=None):
    """Runs a batch to steady; init: optional list of (rho, ux, uy, uz) per domain (None entries
    start from rest).  Returns steps, per-step residual, status (0 steady, 1 not steady, 2
    diverged), wall seconds of the run, and every domain's (rho, ux, uy, uz)."""
    import torch

    from . import BatchSolver
    b = BatchSolver(doms)
    if shape is None:
        b.autotune(trial_steps=4)
    else:
        b.set_shape(*shape)
    if init is not None:
        for k, st in enumerate(init):
            if st is not None:
                b.set_state(k, *st)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    steps, res, status = b.run(tol=tol, max_steps=max_steps, check_every=check_every)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    fields = [b.macroscopic(k) for k in range(len(doms))]
    b.close()
    return steps, res, status, wall, fields


def training_set(metas, fields, status):
    """Device tensors X (features) and Y (u / u_ref, (rho - 1) / u_ref) of the steady domains."""
    import torch
    keep = [k for k in range(len(metas)) if status[k] == 0]
    n = metas[0]["nx"]
    X = torch.empty((len(keep), 4, n, n, n), dtype=torch.float32, device="cuda")
    Y = torch.empty_like(X)
    for j, k in enumerate(keep):
        c = metas[k]
        X[j] = torch.from_numpy(features(c))
        r, ux, uy, uz = fields[k]
        ur = u_ref(c)
        Y[j] = torch.from_numpy(np.stack([ux / ur, uy / ur, uz / ur, (r - 1.0) / ur]).astype(np.float32))
    return X, Y


def train(X, Y, epochs, batch=4, lr=1e-3, width=32, modes=12, layers=4, seed=1, log=None):
    """Trains the operator with its own GPU kernels (Adam, cosine decay); returns (net, losses)."""
    import torch

    from .neural import NeuralOperator
    n = X.shape[-1]
    net = NeuralOperator(D=n, width=width, modes=modes, layers=layers, in_ch=4, out_ch=4, max_batch=batch, seed=seed)
    nb = X.shape[0] // batch
    rng = np.random.default_rng(seed)
    hist, it, total = [], 0, max(1, epochs * nb)
    for ep in range(epochs):
        perm = rng.permutation(X.shape[0])
        el = 0.0
        for i in range(nb):
            idx = torch.from_numpy(perm[i * batch:(i + 1) * batch]).cuda()
            step_lr = lr * 0.5 * (1.0 + math.cos(math.pi * it / total))
            el += net.train_step(X[idx].contiguous(), Y[idx].contiguous(), step_lr)
            it += 1
        hist.append(el / max(nb, 1))
        if log:
            log({"epoch": ep, "loss": hist[-1]})
    return net, hist


def predict(net, metas, density=True):
    """Initial states f^eq(rho_hat, u_hat) for each domain from the operator's prediction (solid
    nodes at rest; density=False keeps rho = 1 and takes only the velocity); returns the list of
    (rho, ux, uy, uz) and the inference wall time."""
    import torch
    n = metas[0]["nx"]
    nb = max(1, int(getattr(net, "max_batch", 1)))  # domains per forward
    out = torch.empty((nb, 4, n, n, n), device="cuda")
    init = []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for j in range(0, len(metas), nb):
        group = metas[j:j + nb]
        x = torch.from_numpy(np.stack([features(c) for c in group])).cuda()
        net.forward(x, out[:len(group)])
        preds = out[:len(group)].cpu().numpy().astype(np.float64)
        for c, p in zip(group, preds):
            ur = u_ref(c)
            fluid = c["mask"] == 0
            u = [np.where(fluid, p[k] * ur, 0.0).astype(np.float32) for k in range(3)]
            rho = np.where(fluid, 1.0 + p[3] * ur, 1.0).astype(np.float32) if density else np.ones_like(u[0])
            init.append((rho, u[0], u[1], u[2]))
    torch.cuda.synchronize()
    return init, time.perf_counter() - t0


def rel_l2(a, b):
    """||a - b|| / ||b|| over the three velocity components."""
    a = np.stack(a[1:4]).astype(np.float64)
    b = np.stack(b[1:4]).astype(np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def compare(doms, init, infer_wall, tol=1e-8, max_steps=400000, shape=None):
    """Cold and warm solves of the same domains to the same tolerance, with the cold fallback for
    warm solves that fail.  Returns a report dict (per-domain lists included)."""
    cs, cr, cst, cwall, cf = solve(doms, tol=tol, max_steps=max_steps, shape=shape)
    ws, wr, wst, wwall, wf = solve(doms, init=init, tol=tol, max_steps=max_steps, shape=shape)
    ws, wr, wst = ws.copy(), wr.copy(), wst.copy()
    failed = [k for k in range(len(doms)) if wst[k] != 0]
    fb_wall = 0.0
    if failed:
        fs, fr, fst, fb_wall, ff = solve([doms[k] for k in failed], tol=tol, max_steps=max_steps, shape=shape)
        for j, k in enumerate(failed):
            ws[k] = ws[k] + fs[j]  # the failed warm steps are charged too
            wr[k], wst[k], wf[k] = fr[j], fst[j], ff[j]
    pred_err = [rel_l2(init[k], cf[k]) if init[k] is not None else 1.0 for k in range(len(doms))]
    field_diff = [rel_l2(wf[k], cf[k]) for k in range(len(doms))]
    ratio = [float(ws[k] / cs[k]) if cs[k] > 0 else float("nan") for k in range(len(doms))]
    warm_total = wwall + fb_wall + infer_wall
    return {
        "domains": len(doms), "tol_per_step": tol, "tol_windowed": tol * CHECK_EVERY, "check_every": CHECK_EVERY,
        "cold_steady": int((cst == 0).sum()), "warm_steady": int((wst == 0).sum()), "warm_fallbacks": failed,
        "cold_steps": cs.tolist(), "warm_steps": ws.tolist(), "step_ratio_warm_over_cold": ratio,
        "cold_steps_total": int(cs.sum()), "warm_steps_total": int(ws.sum()),
        "cold_residual_per_step": cr.tolist(), "warm_residual_per_step": wr.tolist(),
        "cold_residual_windowed_max": float(np.max(cr) * CHECK_EVERY),
        "warm_residual_windowed_max": float(np.max(wr) * CHECK_EVERY),
        "cold_wall_s": cwall, "warm_wall_s": wwall, "fallback_wall_s": fb_wall, "inference_s": infer_wall,
        "wall_speedup": cwall / warm_total if warm_total > 0 else float("nan"),
        "step_ratio_median": float(np.nanmedian(ratio)), "step_ratio_mean": float(np.nanmean(ratio)),
        "domains_faster_warm": int(sum(r < 1.0 for r in ratio)),
        "prediction_rel_error": pred_err, "prediction_rel_error_median": float(np.median(pred_err)),
        "final_field_rel_diff": field_diff, "final_field_rel_diff_max": float(np.max(field_diff)),
        "bound_steps_saved_at_median_pred_error":
            float(math.log(1.0 / max(np.median(pred_err), 1e-12)) / math.log(1.0 / tol)),
    }


def main():
    import torch
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
    ap.add_argument("--json", default=None, help="write the full report (per-domain lists included) here")
    args = ap.parse_args()
    torch.cuda.set_device(0)
    n = args.n
    report = {"config": vars(args)}

    tdoms, tmeta = make_domains(range(args.train), n)
    t0 = time.perf_counter()
    steps, res, status, wall, fields = solve(tdoms, tol=args.tol, max_steps=args.max_steps)
    report["data"] = {"wall_s": time.perf_counter() - t0, "solve_wall_s": wall, "steady": int((status == 0).sum()),
                      "diverged": int((status == 2).sum()), "mean_steps": float(steps.mean()),
                      "max_steps": int(steps.max())}
    print(json.dumps({"stage": "data", **report["data"]}), flush=True)
    X, Y = training_set(tmeta, fields, status)
    del fields
    t0 = time.perf_counter()
    net, hist = train(X, Y, args.epochs, args.batch, args.lr, args.width, args.modes, args.layers,
                      log=lambda d: print(json.dumps(d), flush=True))
    torch.cuda.synchronize()
    report["train"] = {"samples": int(X.shape[0]), "epochs": args.epochs, "wall_s": time.perf_counter() - t0,
                       "loss_first": hist[0] if hist else None, "loss_last": hist[-1] if hist else None,
                       "params": net.param_count, "loss_history": hist}
    del X, Y
    vdoms, vmeta = make_domains(range(args.test_seed0, args.test_seed0 + args.test), n)
    init, infer_wall = predict(net, vmeta)
    report["eval"] = compare(vdoms, init, infer_wall, tol=args.tol, max_steps=args.max_steps)
    summary = {k: v for k, v in report["eval"].items() if not isinstance(v, list) or k == "warm_fallbacks"}
    print(json.dumps({"config": report["config"], "data": report["data"],
                      "train": {k: v for k, v in report["train"].items() if k != "loss_history"},
                      "eval": summary}), flush=True)
    if args.json:
        with open(args.json, "w") as fh:
            json.dump(report, fh)


if __name__ == "__main__":
    main()
