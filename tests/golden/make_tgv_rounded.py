"""Writes tgv64_rounded_oracle.txt: kinetic energy and enstrophy of the decaying Taylor-Green vortex
(64^3 periodic, U0 = 0.05, nu = 1e-4, 5000 steps, every 250 steps) on the FP64 oracle, three ways:
plain FP64, and with the state stored as FP16 or BF16 deviations g = f - w (round to nearest
even after every step; all arithmetic FP64).  The rounding sits in this driver, between oracle
steps; it does none of the method's arithmetic.  The difference between a rounded run and the
plain run is the effect of storage rounding alone, free of any kernel arithmetic.  Calls only
the oracle.  Run from the repository root (about two hours on 8 cores):

    python tests/golden/make_tgv_rounded.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1905_10182_gb300 import inputs  # noqa: E402

N, U0, NU, STEPS, EVERY = 64, 0.05, 1e-4, 5000, 250


def round_fp16(g):
    return g.astype(np.float32).astype(np.float16).astype(np.float64)


def round_bf16(g):
    b = g.astype(np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def run(rounding, threads):
    rho, ux, uy, uz = inputs.taylor_green(N, U0)
    g = oracle.Grid(N, N, N, nu=NU, collision=oracle.COLL_PAPER, threads=threads)
    f = g.init_equilibrium(rho.astype(np.float64), np.stack([ux, uy, uz]).astype(np.float64))
    w = oracle.weights()[:, None, None, None]
    if rounding:
        f = w + rounding(f - w)
    ke, ens = [], []
    for k in range(0, STEPS + 1, EVERY):
        if k:
            if rounding:
                for _ in range(EVERY):
                    f = w + rounding(g.step(f, 1) - w)
            else:
                f = g.step(f, EVERY)
        _, u = g.macroscopic(f)
        ke.append(oracle.kinetic_energy(u))
        ens.append(oracle.enstrophy(u))
        print(rounding.__name__ if rounding else "fp64", k, ke[-1], ens[-1], flush=True)
    return ke, ens


def main():
    threads = int(os.environ.get("ORACLE_THREADS", "0"))
    lines = ["# Taylor-Green vortex 64^3, U0 = 0.05, nu = 1e-4, FP64 oracle (five-step algorithm of Sec. II);",
             "# state rounded after every step to FP16 / BF16 deviations (round to nearest even) or not.",
             "# Written by tests/golden/make_tgv_rounded.py (oracle only).  Values every 250 steps, 0..5000.",
             "# keys: ke_<fp64|fp16|bf16>_<step>, ens_<fp64|fp16|bf16>_<step>"]
    for name, rnd in (("fp64", None), ("fp16", round_fp16), ("bf16", round_bf16)):
        ke, ens = run(rnd, threads)
        for j, k in enumerate(range(0, STEPS + 1, EVERY)):
            lines += [f"ke_{name}_{k} = {ke[j]:.12e}", f"ens_{name}_{k} = {ens[j]:.12e}"]
    with open(os.path.join(HERE, "tgv64_rounded_oracle.txt"), "w") as fh:
        fh.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
