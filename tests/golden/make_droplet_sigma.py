"""Writes droplet_sigma_oracle64.txt: the surface tension of the Shan-Chen static droplet measured on
the FP64 oracle at 64^3 (G = -5.5, nu = 1/6, psi = 1 - exp(-rho), tanh profile rho_l = 2.4,
rho_g = 0.13, width 2, R = 8, 12, 16: the 128^3 benchmark radii 16, 24, 32 halved), after 3000
and 5000 steps.  Calls only the oracle.  Run from the repository root:

    python tests/golden/make_droplet_sigma.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.dirname(HERE))

import oracle  # noqa: E402
from droplet_laplace import laplace  # noqa: E402
from paper_1905_10182_gb300 import inputs  # noqa: E402

G, M, NU = -5.5, 64, 1.0 / 6.0
RADII = (8, 12, 16)
CHECKPOINTS = (3000, 5000)


def main():
    lines = ["# Shan-Chen static droplet on the FP64 oracle (five-step algorithm of Sec. II), 64^3 periodic,",
             "# G = -5.5, nu = 1/6, tanh profile rho_l = 2.4, rho_g = 0.13, width 2, centred at node 32.",
             "# Written by tests/golden/make_droplet_sigma.py (oracle only).  sigma = dp R_eff / 2,",
             "# dp between the centre and the far corner, R_eff the volume-equivalent radius.",
             "# keys: sigma_R<radius>_s<steps>, dp_..., reff_..."]
    for R in RADII:
        g = oracle.Grid(M, M, M, nu=NU, force_kind=oracle.FORCE_SHAN_CHEN, G=G, collision=oracle.COLL_PAPER)
        f = g.init_equilibrium(inputs.droplet_density(M, R).astype(np.float64), np.zeros((3, M, M, M)))
        done = 0
        for s in CHECKPOINTS:
            f = g.step(f, s - done)
            done = s
            rho, _ = g.macroscopic(f)
            dp, reff = laplace(rho, G, M)
            lines += [f"dp_R{R}_s{s} = {dp:.10e}", f"reff_R{R}_s{s} = {reff:.10e}",
                      f"sigma_R{R}_s{s} = {dp * reff / 2.0:.10e}"]
            print(lines[-1], flush=True)
    with open(os.path.join(HERE, "droplet_sigma_oracle64.txt"), "w") as fh:
        fh.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
