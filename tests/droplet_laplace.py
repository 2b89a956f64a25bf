"""Laplace-law measurement on a static-droplet density field (Sec. III, static droplet), used by
the GPU physics test and by the script that stores the oracle's surface tension.

Pressure of the pseudo-potential fluid: p = rho c_s^2 + G c_s^2 psi^2 / 2 = rho / 3 + G psi^2 / 6,
psi = 1 - exp(-rho).  dp is taken between the centre node (n/2, n/2, n/2) and the far corner;
the radius is the volume-equivalent one, R = (3 V / 4 pi)^(1/3) with V = (M - rho_g n^3) /
(rho_l - rho_g) from the measured densities; sigma = dp R / 2.
"""
import math

import numpy as np


def laplace(rho, G, n):
    """(dp, R_eff) of a droplet density field rho (n, n, n)."""
    psi = 1.0 - np.exp(-rho.astype(np.float64))
    p = rho / 3.0 + G * psi ** 2 / 6.0
    c = n // 2
    rl, rg = float(rho[c, c, c]), float(rho[0, 0, 0])
    dp = float(p[c, c, c] - p[0, 0, 0])
    V = (rho.astype(np.float64).sum() - rg * n ** 3) / (rl - rg)
    return dp, (3 * V / (4 * math.pi)) ** (1.0 / 3.0)


def surface_tension(rho, G, n):
    dp, R = laplace(rho, G, n)
    return dp * R / 2.0
