"""Seeded synthetic inputs shared by the tests and the benchmark.

Only random numbers and the geometric / initial-condition recipes of the workloads live here;
none of the lattice Boltzmann arithmetic does.  The same arrays are fed to the CUDA library and
to the FP64 oracle.
"""
from __future__ import annotations

import math

import numpy as np

MASK64 = (1 << 64) - 1


def splitmix64(state: int):
    """One step of splitmix64 (Steele, Lea & Flood 2014): returns (new_state, 64-bit output)."""
    state = (state + 0x9E3779B97F4A7C15) & MASK64
    z = state
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return state, z ^ (z >> 31)


class SplitMix:
    """Counter-based uniform generator over splitmix64, one stream per seed."""

    def __init__(self, seed: int):
        self.state = (int(seed) * 0x9E3779B97F4A7C15 + 0x632BE59BD9B4E019) & MASK64

    def uniform(self, lo=0.0, hi=1.0) -> float:
        self.state, z = splitmix64(self.state)
        return lo + (hi - lo) * ((z >> 11) * (1.0 / (1 << 53)))

    def integer(self, lo: int, hi: int) -> int:
        """Uniform integer in [lo, hi] inclusive."""
        return lo + int(self.uniform() * (hi - lo + 1)) % (hi - lo + 1)


def random_deviations(nx, ny, nz, seed, amp=1e-3, density=None):
    """Population deviations g (27, nz, ny, nx) float32, uniform in [-amp, amp].  With amp well
    below the smallest lattice weight (1/216) every population stays positive.  density: an
    optional (nz, ny, nx) field; (density - 1)/27 is added to all 27 deviations of a node, which
    shifts its mass by density - 1 without moving its momentum."""
    rng = np.random.default_rng(seed)
    g = rng.uniform(-amp, amp, (27, nz, ny, nx))
    if density is not None:
        g += (np.asarray(density, dtype=np.float64) - 1.0)[None] / 27.0
    return g.astype(np.float32)


def random_deviations_device(nx, ny, nz, seed, amp=1e-3, device="cuda"):
    """Population deviations (27, nz, ny, nx) float32, uniform in [-amp, amp], drawn on the device
    by torch's seeded generator (Philox), for grids too large to build on the host (512^3: 14.5 GB).
    The numbers differ from random_deviations with the same seed."""
    import torch
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    g = torch.empty((27, nz, ny, nx), dtype=torch.float32, device=device)
    g.uniform_(-amp, amp, generator=gen)
    return g


def random_force_field(nx, ny, nz, seed, amp=1e-4):
    rng = np.random.default_rng(seed + 7919)
    return rng.uniform(-amp, amp, (3, nz, ny, nx)).astype(np.float32)


def random_mask(nx, ny, nz, seed, fraction=0.2):
    rng = np.random.default_rng(seed + 104729)
    return (rng.random((nz, ny, nx)) < fraction).astype(np.uint8)


def droplet_density(n, radius, rho_l=2.4, rho_g=0.13, width=2.0, center=None):
    """Static-droplet initial density (nz, ny, nx): a tanh profile of the given interface width
    around a sphere of the given radius centred at node (n/2, n/2, n/2) of a periodic n^3 box."""
    c = n / 2 if center is None else center
    ax = np.arange(n, dtype=np.float64)
    z, y, x = np.meshgrid(ax, ax, ax, indexing="ij")
    r = np.sqrt((x - c) ** 2 + (y - c) ** 2 + (z - c) ** 2)
    rho = 0.5 * (rho_l + rho_g) - 0.5 * (rho_l - rho_g) * np.tanh(2.0 * (r - radius) / width)
    return rho.astype(np.float32)


def taylor_green(n, u0, rho0=1.0):
    """Standard 3D Taylor-Green vortex on a periodic n^3 box with x = 2 pi i / n:
    u = u0 sin x cos y cos z, v = -u0 cos x sin y cos z, w = 0, and the matching pressure
    p - p0 = rho0 u0^2 / 16 (cos 2x + cos 2y)(cos 2z + 2) turned into density with c_s^2 = 1/3.
    Returns rho, ux, uy, uz, each (n, n, n) float32 indexed [z, y, x].  The factors are
    separable, so they are formed per axis and broadcast (a 512^3 box needs no FP64 meshgrid)."""
    k = 2.0 * math.pi / n
    a = np.arange(n, dtype=np.float64) * k
    x, y, z = a[None, None, :], a[None, :, None], a[:, None, None]
    ux = (u0 * np.sin(x) * np.cos(y) * np.cos(z)).astype(np.float32)
    uy = (-u0 * np.cos(x) * np.sin(y) * np.cos(z)).astype(np.float32)
    uz = np.zeros((n, n, n), dtype=np.float32)
    p = rho0 * u0 * u0 / 16.0 * (np.cos(2 * x) + np.cos(2 * y)) * (np.cos(2 * z) + 2.0)
    rho = (rho0 + 3.0 * p).astype(np.float32)
    return rho, ux, uy, uz


def orszag_tang(n, u0=0.0203, b0=0.0203):
    """Initial velocity and magnetic field of the three-dimensional Orszag-Tang vortex on a periodic
    2 pi box of n^3 nodes (x = 2 pi i / n), as printed in Sec. III:
    u = u0 (2 sin y, 2 sin x, 0), b = 0.8 b0 (-2 sin 2y + sin z, 2 sin x + sin z, sin x + sin y).
    Returns u, b, each (3, n, n, n) float32 indexed [component, z, y, x]."""
    ax = 2.0 * math.pi * np.arange(n, dtype=np.float64) / n
    z, y, x = np.meshgrid(ax, ax, ax, indexing="ij")
    u = u0 * np.stack([2.0 * np.sin(y), 2.0 * np.sin(x), np.zeros_like(x)])
    b = 0.8 * b0 * np.stack([-2.0 * np.sin(2.0 * y) + np.sin(z), 2.0 * np.sin(x) + np.sin(z), np.sin(x) + np.sin(y)])
    return u.astype(np.float32), b.astype(np.float32)


def sphere_pack(nx, ny, nz, seed, phi_max=0.2, rmin=3, rmax=8, max_tries=2000):
    """Random non-overlapping spheres (radii uniform in [rmin, rmax], centres uniform, rejection
    on overlap) added until the solid fraction reaches a target drawn uniformly in [0, phi_max].
    Returns (mask uint8 (nz, ny, nx), target fraction).  Periodic in x and z; sphere centres keep
    a radius away from the y walls."""
    rng = SplitMix(seed)
    target = rng.uniform(0.0, phi_max)
    mask = np.zeros((nz, ny, nx), dtype=np.uint8)
    spheres = []
    solid = 0
    total = nx * ny * nz
    tries = 0
    while solid < target * total and tries < max_tries:
        tries += 1
        r = rng.integer(rmin, rmax)
        cx, cy, cz = rng.uniform(0, nx), rng.uniform(r, max(r, ny - r)), rng.uniform(0, nz)
        ok = True
        for (sx, sy, sz, sr) in spheres:
            dx = min(abs(cx - sx), nx - abs(cx - sx))
            dz = min(abs(cz - sz), nz - abs(cz - sz))
            if dx * dx + (cy - sy) ** 2 + dz * dz < (r + sr) ** 2:
                ok = False
                break
        if not ok:
            continue
        spheres.append((cx, cy, cz, r))
        # nodes of the bounding box, with periodic wrap in x and z
        xs = np.arange(int(math.floor(cx - r)), int(math.ceil(cx + r)) + 1)
        ys = np.arange(max(0, int(math.floor(cy - r))), min(ny - 1, int(math.ceil(cy + r))) + 1)
        zs = np.arange(int(math.floor(cz - r)), int(math.ceil(cz + r)) + 1)
        Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
        inside = (X - cx) ** 2 + (Y - cy) ** 2 + (Z - cz) ** 2 <= r * r
        zi, yi, xi = Z[inside] % nz, Y[inside], X[inside] % nx
        before = int(mask[zi, yi, xi].sum())
        mask[zi, yi, xi] = 1
        solid += int(mask[zi, yi, xi].sum()) - before
    return mask, target


def porous_channel(seed, size_lo=(32, 32, 32), size_hi=(96, 48, 96)):
    """One forced porous channel: size nx, nz ~ U{32..96}, ny ~ U{32..48}; walls in y; sphere
    pack obstacles with solid fraction up to 0.2; nu ~ U[0.01, 0.1]; F_x ~ U[1e-6, 1e-5]."""
    rng = SplitMix(1_000_003 + seed)
    nx = rng.integer(size_lo[0], size_hi[0])
    ny = rng.integer(size_lo[1], size_hi[1])
    nz = rng.integer(size_lo[2], size_hi[2])
    nu = rng.uniform(0.01, 0.1)
    fx = rng.uniform(1e-6, 1e-5)
    mask, phi = sphere_pack(nx, ny, nz, seed)
    return dict(nx=nx, ny=ny, nz=nz, nu=nu, fx=fx, mask=mask, phi_target=phi, seed=seed)


def porous_cube(seed, n=64, nu_range=(0.01, 0.1)):
    """A forced porous channel on an n^3 grid for the learned warm start: walls in y, sphere-pack
    obstacles (solid fraction target U[0, 0.2]), nu ~ U[nu_range] (default [0.01, 0.1]),
    F_x ~ U[1e-6, 1e-5]."""
    rng = SplitMix(2_000_003 + seed)
    nu = rng.uniform(*nu_range)
    fx = rng.uniform(1e-6, 1e-5)
    mask, phi = sphere_pack(n, n, n, 7_000_001 + seed)
    return dict(nx=n, ny=n, nz=n, nu=nu, fx=fx, mask=mask, phi_target=phi, seed=seed)
