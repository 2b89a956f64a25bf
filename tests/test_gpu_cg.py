"""The colour-gradient two-phase model of App. D on the GPU (lbm_set_colour_gradient) against the
FP64 oracle and against the paper's Rayleigh-Taylor results.

Bound per step: |f^k_gpu - f^k_oracle| <= 128 eps32 S for both colours, S = max(|f|, |u|, |F|)
of the state (full populations are stored, so S is of the order of the density); n steps: n times.
The constant is twice the single-phase one (64, tests/test_gpu_parity.py): the enhanced-equilibrium
terms, of the size of the populations, pass through one more 27-point moment transform before the
inverse, and the recolouring adds another product chain.
"""
import math
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1905_10182_gb300 import Solver, rayleigh_taylor  # noqa: E402
from paper_1905_10182_gb300._native import LbmError  # noqa: E402

EPS32 = 2.0 ** -24
C_STEP = 128.0
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _mixed_state(orc, cg, shape, seed):
    """Both colours present everywhere with O(0.1) order-parameter gradients (well-conditioned
    recolouring directions), small random velocities."""
    nx, ny, nz = shape
    rng = np.random.default_rng(seed)
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    s = np.sin(2 * math.pi * (x / nx + 0.3 * y / ny + 0.2 * z / nz))
    rr = 1.2 * (1.0 + 0.4 * s)
    rb = 0.9 * (1.0 - 0.4 * s)
    u = 0.02 * rng.uniform(-1, 1, (3, nz, ny, nx))
    fr, fb = cg.cg_init(rr, rb, u)
    return fr.astype(np.float32), fb.astype(np.float32)


@pytest.mark.parametrize("walls", [False, True])
def test_two_phase_steps_match_oracle(orc, walls):
    nx, ny, nz = (19, 13, 11)
    prm = dict(rho_r0=1.2, rho_b0=0.9, nu_r=0.05, nu_b=0.12, A=5e-3, beta=0.7, gvec=(1e-4, -2e-4, 5e-5))
    cg = orc.CgGrid(nx, ny, nz, walls_y=walls, **prm)
    fr, fb = _mixed_state(orc, cg, (nx, ny, nz), seed=101)
    s = Solver(nx, ny, nz, nu=prm["nu_r"], walls_y=walls)
    rr0 = fr.astype(np.float64).sum(axis=0)
    rb0 = fb.astype(np.float64).sum(axis=0)
    s.set_colour_gradient(rr0, rb0, rho_r0=prm["rho_r0"], rho_b0=prm["rho_b0"], nu_r=prm["nu_r"], nu_b=prm["nu_b"],
                          A=prm["A"], beta=prm["beta"], g=prm["gvec"])
    s.set_colour_populations(fr, fb)
    f64r, f64b = fr.astype(np.float64), fb.astype(np.float64)
    _, _, u = cg.cg_fields(f64r, f64b)
    S = max(np.abs(f64r + f64b).max(), np.abs(u).max(), 1e-3)
    tol1 = C_STEP * EPS32 * S
    for n in (1, 2, 3):
        s.step(1)
        f64r, f64b = cg.cg_step(f64r, f64b, 1)
        gr, gb = s.get_colour_populations()
        er = np.abs(gr.astype(np.float64) - f64r).max()
        eb = np.abs(gb.astype(np.float64) - f64b).max()
        assert er <= n * tol1 and eb <= n * tol1, (walls, n, er, eb, tol1)
    rr, rb, uo = cg.cg_fields(f64r, f64b)
    grr, grb = s.colour_densities()
    _, ux, uy, uz = s.macroscopic()
    assert np.abs(grr - rr).max() <= 30 * tol1 and np.abs(grb - rb).max() <= 30 * tol1
    assert np.abs(np.stack([ux, uy, uz]) - uo).max() <= 30 * tol1


def test_two_phase_conserves_colour_mass():
    n = 24
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    r = np.sqrt((x - n / 2) ** 2 + (y - n / 2) ** 2 + (z - n / 2) ** 2)
    rr = np.where(r < 6, 1.0, 0.0).astype(np.float32)
    rb = np.where(r < 6, 0.0, 1.0).astype(np.float32)
    s = Solver(n, n, n, nu=0.1)
    s.set_colour_gradient(rr, rb, rho_r0=1.0, rho_b0=1.0, nu_r=0.1, nu_b=0.1, A=1e-3, beta=0.7)
    m0 = [float(a.astype(np.float64).sum()) for a in s.colour_densities()]
    s.step(500)
    m1 = [float(a.astype(np.float64).sum()) for a in s.colour_densities()]
    assert all(abs(a - b) <= 1e-4 * a for a, b in zip(m0, m1)), (m0, m1)


def test_rayleigh_taylor_against_table3():
    """Sec. III, Rayleigh-Taylor instability (W = 64, At = 0.5, Re = 512): the spike and bubble
    positions lie within the range the paper's Table 3 spans over its five methods (present and
    four comparisons, tests/golden/rayleigh_taylor_table3.txt), widened by 0.05 W for the readings
    the paper leaves open (surface-tension amplitude, interface resolution)."""
    tab = np.loadtxt(os.path.join(GOLDEN, "rayleigh_taylor_table3.txt"))
    res = rayleigh_taylor.run(W=64, times=tuple(tab[:, 0]))
    got = np.array([[h["spike"], h["bubble"]] for h in res["history"]])
    spike, bubble = tab[:, 1:6], tab[:, 6:11]
    print("t/t0, spike (ours, present, min..max), bubble (ours, present, min..max):")
    for k in range(len(tab)):
        print(f"  {tab[k, 0]:.1f}  {got[k, 0]:.3f} {spike[k, 0]:.3f} {spike[k].min():.3f}..{spike[k].max():.3f}"
              f"   {got[k, 1]:.3f} {bubble[k, 0]:.3f} {bubble[k].min():.3f}..{bubble[k].max():.3f}")
    assert np.all(np.isfinite(got))
    margin = 0.05
    assert np.all(got[:, 0] >= spike.min(axis=1) - margin) and np.all(got[:, 0] <= spike.max(axis=1) + margin)
    assert np.all(got[:, 1] >= bubble.min(axis=1) - margin) and np.all(got[:, 1] <= bubble.max(axis=1) + margin)


def test_two_phase_rejected_combinations():
    n = 8
    rr, rb = np.ones((n, n, n), np.float32), np.zeros((n, n, n), np.float32)
    kw = dict(rho_r0=1.0, rho_b0=1.0, nu_r=0.1, nu_b=0.1)
    with pytest.raises(LbmError):
        Solver(n, n, n, nu=0.1, storage="fp16").set_colour_gradient(rr, rb, **kw)
    s = Solver(n, n, n, nu=0.1)
    with pytest.raises(LbmError):
        s.set_colour_gradient(rr, rb, rho_r0=1.0, rho_b0=2.0, nu_r=0.1, nu_b=0.1)  # rho_b0 / rho_r0 > 27/19
    s.set_colour_gradient(rr, rb, **kw)
    with pytest.raises(LbmError):
        s.get_populations()
    with pytest.raises(LbmError):
        s.set_magnetic(0.05)


def test_rayleigh_taylor_grid_full_domain_matches_oracle(orc):
    """The two-phase step at the size, parameters and initial state of the Rayleigh-Taylor benchmark
    (64 x 256 x 64, walls in y, heavy fluid rho_h = 3 over light rho_l = 1 with the perturbed
    interface, at rest; nu = 0.005, A = 1e-4, beta = 0.7, g = 0.04^2 / 64): every population of both
    colours of the whole domain against the oracle after 1 and 2 steps, at the per-step bound.

    The state matters.  The recolouring term carries the direction of the order-parameter gradient,
    grad phi / |grad phi|, which is undefined where the gradient vanishes; where |grad phi| is at the
    level of rounding, FP32 and FP64 pick different directions and the colours' split differs by the
    whole recolouring weight (a smooth mixed state on this grid, whose sine has crest planes of zero
    gradient, gave 4e-2 with the colour totals still within 4e-7).  The benchmark's state is well
    conditioned: in the pure phases the gradient is exactly zero on both sides (no recolouring), at
    the interface it is large."""
    W = 64
    nx, ny, nz = W, 4 * W, W
    prm = dict(rho_r0=3.0, rho_b0=1.0, nu_r=0.005, nu_b=0.005, A=1e-4, beta=0.7, gvec=(0.0, -0.04 ** 2 / W, 0.0))
    cg = orc.CgGrid(nx, ny, nz, walls_y=True, **prm)
    rr, rb = rayleigh_taylor.initial_densities(W, prm["rho_r0"], prm["rho_b0"])
    fr, fb = cg.cg_init(rr.astype(np.float64), rb.astype(np.float64))
    fr, fb = fr.astype(np.float32), fb.astype(np.float32)
    s = Solver(nx, ny, nz, nu=prm["nu_r"], walls_y=True)
    s.set_colour_gradient(rr, rb, rho_r0=prm["rho_r0"], rho_b0=prm["rho_b0"], nu_r=prm["nu_r"], nu_b=prm["nu_b"],
                          A=prm["A"], beta=prm["beta"], g=prm["gvec"])
    s.set_colour_populations(fr, fb)
    f64r, f64b = fr.astype(np.float64), fb.astype(np.float64)
    _, _, u = cg.cg_fields(f64r, f64b)
    tol1 = C_STEP * EPS32 * max(np.abs(f64r + f64b).max(), np.abs(u).max(), 1e-3)
    for k in (1, 2):
        s.step(1)
        f64r, f64b = cg.cg_step(f64r, f64b, 1)
        gr, gb = s.get_colour_populations()
        er = np.abs(gr.astype(np.float64) - f64r).max()
        eb = np.abs(gb.astype(np.float64) - f64b).max()
        print(f"Rayleigh-Taylor grid step {k}: red {er:.3e}, blue {eb:.3e} (bound {k * tol1:.3e})")
        assert er <= k * tol1 and eb <= k * tol1, (k, er, eb, tol1)
    s.close()
