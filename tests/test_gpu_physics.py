"""Physics of the benchmark configurations on the GPU path (through the C ABI).

* Four-rolls mill (Sec. III A, run in 2D with nz = 1): the paper's convergence study, N = 8 .. 256 at
  u0 = 1e-3 and 1e-2, second order against the closed form (the paper reports a rate of 1.998,
  tests/golden/four_rolls_mill.txt); one step of the same 2D field-force case against the oracle.
* Static droplet with the Shan-Chen force (Sec. III, static droplet): Laplace's law dp = 2 sigma / R
  at 128^3 for R = 16, 24, 32, and the surface tension against the FP64 oracle's at 64^3.
* Decaying Taylor-Green vortex: the kinetic-energy decay rate equals -2 nu x enstrophy (energy
  equation of periodic incompressible flow), both taken from the FP64 diagnostics of lbm_stats;
  and at low viscosity (nu = 1e-4, 64^3, 5000 steps through the transition) the GPU's kinetic-energy
  and enstrophy curves follow the FP64 oracle's.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from droplet_laplace import surface_tension  # noqa: E402
from golden_util import load_table  # noqa: E402
from paper_1905_10182_gb300 import Solver, inputs  # noqa: E402


def _four_rolls_fields(N, u0):
    """Force field and steady closed form (Eq. tg_vel) of the four-rolls mill on an N x N x 1 grid,
    nu from Re = u0 N / nu = 100."""
    nu = u0 * N / 100.0
    psi = 2 * math.pi / N
    x = np.arange(N)
    X, Y = np.meshgrid(x, x, indexing="xy")  # [y][x]
    Fx = 2 * nu * u0 * psi ** 2 * np.sin(psi * X) * np.sin(psi * Y)
    Fy = 2 * nu * u0 * psi ** 2 * np.cos(psi * X) * np.cos(psi * Y)
    ux_an = u0 * np.sin(psi * X) * np.sin(psi * Y)
    uy_an = u0 * np.cos(psi * X) * np.cos(psi * Y)
    return nu, psi, Fx, Fy, ux_an, uy_an


def _four_rolls_error(N, u0=1e-3):
    """Relative L2 error (Eq. error) of the steady GPU field against Eq. tg_vel.  The run starts
    from f^eq of the closed form and takes 12 e-folding times of the slowest transient."""
    nu, psi, Fx, Fy, ux_an, uy_an = _four_rolls_fields(N, u0)
    s = Solver(N, N, 1, nu=nu)
    z = np.zeros((1, N, N), np.float32)
    s.set_force("field", None, Fx[None].astype(np.float32), Fy[None].astype(np.float32), z)
    s.set_state(np.ones((1, N, N), np.float32), ux_an[None].astype(np.float32), uy_an[None].astype(np.float32), z)
    lam = 2 * nu * psi ** 2  # decay rate of the slowest transient
    s.step(int(12.0 / lam))
    _, ux, uy, _ = s.macroscopic()
    s.close()
    num = np.concatenate([ux[0].ravel(), uy[0].ravel()]).astype(np.float64)
    an = np.concatenate([ux_an.ravel(), uy_an.ravel()])
    return np.linalg.norm(num - an) / np.linalg.norm(an)


FOUR_ROLLS_N = (8, 16, 32, 64, 128, 256)


@pytest.mark.parametrize("u0", [1e-3, 1e-2])
def test_four_rolls_mill_second_order(u0):
    """The convergence study of Sec. III A: N = 8 .. 256 at Re = 100, u0 = 1e-3 and 1e-2.  The
    least-squares rate over all N is within 0.05 of the paper's 1.998, and every pairwise rate
    within 0.15 of 2 (the paper: M1 keeps a rate of about 2 for each N at both velocities)."""
    paper_rate = float(load_table("four_rolls_mill.txt")["rate"])
    errs = np.array([_four_rolls_error(N, u0) for N in FOUR_ROLLS_N])
    rates = np.log2(errs[:-1] / errs[1:])
    slope = -np.polyfit(np.log2(FOUR_ROLLS_N), np.log2(errs), 1)[0]
    print(f"four-rolls mill u0={u0}: errors {errs.tolist()}, pairwise rates {rates.round(4).tolist()}, "
          f"least-squares rate {slope:.4f} (paper: {paper_rate})")
    assert abs(slope - paper_rate) < 0.05, (errs, slope)
    assert np.all(np.abs(rates - 2.0) < 0.15), (errs, rates)


def test_four_rolls_mill_one_step_matches_oracle(orc):
    """One step of the 2D (nz = 1) field-force case against the oracle, from f^eq of the closed
    form plus seeded deviations: the grid and force the convergence study runs."""
    N, u0 = 24, 1e-2
    nu, _, Fx, Fy, ux_an, uy_an = _four_rolls_fields(N, u0)
    F = np.stack([Fx, Fy, np.zeros_like(Fx)])[:, None].astype(np.float32)  # (3, 1, N, N)
    u = np.stack([ux_an, uy_an, np.zeros_like(ux_an)])[:, None]
    og = orc.Grid(N, N, 1, nu=nu, collision=orc.COLL_PAPER, force_kind=orc.FORCE_FIELD, field=F.astype(np.float64))
    w = orc.weights()[:, None, None, None]
    g = (og.init_equilibrium(1.0, u) - w + inputs.random_deviations(N, N, 1, seed=77, amp=1e-4)).astype(np.float32)
    s = Solver(N, N, 1, nu=nu)
    s.set_force("field", None, F[0], F[1], F[2])
    s.set_populations(g)
    f0 = g.astype(np.float64) + w
    S = max(np.abs(g).max(), u0, np.abs(F).max())
    for n in (1, 2):
        s.step(1)
        ref = og.step(f0, n) - w
        err = np.abs(s.get_populations().astype(np.float64) - ref).max()
        assert err <= n * 64 * 2.0 ** -24 * S, (n, err)
    s.close()


def _gpu_sigma(n, R, G=-5.5, steps=20000):
    s = Solver(n, n, n, nu=1 / 6)
    s.set_force("shan_chen", (G,))
    z = np.zeros((n, n, n), np.float32)
    s.set_state(inputs.droplet_density(n, R), z, z, z)
    s.step(steps)
    rho, *_ = s.macroscopic()
    s.close()
    return surface_tension(rho, G, n)


def test_droplet_laplace_law_and_oracle_surface_tension():
    """Laplace's law on the GPU at 128^3 (R = 16, 24, 32, 20000 steps: dp R constant), and the
    surface tension against the FP64 oracle at 64^3 (R = 8, 12, 16; stored by
    tests/golden/make_droplet_sigma.py after 5000 steps, with the 3000-step values showing it has
    settled).  On the same 64^3 runs the GPU agrees with the oracle to 5e-5 relative per radius
    (measured 1.1e-5 to 1.2e-5: FP32 storage against FP64, the same scheme).  Across resolutions
    the measured sigma rises with R at both sizes (the interface keeps its width of about two
    nodes while the curvature falls: 64^3 R = 8..16 gives 0.0595..0.0605, 128^3 R = 16..32 gives
    0.0614..0.0619), so the 128^3 mean lies 2.6 % above the 64^3 mean; the bound is 5 %."""
    G = -5.5
    gold = load_table("droplet_sigma_oracle64.txt")
    so = np.array([float(gold[f"sigma_R{R}_s5000"]) for R in (8, 12, 16)])
    so3 = np.array([float(gold[f"sigma_R{R}_s3000"]) for R in (8, 12, 16)])
    assert np.all(np.abs(so - so3) <= 1e-3 * np.abs(so)), (so, so3)
    g64 = np.array([_gpu_sigma(64, R, G, 5000) for R in (8, 12, 16)])
    d64 = np.abs(g64 - so) / np.abs(so)
    sig = np.array([_gpu_sigma(128, R, G) for R in (16, 24, 32)])
    d128 = abs(sig.mean() - so.mean()) / so.mean()
    print(f"surface tension: GPU 128^3 {sig}, GPU 64^3 {g64}, oracle 64^3 {so}; "
          f"GPU 64^3 vs oracle per radius {d64}, GPU 128^3 mean vs oracle 64^3 mean {d128:.3e}")
    assert sig.std() / sig.mean() < 0.05  # dp R constant: Laplace's law
    assert np.all(d64 <= 5e-5), d64
    assert d128 <= 0.05, d128


def test_taylor_green_energy_decay_rate():
    n, u0, nu = 64, 0.05, 0.005
    rho, ux, uy, uz = inputs.taylor_green(n, u0)
    s = Solver(n, n, n, nu=nu)
    s.set_state(rho, ux, uy, uz)
    s.step(200)
    d = 20
    e0 = s.stats()["kinetic_energy"]
    s.step(d)
    st = s.stats()
    s.step(d)
    e2 = s.stats()["kinetic_energy"]
    rate = (e2 - e0) / (2 * d)
    expect = -2.0 * nu * st["enstrophy"]
    print(f"TGV dE/dt = {rate:.6e}, -2 nu Omega = {expect:.6e}")
    assert rate == pytest.approx(expect, rel=0.03)


def test_taylor_green_low_viscosity_curves_match_oracle(orc):
    """64^3, U0 = 0.05, nu = 1e-4: the vortex goes through its transition (enstrophy grows sixfold,
    then decays) within 5000 steps. Both curves, sampled every 250 steps, stay within 1e-4 relative
    of the FP64 oracle's (measured 2.3e-6 for the energy and 5.9e-6 for the enstrophy): the FP32
    rounding differences are amplified by the flow's instability, while a wrong term (a viscosity
    off by 1 %, a dropped second-order term) moves the enstrophy by percents."""
    n, u0, nu, steps, every = 64, 0.05, 1e-4, 5000, 250
    rho, ux, uy, uz = inputs.taylor_green(n, u0)
    s = Solver(n, n, n, nu=nu)
    s.set_state(rho, ux, uy, uz)
    g = orc.Grid(n, n, n, nu=nu, collision=orc.COLL_PAPER)
    f = g.init_equilibrium(rho.astype(np.float64), np.stack([ux, uy, uz]).astype(np.float64))
    ke, ens = [], []
    for k in range(0, steps + 1, every):
        if k:
            s.step(every)
            f = g.step(f, every)
        st = s.stats()
        _, u = g.macroscopic(f)
        ke.append((st["kinetic_energy"], orc.kinetic_energy(u)))
        ens.append((st["enstrophy"], orc.enstrophy(u)))
    ke, ens = np.array(ke), np.array(ens)
    dke = np.max(np.abs(ke[:, 0] - ke[:, 1]) / ke[:, 1])
    dens = np.max(np.abs(ens[:, 0] - ens[:, 1]) / ens[:, 1])
    print(f"TGV 64^3 nu=1e-4, {steps} steps: max rel. dev. from the oracle: energy {dke:.3e}, "
          f"enstrophy {dens:.3e}; enstrophy peak {ens[:, 1].max() / ens[0, 1]:.2f}x the initial")
    assert ens[:, 1].max() > 4 * ens[0, 1] and ke[-1, 1] < 0.1 * ke[0, 1]
    assert dke <= 1e-4 and dens <= 1e-4
