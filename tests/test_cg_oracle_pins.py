"""Pins of the oracle's colour-gradient model (App. D) against what the mathematics fixes:

* phi_i(alpha) sums to one, equals the D3Q27 weights at alpha = 8/27 and gives the printed
  equation of state p = rho 9 (1 - alpha) / 19 as its second moment;
* the enhanced equilibrium has mass rho and momentum rho u for any density gradient, and (with no
  gradient) the momentum flux rho [9 (1 - alpha)/19 I + u u];
* the perturbation operator (with the squared projection) conserves mass and momentum and its
  second moment is the surface stress (A/9)|grad phi| (n n - I), from the D3Q27 isotropy
  sum_i w_i c c c c = cs^4 (delta delta + 2 sym) and sum_i B_i c c = I/3;
* recolouring keeps each colour's mass, the total populations, and is a plain split without a
  phase gradient;
* one fluid only (no blue, equal reference densities, uniform density) reduces the model to the
  paper's central-moment scheme of Sec. II, step for step.
"""
import numpy as np
import pytest


def test_phi_weights_and_equation_of_state(orc):
    c = orc.velocities().astype(float)
    for alpha in (8 / 27, 0.5, 0.765, 0.1):
        ph = orc.cg_phi(alpha)
        assert ph.sum() == pytest.approx(1.0, abs=1e-15)
        assert np.allclose(np.einsum("i,ia,ib->ab", ph, c, c), 9 * (1 - alpha) / 19 * np.eye(3), atol=1e-15)
    assert np.allclose(orc.cg_phi(8 / 27), orc.weights(), atol=1e-16)


def test_enhanced_equilibrium_moments(orc):
    rng = np.random.default_rng(91)
    c = orc.velocities().astype(float)
    for _ in range(20):
        rho, u, alpha, nu = rng.uniform(0.5, 3), rng.uniform(-0.1, 0.1, 3), rng.uniform(0.2, 0.8), rng.uniform(0.01, 0.2)
        g = rng.uniform(-0.1, 0.1, 3)
        feq = orc.cg_equilibrium(rho, u, alpha, nu, g)
        assert feq.sum() == pytest.approx(rho, abs=1e-14)
        assert np.allclose(feq @ c, rho * u, atol=1e-15)
        f0 = orc.cg_equilibrium(rho, u, alpha, nu, (0, 0, 0))
        P = np.einsum("i,ia,ib->ab", f0, c, c)
        assert np.allclose(P, rho * (9 * (1 - alpha) / 19 * np.eye(3) + np.outer(u, u)), atol=1e-14)


def test_perturbation_conserves_and_gives_surface_stress(orc):
    rng = np.random.default_rng(92)
    c = orc.velocities().astype(float)
    for _ in range(20):
        A, gp = rng.uniform(1e-4, 1e-2), rng.uniform(-0.3, 0.3, 3)
        p = orc.cg_perturbation(A, gp)
        assert abs(p.sum()) < 1e-17 and np.allclose(p @ c, 0.0, atol=1e-17)
        gn = np.linalg.norm(gp)
        n = gp / gn
        assert np.allclose(np.einsum("i,ia,ib->ab", p, c, c), A / 9 * gn * (np.outer(n, n) - np.eye(3)), atol=1e-16)
    assert np.abs(orc.cg_perturbation(1e-3, (0, 0, 0))).max() == 0.0


def test_recolouring_keeps_colour_masses(orc):
    rng = np.random.default_rng(93)
    for _ in range(20):
        rr, rb = rng.uniform(0.01, 2, 2)
        fs = orc.cg_equilibrium(rr + rb, rng.uniform(-0.05, 0.05, 3), 0.5, 0.05) + 1e-3 * rng.uniform(-1, 1, 27)
        fs *= (rr + rb) / fs.sum()
        gp = rng.uniform(-0.2, 0.2, 3)
        fr, fb = orc.cg_recolour(0.7, rr, rb, 0.5, gp, fs)
        assert fr.sum() == pytest.approx(rr, abs=1e-14) and fb.sum() == pytest.approx(rb, abs=1e-14)
        assert np.allclose(fr + fb, fs, atol=1e-16)
        fr0, _ = orc.cg_recolour(0.7, rr, rb, 0.5, (0, 0, 0), fs)
        assert np.allclose(fr0, rr / (rr + rb) * fs, atol=1e-16)


def test_one_fluid_reduces_to_the_paper_scheme(orc):
    n, nu = 10, 0.07
    rng = np.random.default_rng(94)
    u = 0.05 * rng.uniform(-1, 1, (3, n, n, n))
    cg = orc.CgGrid(n, n, n, rho_r0=1.0, rho_b0=1.0, nu_r=nu, nu_b=nu, A=1e-3, beta=0.7)
    fr, fb = cg.cg_init(np.ones((n, n, n)), np.zeros((n, n, n)), u)
    g = orc.Grid(n, n, n, nu=nu, collision=orc.COLL_PAPER)
    f = g.init_equilibrium(np.ones((n, n, n)), u)
    assert np.allclose(fr, f, atol=1e-16) and np.abs(fb).max() == 0.0
    fr1, fb1 = cg.cg_step(fr, fb, 1)
    f1 = g.step(f, 1)
    assert np.abs(fr1 - f1).max() < 1e-13 and np.abs(fb1).max() == 0.0
