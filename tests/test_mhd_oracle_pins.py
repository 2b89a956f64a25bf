"""Pins of the oracle's magnetic-field LBM (App. C: D3Q7 vector populations, Lorentz force j x b)
against what the mathematics and closed forms fix, independent of the oracle's own code:

* the D3Q7 lattice: weights 1/4, 1/8 with sum_l w_l xi_l xi_l = 1/4 I (c_s = 1/2, App. C);
* the equilibrium of App. C has zeroth moment b, electric tensor u b - b u and second moment
  b / 4 (delta), the properties the induction equation rests on;
* the coupled node solve satisfies its defining implicit relations (rho u = sum f c + (F_ext +
  j x b)/2 with j = -(omega_m / c_s^2)(E - 2 u x b)), for random states;
* collision and streaming conserve the total magnetic flux sum_x b exactly on a periodic box;
* a resistive mode b_z = B sin(kx) decays as exp(-eta k^2 t), eta = c_s^2 (1/omega_m - 1/2),
  converging at second order in the grid spacing;
* Hartmann flow (Sec. III: two-dimensional Hartmann flow, periodic in x, driven by a uniform
  force): the steady u_x(y) and induced b_x(y) converge at second order to the closed form
  u = F a^2 / (rho nu Ha tanh Ha) [1 - cosh(Ha y'/a) / cosh Ha], a = L_y / 2,
  Ha = b_y0 a / sqrt(rho nu eta) (the paper's Ha = b_y0 L_y / sqrt(4 rho0 nu eta)).
"""
import math

import numpy as np
import pytest


def test_d3q7_lattice(orc):
    xi, w = orc.mhd_velocities(), orc.mhd_weights()
    assert xi.tolist() == [[0, 0, 0], [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]]
    assert w.sum() == pytest.approx(1.0, abs=1e-15)
    assert np.allclose(np.einsum("l,la,lb->ab", w, xi, xi), 0.25 * np.eye(3), atol=1e-15)
    assert np.allclose(w @ xi, 0.0)


def test_magnetic_equilibrium_moments(orc):
    rng = np.random.default_rng(71)
    xi = orc.mhd_velocities().astype(float)
    for _ in range(20):
        b, u = rng.uniform(-0.3, 0.3, 3), rng.uniform(-0.2, 0.2, 3)
        heq = orc.mhd_equilibrium(b, u)  # (7, 3): [l][alpha]
        assert np.allclose(heq.sum(axis=0), b, atol=1e-15)
        L = np.einsum("lb,la->ba", xi, heq)
        assert np.allclose(L, np.outer(u, b) - np.outer(b, u), atol=1e-15)
        M2 = np.einsum("lb,lc,la->bca", xi, xi, heq)
        assert np.allclose(M2, 0.25 * np.einsum("bc,a->bca", np.eye(3), b), atol=1e-15)


def test_coupled_node_solve_satisfies_its_relations(orc):
    rng = np.random.default_rng(72)
    c = orc.velocities().astype(float)
    xi = orc.mhd_velocities().astype(float)
    for _ in range(30):
        om = rng.uniform(0.6, 1.9)
        rho0 = rng.uniform(0.8, 1.2)
        f = orc.equilibrium(rho0, rng.uniform(-0.1, 0.1, 3)) * (1 + 0.05 * rng.uniform(-1, 1, 27))
        h = orc.mhd_equilibrium(rng.uniform(-0.2, 0.2, 3), rng.uniform(-0.1, 0.1, 3)) + \
            0.01 * rng.uniform(-1, 1, (7, 3))
        Fext = rng.uniform(-1e-3, 1e-3, 3)
        rho, u, FL, j = orc.mhd_node(f, h, Fext, om)
        b = h.sum(axis=0)
        L = np.einsum("lb,la->ba", xi, h)
        E = np.array([L[1, 2] - L[2, 1], L[2, 0] - L[0, 2], L[0, 1] - L[1, 0]])
        assert rho == pytest.approx(f.sum(), abs=1e-15)
        assert np.allclose(j, -(om / 0.25) * (E - 2.0 * np.cross(u, b)), atol=1e-14)
        assert np.allclose(FL, np.cross(j, b), atol=1e-15)
        assert np.allclose(rho * u, f @ c + 0.5 * (Fext + FL), atol=1e-15)


def test_magnetic_flux_conserved(orc):
    n = 8
    rng = np.random.default_rng(73)
    g = orc.MhdGrid(n, n, n, nu=0.05, eta=0.02, collision=orc.COLL_PAPER)
    f = g.init_equilibrium(1 + 0.02 * rng.uniform(-1, 1, (n, n, n)), 0.05 * rng.uniform(-1, 1, (3, n, n, n)))
    h = g.mhd_init(0.1 * rng.uniform(-1, 1, (3, n, n, n)), np.zeros(3))
    flux0 = h.reshape(7, 3, -1).sum(axis=(0, 2))
    f, h = g.mhd_step(f, h, 20)
    assert np.allclose(h.reshape(7, 3, -1).sum(axis=(0, 2)), flux0, rtol=0, atol=1e-12)


def _diffusion_error(orc, N, eta=0.05, B=1e-4):
    k = 2 * math.pi / N
    g = orc.MhdGrid(N, 1, 1, nu=0.1, eta=eta, collision=orc.COLL_PAPER)
    x = np.arange(N)
    b = np.zeros((3, 1, 1, N))
    b[2, 0, 0] = B * np.sin(k * x)
    f = g.init_equilibrium(np.ones((1, 1, N)), np.zeros((3, 1, 1, N)))
    h = g.mhd_init(b, np.zeros(3))
    T = int(0.5 / (eta * k * k))
    f, h = g.mhd_step(f, h, T)
    _, _, bb, _ = g.mhd_fields(f, h)
    amp = 2 * np.mean(bb[2, 0, 0] * np.sin(k * x))
    return abs(amp / (B * math.exp(-eta * k * k * T)) - 1)


def test_resistive_decay_second_order(orc):
    errs = [_diffusion_error(orc, N) for N in (16, 32, 64)]
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert errs[-1] < 2e-3 and all(abs(r - 2) < 0.2 for r in rates), (errs, rates)


def hartmann_closed_form(H, F, nu, eta, Ha):
    """u_x(y), b_x(y) at nodes y = 0..H-1 between halfway walls (y' measured from the centre)."""
    a = H / 2
    B0 = Ha * math.sqrt(nu * eta) / a
    s = (np.arange(H) - (H - 1) / 2) / a
    u = F * a * a / (nu * Ha * math.tanh(Ha)) * (1 - np.cosh(Ha * s) / math.cosh(Ha))
    bx = F * a / B0 * (np.sinh(Ha * s) / math.sinh(Ha) - s)
    return u, bx, B0


def _hartmann_errors(orc, H, Ha=3.0, nu=0.1, eta=0.1, F=1e-6):
    u_ex, bx_ex, B0 = hartmann_closed_form(H, F, nu, eta, Ha)
    g = orc.MhdGrid(1, H, 1, nu=nu, eta=eta, walls_y=True, b_wall=(0, B0, 0), collision=orc.COLL_PAPER,
                    force_kind=orc.FORCE_UNIFORM, force=(F, 0, 0))
    f = g.init_equilibrium(np.ones((1, H, 1)), np.zeros((3, 1, H, 1)))
    h = g.mhd_init(np.array([0.0, B0, 0.0]), np.zeros(3))
    f, h = g.mhd_step(f, h, int(10 * H * H / nu))
    _, u, b, _ = g.mhd_fields(f, h)
    eu = np.linalg.norm(u[0, 0, :, 0] - u_ex) / np.linalg.norm(u_ex)
    eb = np.linalg.norm(b[0, 0, :, 0] - bx_ex) / np.linalg.norm(bx_ex)
    return eu, eb


def test_hartmann_flow_second_order(orc):
    e = [_hartmann_errors(orc, H) for H in (8, 16, 32)]
    for k in range(2):  # u_x, b_x
        rates = [math.log2(e[i][k] / e[i + 1][k]) for i in range(2)]
        assert all(abs(r - 2) < 0.15 for r in rates), (k, e, rates)
    assert e[-1][0] < 3e-3
