"""The magnetic field of App. C on the GPU (lbm_set_magnetic: D3Q7 vector populations in one fused
kernel with the D3Q27 central-moment fluid) against the FP64 oracle and closed forms.

Bound per step, as for the fluid alone: |x_gpu - x_oracle| <= 64 eps32 S for every fluid
deviation and magnetic population x, S = max(|g|, |u|, |F|, |h|) of the state; n steps: n times.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1905_10182_gb300 import Solver, inputs  # noqa: E402
from paper_1905_10182_gb300._native import LbmError  # noqa: E402

EPS32 = 2.0 ** -24
C_STEP = 64.0
RAGGED = (19, 13, 11)


def _state(orc, shape, seed, walls=False):
    """Moving fluid (|u| ~ 0.05) and magnetic populations h^eq(b, u) + noise, |b| ~ 0.1."""
    nx, ny, nz = shape
    rng = np.random.default_rng(seed)
    rho = 1.0 + 0.05 * (rng.random((nz, ny, nx)) - 0.5)
    u = 0.05 * (2 * rng.random((3, nz, ny, nx)) - 1)
    f = orc.Grid(nx, ny, nz, nu=0.1).init_equilibrium(rho, u)
    g = (f - orc.weights()[:, None, None, None] + inputs.random_deviations(nx, ny, nz, seed=seed + 1))
    b = 0.1 * (2 * rng.random((3, nz, ny, nx)) - 1)
    h = orc.MhdGrid(nx, ny, nz, nu=0.1, eta=0.05).mhd_init(b, u) + 1e-3 * rng.uniform(-1, 1, (21, nz, ny, nx))
    return g.astype(np.float32), h.astype(np.float32)


def _bound(orc, g, h, og):
    f = g.astype(np.float64) + orc.weights()[:, None, None, None]
    _, u, _, j = og.mhd_fields(f, h.astype(np.float64))
    b = h.astype(np.float64).reshape(7, 3, *h.shape[1:]).sum(axis=0)
    F = np.cross(j, b, axis=0)
    S = max(np.abs(g).max(), np.abs(u).max(), np.abs(F).max(), np.abs(h).max())
    return C_STEP * EPS32 * S


@pytest.mark.parametrize("walls", [False, True])
def test_coupled_steps_match_oracle(orc, walls):
    nx, ny, nz = RAGGED
    g, h = _state(orc, RAGGED, seed=81)
    bw = (0.02, 0.1, -0.03) if walls else (0.0, 0.0, 0.0)
    F = (2e-4, -1e-4, 5e-5)
    s = Solver(nx, ny, nz, nu=0.07, walls_y=walls)
    s.set_force("uniform", F)
    s.set_magnetic(0.04, b_wall=bw)
    s.set_populations(g)
    s.set_magnetic_populations(h)
    og = orc.MhdGrid(nx, ny, nz, nu=0.07, eta=0.04, b_wall=bw, walls_y=walls, collision=orc.COLL_PAPER,
                     force_kind=orc.FORCE_UNIFORM, force=F)
    f = g.astype(np.float64) + orc.weights()[:, None, None, None]
    hh = h.astype(np.float64)
    tol1 = _bound(orc, g, h, og)
    for n in (1, 2, 3):
        s.step(1)
        f, hh = og.mhd_step(f, hh, 1)
        eg = np.abs(s.get_populations().astype(np.float64) - (f - orc.weights()[:, None, None, None])).max()
        eh = np.abs(s.get_magnetic_populations().astype(np.float64) - hh).max()
        assert eg <= n * tol1 and eh <= n * tol1, (walls, n, eg, eh, tol1)
    # fields through lbm_macroscopic / lbm_magnetic (u includes (F + j x b)/2)
    rho_o, u_o, b_o, j_o = og.mhd_fields(f, hh)
    _, ux, uy, uz = s.macroscopic()
    b, j = s.magnetic()
    assert np.abs(np.stack([ux, uy, uz]) - u_o).max() <= 8 * tol1
    assert np.abs(b - b_o).max() <= 8 * tol1
    # j is a difference of O(b) populations times 4 omega_m
    assert np.abs(j - j_o).max() <= 8 * tol1 * 4 * og.omega_m * 4


def _hartmann_gpu(H, Ha=3.0, nu=0.1, eta=0.1, F=1e-6):
    a = H / 2
    B0 = Ha * math.sqrt(nu * eta) / a
    s = Solver(1, H, 1, nu=nu, walls_y=True)
    s.set_force("uniform", (F, 0.0, 0.0))
    s.set_magnetic(eta, b=(0.0, B0, 0.0), b_wall=(0.0, B0, 0.0))
    s.step(int(10 * H * H / nu))
    _, ux, _, _ = s.macroscopic()
    sc = (np.arange(H) - (H - 1) / 2) / a
    ex = F * a * a / (nu * Ha * math.tanh(Ha)) * (1 - np.cosh(Ha * sc) / math.cosh(Ha))
    return np.linalg.norm(ux[0, :, 0] - ex) / np.linalg.norm(ex)


def test_hartmann_flow_second_order():
    """Sec. III, Hartmann flow (periodic in x, driven by a uniform force): the GPU's steady profile
    converges at second order to the closed form, like the oracle's (tests/test_mhd_oracle_pins.py)."""
    e = [_hartmann_gpu(H) for H in (8, 16, 32)]
    rates = [math.log2(e[i] / e[i + 1]) for i in range(2)]
    print(f"GPU Hartmann errors {e}, rates {rates}")
    assert all(abs(r - 2) < 0.2 for r in rates) and e[-1] < 3e-3, (e, rates)


def test_orszag_tang_100_steps_match_oracle(orc):
    n, steps = 24, 100
    u, b = inputs.orszag_tang(n)
    nu = eta = 0.02
    s = Solver(n, n, n, nu=nu)
    rho = np.ones((n, n, n), np.float32)
    s.set_state(rho, *u)
    s.set_magnetic(eta, b=b)
    og = orc.MhdGrid(n, n, n, nu=nu, eta=eta, collision=orc.COLL_PAPER)
    g0 = s.get_populations()
    h0 = s.get_magnetic_populations()
    # the GPU's initial state (f^eq(rho, u), h^eq(b, u) in FP32) against the oracle's own
    f = og.init_equilibrium(rho.astype(np.float64), u.astype(np.float64))
    h = og.mhd_init(b.astype(np.float64), u.astype(np.float64))
    tol1 = _bound(orc, g0, h0, og)
    assert np.abs(g0 - (f - orc.weights()[:, None, None, None])).max() <= tol1
    assert np.abs(h0 - h).max() <= tol1
    f = g0.astype(np.float64) + orc.weights()[:, None, None, None]  # both continue from the same state
    h = h0.astype(np.float64)
    s.step(steps)
    f, h = og.mhd_step(f, h, steps)
    eg = np.abs(s.get_populations().astype(np.float64) - (f - orc.weights()[:, None, None, None])).max()
    eh = np.abs(s.get_magnetic_populations().astype(np.float64) - h).max()
    _, _, _, j_o = og.mhd_fields(f, h)
    _, j = s.magnetic()
    jmax_o, jmax = np.sqrt((j_o ** 2).sum(0)).max(), np.sqrt((j.astype(np.float64) ** 2).sum(0)).max()
    print(f"Orszag-Tang {n}^3, {steps} steps: max dg {eg:.2e}, max dh {eh:.2e} (bound {steps * tol1:.2e}); "
          f"j_max {jmax:.6e} vs oracle {jmax_o:.6e}")
    assert eg <= steps * tol1 and eh <= steps * tol1
    assert abs(jmax - jmax_o) <= 1e-4 * jmax_o


def test_magnetic_field_rejected_combinations(tmp_path):
    with pytest.raises(LbmError):
        Solver(8, 8, 8, nu=0.1, storage="fp16").set_magnetic(0.05)
    with pytest.raises(LbmError):
        Solver(8, 8, 8, nu=0.1, mask=np.zeros((8, 8, 8), np.uint8)).set_magnetic(0.05)
    s = Solver(8, 8, 8, nu=0.1)
    s.set_magnetic(0.05)
    with pytest.raises(LbmError):
        s.save(tmp_path / "c.bin")
    with pytest.raises(LbmError):
        s.set_force("kolmogorov", (1e-5,))
        s.step(1)


def test_orszag_tang_128_full_domain_matches_oracle(orc):
    """The magnetic step at the size and parameters of the Orszag-Tang benchmark (128^3 periodic,
    nu = eta = 0.005, the fused kernel the bench times), from a seeded non-equilibrium state with
    |u| ~ 0.05 and |b| ~ 0.1: every fluid deviation and magnetic population of the whole domain
    against the oracle after 1 and 2 steps, at the per-step bound."""
    n = 128
    g, h = _state(orc, (n, n, n), seed=91)
    s = Solver(n, n, n, nu=0.005)
    s.set_magnetic(0.005)
    s.set_populations(g)
    s.set_magnetic_populations(h)
    og = orc.MhdGrid(n, n, n, nu=0.005, eta=0.005, collision=orc.COLL_PAPER)
    w = orc.weights()[:, None, None, None]
    f = g.astype(np.float64) + w
    hh = h.astype(np.float64)
    tol1 = _bound(orc, g, h, og)
    for k in (1, 2):
        s.step(1)
        f, hh = og.mhd_step(f, hh, 1)
        eg = np.abs(s.get_populations().astype(np.float64) - (f - w)).max()
        eh = np.abs(s.get_magnetic_populations().astype(np.float64) - hh).max()
        print(f"Orszag-Tang grid 128^3 step {k}: fluid {eg:.3e}, magnetic {eh:.3e} (bound {k * tol1:.3e})")
        assert eg <= k * tol1 and eh <= k * tol1, (k, eg, eh, tol1)
    s.close()
