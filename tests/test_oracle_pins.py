"""Pins of the FP64 oracle against what the paper and the mathematics fix (CPU only).

Each test names the passage of arXiv 1905.10182 it checks.  None of them re-types the
oracle's own formula: they use the paper's printed tables (tests/golden/), closed forms,
invariants, textbook special cases and brute force on tiny grids.
"""
import itertools
import math

import numpy as np
import pytest

from golden_util import evaluate, load_table

CS2 = 1.0 / 3.0
W1 = {0: 2.0 / 3.0, 1: 1.0 / 6.0, -1: 1.0 / 6.0}  # D1Q3 weights


def _rand_state(orc, rng, umax=0.1, noise=1e-3):
    rho = rng.uniform(0.8, 1.2)
    u = rng.uniform(-umax, umax, 3)
    f = orc.equilibrium(rho, u) * (1.0 + rng.uniform(-noise, noise, 27) * 30)
    F = rng.uniform(-1e-2, 1e-2, 3)
    return f, F


def _macro(c, f, F):
    rho = f.sum()
    u = (f @ c + 0.5 * np.asarray(F)) / rho
    return rho, u


# --------------------------------------------------------------------------- lattice
def test_velocity_table_matches_paper(orc):
    """Sec. II: the printed D3Q27 velocity list and weights."""
    tab = {}
    for line in open(__import__("golden_util").GOLDEN + "/d3q27_velocities.txt"):
        line = line.split("#", 1)[0].strip()
        if line:
            k, v = line.split("=", 1)
            tab[k.strip()] = v.split()
    c = orc.velocities()
    for a, key in enumerate(("cx", "cy", "cz")):
        assert list(c[:, a]) == [int(s) for s in tab[key]]
    w = orc.weights()
    expect = [float(eval(s)) for s in tab["w"]]
    assert np.allclose(w, expect, rtol=0, atol=1e-16)


def test_weights_are_d1q3_products_and_isotropic(orc):
    """D3Q27 is the tensor product of D1Q3 (App. A); sum w = 1, sum w c c = c_s^2 I."""
    c, w = orc.velocities(), orc.weights()
    for i in range(27):
        assert w[i] == pytest.approx(W1[c[i, 0]] * W1[c[i, 1]] * W1[c[i, 2]], abs=1e-16)
    assert w.sum() == pytest.approx(1.0, abs=1e-15)
    M2 = np.einsum("i,ia,ib->ab", w, c, c)
    assert np.allclose(M2, CS2 * np.eye(3), atol=1e-15)
    assert len({tuple(v) for v in c}) == 27
    for i in range(27):
        j = orc.opposite(i)
        assert (c[j] == -c[i]).all()


def test_hermite_discrete_orthogonality(orc):
    """App. A: the 27 tensor-product Hermite polynomials (<= 2 per axis) are orthogonal under
    the lattice weights with norm nx! ny! nz! c_s^(2n)."""
    w = orc.weights()
    idx = list(itertools.product(range(3), repeat=3))
    H = np.array([[orc.hermite(i, *n) for i in range(27)] for n in idx])
    G = (H * w) @ H.T
    fact = [1, 1, 2]
    norm = np.diag([fact[a] * fact[b] * fact[c] * CS2 ** (a + b + c) for a, b, c in idx])
    assert np.allclose(G, norm, atol=1e-15)


# --------------------------------------------------------------------------- equilibrium
def _psi1d(cc, u):
    """Tensor-product factor of the complete D1Q3 equilibrium: the three populations with
    moments 1, u, u^2 + c_s^2."""
    return 2.0 / 3.0 - u * u if cc == 0 else (1.0 / 6.0 + cc * u / 2.0 + u * u / 2.0)


def test_equilibrium_product_form(orc):
    """Eq. eq:truncation with all 27 tensors factorises into three D1Q3 equilibria."""
    rng = np.random.default_rng(0)
    c = orc.velocities()
    for _ in range(50):
        rho, u = rng.uniform(0.5, 2.0), rng.uniform(-0.4, 0.4, 3)
        feq = orc.equilibrium(rho, u)
        prod = np.array([rho * _psi1d(c[i, 0], u[0]) * _psi1d(c[i, 1], u[1]) * _psi1d(c[i, 2], u[2])
                         for i in range(27)])
        assert np.allclose(feq, prod, rtol=0, atol=2e-15)


def test_equilibrium_raw_moments_are_maxwellian(orc):
    """All 27 raw moments (<= 2 per axis) of the complete equilibrium equal the Maxwellian's:
    prod_a m_a(u_a) with m_0 = 1, m_1 = u, m_2 = u^2 + c_s^2."""
    rng = np.random.default_rng(1)
    c = orc.velocities().astype(float)
    for _ in range(20):
        rho, u = rng.uniform(0.5, 2.0), rng.uniform(-0.3, 0.3, 3)
        feq = orc.equilibrium(rho, u)
        for a, b, d in itertools.product(range(3), repeat=3):
            mom = (feq * c[:, 0] ** a * c[:, 1] ** b * c[:, 2] ** d).sum()
            ex = rho
            for k, p in zip((a, b, d), u):
                ex *= (1.0, p, p * p + CS2)[k]
            assert mom == pytest.approx(ex, abs=3e-15)


def test_second_order_equilibrium_is_textbook(orc):
    """Eq. eq:truncation truncated at H^(2) is the classical second-order equilibrium."""
    rng = np.random.default_rng(2)
    c, w = orc.velocities(), orc.weights()
    for _ in range(20):
        rho, u = rng.uniform(0.5, 2.0), rng.uniform(-0.3, 0.3, 3)
        cu = c @ u
        classic = w * rho * (1 + cu / CS2 + cu ** 2 / (2 * CS2 ** 2) - (u @ u) / (2 * CS2))
        assert np.allclose(orc.equilibrium(rho, u, order=2), classic, atol=1e-15)


def test_equilibrium_central_moments_golden(orc):
    """Eq. equil_central_moments6: only k0, k9, k17, k18, k26 are nonzero."""
    tab = load_table("equilibrium_cms.txt")
    rng = np.random.default_rng(3)
    for _ in range(30):
        rho, u = rng.uniform(0.5, 2.0), rng.uniform(-0.4, 0.4, 3)
        k = orc.central_moments(u, orc.equilibrium(rho, u))
        for j in range(27):
            ex = evaluate(tab[f"k{j}"], rho=rho, cs2=CS2) if f"k{j}" in tab else 0.0
            assert k[j] == pytest.approx(ex, abs=2e-15), j


# --------------------------------------------------------------------------- forcing
def _dpsi1d(cc, u):
    return -2.0 * u if cc == 0 else (cc / 2.0 + u)


def test_forcing_is_force_dot_velocity_gradient_of_equilibrium(orc):
    """Eq. generalForcing/forcing: F_i = F . grad_u (f_i^eq / rho) (force-density reading)."""
    rng = np.random.default_rng(4)
    c = orc.velocities()
    for _ in range(50):
        u, F = rng.uniform(-0.4, 0.4, 3), rng.uniform(-1, 1, 3)
        Fi = orc.forcing_term(F, u)
        ex = np.zeros(27)
        for i in range(27):
            p = [_psi1d(c[i, a], u[a]) for a in range(3)]
            dp = [_dpsi1d(c[i, a], u[a]) for a in range(3)]
            ex[i] = F[0] * dp[0] * p[1] * p[2] + F[1] * p[0] * dp[1] * p[2] + F[2] * p[0] * p[1] * dp[2]
        assert np.allclose(Fi, ex, atol=2e-15)


def test_forcing_moments(orc):
    """sum F_i = 0, sum F_i c = F, sum F_i c c = u F + F u (Eq. macroscopic's F/2 relies on these)."""
    rng = np.random.default_rng(5)
    c = orc.velocities().astype(float)
    for _ in range(20):
        u, F = rng.uniform(-0.3, 0.3, 3), rng.uniform(-1, 1, 3)
        Fi = orc.forcing_term(F, u)
        assert Fi.sum() == pytest.approx(0.0, abs=1e-15)
        assert np.allclose(Fi @ c, F, atol=1e-15)
        assert np.allclose(np.einsum("i,ia,ib->ab", Fi, c, c), np.outer(u, F) + np.outer(F, u), atol=1e-15)


def test_second_order_forcing_is_guo(orc):
    """Sec. II: truncated at H^(2), the forcing term is Guo et al.'s."""
    rng = np.random.default_rng(6)
    c, w = orc.velocities().astype(float), orc.weights()
    for _ in range(20):
        u, F = rng.uniform(-0.3, 0.3, 3), rng.uniform(-1, 1, 3)
        guo = w * (((c - u) / CS2 + np.outer(c @ u, np.ones(3)) * c / CS2 ** 2) @ F)
        assert np.allclose(orc.forcing_term(F, u, order=2), guo, atol=1e-15)


@pytest.mark.parametrize("order", [2, 3, 4, 5, 6])
def test_forcing_central_moments_golden(orc, order):
    """The five printed tables of forcing CMs (Sec. II), truncations H^(2) .. H^(6)."""
    tab = load_table(f"forcing_cms_order{order}.txt")
    rng = np.random.default_rng(10 + order)
    for _ in range(30):
        u, F = rng.uniform(-0.4, 0.4, 3), rng.uniform(-1, 1, 3)
        R = orc.central_moments(u, orc.forcing_term(F, u, order=order))
        env = dict(ux=u[0], uy=u[1], uz=u[2], Fx=F[0], Fy=F[1], Fz=F[2], cs2=CS2)
        for j in range(27):
            ex = evaluate(tab[f"R{j}"], **env) if f"R{j}" in tab else 0.0
            assert R[j] == pytest.approx(ex, abs=3e-15), (order, j)


def test_order3_table_printed_R26_is_garbled(orc):
    """The printed R26 of the H^(3) table does not match T^T F_i; the sign-consistent reading does."""
    tab = load_table("forcing_cms_order3.txt")
    u, F = np.array([0.2, -0.15, 0.3]), np.array([0.4, 0.7, -0.5])
    R = orc.central_moments(u, orc.forcing_term(F, u, order=3))
    env = dict(ux=u[0], uy=u[1], uz=u[2], Fx=F[0], Fy=F[1], Fz=F[2], cs2=CS2)
    assert abs(evaluate(tab["R26_printed"], **env) - R[26]) > 1e-3
    assert R[26] == pytest.approx(evaluate(tab["R26"], **env), abs=1e-15)


# --------------------------------------------------------------------------- basis / inverse
def test_basis_determinant_is_shift_invariant(orc):
    """T(u) = T(0) times a unit-triangular shift of monomials, so det T(u) = det T(0) != 0."""
    d0 = np.linalg.det(orc.basis([0, 0, 0]))
    assert abs(d0) > 1.0
    rng = np.random.default_rng(7)
    for _ in range(10):
        u = rng.uniform(-0.5, 0.5, 3)
        assert np.linalg.det(orc.basis(u)) == pytest.approx(d0, rel=1e-10)


def test_fast_inverse_equals_literal_solve(orc):
    """The fast CM transform cited after Eq. system reproduces (T^T)^-1 k to rounding."""
    rng = np.random.default_rng(8)
    for _ in range(50):
        u, k = rng.uniform(-0.4, 0.4, 3), rng.normal(size=27)
        a, b = orc.inverse_literal(u, k), orc.inverse_fast(u, k)
        assert np.abs(a - b).max() <= 1e-13 * max(1.0, np.abs(k).max())
        assert np.allclose(orc.central_moments(u, a), k, atol=1e-13)


# --------------------------------------------------------------------------- collision
def test_single_rate_literal_collision_is_bgk(orc):
    """Lambda = omega I in the CM collision equals BGK with the same complete f^eq and F_i
    (Eq. collision), for any omega."""
    rng = np.random.default_rng(9)
    for _ in range(20):
        om = rng.uniform(0.3, 1.95)
        lit = orc.Grid(1, 1, 1, omega=om, collision=orc.COLL_LITERAL, lambdas=[om] * 27)
        bgk = orc.Grid(1, 1, 1, omega=om, collision=orc.COLL_BGK)
        f, F = _rand_state(orc, rng)
        assert np.abs(lit.collide(f, F) - bgk.collide(f, F)).max() < 5e-16 * 30


def test_truncated_single_rate_literal_is_textbook_guo_bgk(orc):
    """Models M4/M5 of Sec. III through the literal definition: with Lambda = omega I and both
    expansions cut at H^(2), the CM collision is BGK with the classical second-order equilibrium
    and Guo et al.'s forcing term, both written out here from their textbook forms."""
    rng = np.random.default_rng(31)
    c, w = orc.velocities().astype(float), orc.weights()
    for _ in range(20):
        om = rng.uniform(0.3, 1.95)
        f, F = _rand_state(orc, rng, umax=0.2)
        rho, u = _macro(c, f, F)
        cu = c @ u
        feq2 = w * rho * (1 + 3 * cu + 4.5 * cu ** 2 - 1.5 * (u @ u))
        guo = w * (3 * (c - u) @ F + 9 * cu * (c @ F))
        lit = orc.Grid(1, 1, 1, omega=om, collision=orc.COLL_LITERAL, lambdas=[om] * 27, eq_order=2, force_order=2)
        ex = f + om * (feq2 - f) + (1 - om / 2) * guo
        assert np.abs(lit.collide(f, F) - ex).max() < 1e-14


@pytest.mark.parametrize("orders", [(6, 2), (2, 2), (2, 6)])
def test_truncations_change_only_moments_of_order_three_and_up(orc, orders):
    """With the paper's Lambda, cutting f^eq and/or F_i at H^(2) leaves the post-collision central
    moments k0..k9 (orders <= 2, including the omega-relaxed k4..k8) unchanged: the D3Q27
    quadrature reproduces the second-order moments of every truncation of order >= 2."""
    rng = np.random.default_rng(32)
    c = orc.velocities().astype(float)
    for _ in range(20):
        om = rng.uniform(0.5, 1.99)
        f, F = _rand_state(orc, rng, umax=0.2)
        _, u = _macro(c, f, F)
        full6 = orc.Grid(1, 1, 1, omega=om, collision=orc.COLL_LITERAL).collide(f, F)
        trunc = orc.Grid(1, 1, 1, omega=om, collision=orc.COLL_LITERAL, eq_order=orders[0],
                         force_order=orders[1]).collide(f, F)
        dk = orc.central_moments(u, trunc - full6)
        assert np.abs(dk[:10]).max() < 1e-15
        assert np.abs(dk[10:]).max() > 1e-6


def test_paper_lambda_at_omega_one_is_bgk(orc):
    """Eq. eq:relaxationMatrix at omega = 1 is the identity, so the scheme is BGK at nu = 1/6."""
    rng = np.random.default_rng(10)
    bgk = orc.Grid(1, 1, 1, omega=1.0, collision=orc.COLL_BGK)
    for coll in (orc.COLL_LITERAL, orc.COLL_PAPER):
        g = orc.Grid(1, 1, 1, omega=1.0, collision=coll)
        for _ in range(10):
            f, F = _rand_state(orc, rng)
            assert np.abs(g.collide(f, F) - bgk.collide(f, F)).max() < 1e-14


def test_paper_algorithm_equals_definition(orc):
    """The five-step summary of Sec. II (closed-form k*, fast inverse) equals the literal
    definition k* = (I-L)k + L k^eq + (I-L/2) R, f* = (T^T)^-1 k*."""
    rng = np.random.default_rng(11)
    for _ in range(40):
        om = rng.uniform(0.5, 1.99)
        f, F = _rand_state(orc, rng, umax=0.2)
        a = orc.Grid(1, 1, 1, omega=om, collision=orc.COLL_LITERAL).collide(f, F)
        b = orc.Grid(1, 1, 1, omega=om, collision=orc.COLL_PAPER).collide(f, F)
        assert np.abs(a - b).max() <= 1e-13


def test_post_collision_central_moments_golden(orc):
    """Eq. post_collision_central_moments_forcing: T^T f* (at the pre-collision u) has the
    printed 19 nonzero entries and zeros elsewhere."""
    tab = load_table("post_collision_cms.txt")
    rng = np.random.default_rng(12)
    c = orc.velocities().astype(float)
    for _ in range(20):
        om = rng.uniform(0.5, 1.99)
        f, F = _rand_state(orc, rng, umax=0.2)
        rho, u = _macro(c, f, F)
        k = orc.central_moments(u, f)
        fs = orc.Grid(1, 1, 1, omega=om, collision=orc.COLL_LITERAL).collide(f, F)
        ks = orc.central_moments(u, fs)
        env = dict(rho=rho, Fx=F[0], Fy=F[1], Fz=F[2], cs2=CS2, omega=om,
                   k4=k[4], k5=k[5], k6=k[6], k7=k[7], k8=k[8])
        for j in range(27):
            ex = evaluate(tab[f"k{j}"], **env) if f"k{j}" in tab else 0.0
            assert ks[j] == pytest.approx(ex, abs=1e-14), j


def test_collision_conserves_mass_and_adds_momentum(orc):
    """sum f* = sum f and sum f* c = sum f c + F (from k0* = rho, k1..3* = F/2 with u from
    Eq. macroscopic)."""
    rng = np.random.default_rng(13)
    c = orc.velocities().astype(float)
    for coll in (orc.COLL_LITERAL, orc.COLL_PAPER, orc.COLL_BGK):
        g = orc.Grid(1, 1, 1, omega=1.3, collision=coll)
        for _ in range(10):
            f, F = _rand_state(orc, rng)
            fs = g.collide(f, F)
            assert fs.sum() == pytest.approx(f.sum(), abs=1e-15)
            assert np.allclose(fs @ c, f @ c + F, atol=1e-15)


def test_equilibrium_is_fixed_point_without_force(orc):
    """f = f^eq(rho, u), F = 0: every post-collision CM equals its pre-collision value."""
    rng = np.random.default_rng(14)
    g = orc.Grid(1, 1, 1, omega=1.7, collision=orc.COLL_PAPER)
    for _ in range(10):
        feq = orc.equilibrium(rng.uniform(0.5, 2), rng.uniform(-0.3, 0.3, 3))
        assert np.allclose(g.collide(feq), feq, atol=1e-15)


# --------------------------------------------------------------------------- streaming
def _brute_stream(c, opp, lab, nx, ny, nz, walls_y, mask):
    """Pure-Python Eq. streaming with halfway bounce-back, one step, f* = f."""
    out = lab.copy()
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                if mask is not None and mask[z, y, x]:
                    continue
                for i in range(27):
                    sx, sy, sz = x - c[i, 0], y - c[i, 1], z - c[i, 2]
                    blocked = False
                    if walls_y and not (0 <= sy < ny):
                        blocked = True
                    sx, sy, sz = sx % nx, sy % ny, sz % nz
                    if not blocked and mask is not None and mask[sz, sy, sx]:
                        blocked = True
                    out[i, z, y, x] = lab[opp[i], z, y, x] if blocked else lab[i, sz, sy, sx]
    return out


@pytest.mark.parametrize("walls,use_mask", [(False, False), (True, False), (True, True), (False, True)])
def test_streaming_matches_brute_force(orc, walls, use_mask):
    """Eq. streaming + halfway bounce-back on a ragged 5x4x3 grid, bit-exact labels."""
    nx, ny, nz = 5, 4, 3
    rng = np.random.default_rng(15)
    mask = (rng.random((nz, ny, nx)) < 0.25).astype(np.uint8) if use_mask else None
    c = orc.velocities()
    opp = [orc.opposite(i) for i in range(27)]
    lab = np.arange(27 * nx * ny * nz, dtype=np.float64).reshape(27, nz, ny, nx)
    g = orc.Grid(nx, ny, nz, omega=1.0, collision=orc.COLL_NONE, walls_y=walls, mask=mask)
    got = lab.copy()
    ref = lab.copy()
    for _ in range(3):
        got = g.step(got, 1)
        ref = _brute_stream(c, opp, ref, nx, ny, nz, walls, mask)
        assert np.array_equal(got, ref)


def test_periodic_streaming_returns_after_period(orc):
    """On a periodic L^3 grid, L free-streaming steps are the identity."""
    L = 4
    lab = np.arange(27 * L ** 3, dtype=np.float64).reshape(27, L, L, L)
    g = orc.Grid(L, L, L, omega=1.0, collision=orc.COLL_NONE)
    assert np.array_equal(g.step(lab, L), lab)
    assert not np.array_equal(g.step(lab, 1), lab)


def test_sampled_step_matches_full_step(orc):
    """orc_step_sampled (used for parity at full size) equals orc_step at the sampled nodes."""
    rng = np.random.default_rng(16)
    nx, ny, nz = 6, 5, 4
    mask = (rng.random((nz, ny, nx)) < 0.2).astype(np.uint8)
    for kw in (dict(walls_y=True, mask=mask, force_kind=orc.FORCE_UNIFORM, force=(1e-4, 2e-5, 0)),
               dict(force_kind=orc.FORCE_SHAN_CHEN, G=-5.0)):
        g = orc.Grid(nx, ny, nz, nu=0.1, **kw)
        rho = rng.uniform(0.2, 2.0, (nz, ny, nx))
        f = g.init_equilibrium(rho, rng.uniform(-0.05, 0.05, (3, nz, ny, nx)))
        f *= 1 + rng.uniform(-1e-3, 1e-3, f.shape)
        full = g.step(f, 1).reshape(27, -1)
        nodes = rng.choice(nx * ny * nz, 25, replace=False)
        assert np.allclose(g.step_sampled(f, nodes), full[:, nodes].T, rtol=0, atol=1e-15)


# --------------------------------------------------------------------------- closed forms
def test_kolmogorov_translation_invariance(orc):
    """A y-only force keeps the flow y-only: a 3D grid equals the 1D-reduced run bit for bit."""
    kw = dict(nu=0.05, force_kind=orc.FORCE_KOLMOGOROV, force=(1e-5, 0, 0))
    g3, g1 = orc.Grid(4, 16, 3, **kw), orc.Grid(1, 16, 1, **kw)
    f3 = g3.step(g3.init_equilibrium(1.0, np.zeros((3, 3, 16, 4))), 50)
    f1 = g1.step(g1.init_equilibrium(1.0, np.zeros((3, 1, 16, 1))), 50)
    assert np.array_equal(f3, np.broadcast_to(f1, f3.shape))


def _kolmogorov_profile(orc, N, nu, F0, steps):
    g = orc.Grid(1, N, 1, nu=nu, force_kind=orc.FORCE_KOLMOGOROV, force=(F0, 0, 0))
    f = g.step(g.init_equilibrium(1.0, np.zeros((3, 1, N, 1))), steps)
    rho, u = g.macroscopic(f)
    return u[0, 0, :, 0], u[1, 0, :, 0]


def test_kolmogorov_transient_closed_form(orc):
    """Kolmogorov flow, 32 nodes, nu = 0.05, F0 = 1e-5, 2000 steps: u_x follows
    U0 (1 - exp(-nu k^2 t)) sin(k y), U0 = F0/(nu k^2), within 1e-2 U0."""
    N, nu, F0, t = 32, 0.05, 1e-5, 2000
    ux, uy = _kolmogorov_profile(orc, N, nu, F0, t)
    k = 2 * math.pi / N
    U0 = F0 / (nu * k * k)
    y = np.arange(N)
    ex = U0 * (1 - math.exp(-nu * k * k * t)) * np.sin(k * y)
    assert np.abs(ux - ex).max() <= 1e-2 * U0
    assert np.abs(uy).max() < 1e-6 * U0  # only O(u^2) compressibility effects


def test_kolmogorov_second_order_convergence(orc):
    """Steady Kolmogorov flow converges at second order in the grid spacing (Sec. III A reports
    second order for the forced four-rolls mill)."""
    nu, F0 = 0.05, 1e-5
    errs = []
    for N in (16, 32, 64):
        k = 2 * math.pi / N
        steps = int(12 / (nu * k * k))
        ux, _ = _kolmogorov_profile(orc, N, nu, F0, steps)
        ex = F0 / (nu * k * k) * np.sin(k * np.arange(N))
        errs.append(np.linalg.norm(ux - ex) / np.linalg.norm(ex))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(1.9 < r < 2.1 for r in rates), (errs, rates)


def test_poiseuille_second_order_convergence(orc):
    """Force-driven channel with halfway bounce-back walls (y = -1/2, H - 1/2):
    u_x = F/(2 nu) (y + 1/2)(H - y - 1/2), recovered at second order."""
    nu, F = 0.05, 1e-6
    errs = []
    for H in (8, 16, 32):
        g = orc.Grid(1, H, 1, nu=nu, walls_y=True, force_kind=orc.FORCE_UNIFORM, force=(F, 0, 0))
        steps = int(10 * H * H / (nu * math.pi ** 2))
        f = g.step(g.init_equilibrium(1.0, np.zeros((3, 1, H, 1))), steps)
        _, u = g.macroscopic(f)
        yy = np.arange(H) + 0.5
        ex = F / (2 * nu) * yy * (H - yy)
        errs.append(np.abs(u[0, 0, :, 0] - ex).max() / ex.max())
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert errs[0] < 2e-2 and all(1.8 < r < 2.2 for r in rates), (errs, rates)


def test_shan_chen_force_sine_closed_form(orc):
    """Sec. III static droplet force: for psi(x) = a + b sin(2 pi x/N), sum_i w_i c_i psi(x+c_i)
    = (b/3) sin(2 pi/N) cos(2 pi x/N) e_x, so F_x = -G psi (b/3) sin(2pi/N) cos(2pi x/N)."""
    N, a, b, G = 16, 0.5, 0.2, -5.5
    x = np.arange(N)
    psi = a + b * np.sin(2 * math.pi * x / N)
    rho1 = -np.log(1.0 - psi)
    rho = np.broadcast_to(rho1, (3, 4, N)).copy()
    g = orc.Grid(N, 4, 3, nu=1 / 6, force_kind=orc.FORCE_SHAN_CHEN, G=G)
    f = g.init_equilibrium(rho, np.zeros((3, 3, 4, N)))
    F = g.force_field(f)
    ex = -G * psi * (b / 3) * math.sin(2 * math.pi / N) * np.cos(2 * math.pi * x / N)
    assert np.allclose(F[0], np.broadcast_to(ex, (3, 4, N)), rtol=0, atol=1e-14)
    assert np.abs(F[1]).max() < 1e-14 and np.abs(F[2]).max() < 1e-14


def test_shan_chen_droplet_conserves_mass(orc):
    """Collision conserves mass and periodic streaming moves it: total mass is constant."""
    N = 12
    g = orc.Grid(N, N, N, nu=1 / 6, force_kind=orc.FORCE_SHAN_CHEN, G=-5.5)
    z, y, x = np.meshgrid(*(np.arange(N),) * 3, indexing="ij")
    r = np.sqrt((x - N / 2) ** 2 + (y - N / 2) ** 2 + (z - N / 2) ** 2)
    rho = 0.5 * (2.4 + 0.13) - 0.5 * (2.4 - 0.13) * np.tanh(2 * (r - 3.5) / 2)
    f = g.init_equilibrium(rho, np.zeros((3, N, N, N)))
    m0 = f.sum()
    f = g.step(f, 40)
    assert abs(f.sum() - m0) <= 1e-12 * m0
    assert np.isfinite(f).all()
