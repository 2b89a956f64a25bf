"""Batched solver (lbm_batch_*): uneven domains advanced by one persistent launch per step.

Each batch domain must evolve exactly as the same domain run alone (same per-node arithmetic), and
match the FP64 oracle within the per-step bound of test_gpu_parity; run-to-steady retires converged
domains; the autotuner returns a valid shape and leaves the batch at rest.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1905_10182_gb300 import BatchSolver, Solver, inputs  # noqa: E402

EPS32 = 2.0 ** -24


def _domains():
    rng = np.random.default_rng(31)
    doms = []
    for k, (nx, ny, nz) in enumerate([(19, 13, 11), (32, 16, 8), (7, 21, 5), (40, 9, 13), (16, 16, 16)]):
        mask = inputs.random_mask(nx, ny, nz, seed=40 + k, fraction=0.12) if k % 2 == 0 else None
        doms.append(dict(nx=nx, ny=ny, nz=nz, nu=float(rng.uniform(0.02, 0.15)),
                         force=(float(rng.uniform(1e-5, 1e-4)), 0.0, float(rng.uniform(-1e-5, 1e-5))),
                         walls_y=bool(k != 4), mask=mask))
    return doms


def test_batch_domains_match_single_domain_runs():
    doms = _domains()
    b = BatchSolver(doms)
    b.step(7)
    for k, d in enumerate(doms):
        s = Solver(d["nx"], d["ny"], d["nz"], nu=d["nu"], walls_y=d["walls_y"], mask=d["mask"])
        s.set_force("uniform", d["force"])
        s.step(7)
        assert np.array_equal(b.get_populations(k), s.get_populations()), k


def test_batch_domain_matches_oracle(orc):
    doms = _domains()
    b = BatchSolver(doms)
    for k in (0, 3):
        d = doms[k]
        rho = np.ones((d["nz"], d["ny"], d["nx"]), np.float32) * 1.02
        u = np.zeros((3,) + rho.shape, np.float32)
        u[0] = 0.01
        b.set_state(k, rho, u[0], u[1], u[2])
    b.step(3)
    for k in (0, 3):
        d = doms[k]
        og = orc.Grid(d["nx"], d["ny"], d["nz"], nu=d["nu"], walls_y=d["walls_y"], mask=d["mask"],
                      collision=orc.COLL_PAPER, force_kind=orc.FORCE_UNIFORM, force=d["force"])
        rho = np.full((d["nz"], d["ny"], d["nx"]), 1.02)
        u = np.zeros((3,) + rho.shape)
        u[0] = 0.01
        f = og.step(og.init_equilibrium(rho.astype(np.float32).astype(np.float64),
                                        u.astype(np.float32).astype(np.float64)), 3)
        ref = f - orc.weights()[:, None, None, None]
        fluid = np.ones(rho.shape, bool) if d["mask"] is None else d["mask"] == 0
        err = np.abs(b.get_populations(k) - ref)[:, fluid].max()
        assert err <= 3 * 64 * EPS32 * 0.05, (k, err)


def test_batch_run_to_steady_retires_domains():
    """Clean channels of three heights: each reaches residual 1e-8 and retires; the steady profile
    is the halfway-bounce-back Poiseuille parabola to second-order accuracy."""
    doms = [dict(nx=4, ny=H, nz=4, nu=0.1, force=(1e-6, 0, 0), walls_y=True) for H in (8, 12, 16)]
    b = BatchSolver(doms)
    steps, res, status = b.run(tol=1e-8, max_steps=40000, check_every=100)
    assert (status == 0).all(), (steps, res, status)
    assert steps[0] < steps[1] < steps[2]  # wider channels relax more slowly (rate nu (pi/H)^2)
    assert b.active == 0
    for k, H in enumerate((8, 12, 16)):
        _, ux, _, _ = b.macroscopic(k)
        y = np.arange(H) + 0.5
        ex = 1e-6 / (2 * 0.1) * y * (H - y)
        err = np.abs(ux[0, :, 0] - ex).max() / ex.max()
        assert err < 3.0 / H ** 2, (H, err)


def test_batch_autotune_resets_to_rest():
    doms = _domains()
    b = BatchSolver(doms)
    out = b.autotune(trial_steps=4)
    # blocks_per_sm = 0: one block per tile
    assert out["tile"] in (64, 128, 256) and out["blocks_per_sm"] >= 0 and out["mlups"] > 0
    assert b.time == 0
    for k in range(len(doms)):
        assert np.abs(b.get_populations(k)).max() == 0.0
    b.step(7)  # results after tuning equal the default shape's results
    s = Solver(doms[1]["nx"], doms[1]["ny"], doms[1]["nz"], nu=doms[1]["nu"], walls_y=doms[1]["walls_y"])
    s.set_force("uniform", doms[1]["force"])
    s.step(7)
    assert np.array_equal(b.get_populations(1), s.get_populations())


@pytest.mark.parametrize("shape", [(64, 0, "strided"), (128, 2, "strided"), (128, 1, "contiguous"),
                                   (256, 4, "contiguous"), (64, 8, "strided_prefetch"), (128, 1, "strided_prefetch")])
def test_batch_launch_shapes_bit_identical(shape):
    """Every launch shape and schedule (strided, contiguous runs or strided with L2 prefetch) gives the same
    populations, bit for bit, as the single-domain solver."""
    doms = _domains()
    b = BatchSolver(doms)
    b.set_shape(*shape)
    b.step(9)
    for k, d in enumerate(doms):
        s = Solver(d["nx"], d["ny"], d["nz"], nu=d["nu"], walls_y=d["walls_y"], mask=d["mask"])
        s.set_force("uniform", d["force"])
        s.step(9)
        assert np.array_equal(b.get_populations(k), s.get_populations()), (shape, k)


@pytest.mark.parametrize("shape", [(64, 8, "strided_prefetch"), None], ids=["bench-shape", "autotuned"])
def test_full_batch_512_channels_match_oracle(orc, shape):
    """The batched step at the full size of the porous-channel benchmark: all 512 channels
    (inputs.porous_channel seeds 0..511, 85.8 M nodes) in one batch with the bench's launch shape
    (or the autotuner's), 16 of them (spread over the tile list, the largest included) started from
    f^eq of seeded (rho, u) fields and compared, every fluid node and population, with the
    oracle's whole-domain steps after 1 and 2 steps (both AA parities), at the per-step bound
    64 eps32 S of the single-domain parity tests."""
    chans = [inputs.porous_channel(sd) for sd in range(512)]
    doms = [dict(nx=c["nx"], ny=c["ny"], nz=c["nz"], nu=c["nu"], force=(c["fx"], 0.0, 0.0), walls_y=True,
                 mask=c["mask"]) for c in chans]
    sizes = np.array([c["nx"] * c["ny"] * c["nz"] for c in chans])
    pick = sorted(set(np.linspace(0, 511, 15).astype(int).tolist() + [int(np.argmax(sizes))]))
    b = BatchSolver(doms)
    if shape is None:
        b.autotune(trial_steps=4)
    else:
        b.set_shape(*shape)
    rng = np.random.default_rng(77)
    start = {}
    for k in pick:
        d = doms[k]
        shp = (d["nz"], d["ny"], d["nx"])
        rho = (1.0 + 0.02 * (rng.random(shp) - 0.5)).astype(np.float32)
        u = (0.04 * (rng.random((3,) + shp) - 0.5)).astype(np.float32)
        b.set_state(k, rho, u[0], u[1], u[2])
        start[k] = (rho, u)
    for n in (1, 2):
        b.step(1)
        for k in pick:
            d = doms[k]
            og = orc.Grid(d["nx"], d["ny"], d["nz"], nu=d["nu"], walls_y=True, mask=d["mask"],
                          collision=orc.COLL_PAPER, force_kind=orc.FORCE_UNIFORM, force=d["force"])
            rho, u = start[k]
            f0 = og.init_equilibrium(rho.astype(np.float64), u.astype(np.float64))
            ref = og.step(f0, n) - orc.weights()[:, None, None, None]
            fluid = d["mask"] == 0
            g0 = f0 - orc.weights()[:, None, None, None]
            S = max(np.abs(g0).max(), 0.02, abs(d["force"][0]))
            err = np.abs(b.get_populations(k) - ref)[:, fluid].max()
            assert err <= n * 64 * EPS32 * S, (k, n, err)
    b.close()
