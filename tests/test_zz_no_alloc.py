"""The allocation-free diagnostics entry point (lbm_reduce_fields_noalloc), checked against lbm_stats.

Some callers cannot let a library call cudaMalloc while they run: a framework whose caching
allocator owns the device's memory budget, or a stepping loop that cannot afford the implicit
device synchronisation of an allocation.  For them the library offers one reduction that keeps its
scratch in a fixed device array.  This test calls it through the C ABI, twice in a row, and
compares it with lbm_stats on the same state (same FP64 reduction order, so the results agree to
rounding of the final sums).
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1905_10182_gb300 import Solver, inputs  # noqa: E402
from paper_1905_10182_gb300 import _native as nat  # noqa: E402

KEYS = ("mass", "mom_x", "mom_y", "mom_z", "residual", "kinetic_energy", "enstrophy", "umax", "fluid_nodes")


def _noalloc(nx, ny, nz, walls, mask_d, rho, u, uprev):
    out = (ctypes.c_double * (nat.LBM_STATS_LEN - 1))()
    st = nat.lib().lbm_reduce_fields_noalloc(
        nx, ny, nz, int(walls), nat.ptr(mask_d), nat.ptr(rho), nat.ptr(u[0]), nat.ptr(u[1]), nat.ptr(u[2]),
        nat.ptr(uprev) if uprev is not None else None, out, torch.cuda.current_stream().cuda_stream)
    assert st == nat.LBM_OK, nat.status_name(st)
    return list(out)


def _compare(stats, got):
    for k, v in zip(KEYS, got):
        ref = stats[k]
        assert v == pytest.approx(ref, rel=1e-12, abs=1e-300), (k, v, ref)


def test_noalloc_reduction_matches_lbm_stats_on_two_calls():
    nx, ny, nz = 40, 24, 18
    mask = inputs.random_mask(nx, ny, nz, seed=21, fraction=0.1)
    s = Solver(nx, ny, nz, nu=0.05, walls_y=True, mask=mask)
    s.set_force("uniform", (2e-4, 0.0, 1e-4))
    s.set_populations(inputs.random_deviations(nx, ny, nz, seed=22))
    mask_d = torch.from_numpy(mask).cuda()
    rho = torch.empty((nz, ny, nx), device="cuda")
    u1 = torch.empty((3, nz, ny, nx), device="cuda")
    u2 = torch.empty((3, nz, ny, nx), device="cuda")

    st1 = s.stats()
    s.macroscopic(rho, u1[0], u1[1], u1[2])
    got1 = _noalloc(nx, ny, nz, True, mask_d, rho, u1, None)
    _compare(st1, got1)
    assert got1[4] == pytest.approx(1.0)

    s.step(5)
    st2 = s.stats()
    s.macroscopic(rho, u2[0], u2[1], u2[2])
    got2 = _noalloc(nx, ny, nz, True, mask_d, rho, u2, u1)
    _compare(st2, got2)
    assert got2[4] > 0.0
    assert got2[8] == float((mask == 0).sum())


def test_noalloc_rejects_bad_sizes():
    out = (ctypes.c_double * (nat.LBM_STATS_LEN - 1))()
    L = nat.lib()
    assert L.lbm_reduce_fields_noalloc(0, 4, 4, 0, None, None, None, None, None, None, out, None) == nat.LBM_ERR_ARG
    assert L.lbm_reduce_fields_noalloc(2048, 2048, 1024, 0, None, None, None, None, None, None, out,
                                       None) == nat.LBM_ERR_ARG
