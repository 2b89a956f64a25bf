"""Parity at the full sizes and launch configurations of the benchmark workloads, on sampled nodes.

The store of a 512^3 grid (27 x 134 M values, 14.5 GB in FP32) cannot be stepped by the oracle as a
whole, so the check is local (tests/sampled_boxes.py): for each sampled node the initial
populations of the periodic box that determines it after s steps are gathered on the device (torch
indexing of the input tensor, never a whole-store host copy), the oracle steps all boxes at once,
and the centre of each box is compared element by element with the GPU's populations at that
node (read back with lbm_get_populations into a device tensor).

Bound per step, as in the small-grid parity tests: |g_gpu - g_oracle| <= 64 eps32 S plus half an
ulp of the stored format for 16-bit storage, S = max(|g|, |u|, |F|) over the boxes; s steps: s
times that.

What this covers beyond the small grids: the 64-bit element offsets of the single-domain kernels
(27 N > 2^32 at 512^3), the L2 prefetch (on when the store exceeds L2), the two-nodes-per-thread
16-bit kernel and its psi pass on the real row length and grid, both AA parities.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1905_10182_gb300 import Solver, inputs  # noqa: E402
from sampled_boxes import box_indices, oracle_centres, sample_nodes  # noqa: E402

EPS32 = 2.0 ** -24
C_STEP = 64.0


def storage_round(g, storage):
    """Round FP32 deviations to the stored precision (round to nearest even), as the codec does."""
    g = np.asarray(g, dtype=np.float32)
    if storage == "fp16":
        return g.astype(np.float16).astype(np.float32)
    if storage == "bf16":
        b = g.view(np.uint32).astype(np.uint64)
        b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
        return b.astype(np.uint32).view(np.float32)
    return g


def half_ulp(m, storage):
    if storage == "fp32":
        return 0.0
    e = math.floor(math.log2(max(m, 1e-30)))
    return 2.0 ** (e - (10 if storage == "fp16" else 7)) / 2.0


def gather(t, idx):
    """Values of a device tensor (27, nz, ny, nx) at flat node indices idx (any shape) -> host
    float32 array (27,) + idx.shape."""
    flat = t.reshape(27, -1)
    it = torch.from_numpy(np.ascontiguousarray(idx.reshape(-1))).to(device=t.device, dtype=torch.int64)
    return flat[:, it].cpu().numpy().reshape((27,) + idx.shape)


def check_sampled(orc, s, g0, storage, okw, reach, steps_list, nodes, label):
    """Step the solver through steps_list (cumulative step counts from the state g0) and compare
    each time with the oracle on the boxes of the sampled nodes."""
    shape = tuple(g0.shape[1:])
    w = orc.weights()
    out = torch.empty_like(g0)
    done = 0
    for steps in steps_list:
        s.step(steps - done)
        done = steps
        s.get_populations(out)
        got = gather(out, nodes).T.astype(np.float64)  # (K, 27)
        r = reach * steps
        idx = box_indices(nodes, shape, r)
        g_box = storage_round(gather(g0, idx), storage).astype(np.float64)
        ref, S = oracle_centres(orc, g_box + w[:, None, None, None, None], r, steps, okw)
        ref -= w[None, :]
        err = np.abs(got - ref).max()
        tol = steps * (C_STEP * EPS32 * S + half_ulp(np.abs(ref).max(), storage))
        print(f"{label} {storage} step {steps}: max |g - g_oracle| = {err:.3e} (bound {tol:.3e}, S = {S:.3e}, "
              f"{len(nodes)} nodes)")
        assert err <= tol, (label, storage, steps, err, tol)
    del out


@pytest.fixture
def free_device_memory():
    yield
    torch.cuda.synchronize()
    torch.cuda.empty_cache()


@pytest.mark.parametrize("storage", ["fp32", "fp16", "bf16"])
def test_taylor_green_512_sampled(orc, storage, free_device_memory):
    """512^3 periodic grid at nu = 1e-4 (the Taylor-Green workload's grid, viscosity and launch
    path): one and two steps from a seeded random state (deviations up to 4e-3, so every population
    stays positive), checked at about 3000 sampled nodes."""
    n = 512
    g0 = inputs.random_deviations_device(n, n, n, seed=512, amp=4e-3)
    s = Solver(n, n, n, nu=1e-4, storage=storage)
    s.set_populations(g0)
    nodes = sample_nodes((n, n, n), 3000, seed=513)
    check_sampled(orc, s, g0, storage, dict(nu=1e-4), 1, (1, 2), nodes, "taylor-green 512^3")
    s.close()
    del g0


@pytest.mark.parametrize("storage", ["fp32", "fp16", "bf16"])
def test_droplet_128_sampled(orc, storage, free_device_memory):
    """The Shan-Chen droplet workload at 128^3 (G = -5.5, nu = 1/6, psi pass + stencil in the
    collide kernel): one and two steps from the droplet density plus seeded deviations, checked at
    about 3000 sampled nodes."""
    N = 128
    rho = inputs.droplet_density(N, radius=24)
    g = inputs.random_deviations(N, N, N, seed=9, density=rho)
    g0 = torch.from_numpy(g).cuda()
    s = Solver(N, N, N, nu=1 / 6, storage=storage)
    s.set_force("shan_chen", (-5.5,))
    s.set_populations(g0)
    nodes = sample_nodes((N, N, N), 3000, seed=10)
    okw = dict(nu=1 / 6, force_kind=orc.FORCE_SHAN_CHEN, G=-5.5)
    check_sampled(orc, s, g0, storage, okw, 2, (1, 2), nodes, "droplet 128^3")
    s.close()
