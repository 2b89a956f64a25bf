"""The local (box) evaluation used by the full-size GPU parity tests equals the oracle's step of
the whole grid at every sampled node, bit for bit (the same arithmetic on the same inputs)."""
import numpy as np
import pytest

from paper_1905_10182_gb300 import inputs
from sampled_boxes import box_indices, oracle_centres, sample_nodes


@pytest.mark.parametrize("shan_chen", [False, True])
@pytest.mark.parametrize("steps", [1, 2])
def test_boxes_equal_whole_grid(orc, shan_chen, steps):
    nx, ny, nz = 22, 15, 13
    rho = 1.0 + 0.3 * np.random.default_rng(31).random((nz, ny, nx))
    g = inputs.random_deviations(nx, ny, nz, seed=32, amp=4e-3, density=rho).astype(np.float64)
    w = orc.weights()[:, None, None, None]
    okw = dict(nu=0.08)
    if shan_chen:
        okw.update(force_kind=orc.FORCE_SHAN_CHEN, G=-5.5)
    whole = orc.Grid(nx, ny, nz, collision=orc.COLL_PAPER, **okw).step(g + w, steps).reshape(27, -1)
    nodes = sample_nodes((nz, ny, nx), 60, seed=33)
    r = steps * (2 if shan_chen else 1)
    idx = box_indices(nodes, (nz, ny, nx), r)
    boxes = (g + w).reshape(27, -1)[:, idx]
    got, S = oracle_centres(orc, boxes, r, steps, okw)
    assert np.array_equal(got, whole[:, nodes].T)
    assert S > 0
    # a box one node too small does not reproduce the whole-grid step
    small = box_indices(nodes, (nz, ny, nx), r - 1)
    bad, _ = oracle_centres(orc, (g + w).reshape(27, -1)[:, small], r - 1, steps, okw)
    assert not np.allclose(bad, whole[:, nodes].T, rtol=0, atol=1e-12)
