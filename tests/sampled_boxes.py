"""Local oracle evaluation at sampled nodes of grids too large for the oracle as a whole.

After s steps a node's populations depend only on the state inside the periodic box of radius r
around it: r = s without a force stencil, r = 2 s with the Shan-Chen force (streaming reaches one
node per step, the 26-neighbour psi stencil one more).  The boxes of all sampled nodes are laid
side by side along x into one oracle grid; after s oracle steps the centre of each box holds the
node's populations.  A box's edge nodes see the neighbouring box through the periodic wrap, but
nothing from there reaches the centre within s steps.  tests/test_sampled_boxes_cpu.py pins this
against the oracle's whole-grid step.
"""
import numpy as np


def sample_nodes(shape, count, seed):
    """count random nodes plus the corners and the row ends (x = 0, 1, nx-2, nx-1) of random rows:
    the wrapped first pair (nx-1, 0) of the 16-bit kernel's odd step and the last planes of the
    store, where the element offsets are largest."""
    nz, ny, nx = shape
    rng = np.random.default_rng(seed)
    N = nx * ny * nz
    picks = [rng.choice(N, min(count, N), replace=False)]
    for z in (0, nz - 1):
        for y in (0, ny - 1):
            for x in (0, nx - 1):
                picks.append(np.array([(z * ny + y) * nx + x]))
    rows = rng.integers(0, ny * nz, 16)
    for x in sorted({0, min(1, nx - 1), max(nx - 2, 0), nx - 1}):
        picks.append(rows * nx + x)
    return np.unique(np.concatenate(picks))


def box_indices(nodes, shape, r):
    """Flat node indices of the periodic (2r+1)^3 box around each node, shaped (K, m, m, m) as
    [node][lz][ly][lx]."""
    nz, ny, nx = shape
    x, y, z = nodes % nx, (nodes // nx) % ny, nodes // (nx * ny)
    o = np.arange(-r, r + 1)
    Z = (z[:, None, None, None] + o[None, :, None, None]) % nz
    Y = (y[:, None, None, None] + o[None, None, :, None]) % ny
    X = (x[:, None, None, None] + o[None, None, None, :]) % nx
    return (Z * ny + Y) * nx + X


def oracle_centres(orc, f_boxes, r, steps, okw):
    """f_boxes: full populations (27, K, m, m, m), m = 2r + 1.  Returns the populations at the
    centre of each box after `steps` oracle steps, shaped (K, 27), and the scale
    S = max(|g|, |u|, |F|) of the initial state (g = f - w, the deviations)."""
    m = 2 * r + 1
    K = f_boxes.shape[1]
    f = np.ascontiguousarray(f_boxes.transpose(0, 2, 3, 1, 4).reshape(27, m, m, K * m))
    og = orc.Grid(K * m, m, m, collision=orc.COLL_PAPER, **okw)
    rho = f.sum(axis=0)
    c = orc.velocities().astype(float)
    u = np.einsum("ia,izyx->azyx", c, f) / rho
    S = max(np.abs(f - orc.weights()[:, None, None, None]).max(), np.abs(u).max())
    if okw.get("force_kind") == orc.FORCE_SHAN_CHEN:
        S = max(S, np.abs(og.force_field(f)).max())
    out = og.step(f, steps)
    return np.ascontiguousarray(out[:, r, r, r::m].T), S
