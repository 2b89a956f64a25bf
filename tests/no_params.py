"""Seeded host-side parameters for the neural-operator tests, so that the oracle and the GPU start
from the same numbers and none of them comes from the library's own initialiser.

Distribution per block (the usual fan-in scaling): the lift P and the 1x1 maps Wc, Q uniform in
+-1/sqrt(fan_in); the mode matrices uniform in [0, 1/W^2) (a positive mean, so the spectral path
carries signal through all layers); biases uniform in +-0.1.
"""
import numpy as np


def host_params(layout, W, seed):
    lay, n = layout
    rng = np.random.default_rng(seed)
    theta = np.empty(n, dtype=np.float32)
    for name, (off, shp) in lay.items():
        cnt = int(np.prod(shp))
        if name.startswith("Wm"):
            v = rng.uniform(0.0, 1.0 / (W * W), cnt)
        elif name in ("P", "Q") or name.startswith("Wc"):
            fan_in = shp[1]
            v = rng.uniform(-1.0, 1.0, cnt) / np.sqrt(fan_in)
        else:
            v = rng.uniform(-0.1, 0.1, cnt)
        theta[off:off + cnt] = v
    return theta
