"""Guard bands around the population store: a caller-owned store (lbm_desc.store) sits between two
bands of a known byte pattern; after steps of both AA parities on every kernel path (one node or
two nodes per thread, walls and masks, the Shan-Chen stencil, the M5 variant) no band byte may have
changed.  An out-of-range write of any stream-collide kernel lands in a band."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1905_10182_gb300 import Solver, inputs  # noqa: E402
from paper_1905_10182_gb300._native import LbmDesc, lib  # noqa: E402

GUARD = 1 << 16  # bytes on each side, a multiple of 256
PATTERN = 0xA5

CASES = [
    ("fp32", (19, 13, 11), {}, None),
    ("fp16", (66, 5, 4), {}, None),                      # two nodes per thread
    ("bf16", (20, 13, 11), {}, ("shan_chen", (-5.5,))),  # pair kernel with the psi stencil
    ("fp16", (19, 5, 4), {}, None),                      # one node per thread (odd nx)
    ("fp32", (19, 13, 11), {"walls_y": True, "mask": True}, ("uniform", (1e-4, 0, 0))),
    ("fp16", (19, 13, 11), {"walls_y": True}, ("uniform", (1e-4, 0, 0))),
    ("fp32", (20, 12, 10), {}, ("field", None)),
]


@pytest.mark.parametrize("storage,shape,kw,force", CASES)
def test_store_guard_bands_untouched(storage, shape, kw, force):
    nx, ny, nz = shape
    kw = dict(kw)
    if kw.pop("mask", False):
        kw["mask"] = inputs.random_mask(nx, ny, nz, seed=7, fraction=0.15)
    d = LbmDesc()
    d.nx, d.ny, d.nz = nx, ny, nz
    d.storage = {"fp32": 0, "fp16": 1, "bf16": 2}[storage]
    nbytes = lib().lbm_store_bytes(ctypes.byref(d))
    buf = torch.full((nbytes + 2 * GUARD,), PATTERN, dtype=torch.uint8, device="cuda")
    s = Solver(nx, ny, nz, nu=0.08, storage=storage, store=buf[GUARD:GUARD + nbytes], **kw)
    if force:
        if force[0] == "field":
            F = inputs.random_force_field(nx, ny, nz, seed=3)
            s.set_force("field", None, F[0], F[1], F[2])
        else:
            s.set_force(*force)
    s.set_populations(inputs.random_deviations(nx, ny, nz, seed=9))
    s.step(5)
    if storage == "fp32" and not kw:
        s.set_hermite_orders(2, 2)
        s.step(3)
    s.synchronize()
    bands = torch.cat([buf[:GUARD], buf[GUARD + nbytes:]]).cpu().numpy()
    assert np.all(bands == PATTERN), np.flatnonzero(bands != PATTERN)[:10]
