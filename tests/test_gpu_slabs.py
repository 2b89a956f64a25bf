"""z-slab decomposition on one GPU: slabs exchanging halos through device buffers reproduce the
single-domain run bit for bit (same per-node arithmetic, same stream order of every slot)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1905_10182_gb300 import Solver, inputs  # noqa: E402
from paper_1905_10182_gb300.slabs import LocalRing, SolverSlab  # noqa: E402


@pytest.mark.parametrize("heights,walls,storage,nx", [
    ((12,), False, "fp32", 21), ((5, 7), False, "fp32", 21), ((3, 3, 4, 2), True, "fp32", 21), ((6, 6), True, "fp32", 21),
    ((5, 7), False, "fp16", 20), ((3, 3, 4, 2), False, "bf16", 66)])  # 16-bit, even nx: two nodes per thread
def test_slabs_match_single_domain(heights, walls, storage, nx):
    ny, nz = 10, sum(heights)
    g = inputs.random_deviations(nx, ny, nz, seed=51)
    ref = Solver(nx, ny, nz, nu=0.04, walls_y=walls, storage=storage)
    ref.set_force("uniform", (1e-4, 0.0, -5e-5))
    ref.set_populations(g)
    ref.step(8)
    slabs, z = [], 0
    for h in heights:
        s = Solver(nx, ny, h, nu=0.04, walls_y=walls, slab_z=True, storage=storage)
        s.set_force("uniform", (1e-4, 0.0, -5e-5))
        s.set_populations(g[:, z:z + h])
        slabs.append(s)
        z += h
    LocalRing([SolverSlab(s) for s in slabs]).step(8)
    got = np.concatenate([s.get_populations() for s in slabs], axis=1)
    assert np.array_equal(got, ref.get_populations())
    # the slabs' FP64 mass adds up to the domain's
    assert sum(s.stats()["mass"] for s in slabs) == pytest.approx(ref.stats()["mass"], rel=1e-12)
