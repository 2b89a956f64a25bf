"""z-slab exchange schedule (paper_1905_10182_gb300.slabs) on CPU: slabs of an AA store stepped
with the oracle's collision, in one process and as two gloo ranks, must reproduce the oracle's
unsplit two-array run bit for bit."""
import os
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")

HERE = os.path.dirname(os.path.abspath(__file__))
NX, NY, NZ, NU, FORCE = 3, 2, 5, 0.05, (2e-4, -1e-4, 3e-4)


def _initial(orc):
    rng = np.random.default_rng(5)
    w = orc.weights()[:, None, None, None]
    return w + rng.uniform(-1e-3, 1e-3, (27, NZ, NY, NX))


def _reference(orc, f0, steps, walls=False):
    g = orc.Grid(NX, NY, NZ, nu=NU, collision=orc.COLL_PAPER, force_kind=orc.FORCE_UNIFORM, force=FORCE,
                 walls_y=walls)
    return g.step(f0, steps)


@pytest.mark.parametrize("heights,walls", [((5,), False), ((2, 3), False), ((1, 3, 1), False), ((2, 3), True),
                                           ((5,), True)])
def test_local_ring_matches_unsplit(orc, heights, walls):
    from aa_slab_cpu import AASlabCPU
    from paper_1905_10182_gb300.slabs import LocalRing
    f0 = _initial(orc)
    slabs, z = [], 0
    for h in heights:
        slabs.append(AASlabCPU(orc, f0[:, z:z + h], NU, FORCE, walls_y=walls))
        z += h
    LocalRing(slabs).step(4)
    got = np.concatenate([s.natural() for s in slabs], axis=1)
    assert np.array_equal(got, _reference(orc, f0, 4, walls))


def _rank_main(rank, world, port, out):
    sys.path.insert(0, HERE)
    sys.path.insert(0, os.path.dirname(HERE))
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    from aa_slab_cpu import AASlabCPU
    from paper_1905_10182_gb300.slabs import DistRing
    f0 = _initial(oracle)
    bounds = [0, 2, NZ]
    slab = AASlabCPU(oracle, f0[:, bounds[rank]:bounds[rank + 1]], NU, FORCE, walls_y=True)
    DistRing(slab).step(4)
    np.save(os.path.join(out, f"slab{rank}.npy"), slab.natural())
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_match_unsplit(orc, tmp_path):
    import socket
    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    got = np.concatenate([np.load(tmp_path / f"slab{r}.npy") for r in range(2)], axis=1)
    assert np.array_equal(got, _reference(orc, _initial(orc), 4, walls=True))
