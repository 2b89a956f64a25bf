"""z-slab decomposition of one periodic domain (one slab per rank, or several in one process).

The exchange schedule follows lbm_halo_pack / lbm_halo_unpack in include/cmlbm.h: even AA steps are
local; an odd step needs, across each face, the 9 populations that point into the slab before it
(stage 0) and returns the 9 it pushed out after it (stage 1).  A backend is one slab with
  parity() -> 0 | 1,  step(),  pack(face, stage) -> buffer,  unpack(face, stage, buffer);
a ring delivers, for every slab, the buffer its lower neighbour sent up and the one its upper
neighbour sent down.
"""
from __future__ import annotations


class SolverSlab:
    """A GPU slab: a Solver created with slab_z=True (see Solver)."""

    def __init__(self, solver):
        import torch
        self.s = solver
        nbytes = solver.halo_bytes
        self._bufs = {(f, st): torch.empty(nbytes, dtype=torch.uint8, device="cuda") for f in (0, 1) for st in (0, 1)}

    def parity(self):
        return self.s.parity

    def step(self):
        self.s.step(1)

    def pack(self, face, stage):
        b = self._bufs[(face, stage)]
        self.s.halo_pack(face, stage, b)
        return b

    def unpack(self, face, stage, buf):
        self.s.halo_unpack(face, stage, buf)


class LocalRing:
    """All slabs of the domain in one process, bottom to top, periodic."""

    def __init__(self, slabs):
        self.slabs = list(slabs)

    def exchange(self, stage):
        n = len(self.slabs)
        down = [s.pack(0, stage) for s in self.slabs]
        up = [s.pack(1, stage) for s in self.slabs]
        # a slab's upper face receives what the slab above sent down, its lower face what the
        # slab below sent up; copies decouple the send buffers from the receive side
        from_above = [down[(k + 1) % n].clone() if hasattr(down[0], "clone") else down[(k + 1) % n].copy()
                      for k in range(n)]
        from_below = [up[(k - 1) % n].clone() if hasattr(up[0], "clone") else up[(k - 1) % n].copy()
                      for k in range(n)]
        for k, s in enumerate(self.slabs):
            s.unpack(1, stage, from_above[k])
            s.unpack(0, stage, from_below[k])

    def step(self, nsteps=1):
        for _ in range(nsteps):
            odd = self.slabs[0].parity() == 1
            if odd:
                self.exchange(0)
            for s in self.slabs:
                s.step()
            if odd:
                self.exchange(1)


class DistRing:
    """One slab per torch.distributed rank (NCCL with CUDA buffers, gloo with CPU buffers)."""

    def __init__(self, slab, group=None):
        import torch.distributed as dist
        self.slab = slab
        self.dist = dist
        self.group = group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)

    def exchange(self, stage):
        d = self.dist
        down, up = self.slab.pack(0, stage), self.slab.pack(1, stage)
        if self.world == 1:
            self.slab.unpack(1, stage, down.clone())
            self.slab.unpack(0, stage, up.clone())
            return
        below, above = (self.rank - 1) % self.world, (self.rank + 1) % self.world
        from_above, from_below = down.clone(), up.clone()
        g = self.group
        gb = d.get_global_rank(g, below) if g is not None else below
        ga = d.get_global_rank(g, above) if g is not None else above
        ops = [d.P2POp(d.isend, down, gb, g), d.P2POp(d.isend, up, ga, g),
               d.P2POp(d.irecv, from_above, ga, g), d.P2POp(d.irecv, from_below, gb, g)]
        for r in d.batch_isend_irecv(ops):
            r.wait()
        self.slab.unpack(1, stage, from_above)
        self.slab.unpack(0, stage, from_below)

    def step(self, nsteps=1):
        for _ in range(nsteps):
            odd = self.slab.parity() == 1
            if odd:
                self.exchange(0)
            self.slab.step()
            if odd:
                self.exchange(1)
