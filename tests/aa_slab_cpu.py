"""CPU test double of one GPU z slab: an AA in-place store with ghost planes, stepped in pure
Python with the oracle's per-node collision.  It exercises the slab exchange schedule of
paper_1905_10182_gb300.slabs on CPU-only machines (single process or gloo ranks)."""
import numpy as np


class AASlabCPU:
    def __init__(self, orc, f_local, nu, force, walls_y=False):
        self.orc = orc
        self.walls = walls_y
        self.c = orc.velocities()
        self.opp = [orc.opposite(i) for i in range(27)]
        self.up = [i for i in range(27) if self.c[i, 2] == 1]
        self.down = [i for i in range(27) if self.c[i, 2] == -1]
        self.g = orc.Grid(1, 1, 1, nu=nu, collision=orc.COLL_PAPER)
        self.F = np.asarray(force, dtype=np.float64)
        q, nz, ny, nx = f_local.shape
        self.nz, self.ny, self.nx = nz, ny, nx
        self.f = np.zeros((27, nz + 2, ny, nx))
        self.f[:, 1:nz + 1] = f_local
        self.par = 0

    def parity(self):
        return self.par

    def step(self):
        nx, ny, c, opp = self.nx, self.ny, self.c, self.opp
        new = self.f.copy()  # slot sets of nodes are disjoint: writing into a copy equals in place
        for z in range(1, self.nz + 1):
            for y in range(ny):
                for x in range(nx):
                    if self.par == 0:
                        gs = self.g.collide(self.f[:, z, y, x], self.F)
                        for i in range(27):
                            new[opp[i], z, y, x] = gs[i]
                    else:
                        g = np.array([self.f[i, z, y, x] if self._blocked(y - c[i, 1]) else
                                      self.f[opp[i], z - c[i, 2], (y - c[i, 1]) % ny, (x - c[i, 0]) % nx]
                                      for i in range(27)])
                        gs = self.g.collide(g, self.F)
                        for i in range(27):
                            if self._blocked(y + c[i, 1]):
                                new[opp[i], z, y, x] = gs[i]  # halfway bounce-back
                            else:
                                new[i, z + c[i, 2], (y + c[i, 1]) % ny, (x + c[i, 0]) % nx] = gs[i]
        self.f = new
        self.par ^= 1

    def _blocked(self, yy):
        return self.walls and not (0 <= yy < self.ny)

    def _where(self, face, stage, pack):
        top = self.nz + 1
        if pack:
            return {(0, 0): (1, self.up), (1, 0): (top - 1, self.down),
                    (0, 1): (0, self.down), (1, 1): (top, self.up)}[(face, stage)]
        return {(0, 0): (0, self.down), (1, 0): (top, self.up),
                (0, 1): (1, self.up), (1, 1): (top - 1, self.down)}[(face, stage)]

    def pack(self, face, stage):
        import torch
        z, slots = self._where(face, stage, True)
        return torch.from_numpy(np.ascontiguousarray(self.f[slots, z]))

    def unpack(self, face, stage, buf):
        z, slots = self._where(face, stage, False)
        buf = np.asarray(buf)
        for k, i in enumerate(slots):
            for y in range(self.ny):
                # after the odd step, a slot whose source lies behind a wall keeps this node's
                # bounce-back: nothing across the face pushed it
                if stage == 1 and self._blocked(y - self.c[i, 1]):
                    continue
                self.f[i, z, y] = buf[k, y]

    def natural(self):
        assert self.par == 0
        return self.f[:, 1:self.nz + 1].copy()
