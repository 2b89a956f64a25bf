"""Python face of the C ABI in include/cmlbm.h (same calls, same names, marshalling only).

Arrays may be numpy arrays (host) or torch tensors (host or CUDA); the library detects which.
Fields are (nz, ny, nx) float32, populations (27, nz, ny, nx) float32 deviations f_i - w_i rho0.
By default the population store is a torch CUDA tensor and work runs on torch's current stream.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _native as nat

STORAGE = {"fp32": nat.LBM_FP32, "fp16": nat.LBM_FP16_DEV, "bf16": nat.LBM_BF16_DEV}
FORCE = {"none": nat.LBM_FORCE_NONE, "uniform": nat.LBM_FORCE_UNIFORM, "kolmogorov": nat.LBM_FORCE_KOLMOGOROV,
         "field": nat.LBM_FORCE_FIELD, "shan_chen": nat.LBM_FORCE_SHAN_CHEN}


def _f32(a):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        import torch
        return a.to(torch.float32).contiguous()
    return np.ascontiguousarray(a, dtype=np.float32)


class Solver:
    """One D3Q27 central-moment LBM domain on the current CUDA device."""

    def __init__(self, nx, ny, nz, nu, rho0=1.0, walls_y=False, mask=None, storage="fp32", stream=None,
                 torch_store=True):
        self._lib = nat.lib()
        self.shape = (int(nz), int(ny), int(nx))
        self.N = int(nx) * int(ny) * int(nz)
        d = nat.LbmDesc()
        d.nx, d.ny, d.nz = int(nx), int(ny), int(nz)
        d.nu, d.rho0 = float(nu), float(rho0)
        d.walls_y = int(bool(walls_y))
        self._mask = None
        if mask is not None:
            if hasattr(mask, "data_ptr"):
                import torch
                self._mask = mask.to(torch.uint8).contiguous()
            else:
                self._mask = np.ascontiguousarray(mask, dtype=np.uint8)
            d.mask = nat.ptr(self._mask)
        d.storage = STORAGE[storage] if isinstance(storage, str) else int(storage)
        self.storage = storage
        self._store = None
        if stream is None or torch_store:
            import torch
            if stream is None:
                stream = torch.cuda.current_stream().cuda_stream
            if torch_store:
                nbytes = self._lib.lbm_store_bytes(ctypes.byref(d))
                if nbytes == 0:
                    raise nat.LbmError(nat.LBM_ERR_ARG, "invalid grid")
                self._store = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
                d.store = self._store.data_ptr()
        d.stream = int(stream) if stream else None
        self.desc = d
        h = ctypes.c_void_p()
        st = self._lib.lbm_create(ctypes.byref(d), ctypes.byref(h))
        if st != nat.LBM_OK:
            raise nat.LbmError(st, self._lib.lbm_last_error(None).decode())
        self._h = h

    # -- helpers
    def _check(self, st):
        if st != nat.LBM_OK:
            raise nat.LbmError(st, self._lib.lbm_last_error(self._h).decode())

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            self._lib.lbm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- the C ABI
    def set_force(self, kind, params=None, fx=None, fy=None, fz=None):
        k = FORCE[kind] if isinstance(kind, str) else int(kind)
        par = None
        if params is not None:
            arr = (ctypes.c_double * 4)(*([float(v) for v in params] + [0.0] * (4 - len(params))))
            par = arr
        self._keep = [_f32(fx), _f32(fy), _f32(fz)]
        self._check(self._lib.lbm_set_force(self._h, k, par, *(nat.ptr(a) for a in self._keep)))

    def set_state(self, rho, ux, uy, uz):
        arrs = [_f32(a) for a in (rho, ux, uy, uz)]
        self._check(self._lib.lbm_set_state(self._h, *(nat.ptr(a) for a in arrs)))

    def set_populations(self, g):
        g = _f32(g)
        self._check(self._lib.lbm_set_populations(self._h, nat.ptr(g)))

    def get_populations(self, out=None):
        if out is None:
            out = np.empty((27,) + self.shape, dtype=np.float32)
        self._check(self._lib.lbm_get_populations(self._h, nat.ptr(out)))
        return out

    def step(self, nsteps=1):
        self._check(self._lib.lbm_step(self._h, int(nsteps)))

    def stream_only(self, nsteps=1):
        self._check(self._lib.lbm_stream_only(self._h, int(nsteps)))

    def macroscopic(self, rho=None, ux=None, uy=None, uz=None):
        """Fills the given outputs (numpy/torch, N floats) or returns four new numpy arrays."""
        if rho is None and ux is None and uy is None and uz is None:
            rho, ux, uy, uz = (np.empty(self.shape, dtype=np.float32) for _ in range(4))
        self._check(self._lib.lbm_macroscopic(self._h, *(nat.ptr(a) for a in (rho, ux, uy, uz))))
        return rho, ux, uy, uz

    def stats(self):
        out = (ctypes.c_double * nat.LBM_STATS_LEN)()
        self._check(self._lib.lbm_stats(self._h, out))
        keys = ("mass", "mom_x", "mom_y", "mom_z", "residual", "kinetic_energy", "enstrophy", "umax",
                "fluid_nodes", "step")
        return dict(zip(keys, list(out)))

    def profile(self, every=1):
        """Record kernel times of every every-th step (0: off)."""
        self._check(self._lib.lbm_profile(self._h, int(every)))

    def profile_read(self):
        out = (ctypes.c_double * nat.LBM_PROFILE_LEN)()
        self._check(self._lib.lbm_profile_read(self._h, out))
        return dict(collide_ms=out[0], collide_launches=int(out[1]), psi_ms=out[2], psi_launches=int(out[3]))

    def synchronize(self):
        self._check(self._lib.lbm_synchronize(self._h))

    @property
    def time(self):
        return self._lib.lbm_time(self._h)
