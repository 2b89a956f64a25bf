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
                 torch_store=True, slab_z=False, store=None):
        """store: an optional caller-owned CUDA uint8 tensor of at least lbm_store_bytes bytes,
        256-byte aligned, used as the population store (kept alive by the solver)."""
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
        d.slab_z = int(bool(slab_z))
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
                if store is not None:
                    if store.numel() * store.element_size() < nbytes:
                        raise nat.LbmError(nat.LBM_ERR_ARG, "store smaller than lbm_store_bytes")
                    self._store = store
                else:
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

    # Hermite truncation orders (equilibrium, forcing) of the models compared in Sec. III
    MODELS = {"M1": (6, 6), "M4": (6, 2), "M5": (2, 2)}

    def set_hermite_orders(self, eq_order, force_order):
        self._check(self._lib.lbm_set_hermite_orders(self._h, int(eq_order), int(force_order)))

    def set_model(self, name):
        """'M1' (complete expansions, default), 'M4' (Guo forcing) or 'M5' (second-order both)."""
        self.set_hermite_orders(*self.MODELS[name])

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

    # -- magnetic field (App. C)
    def set_magnetic(self, eta, b=None, b_wall=(0.0, 0.0, 0.0)):
        """Turns on the D3Q7 magnetic field: b = (bx, by, bz) arrays of the grid's shape (None: zero)
        or a constant 3-vector; b_wall is held at the y walls."""
        if b is not None and all(np.isscalar(v) for v in b):
            b = [np.full(self.shape, float(v), dtype=np.float32) for v in b]
        self._keep_b = [None, None, None] if b is None else [_f32(a) for a in b]
        bw = (ctypes.c_double * 3)(*[float(v) for v in b_wall])
        self._check(self._lib.lbm_set_magnetic(self._h, float(eta), bw, *(nat.ptr(a) for a in self._keep_b)))

    def get_magnetic_populations(self, out=None):
        if out is None:
            out = np.empty((21,) + self.shape, dtype=np.float32)
        self._check(self._lib.lbm_get_magnetic_populations(self._h, nat.ptr(out)))
        return out

    def set_magnetic_populations(self, h):
        h = _f32(h)
        self._check(self._lib.lbm_set_magnetic_populations(self._h, nat.ptr(h)))

    def magnetic(self):
        """b and j = curl b (each (3,) + shape, float32) at the current time."""
        out = [np.empty(self.shape, dtype=np.float32) for _ in range(6)]
        self._check(self._lib.lbm_magnetic(self._h, *(nat.ptr(a) for a in out)))
        return np.stack(out[:3]), np.stack(out[3:])

    # -- colour-gradient two-phase model (App. D)
    def set_colour_gradient(self, rho_r, rho_b, rho_r0, rho_b0, nu_r, nu_b, A=1e-4, beta=0.7, g=(0.0, 0.0, 0.0)):
        """Turns on the red/blue model from the colour densities rho_r, rho_b (grid-shaped, at rest)."""
        prm = nat.LbmCgParams(float(rho_r0), float(rho_b0), float(nu_r), float(nu_b), float(A), float(beta),
                              (ctypes.c_double * 3)(*[float(v) for v in g]))
        rr, rb = _f32(rho_r), _f32(rho_b)
        self._check(self._lib.lbm_set_colour_gradient(self._h, ctypes.byref(prm), nat.ptr(rr), nat.ptr(rb)))

    def colour_densities(self):
        rr, rb = (np.empty(self.shape, dtype=np.float32) for _ in range(2))
        self._check(self._lib.lbm_colour_densities(self._h, nat.ptr(rr), nat.ptr(rb)))
        return rr, rb

    def get_colour_populations(self):
        fr, fb = (np.empty((27,) + self.shape, dtype=np.float32) for _ in range(2))
        self._check(self._lib.lbm_get_colour_populations(self._h, nat.ptr(fr), nat.ptr(fb)))
        return fr, fb

    def set_colour_populations(self, fr, fb):
        fr, fb = _f32(fr), _f32(fb)
        self._check(self._lib.lbm_set_colour_populations(self._h, nat.ptr(fr), nat.ptr(fb)))

    def stats(self):
        out = (ctypes.c_double * nat.LBM_STATS_LEN)()
        self._check(self._lib.lbm_stats(self._h, out))
        keys = ("mass", "mom_x", "mom_y", "mom_z", "residual", "kinetic_energy", "enstrophy", "umax",
                "fluid_nodes", "step")
        return dict(zip(keys, list(out)))

    def save(self, path):
        self._check(self._lib.lbm_save(self._h, str(path).encode()))

    def load(self, path):
        self._check(self._lib.lbm_load(self._h, str(path).encode()))

    # -- z slabs (see paper_1905_10182_gb300.slabs)
    @property
    def halo_bytes(self):
        return self._lib.lbm_halo_bytes(self._h)

    @property
    def parity(self):
        return self._lib.lbm_parity(self._h)

    def halo_pack(self, face, stage, buf):
        self._check(self._lib.lbm_halo_pack(self._h, int(face), int(stage), nat.ptr(buf)))

    def halo_unpack(self, face, stage, buf):
        self._check(self._lib.lbm_halo_unpack(self._h, int(face), int(stage), nat.ptr(buf)))

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


# launch schedules of the batched step (lbm_batch_set_shape)
SCHEDULES = ("strided", "contiguous", "strided_prefetch")


class BatchSolver:
    """Many independent domains advanced together (lbm_batch_* of the C ABI)."""

    def __init__(self, domains, rho0=1.0, stream=None):
        """domains: list of dicts with nx, ny, nz, nu, and optional force (3-tuple), walls_y, mask."""
        self._lib = nat.lib()
        n = len(domains)
        arr = (nat.LbmDomain * n)()
        self._masks = []
        self.shapes = []
        for k, d in enumerate(domains):
            a = arr[k]
            a.nx, a.ny, a.nz = int(d["nx"]), int(d["ny"]), int(d["nz"])
            a.nu = float(d["nu"])
            f = d.get("force", (0.0, 0.0, 0.0))
            for j in range(3):
                a.force[j] = float(f[j])
            a.walls_y = int(bool(d.get("walls_y", False)))
            m = d.get("mask")
            if m is not None:
                m = np.ascontiguousarray(m, dtype=np.uint8)
                self._masks.append(m)
                a.mask = m.ctypes.data
            self.shapes.append((a.nz, a.ny, a.nx))
        if stream is None:
            import torch
            stream = torch.cuda.current_stream().cuda_stream
        h = ctypes.c_void_p()
        st = self._lib.lbm_batch_create(arr, n, float(rho0), ctypes.c_void_p(int(stream)) if stream else None,
                                        ctypes.byref(h))
        if st != nat.LBM_OK:
            raise nat.LbmError(st, "lbm_batch_create failed")
        self._h = h
        self.count = n

    def _check(self, st):
        if st != nat.LBM_OK:
            raise nat.LbmError(st, self._lib.lbm_batch_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            self._lib.lbm_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def nodes(self):
        return self._lib.lbm_batch_nodes(self._h)

    @property
    def active(self):
        return self._lib.lbm_batch_active(self._h)

    @property
    def time(self):
        return self._lib.lbm_batch_time(self._h)

    def autotune(self, trial_steps=20):
        out = (ctypes.c_double * 4)()
        self._check(self._lib.lbm_batch_autotune(self._h, int(trial_steps), out))
        return dict(mlups=out[0], tile=int(out[1]), blocks_per_sm=int(out[2]),
                    schedule=SCHEDULES[int(out[3])])

    def set_shape(self, tile, blocks_per_sm, schedule="strided"):
        """Launch shape without tuning (tile: nodes per tile; blocks_per_sm 0: one block per tile)."""
        sch = SCHEDULES.index(schedule) if isinstance(schedule, str) else int(schedule)
        self._check(self._lib.lbm_batch_set_shape(self._h, int(tile), int(blocks_per_sm), sch))

    def step(self, nsteps=1):
        self._check(self._lib.lbm_batch_step(self._h, int(nsteps)))

    def run(self, tol=1e-8, max_steps=100000, check_every=100):
        n = self.count
        steps = (ctypes.c_longlong * n)()
        res = (ctypes.c_double * n)()
        status = (ctypes.c_int * n)()
        self._check(self._lib.lbm_batch_run(self._h, float(tol), int(max_steps), int(check_every), steps, res, status))
        return np.array(steps[:]), np.array(res[:]), np.array(status[:])

    def set_state(self, k, rho, ux, uy, uz):
        arrs = [_f32(a) for a in (rho, ux, uy, uz)]
        self._check(self._lib.lbm_batch_set_state(self._h, int(k), *(nat.ptr(a) for a in arrs)))

    def macroscopic(self, k):
        outs = [np.empty(self.shapes[k], dtype=np.float32) for _ in range(4)]
        self._check(self._lib.lbm_batch_macroscopic(self._h, int(k), *(nat.ptr(a) for a in outs)))
        return outs

    def get_populations(self, k):
        out = np.empty((27,) + self.shapes[k], dtype=np.float32)
        self._check(self._lib.lbm_batch_get_populations(self._h, int(k), nat.ptr(out)))
        return out
