"""FP64 CPU oracle of the D3Q27 central-moment LBM with forcing -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may import
this package.  The product library (``paper_1905_10182_gb300``) never imports, links or runs
anything here, and this package imports nothing from it.

The arithmetic lives in ``cmlbm_oracle.c`` (plain C, FP64, OpenMP over nodes); this module
builds it with gcc and exposes numpy-friendly wrappers.  Populations are full values f_i
(not deviations) in the layout f[i, z, y, x].
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "cmlbm_oracle.c")
LIB = os.path.join(HERE, "_build", "libcmlbm_oracle.so")

Q = 27
COLL_LITERAL, COLL_PAPER, COLL_BGK, COLL_NONE = 0, 1, 2, 3
FORCE_NONE, FORCE_UNIFORM, FORCE_KOLMOGOROV, FORCE_FIELD, FORCE_SHAN_CHEN = 0, 1, 2, 3, 4


def build(force: bool = False) -> str:
    """Compile the oracle shared library with gcc (portable flags only: x86_64 and aarch64)."""
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    srcs = [SRC, os.path.join(HERE, "cmlbm_oracle.h")]
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= max(os.path.getmtime(s) for s in srcs)):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-o", tmp, SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


class _Desc(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("omega", ctypes.c_double), ("rho0", ctypes.c_double),
        ("walls_y", ctypes.c_int),
        ("mask", ctypes.c_void_p),
        ("collision", ctypes.c_int),
        ("eq_order", ctypes.c_int), ("force_order", ctypes.c_int),
        ("lambda_", ctypes.c_void_p),
        ("force_kind", ctypes.c_int),
        ("force", ctypes.c_double * 3),
        ("G", ctypes.c_double),
        ("fx", ctypes.c_void_p), ("fy", ctypes.c_void_p), ("fz", ctypes.c_void_p),
        ("threads", ctypes.c_int),
    ]


class _CG(ctypes.Structure):
    _fields_ = [("grid", ctypes.POINTER(_Desc)), ("rho_r0", ctypes.c_double), ("rho_b0", ctypes.c_double),
                ("nu_r", ctypes.c_double), ("nu_b", ctypes.c_double), ("A", ctypes.c_double),
                ("beta", ctypes.c_double), ("gvec", ctypes.c_double * 3)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = build()
        L = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        L.orc_velocities.argtypes = [ctypes.POINTER(ctypes.c_int)]
        L.orc_weights.argtypes = [dp]
        L.orc_opposite.argtypes = [ctypes.c_int]
        L.orc_opposite.restype = ctypes.c_int
        L.orc_hermite.argtypes = [ctypes.c_int] * 4
        L.orc_hermite.restype = ctypes.c_double
        L.orc_equilibrium.argtypes = [ctypes.c_double, dp, ctypes.c_int, dp]
        L.orc_forcing_term.argtypes = [dp, dp, ctypes.c_int, dp]
        L.orc_basis.argtypes = [dp, dp]
        L.orc_central_moments.argtypes = [dp, dp, dp]
        L.orc_inverse_literal.argtypes = [dp, dp, dp]
        L.orc_inverse_literal.restype = ctypes.c_int
        L.orc_inverse_fast.argtypes = [dp, dp, dp]
        for name in ("orc_collide",):
            getattr(L, name).argtypes = [ctypes.POINTER(_Desc), dp, dp, dp]
            getattr(L, name).restype = ctypes.c_int
        L.orc_force_field.argtypes = [ctypes.POINTER(_Desc), dp, dp]
        L.orc_force_field.restype = ctypes.c_int
        L.orc_macroscopic.argtypes = [ctypes.POINTER(_Desc), dp, dp, dp]
        L.orc_macroscopic.restype = ctypes.c_int
        L.orc_init_equilibrium.argtypes = [ctypes.POINTER(_Desc), dp, dp, dp]
        L.orc_init_equilibrium.restype = ctypes.c_int
        L.orc_step.argtypes = [ctypes.POINTER(_Desc), dp, ctypes.c_int]
        L.orc_step.restype = ctypes.c_int
        L.orc_step_sampled.argtypes = [ctypes.POINTER(_Desc), dp, ctypes.POINTER(ctypes.c_longlong),
                                       ctypes.c_int, dp]
        L.orc_step_sampled.restype = ctypes.c_int
        L.orc_mhd_velocities.argtypes = [ctypes.POINTER(ctypes.c_int)]
        L.orc_mhd_weights.argtypes = [dp]
        L.orc_mhd_equilibrium.argtypes = [dp, dp, dp]
        L.orc_mhd_moments.argtypes = [dp, dp, dp]
        L.orc_mhd_node.argtypes = [dp, dp, dp, ctypes.c_double, dp, dp, dp, dp]
        L.orc_mhd_init.argtypes = [ctypes.POINTER(_Desc), dp, dp, dp]
        L.orc_mhd_init.restype = ctypes.c_int
        L.orc_mhd_step.argtypes = [ctypes.POINTER(_Desc), ctypes.c_double, dp, dp, dp, ctypes.c_int]
        L.orc_mhd_step.restype = ctypes.c_int
        L.orc_mhd_fields.argtypes = [ctypes.POINTER(_Desc), ctypes.c_double, dp, dp, dp, dp, dp, dp]
        L.orc_mhd_fields.restype = ctypes.c_int
        L.orc_cg_phi.argtypes = [ctypes.c_double, dp]
        L.orc_cg_equilibrium.argtypes = [ctypes.c_double, dp, ctypes.c_double, ctypes.c_double, dp, dp]
        L.orc_cg_perturbation.argtypes = [ctypes.c_double, dp, dp]
        L.orc_cg_recolour.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double, dp, dp,
                                      dp, dp]
        for name in ("orc_cg_init",):
            getattr(L, name).argtypes = [ctypes.POINTER(_CG), dp, dp, dp, dp, dp]
            getattr(L, name).restype = ctypes.c_int
        L.orc_cg_step.argtypes = [ctypes.POINTER(_CG), dp, dp, ctypes.c_int]
        L.orc_cg_step.restype = ctypes.c_int
        L.orc_cg_fields.argtypes = [ctypes.POINTER(_CG), dp, dp, dp, dp, dp]
        L.orc_cg_fields.restype = ctypes.c_int
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _vec(v, n=3):
    a = np.ascontiguousarray(np.asarray(v, dtype=np.float64).reshape(n))
    return a


# --------------------------------------------------------------------------- lattice
def velocities() -> np.ndarray:
    c = (ctypes.c_int * (Q * 3))()
    lib().orc_velocities(c)
    return np.array(c[:], dtype=np.int64).reshape(Q, 3)


def weights() -> np.ndarray:
    w = np.zeros(Q)
    lib().orc_weights(_dp(w))
    return w


def opposite(i: int) -> int:
    return lib().orc_opposite(i)


def hermite(i: int, nx: int, ny: int, nz: int) -> float:
    return lib().orc_hermite(i, nx, ny, nz)


def equilibrium(rho, u, order=6) -> np.ndarray:
    out = np.zeros(Q)
    uu = _vec(u)
    lib().orc_equilibrium(float(rho), _dp(uu), int(order), _dp(out))
    return out


def forcing_term(F, u, order=6) -> np.ndarray:
    out = np.zeros(Q)
    FF, uu = _vec(F), _vec(u)
    lib().orc_forcing_term(_dp(FF), _dp(uu), int(order), _dp(out))
    return out


def basis(u) -> np.ndarray:
    T = np.zeros((Q, Q))
    uu = _vec(u)
    lib().orc_basis(_dp(uu), _dp(T))
    return T


def central_moments(u, v) -> np.ndarray:
    k = np.zeros(Q)
    uu, vv = _vec(u), _vec(v, Q)
    lib().orc_central_moments(_dp(uu), _dp(vv), _dp(k))
    return k


def inverse_literal(u, k) -> np.ndarray:
    v = np.zeros(Q)
    uu, kk = _vec(u), _vec(k, Q)
    st = lib().orc_inverse_literal(_dp(uu), _dp(kk), _dp(v))
    if st:
        raise RuntimeError(f"orc_inverse_literal failed ({st})")
    return v


def inverse_fast(u, k) -> np.ndarray:
    v = np.zeros(Q)
    uu, kk = _vec(u), _vec(k, Q)
    lib().orc_inverse_fast(_dp(uu), _dp(kk), _dp(v))
    return v


# --------------------------------------------------------------------------- grid
class Grid:
    """Parameters of an oracle run; owns the numpy arrays the C descriptor points at."""

    def __init__(self, nx, ny, nz, nu=None, omega=None, rho0=1.0, walls_y=False, mask=None,
                 collision=COLL_PAPER, eq_order=6, force_order=6, lambdas=None,
                 force_kind=FORCE_NONE, force=(0.0, 0.0, 0.0), G=0.0, field=None, threads=0):
        if omega is None:
            omega = 1.0 / (3.0 * nu + 0.5)
        self.shape = (int(nz), int(ny), int(nx))
        self.N = int(nx) * int(ny) * int(nz)
        d = _Desc()
        d.nx, d.ny, d.nz = int(nx), int(ny), int(nz)
        d.omega = float(omega)
        d.rho0 = float(rho0)
        d.walls_y = int(bool(walls_y))
        self._mask = None
        if mask is not None:
            self._mask = np.ascontiguousarray(np.asarray(mask, dtype=np.uint8).reshape(-1))
            d.mask = self._mask.ctypes.data
        d.collision = int(collision)
        d.eq_order, d.force_order = int(eq_order), int(force_order)
        self._lam = None
        if lambdas is not None:
            self._lam = _vec(lambdas, Q)
            d.lambda_ = self._lam.ctypes.data
        d.force_kind = int(force_kind)
        for k in range(3):
            d.force[k] = float(force[k])
        d.G = float(G)
        self._field = None
        if field is not None:
            self._field = [np.ascontiguousarray(np.asarray(a, dtype=np.float64).reshape(-1)) for a in field]
            d.fx, d.fy, d.fz = (a.ctypes.data for a in self._field)
        d.threads = int(threads)
        self.desc = d

    def _check(self, st, what):
        if st:
            raise RuntimeError(f"oracle {what} failed with status {st}")

    def collide(self, f, F=(0.0, 0.0, 0.0)) -> np.ndarray:
        ff, FF = _vec(f, Q), _vec(F)
        out = np.zeros(Q)
        self._check(lib().orc_collide(ctypes.byref(self.desc), _dp(ff), _dp(FF), _dp(out)), "collide")
        return out

    def init_equilibrium(self, rho, u) -> np.ndarray:
        rho = np.ascontiguousarray(np.broadcast_to(np.asarray(rho, dtype=np.float64), self.shape)).reshape(-1)
        u = np.ascontiguousarray(np.asarray(u, dtype=np.float64).reshape(3, -1))
        f = np.zeros((Q,) + self.shape)
        self._check(lib().orc_init_equilibrium(ctypes.byref(self.desc), _dp(rho), _dp(u), _dp(f)), "init")
        return f

    def step(self, f: np.ndarray, nsteps: int = 1) -> np.ndarray:
        """Advance a copy of f (shape (27, nz, ny, nx)) by nsteps; returns the new array."""
        g = np.ascontiguousarray(f, dtype=np.float64).copy()
        self._check(lib().orc_step(ctypes.byref(self.desc), _dp(g), int(nsteps)), "step")
        return g

    def step_sampled(self, f: np.ndarray, nodes) -> np.ndarray:
        f = np.ascontiguousarray(f, dtype=np.float64)
        nodes = np.ascontiguousarray(np.asarray(nodes, dtype=np.int64))
        out = np.zeros((len(nodes), Q))
        self._check(lib().orc_step_sampled(ctypes.byref(self.desc), _dp(f),
                                           nodes.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)),
                                           len(nodes), _dp(out)), "step_sampled")
        return out

    def force_field(self, f) -> np.ndarray:
        f = np.ascontiguousarray(f, dtype=np.float64)
        F = np.zeros((3,) + self.shape)
        self._check(lib().orc_force_field(ctypes.byref(self.desc), _dp(f), _dp(F)), "force_field")
        return F

    def macroscopic(self, f):
        f = np.ascontiguousarray(f, dtype=np.float64)
        rho = np.zeros(self.shape)
        u = np.zeros((3,) + self.shape)
        self._check(lib().orc_macroscopic(ctypes.byref(self.desc), _dp(f), _dp(rho), _dp(u)), "macroscopic")
        return rho, u


# --------------------------------------------------------------------------- magnetic field (App. C)
QM = 7


def mhd_velocities() -> np.ndarray:
    c = (ctypes.c_int * (QM * 3))()
    lib().orc_mhd_velocities(c)
    return np.array(list(c), dtype=np.int64).reshape(QM, 3)


def mhd_weights() -> np.ndarray:
    w = np.zeros(QM)
    lib().orc_mhd_weights(_dp(w))
    return w


def mhd_equilibrium(b, u) -> np.ndarray:
    """h_la^eq as an array (7, 3)."""
    out = np.zeros(3 * QM)
    lib().orc_mhd_equilibrium(_dp(_vec(b)), _dp(_vec(u)), _dp(out))
    return out.reshape(QM, 3)


def mhd_moments(h):
    """b = sum_l h_l and E_g = eps_gba sum_l xi_lb h_la of one node, h shaped (7, 3)."""
    b, E = np.zeros(3), np.zeros(3)
    lib().orc_mhd_moments(_dp(_vec(np.asarray(h).reshape(-1), 3 * QM)), _dp(b), _dp(E))
    return b, E


def mhd_node(f, h, Fext, omega_m):
    """rho, u, Lorentz force, current of one node."""
    rho = np.zeros(1)
    u, FL, j = np.zeros(3), np.zeros(3), np.zeros(3)
    lib().orc_mhd_node(_dp(_vec(f, Q)), _dp(_vec(np.asarray(h).reshape(-1), 3 * QM)), _dp(_vec(Fext)),
                       float(omega_m), _dp(rho), _dp(u), _dp(FL), _dp(j))
    return float(rho[0]), u, FL, j


class MhdGrid(Grid):
    """A Grid with the magnetic populations of App. C: h has shape (21, nz, ny, nx), entry 3 l + a."""

    def __init__(self, nx, ny, nz, eta=None, omega_m=None, b_wall=(0.0, 0.0, 0.0), **kw):
        super().__init__(nx, ny, nz, **kw)
        if omega_m is None:
            omega_m = 1.0 / (eta / 0.25 + 0.5)
        self.omega_m = float(omega_m)
        self.b_wall = _vec(b_wall)

    def _field3(self, v):
        """(3,) constant or (3, nz, ny, nx) field -> contiguous (3, N) float64."""
        v = np.asarray(v, dtype=np.float64)
        if v.ndim == 1:
            v = v.reshape(3, 1, 1, 1)
        return np.ascontiguousarray(np.broadcast_to(v, (3,) + self.shape)).reshape(3, -1)

    def mhd_init(self, b, u) -> np.ndarray:
        """h = h^eq(b, u)."""
        b, u = self._field3(b), self._field3(u)
        h = np.zeros((3 * QM,) + self.shape)
        self._check(lib().orc_mhd_init(ctypes.byref(self.desc), _dp(b), _dp(u), _dp(h)), "mhd_init")
        return h

    def mhd_step(self, f, h, nsteps=1):
        """Advance copies of f and h by nsteps of the coupled scheme; returns (f, h)."""
        f = np.ascontiguousarray(f, dtype=np.float64).copy()
        h = np.ascontiguousarray(h, dtype=np.float64).copy()
        self._check(lib().orc_mhd_step(ctypes.byref(self.desc), self.omega_m, _dp(self.b_wall), _dp(f), _dp(h),
                                       int(nsteps)), "mhd_step")
        return f, h

    def mhd_fields(self, f, h):
        """rho, u, b, j at the current time."""
        f = np.ascontiguousarray(f, dtype=np.float64)
        h = np.ascontiguousarray(h, dtype=np.float64)
        rho = np.zeros(self.shape)
        u, b, j = (np.zeros((3,) + self.shape) for _ in range(3))
        self._check(lib().orc_mhd_fields(ctypes.byref(self.desc), self.omega_m, _dp(f), _dp(h), _dp(rho), _dp(u),
                                         _dp(b), _dp(j)), "mhd_fields")
        return rho, u, b, j


# --------------------------------------------------------------------------- colour gradient (App. D)
def cg_phi(alpha) -> np.ndarray:
    out = np.zeros(Q)
    lib().orc_cg_phi(float(alpha), _dp(out))
    return out


def cg_equilibrium(rho, u, alpha, nu, grad_rho=(0.0, 0.0, 0.0)) -> np.ndarray:
    out = np.zeros(Q)
    lib().orc_cg_equilibrium(float(rho), _dp(_vec(u)), float(alpha), float(nu), _dp(_vec(grad_rho)), _dp(out))
    return out


def cg_perturbation(A, grad_phi) -> np.ndarray:
    out = np.zeros(Q)
    lib().orc_cg_perturbation(float(A), _dp(_vec(grad_phi)), _dp(out))
    return out


def cg_recolour(beta, rho_r, rho_b, alpha, grad_phi, fs):
    fr, fb = np.zeros(Q), np.zeros(Q)
    lib().orc_cg_recolour(float(beta), float(rho_r), float(rho_b), float(alpha), _dp(_vec(grad_phi)),
                          _dp(_vec(fs, Q)), _dp(fr), _dp(fb))
    return fr, fb


class CgGrid(Grid):
    """Two-colour populations (fr, fb, each (27, nz, ny, nx)) of the colour-gradient model (App. D)."""

    def __init__(self, nx, ny, nz, rho_r0, rho_b0, nu_r, nu_b, A=0.0, beta=0.7, gvec=(0.0, 0.0, 0.0), **kw):
        super().__init__(nx, ny, nz, nu=nu_r, **kw)
        m = _CG()
        m.grid = ctypes.pointer(self.desc)
        m.rho_r0, m.rho_b0, m.nu_r, m.nu_b = float(rho_r0), float(rho_b0), float(nu_r), float(nu_b)
        m.A, m.beta = float(A), float(beta)
        for k in range(3):
            m.gvec[k] = float(gvec[k])
        self.cg = m

    def cg_init(self, rho_r, rho_b, u=None):
        rr = np.ascontiguousarray(np.broadcast_to(np.asarray(rho_r, np.float64), self.shape)).reshape(-1)
        rb = np.ascontiguousarray(np.broadcast_to(np.asarray(rho_b, np.float64), self.shape)).reshape(-1)
        uu = np.zeros((3, self.N)) if u is None else np.ascontiguousarray(np.asarray(u, np.float64).reshape(3, -1))
        fr, fb = np.zeros((Q,) + self.shape), np.zeros((Q,) + self.shape)
        self._check(lib().orc_cg_init(ctypes.byref(self.cg), _dp(rr), _dp(rb), _dp(uu), _dp(fr), _dp(fb)), "cg_init")
        return fr, fb

    def cg_step(self, fr, fb, nsteps=1):
        fr = np.ascontiguousarray(fr, dtype=np.float64).copy()
        fb = np.ascontiguousarray(fb, dtype=np.float64).copy()
        self._check(lib().orc_cg_step(ctypes.byref(self.cg), _dp(fr), _dp(fb), int(nsteps)), "cg_step")
        return fr, fb

    def cg_fields(self, fr, fb):
        fr = np.ascontiguousarray(fr, dtype=np.float64)
        fb = np.ascontiguousarray(fb, dtype=np.float64)
        rr, rb = np.zeros(self.shape), np.zeros(self.shape)
        u = np.zeros((3,) + self.shape)
        self._check(lib().orc_cg_fields(ctypes.byref(self.cg), _dp(fr), _dp(fb), _dp(rr), _dp(rb), _dp(u)), "cg_fields")
        return rr, rb, u


# --------------------------------------------------------------------------- diagnostics
def kinetic_energy(u, fluid=None) -> float:
    """Mean of |u|^2 / 2 over fluid nodes (FP64)."""
    e = 0.5 * (u[0] ** 2 + u[1] ** 2 + u[2] ** 2)
    return float(e[fluid].mean() if fluid is not None else e.mean())


def enstrophy(u) -> float:
    """Mean of |curl u|^2 / 2 with second-order central differences on a periodic grid.
    u has shape (3, nz, ny, nx)."""
    def d(a, axis):
        return 0.5 * (np.roll(a, -1, axis=axis) - np.roll(a, 1, axis=axis))
    ux, uy, uz = u
    wx = d(uz, 1) - d(uy, 0)
    wy = d(ux, 0) - d(uz, 2)
    wz = d(uy, 2) - d(ux, 1)
    return float((0.5 * (wx ** 2 + wy ** 2 + wz ** 2)).mean())
