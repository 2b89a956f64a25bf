"""C-ABI checks that need no GPU: the library builds and loads, every entry point declared in
include/cmlbm.h is exported, and argument validation answers before any device work."""
import ctypes
import subprocess

import pytest


@pytest.fixture(scope="module")
def nat():
    from paper_1905_10182_gb300 import _native
    _native.lib()
    return _native


def test_every_declared_symbol_is_exported(nat):
    declared = nat.declared_symbols()
    assert len(declared) >= 14
    out = subprocess.run(["nm", "-D", "--defined-only", nat._build.LIB], capture_output=True, text=True,
                         check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    missing = [s for s in declared if s not in exported]
    assert not missing, missing
    for s in declared:
        assert hasattr(nat.lib(), s)


def test_store_bytes(nat):
    d = nat.LbmDesc()
    d.nx, d.ny, d.nz, d.nu, d.rho0 = 5, 3, 7, 0.1, 1.0
    for storage, size in ((nat.LBM_FP32, 4), (nat.LBM_FP16_DEV, 2), (nat.LBM_BF16_DEV, 2)):
        d.storage = storage
        assert nat.lib().lbm_store_bytes(ctypes.byref(d)) == 27 * 5 * 3 * 7 * size
    d.storage = 9
    assert nat.lib().lbm_store_bytes(ctypes.byref(d)) == 0
    d.storage, d.nx = 0, 0
    assert nat.lib().lbm_store_bytes(ctypes.byref(d)) == 0


@pytest.mark.parametrize("field,value", [("nx", 0), ("ny", -1), ("nu", 0.0), ("rho0", -1.0), ("storage", 5)])
def test_create_rejects_bad_arguments_without_a_gpu(nat, field, value):
    d = nat.LbmDesc()
    d.nx, d.ny, d.nz, d.nu, d.rho0, d.storage = 4, 4, 4, 0.1, 1.0, 0
    setattr(d, field, value)
    h = ctypes.c_void_p(123)
    st = nat.lib().lbm_create(ctypes.byref(d), ctypes.byref(h))
    assert st == nat.LBM_ERR_ARG
    assert not h.value
    assert nat.lib().lbm_last_error(None)


def test_null_handles(nat):
    L = nat.lib()
    L.lbm_destroy(None)
    assert L.lbm_step(None, 1) == nat.LBM_ERR_ARG
    assert L.lbm_time(None) == -1
    assert L.lbm_status_string(nat.LBM_ERR_DIVERGED) == b"LBM_ERR_DIVERGED"
    d = nat.LbmDesc()
    d.nx = d.ny = d.nz = 4
    d.nu, d.rho0 = 0.1, 1.0
    assert L.lbm_create(ctypes.byref(d), None) == nat.LBM_ERR_ARG


def test_huge_grid_rejected(nat):
    d = nat.LbmDesc()
    d.nx, d.ny, d.nz, d.nu, d.rho0 = 2048, 2048, 1024, 0.1, 1.0
    h = ctypes.c_void_p()
    assert nat.lib().lbm_create(ctypes.byref(d), ctypes.byref(h)) == nat.LBM_ERR_ARG
