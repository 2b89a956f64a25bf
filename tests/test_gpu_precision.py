"""Where the drift of 16-bit population storage comes from (the third benchmark configuration's
Taylor-Green vortex at 64^3, U0 = 0.05, nu = 1e-4, 5000 steps through the transition).

tests/golden/tgv64_rounded_oracle.txt holds the FP64 oracle's kinetic energy and enstrophy every
250 steps, plain and with its state rounded to FP16 or BF16 deviations after every step (the
rounding sits between oracle steps, so the stored curves carry storage rounding and no other
error).  The GPU's 16-bit kernels store the same rounded deviations but compute each step in FP32
with the direct-form collision.  If the GPU follows the rounded oracle much more closely than the
rounded oracle follows the plain one, the drift is the storage rounding and not the kernels'
arithmetic.

Measured (deterministic on both sides): BF16 storage rounding alone moves the energy by 6.4 %
and the enstrophy by 11.6 % (D_storage); the GPU's BF16 run stays within 0.87 % and 0.93 % of the
rounded oracle (D_kernel), so BF16's drift is the storage rounding.  FP16 storage moves the curves
by 0.085 % and 0.13 %, and the GPU differs from the rounded oracle by 0.22 % and 0.16 %: the
same small order, since two FP16 trajectories whose rounding decisions differ wherever an FP32
and an FP64 result straddle a rounding boundary separate through the transition; FP16 drifts by
at most 0.13 % from the plain oracle.

Asserted, energy and enstrophy: BF16, D_kernel <= D_storage / 4 and D_kernel <= 2e-2; FP16, the
GPU within 3e-3 of the plain oracle and D_kernel <= 5e-3 (about twice the measured values).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from golden_util import load_table  # noqa: E402
from paper_1905_10182_gb300 import Solver, inputs  # noqa: E402

N, U0, NU, STEPS, EVERY = 64, 0.05, 1e-4, 5000, 250


def _gpu_curves(storage):
    rho, ux, uy, uz = inputs.taylor_green(N, U0)
    s = Solver(N, N, N, nu=NU, storage=storage)
    s.set_state(rho, ux, uy, uz)
    ke, ens = [], []
    for k in range(0, STEPS + 1, EVERY):
        if k:
            s.step(EVERY)
        st = s.stats()
        ke.append(st["kinetic_energy"])
        ens.append(st["enstrophy"])
    s.close()
    return np.array(ke), np.array(ens)


@pytest.mark.parametrize("storage", ["fp16", "bf16"])
def test_storage_rounding_explains_the_drift(storage):
    gold = load_table("tgv64_rounded_oracle.txt")
    ks = range(0, STEPS + 1, EVERY)
    ref = {q: np.array([float(gold[f"{q}_fp64_{k}"]) for k in ks]) for q in ("ke", "ens")}
    rnd = {q: np.array([float(gold[f"{q}_{storage}_{k}"]) for k in ks]) for q in ("ke", "ens")}
    gpu = dict(zip(("ke", "ens"), _gpu_curves(storage)))
    for q in ("ke", "ens"):
        d_storage = np.max(np.abs(rnd[q] - ref[q]) / ref[q])
        d_kernel = np.max(np.abs(gpu[q] - rnd[q]) / ref[q])
        d_total = np.max(np.abs(gpu[q] - ref[q]) / ref[q])
        print(f"{storage} {q}: GPU vs FP64 oracle {d_total:.3e}; rounded oracle vs FP64 oracle (storage) "
              f"{d_storage:.3e}; GPU vs rounded oracle (kernel arithmetic) {d_kernel:.3e}")
        if storage == "bf16":
            assert d_kernel <= 0.25 * d_storage and d_kernel <= 2e-2, (q, d_kernel, d_storage)
        else:
            assert d_total <= 3e-3 and d_kernel <= 5e-3, (q, d_total, d_kernel)
