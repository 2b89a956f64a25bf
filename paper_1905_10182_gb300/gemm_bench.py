"""Timing of the tcgen05 BF16 GEMM (lbm_gemm_bf16) and of the neural operator's training step.

Prints one JSON line per case: a large square product (compute-bound: TFLOP/s against the dense
BF16 peak) and the operator's own products at the warm-start configuration (64^3, width 32, 12
modes, batch 4: memory-bound, GB/s of A + B read and C written against the HBM copy peak), then
the time of one training step (forward, backward, Adam) of that operator.  CUDA events on the
launching stream, after warm-up.

    python -m paper_1905_10182_gb300.gemm_bench [--profile-shapes | --train-step]
"""
from __future__ import annotations

import ctypes
import json
import os

import numpy as np


def _peaks():
    path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "MEASURED_PEAKS.json")
    try:
        p = json.load(open(path))
        return p.get("bf16_tflops"), p.get("hbm_gbs"), "measured"
    except (OSError, ValueError):
        return 1900.0, 6800.0, "fallback"


def time_gemm(M, N, K, batch, sa, sb, sc, reps=20):
    """sa = (sam, sak, sab) etc. in elements; A, B BF16 and C FP32 device buffers sized from the
    strides; returns milliseconds per call."""
    import torch

    from . import _native as nat

    def extent(strides, dims):
        return 1 + sum((d - 1) * s for d, s in zip(dims, strides))
    A = torch.randn(extent(sa, (M, K, batch)), device="cuda").to(torch.bfloat16)
    B = torch.randn(extent(sb, (K, N, batch)), device="cuda").to(torch.bfloat16)
    C = torch.empty(extent(sc, (M, N, batch)), device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    lib = nat.lib()

    def call():
        r = lib.lbm_gemm_bf16(M, N, K, batch, A.data_ptr(), *sa, B.data_ptr(), *sb, C.data_ptr(), *sc, 0,
                              ctypes.c_float(1.0), 0, err.data_ptr(), st)
        if r != nat.LBM_OK:
            raise nat.LbmError(r, "lbm_gemm_bf16")
    for _ in range(3):
        call()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        call()
    e1.record()
    torch.cuda.synchronize()
    if int(err.item()):
        raise RuntimeError("a GEMM wait timed out")
    return e0.elapsed_time(e1) / reps


def profile_shapes():
    """One timed launch (after 3 warm-ups) of the square, x-DFT and 1x1-map products, in that order:
    launches 3, 7 and 11 of k_gemm_bf16_tc, for an ncu capture."""
    n = 8192
    D, W, MX, B = 64, 32, 12, 4
    S, BWD = D ** 3, B * W * D
    time_gemm(n, n, n, 1, (n, 1, 0), (n, 1, 0), (n, 1, 0), reps=1)
    time_gemm(D, 2 * MX, D, BWD, (D, 1, D * D), (2 * MX, 1, 0), (1, D, 2 * MX * D), reps=1)
    time_gemm(S, W, W, B, (1, S, W * S), (1, W, 0), (1, S, W * S), reps=1)


def main():
    import sys

    import torch
    torch.cuda.set_device(0)
    if "--profile-shapes" in sys.argv:
        profile_shapes()
        return
    if "--train-step" in sys.argv:
        print(json.dumps(train_step_time()), flush=True)
        return
    tf_peak, gb_peak, src = _peaks()
    n = 8192
    ms = time_gemm(n, n, n, 1, (n, 1, 0), (n, 1, 0), (n, 1, 0), reps=5)
    tf = 2.0 * n ** 3 / (ms * 1e-3) / 1e12
    print(json.dumps({"case": f"square {n}^3 row-major", "ms": ms, "tflops": tf, "peak_tflops": tf_peak,
                      "frac": tf / tf_peak, "peak_source": src}), flush=True)
    # the operator's products at D = 64, width 32, 12 modes, batch 4 (strides as the model uses them)
    D, W, MX, B = 64, 32, 12, 4
    MY = MZ = 2 * MX
    S, BWD = D ** 3, B * W * D
    cases = [
        ("x DFT", D, 2 * MX, D, BWD, (D, 1, D * D), (2 * MX, 1, 0), (1, D, 2 * MX * D)),
        ("y DFT", BWD * MX, 2 * MY, 2 * D, 1, (2 * D, 1, 0), (2 * MY, 1, 0), (2 * MY, 1, 0)),
        ("z DFT", B * W * MX * MY, 2 * MZ, 2 * D, 1, (2 * D, 1, 0), (2 * MZ, 1, 0), (2 * MZ, 1, 0)),
        ("inverse x", D, D, 2 * MX, BWD, (1, D, 2 * MX * D), (D, 1, 0), (D, 1, D * D)),
        ("1x1 map", S, W, W, B, (1, S, W * S), (1, W, 0), (1, S, W * S)),
    ]
    for name, M, N, K, nb, sa, sb, sc in cases:
        ms = time_gemm(M, N, K, nb, sa, sb, sc)
        byts = nb * (2 * (M * K + K * N) + 4 * M * N)
        flops = 2.0 * nb * M * N * K
        print(json.dumps({"case": f"operator {name}", "M": M, "N": N, "K": K, "batch": nb, "ms": ms,
                          "gbs": byts / (ms * 1e-3) / 1e9, "peak_gbs": gb_peak,
                          "frac_hbm": byts / (ms * 1e-3) / 1e9 / gb_peak,
                          "tflops": flops / (ms * 1e-3) / 1e12}), flush=True)
    print(json.dumps(train_step_time()), flush=True)


def train_step_time(steps=10):
    """One training step of the operator (batch 4, 64^3, width 32, 12 modes): 3 warm-up steps, then
    the mean over `steps`."""
    import torch

    from .neural import NeuralOperator
    D, W, MX, B = 64, 32, 12, 4
    net = NeuralOperator(D=D, width=W, modes=MX, layers=4, in_ch=4, out_ch=4, max_batch=B, seed=1)
    rng = np.random.default_rng(0)
    x = torch.from_numpy(rng.normal(size=(B, 4, D, D, D)).astype(np.float32)).cuda()
    y = torch.from_numpy(rng.normal(size=(B, 4, D, D, D)).astype(np.float32)).cuda()
    for _ in range(3):
        net.train_step(x, y, 1e-4)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        net.train_step(x, y, 1e-4)
    e1.record()
    torch.cuda.synchronize()
    net.close()
    return {"case": "operator train step (forward, backward, Adam), batch 4, 64^3, width 32, 12 modes",
            "ms": e0.elapsed_time(e1) / steps}


if __name__ == "__main__":
    main()
