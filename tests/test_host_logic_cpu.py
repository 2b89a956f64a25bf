"""Host-side logic of the kernels and of bench.py, checked on the CPU.

* The magic-number division the kernels use for their index maps (FastDiv in lbm_device.cuh):
  for a divisor d >= 2, l = ceil(log2 d), m = ceil(2^(31 + l) / d), s = l - 1, the quotient of any
  dividend n < 2^31 is umulhi(n, m) >> s, because m d - 2^(31 + l) < 2^l.  Checked here for the
  construction itself, over every divisor up to 4096, a spread of larger ones and dividends at the
  edges of each quotient step.
* bench.py's kernel-time sampling: every timed run of at least two steps records at least one step
  pair, whatever its warm-up (a run with none cannot report a roofline).
"""
import importlib.util
import os

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def magic(d):
    l = (d - 1).bit_length()  # ceil(log2 d) for d >= 2
    return (2 ** (31 + l) + d - 1) // d, l - 1


def test_magic_number_division_is_exact():
    rng = np.random.default_rng(5)
    divisors = list(range(2, 4097)) + [int(v) for v in rng.integers(4097, 2 ** 31, 2000)] + [2 ** 31 - 1, 2 ** 30 + 1]
    for d in divisors:
        m, s = magic(d)
        assert m < 2 ** 32, d
        q = np.arange(0, (2 ** 31 - 1) // d + 1, max(1, ((2 ** 31 - 1) // d) // 500), dtype=np.uint64)
        n = np.concatenate([q * np.uint64(d), q * np.uint64(d) + np.uint64(d - 1), q * np.uint64(d) - np.uint64(1)])
        n = n[(n < 2 ** 31)]
        n = np.concatenate([n, np.array([0, 2 ** 31 - 1], dtype=np.uint64)])
        hi = (n * np.uint64(m)) >> np.uint64(32)
        assert np.array_equal(hi >> np.uint64(s), n // np.uint64(d)), d


def test_bench_samples_kernel_times_in_every_run():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    for steps in (2, 3, 7, 20, 100, 255, 256, 2000):
        every = bench.profile_every(steps)
        for warmup in range(0, 70):
            sampled = [t for t in range(warmup, warmup + steps) if t % every in (0, 1)]
            assert sampled, (steps, warmup, every)
    assert bench.profile_every(2000) == bench.PROFILE_EVERY
