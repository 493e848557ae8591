"""Pins for the oracle's random-number side: Philox4x32-10, the FP32 log and
sincos it uses, and the Box-Muller normals of the Gaussian sketch (Section 2.3,
"Gaussian Ensemble").  Each pin is independent of the oracle's own code:
library functions, statistics and exact properties."""
import math

import numpy as np
import pytest
from scipy import stats

import oracle as o


# ------------------------------------------------------------------ Philox
def test_philox_is_a_bijection_on_a_counter_set():
    # Each round is invertible for a fixed key, so distinct counters never
    # collide; 20000 consecutive counters give 20000 distinct 128-bit outputs.
    seen = set()
    for c in range(20000):
        seen.add(tuple(o.philox4x32_10([c, 0, 7, 0], [123, 456])))
    assert len(seen) == 20000


def test_philox_output_bits_are_balanced():
    # every output bit is 1 with probability 1/2 (4 * 32 bits, 8192 draws)
    bits = np.zeros(128)
    N = 8192
    for c in range(N):
        x = o.philox4x32_10([c, c >> 5, 3, 1], [0xDEADBEEF, 42])
        for w in range(4):
            for b in range(32):
                bits[32 * w + b] += (int(x[w]) >> b) & 1
    frac = bits / N
    # 6 sigma band for a binomial(N, 1/2) fraction
    assert np.all(np.abs(frac - 0.5) < 6 * 0.5 / math.sqrt(N))


def test_philox_avalanche_on_counter_and_key():
    # flipping one input bit flips about half of the 128 output bits
    rng = np.random.default_rng(5)
    flips = []
    for _ in range(400):
        c = [int(v) for v in rng.integers(0, 2**32, 4, dtype=np.uint64)]
        k = [int(v) for v in rng.integers(0, 2**32, 2, dtype=np.uint64)]
        base = o.philox4x32_10(c, k)
        w, b = int(rng.integers(0, 6)), int(rng.integers(0, 32))
        c2, k2 = list(c), list(k)
        if w < 4:
            c2[w] ^= 1 << b
        else:
            k2[w - 4] ^= 1 << b
        x = o.philox4x32_10(c2, k2)
        flips.append(sum(bin(int(a) ^ int(bb)).count("1") for a, bb in zip(base, x)))
    assert abs(np.mean(flips) - 64.0) < 1.5


# ------------------------------------------------------------------ FP32 log
def test_logf_within_two_ulp_of_true_log():
    # all u = n 2^-24 for a spread of n, plus every power of two
    ns = np.unique(np.concatenate([np.arange(1, 5000), np.linspace(1, 2**24, 20001).astype(np.int64),
                                   2 ** np.arange(25), 2 ** np.arange(1, 25) - 1]))
    worst = 0.0
    for n in ns:
        u = np.float32(float(n) * 2.0**-24)
        got = float(o.logf(float(u)))
        exact = math.log(float(u))
        if exact == 0.0:
            assert got == 0.0
            continue
        ulp = float(np.spacing(np.float32(abs(exact))))
        worst = max(worst, abs(got - exact) / ulp)
    assert worst <= 2.0, worst


# ------------------------------------------------------------------ sincos
def test_sincos2pi_matches_library_within_single_precision():
    ns = np.unique(np.concatenate([np.arange(1, 3000), np.linspace(1, 2**24, 30001).astype(np.int64),
                                   [2**21, 2**22, 2**23, 3 * 2**22, 2**24, 2**21 - 1, 2**21 + 1]]))
    worst = 0.0
    for n in ns:
        s, c = o.sincos2pi(int(n))
        th = 2.0 * math.pi * float(n) * 2.0**-24
        worst = max(worst, abs(float(s) - math.sin(th)), abs(float(c) - math.cos(th)))
        assert abs(float(s) ** 2 + float(c) ** 2 - 1.0) < 3e-7
    assert worst < 2.5e-7, worst


def test_sincos2pi_exact_quadrant_points():
    # u = 1/4, 1/2, 3/4, 1 land exactly on the axes
    assert o.sincos2pi(2**22) == (np.float32(1.0), np.float32(0.0))
    assert o.sincos2pi(2**23) == (np.float32(0.0), np.float32(-1.0)) or \
        o.sincos2pi(2**23) == (np.float32(-0.0), np.float32(-1.0))
    s, c = o.sincos2pi(3 * 2**22)
    assert (s, abs(c)) == (np.float32(-1.0), np.float32(0.0))
    s, c = o.sincos2pi(2**24)
    assert (abs(s), c) == (np.float32(0.0), np.float32(1.0))


# ------------------------------------------------------------------ normals
def test_normals_are_standard_normal():
    z = o.omega_z(seed=0, s=128, i0=0, rows=2000).ravel().astype(np.float64)  # 256000 values
    assert abs(z.mean()) < 6 / math.sqrt(z.size)
    assert abs(z.var() - 1.0) < 6 * math.sqrt(2.0 / z.size)
    assert abs(stats.kurtosis(z, fisher=False) - 3.0) < 0.05
    assert stats.kstest(z, "norm").pvalue > 1e-4


def test_normals_independent_across_rows_and_columns():
    z = o.omega_z(seed=7, s=64, i0=10**6, rows=4000).astype(np.float64)
    c = np.corrcoef(z.T)                       # 64 x 64 correlation between sketch rows
    off = c[~np.eye(64, dtype=bool)]
    assert np.max(np.abs(off)) < 6 / math.sqrt(4000)
    c2 = np.corrcoef(z)[:200, :200]            # between columns (rows of A)
    assert np.max(np.abs(c2[~np.eye(200, dtype=bool)])) < 0.6


def test_omega_layout_and_odd_s():
    # z_out[(i - i0) * s + r]: rows 4k..4k+3 of column i are one Philox call
    z = o.omega_z(seed=3, s=10, i0=5, rows=3)
    for i in range(3):
        for k in range(3):
            q = o.normal4(3, 5 + i, k, 0)
            for t in range(4):
                if 4 * k + t < 10:
                    assert z[i, 4 * k + t] == q[t]
    # odd s drops the surplus of the last call; shorter s is a prefix
    z7 = o.omega_z(seed=3, s=7, i0=5, rows=3)
    assert np.array_equal(z7, z[:, :7])


def test_seed_and_large_row_index_change_the_stream():
    a = o.omega_z(1, 8, 0, 4)
    b = o.omega_z(2, 8, 0, 4)
    assert not np.array_equal(a, b)
    hi = o.omega_z(1, 8, 2**32, 4)             # i_hi word of the counter in use
    assert not np.array_equal(a, hi)
    assert np.all(np.isfinite(hi))


def test_sketch_variance_is_one_over_s():
    # Omega has N(0, 1/s) entries: E ||Omega x||^2 = ||x||^2 for a unit vector x
    m, s = 4000, 64
    Om = o.omega(seed=11, s=s, m=m)
    x = np.ones(m) / math.sqrt(m)
    vals = [np.sum((o.omega(seed=sd, s=s, m=m) @ x) ** 2) for sd in range(20)]
    assert abs(np.mean(vals) - 1.0) < 6 * math.sqrt(2.0 / s / 20)
    assert abs(Om.var() * s - 1.0) < 0.02
