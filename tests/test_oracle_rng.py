"""Pins for the oracle's random streams.

* Philox4x32-10 against an independent library implementation (cuRAND's host
  generator, run on the CPU): its output word 4q+j is word j of the block with key
  (seed lo, seed hi) and counter (c0|c1 = q div 65536, c2 = q mod 65536, c3 = 0),
  which exercises both key words and the counter words c0, c1, c2.
* uniforms, Box-Muller normals, Poisson counts, jump times and jump sizes against
  their laws (exact values, scipy CDFs, Kolmogorov-Smirnov and chi-square tests).
  The jump-time test pins the per-step construction against the paper's exponential
  inter-arrival sampling (Sec. 5.3 eq:collision_time_Poisson, Algorithm 5.2).
"""
import ctypes
import os

import numpy as np
import pytest
from scipy import stats

import oracle
import workloads

MASK = 0xFFFFFFFF


def _curand():
    for path in ("/usr/local/cuda/lib64/libcurand.so", "libcurand.so", "libcurand.so.10"):
        try:
            return ctypes.CDLL(path)
        except OSError:
            continue
    return None


def _curand_words(lib, seed, offset, n):
    gen = ctypes.c_void_p()
    assert lib.curandCreateGeneratorHost(ctypes.byref(gen), 161) == 0  # PHILOX4_32_10
    assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
    assert lib.curandSetGeneratorOffset(gen, ctypes.c_ulonglong(offset)) == 0
    out = np.zeros(n, dtype=np.uint32)
    assert lib.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(n)) == 0
    lib.curandDestroyGenerator(gen)
    return out


@pytest.mark.parametrize("seed", [0, 1, 0x123456789ABCDEF, 0xFFFFFFFFFFFFFFFF, 2**32 + 5])
def test_philox_matches_curand_host(seed):
    lib = _curand()
    if lib is None:
        pytest.skip("cuRAND not loadable")
    key = (seed & MASK, seed >> 32)
    for offset_q in (0, 65536 * 3 + 100, 65536 * 70000, (1 << 48) + 65536 * 9 + 7):
        n = 4 * 64
        words = _curand_words(lib, seed, 4 * offset_q, n)
        for b in range(0, n // 4, 7):
            q = offset_q + b
            c0, c2 = q // 65536, q % 65536
            got = oracle.philox(key, (c0 & MASK, c0 >> 32, c2, 0))
            assert got == [int(x) for x in words[4 * b: 4 * b + 4]], (seed, q)


def test_philox_counter_avalanche():
    """Flipping any single counter or key bit changes about half of the 128 output bits."""
    base_key, base_ctr = (0x01234567, 0x89ABCDEF), (5, 77, 1 << 24, 3)
    ref = oracle.philox(base_key, base_ctr)
    flips = []
    for word in range(6):
        for bit in range(0, 32, 3):
            k, c = list(base_key), list(base_ctr)
            if word < 4:
                c[word] ^= 1 << bit
            else:
                k[word - 4] ^= 1 << bit
            o = oracle.philox(k, c)
            flips.append(sum(bin(a ^ b).count("1") for a, b in zip(o, ref)))
    flips = np.array(flips)
    assert 56 < flips.mean() < 72
    assert flips.min() > 35


def test_u01_exact_values():
    assert oracle.u01(0) == 2.0 ** -24
    assert oracle.u01(0xFFFFFFFF) == 1.0 - 2.0 ** -24
    for w in (0x200, 0x12345678, 0x80000000):
        assert oracle.u01(w) == ((w >> 9) * 2 + 1) * 2.0 ** -24


@pytest.mark.parametrize("mu", [1e-6, 0.01, 0.4, 2.0, 5.0])
def test_poisson_thresholds_match_cdf(mu):
    thr = oracle.poisson_thresholds(mu)
    cdf = stats.poisson.cdf(np.arange(16), mu)
    assert all(thr[i] <= thr[i + 1] for i in range(15))
    for n in range(16):
        # floor() puts the threshold within one unit of 2^-32 below 2^32 F(n)
        assert -1e-14 <= cdf[n] - thr[n] / 2.0 ** 32 < 2.0 ** -32 + 1e-14


def test_poisson_thresholds_degenerate():
    # mu = 0: every threshold is 2^32, so no 32-bit word ever counts a jump
    assert oracle.poisson_thresholds(0.0) == [2 ** 32] * 16


def _many_draws(p, ks, ms):
    return [oracle.step_draws(p, k, m) for k in ks for m in ms]


def test_normals_are_standard():
    p = workloads.linear_family(8, M=64, Nt=64, lam=0.0)
    z = np.concatenate([dr["Z"][0] for dr in _many_draws(p, range(64), range(40))])
    assert z.size == 64 * 40 * 8
    assert stats.kstest(z, "norm").pvalue > 1e-3
    assert abs(z.mean()) < 4 / np.sqrt(z.size)
    assert abs(z.var() - 1) < 5 * np.sqrt(2 / z.size)
    # odd d: the second value of the last pair is discarded, the first is used
    p1 = workloads.lq_scalar(M=64, Nt=64)
    z1 = np.array([dr["Z"][0][0] for dr in _many_draws(p1, range(64), range(40))])
    assert stats.kstest(z1, "norm").pvalue > 1e-3


def test_jump_counts_are_poisson():
    p = workloads.lq_scalar(M=400, Nt=10).replace(lam=15.0)  # mu = lambda dt = 1.5
    mu = p.lam * p.dt
    n = np.array([dr["n"] for dr in _many_draws(p, range(10), range(400))])
    counts = np.bincount(n, minlength=9)[:9].astype(float)
    expected = stats.poisson.pmf(np.arange(9), mu) * n.size
    expected[-1] += stats.poisson.sf(8, mu) * n.size
    counts[-1] += (n > 8).sum()
    chi2 = ((counts - expected) ** 2 / expected).sum()
    assert stats.chi2.sf(chi2, df=8) > 1e-3


def test_jump_times_sizes_and_interarrivals():
    """Times are sorted and uniform within a step; the jumps of one path form a
    Poisson process, so the gaps between consecutive jump times are Exp(lambda)."""
    p = workloads.lq_scalar(M=8, Nt=400).replace(lam=40.0)
    dt = p.dt
    gaps, thetas, sizes = [], [], []
    for m in range(8):
        times = []
        for k in range(p.Nt):
            dr = oracle.step_draws(p, k, m)
            th = dr["theta"]
            assert np.all(np.diff(th) >= 0)
            assert np.isclose(dr["delta"].sum(), dt, rtol=0, atol=1e-15)
            thetas.extend(th)
            sizes.extend(dr["xi_hat"][:, 0])
            times.extend(k * dt + dt * th)
        gaps.extend(np.diff(times))
    assert stats.kstest(thetas, "uniform").pvalue > 1e-3
    assert stats.kstest(np.array(gaps) * p.lam, "expon").pvalue > 1e-3
    assert stats.kstest(sizes, "norm").pvalue > 1e-3


def test_uniform_jump_sizes():
    p = workloads.double_well(M=8, Nt=400).replace(lam=100.0)
    xs = []
    for m in range(4):
        for k in range(0, 400, 2):
            dr = oracle.step_draws(p, k, m)
            xs.extend(dr["xi_hat"].ravel())
    xs = np.array(xs)
    assert xs.min() > -1 and xs.max() < 1
    assert stats.kstest(xs, "uniform", args=(-1, 2)).pvalue > 1e-3


def test_streams_depend_on_seed_epoch_path_step():
    p = workloads.double_well(M=8, Nt=8)
    a = oracle.step_draws(p, 3, 5)["Z"][0]
    for q in (p.replace(seed=1), p.replace(epoch=1)):
        assert not np.allclose(oracle.step_draws(q, 3, 5)["Z"][0], a)
    assert not np.allclose(oracle.step_draws(p, 4, 5)["Z"][0], a)
    assert not np.allclose(oracle.step_draws(p, 3, 6)["Z"][0], a)


def test_poisson_count_boundaries():
    """The count is #{n : T_n <= w}: a word equal to a threshold counts it."""
    thr = oracle.poisson_thresholds(0.5)
    assert oracle.poisson_count(0, thr) == 0
    assert oracle.poisson_count(thr[0] - 1, thr) == 0
    assert oracle.poisson_count(thr[0], thr) == 1
    assert oracle.poisson_count(thr[1] - 1, thr) == 1
    assert oracle.poisson_count(thr[1], thr) == 2
    assert oracle.poisson_count(0xFFFFFFFF, thr) == sum(1 for t in thr if t <= 0xFFFFFFFF)


def test_normal_pair_radius_and_angle_words():
    """Convention: the first word sets the radius, the second the angle."""
    w_small = 0x00000200          # U = 1.5 * 2^-23: large radius
    w_quarter = 0x40000000        # U = 1/4 + 2^-24: angle pi/2 + tiny
    z0, z1 = oracle.normal_pair(w_small, w_quarter)
    r = np.sqrt(-2 * np.log(oracle.u01(w_small)))
    assert r > 5.5
    assert abs(z1 - r) < 1e-6 * r and abs(z0) < 1e-5 * r
    # angle 0 (U -> 2^-24): the pair lies on the positive first axis
    z0, z1 = oracle.normal_pair(0x80000000, 0)
    assert z0 > 0 and abs(z1) < 1e-6
