"""Pins of the oracle's random operators (no GPU)."""

import math
import os

import numpy as np
import pytest

from oracle import rng

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_lines(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [ln.strip() for ln in f if ln.strip() and not ln.startswith("#")]


def test_splitmix64_published_outputs():
    want = [int(h, 16) for h in _golden_lines("splitmix64_seed0.txt")]
    assert rng.splitmix64_sequence(0, len(want)) == want


def _py_mix64(z):
    M = (1 << 64) - 1
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M
    return z ^ (z >> 31)


def test_counter_hash_definition_with_python_integers():
    seed, stream = 123456789, 2
    i = np.array([0, 1, 7, 2**40 + 3], dtype=np.uint64)
    got = rng.counter_hash(seed, stream, i)
    for ii, g in zip(i.tolist(), got.tolist()):
        x = (seed * 0x9E3779B97F4A7C15 + (stream << 56) + ii) & ((1 << 64) - 1)
        assert g == _py_mix64(x)


def test_mix64_is_a_bijection_on_a_sample():
    # inverse of x ^= x >> s and of multiplication by an odd constant mod 2^64
    M = (1 << 64) - 1

    def unxorshift(y, s):
        x = y
        for _ in range(64 // s + 1):
            x = y ^ (x >> s)
        return x

    def inv(y):
        y = unxorshift(y, 31)
        y = (y * pow(0x94D049BB133111EB, -1, 1 << 64)) & M
        y = unxorshift(y, 27)
        y = (y * pow(0xBF58476D1CE4E5B9, -1, 1 << 64)) & M
        return unxorshift(y, 30)

    xs = np.random.default_rng(0).integers(0, 2**63, 64, dtype=np.uint64) * np.uint64(2) + np.uint64(1)
    for x, y in zip(xs.tolist(), rng.mix64(xs).tolist()):
        assert inv(y) == x


def test_signs_are_the_top_bit_and_balanced():
    N = 1 << 16
    d = rng.srht_signs(7, N)
    h = rng.counter_hash(7, rng.STREAM_SIGN, np.arange(N, dtype=np.uint64))
    assert np.array_equal(d < 0, (h >> np.uint64(63)) == 1)
    assert set(np.unique(d)) == {-1.0, 1.0}
    # binomial(N, 1/2): |sum| beyond 5 sigma is a broken generator
    assert abs(d.sum()) < 5 * math.sqrt(N)


@pytest.mark.parametrize("N,k", [(64, 1), (64, 64), (1000, 17), (4096, 512)])
def test_sample_is_k_smallest_keys_in_increasing_order(N, k):
    idx = rng.srht_sample(11, N, k)
    keys = rng.counter_hash(11, rng.STREAM_SAMPLE, np.arange(N, dtype=np.uint64)).tolist()
    brute = sorted(sorted(range(N), key=lambda i: keys[i])[:k])
    assert idx.tolist() == brute
    assert len(set(idx.tolist())) == k and np.all(np.diff(idx) > 0)


def test_sample_is_uniform_over_positions():
    N, k, trials = 256, 32, 400
    counts = np.zeros(N)
    for s in range(trials):
        counts[rng.srht_sample(s, N, k)] += 1
    expect = trials * k / N
    chi2 = ((counts - expect) ** 2 / expect).sum()
    assert chi2 < N + 6 * math.sqrt(2 * N)  # chi-square with N-1 dof, generous bound


def test_series_log_matches_math_log():
    x = np.concatenate([np.random.default_rng(1).uniform(0, 1, 20000) + 1e-300,
                        2.0 ** -np.arange(0, 54), [1.0, 0.5, 0.75, 1 - 2**-53]])
    got = rng.series_log(x)
    ref = np.array([math.log(v) for v in x])
    assert np.all(np.abs(got - ref) <= 4 * np.spacing(np.maximum(np.abs(ref), 1e-300)) + 1e-300)
    assert rng.series_log(np.array([1.0]))[0] == 0.0


def test_series_cos_turns_matches_math_cos():
    t = np.concatenate([np.random.default_rng(2).uniform(0, 1, 20000), np.arange(16) / 16])
    got = rng.series_cos_turns(t)
    ref = np.array([math.cos(2 * math.pi * v) for v in t])
    assert np.max(np.abs(got - ref)) < 2e-15
    special = rng.series_cos_turns(np.array([0.0, 0.25, 0.5, 0.75]))
    assert special[0] == 1.0 and special[1] == 0.0 and special[2] == -1.0 and special[3] == 0.0


def test_gaussian_values_are_standard_normal():
    from scipy import stats

    g = rng.gaussian_values(42, np.arange(200000, dtype=np.uint64))
    assert abs(g.mean()) < 5 / math.sqrt(g.size)
    assert abs(g.var() - 1) < 0.02
    assert stats.kstest(g, "norm").pvalue > 1e-4
    # Box-Muller by definition, with library log/cos, agrees to rounding
    h1 = rng.counter_hash(42, 3, np.arange(100, dtype=np.uint64))
    h2 = rng.counter_hash(42, 4, np.arange(100, dtype=np.uint64))
    u1 = ((h1 >> np.uint64(11)) + np.uint64(1)).astype(np.float64) * 2.0**-53
    u2 = (h2 >> np.uint64(11)).astype(np.float64) * 2.0**-53
    ref = np.sqrt(-2 * np.log(u1)) * np.cos(2 * np.pi * u2)
    assert np.max(np.abs(g[:100] - ref)) < 1e-13


def _bf16_neighbours(x):
    b = np.float32(x).view(np.uint32) & np.uint32(0xFFFF0000)
    lo = np.uint32(b).view(np.float32)
    hi = np.uint32(b + np.uint32(0x10000)).view(np.float32)
    return float(lo), float(hi), int(b >> np.uint32(16))


def test_bf16_rounding_is_nearest_even():
    xs = np.random.default_rng(3).standard_normal(3000).astype(np.float32)
    xs = np.concatenate([xs, np.float32([1 + 2**-8, 1 + 3 * 2**-8, -(1 + 2**-8), 1.0])])
    got = rng.bf16_round(xs)
    for x, g in zip(xs.tolist(), got.tolist()):
        lo, hi, lobits = _bf16_neighbours(x)
        dlo, dhi = abs(x - lo), abs(x - hi)
        want = lo if dlo < dhi else hi if dhi < dlo else (lo if lobits % 2 == 0 else hi)
        assert g == want


def test_round_to_dtype_f16_and_f32():
    x = np.random.default_rng(4).standard_normal(1000)
    assert np.array_equal(rng.round_to_dtype(x, "f32"), x.astype(np.float32).astype(np.float64))
    assert np.array_equal(rng.round_to_dtype(x, "f16"), x.astype(np.float32).astype(np.float16).astype(np.float64))
    assert np.array_equal(rng.round_to_dtype(x, "f64"), x)
