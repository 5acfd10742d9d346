"""Counter-based random operators of the sketches (oracle side).

The paper only says that a seed is drawn and shared (Section 2.3: the Gaussian
sketch "can be drawn from a seed during the product", the SRHT uses random
signs and a uniform row sample).  It fixes no generator, so this project fixes
one, written here from its published definition and written again,
independently, in the CUDA library:

* ``mix64`` is the SplitMix64 output function (Steele, Lea & Flood,
  "Fast splittable pseudorandom number generators", OOPSLA 2014).
* ``counter_hash(seed, stream, i) = mix64(seed*G + stream*2**56 + i mod 2**64)``
  with ``G = 0x9E3779B97F4A7C15``.  ``mix64`` is a bijection of 64-bit words,
  so distinct counters inside one stream give distinct outputs.
* Signs of the SRHT (stream 1): ``D_i = -1`` when the top bit of the hash is set.
* Row sample of the SRHT (stream 2): the ``k`` indices in ``[0, N)`` with the
  smallest hash, returned in increasing order (sampling without replacement).
* Gaussian entries (streams 3 and 4, counter ``r*n + c`` for entry (r, c) of the
  k x n operator): Box-Muller, ``g = sqrt(-2 ln u1) cos(2 pi u2)`` with
  ``u1 = (h3 >> 11 + 1) 2^-53`` and ``u2 = (h4 >> 11) 2^-53``.  ``ln`` and ``cos``
  are evaluated by the atanh and Taylor series below using only correctly
  rounded ``+ - * /`` and ``sqrt`` (no fused multiply-add), so the value is the
  same bit pattern on any IEEE machine that evaluates the same expression.
"""

from __future__ import annotations

import numpy as np

MASK64 = (1 << 64) - 1
GOLDEN = 0x9E3779B97F4A7C15
STREAM_SIGN = 1
STREAM_SAMPLE = 2
STREAM_GAUSS_U1 = 3
STREAM_GAUSS_U2 = 4

_U = np.uint64


def mix64(z):
    """SplitMix64 output function on a uint64 array (wrap-around arithmetic)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> _U(30))) * _U(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> _U(27))) * _U(0x94D049BB133111EB)
    return z ^ (z >> _U(31))


def splitmix64_sequence(state: int, count: int) -> list[int]:
    """The SplitMix64 generator itself: state += G, output mix64(state)."""
    out = []
    for _ in range(count):
        state = (state + GOLDEN) & MASK64
        out.append(int(mix64(np.array([state], dtype=np.uint64))[0]))
    return out


def counter_base(seed: int, stream: int) -> int:
    return (seed * GOLDEN + (stream << 56)) & MASK64


def counter_hash(seed: int, stream: int, i) -> np.ndarray:
    """mix64(seed*G + stream*2^56 + i) for an integer array ``i``."""
    i = np.asarray(i, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return mix64(_U(counter_base(seed, stream)) + i)


def srht_signs(seed: int, N: int) -> np.ndarray:
    """Diagonal D of the SRHT (Section 2.3): +1.0 / -1.0 as float64, length N."""
    h = counter_hash(seed, STREAM_SIGN, np.arange(N, dtype=np.uint64))
    return np.where((h >> _U(63)) == _U(1), -1.0, 1.0)


def srht_sample(seed: int, N: int, k: int) -> np.ndarray:
    """Rows kept by P (Section 2.3): the k smallest keys, increasing index order."""
    if not 0 < k <= N:
        raise ValueError("need 0 < k <= N")
    keys = counter_hash(seed, STREAM_SAMPLE, np.arange(N, dtype=np.uint64))
    order = np.argsort(keys, kind="stable")
    return np.sort(order[:k]).astype(np.int64)


# ---------------------------------------------------------------------------
# Elementary functions from their series, basic IEEE operations only.
# ---------------------------------------------------------------------------

LN2 = 0.6931471805599453  # nearest double to ln 2
HALF_PI = 1.5707963267948966  # nearest double to pi/2
ATANH_TERMS = 12  # odd powers s^1 .. s^23; |s| <= 3 - 2 sqrt 2 makes s^25/25 < 1e-19
TRIG_TERMS = 10  # y^0 .. y^19 with |y| <= pi/4


def _inverse_odd() -> list[float]:
    """1/(2i+1) for i < ATANH_TERMS, each one correctly rounded division."""
    return [1.0 / float(2 * i + 1) for i in range(ATANH_TERMS)]


def _inverse_factorials() -> list[float]:
    """f[0] = 1, f[n] = f[n-1] / n in double precision (n <= 2*TRIG_TERMS)."""
    f = [1.0]
    for n in range(1, 2 * TRIG_TERMS):
        f.append(f[-1] / float(n))
    return f


def series_log(x: np.ndarray) -> np.ndarray:
    """ln x for x in (0, 1]: x = f 2^e with f in [1/sqrt2, sqrt2),
    ln f = 2 atanh((f-1)/(f+1)) summed as a Horner polynomial in s^2."""
    x = np.asarray(x, dtype=np.float64)
    f, e = np.frexp(x)  # f in [0.5, 1), exact
    low = f < 0.7071067811865476
    f = np.where(low, f * 2.0, f)  # exact scaling
    e = np.where(low, e - 1, e).astype(np.float64)
    s = (f - 1.0) / (f + 1.0)
    s2 = s * s
    inv = _inverse_odd()
    p = np.full_like(s, inv[-1])
    for c in reversed(inv[:-1]):
        p = p * s2 + c
    return e * LN2 + 2.0 * (s * p)


def _sin_cos_small(y: np.ndarray):
    """sin y and cos y for 0 <= y <= pi/4 by their Taylor series (Horner in y^2)."""
    f = _inverse_factorials()
    y2 = y * y
    # cos: sum_k (-1)^k y^(2k)/(2k)!
    pc = np.full_like(y, f[2 * (TRIG_TERMS - 1)] * (-1.0) ** (TRIG_TERMS - 1))
    for kk in range(TRIG_TERMS - 2, -1, -1):
        pc = pc * y2 + (f[2 * kk] if kk % 2 == 0 else -f[2 * kk])
    # sin: y * sum_k (-1)^k y^(2k)/(2k+1)!
    ps = np.full_like(y, f[2 * TRIG_TERMS - 1] * (-1.0) ** (TRIG_TERMS - 1))
    for kk in range(TRIG_TERMS - 2, -1, -1):
        ps = ps * y2 + (f[2 * kk + 1] if kk % 2 == 0 else -f[2 * kk + 1])
    return y * ps, pc


def series_cos_turns(t: np.ndarray) -> np.ndarray:
    """cos(2 pi t) for t in [0, 1) via quarter-turn reduction (all reductions exact)."""
    t = np.asarray(t, dtype=np.float64)
    t4 = 4.0 * t
    q = np.floor(t4)
    r = t4 - q  # in [0, 1)
    flip = r > 0.5
    rr = np.where(flip, 1.0 - r, r)
    y = HALF_PI * rr
    sn, cs = _sin_cos_small(y)
    # cos(pi/2 r) and sin(pi/2 r) for the unreduced r
    c_r = np.where(flip, sn, cs)
    s_r = np.where(flip, cs, sn)
    qi = q.astype(np.int64)
    return np.select([qi == 0, qi == 1, qi == 2], [c_r, -s_r, -c_r], default=s_r)


def gaussian_values(seed: int, counters: np.ndarray) -> np.ndarray:
    """Box-Muller N(0,1) values for the given counters, in float64."""
    counters = np.asarray(counters, dtype=np.uint64)
    h1 = counter_hash(seed, STREAM_GAUSS_U1, counters)
    h2 = counter_hash(seed, STREAM_GAUSS_U2, counters)
    u1 = ((h1 >> _U(11)) + _U(1)).astype(np.float64) * (2.0 ** -53)
    u2 = (h2 >> _U(11)).astype(np.float64) * (2.0 ** -53)
    rad = np.sqrt(-2.0 * series_log(u1))
    return rad * series_cos_turns(u2)


# ---------------------------------------------------------------------------
# Storage rounding of the Gaussian entries.
# ---------------------------------------------------------------------------

DTYPES = ("f64", "f32", "bf16", "f16")


def bf16_round(x32: np.ndarray) -> np.ndarray:
    """Round float32 values to bfloat16 (round to nearest, ties to even);
    returns the bfloat16 values widened to float32."""
    b = np.asarray(x32, dtype=np.float32).view(np.uint32).astype(np.uint64)
    bias = _U(0x7FFF) + ((b >> _U(16)) & _U(1))
    r = ((b + bias) >> _U(16)) << _U(16)
    return r.astype(np.uint32).view(np.float32)


def round_to_dtype(x64: np.ndarray, dtype: str) -> np.ndarray:
    """Value stored for a float64 number in the given format, returned as float64.
    Narrow formats go through float32 first (two roundings, both to nearest even)."""
    x64 = np.asarray(x64, dtype=np.float64)
    if dtype == "f64":
        return x64.copy()
    x32 = x64.astype(np.float32)
    if dtype == "f32":
        return x32.astype(np.float64)
    if dtype == "bf16":
        return bf16_round(x32).astype(np.float64)
    if dtype == "f16":
        return x32.astype(np.float16).astype(np.float64)
    raise ValueError(dtype)


def gaussian_block(seed: int, n: int, rows, cols, dtype: str = "f64") -> np.ndarray:
    """Entries G[r, c] of the k x n standard Gaussian matrix (before the 1/sqrt(k)
    factor of Section 2.3) for r in ``rows`` and c in ``cols``, rounded to the
    storage format ``dtype``."""
    rows = np.asarray(rows, dtype=np.uint64)
    cols = np.asarray(cols, dtype=np.uint64)
    ctr = rows[:, None] * _U(n) + cols[None, :]
    return round_to_dtype(gaussian_values(seed, ctr.ravel()), dtype).reshape(ctr.shape)
