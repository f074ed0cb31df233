"""Seeded synthetic inputs shaped like the workloads of arXiv 2204.09131.

This module holds no part of the estimator or the searches: it only draws series.
Both the tests (CUDA path and oracle) and ``bench.py`` take their inputs from here.

Generator: SplitMix64 (Steele, Lea and Flood 2014), output number ``n`` of the stream
with state ``seed`` is ``mix(seed + n * 0x9E3779B97F4A7C15)``; uniforms are the top 53
bits; normals come from the Box-Muller transform in binary64 and are cast to float32.

Seed recipe: ``seed = 20220419 ^ (cfg << 40) ^ (series << 20) ^ stream``.

The relation shapes follow the paper's synthetic relations (Table "Identify different
types of correlation relations", Sec. 8.4.1): linear, quadratic, sinusoidal,
exponential; the planted-segment layout stands in for the paper's real datasets,
which are not available.
"""
from __future__ import annotations

import math

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_MASK = (1 << 64) - 1


def seed_for(cfg: int, series: int, stream: int = 0) -> int:
    return (20220419 ^ (cfg << 40) ^ (series << 20) ^ stream) & _MASK


def splitmix64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Outputs number offset+1 .. offset+n of the SplitMix64 stream with state ``seed``."""
    idx = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & _MASK) + idx * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Uniform doubles in [0, 1)."""
    return (splitmix64(seed, n, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal(seed: int, n: int) -> np.ndarray:
    """Standard normal doubles by Box-Muller (two uniforms per pair of outputs)."""
    half = (n + 1) // 2
    u = uniform(seed, 2 * half)
    u1 = 1.0 - u[0::2]              # (0, 1]
    u2 = u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    th = 2.0 * math.pi * u2
    out = np.empty(2 * half, dtype=np.float64)
    out[0::2] = r * np.cos(th)
    out[1::2] = r * np.sin(th)
    return out[:n]


def laplace(seed: int, n: int) -> np.ndarray:
    """Unit-variance Laplace doubles by inverse CDF."""
    u = uniform(seed, n) - 0.5
    b = 1.0 / math.sqrt(2.0)
    return -b * np.sign(u) * np.log1p(-2.0 * np.abs(u))


def uniform_unit(seed: int, n: int) -> np.ndarray:
    """Unit-variance uniform doubles on [-sqrt(3), sqrt(3))."""
    return (2.0 * uniform(seed, n) - 1.0) * math.sqrt(3.0)


def loguniform_int(u: float, lo: int, hi: int) -> int:
    return int(round(math.exp(math.log(lo) + u * (math.log(hi) - math.log(lo)))))


def quantize(v: np.ndarray, step_inv: float = 10.0) -> np.ndarray:
    """(float)(nearbyint((double)v * 10) / 10): values on a 0.1 grid, heavy ties."""
    return (np.rint(np.asarray(v, dtype=np.float64) * step_inv) / step_inv).astype(np.float32)


# ---------------------------------------------------------------------------
# Workloads
# ---------------------------------------------------------------------------

def planted_small_pair(n: int = 2000, cfg: int = 1):
    """One pair: X ~ N(0,1); Y = X + N(0, 0.1^2) on [400, 700), Y = X^2 + N(0, 0.1^2) on
    [1200, 1500), Y ~ N(0,1) iid elsewhere.  Returns float32 (x, y)."""
    x = normal(seed_for(cfg, 0), n)
    y = normal(seed_for(cfg, 1), n)
    e = 0.1 * normal(seed_for(cfg, 2), n)
    a0, a1 = min(400, n), min(700, n)
    b0, b1 = min(1200, n), min(1500, n)
    y[a0:a1] = x[a0:a1] + e[a0:a1]
    y[b0:b1] = x[b0:b1] ** 2 + e[b0:b1]
    return x.astype(np.float32), y.astype(np.float32)


RELATIONS = ("linear", "quadratic", "sine", "exp")


def _relation(kind: str, x: np.ndarray, sign: float) -> np.ndarray:
    if kind == "linear":
        return sign * x
    if kind == "quadratic":
        return x * x
    if kind == "sine":
        return np.sin(3.0 * x)
    return np.exp(x)


def planted_pair(cfg: int, pair: int, n: int, coverage: float = 0.3, len_lo: int = 50,
                 len_hi: int = 5000, snrs=(0.5, 2.0, 10.0), background: str = "gaussian"):
    """A pair of float32 series with planted relation segments.

    Background: iid N(0,1) for X and Y (``background="gaussian"``), or independent noise
    segments whose family is drawn per gap from {gaussian, uniform, laplace}
    (``background="mixed"``).  Segments: lengths log-uniform in [len_lo, len_hi], gaps
    random, until ``coverage`` of the series is covered; Y = sqrt(s/(1+s)) f(X)/std(f)
    + sqrt(1/(1+s)) N(0,1) with f drawn from linear / quadratic / sin(3X) / exp(X)
    and the signal-to-noise ratio s drawn from ``snrs``.
    Returns (x, y, segments) with segments = [(start, end_exclusive, kind, snr)].
    """
    sx = seed_for(cfg, 2 * pair, 0)
    sy = seed_for(cfg, 2 * pair + 1, 0)
    x = normal(sx, n)
    y = normal(sy, n)
    if background == "mixed":
        x = _mixed_noise(seed_for(cfg, 2 * pair, 7), n)
        y = _mixed_noise(seed_for(cfg, 2 * pair + 1, 7), n)
    ctl = uniform(seed_for(cfg, 2 * pair, 1), 4 * (n // max(len_lo, 1) + 8))
    noise = normal(seed_for(cfg, 2 * pair, 2), n)
    segs = []
    q = 0
    gap_ratio = (1.0 - coverage) / max(coverage, 1e-9)
    L0 = loguniform_int(ctl[q], len_lo, len_hi); q += 1
    pos = int(ctl[q] * 2.0 * gap_ratio * L0); q += 1
    covered = 0
    while covered < coverage * n and q + 4 <= ctl.shape[0]:
        L = loguniform_int(ctl[q], len_lo, len_hi); q += 1
        if pos + L > n:
            break
        kind = RELATIONS[int(ctl[q] * len(RELATIONS)) % len(RELATIONS)]; q += 1
        snr = float(snrs[int(ctl[q] * len(snrs)) % len(snrs)]); q += 1
        sign = 1.0 if ctl[q] < 0.5 else -1.0; q += 1
        xs = x[pos:pos + L]
        f = _relation(kind, xs, sign)
        sd = f.std()
        f = (f - f.mean()) / (sd if sd > 0 else 1.0)
        y[pos:pos + L] = math.sqrt(snr / (1.0 + snr)) * f + \
            math.sqrt(1.0 / (1.0 + snr)) * noise[pos:pos + L]
        segs.append((pos, pos + L, kind, snr))
        covered += L
        gap = int(ctl[q] * 2.0 * gap_ratio * L) if q < ctl.shape[0] else 0; q += 1
        pos += L + gap
    return x.astype(np.float32), y.astype(np.float32), segs


def tied_pair(pair: int, n: int, cfg: int = 5):
    """A tie-heavy pair: both series of :func:`planted_pair` with planted multi-scale
    relations of 100..50,000 samples, quantised to 0.1 steps (many equal values, equal
    distances and duplicate points).  Returns float32 (x, y, segments)."""
    x, y, segs = planted_pair(cfg, pair, n, len_lo=100, len_hi=min(50000, max(100, n // 2)))
    return quantize(x), quantize(y), segs


def _mixed_noise(seed: int, n: int) -> np.ndarray:
    """Independent noise in segments of 100..10000 samples, each from a family drawn
    from {gaussian, uniform, laplace} (unit variance)."""
    ctl = uniform(seed, 2 * (n // 100 + 4))
    out = np.empty(n, dtype=np.float64)
    pos, q, part = 0, 0, 0
    while pos < n:
        L = min(n - pos, loguniform_int(ctl[q % ctl.shape[0]], 100, 10000)); q += 1
        fam = int(ctl[q % ctl.shape[0]] * 3) % 3; q += 1
        s = (seed + 0x1000 * (part + 1)) & _MASK
        if fam == 0:
            out[pos:pos + L] = normal(s, L)
        elif fam == 1:
            out[pos:pos + L] = uniform_unit(s, L)
        else:
            out[pos:pos + L] = laplace(s, L)
        pos += L
        part += 1
    return out


def gaussian_pair(seed: int, m: int, rho: float):
    """m samples of a bivariate normal with correlation rho, float32."""
    a = normal(seed, m)
    b = normal(seed ^ 0x5A5A5A5A, m)
    return a.astype(np.float32), (rho * a + math.sqrt(1.0 - rho * rho) * b).astype(np.float32)


def stride_windows(n: int, sizes, stride: int = 1):
    """All windows [s, s+m-1] of the given sizes at the given stride: list of (start, m)."""
    out = []
    for m in sizes:
        for s in range(0, n - m + 1, stride):
            out.append((s, m))
    return out
