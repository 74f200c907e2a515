"""Seeded synthetic time series shaped like the paper's workloads.

This module is shared by the FP64 oracle side (tests) and the CUDA side
(tests, bench, smoke).  It only draws numbers: it holds none of the
discord arithmetic (no means, deviations, distances or thresholds), so the
two sides share inputs and nothing else.

Every series is float32 (the paper's time series are real-valued, Eq. 1;
the C ABI takes float32).  All randomness comes from numpy's PCG64 with an
explicit seed, so a given (config, seed) always yields the same bytes.

Workloads (the paper's real datasets, Tab. 1 of Sec. 4.1, are not shipped;
these stand in for their shapes):

* ``tiny``      -- Gaussian random walk, n=2000, seed 0, lengths 32..40, top-1.
* ``sine100k``  -- sine of period 200 + N(0, 0.1^2) noise, n=100000, five
                   length-150 phase-flipped 1.5x-amplitude anomalies,
                   lengths 128..256, top-3 (stands in for the periodic ECG /
                   space-shuttle series).
* ``rw250k``    -- Gaussian random walk, n=250000, seed 7, lengths 64..512,
                   top-1 (stands in for RandomWalk1M/2M).
* ``batch256``  -- 256 series, n ~ U[5000, 60000], half random walks, half
                   noisy sines with 1-3 anomalies; per-series lengths
                   [minL, minL+64], minL ~ U[32, 256], top-1.
* ``beats1m``   -- quasi-periodic Gaussian-bump beats, n=1000000, period
                   250 +- 10, N(0, 0.05^2) noise, 20 widened or inverted
                   beats, lengths 100..1000, top-1 plus the heatmap
                   (stands in for ECG / Koski-ECG and the PolyTER case
                   study of Sec. 5).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Workload",
    "random_walk",
    "noisy_sine",
    "beats",
    "pick_starts",
    "workload",
    "WORKLOADS",
    "points_x_lengths",
]


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def random_walk(n: int, seed: int, t0: float = 0.0) -> np.ndarray:
    """Cumulative sum of N(0, 1) steps starting at ``t0`` (float32)."""
    steps = _rng(seed).standard_normal(n)
    steps[0] = 0.0
    return (t0 + np.cumsum(steps)).astype(np.float32)


def pick_starts(rng: np.random.Generator, n: int, count: int, length: int,
                gap: int, margin: int) -> list[int]:
    """Draw ``count`` anomaly starts uniformly, pairwise at least ``gap`` apart,
    each at least ``margin`` away from both ends of the series."""
    lo, hi = margin, n - length - margin
    if hi <= lo:
        raise ValueError("series too short for the requested anomalies")
    starts: list[int] = []
    for _ in range(100000):
        if len(starts) == count:
            break
        s = int(rng.integers(lo, hi))
        if all(abs(s - o) >= gap for o in starts):
            starts.append(s)
    if len(starts) != count:
        raise ValueError("could not place anomalies")
    return sorted(starts)


def noisy_sine(n: int, period: float, noise: float, seed: int,
               anomalies: list[tuple[int, int]] = (),
               flip_amp: float = 1.5) -> np.ndarray:
    """``sin(2 pi k / period) + N(0, noise^2)``; each ``(start, length)`` in
    ``anomalies`` replaces that window by the phase-flipped sine scaled by
    ``flip_amp`` (plus the same noise)."""
    rng = _rng(seed)
    k = np.arange(n, dtype=np.float64)
    x = np.sin(2.0 * np.pi * k / period)
    for s, ln in anomalies:
        x[s:s + ln] = -flip_amp * np.sin(2.0 * np.pi * k[s:s + ln] / period)
    x += noise * rng.standard_normal(n)
    return x.astype(np.float32)


def beats(n: int, seed: int, period: int = 250, jitter: int = 10,
          width: float = 15.0, noise: float = 0.05, n_odd: int = 20) -> tuple[np.ndarray, list[int]]:
    """Gaussian-bump beats every ``period +- U[-jitter, jitter]`` samples plus
    N(0, noise^2); ``n_odd`` beats (drawn with ``seed``) are abnormal: the
    first half widened 2x, the second half inverted.  Returns the series and
    the centres of the abnormal beats."""
    rng = _rng(seed)
    centres = []
    c = period // 2
    while c < n - period // 2:
        centres.append(c)
        c += period + int(rng.integers(-jitter, jitter + 1))
    centres = np.asarray(centres)
    odd_pos = np.sort(rng.choice(np.arange(4, len(centres) - 4), size=n_odd, replace=False))
    widened = set(odd_pos[: n_odd // 2].tolist())
    inverted = set(odd_pos[n_odd // 2:].tolist())
    x = noise * rng.standard_normal(n)
    half = int(8 * width)
    for b, cc in enumerate(centres):
        w = width * (2.0 if b in widened else 1.0)
        amp = -1.0 if b in inverted else 1.0
        lo, hi = max(0, cc - 2 * half), min(n, cc + 2 * half + 1)
        k = np.arange(lo, hi, dtype=np.float64)
        x[lo:hi] += amp * np.exp(-0.5 * ((k - cc) / w) ** 2)
    return x.astype(np.float32), [int(centres[b]) for b in odd_pos]


@dataclass
class Workload:
    """One discord-discovery job: series plus the length range and top-K."""
    name: str
    series: list[np.ndarray]
    minL: list[int]
    maxL: list[int]
    topK: int
    heatmap: bool = False
    notes: dict = field(default_factory=dict)

    @property
    def units(self) -> int:
        """Points x lengths: sum over series and lengths of n - m + 1."""
        return points_x_lengths([len(s) for s in self.series], self.minL, self.maxL)


def points_x_lengths(ns, minLs, maxLs) -> int:
    tot = 0
    for n, a, b in zip(ns, minLs, maxLs):
        for m in range(a, b + 1):
            tot += n - m + 1
    return tot


def _tiny() -> Workload:
    return Workload("tiny", [random_walk(2000, seed=0)], [32], [40], 1)


def _sine100k() -> Workload:
    n, minL, maxL, alen = 100_000, 128, 256, 150
    starts = pick_starts(_rng(2), n, 5, alen, gap=2 * maxL, margin=2 * maxL)
    x = noisy_sine(n, 200.0, 0.1, seed=2002, anomalies=[(s, alen) for s in starts])
    return Workload("sine100k", [x], [minL], [maxL], 3, notes={"anomaly_starts": starts})


def _rw250k() -> Workload:
    return Workload("rw250k", [random_walk(250_000, seed=7)], [64], [512], 1)


def _batch256(count: int = 256) -> Workload:
    rng = _rng(4)
    series, mins, maxs, starts_all = [], [], [], []
    for s in range(count):
        n = int(rng.integers(5000, 60001))
        minL = int(rng.integers(32, 257))
        maxL = minL + 64
        sub_seed = int(rng.integers(0, 2**31 - 1))
        if s % 2 == 0:
            x = random_walk(n, seed=sub_seed)
            st = []
        else:
            period = float(rng.uniform(50.0, 400.0))
            na = int(rng.integers(1, 4))
            alen = int(rng.integers(minL, minL + 65))
            st = pick_starts(rng, n, na, alen, gap=2 * maxL, margin=2 * maxL)
            x = noisy_sine(n, period, 0.1, seed=sub_seed, anomalies=[(a, alen) for a in st])
        series.append(x)
        mins.append(minL)
        maxs.append(maxL)
        starts_all.append(st)
    return Workload("batch256", series, mins, maxs, 1, notes={"anomaly_starts": starts_all})


def _beats1m() -> Workload:
    x, odd = beats(1_000_000, seed=5)
    return Workload("beats1m", [x], [100], [1000], 1, heatmap=True, notes={"odd_beats": odd})


WORKLOADS = {
    "tiny": _tiny,
    "sine100k": _sine100k,
    "rw250k": _rw250k,
    "batch256": _batch256,
    "beats1m": _beats1m,
}


def workload(name: str) -> Workload:
    """Build the named workload (deterministic)."""
    return WORKLOADS[name]()
