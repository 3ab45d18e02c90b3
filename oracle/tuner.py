"""Tuner oracle -- TEST INFRASTRUCTURE ONLY.

Plain restatements used to check the library's auto-tuner (kt_tune):

* the objective, Eq. 1 of the paper (Section 3.1): x* = argmin over the search
  space of the measured runtime f(K_x); ties are broken by the
  lexicographically smallest (band, tile, threads, cols_per_block, unroll);
* the search spaces: the paper's own (Section 5.2 table) and the one this
  library tunes over (tile x band x threads x cols_per_block x unroll); which
  points of a space are valid is a user-supplied constraint (Section 3.1), here
  the library's launch contract, so it is not restated here;
* SplitMix64 (Steele, Lea & Flood 2014), the counter-based generator both
  sides use to draw the random-5% baseline sample;
* summary ratios: optimal / median / default runtimes.
"""
from __future__ import annotations

import itertools

import numpy as np

TILES = (16, 32, 64, 128)
BANDS = (16, 32, 64)
THREADS = tuple(range(64, 1025, 64))
CPBS = (1, 2, 4, 8)
UNROLLS = (1, 2, 4)

MASK64 = (1 << 64) - 1


def space(tiles=TILES, bands=BANDS, threads=THREADS, cpbs=CPBS, unrolls=UNROLLS):
    """All configurations, ordered lexicographically by (band, tile, threads, cpb, unroll)."""
    return [(b, t, th, c, u) for b, t, th, c, u in itertools.product(sorted(bands), sorted(tiles), sorted(threads),
                                                                      sorted(cpbs), sorted(unrolls))]


def argmin(times: dict):
    """Eq. 1: the configuration with the smallest runtime; ties -> smallest tuple."""
    finite = {k: v for k, v in times.items() if v is not None and np.isfinite(v)}
    if not finite:
        return None
    best = min(finite.values())
    return min(k for k, v in finite.items() if v == best)


def ratios(times: dict, default_cfg):
    """(optimal_ms, median_ms, default_ms, median/optimal, default/optimal)."""
    vals = np.array([v for v in times.values() if v is not None and np.isfinite(v)])
    opt = float(vals.min())
    med = float(np.median(vals))
    dflt = times.get(default_cfg)
    return opt, med, dflt, med / opt, (dflt / opt if dflt else None)


def splitmix64(state: int):
    """One SplitMix64 step: returns (new_state, output)."""
    state = (state + 0x9E3779B97F4A7C15) & MASK64
    z = state
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return state, z ^ (z >> 31)


def random_subset(count: int, k: int, seed: int):
    """k distinct indices of range(count) by a partial Fisher-Yates shuffle driven by SplitMix64."""
    idx = list(range(count))
    state = seed & MASK64
    for i in range(min(k, count)):
        state, r = splitmix64(state)
        j = i + r % (count - i)
        idx[i], idx[j] = idx[j], idx[i]
    return idx[: min(k, count)]
