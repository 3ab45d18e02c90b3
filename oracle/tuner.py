"""Tuner oracle -- TEST INFRASTRUCTURE ONLY.

Plain restatements used to check the library's auto-tuner (kt_tune):

* the objective, Eq. 1 of the paper (Section 3.1): x* = argmin over the search
  space of the measured runtime f(K_x); ties are broken by the
  lexicographically smallest (band, tile, threads, cols_per_block, unroll);
* the search spaces: the paper's own (Section 5.2 table) and the one this
  library tunes over (tile x band x threads x cols_per_block x unroll);
* the validity rule of the trailing-update kernels, written out from its
  definition (the block tiles the strip into 4-column groups and the band into
  groups of 1, 2, 4 or 8 reflectors; a staged tile splits into whole 4-row
  sub-blocks per thread; shared memory <= 227 KB);
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


def smem_bytes(side, elem, nb, tile, w):
    """Shared memory of the register-tiled update: X tile, V tile (padded by 4), W."""
    return elem * (tile * w + tile * (nb + 4) + nb * w)


def tma_smem_bytes(b, tile, stages):
    """Shared memory of the TMA-streamed FP32 kernels: `stages` copies of the larger
    stage (QR projection: tile/32 boxes of 32 rows x 128 columns of X plus 32 x b of V;
    column-streaming kernels: 64/b boxes of 32 rows x tile columns plus tile x b of Q),
    plus 1 KiB to align the 128-byte-swizzled boxes."""
    qr = (tile // 32) * (128 * 128 + b * 128)
    cols = (64 // b) * tile * 128 + tile * b * 4
    return stages * max(qr, cols) + 1024


def valid_tma(cfg):
    """Validity of (band, tile, threads, cpb, unroll) for the TMA-streamed FP32 kernels,
    which read it as (band, stage depth, consumer threads, pipeline stages, waves):
    band 16/32/64; stage depth 32/64/128; 2, 4 or 8 consumer warps, a whole number
    of 16-reflector groups; 2, 4 or 8 stages; 1, 2 or 4 waves; shared memory
    <= 226 KiB."""
    b, tile, threads, cpb, unroll = cfg
    if b not in (16, 32, 64) or tile not in (32, 64, 128) or threads not in (64, 128, 256):
        return False
    if (threads // 32) % (b // 16):
        return False
    if cpb not in (2, 4, 8) or unroll not in (1, 2, 4):
        return False
    return tma_smem_bytes(b, tile, cpb) <= 226 * 1024


def valid(side, elem, cfg):
    """Validity of (band, tile, threads, cpb, unroll) for the trailing-update kernels.
    FP32 at band 16/32/64 runs the TMA-streamed kernels (valid_tma).  Otherwise
    (band widths divisible by 4) the register-tiled kernels: the block is (w/4 column
    groups) x (band/R reflector groups) with R in {1, 2, 4, 8}; a staged tile gives
    each thread a whole number of 4-row sub-blocks; shared memory <= 227 KiB."""
    b, tile, threads, cpb, unroll = cfg
    if elem == 4 and b in (16, 32, 64):
        return valid_tma(cfg)
    if b % 4 or not (4 <= b <= 64):
        return False
    if threads % 32 or not (32 <= threads <= 1024):
        return False
    if cpb not in (1, 2, 4, 8) or unroll not in (1, 2, 4):
        return False
    w = 32 * cpb
    ncg = w // 4
    if threads % ncg:
        return False
    nrg = threads // ncg
    if b % nrg or b // nrg not in (1, 2, 4, 8):
        return False
    if not (4 <= tile <= 256) or tile % (4 * nrg):
        return False
    return smem_bytes(side, elem, b, tile, w) <= 227 * 1024


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
