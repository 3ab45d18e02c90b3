"""Pins for the tuner oracle (Eq. 1 argmin, search spaces, SplitMix64)."""
import os

import numpy as np

from oracle import tuner

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def read_space(name):
    vals = {}
    for line in open(os.path.join(GOLDEN, name)):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        k, *v = line.split()
        vals[k] = [int(x) for x in v]
    return vals


def test_paper_search_space_size():
    # Section 5.2's table: TS x TH x split-K x CPB = 5 * 5 * 8 * 8
    sp = read_space("paper_search_space.txt")
    pts = tuner.space(tiles=sp["tile_size_TS"], bands=sp["tile_height_TH"], threads=sp["split_k_K"],
                      cpbs=sp["cols_per_block_CPB"], unrolls=(1,))
    assert len(pts) == 1600
    assert len(set(pts)) == 1600


def test_library_space_size_and_order():
    pts = tuner.space()
    assert len(pts) == 4 * 3 * 16 * 4 * 3 == 2304
    assert pts == sorted(pts)
    assert pts[0] == (16, 16, 64, 1, 1) and pts[-1] == (64, 128, 1024, 8, 4)


def test_argmin_on_known_surface():
    # f = (log2 tile - 5)^2 + ((threads - 384) / 64)^2 + (cpb - 2)^2 + unroll + band / 16: unique minimum
    times = {c: (np.log2(c[1]) - 5) ** 2 + ((c[2] - 384) / 64) ** 2 + (c[3] - 2) ** 2 + c[4] + c[0] / 16
             for c in tuner.space()}
    assert tuner.argmin(times) == (16, 32, 384, 2, 1)


def test_argmin_ties_and_failures():
    times = {(32, 64, 128, 1, 1): 2.0, (16, 64, 128, 1, 1): 2.0, (16, 32, 64, 2, 2): 3.0,
             (16, 16, 64, 1, 1): float("nan"), (64, 16, 64, 1, 1): None}
    assert tuner.argmin(times) == (16, 64, 128, 1, 1)
    assert tuner.argmin({(1, 1, 1, 1, 1): None}) is None


def test_ratios():
    times = {("a",): 1.0, ("b",): 2.0, ("c",): 4.0, ("d",): 8.0, ("e",): 10.0}
    opt, med, dflt, r_med, r_def = tuner.ratios(times, ("c",))
    assert (opt, med, dflt, r_med, r_def) == (1.0, 4.0, 4.0, 4.0, 4.0)


def test_splitmix64_reference_outputs():
    # SplitMix64 from state 0: the first outputs of the published generator
    s = 0
    outs = []
    for _ in range(3):
        s, z = tuner.splitmix64(s)
        outs.append(z)
    assert outs == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_random_subset_distinct_and_deterministic():
    a = tuner.random_subset(2304, 116, seed=7)
    b = tuner.random_subset(2304, 116, seed=7)
    c = tuner.random_subset(2304, 116, seed=8)
    assert a == b and a != c
    assert len(set(a)) == 116 and all(0 <= i < 2304 for i in a)
