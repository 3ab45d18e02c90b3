"""The tuner's host logic in libnla.so (no GPU calls).

The search space's order and the random sample are checked against the tuner
oracle (Section 3.1's space, SplitMix64).  Which points are valid is the
library's launch contract, not something the paper fixes (Section 3.1: the
constraints are user-supplied): its documented cases are checked here, and so
is its agreement with the workspace query, which must return NLA_ERR_CONFIG for
exactly the points kt_cfg_valid rejects.  The GPU half of the contract (every
admitted point launches and gives the oracle's singular values) is in
test_gpu_tuner.py.
"""
import ctypes

import numpy as np
import pytest

from oracle import tuner as otuner


@pytest.fixture(scope="module")
def kt():
    from paper_2608_21227_gb300 import _build

    _build.build()
    from paper_2608_21227_gb300 import kt as _kt

    return _kt


def test_space_matches_oracle(kt):
    assert kt.space() == otuner.space()


def test_validity_rule_cases(kt):
    L, F64, F32 = 0, 0, 1
    # register-tiled (FP64): the default configuration: w = 64 (16 column groups), 8
    # reflector groups of R = 4, 64-row tiles = 8 rows per thread, 8 * (64*64 + 64*36 + 32*64) B
    assert kt.cfg_valid(L, F64, (32, 64, 128, 2, 1))
    assert not kt.cfg_valid(L, F64, (32, 32, 96, 1, 1))      # 96 threads: 12 reflector groups do not divide 32
    assert not kt.cfg_valid(L, F64, (32, 16, 256, 1, 1))     # R = 1 but a 16-row tile gives 0.5 rows per thread
    assert kt.cfg_valid(L, F64, (32, 128, 256, 1, 1))        # 128 rows / 32 groups = 4 rows per thread
    assert not kt.cfg_valid(L, F64, (64, 128, 1024, 8, 1))   # 8 * (128*256 + 128*68 + 64*256) > 227 KiB
    # TMA-streamed (FP32, band 16/32/64): (band, stage depth, consumer threads, stages, waves)
    assert kt.cfg_valid(L, F32, (32, 64, 128, 2, 1))         # 2 * 40960 + 1024 B
    assert not kt.cfg_valid(L, F32, (16, 128, 256, 4, 1))    # 4 * 73728 + 1024 > 226 KiB
    assert kt.cfg_valid(L, F32, (64, 32, 128, 8, 4))         # 8 * 24576 + 1024 fits
    assert not kt.cfg_valid(L, F32, (64, 32, 64, 2, 1))      # 2 consumer warps < 4 reflector groups of 16
    assert not kt.cfg_valid(L, F32, (16, 16, 64, 2, 1))      # stage depth is a whole 32-row box
    assert not kt.cfg_valid(L, F32, (16, 64, 128, 1, 1))     # a ring needs at least 2 stages
    assert not kt.cfg_valid(L, F32, (64, 128, 1024, 8, 1))   # at most 8 consumer warps
    for dt in (F64, F32):
        n_valid = sum(kt.cfg_valid(L, dt, c) for c in kt.space())
        assert 0 < n_valid < 2304


@pytest.mark.parametrize("dtype", [0, 1])
def test_workspace_query_enforces_the_rule(kt, dtype):
    # the workspace query rejects (NLA_ERR_CONFIG) exactly the points kt_cfg_valid rejects
    from paper_2608_21227_gb300 import nla

    for c in kt.space():
        ok = kt.cfg_valid(kt.KT_GESVD, dtype, c)
        try:
            nla.gesvd_vals_workspace(256, 200, dtype, cfg=c)
            got = True
        except nla.NLAError as e:
            assert e.status == 3, (c, e.status)
            got = False
        assert got == bool(ok), c


def test_default_config_is_valid(kt):
    for dt in (0, 1):
        assert kt.cfg_valid(0, dt, (32, 64, 128, 2, 1)) and kt.cfg_valid(1, dt, (32, 64, 128, 2, 1))


@pytest.mark.parametrize("count,k,seed", [(294, 15, 1), (2304, 116, 7), (10, 10, 3), (5, 0, 9)])
def test_random_subset_matches_oracle(kt, count, k, seed):
    assert kt.random_subset(count, k, seed) == otuner.random_subset(count, k, seed)


def test_features_layout(kt):
    f = kt.features(1, 8192, 4096, 1, 2, (32, 64, 128, 2, 4))
    want = np.zeros(15, dtype=np.float32)
    want[1] = 1
    want[3:10] = np.log2([32, 64, 128, 2, 4, 8192, 4096])
    want[11] = 1  # FP32
    want[14] = 1  # BF16 update
    assert np.allclose(f, want)
