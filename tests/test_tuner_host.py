"""The tuner's host logic in libnla.so (no GPU calls) against the tuner oracle."""
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


@pytest.mark.parametrize("kernel,side", [(0, 0), (1, 1)])
@pytest.mark.parametrize("dtype,elem", [(0, 8), (1, 4)])
def test_validity_matches_oracle(kt, kernel, side, dtype, elem):
    lib_valid = [kt.cfg_valid(kernel, dtype, c) for c in otuner.space()]
    ora_valid = [otuner.valid(side, elem, c) for c in otuner.space()]
    assert lib_valid == ora_valid


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
