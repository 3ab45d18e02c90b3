"""GPU tests of the auto-tuner: Eq. 1 argmin over measured runtimes, cache/resume,
the random-sample baseline, pipeline-level band choice and the installed table."""
import csv
import ctypes
import math
import os

import numpy as np
import pytest

from oracle import tuner as otuner

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kt():
    from paper_2608_21227_gb300 import kt as _kt

    _kt.lib()
    return _kt


def read_cache(path):
    rows = []
    with open(path) as f:
        for r in csv.DictReader(f):
            rows.append({k: float(v) if k == "median_ms" else int(v) for k, v in r.items()})
    return rows


def cfg_of(r):
    return (r["band"], r["tile"], r["threads"], r["cpb"], r["unroll"])


def test_exhaustive_is_eq1_argmin(kt, tmp_path):
    cache = str(tmp_path / "c.csv")
    res = kt.tune(kt.KT_TRAIL_LEFT, 1024, 1024, 1, band=32, reps=3, cache=cache)
    rows = read_cache(cache)
    valid = [c for c in kt.space() if c[0] == 32 and kt.cfg_valid(kt.KT_TRAIL_LEFT, 1, c)]
    assert res["evaluated"] == len(rows) == res["valid"] == len(valid)
    assert res["failed"] == 0 and all(r["status"] == 0 for r in rows)
    times = {cfg_of(r): r["median_ms"] for r in rows}
    assert res["best"] == otuner.argmin(times)
    assert math.isclose(res["best_ms"], min(times.values()), rel_tol=1e-6)
    assert math.isclose(res["median_ms"], float(np.median(list(times.values()))), rel_tol=1e-6)
    assert res["default_ms"] > 0 and res["median_ms"] >= res["best_ms"]
    # resume: everything comes from the cache, same answer
    res2 = kt.tune(kt.KT_TRAIL_LEFT, 1024, 1024, 1, band=32, reps=3, cache=cache)
    assert res2["best"] == res["best"] and len(read_cache(cache)) == len(rows)


def test_lq_side_and_fp64(kt, tmp_path):
    cache = str(tmp_path / "r.csv")
    res = kt.tune(kt.KT_TRAIL_RIGHT, 512, 512, 0, band=16, reps=2, cache=cache)
    rows = read_cache(cache)
    assert res["failed"] == 0 and res["evaluated"] == len(rows) > 0
    assert res["best"] == otuner.argmin({cfg_of(r): r["median_ms"] for r in rows})


def test_random_sample_is_the_oracle_subset(kt, tmp_path):
    cache = str(tmp_path / "rnd.csv")
    res = kt.tune(kt.KT_TRAIL_LEFT, 768, 768, 1, band=16, reps=2, strategy=kt.KT_RANDOM, budget_frac=0.1,
                  cache=cache, seed=12345)
    valid = [c for c in kt.space() if c[0] == 16 and kt.cfg_valid(kt.KT_TRAIL_LEFT, 1, c)]
    k = max(1, math.ceil(0.1 * res["valid"]))
    assert res["valid"] == len(valid) and res["evaluated"] == k
    # the sample is the oracle's SplitMix64 subset of the valid list (in space order)
    want = {valid[i] for i in otuner.random_subset(len(valid), k, 12345)}
    got = {cfg_of(r) for r in read_cache(cache)}
    assert got == want


def test_pipeline_band_choice_and_table(kt, tmp_path):
    res = kt.tune(kt.KT_GESVD, 1024, 1024, 1, reps=2)
    assert res["best"][0] in (16, 32, 64) and res["evaluated"] == 3
    table = str(tmp_path / "t.kt")
    kt.write_table(table, 0, 1024, 1024, 1, 0, res["best"], res["best_ms"])
    kt.write_table(table, 1, 1024, 1024, 1, 0, res["best"], res["best_ms"])
    kt.load_config(table)
    L = kt.lib()
    from paper_2608_21227_gb300 import nla

    out = nla.Cfg()
    L.nla_tuned_lookup.argtypes = [ctypes.c_int] * 5 + [ctypes.POINTER(nla.Cfg)]
    assert L.nla_tuned_lookup(2000, 2000, 1, 0, 0, ctypes.byref(out)) == 1
    assert out.as_tuple() == tuple(res["best"])
    assert L.nla_tuned_lookup(2000, 2000, 0, 0, 0, ctypes.byref(out)) == 0  # no FP64 entry
    # the pipeline runs with the installed table and stays correct
    import oracle
    from paper_2608_21227_gb300 import inputs
    from _util import err_rel, to_device_colmajor, tol_for

    A = inputs.uniform(1024, 1024, 77, dtype=np.float32).astype(np.float64)
    S, info = nla.gesvd_vals(to_device_colmajor(A, torch.float32))
    torch.cuda.synchronize()
    assert int(info.item()) == 0
    assert err_rel(S.cpu().numpy(), oracle.svdvals(A)) <= tol_for(1, 1024)
    kt.load_config(None)


@pytest.mark.parametrize("dtype", [0, 1])
def test_validity_contract(kt, dtype):
    # the launch contract on this device: every point kt_cfg_valid admits runs the whole
    # SVD and gives the oracle's singular values; every point it rejects is refused
    # up front with NLA_ERR_CONFIG (nothing enqueued)
    import oracle
    from paper_2608_21227_gb300 import inputs, nla
    from _util import err_rel, to_device_colmajor, tol_for

    m, n = 200, 160
    A = inputs.uniform(m, n, 91)
    if dtype == 1:
        A = A.astype(np.float32).astype(np.float64)
    ref = oracle.svdvals(A)
    t0 = to_device_colmajor(A, torch.float64 if dtype == 0 else torch.float32)
    admitted = 0
    for c in kt.space():
        ok = kt.cfg_valid(kt.KT_GESVD, dtype, c)
        t = t0.clone()
        if ok:
            S, info = nla.gesvd_vals(t, cfg=nla.Cfg.make(*c))
            torch.cuda.synchronize()
            assert int(info.item()) == 0, c
            assert err_rel(S.double().cpu().numpy(), ref) <= tol_for(dtype, m), c
            admitted += 1
        else:
            with pytest.raises(nla.NLAError) as ei:
                nla.gesvd_vals(t, cfg=nla.Cfg.make(*c))
            assert ei.value.status == 3, c
    assert admitted > 0
