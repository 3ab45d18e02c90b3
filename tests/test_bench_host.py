"""Host-side arithmetic behind the benchmark line and the tuning scripts (no GPU): the
metric's flop count, the roofline's algorithmic bytes of the trailing update, and the
sweep-cache reader that feeds the cost model."""
import importlib.util
import os

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_flop_count_is_householder_bidiagonalisation():
    # 4 m n^2 - 4 n^3 / 3 (m >= n), the count the metric divides by; symmetric in (m, n)
    b = _bench()
    assert b.flops(8192, 8192) == 4.0 * 8192 ** 3 - 4.0 * 8192 ** 3 / 3.0
    assert b.flops(300, 200) == pytest.approx(4 * 300 * 200 ** 2 - 4 * 200 ** 3 / 3)
    assert b.flops(200, 300) == b.flops(300, 200)


def test_trailing_update_bytes_small_case_by_hand():
    # n = 32, b = 16: one panel step; the QR-side block is 32 x 16 (rows kb.., columns kb+b..),
    # the LQ-side block 16 x 16; three passes (read, read, write) of 4-byte entries
    b = _bench()
    assert b.trail_bytes_per_step(32, 32, 16, 0) == 3 * 4 * 32 * 16
    assert b.trail_bytes_per_step(32, 32, 16, 1) == 3 * 4 * 16 * 16
    assert b.trail_bytes_per_step(16, 16, 16, 0) == 0  # one panel, nothing trails it


def test_trailing_update_bytes_closed_form_at_the_headline_size():
    # n = 8192, b = 16: sum over k < n/b - 1 of 12 (n - kb)(n - (k+1)b) (QR) and 12 (n - (k+1)b)^2 (LQ)
    b = _bench()
    n, bb = 8192, 16
    k = np.arange(n // bb - 1, dtype=np.int64)
    qr = int(12 * np.sum((n - k * bb) * (n - (k + 1) * bb)))
    lq = int(12 * np.sum((n - (k + 1) * bb) ** 2))
    assert b.trail_bytes_per_step(n, n, bb, 0) == qr
    assert b.trail_bytes_per_step(n, n, bb, 1) == lq
    # ~ 24 n^3 / (3 b): the continuum estimate of the same sum
    assert qr + lq == pytest.approx(24 * n ** 3 / (3 * bb), rel=2e-3)


def test_trailing_update_flops_are_4_b_per_entry():
    b = _bench()
    n, bb = 1024, 16
    for side in (0, 1):
        assert b.trail_flops_per_step(n, n, bb, side) == pytest.approx(
            4 * bb * b.trail_bytes_per_step(n, n, bb, side) / 12)


def test_sweep_cache_reader_accepts_both_row_widths(tmp_path):
    # rows written before and after the objective column was added, under the older header
    tune = pytest.importorskip("paper_2608_21227_gb300.tune")
    p = tmp_path / "cache.csv"
    p.write_text("kernel,m,n,dtype,update,band,tile,threads,cpb,unroll,median_ms,status\n"
                 "0,1024,1024,1,0,16,64,128,2,1,0.5,0\n"
                 "1,1024,1024,1,0,16,64,128,2,1,0.25,0,0\n"
                 "1,1024,1024,1,0,16,64,128,2,1,9.5,0,1\n"  # an energy row: not a runtime
                 "0,1024,1024,1,0,16,64,128,2,1,0.0,3\n")   # a failed configuration
    rows = tune.read_cache(str(p))
    assert [(r["kernel"], r["median_ms"]) for r in rows] == [(0, 0.5), (1, 0.25)]
    assert rows[1]["objective"] == 0
