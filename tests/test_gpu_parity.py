"""GPU parity: singular values from the CUDA path (through the C ABI) against the FP64 oracle.

Acceptance: max_i |sigma_gpu_i - sigma_oracle_i| / sigma_1 <= 1e-12 N (FP64),
<= 5e-6 N (FP32), N = max(m, n).
"""
import numpy as np
import pytest

import oracle
from paper_2608_21227_gb300 import inputs
from _util import err_rel, from_device_colmajor, to_device_colmajor, tol_for

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DT = {0: torch.float64, 1: torch.float32}


@pytest.fixture(scope="module")
def nla():
    from paper_2608_21227_gb300 import nla as _nla

    _nla.lib()
    return _nla


def run(nla, A, dt, **kw):
    t = to_device_colmajor(A, DT[dt])
    S, info = nla.gesvd_vals(t, **kw)
    torch.cuda.synchronize()
    assert int(info.item()) == 0, f"info {int(info.item())}"
    return S.cpu().numpy().astype(np.float64), t


SHAPES = [
    (256, 256, 32),   # the plain-method configuration: 256 x 256, tile 32, band 32
    (300, 200, 32),   # tall, ragged last tile
    (200, 300, 32),   # wide: transposed in the workspace
    (129, 129, 16),
    (97, 61, 8),
    (64, 64, 64),
    (33, 33, 32),     # last panel one column wide
    (520, 260, 64),
    (1000, 1000, 32),
    (700, 650, 64),
]


@pytest.mark.parametrize("dt", [0, 1])
@pytest.mark.parametrize("m,n,b", SHAPES)
def test_gesvd_vs_oracle(nla, dt, m, n, b):
    A = inputs.gaussian(m, n, 1000 + m + n + b)
    if dt == 1:
        A = A.astype(np.float32).astype(np.float64)  # the FP32 path sees exactly these values
    ref = oracle.svdvals(A)
    got, _ = run(nla, A, dt, cfg=nla.Cfg.make(band=b))
    assert err_rel(got, ref) <= tol_for(dt, max(m, n))
    assert np.all(np.diff(got) <= 0), "not descending"
    assert np.all(got >= 0)


@pytest.mark.parametrize("dt", [0, 1])
@pytest.mark.parametrize("m,n", [(1, 1), (1, 7), (7, 1), (2, 2), (5, 3), (3, 5), (17, 2), (40, 40)])
def test_tiny_shapes(nla, dt, m, n):
    A = inputs.uniform(m, n, 77 + m * 13 + n)
    if dt == 1:
        A = A.astype(np.float32).astype(np.float64)
    ref = oracle.svdvals(A)
    got, _ = run(nla, A, dt)
    assert err_rel(got, ref) <= tol_for(dt, max(m, n))


@pytest.mark.parametrize("dt", [0, 1])
@pytest.mark.parametrize("kappa", [1.0, 1e4, 1e8])
def test_prescribed_sigma(nla, dt, kappa):
    m, n = 600, 500
    sigma = inputs.geometric_sigma(n, kappa)
    A = inputs.prescribed(m, n, sigma, seed=31)
    if dt == 1:
        A = A.astype(np.float32).astype(np.float64)
    ref = oracle.svdvals(A)
    got, _ = run(nla, A, dt, cfg=nla.Cfg.make(band=32))
    assert err_rel(got, ref) <= tol_for(dt, m)
    if dt == 0:
        assert err_rel(got, sigma) <= tol_for(dt, m)


def test_degenerate_inputs(nla):
    # zero matrix, rank one, repeated singular values
    for A, ref in [
        (np.zeros((50, 40)), np.zeros(40)),
        (np.outer(np.arange(1, 61.0), np.ones(45)), None),
        (np.kron(np.eye(3), inputs.haar(20, 20, np.random.default_rng(5))), np.ones(60)),
    ]:
        if ref is None:
            ref = oracle.svdvals(A)
        got, _ = run(nla, A, 0, cfg=nla.Cfg.make(band=16))
        assert err_rel(got, ref) <= tol_for(0, max(A.shape)) or np.max(np.abs(got - ref)) <= 1e-13


def test_empty_is_noop(nla):
    lib = nla.lib()
    assert lib.nla_gesvd_vals(0, 5, 0, None, 1, None, None, 0, None, None, None) == 0
    assert lib.nla_gesvd_vals(5, 0, 0, None, 5, None, None, 0, None, None, None) == 0


def test_preserve_a_and_determinism(nla):
    A = inputs.gaussian(300, 300, 9)
    t = to_device_colmajor(A, torch.float64)
    S1, _ = nla.gesvd_vals(t, preserve_a=True)
    S2, _ = nla.gesvd_vals(t, preserve_a=True)
    torch.cuda.synchronize()
    assert np.array_equal(from_device_colmajor(t), A), "preserve_a modified A"
    assert torch.equal(S1, S2), "results differ between identical runs"


def test_oversized_config_rejected(nla):
    # 1024 threads cannot tile a 64-column strip and 64 reflectors with 32-row
    # tiles: rejected up front as a configuration error, not a failed launch
    A = inputs.gaussian(256, 256, 3)
    t = to_device_colmajor(A, torch.float64)
    with pytest.raises(nla.NLAError) as ei:
        nla.gesvd_vals(t, cfg=nla.Cfg.make(band=64, tile=32, threads=1024, cols_per_block=2, unroll=1))
    assert ei.value.status == 3


def test_invalid_config_rejected(nla):
    A = inputs.gaussian(64, 64, 3)
    t = to_device_colmajor(A, torch.float64)
    with pytest.raises(nla.NLAError) as ei:
        nla.gesvd_vals(t, cfg=nla.Cfg.make(band=32, tile=32, threads=96, cols_per_block=1, unroll=1))
    assert ei.value.status == 3


def _spread_valid_configs(count):
    from paper_2608_21227_gb300 import kt

    pts = [c for c in kt.space() if kt.cfg_valid(kt.KT_GESVD, 0, c)]
    step = max(1, len(pts) // count)
    return pts[::step][:count]


@pytest.mark.parametrize("i", range(8))
def test_configs_agree(nla, i):
    cfg = _spread_valid_configs(8)[i]
    A = inputs.uniform(400, 333, 11)
    ref = oracle.svdvals(A)
    got, _ = run(nla, A, 0, cfg=nla.Cfg.make(*cfg))
    assert err_rel(got, ref) <= tol_for(0, 400)


def test_full_size_fp64_prescribed(nla):
    # 8192 x 8192 FP64 with prescribed geometric sigma (1 -> 1e-6): the pin holds at any size.
    n = 8192
    sigma = inputs.geometric_sigma(n, 1e6)
    At = inputs.prescribed_device(n, n, sigma, seed=208, device="cuda")
    fro2 = float((At * At).sum().item())
    S, info = nla.gesvd_vals(At)
    torch.cuda.synchronize()
    assert int(info.item()) == 0
    got = S.cpu().numpy()
    assert err_rel(got, sigma) <= tol_for(0, n)
    assert abs(float(np.sum(got * got)) - fro2) <= 1e-12 * n * fro2


def test_full_size_fp32_uniform_frobenius(nla):
    # 8192 x 8192 FP32 U[-1, 1]: sum sigma^2 = ||A||_F^2 and sampled agreement with the FP64 path
    n = 8192
    At = inputs.uniform_device(n, n, seed=216, dtype=torch.float32)
    A64 = At.double()
    fro2 = float((A64 * A64).sum().item())
    S32, info = nla.gesvd_vals(At)
    S64, info64 = nla.gesvd_vals(A64)
    torch.cuda.synchronize()
    assert int(info.item()) == 0 and int(info64.item()) == 0
    s32 = S32.double().cpu().numpy()
    s64 = S64.cpu().numpy()
    assert abs(float(np.sum(s64 * s64)) - fro2) <= 1e-12 * n * fro2
    assert err_rel(s32, s64) <= tol_for(1, n)
