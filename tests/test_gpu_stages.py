"""Stage-level GPU parity: each stage's output checked by the FP64 oracle."""
import numpy as np
import pytest

import oracle
from paper_2608_21227_gb300 import inputs
from _util import band_dense, err_rel, from_device_colmajor, to_device_colmajor, tol_for

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nla():
    from paper_2608_21227_gb300 import nla as _nla

    _nla.lib()
    return _nla


@pytest.mark.parametrize("dt", [0, 1])
@pytest.mark.parametrize("m,n,b", [(300, 200, 16), (256, 256, 32), (150, 150, 64), (90, 45, 8),
                                   # FP32: several 128-row strips, column splits and ragged tails of the
                                   # TMA / tensor-core projections on both sides
                                   (1100, 900, 16), (1032, 1000, 32), (1064, 1064, 64)])
def test_stage1_band(nla, dt, m, n, b):
    A = inputs.gaussian(m, n, 500 + m + b)
    tdt = torch.float64 if dt == 0 else torch.float32
    if dt == 1:
        A = A.astype(np.float32).astype(np.float64)
    t = to_device_colmajor(A, tdt)
    tauq, taup, info = nla.gebrd_band(t, b)
    ABt = nla.band_extract(t, b)
    torch.cuda.synchronize()
    assert int(info.item()) == 0
    D = band_dense(ABt, b)
    # structure: nothing outside the upper band 0 <= j - i <= b
    i, j = np.indices(D.shape)
    assert np.all(D[(j - i < 0) | (j - i > b)] == 0)
    # Frobenius norm and singular values preserved (Section 5.1.1: orthogonal reduction)
    fro = np.linalg.norm(A)
    tolf = (1e-13 if dt == 0 else 1e-6) * m
    assert abs(np.linalg.norm(D) - fro) <= tolf * fro
    assert err_rel(oracle.svdvals(D), oracle.svdvals(A)) <= tol_for(dt, m)
    # the lower part of the panel holds reflectors, the band the reduced matrix
    full = from_device_colmajor(t)
    assert np.allclose(np.triu(full[:n, :n]) * ((j - i) <= b), D, atol=0, rtol=0)


@pytest.mark.parametrize("dt", [0, 1])
@pytest.mark.parametrize("n,b", [(200, 16), (256, 32), (130, 64), (50, 2), (64, 3), (3, 2)])
def test_stage2_bulge_chase(nla, dt, n, b):
    g = np.random.default_rng(600 + n + b)
    D = np.triu(g.standard_normal((n, n))) * (np.subtract.outer(np.arange(n), np.arange(n)) >= -b)
    if dt == 1:
        D = D.astype(np.float32).astype(np.float64)
    tdt = torch.float64 if dt == 0 else torch.float32
    t = to_device_colmajor(D, tdt)
    ABt = nla.band_extract(t, b)
    d, e, info = nla.band2bd(ABt, b)
    torch.cuda.synchronize()
    assert int(info.item()) == 0
    dn, en = d.cpu().numpy(), e.cpu().numpy()
    fro2 = float(np.sum(D * D))
    tolf = (1e-13 if dt == 0 else 1e-6) * n
    assert abs(np.sum(dn * dn) + np.sum(en * en) - fro2) <= tolf * fro2
    assert err_rel(oracle.bdsvd(dn, en), oracle.svdvals(D)) <= tol_for(dt, n)


@pytest.mark.parametrize("n", [1, 2, 3, 50, 333, 1024])
def test_stage3_bisection_vs_oracle(nla, n):
    g = np.random.default_rng(700 + n)
    d = g.standard_normal(n)
    e = g.standard_normal(max(n - 1, 0))
    S, info = nla.bdsvd_vals(torch.from_numpy(d).cuda(), torch.from_numpy(e).cuda())
    torch.cuda.synchronize()
    assert int(info.item()) == 0
    assert err_rel(S.cpu().numpy(), oracle.bdsvd(d, e)) <= 1e-12 * max(n, 1)


def test_stage3_closed_forms(nla):
    n = 400
    S, _ = nla.bdsvd_vals(torch.ones(n, dtype=torch.float64).cuda(), torch.ones(n - 1, dtype=torch.float64).cuda())
    k = np.arange(1, n + 1)
    assert err_rel(S.cpu().numpy(), 2 * np.cos(k * np.pi / (2 * n + 1))) <= 1e-13 * n
    d = np.array([3.0, 0.0, -2.0, 0.0, 1.0, 5.0])
    S, _ = nla.bdsvd_vals(torch.from_numpy(d).cuda(), torch.zeros(5, dtype=torch.float64).cuda())
    assert err_rel(S.cpu().numpy(), np.sort(np.abs(d))[::-1]) <= 1e-15
    e = np.array([1.0, 2.0, 0.5, 1.5, 0.25])
    S, _ = nla.bdsvd_vals(torch.from_numpy(d).cuda(), torch.from_numpy(e).cuda())
    assert err_rel(S.cpu().numpy(), oracle.bdsvd(d, e)) <= 1e-13
