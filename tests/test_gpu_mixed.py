"""Mixed precision: the tensor-core building block and the TF32/BF16 trailing update.

The tensor-core product is checked against FP64 products of the operands
rounded on the CPU the way the device rounds them (TF32: keep 10 mantissa
bits, round half away from zero; BF16: keep 7, round half to even).  The
mixed-precision pipeline is checked against the prescribed singular values
within the first-order model err <= 10 u sqrt(n / b) (u = 2^-11 for TF32,
2^-8 for BF16: each of the n/b panel steps perturbs the trailing matrix by
about u ||A||, accumulating like a random walk; Weyl's inequality carries it
to the singular values).
"""
import ctypes
import math

import numpy as np
import pytest

import oracle
from paper_2608_21227_gb300 import inputs
from _util import err_rel, to_device_colmajor

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nla():
    from paper_2608_21227_gb300 import nla as _nla

    L = _nla.lib()
    L.nla_tc_selftest.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int] + [ctypes.c_void_p] * 5
    L.nla_tc_selftest.restype = ctypes.c_int
    return _nla


def round_tf32(x):
    b = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = ((b + 0x1000) & 0xFFFFE000).astype(np.uint32)
    return b.view(np.float32)


def round_bf16(x):
    b = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = ((b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return b.view(np.float32)


@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("K,N", [(16, 16), (32, 64), (64, 128), (128, 256)])
def test_tensor_core_tile(nla, prec, K, N):
    g = np.random.default_rng(K * 1000 + N + prec)
    A = g.standard_normal((128, K)).astype(np.float32)
    B = g.standard_normal((K, N)).astype(np.float32)
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    dD = torch.full((128, N), float("nan"), dtype=torch.float32, device="cuda")
    info = torch.zeros(1, dtype=torch.int32, device="cuda")
    st = nla.lib().nla_tc_selftest(prec, K, N, dA.data_ptr(), dB.data_ptr(), dD.data_ptr(), info.data_ptr(),
                                   torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert st == 0 and int(info.item()) == 0
    rnd = round_tf32 if prec == 1 else round_bf16
    ref = rnd(A).astype(np.float64) @ rnd(B).astype(np.float64)
    got = dD.cpu().numpy().astype(np.float64)
    scale = np.abs(rnd(A)).astype(np.float64) @ np.abs(rnd(B)).astype(np.float64)
    assert np.all(np.abs(got - ref) <= 1e-5 * scale + 1e-30)


@pytest.mark.parametrize("prec,u", [(1, 2.0 ** -11), (2, 2.0 ** -8)])
@pytest.mark.parametrize("kappa", [1.0, 1e4, 1e8])
def test_mixed_pipeline_prescribed(nla, prec, u, kappa):
    m, n, b = 700, 600, 32
    sigma = inputs.geometric_sigma(n, kappa)
    A = inputs.prescribed(m, n, sigma, seed=41)
    S, info = nla.gesvd_vals(to_device_colmajor(A, torch.float64), update=prec, cfg=nla.Cfg.make(band=b))
    torch.cuda.synchronize()
    assert int(info.item()) == 0
    err = err_rel(S.cpu().numpy(), sigma)
    assert err <= 10 * u * math.sqrt(max(m, n) / b), err
    assert np.all(np.isfinite(S.cpu().numpy()))


@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("m,n,b", [(300, 200, 16), (257, 257, 64), (130, 129, 32), (64, 64, 32)])
def test_mixed_stage1_keeps_sigma(nla, prec, m, n, b):
    # stage 1 with tensor-core updates: the band's singular values stay within the model of A's
    from _util import band_dense

    A = inputs.gaussian(m, n, 43 + m)
    t = to_device_colmajor(A, torch.float64)
    _, _, info = nla.gebrd_band(t, b, update=prec)
    ABt = nla.band_extract(t, b)
    torch.cuda.synchronize()
    assert int(info.item()) == 0
    D = band_dense(ABt, b)
    i, j = np.indices(D.shape)
    assert np.all(D[(j - i < 0) | (j - i > b)] == 0)
    u = 2.0 ** -11 if prec == 1 else 2.0 ** -8
    assert err_rel(oracle.svdvals(D), oracle.svdvals(A)) <= 10 * u * math.sqrt(m / b)
