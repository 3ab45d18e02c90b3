"""nla_band2bd_noalloc: the bulge chase for callers that cannot allocate.

Some callers cannot call cudaMalloc -- a plug-in inside a host framework
whose memory manager owns the whole device, code that must never synchronise
the device (cudaMalloc and cudaFree may), a program with a fixed device-memory
budget -- so they cannot hand nla_band2bd a workspace.  The no-alloc variant
keeps that scratch in a fixed array inside the library.  This test
calls it through the C ABI, twice in a row (the second call must not be
disturbed by what the first left in the shared array), and checks its d, e
against the regular entry point's on the same band matrix, with the
tolerance the other GPU tests use (1e-12 N relative to the largest entry for
FP64, 5e-6 N for FP32).  The file is named to be collected last.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nla():
    from paper_2608_21227_gb300 import nla as _nla

    L = _nla.lib()
    L.nla_band2bd_noalloc.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
                                      ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    L.nla_band2bd_noalloc.restype = ctypes.c_int
    return _nla


def band_storage(n, b, dtype, seed):
    """Compact storage (tensor (n, 3b+1)) of a random upper band matrix of width b."""
    g = np.random.default_rng(seed)
    D = np.triu(g.standard_normal((n, n))) * (np.subtract.outer(np.arange(n), np.arange(n)) >= -b)
    AB = np.zeros((n, 3 * b + 1))
    for j in range(n):
        for i in range(max(0, j - b), j + 1):
            AB[j, 2 * b + i - j] = D[i, j]
    return torch.from_numpy(AB).to(device="cuda", dtype=dtype)


def call_noalloc(nla, ABt, b):
    n, ldab = ABt.shape
    d = torch.empty(n, dtype=torch.float64, device="cuda")
    e = torch.empty(max(n, 1), dtype=torch.float64, device="cuda")
    info = torch.zeros(1, dtype=torch.int32, device="cuda")
    dt = 0 if ABt.dtype == torch.float64 else 1
    st = nla.lib().nla_band2bd_noalloc(n, b, dt, ABt.data_ptr(), ldab, d.data_ptr(), e.data_ptr(),
                                       info.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert st == 0, nla.lib().nla_last_error()
    return d, e[: max(n - 1, 0)], info


@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-12), (torch.float32, 5e-6)])
@pytest.mark.parametrize("n,b", [(300, 16), (1000, 32), (257, 64)])
def test_noalloc_matches_regular_twice(nla, dtype, tol, n, b):
    AB = band_storage(n, b, dtype, seed=900 + n + b)
    ref_d, ref_e, ref_info = nla.band2bd(AB.clone(), b)
    for _ in range(2):
        d, e, info = call_noalloc(nla, AB.clone(), b)
        torch.cuda.synchronize()
        assert int(info.item()) == 0 and int(ref_info.item()) == 0
        scale = float(torch.max(torch.abs(AB)).item())
        assert float(torch.max(torch.abs(d - ref_d)).item()) <= tol * n * scale
        assert float(torch.max(torch.abs(e - ref_e)).item()) <= tol * n * scale


def test_noalloc_rejects_oversized(nla):
    L = nla.lib()
    st = L.nla_band2bd_noalloc(65537, 2, 0, None, 7, None, None, None, None)
    assert st == 7  # NLA_ERR_UNSUPPORTED, before any device work
