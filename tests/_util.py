"""Shared helpers for the tests (no method arithmetic here)."""
import numpy as np

EPS64 = np.finfo(np.float64).eps


def err_rel(got, ref):
    """max_i |got_i - ref_i| / ref_1: absolute singular-value error relative to sigma_max."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    assert got.shape == ref.shape, (got.shape, ref.shape)
    if ref.size == 0:
        return 0.0
    scale = ref[0] if ref[0] > 0 else 1.0
    return float(np.max(np.abs(got - ref)) / scale)


def tol_for(dtype_code, N):
    """Acceptance bound on err_rel: 1e-12 N for FP64, 5e-6 N for FP32 (N = max(m, n))."""
    return (1e-12 if dtype_code == 0 else 5e-6) * N


def to_device_colmajor(A, torch_dtype, device="cuda"):
    """A CUDA tensor whose memory is the column-major copy of the numpy matrix A."""
    import torch

    return torch.from_numpy(np.ascontiguousarray(np.asarray(A).T)).to(device=device, dtype=torch_dtype)


def from_device_colmajor(t):
    """Inverse of to_device_colmajor."""
    return t.detach().cpu().numpy().T.astype(np.float64)


def band_dense(ABt, band):
    """Dense n x n matrix from compact band storage (tensor (n, 3b+1), entry (i,j) at row 2b+i-j)."""
    AB = ABt.detach().cpu().numpy().astype(np.float64)  # AB[j, q]
    n = AB.shape[0]
    D = np.zeros((n, n))
    for j in range(n):
        for q in range(AB.shape[1]):
            i = q - 2 * band + j
            if 0 <= i < n:
                D[i, j] = AB[j, q]
    return D
