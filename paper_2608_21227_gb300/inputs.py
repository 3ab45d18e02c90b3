"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module generates matrices only; it contains none of the arithmetic of
the singular-value method.  All randomness comes from numpy's PCG64
(``numpy.random.default_rng``) or, for sizes too large to build on the host,
from a seeded ``torch.Generator`` on the GPU.

Recipes (matching the workloads named by the library's benchmark configs):

* ``gaussian``     -- entries iid N(0, 1).
* ``uniform``      -- entries iid U[-1, 1].
* ``haar``         -- an n x k matrix with orthonormal columns, distributed
                      as the first k columns of a Haar orthogonal matrix:
                      Q of the QR of a Gaussian matrix with each column
                      multiplied by the sign of R's diagonal (Mezzadri 2007).
* ``prescribed``   -- U diag(sigma) V^T with Haar U (m x p) and V (n x p);
                      its singular values are sigma up to the FP64 forming
                      error.
* ``geometric_sigma`` -- sigma_i = kappa^{-(i-1)/(p-1)}.
* ``batch_shapes`` -- n ~ U{lo..hi}, r ~ U[1, 4], m = floor(n r + 0.5).
"""
from __future__ import annotations

import numpy as np


def rng(seed) -> np.random.Generator:
    return np.random.default_rng(seed)


def gaussian(m: int, n: int, seed, dtype=np.float64) -> np.ndarray:
    a = rng(seed).standard_normal((n, m)).T  # column-major m x n
    return np.asfortranarray(a.astype(dtype, copy=False))


def uniform(m: int, n: int, seed, dtype=np.float64) -> np.ndarray:
    a = rng(seed).uniform(-1.0, 1.0, size=(n, m)).T
    return np.asfortranarray(a.astype(dtype, copy=False))


def haar(n: int, k: int, g: np.random.Generator) -> np.ndarray:
    """n x k with orthonormal columns, Haar-distributed (Mezzadri 2007)."""
    z = g.standard_normal((n, k))
    q, r = np.linalg.qr(z, mode="reduced")
    s = np.sign(np.diag(r))
    s[s == 0] = 1.0
    return q * s[None, :]


def geometric_sigma(p: int, kappa: float) -> np.ndarray:
    if p == 1:
        return np.ones(1)
    i = np.arange(p, dtype=np.float64)
    return kappa ** (-i / (p - 1))


def prescribed(m: int, n: int, sigma, seed, dtype=np.float64) -> np.ndarray:
    """U diag(sigma) V^T with Haar U, V (host, FP64 forming)."""
    sigma = np.asarray(sigma, dtype=np.float64)
    p = min(m, n)
    assert sigma.shape == (p,)
    g = rng(seed)
    U = haar(m, p, g)
    V = haar(n, p, g)
    a = (U * sigma[None, :]) @ V.T
    return np.asfortranarray(a.astype(dtype, copy=False))


def prescribed_device(m: int, n: int, sigma, seed: int, device="cuda", form_dtype=None):
    """Large U diag(sigma) V^T built on the GPU with a seeded torch.Generator.

    Returns a torch tensor of shape (n, m) in row-major order, i.e. the
    column-major m x n matrix the library expects.  The orthogonal factors are
    Haar (Mezzadri sign fix).  ``form_dtype`` (default float64) is the
    precision of the final product.
    """
    import torch

    form_dtype = form_dtype or torch.float64
    p = min(m, n)
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))

    def haar_t(rows):
        z = torch.randn(rows, p, generator=g, device=device, dtype=torch.float64)
        q, r = torch.linalg.qr(z, mode="reduced")
        s = torch.sign(torch.diagonal(r))
        s[s == 0] = 1.0
        return q * s[None, :]

    U = haar_t(m)
    V = haar_t(n)
    sig = torch.as_tensor(np.asarray(sigma, dtype=np.float64), device=device)
    # column-major A (m x n) == row-major A^T (n x m) = V diag(sigma) U^T
    At = (V.to(form_dtype) * sig.to(form_dtype)[None, :]) @ U.to(form_dtype).T
    del U, V
    return At.contiguous()


def uniform_device(m: int, n: int, seed: int, dtype=None, device="cuda"):
    """U[-1, 1] entries generated on the GPU (row-major (n, m) == column-major m x n)."""
    import torch

    dtype = dtype or torch.float64
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    t = torch.empty(n, m, dtype=dtype, device=device)
    t.uniform_(-1.0, 1.0, generator=g)
    return t


def batch_shapes(count: int, seed, n_lo: int = 8, n_hi: int = 256):
    """Shapes of a batch of uneven matrices: n ~ U{n_lo..n_hi}, m/n ~ U[1, 4]."""
    g = rng(seed)
    n = g.integers(n_lo, n_hi + 1, size=count)
    r = g.uniform(1.0, 4.0, size=count)
    m = np.floor(n * r + 0.5).astype(np.int64)
    return m.astype(np.int64), n.astype(np.int64)


def batch_matrices(shapes, seed, dtype=np.float32):
    """Matrix i of a batch uses the sub-stream default_rng([seed, i]), entries N(0, 1)."""
    ms, ns = shapes
    return [gaussian(int(ms[i]), int(ns[i]), [seed, i], dtype=dtype) for i in range(len(ms))]
