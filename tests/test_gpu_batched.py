"""Batched persistent path: every matrix against the FP64 oracle (FP32 tolerance 5e-6 N)."""
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

    _nla.lib()
    return _nla


def make_batch(nla, mats):
    return nla.Batch([to_device_colmajor(A, torch.float32) for A in mats])


def check(batch_S, info, mats, tol_scale=5e-6):
    torch.cuda.synchronize()
    assert np.all(info.cpu().numpy()[: len(mats)] == 0)
    for A, S in zip(mats, batch_S):
        ref = oracle.svdvals(A.astype(np.float64))
        assert err_rel(S.cpu().numpy(), ref) <= tol_scale * max(A.shape), A.shape


def test_uneven_shapes_vs_oracle(nla):
    ms, ns = inputs.batch_shapes(300, seed=33)
    mats = [inputs.gaussian(int(m), int(n), [33, i], dtype=np.float32) for i, (m, n) in enumerate(zip(ms, ns))]
    # every fifth matrix is handed over wide (m < n)
    mats = [A.T.copy() if i % 5 == 0 else A for i, A in enumerate(mats)]
    b = make_batch(nla, mats)
    S, info = nla.gesvd_vals_batched(b)
    check(S, info, mats)


def test_tiny_and_degenerate(nla):
    g = np.random.default_rng(5)
    mats = [g.standard_normal((1, 1)), g.standard_normal((1, 6)), g.standard_normal((6, 1)), np.zeros((8, 8)),
            np.outer(np.arange(1.0, 11.0), np.ones(5)), g.standard_normal((17, 16)), g.standard_normal((256, 256)),
            g.standard_normal((1024, 256))]
    mats = [A.astype(np.float32) for A in mats]
    b = make_batch(nla, mats)
    S, info = nla.gesvd_vals_batched(b)
    torch.cuda.synchronize()
    assert np.all(info.cpu().numpy() == 0)
    for A, s in zip(mats, S):
        ref = oracle.svdvals(A.astype(np.float64))
        assert np.max(np.abs(s.cpu().numpy() - ref)) <= 5e-6 * max(A.shape) * max(ref[0], 1e-30) + 1e-30


def test_ten_thousand_matrices_sampled(nla):
    # the batched workload: 10,000 FP32 matrices, n ~ U{8..256}, m/n ~ U[1, 4], N(0, 1)
    ms, ns = inputs.batch_shapes(10000, seed=3)
    mats = [inputs.gaussian(int(m), int(n), [3, i], dtype=np.float32) for i, (m, n) in enumerate(zip(ms, ns))]
    b = make_batch(nla, mats)
    S, info = nla.gesvd_vals_batched(b)
    torch.cuda.synchronize()
    assert np.all(info.cpu().numpy() == 0)
    sample = np.random.default_rng(0).choice(10000, size=60, replace=False)
    for i in sample:
        ref = oracle.svdvals(mats[i].astype(np.float64))
        assert err_rel(S[i].cpu().numpy(), ref) <= 5e-6 * max(mats[i].shape)


def test_graph_capture_replay(nla):
    # the whole batched call (prep + persistent kernel) is captured once and replayed;
    # work is handed out dynamically, so replays agree with the direct call to rounding
    ms, ns = inputs.batch_shapes(200, seed=7)
    mats = [inputs.gaussian(int(m), int(n), [7, i], dtype=np.float32) for i, (m, n) in enumerate(zip(ms, ns))]
    b = make_batch(nla, mats)
    S0, _ = nla.gesvd_vals_batched(b)
    torch.cuda.synchronize()
    first = [s.clone() for s in S0]
    for s in b.S:
        s.fill_(float("nan"))
    st = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(st):
        with torch.cuda.graph(g, stream=st):
            nla.gesvd_vals_batched(b, stream=st)
    for _ in range(2):
        g.replay()
        torch.cuda.synchronize()
        assert np.all(b.info.cpu().numpy() == 0)
        for A, a, s in zip(mats, first, b.S):
            sv = s.cpu().numpy().astype(np.float64)
            assert np.all(np.isfinite(sv))
            assert err_rel(sv, a.cpu().numpy().astype(np.float64)) <= 5e-6 * max(A.shape)
    check(b.S, b.info, mats[:40])


def test_unsorted_batch_over_the_sort_limit(nla):
    # above 16,384 matrices the batch is not sorted: the persistent kernel then also takes
    # the matrices too large for shared memory (global scratch); every 1000th is one
    g = np.random.default_rng(11)
    count = 16400
    mats = []
    for i in range(count):
        if i % 1000 == 500:
            mats.append(g.standard_normal((300, 200)).astype(np.float32))  # 60,000 elements
        else:
            n = int(g.integers(2, 9))
            mats.append(g.standard_normal((n + int(g.integers(0, 5)), n)).astype(np.float32))
    b = make_batch(nla, mats)
    S, info = nla.gesvd_vals_batched(b)
    torch.cuda.synchronize()
    assert np.all(info.cpu().numpy() == 0)
    check_ids = [i for i in range(count) if i % 1000 == 500] + list(range(0, count, 997))
    for i in check_ids:
        ref = oracle.svdvals(mats[i].astype(np.float64))
        assert err_rel(S[i].cpu().numpy(), ref) <= 5e-6 * max(mats[i].shape), (i, mats[i].shape)
