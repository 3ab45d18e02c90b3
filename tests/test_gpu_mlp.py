"""GPU tests of the learned cost model's kernels against the FP64 MLP oracle."""
import numpy as np
import pytest

from oracle import mlp as omlp

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kt():
    from paper_2608_21227_gb300 import kt as _kt

    _kt.lib()
    return _kt


def pack(params):
    return np.concatenate([np.concatenate([W.ravel(), b]) for W, b in params]).astype(np.float32)


def unpack(vec, params_like):
    out, o = [], 0
    for W, b in params_like:
        nW = W.size
        out.append((vec[o:o + nW].reshape(W.shape), vec[o + nW:o + nW + b.size]))
        o += nW + b.size
    return out


def test_forward_backward_match_oracle(kt):
    params = omlp.init(15, seed=3)
    p32 = pack(params)
    assert p32.size == kt.mlp_param_count()
    params = unpack(p32.astype(np.float64), params)  # the oracle sees the FP32-rounded weights
    g = np.random.default_rng(4)
    X = g.standard_normal((200, 15)).astype(np.float32)
    y = g.standard_normal(200).astype(np.float32)
    pred, grads = kt.mlp_forward_backward(torch.from_numpy(p32).cuda(), torch.from_numpy(X).cuda(),
                                          torch.from_numpy(y).cuda())
    torch.cuda.synchronize()
    p_ref, _ = omlp.forward(params, X.astype(np.float64))
    g_ref = omlp.backward(params, X.astype(np.float64), y.astype(np.float64))
    assert np.max(np.abs(pred.cpu().numpy() - p_ref)) <= 1e-3 * max(1.0, np.max(np.abs(p_ref)))
    g_gpu = unpack(grads.cpu().numpy().astype(np.float64), params)
    for (gW, gb), (rW, rb) in zip(g_gpu, g_ref):
        for a, r in ((gW, rW), (gb, rb)):
            assert np.max(np.abs(a - r)) <= 1e-3 * max(1e-6, np.max(np.abs(r)))


def test_adam_step_matches_oracle(kt):
    params = omlp.init(15, seed=5)
    p32 = pack(params)
    params = unpack(p32.astype(np.float64), params)
    g = np.random.default_rng(6)
    grads = [(g.standard_normal(W.shape), g.standard_normal(b.shape)) for W, b in params]
    g32 = pack(grads)
    grads = unpack(g32.astype(np.float64), grads)
    opt = omlp.Adam(params, lr=1e-2)
    P = torch.from_numpy(p32).cuda()
    G = torch.from_numpy(g32).cuda()
    M = torch.zeros_like(P)
    V = torch.zeros_like(P)
    ref = params
    for t in range(1, 4):
        kt.mlp_adam_step(P, G, M, V, t, 1e-2)
        ref = opt.step(ref, grads)
    torch.cuda.synchronize()
    assert np.max(np.abs(P.cpu().numpy() - pack(ref))) <= 1e-5


def test_training_learns_a_known_surface(kt, tmp_path):
    # log runtime = a smooth function of the features; the trained model must fit it
    g = np.random.default_rng(7)
    X = g.uniform(0, 1, size=(4096, 15)).astype(np.float32)
    y = (np.sin(3 * X[:, 0]) + X[:, 1] * X[:, 2] - 0.5 * X[:, 3] ** 2).astype(np.float32)
    model = str(tmp_path / "m.bin")
    loss = kt.mlp_train(X, y, epochs=60, batch=256, lr=2e-3, seed=1, model_path=model)
    pred = kt.mlp_predict(model, X[:512])
    mse = float(np.mean((pred - y[:512]) ** 2))
    assert mse < 0.1 * float(np.var(y)), (mse, float(np.var(y)), loss)
