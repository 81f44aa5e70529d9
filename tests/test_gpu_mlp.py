"""The latency model's CUDA training and inference kernels against a plain
float64 NumPy restatement of the same model: standardisation, ReLU MLP forward,
MSE gradient, backward pass and Adam, from the same initial parameters."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2606_16359_b300 as fe  # noqa: E402


def unpack(params, dims):
    Ws, bs, o = [], [], 0
    for l in range(len(dims) - 1):
        n = dims[l] * dims[l + 1]
        Ws.append(params[o:o + n].reshape(dims[l + 1], dims[l]).astype(np.float64))
        o += n
        bs.append(params[o:o + dims[l + 1]].astype(np.float64))
        o += dims[l + 1]
    return Ws, bs


def ref_train(params, dims, X, y, steps, lr, wd):
    Ws, bs = unpack(params, dims)
    xm, xs = X.mean(0), X.std(0)
    xs = np.where(xs ** 2 > 1e-12, xs, 1.0)
    ym, ys = y.mean(), y.std()
    Z, t = (X - xm) / xs, (y - ym) / ys
    mW = [np.zeros_like(W) for W in Ws]
    vW = [np.zeros_like(W) for W in Ws]
    mb = [np.zeros_like(b) for b in bs]
    vb = [np.zeros_like(b) for b in bs]
    L, n = len(Ws), len(y)
    for step in range(1, steps + 1):
        acts = [Z]
        for l in range(L):
            a = acts[-1] @ Ws[l].T + bs[l]
            acts.append(a if l == L - 1 else np.maximum(a, 0))
        d = 2 * (acts[-1][:, 0] - t)[:, None] / n
        gW, gb = [None] * L, [None] * L
        for l in range(L - 1, -1, -1):
            gW[l] = d.T @ acts[l]
            gb[l] = d.sum(0)
            if l > 0:
                d = (d @ Ws[l]) * (acts[l] > 0)
        for l in range(L):
            for P_, G, M, V in ((Ws, gW, mW, vW), (bs, gb, mb, vb)):
                M[l] = 0.9 * M[l] + 0.1 * G[l]
                V[l] = 0.999 * V[l] + 0.001 * G[l] ** 2
                mh, vh = M[l] / (1 - 0.9 ** step), V[l] / (1 - 0.999 ** step)
                P_[l] = P_[l] - lr * (mh / (np.sqrt(vh) + 1e-8) + wd * P_[l])
    def predict(Xq):
        a = (Xq - xm) / xs
        for l in range(L):
            a = a @ Ws[l].T + bs[l]
            if l < L - 1:
                a = np.maximum(a, 0)
        return a[:, 0] * ys + ym
    return Ws, bs, predict


def test_mlp_train_and_predict_match_numpy():
    rng = np.random.default_rng(0)
    X = rng.normal(size=(96, 7)) * np.array([1, 10, 0.1, 3, 1, 1, 5]) + 2
    y = np.sin(X[:, 0]) + 0.1 * X[:, 1] - X[:, 3] ** 2 * 0.05
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        m = fe.MLP(7, hidden=64, n_hidden=3, seed=3)
        p0 = m.params()
        dims = [7, 64, 64, 64, 1]
        assert p0.size == sum(dims[l] * dims[l + 1] + dims[l + 1] for l in range(4))
        steps, lr, wd = 40, 3e-3, 1e-4
        m.train(X.astype(np.float32), y.astype(np.float32), steps=steps, lr=lr, weight_decay=wd)
        got = m.params()
        pred = m.predict(X[:10].astype(np.float32))
    Ws, bs, predict = ref_train(p0, dims, X.astype(np.float32).astype(np.float64),
                                y.astype(np.float32).astype(np.float64), steps, lr, wd)
    want = np.concatenate([np.concatenate([W.ravel(), b]) for W, b in zip(Ws, bs)])
    assert np.allclose(got, want, rtol=2e-3, atol=2e-4), np.abs(got - want).max()
    assert np.allclose(pred, predict(X[:10]), rtol=1e-3, atol=1e-3)


def test_mlp_learns_and_is_deterministic():
    rng = np.random.default_rng(1)
    X = rng.uniform(-2, 2, size=(256, 4)).astype(np.float32)
    y = (X[:, 0] * X[:, 1] + np.abs(X[:, 2]) - X[:, 3]).astype(np.float32)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        outs = []
        for _ in range(2):
            m = fe.MLP(4, seed=11)
            loss = m.train(X, y, steps=1500, lr=2e-3)
            outs.append(m.params())
        pred = m.predict(X)
    assert loss < 0.05
    assert np.array_equal(outs[0], outs[1])
    assert np.sqrt(np.mean((pred - y) ** 2)) < 0.3 * y.std()
