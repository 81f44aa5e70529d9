"""Pins of the FP64 plaintext layers (oracle/plain.py), the ground truth that
decrypted results are compared with.  Each layer is checked against a library
routine or a brute-force sum written independently of it:

- conv2d (Eq. 2, valid cross-correlation) against scipy.signal.correlate2d
  summed over input channels, with non-symmetric kernels so that a transposed
  or flipped kernel fails, and stride 2 as the stride-1 result subsampled;
- depthwise conv against per-channel correlate2d;
- avgpool2 against a reshape-mean of the 2x2 windows;
- fc against an explicit double loop;
- the LeNet-shaped composition against the layers applied one by one, with the
  flatten order (channel, row, column) that FC 256 = 16 x 4 x 4 needs.
"""
import numpy as np
import pytest
from scipy.signal import correlate2d

from oracle import plain


@pytest.mark.parametrize("H,Cin,Cout,K", [(8, 1, 2, 3), (9, 3, 4, 5), (6, 2, 3, 1)])
def test_conv2d_is_valid_cross_correlation(H, Cin, Cout, K):
    rng = np.random.default_rng(H * 100 + K)
    x = rng.normal(size=(2, Cin, H, H + 1))
    w = rng.normal(size=(Cout, Cin, K, K))
    y = plain.conv2d(x, w)
    assert y.shape == (2, Cout, H - K + 1, H + 2 - K)
    for b in range(2):
        for o in range(Cout):
            want = sum(correlate2d(x[b, c], w[o, c], mode="valid") for c in range(Cin))
            assert np.allclose(y[b, o], want, rtol=0, atol=1e-12)
    # a flipped kernel (convolution instead of correlation) gives another answer
    yf = plain.conv2d(x, w[:, :, ::-1, ::-1].copy())
    if K > 1:
        assert not np.allclose(yf, y)


def test_conv2d_stride_two_is_subsampled_stride_one():
    rng = np.random.default_rng(5)
    x = rng.normal(size=(1, 3, 11, 11))
    w = rng.normal(size=(2, 3, 3, 3))
    y1 = plain.conv2d(x, w)
    y2 = plain.conv2d(x, w, stride=2)
    assert np.allclose(y2, y1[:, :, ::2, ::2], rtol=0, atol=1e-12)


def test_depthwise_conv_is_per_channel_correlation():
    rng = np.random.default_rng(6)
    x = rng.normal(size=(2, 4, 7, 7))
    w = rng.normal(size=(4, 1, 3, 3))
    y = plain.conv2d(x, w, depthwise=True)
    for b in range(2):
        for c in range(4):
            assert np.allclose(y[b, c], correlate2d(x[b, c], w[c, 0], mode="valid"), rtol=0, atol=1e-12)


def test_avgpool_and_fc_and_activation():
    rng = np.random.default_rng(7)
    x = rng.normal(size=(3, 2, 8, 6))
    want = x.reshape(3, 2, 4, 2, 3, 2).mean(axis=(3, 5))
    assert np.allclose(plain.avgpool2(x), want, rtol=0, atol=1e-14)
    v = rng.normal(size=(4, 5))
    w = rng.normal(size=(3, 5))
    loop = np.array([[sum(v[b, f] * w[n, f] for f in range(5)) for n in range(3)] for b in range(4)])
    assert np.allclose(plain.fc(v, w), loop, rtol=0, atol=1e-12)
    assert np.allclose(plain.poly_act(v, 2.0, -1.0, 0.5), 2 * v ** 2 - v + 0.5)


def test_lenet_composition_and_flatten_order():
    import workloads as W
    wts = W.lenet_weights(0)
    x = W.lenet_input(0, 3)
    h = plain.avgpool2(plain.conv2d(x, wts["conv1"]) ** 2)
    assert h.shape == (3, 6, 12, 12)
    h = plain.avgpool2(plain.conv2d(h, wts["conv2"]) ** 2)
    assert h.shape == (3, 16, 4, 4)
    f = np.stack([[h[b, c, i, j] for c in range(16) for i in range(4) for j in range(4)] for b in range(3)])
    y = f @ wts["fc1"].T @ wts["fc2"].T @ wts["fc3"].T
    assert np.allclose(plain.lenet(x, wts), y, rtol=1e-12, atol=1e-12)
