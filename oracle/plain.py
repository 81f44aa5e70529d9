"""FP64 plaintext reference of the layers the encrypted path evaluates.

Test infrastructure only (see oracle/__init__.py).

conv2d is Eq. 2 written out literally: Y[o, h, w] = sum_c sum_{i, j}
X[c, h + i, w + j] K[o, c, i, j] (valid cross-correlation; stride s keeps the
outputs with h, w divisible by s).  The activation, pooling and FC layers are
the ones named in the implementation paragraph of the evaluation setup:
a x^2 + b x + c activation, 2x2 average pooling, fully connected layers.
"""
import numpy as np


def conv2d(x, w, stride=1, depthwise=False):
    """x: (BS, Cin, H, W); w: (Cout, Cin, K, K), or (C, 1, K, K) when depthwise."""
    BS, Cin, H, W = x.shape
    K = w.shape[-1]
    Ho, Wo = (H - K) // stride + 1, (W - K) // stride + 1
    Cout = Cin if depthwise else w.shape[0]
    y = np.zeros((BS, Cout, Ho, Wo), dtype=np.float64)
    for o in range(Cout):
        chans = [o] if depthwise else range(Cin)
        for c in chans:
            wk = w[o, 0] if depthwise else w[o, c]
            for i in range(K):
                for j in range(K):
                    y[:, o] += wk[i, j] * x[:, c, i:i + stride * (Ho - 1) + 1:stride,
                                             j:j + stride * (Wo - 1) + 1:stride]
    return y


def poly_act(x, a=1.0, b=0.0, c=0.0):
    return a * x * x + b * x + c


def avgpool2(x):
    BS, C, H, W = x.shape
    Ho, Wo = H // 2, W // 2
    x = x[:, :, :2 * Ho, :2 * Wo]
    return 0.25 * (x[:, :, 0::2, 0::2] + x[:, :, 1::2, 0::2] + x[:, :, 0::2, 1::2] + x[:, :, 1::2, 1::2])


def fc(x, w):
    """x: (BS, F); w: (F_out, F)."""
    return x @ w.T


def lenet(x, weights, act=(1.0, 0.0, 0.0)):
    """conv5x5 1->6, act, avgpool2, conv5x5 6->16, act, avgpool2, FC 256->120->84->10;
    act = (a, b, c) of a x^2 + b x + c (x^2 by default)."""
    h = avgpool2(poly_act(conv2d(x, weights["conv1"]), *act))
    h = avgpool2(poly_act(conv2d(h, weights["conv2"]), *act))
    h = h.reshape(h.shape[0], -1)
    h = fc(h, weights["fc1"])
    h = fc(h, weights["fc2"])
    return fc(h, weights["fc3"])
