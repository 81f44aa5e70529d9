"""Plaintext FP64 reference of the encrypted layers (what a client would compute
in the clear), used to report the decrypted error of the benchmark workloads.
Valid cross-correlation as in Eq. 2 (torch.nn.functional.conv2d, float64)."""
import numpy as np


def conv2d(x, w, stride=1, depthwise=False):
    import torch
    import torch.nn.functional as F
    xt = torch.from_numpy(np.asarray(x, dtype=np.float64))
    wt = torch.from_numpy(np.asarray(w, dtype=np.float64))
    y = F.conv2d(xt, wt, stride=stride, groups=xt.shape[1] if depthwise else 1)
    return y.numpy()


def poly_act(x, a, b, c):
    """a x^2 + b x + c elementwise (float64)."""
    x = np.asarray(x, dtype=np.float64)
    return a * x * x + b * x + c


def lenet(x, weights):
    """The LeNet-5-shaped network in the clear (float64): two 5x5 valid convs,
    each followed by x^2 and 2x2 average pooling, then FC 256 -> 120 -> 84 -> 10
    with no activation between the FC layers."""
    import torch
    import torch.nn.functional as F
    t = lambda a: torch.from_numpy(np.asarray(a, dtype=np.float64))
    h = t(x)
    for name in ("conv1", "conv2"):
        h = F.avg_pool2d(F.conv2d(h, t(weights[name])) ** 2, 2)
    h = h.flatten(1)
    for name in ("fc1", "fc2", "fc3"):
        h = F.linear(h, t(weights[name]))
    return h.numpy()
