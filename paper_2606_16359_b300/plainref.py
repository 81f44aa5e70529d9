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
