"""Seeded synthetic workloads: shapes, parameter sets and input tensors.

This module is the only one that both the CUDA path and the CPU oracle read.
It holds shapes and seeded random tensors, and none of the method's arithmetic.

The paper evaluates on MNIST / CIFAR-10 / ImageNet with trained weights, which
are not available here; uniform inputs and normally distributed weights of the
same shapes stand in for them.

Parameter sets (ring degree, prime counts and sizes, scale):
  conv1     one encrypted 5x5 conv 1->6 on a 28x28 input, N = 2^13,
            3 x 30-bit primes + 1 special prime, scale 2^25, fragment 4x4.
  lenet     LeNet-5-shaped network at N = 2^14, 8 x 40-bit + 2 special primes,
            scale 2^35, BS = 128 (the largest slot batch at S = 4).
  mobilenet three depthwise-3x3 + pointwise blocks at N = 2^16,
            24 x 36-bit + 4 special primes, scale 2^32.
The special-prime size is not fixed by these descriptions; conv1 uses a 50-bit
special prime (the hybrid key-switch noise with a 30-bit one is too large at
scale 2^25), the others continue the ciphertext primes' sequence.
"""
import numpy as np

PARAMS = {
    "conv1": dict(logN=13, n_q=3, k=1, bits=30, pbits=50, delta=2.0 ** 25),
    "lenet": dict(logN=14, n_q=8, k=2, bits=40, pbits=40, delta=2.0 ** 35),
    "mobilenet": dict(logN=16, n_q=24, k=4, bits=36, pbits=36, delta=2.0 ** 32),
    # reduced ring sizes with the same structure, for fast parity cases
    "tiny": dict(logN=10, n_q=3, k=1, bits=30, pbits=50, delta=2.0 ** 25),
    "lenet_small": dict(logN=12, n_q=8, k=2, bits=40, pbits=40, delta=2.0 ** 35),
    "mobilenet_small": dict(logN=12, n_q=6, k=2, bits=36, pbits=36, delta=2.0 ** 32),
}

# (H, Cin, Cout) of the three MobileNet-shaped blocks (depthwise 3x3 then 1x1)
MOBILENET_BLOCKS = [(112, 32, 64), (56, 128, 128), (14, 512, 512)]


def _rng(seed, stream):
    return np.random.default_rng([seed, stream])


def uniform_input(seed, shape, lo=0.0, hi=1.0, stream=0):
    """Activation tensor (BS, C, H, W) ~ U[lo, hi)."""
    return _rng(seed, stream).uniform(lo, hi, size=shape)


def normal_weight(seed, shape, std, stream=1):
    return _rng(seed, stream).normal(0.0, std, size=shape)


def conv1_workload(seed=0):
    """Config "single encrypted conv layer": x 1x1x28x28 ~ U[0,1), W 6x1x5x5 ~ N(0, 1/25)."""
    x = uniform_input(seed, (1, 1, 28, 28))
    w = normal_weight(seed, (6, 1, 5, 5), 1.0 / 5.0)
    return x, w


def lenet_weights(seed=0):
    """Random-init N(0, 1/fan_in) weights of the LeNet-5-shaped network."""
    shapes = {"conv1": (6, 1, 5, 5), "conv2": (16, 6, 5, 5), "fc1": (120, 256), "fc2": (84, 120),
              "fc3": (10, 84)}
    out = {}
    for i, (name, shp) in enumerate(shapes.items()):
        fan_in = int(np.prod(shp[1:]))
        out[name] = normal_weight(seed, shp, 1.0 / np.sqrt(fan_in), stream=10 + i)
    return out


def lenet_input(seed, BS):
    return uniform_input(seed, (BS, 1, 28, 28))


def mobilenet_block(seed, H, Cin, Cout, BS=1, block=0):
    """Depthwise 3x3 (Cin) then pointwise Cin->Cout; inputs ~ U[-1, 1),
    weights N(0, 1/fan_in)."""
    x = uniform_input(seed, (BS, Cin, H, H), -1.0, 1.0, stream=100 + block)
    wd = normal_weight(seed, (Cin, 1, 3, 3), 1.0 / 3.0, stream=200 + block)
    wp = normal_weight(seed, (Cout, Cin, 1, 1), 1.0 / np.sqrt(Cin), stream=300 + block)
    return x, wd, wp


def synthetic_layers(seed=0, n=200):
    """Config "learned fragment/schedule proposer": n conv layers drawn with seed:
    H = W log-uniform over [8, 224] (rounded to an integer), Cin and Cout
    log-uniform over [3, 512], K in {1, 3, 5}, stride in {1, 2},
    N in {2^14, 2^16}.  Returns a list of dicts; the first 80 % are the training
    split, the rest the test split."""
    rng = _rng(seed, 400)
    out = []
    for i in range(n):
        H = int(round(float(np.exp(rng.uniform(np.log(8), np.log(224))))))
        Cin = int(round(float(np.exp(rng.uniform(np.log(3), np.log(512))))))
        Cout = int(round(float(np.exp(rng.uniform(np.log(3), np.log(512))))))
        K = int(rng.choice([1, 3, 5]))
        stride = int(rng.choice([1, 2]))
        logN = int(rng.choice([14, 16]))
        out.append(dict(id=i, H=H, W=H, Cin=Cin, Cout=Cout, K=K, stride=stride, logN=logN,
                        split="train" if i < int(0.8 * n) else "test"))
    return out
