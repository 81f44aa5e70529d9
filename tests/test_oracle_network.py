"""CPU pin of the oracle's network chain: the LeNet-shaped network (conv, x^2,
pool, conv, x^2, pool, FC x3; Sec. 5, Implementation paragraph) evaluated
encrypted by the oracle at a reduced ring with the LeNet prime structure
(N = 2^10, 8 x 40-bit + 2 special primes, scale 2^35, the largest slot batch
BS = 8), decrypted and compared with the FP64 network of oracle/plain.py.

This pins the scale rule `henn.weight_scale` and the level chain on the CPU:
every linear layer's rescale must land on the scale the rule promises (Delta,
or sqrt(Delta q_{l-1}) before an x^2, whose own rescale brings it back to
Delta), and the decrypted logits must match the plaintext network."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import ckks, fragment, henn, plain


@pytest.fixture(scope="module")
def lenet_run():
    logN, delta = 10, 2.0 ** 35
    pr = ckks.Params(logN, 8, 2, 40, 40)
    BS = pr.N // 2 // 64  # S = 4 on the 28x28 input: m = 8, one channel per ciphertext
    wts = W.lenet_weights(0)
    lay = henn.lenet_layouts(pr.N, BS)
    keys = ckks.KeySet(pr, 9, rot_steps=henn.lenet_rotation_steps(pr.N, BS), relin=True)
    x = W.lenet_input(0, BS)
    slots = fragment.pack(lay, x)
    cts = [ckks.encrypt(pr, keys.sk, ckks.encode(pr, slots[i], pr.L, delta), 3, i) for i in range(lay.n_ct)]
    cnt = henn.Counters()
    out, P = henn.he_lenet(pr, keys, cts, lay, wts, delta, cnt=cnt)
    y = henn.lenet_decode_logits([ckks.decrypt(pr, keys.sk, c) for c in out], P, BS)
    return dict(pr=pr, delta=delta, BS=BS, x=x, wts=wts, out=out, y=y, cnt=cnt)


def test_lenet_chain_decrypts_to_the_fp64_network(lenet_run):
    r = lenet_run
    ref = plain.lenet(r["x"], r["wts"])
    assert np.abs(r["y"] - ref).max() < 1e-3
    # the logits are not trivially small: the comparison has something to compare
    assert np.abs(ref).max() > 0.1


def test_lenet_level_chain_and_final_scale(lenet_run):
    """Seven levels are consumed (conv, x^2, conv, x^2, FC x3) of the eight
    primes, and the final scale is Delta up to floating-point rounding of the
    scale bookkeeping."""
    r = lenet_run
    assert all(c.level == 0 for c in r["out"])
    assert r["out"][0].scale == pytest.approx(r["delta"], rel=1e-9)
    # Table 4 invariant: key switches - rotations = relinearisations, one per x^2 ciphertext
    cnt = r["cnt"]
    assert cnt.keyswitch - cnt.rot == cnt.cmult > 0


def test_weight_scale_lands_on_delta_or_its_square_root_form():
    """The rule of Sec. 4.3 / Sec. 5 restated as its purpose: a layer at level l
    with input scale s encodes at w = (t / s) q_l, so that s w / q_l = t, with
    t = Delta, or t = sqrt(Delta q_{l-1}) when x^2 follows (then t^2 / q_{l-1}
    = Delta after the activation's rescale).  Checked at every level of the
    LeNet prime chain and for input scales off Delta."""
    pr = ckks.Params(10, 8, 2, 40, 40)
    delta = 2.0 ** 35
    for level in range(1, pr.L + 1):
        q_l, q_lm1 = float(pr.moduli[level]), float(pr.moduli[level - 1])
        for s_in in (delta, delta * 1.37, delta / 3.1):
            w = henn.weight_scale(pr, level, s_in, delta, False)
            assert s_in * w / q_l == pytest.approx(delta, rel=1e-12)
            w = henn.weight_scale(pr, level, s_in, delta, True)
            t = s_in * w / q_l
            assert t == pytest.approx(math.sqrt(delta * q_lm1), rel=1e-12)
            assert t * t / q_lm1 == pytest.approx(delta, rel=1e-12)
