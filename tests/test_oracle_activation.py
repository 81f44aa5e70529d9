"""Pins of the oracle's polynomial activation a x^2 + b x + c (Sec. 5,
Implementation paragraph) and of AAC with its plaintext mask (Sec. 4.3, last
paragraph), against what the mathematics fixes: the FP64 polynomial, the
special case that reduces to the x^2 layer residue for residue, and the
replication of the valid channel blocks when the empty ones hold garbage."""
import numpy as np
import pytest

import workloads as W
from oracle import ckks, fragment, henn, plain


@pytest.fixture(scope="module")
def setup():
    pr = ckks.Params(10, 4, 1, 40, 40)
    keys = ckks.KeySet(pr, 12, rot_steps=[1, -128, -256], relin=True)
    return pr, keys


def test_nearest_int_rounds_half_away_from_zero_exactly():
    assert [ckks.nearest_int(v) for v in (0.5, -0.5, 1.5, -2.5, 2.4999999, -0.49999999999999994)] == \
        [1, -1, 2, -3, 2, 0]
    # the largest double below 1/2 rounds to 0 (a naive floor(x + 0.5) gives 1)
    assert ckks.nearest_int(0.49999999999999994) == 0
    big = 3.0 * 2.0 ** 70 + 2.0 ** 20
    assert ckks.nearest_int(big) == 3 * 2 ** 70 + 2 ** 20
    assert ckks.nearest_int(-big) == -(3 * 2 ** 70 + 2 ** 20)


def _decrypt2(pr, keys, ct):
    """Decrypt on the two limbs q_0 q_1 (CRT with Python integers, centred), for
    messages above q_0 / 2."""
    from oracle import _core as C
    q0, q1 = int(pr.moduli[0]), int(pr.moduli[1])
    r = []
    for t in (0, 1):
        q = pr.moduli[t]
        r.append([int(v) for v in pr.intt(C.vec_add(ct.c0[t], C.vec_mul(ct.c1[t], keys.sk.ntt[t], q), q), t)])
    Q, inv = q0 * q1, pow(q0, -1, q1)
    m = []
    for a0, a1 in zip(*r):
        v = a0 + q0 * (((a1 - a0) * inv) % q1)
        m.append(v - Q if v > Q // 2 else v)
    return C.decode(np.array(m, dtype=np.int64), pr.logN, ct.scale)


def _enc(pr, keys, z, scale, seed):
    return ckks.encrypt(pr, keys.sk, ckks.encode(pr, z, pr.L, scale), seed, 0)


def test_poly_act_with_a1_b0_c0_is_the_square_layer_residue_for_residue(setup):
    pr, keys = setup
    z = np.random.default_rng(1).uniform(-1, 1, pr.N // 2)
    ct = _enc(pr, keys, z, 2.0 ** 35, 3)
    sq = henn.he_square(pr, keys, [ct])[0]
    pa = henn.he_poly_act(pr, keys, [ct], 1.0, 0.0, 0.0)[0]
    assert np.array_equal(pa.as_array(), sq.as_array())
    assert pa.scale == sq.scale and pa.level == sq.level == pr.L - 1


@pytest.mark.parametrize("a,b,c", [(0.125, 0.5, 0.25), (-0.3, 0.2, -0.1), (2.0, 0.0, 0.0), (0.0, 0.7, 0.3),
                                   (0.0, 0.0, -0.4), (1e-3, 1.0, 0.0)])
def test_poly_act_decrypts_to_the_fp64_polynomial(setup, a, b, c):
    pr, keys = setup
    z = np.random.default_rng(2).uniform(-1, 1, pr.N // 2)
    ct = _enc(pr, keys, z, 2.0 ** 35, 4)
    out = henn.he_poly_act(pr, keys, [ct], a, b, c)[0]
    assert out.level == pr.L - 1
    y = ckks.decrypt(pr, keys.sk, out)
    assert np.abs(y - (a * z * z + b * z + c)).max() < 1e-3
    if a != 0:
        assert out.scale == (ct.scale * ct.scale) / (float(pr.moduli[pr.L]) * abs(a))
    else:
        assert out.scale == ct.scale


def test_masked_aac_replicates_valid_blocks_over_garbage(setup):
    """Empty channel blocks that hold garbage (here the constant an activation
    with c != 0 leaves there) break the plain rotate-and-add replication; the
    mask at Delta_2 zeroes them first, and the output decrypts at scale
    s Delta_2 to every channel position c holding channel c mod c_valid."""
    pr, keys = setup
    lay = fragment.Layout(pr.N, 8, 8, 8, 1, 1)  # m = 8, cpc = 8, 64 slots per channel block
    c_valid, blk = 2, lay.blk
    rng = np.random.default_rng(3)
    valid = rng.uniform(-1, 1, c_valid * blk)
    z = np.concatenate([valid, np.full(pr.N // 2 - c_valid * blk, 0.37)])  # garbage in the empty blocks
    ct = _enc(pr, keys, z, 2.0 ** 35, 5)
    want = np.tile(valid, lay.cpc // c_valid)
    plain_out = henn.aac_compress(pr, keys, [ct], lay, c_valid)[0]
    assert np.abs(ckks.decrypt(pr, keys.sk, plain_out) - want).max() > 0.1  # the garbage got added in
    d2 = 2.0 ** 20
    out = henn.aac_compress_masked(pr, keys, [ct], lay, c_valid, d2)[0]
    assert out.level == pr.L and out.scale == ct.scale * d2
    # the message at scale 2^55 exceeds q_0: decrypt it on q_0 q_1
    assert np.abs(_decrypt2(pr, keys, out) - want).max() < 1e-3
    mask = henn.aac_mask_slots(lay, c_valid)
    assert mask.sum() == c_valid * blk and set(np.unique(mask)) == {0.0, 1.0}


def test_conv_act_masked_aac_conv_chain_matches_fp64():
    """A channel-reducing 1x1 conv (4 -> 2 channels), the activation
    0.25 x^2 + 0.5 x + 0.3 (c != 0 fills the empty channel blocks), AAC with
    its mask at Delta_2 = 2^20, then a 1x1 conv 2 -> 4 reading the replicated
    channels, whose weights take the scale Delta_1 from the scale rule with the
    input scale s Delta_2: one rescale follows mask and weights together."""
    pr = ckks.Params(10, 5, 1, 40, 40)
    delta, d2 = 2.0 ** 35, 2.0 ** 20
    a, b, c = 0.25, 0.5, 0.3
    H, C0, C1, C2 = 8, 4, 2, 4
    rng = np.random.default_rng(6)
    x = rng.uniform(-1, 1, (1, C0, H, H))
    w1 = rng.normal(0, 0.5, (C1, C0, 1, 1))
    w2 = rng.normal(0, 0.5, (C2, C1, 1, 1))
    lay = fragment.Layout(pr.N, H, H, C0, 1, 1)
    lay1 = fragment.Layout(pr.N, H, H, C1, 1, 1)
    steps = set(henn.conv_rotation_steps(lay, C0, C1, 1)) | set(henn.aac_rotation_steps(lay1, C1))
    steps |= set(henn.conv_rotation_steps(lay1, C1, C2, 1, in_period=C1))
    keys = ckks.KeySet(pr, 8, rot_steps=sorted(steps), relin=True)
    slots = fragment.pack(lay, x)
    cts = [ckks.encrypt(pr, keys.sk, ckks.encode(pr, slots[i], pr.L, delta), 9, i) for i in range(lay.n_ct)]
    lv = pr.L
    h, l1 = henn.he_conv(pr, keys, cts, lay, w1, w_scale=henn.weight_scale(pr, lv, delta, delta, True))
    h = henn.he_poly_act(pr, keys, h, a, b, c)
    h = henn.aac_compress_masked(pr, keys, h, l1, C1, d2)
    lv = h[0].level
    ws = henn.weight_scale(pr, lv, h[0].scale, delta, False)
    out, l2 = henn.he_conv(pr, keys, h, l1, w2, in_period=C1, w_scale=ws)
    y = fragment.unpack(l2, np.stack([ckks.decrypt(pr, keys.sk, o) for o in out]))
    t = plain.conv2d(x, w1)
    ref = plain.conv2d(a * t * t + b * t + c, w2)
    assert np.abs(y - ref).max() < 1e-3
    assert out[0].scale == pytest.approx(delta, rel=1e-9)
