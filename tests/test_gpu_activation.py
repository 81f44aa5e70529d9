"""GPU parity of the polynomial activation a x^2 + b x + c (Sec. 5,
Implementation), AAC with its plaintext mask (Sec. 4.3, last paragraph), the
library's scale rule and the FC-from-layout plans, through the C ABI, against
the oracle (residues bit for bit) and the FP64 definitions."""
import numpy as np
import pytest

import workloads as W
from oracle import ckks, fragment, henn, plain

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2606_16359_b300 as fe  # noqa: E402
from paper_2606_16359_b300.net import LeNet  # noqa: E402

ARGS = (10, 4, 1, 40, 40)
DELTA = 2.0 ** 35


def u64(t):
    return t.detach().cpu().numpy().view(np.uint64)


@pytest.fixture(scope="module")
def env():
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        ctx = fe.Context(*ARGS)
        sk = ctx.sk_gen(12)
        evk = ctx.evk_gen(sk, 12, [1, -128, -256], relin=True)
    pr = ckks.Params(*ARGS)
    keys = ckks.KeySet(pr, 12, rot_steps=[1, -128, -256], relin=True)
    return s, ctx, sk, evk, pr, keys


@pytest.mark.parametrize("a,b,c", [(1.0, 0.0, 0.0), (0.125, 0.5, 0.25), (-0.3, 0.2, -0.1), (0.0, 0.7, 0.3),
                                   (1e-3, 1.0, 0.0)])
def test_poly_act_bit_exact_to_the_oracle(env, a, b, c):
    s, ctx, sk, evk, pr, keys = env
    z = np.random.default_rng(2).uniform(-1, 1, (2, pr.N // 2))
    with torch.cuda.stream(s):
        ct = ctx.encrypt(sk, torch.from_numpy(z), ctx.L, DELTA, 4, ct_id0=0)
        out, sc = ctx.he_poly_act(evk, ct, ctx.L, DELTA, a, b, c)
        got = u64(out)
        y = ctx.decrypt(sk, out, ctx.L - 1, sc).cpu().numpy()
        if (a, b, c) == (1.0, 0.0, 0.0):
            assert np.array_equal(got, u64(ctx.he_square(evk, ct, ctx.L)))
        assert sc == ctx.poly_act_scale(ctx.L, DELTA, a)
    octs = [ckks.encrypt(pr, keys.sk, ckks.encode(pr, z[i], pr.L, DELTA), 4, i) for i in range(2)]
    oout = henn.he_poly_act(pr, keys, octs, a, b, c)
    assert np.array_equal(got, np.stack([o.as_array() for o in oout]))
    assert sc == oout[0].scale
    assert np.abs(y - (a * z * z + b * z + c)).max() < 1e-3


def test_masked_compress_bit_exact_to_the_oracle(env):
    s, ctx, sk, evk, pr, keys = env
    c_valid, d2 = 2, 2.0 ** 20
    rng = np.random.default_rng(3)
    blk = 64
    z = np.concatenate([rng.uniform(-1, 1, c_valid * blk), np.full(pr.N // 2 - c_valid * blk, 0.37)])
    with torch.cuda.stream(s):
        lay = ctx.layout(8, 8, 8, 1, 1)
        assert lay.cpc == 8 and lay.m == 8
        ct = ctx.encrypt(sk, torch.from_numpy(z[None]), ctx.L, DELTA, 5, ct_id0=0)
        out, sc = ctx.compress_masked(evk, lay, c_valid, d2, ct, ctx.L, DELTA)
        got = u64(out)
    olay = fragment.Layout(pr.N, 8, 8, 8, 1, 1)
    oct0 = ckks.encrypt(pr, keys.sk, ckks.encode(pr, z, pr.L, DELTA), 5, 0)
    oout = henn.aac_compress_masked(pr, keys, [oct0], olay, c_valid, d2)
    assert np.array_equal(got[0], oout[0].as_array())
    assert sc == oout[0].scale == DELTA * d2


def test_scale_rule_matches_the_oracle(env):
    s, ctx, sk, evk, pr, keys = env
    for level in range(1, pr.L + 1):
        for s_in in (DELTA, DELTA * 1.37):
            for a in (0.0, 1.0, 0.125, -0.3):
                assert ctx.weight_scale(level, s_in, DELTA, a) == henn.weight_scale(pr, level, s_in, DELTA, a)
    with pytest.raises(fe.FencError):
        ctx.weight_scale(0, DELTA, DELTA)


def test_conv_act_masked_aac_conv_chain_bit_exact_and_fp64():
    """Channel-reducing 1x1 conv 4 -> 2, 0.25 x^2 + 0.5 x + 0.3 (fills the empty
    channel blocks with 0.3), masked AAC at Delta_2 = 2^20, 1x1 conv 2 -> 4 on
    the replicated channels with its weights at the scale the rule gives
    (Delta_1 = q_l t / (s Delta_2)): residues equal the oracle's, decryption
    equals the FP64 chain."""
    args = (10, 5, 1, 40, 40)
    a, b, c, d2 = 0.25, 0.5, 0.3, 2.0 ** 20
    H, C0, C1, C2 = 8, 4, 2, 4
    rng = np.random.default_rng(6)
    x = rng.uniform(-1, 1, (1, C0, H, H))
    w1 = rng.normal(0, 0.5, (C1, C0, 1, 1))
    w2 = rng.normal(0, 0.5, (C2, C1, 1, 1))
    pr = ckks.Params(*args)
    lay = fragment.Layout(pr.N, H, H, C0, 1, 1)
    lay1 = fragment.Layout(pr.N, H, H, C1, 1, 1)
    steps = set(henn.conv_rotation_steps(lay, C0, C1, 1)) | set(henn.aac_rotation_steps(lay1, C1))
    steps |= set(henn.conv_rotation_steps(lay1, C1, C2, 1, in_period=C1))
    steps = sorted(steps)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        ctx = fe.Context(*args)
        L = ctx.L
        sk = ctx.sk_gen(8)
        evk = ctx.evk_gen(sk, 8, steps, relin=True)
        glay = ctx.layout(H, H, C0, 1, 1)
        p1 = ctx.plan_conv(glay, C1, 1, level=L)
        assert sorted(set(p1.steps)) == sorted(set(henn.conv_rotation_steps(lay, C0, C1, 1)))
        pt1 = ctx.load_weights(p1, w1, ctx.weight_scale(L, DELTA, DELTA, a))
        ct = ctx.encrypt(sk, ctx.pack(glay, torch.from_numpy(x)), L, DELTA, 9, ct_id0=0)
        h = ctx.he_conv(evk, p1, pt1, ct)
        sc = ctx.plan_out_scale(p1, DELTA)
        h, sc = ctx.he_poly_act(evk, h, L - 1, sc, a, b, c)
        l1 = p1.out_layout
        h, sc = ctx.compress_masked(evk, l1, C1, d2, h, L - 2, sc)
        p2 = ctx.plan_conv(l1, C2, 1, in_period=C1, level=L - 2)
        pt2 = ctx.load_weights(p2, w2, ctx.weight_scale(L - 2, sc, DELTA))
        out = ctx.he_conv(evk, p2, pt2, h)
        sc2 = ctx.plan_out_scale(p2, sc)
        got = u64(out)
        y = ctx.unpack(p2.out_layout, ctx.decrypt(sk, out, L - 3, sc2)).cpu().numpy()
        assert ctx.device_status() == 0
    keys = ckks.KeySet(pr, 8, rot_steps=steps, relin=True)
    slots = fragment.pack(lay, x)
    cts = [ckks.encrypt(pr, keys.sk, ckks.encode(pr, slots[i], pr.L, DELTA), 9, i) for i in range(lay.n_ct)]
    oh, ol1 = henn.he_conv(pr, keys, cts, lay, w1, w_scale=henn.weight_scale(pr, pr.L, DELTA, DELTA, a))
    oh = henn.he_poly_act(pr, keys, oh, a, b, c)
    oh = henn.aac_compress_masked(pr, keys, oh, ol1, C1, d2)
    oout, _ = henn.he_conv(pr, keys, oh, ol1, w2, in_period=C1,
                           w_scale=henn.weight_scale(pr, oh[0].level, oh[0].scale, DELTA, 0))
    assert np.array_equal(got, np.stack([o.as_array() for o in oout]))
    assert sc2 == oout[0].scale
    t = plain.conv2d(x, w1)
    assert np.abs(y - plain.conv2d(a * t * t + b * t + c, w2)).max() < 1e-3


def test_lenet_with_a_general_activation_bit_exact_at_a_reduced_ring():
    """The LeNet-shaped network with 0.125 x^2 + 0.5 x + 0.25 in place of x^2:
    every scale from the library (fe_weight_scale with the activation's a,
    fe_plan_out_scale, fe_poly_act_scale), the FC plans from the pooled layout
    (fe_plan_fc_layout, fe_plan_fc_next) and the logits read back by
    fe_fc_unpack; the residues equal the oracle's and the logits the FP64
    network's."""
    logN, act = 11, (0.125, 0.5, 0.25)
    wts = W.lenet_weights(0)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        ctx = fe.Context(logN, 8, 2, 40, 40)
        net = LeNet(ctx, DELTA, wts, key_seed=9, act=act)
        x = W.lenet_input(0, net.BS)
        out = net.forward(net.encrypt(x, seed=3), mode=1)
        got = u64(out)
        y = net.decode_logits(out)
    pr = ckks.Params(logN, 8, 2, 40, 40)
    lay = henn.lenet_layouts(pr.N, net.BS)
    keys = ckks.KeySet(pr, 9, rot_steps=henn.lenet_rotation_steps(pr.N, net.BS), relin=True)
    slots = fragment.pack(lay, x)
    octs = [ckks.encrypt(pr, keys.sk, ckks.encode(pr, slots[i], pr.L, DELTA), 3, i) for i in range(lay.n_ct)]
    oout, P = henn.he_lenet(pr, keys, octs, lay, wts, DELTA, act=act)
    assert np.array_equal(got, np.stack([c.as_array() for c in oout]))
    assert oout[0].scale == net.out_scale
    assert np.abs(y - plain.lenet(x, wts, act)).max() < 1e-3
