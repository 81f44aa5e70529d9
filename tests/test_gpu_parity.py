"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Residues must be bit-exact: NTT, keys, encoding, encryption, rotation,
rescale, PMult, the fragment convolution (plain and batched paths), FC, x^2,
pooling and AAC, from the same seeds and seeded inputs.  Decrypted outputs are
also checked against the FP64 definitions within 1e-3.
"""
import numpy as np
import pytest

import workloads as W
from oracle import _core as C
from oracle import ckks, fragment, henn, plain

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2606_16359_b300 as fe  # noqa: E402


def u64(t):
    return t.detach().cpu().numpy().view(np.uint64)


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int64)).cuda()


def oracle_ct_array(cts):
    return np.stack([c.as_array() for c in cts])


class Pair:
    """A parameter set instantiated on both sides."""

    def __init__(self, logN, n_q, k, bits, pbits=None):
        self.pr = ckks.Params(logN, n_q, k, bits, pbits)
        self.g = fe.Context(logN, n_q, k, bits, pbits if pbits is not None else bits)
        assert self.g.moduli == self.pr.moduli


@pytest.fixture(scope="module")
def tiny():
    p = W.PARAMS["tiny"]
    return Pair(p["logN"], p["n_q"], p["k"], p["bits"], p["pbits"])


@pytest.fixture(scope="module")
def ks2():
    return Pair(7, 4, 2, 40)


@pytest.mark.parametrize("args", [(10, 3, 1, 30, 50), (12, 4, 2, 40, 40), (13, 2, 1, 36, 60), (16, 2, 1, 36, 36),
                                  (14, 3, 2, 40, 40)])
def test_ntt_parity(args):
    pr = ckks.Params(*args)
    g = fe.Context(*args)
    assert g.moduli == pr.moduli
    rng = np.random.default_rng(args[0])
    a = np.stack([rng.integers(0, q, pr.N, dtype=np.uint64) for q in pr.moduli])[None]
    d = to_dev(a)
    g.ntt(d)
    want = np.stack([pr.ntt(a[0, i], i) for i in range(len(pr.moduli))])
    assert np.array_equal(u64(d)[0], want)
    g.ntt(d, inverse=True)
    assert np.array_equal(u64(d)[0], a[0])


@pytest.mark.parametrize("which", ["tiny", "ks2"])
def test_keys_parity(which, tiny, ks2):
    P = tiny if which == "tiny" else ks2
    pr, g = P.pr, P.g
    steps = [1, 5, -3]
    keys = ckks.KeySet(pr, 77, rot_steps=steps, relin=True)
    sk = g.sk_gen(77)
    assert np.array_equal(u64(sk), keys.sk.ntt)
    evk = g.evk_gen(sk, 77, steps, relin=True)
    kb = u64(evk.buf)
    dnum = len(pr.digits(pr.L))
    nm = len(pr.moduli)
    per = dnum * 2 * nm * pr.N
    for idx, r in enumerate(sorted(steps)):
        sw = keys.rot[pr.galois(r)]
        got = kb[idx * per:(idx + 1) * per].reshape(dnum, 2, nm, pr.N)
        for j in range(dnum):
            assert np.array_equal(got[j, 0], sw.b[j]) and np.array_equal(got[j, 1], sw.a[j])
    got = kb[len(steps) * per:(len(steps) + 1) * per].reshape(dnum, 2, nm, pr.N)
    for j in range(dnum):
        assert np.array_equal(got[j, 0], keys.relin.b[j]) and np.array_equal(got[j, 1], keys.relin.a[j])


def test_evk_upload_from_host_equals_generated(tiny):
    """Keys generated on one side and indexed from their host bytes on the
    other (fe_evk_upload) give the same rotations and relinearisations bit for
    bit; host bytes shorter than the keys are rejected."""
    pr, g = tiny.pr, tiny.g
    sk = g.sk_gen(21)
    steps = [-2, 1, 5]
    evk = g.evk_gen(sk, 21, steps, relin=True)
    host = evk.buf.cpu()
    evk2 = g.evk_upload(host, evk.steps, relin=True)
    z = np.random.default_rng(21).uniform(-1, 1, (2, pr.N // 2))
    ct = g.encrypt(sk, torch.from_numpy(z), pr.L, 2.0 ** 25, seed=3)
    for r in steps:
        assert np.array_equal(u64(g.rotate(evk, ct, pr.L, r)), u64(g.rotate(evk2, ct, pr.L, r))), r
    assert np.array_equal(u64(g.he_square(evk, ct, pr.L)), u64(g.he_square(evk2, ct, pr.L)))
    with pytest.raises(fe.FencError):
        g.evk_upload(host[:16], evk.steps, relin=True)


def test_chacha20_generator_parity():
    """ChaCha20 (RFC 8439) as the generator on both sides: the secret key, the
    evaluation keys (b and a of every digit), fresh ciphertexts and a rotation
    are bit-exact to the oracle's, and differ from the SplitMix64 ones."""
    key6 = [0x01234567, 0x89abcdef, 0x0badf00d, 0xdeadbeef, 0x13579bdf, 0x2468ace0]
    P = Pair(10, 3, 1, 30, 50)
    pr, g = P.pr, P.g
    g.set_generator("chacha20", key6)
    C.set_generator("chacha20", np.array(key6, dtype=np.uint32))
    try:
        steps = [1, -3]
        keys = ckks.KeySet(pr, 5, rot_steps=steps, relin=True)
        sk = g.sk_gen(5)
        assert np.array_equal(u64(sk), keys.sk.ntt)
        evk = g.evk_gen(sk, 5, steps, relin=True)
        kb = u64(evk.buf)
        dnum, nm = len(pr.digits(pr.L)), len(pr.moduli)
        per = dnum * 2 * nm * pr.N
        for idx, r in enumerate(sorted(steps)):
            got = kb[idx * per:(idx + 1) * per].reshape(dnum, 2, nm, pr.N)
            sw = keys.rot[pr.galois(r)]
            for j in range(dnum):
                assert np.array_equal(got[j, 0], sw.b[j]) and np.array_equal(got[j, 1], sw.a[j])
        z = np.random.default_rng(8).uniform(-1, 1, (2, pr.N // 2))
        octs = [ckks.encrypt(pr, keys.sk, ckks.encode(pr, z[i], pr.L, 2.0 ** 25), 2, i) for i in range(2)]
        ct = g.encrypt(sk, torch.from_numpy(z), pr.L, 2.0 ** 25, seed=2)
        assert np.array_equal(u64(ct), oracle_ct_array(octs))
        for r in steps:
            want = oracle_ct_array([ckks.rotate(pr, keys, c, r) for c in octs])
            assert np.array_equal(u64(g.rotate(evk, ct, pr.L, r)), want), r
        y = g.decrypt(sk, g.rotate(evk, ct, pr.L, 1), pr.L, 2.0 ** 25).cpu().numpy()
        assert np.abs(y - np.roll(z, -1, axis=1)).max() < 1e-3
    finally:
        C.set_generator("splitmix64")
    g2 = fe.Context(10, 3, 1, 30, 50)
    assert not np.array_equal(u64(g2.sk_gen(5)), u64(sk))


def test_encode_encrypt_decrypt_parity(tiny):
    pr, g = tiny.pr, tiny.g
    rng = np.random.default_rng(3)
    z = rng.uniform(-1, 1, (3, pr.N // 2))
    for scale, level in [(2.0 ** 25, pr.L), (float(pr.q[-1]), 1), (2.0 ** 40 * 1.37, 2)]:
        pt = g.encode(torch.from_numpy(z), level, scale)
        want = np.stack([ckks.encode(pr, z[i], level, scale).m for i in range(3)])
        assert np.array_equal(u64(pt), want)
    keys = ckks.KeySet(pr, 5)
    sk = g.sk_gen(5)
    ct = g.encrypt(sk, torch.from_numpy(z), pr.L, 2.0 ** 25, seed=9, ct_id0=4)
    want = oracle_ct_array([ckks.encrypt(pr, keys.sk, ckks.encode(pr, z[i], pr.L, 2.0 ** 25), 9, 4 + i)
                            for i in range(3)])
    assert np.array_equal(u64(ct), want)
    dec = g.decrypt(sk, ct, pr.L, 2.0 ** 25).cpu().numpy()
    assert np.abs(dec - z).max() < 1e-5
    dec0 = g.decrypt(sk, ct[:, :, :1].contiguous(), 0, 2.0 ** 25).cpu().numpy()
    assert np.abs(dec0 - z).max() < 1e-5


@pytest.mark.parametrize("which", ["tiny", "ks2"])
def test_rotate_rescale_pmult_add_parity(which, tiny, ks2):
    P = tiny if which == "tiny" else ks2
    pr, g = P.pr, P.g
    steps = [1, 3, -2, pr.N // 8]
    keys = ckks.KeySet(pr, 11, rot_steps=steps)
    sk = g.sk_gen(11)
    evk = g.evk_gen(sk, 11, steps)
    rng = np.random.default_rng(4)
    z = rng.uniform(-1, 1, (2, pr.N // 2))
    octs = [ckks.encrypt(pr, keys.sk, ckks.encode(pr, z[i], pr.L, 2.0 ** 25), 2, i) for i in range(2)]
    ct = g.encrypt(sk, torch.from_numpy(z), pr.L, 2.0 ** 25, seed=2)
    assert np.array_equal(u64(ct), oracle_ct_array(octs))
    wants = {}
    for r in steps:
        got = g.rotate(evk, ct, pr.L, r)
        wants[r] = oracle_ct_array([ckks.rotate(pr, keys, c, r) for c in octs])
        assert np.array_equal(u64(got), wants[r]), r
    # hoisted: one ModUp per ciphertext for every step (and the identity step 0)
    many = u64(g.rotate_many(evk, ct, pr.L, steps + [0]))
    for j, r in enumerate(steps):
        assert np.array_equal(many[j], wants[r]), r
    assert np.array_equal(many[len(steps)], u64(ct))
    w = rng.uniform(-1, 1, (2, pr.N // 2))
    pts = g.encode(torch.from_numpy(w), pr.L, float(pr.q[pr.L]))
    opts = [ckks.encode(pr, w[i], pr.L, float(pr.q[pr.L])) for i in range(2)]
    pm = g.pmult(ct, pts, pr.L)
    opm = [ckks.pmult(pr, octs[i], opts[i]) for i in range(2)]
    assert np.array_equal(u64(pm), oracle_ct_array(opm))
    rs = g.rescale(pm, pr.L)
    assert np.array_equal(u64(rs), oracle_ct_array([ckks.rescale(pr, c) for c in opm]))
    ad = g.add(ct, ct, pr.L)
    assert np.array_equal(u64(ad), oracle_ct_array([ckks.add(pr, c, c) for c in octs]))


ORACLE_HOIST = {0: "single", 1: "double", 2: "double_fused"}


def run_conv_pair(P, x, w, S, stride=1, depthwise=False, seed=3, delta=2.0 ** 25, modes=(0, 1), bsgs_n1=0,
                  double_hoist=False, check_counts=True):
    pr, g = P.pr, P.g
    BS, C, H, _ = x.shape
    Cout = w.shape[0]
    K = w.shape[-1]
    olay = fragment.Layout(pr.N, H, H, C, BS, S)
    steps = henn.conv_rotation_steps(olay, C, Cout, K, stride, depthwise, bsgs_n1=bsgs_n1)
    keys = ckks.KeySet(pr, seed, rot_steps=steps)
    slots = fragment.pack(olay, x)
    octs = [ckks.encrypt(pr, keys.sk, ckks.encode(pr, slots[i], pr.L, delta), 17, i) for i in range(olay.n_ct)]
    ocnt = henn.Counters()
    oout, oolay = henn.he_conv(pr, keys, octs, olay, w, stride=stride, depthwise=depthwise, cnt=ocnt,
                               bsgs_n1=bsgs_n1, hoist=ORACLE_HOIST[fe._hoisting(double_hoist)])
    want = oracle_ct_array(oout)

    lay = g.layout(H, H, C, BS, S)
    plan = g.plan_conv(lay, Cout, K, stride=stride, depthwise=depthwise, level=pr.L, bsgs_n1=bsgs_n1,
                       double_hoist=double_hoist)
    assert sorted(plan.steps) == sorted(steps)
    if check_counts:  # the plan is structural; the oracle also drops plaintexts that are zero by value
        assert plan.info.n_inner_rot + plan.info.n_outer_rot == ocnt.rot
        assert plan.info.n_pt == ocnt.pmult
    sk = g.sk_gen(seed)
    evk = g.evk_gen(sk, seed, plan.steps)
    xs = g.pack(lay, torch.from_numpy(x))
    assert np.array_equal(xs.cpu().numpy(), slots)
    ct = g.encrypt(sk, xs, pr.L, delta, seed=17)
    pt = g.load_weights(plan, w, float(pr.q[pr.L]))
    outs = {}
    for mode in modes:
        outs[mode] = g.he_conv(evk, plan, pt, ct, mode=mode)
        assert np.array_equal(u64(outs[mode]), want), f"mode {mode}"
    y = g.unpack(plan.out_layout, g.decrypt(sk, outs[modes[-1]], pr.L - 1, delta)).cpu().numpy()
    ref = plain.conv2d(x, w, stride=stride, depthwise=depthwise)
    assert np.abs(y - ref).max() < 1e-3
    return plan, outs


@pytest.mark.parametrize("H,C,Co,K,BS,S,stride", [
    (8, 3, 5, 3, 2, 2, 1),
    (8, 3, 5, 3, 1, 4, 1),
    (9, 2, 3, 3, 2, 2, 2),
    (6, 20, 18, 3, 1, 1, 1),
    (7, 2, 2, 5, 1, 3, 1),
])
def test_conv_parity(tiny, H, C, Co, K, BS, S, stride):
    rng = np.random.default_rng(H * 100 + C)
    x = rng.uniform(0, 1, (BS, C, H, H))
    w = rng.normal(0, 1 / K, (Co, C, K, K))
    run_conv_pair(tiny, x, w, S, stride)


@pytest.mark.parametrize("n1,dh", [(0, False), (2, False), (0, 2)])
def test_conv_parity_empty_sums(tiny, n1, dh):
    """Outputs with no nonzero term are the zero ciphertext on both sides: with
    H = 6, K = 5, S = 4 the fragments u', v' > H - K hold no valid output (12 of
    16 outputs), and all-zero weights empty every output; single hoisting with
    linear and baby-step / giant-step outer rotations, and fused double hoisting."""
    rng = np.random.default_rng(70 + n1)
    x = rng.uniform(0, 1, (1, 2, 6, 6))
    plan, outs = run_conv_pair(tiny, x, rng.normal(0, 1 / 5, (3, 2, 5, 5)), 4, bsgs_n1=n1, double_hoist=dh)
    res = u64(outs[1]).reshape(plan.info.n_out_ct, -1)
    assert int((~res.any(axis=1)).sum()) == 12
    plan, outs = run_conv_pair(tiny, x, np.zeros((3, 2, 5, 5)), 4, bsgs_n1=n1, double_hoist=dh,
                               check_counts=False)
    assert not u64(outs[1]).any() and not u64(outs[0]).any()
    assert tiny.g.device_status() == 0


@pytest.mark.parametrize("H,C,Co,K,S", [
    (6, 1, 1, 1, 1),   # one channel, 1x1 kernel: no rotation at all
    (5, 2, 3, 5, 1),   # kernel as large as the map: one valid output per channel
    (5, 3, 2, 5, 2),   # the same with S = 2: three of the four output fragments are empty
])
def test_conv_parity_degenerate_shapes(tiny, H, C, Co, K, S):
    rng = np.random.default_rng(H * 31 + C + K)
    x = rng.uniform(0, 1, (1, C, H, H))
    plan, _ = run_conv_pair(tiny, x, rng.normal(0, 1 / K, (Co, C, K, K)), S)
    if K == 1 and C == 1:
        assert plan.info.n_inner_rot == 0 and plan.info.n_outer_rot == 0 and not plan.steps
    assert tiny.g.device_status() == 0


def test_conv_parity_depthwise_and_two_prime_digits(ks2):
    rng = np.random.default_rng(9)
    x = rng.uniform(-1, 1, (1, 4, 6, 6))
    w = rng.normal(0, 1 / 3, (4, 1, 3, 3))
    run_conv_pair(ks2, x, w, 1, depthwise=True)
    w2 = rng.normal(0, 0.3, (5, 4, 1, 1))
    run_conv_pair(ks2, x, w2, 1)


def test_conv1_configuration_bit_exact():
    """The single-conv configuration at full size (N = 2^13): residues bit-exact
    to the oracle in both paths, decrypted error <= 1e-3 against Eq. 2."""
    p = W.PARAMS["conv1"]
    P = Pair(p["logN"], p["n_q"], p["k"], p["bits"], p["pbits"])
    x, w = W.conv1_workload(0)
    plan, _ = run_conv_pair(P, x, w, 4, delta=p["delta"])
    assert (plan.info.n_inner_rot, plan.info.n_outer_rot, plan.info.n_pt) == (48, 80, 2400)


def test_square_pool_fc_parity():
    pr_args = (10, 4, 1, 40, 50)
    P = Pair(*pr_args)
    pr, g = P.pr, P.g
    rng = np.random.default_rng(7)
    olay = fragment.Layout(pr.N, 4, 4, 2, 4, 2)
    x = rng.uniform(0, 1, (4, 2, 4, 4))
    Pp = olay.cpc * olay.m * olay.m
    steps = henn.fc_rotation_steps(Pp, olay.BS)
    keys = ckks.KeySet(pr, 3, rot_steps=steps, relin=True)
    slots = fragment.pack(olay, x)
    octs = [ckks.encrypt(pr, keys.sk, ckks.encode(pr, slots[i], pr.L, 2.0 ** 35), 1, i) for i in range(olay.n_ct)]
    osq = henn.he_square(pr, keys, octs)
    opool, opl = henn.he_avgpool2(pr, osq, olay)
    sk = g.sk_gen(3)
    evk = g.evk_gen(sk, 3, steps, relin=True)
    lay = g.layout(4, 4, 2, 4, 2)
    ct = g.encrypt(sk, torch.from_numpy(slots), pr.L, 2.0 ** 35, seed=1)
    sq = g.he_square(evk, ct, pr.L)
    assert np.array_equal(u64(sq), oracle_ct_array(osq))
    pooled, pl = g.he_avgpool(lay, sq, pr.L - 1)
    assert np.array_equal(u64(pooled), oracle_ct_array(opool))
    wfc = rng.normal(0, 0.3, (7, 8))
    m = opl.m

    def feat(c_ct, p):
        c_loc, k = divmod(p, m * m)
        c = c_ct * opl.cpc + c_loc
        bi, bj = divmod(k, m)
        if c >= opl.C or bi >= opl.H or bj >= opl.W:
            return -1
        return (c * opl.H + bi) * opl.W + bj

    ofc = henn.he_fc(pr, keys, opool, feat, Pp, opl.BS, wfc)
    ftab = np.array([[feat(c, p) for p in range(Pp)] for c in range(len(opool))], dtype=np.int32)
    plan = g.plan_fc(len(opool), Pp, opl.BS, ftab, 8, 7, pr.L - 1)
    pt = g.load_weights(plan, wfc, float(pr.q[pr.L - 1]))
    for mode in (0, 1):
        out = g.he_fc(evk, plan, pt, pooled, mode=mode)
        assert np.array_equal(u64(out), oracle_ct_array(ofc)), mode
    # outputs Pp .. Pp + 2 with all-zero weights: their ciphertext is the zero
    # ciphertext on both sides (an empty sum in the oracle)
    wz = np.zeros((Pp + 3, 8))
    wz[:7] = wfc
    ofz = henn.he_fc(pr, keys, opool, feat, Pp, opl.BS, wz)
    planz = g.plan_fc(len(opool), Pp, opl.BS, ftab, 8, Pp + 3, pr.L - 1)
    ptz = g.load_weights(planz, wz, float(pr.q[pr.L - 1]))
    for mode in (0, 1):
        out = u64(g.he_fc(evk, planz, ptz, pooled, mode=mode))
        assert np.array_equal(out, oracle_ct_array(ofz)), mode
        assert not out[1].any()


def test_aac_compress_parity(tiny):
    pr, g = tiny.pr, tiny.g
    rng = np.random.default_rng(6)
    olay = fragment.Layout(pr.N, 8, 8, 2, 1, 1)  # cpc = 8, 2 valid channels
    x = rng.uniform(-1, 1, (1, 2, 8, 8))
    steps = henn.aac_rotation_steps(olay, 2)
    keys = ckks.KeySet(pr, 4, rot_steps=steps)
    slots = fragment.pack(olay, x)
    octs = [ckks.encrypt(pr, keys.sk, ckks.encode(pr, slots[0], pr.L, 2.0 ** 25), 1, 0)]
    want = oracle_ct_array(henn.aac_compress(pr, keys, octs, olay, 2))
    sk = g.sk_gen(4)
    evk = g.evk_gen(sk, 4, steps)
    lay = g.layout(8, 8, 2, 1, 1)
    ct = g.encrypt(sk, torch.from_numpy(slots), pr.L, 2.0 ** 25, seed=1)
    got = g.compress(evk, lay, 2, ct, pr.L)
    assert np.array_equal(u64(got), want)
    dec = g.decrypt(sk, got, pr.L, 2.0 ** 25).cpu().numpy()[0].reshape(8, -1)
    for c in range(8):
        assert np.abs(dec[c] - slots[0].reshape(8, -1)[c % 2]).max() < 1e-4


@pytest.mark.parametrize("H,W_,C,BS,S", [(28, 28, 1, 2, 4), (7, 5, 3, 2, 2), (14, 14, 20, 1, 1), (9, 9, 5, 2, 3)])
def test_fragment_pack_unpack_parity(tiny, H, W_, C, BS, S):
    """Algorithm 1 slot map on the GPU equals the oracle's, element for element,
    including ragged maps (H, W not multiples of S; C not a multiple of cpc)."""
    rng = np.random.default_rng(H * 10 + C)
    x = rng.uniform(-1, 1, (BS, C, H, W_))
    lay = tiny.g.layout(H, W_, C, BS, S)
    olay = fragment.Layout(tiny.pr.N, H, W_, C, BS, S)
    assert (lay.m, lay.cpc, lay.n_ct) == (olay.m, olay.cpc, olay.n_ct)
    slots = tiny.g.pack(lay, torch.from_numpy(x))
    want = fragment.pack(olay, x)
    assert np.array_equal(slots.cpu().numpy(), np.asarray(want))
    back = tiny.g.unpack(lay, slots).cpu().numpy()
    assert np.array_equal(back, x)


@pytest.mark.parametrize("H,C,Co,K,BS,S,stride", [(8, 3, 5, 3, 2, 2, 1), (9, 2, 3, 3, 2, 2, 2), (16, 4, 4, 5, 1, 4, 1),
                                                   (6, 20, 18, 3, 1, 1, 1)])
def test_planner_inner_count_matches_rotation_model(tiny, H, C, Co, K, BS, S, stride):
    """The planner executes exactly the inner rotations the host model counts."""
    lay = tiny.g.layout(H, H, C, BS, S)
    plan = tiny.g.plan_conv(lay, Co, K, stride=stride, level=tiny.g.L)
    r = fe.rotation_model(tiny.pr.N, H, H, C, Co, K, S, BS, stride)
    assert plan.info.n_inner_rot == r["executed_inner"]


@pytest.mark.parametrize("H,C,Co,K,BS,S", [(8, 3, 5, 3, 2, 2), (6, 20, 18, 3, 1, 1)])
def test_layer_batch_each_request_equals_alone(tiny, H, C, Co, K, BS, S):
    """Three requests through one batched launch (keys grouped across them): each
    request's output residues equal running it alone, in both paths, and the
    plain per-op batch equals the batched one."""
    g, pr = tiny.g, tiny.pr
    rng = np.random.default_rng(H + C)
    w = rng.normal(0, 1 / K, (Co, C, K, K))
    lay = g.layout(H, H, C, BS, S)
    plan = g.plan_conv(lay, Co, K, level=pr.L)
    sk = g.sk_gen(5)
    evk = g.evk_gen(sk, 5, plan.steps)
    pt = g.load_weights(plan, w, float(pr.q[pr.L]))
    cts = []
    for r in range(3):
        x = rng.uniform(0, 1, (BS, C, H, H))
        cts.append(g.encrypt(sk, g.pack(lay, torch.from_numpy(x)), pr.L, 2.0 ** 25, seed=30 + r))
    alone = [u64(g.he_conv(evk, plan, pt, ct, mode=1)) for ct in cts]
    batch_in = torch.cat(cts, 0).contiguous()
    n_out = plan.info.n_out_ct
    for mode in (1, 0):
        out = u64(g.he_layer_batch(evk, plan, pt, batch_in, 3, mode=mode))
        for r in range(3):
            assert np.array_equal(out[r * n_out:(r + 1) * n_out], alone[r]), (mode, r)
    # the smallest workspace (one outer rotation at a time) gives the same result
    ws = g.workspace(g.workspace_bytes(plan, 3, minimum=True))
    out = u64(g.he_layer_batch(evk, plan, pt, batch_in, 3, ws=ws))
    assert np.array_equal(out, np.concatenate(alone))



@pytest.mark.parametrize("H,C,Co,K,BS,S,stride,n1", [
    (6, 20, 18, 3, 1, 1, 1, 4),
    (4, 12, 10, 1, 2, 1, 1, 2),
    (8, 6, 9, 3, 1, 2, 2, 4),
    (6, 8, 8, 1, 1, 1, 1, 3),
])
def test_conv_parity_bsgs(tiny, H, C, Co, K, BS, S, stride, n1):
    """Baby-step / giant-step outer rotations: residues bit-exact to the oracle's
    schedule in both paths, decrypted within 1e-3 of FP64."""
    rng = np.random.default_rng(H * 10 + C + n1)
    x = rng.uniform(0, 1, (BS, C, H, H))
    w = rng.normal(0, 1 / K, (Co, C, K, K))
    plan, _ = run_conv_pair(tiny, x, w, S, stride, bsgs_n1=n1)
    assert plan.info.bsgs_n1 == min(n1, plan.in_layout.cpc)



def test_mac_ways_do_not_change_residues(tiny):
    """The MAC tile (outputs sharing ciphertext loads) is a pure schedule choice."""
    g, pr = tiny.g, tiny.pr
    rng = np.random.default_rng(7)
    w = rng.normal(0, 0.3, (12, 12, 1, 1))
    lay = g.layout(4, 4, 12, 2, 1)
    plan = g.plan_conv(lay, 12, 1, level=pr.L, bsgs_n1=4)
    sk = g.sk_gen(8)
    evk = g.evk_gen(sk, 8, plan.steps)
    pt = g.load_weights(plan, w, float(pr.q[pr.L]))
    ct = g.encrypt(sk, g.pack(lay, torch.from_numpy(rng.uniform(0, 1, (2, 12, 4, 4)))), pr.L, 2.0 ** 25, seed=9)
    outs = []
    for ways in (1, 2, 4):
        g.plan_set_mac_ways(plan, ways)
        outs.append(u64(g.he_conv(evk, plan, pt, ct, mode=1)))
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])
    assert g.device_status() == 0



@pytest.mark.parametrize("H,C,Co,K,BS,S,stride,n1,dw", [
    (8, 3, 5, 3, 2, 2, 1, 0, False),
    (6, 4, 4, 3, 1, 1, 1, 0, True),
    (6, 20, 18, 3, 1, 1, 1, 4, False),
    (8, 6, 9, 3, 1, 2, 2, 4, False),
])
def test_conv_parity_double_hoisted(tiny, H, C, Co, K, BS, S, stride, n1, dw):
    """Double hoisting (rotations and MAC on Q P, one ModDown per partial sum):
    residues bit-exact to the oracle's schedule in both paths, within 1e-3 of FP64."""
    rng = np.random.default_rng(H * 7 + C + n1)
    x = rng.uniform(0, 1, (BS, C, H, H))
    w = rng.normal(0, 1 / K, ((C if dw else Co), 1 if dw else C, K, K))
    plan, _ = run_conv_pair(tiny, x, w, S, stride, depthwise=dw, bsgs_n1=n1, double_hoist=True)
    assert plan.info.double_hoist == 1
    assert tiny.g.device_status() == 0



@pytest.mark.parametrize("H,C,Co,K,BS,S,stride,n1,dw", [
    (6, 4, 4, 3, 1, 1, 1, 0, True),    # depthwise: no outer rotation, fused
    (8, 3, 3, 3, 2, 2, 1, 0, True),    # depthwise, S = 2, two images
    (6, 8, 8, 1, 1, 1, 1, 8, False),   # BSGS with n1 = cpc: no giant step, fused
    (6, 20, 18, 3, 1, 1, 1, 4, False), # giant steps: plain double hoisting
])
def test_conv_parity_fused_moddown_rescale(tiny, H, C, Co, K, BS, S, stride, n1, dw):
    """Hoisting 2 (double hoisting, ModDown and rescale as one division by
    q_l P when the layer has no outer rotation): residues bit-exact to the
    oracle's "double_fused" schedule in both paths, within 1e-3 of FP64."""
    rng = np.random.default_rng(H * 13 + C + n1)
    x = rng.uniform(0, 1, (BS, C, H, H))
    w = rng.normal(0, 1 / K, ((C if dw else Co), 1 if dw else C, K, K))
    plan, _ = run_conv_pair(tiny, x, w, S, stride, depthwise=dw, bsgs_n1=n1, double_hoist=2)
    assert plan.info.double_hoist == 2
    assert tiny.g.device_status() == 0


@pytest.mark.parametrize("n1", [0, 4])
def test_per_operation_path(tiny, n1):
    """Mode 2 composes the layer from single-ciphertext operations (every
    rotation a key switch of its own, one PMult per term, one rescale per
    output): residues equal to the oracle's single-hoisted schedule, and on a
    plan whose plaintexts are encoded on Q P (double hoisting) equal to the
    single-hoisted plan's."""
    rng = np.random.default_rng(11 + n1)
    x = rng.uniform(0, 1, (1, 20, 6, 6))
    w = rng.normal(0, 1 / 3, (18, 20, 3, 3))
    plan, outs = run_conv_pair(tiny, x, w, 1, bsgs_n1=n1, modes=(1, 2))
    g = tiny.g
    lay = g.layout(6, 6, 20, 1, 1)
    dplan = g.plan_conv(lay, 18, 3, level=tiny.pr.L, bsgs_n1=n1, double_hoist=True)
    sk = g.sk_gen(3)
    evk = g.evk_gen(sk, 3, dplan.steps)
    ct = g.encrypt(sk, g.pack(lay, torch.from_numpy(x)), tiny.pr.L, 2.0 ** 25, seed=17)
    pt = g.load_weights(dplan, w, float(tiny.pr.q[tiny.pr.L]))
    assert np.array_equal(u64(g.he_conv(evk, dplan, pt, ct, mode=2)), u64(outs[2]))
    assert g.device_status() == 0


@pytest.fixture(scope="module", params=[36, 40])
def narrow(request):
    """Every modulus in [2^26, 2^40) (narrow reductions).  With a 36-bit special
    prime every modulus is below 2^36: the MAC and base conversion split their
    products at bit 24 (Acc36); with a 40-bit one the MAC keeps three 32-bit
    words (Acc40)."""
    return Pair(10, 3, 1, 30, request.param)


@pytest.mark.parametrize("dh", [False, 2])
def test_split_sums_below_2_40_bit_exact(narrow, dh):
    """With every modulus below 2^40 the MAC and base conversion use split sums
    (Acc36 below 2^36, Acc40 up to 2^40) and the key inner product the narrow
    reduction; depthwise and pointwise (BSGS) layers give the oracle's residues
    in both paths, and MAC items of 1, 2 and 4 outputs agree."""
    rng = np.random.default_rng(40 + int(dh))
    x = rng.uniform(0, 1, (1, 12, 6, 6))
    run_conv_pair(narrow, x, rng.normal(0, 1 / 3, (12, 1, 3, 3)), 1, depthwise=True, double_hoist=dh)
    w = rng.normal(0, 0.3, (12, 12, 1, 1))
    plan, outs = run_conv_pair(narrow, x, w, 1, bsgs_n1=4, double_hoist=dh)
    g, pr = narrow.g, narrow.pr
    lay = g.layout(6, 6, 12, 1, 1)
    sk = g.sk_gen(3)
    evk = g.evk_gen(sk, 3, plan.steps)
    ct = g.encrypt(sk, g.pack(lay, torch.from_numpy(x)), pr.L, 2.0 ** 25, seed=17)
    pt = g.load_weights(plan, w, float(pr.q[pr.L]))
    for ways in (1, 2, 4):
        g.plan_set_mac_ways(plan, ways)
        assert np.array_equal(u64(g.he_conv(evk, plan, pt, ct, mode=1)), u64(outs[1])), f"ways {ways}"
    assert g.device_status() == 0


@pytest.mark.parametrize("pbits,hb", [(36, 1), (45, 2), (52, 4)])
def test_compact_plaintext_widths(pbits, hb):
    """Plan plaintexts are stored as a 32-bit low plane plus a 1-, 2- or 4-byte
    high plane, chosen by the widest modulus; every width gives the oracle's
    residues in both paths, with plaintexts on Q (single hoisting) and on Q P
    (double hoisting, where the special primes set the width)."""
    P = Pair(10, 3, 1, 30, pbits)
    rng = np.random.default_rng(pbits)
    x = rng.uniform(0, 1, (1, 6, 6, 6))
    w = rng.normal(0, 1 / 3, (5, 6, 3, 3))
    for dh in (False, True):
        plan, _ = run_conv_pair(P, x, w, 1, bsgs_n1=2, double_hoist=dh)
        nl = P.pr.L + 1 + (P.pr.k if dh else 0)
        assert plan.info.pt_bytes == plan.info.n_pt * nl * (4 + hb) * P.pr.N
    assert P.g.device_status() == 0


@pytest.mark.parametrize("logN", [14, 16])
def test_ntt_radix16_equals_radix8_and_oracle(logN):
    """The radix-16 and radix-4 round variants of the NTT give the same residues."""
    g = fe.Context(logN, 3, 1, 36, 36)
    pr = ckks.Params(logN, 3, 1, 36, 36)
    rng = np.random.default_rng(logN)
    a = np.stack([rng.integers(0, q, pr.N, dtype=np.uint64) for q in pr.moduli])
    outs = []
    for radix in (8, 16, 4):
        g.set_ntt_radix(radix)
        d = to_dev(a[None])
        g.ntt(d)
        fwd = u64(d)[0]
        g.ntt(d, inverse=True)
        outs.append((fwd, u64(d)[0]))
    g.set_ntt_radix(8)
    for o in outs[1:]:
        assert np.array_equal(outs[0][0], o[0]) and np.array_equal(o[1], a)
    for t in range(pr.n_mod if hasattr(pr, "n_mod") else len(pr.moduli)):
        assert np.array_equal(outs[1][0][t], pr.ntt(a[t], t))


@pytest.mark.parametrize("logN,radix", [(11, 8), (14, 16), (16, 8), (16, 16)])
def test_ntt_36bit_shoup_form_equals_general_form_and_oracle(logN, radix):
    """With every modulus below 2^36 the transforms take the Shoup product in
    32-bit pieces (fe_ctx_set_ntt_q36); it gives the residues of the general
    64-bit form and of the oracle, forward and inverse, including inputs at
    q - 1 everywhere (the largest values the forward transform's lazy stages
    build up)."""
    g = fe.Context(logN, 3, 2, 36, 36)
    pr = ckks.Params(logN, 3, 2, 36, 36)
    rng = np.random.default_rng(logN + radix)
    rnd = np.stack([rng.integers(0, q, pr.N, dtype=np.uint64) for q in pr.moduli])
    top = np.stack([np.full(pr.N, q - 1, dtype=np.uint64) for q in pr.moduli])
    g.set_ntt_radix(radix)
    for a in (rnd, top):
        res = []
        for q36 in (True, False):
            g.set_ntt_q36(q36)
            d = to_dev(a[None])
            g.ntt(d)
            fwd = u64(d)[0]
            g.ntt(d, inverse=True)
            res.append((fwd, u64(d)[0]))
        assert np.array_equal(res[0][0], res[1][0]) and np.array_equal(res[0][1], a) and np.array_equal(res[1][1], a)
        for t in range(len(pr.moduli)):
            assert np.array_equal(res[0][0][t], pr.ntt(a[t], t))
    g.set_ntt_q36(True)
    g.set_ntt_radix(8)


@pytest.mark.parametrize("logN", [11, 14, 16])
def test_ntt_data_paths_equal_the_oracle(logN):
    """Every NTT data path (fe_ctx_set_ntt_path): two passes whose first and
    last rounds touch global memory directly (0, default), two passes staged
    through shared memory (1), one pass on 8-CTA clusters exchanging the limb
    through distributed shared memory (2, N = 2^16), and the forward forms of
    fe_ctx_set_ntt_forward (per-stage reduction, 36-bit product); each gives the
    residues forward and returns the input inverse, on random residues and on
    q - 1 everywhere, in place and out of place (the key switch's ModUp
    transforms a converted copy)."""
    g = fe.Context(logN, 3, 2, 36, 36)
    pr = ckks.Params(logN, 3, 2, 36, 36)
    rng = np.random.default_rng(logN + 7)
    rnd = np.stack([rng.integers(0, q, pr.N, dtype=np.uint64) for q in pr.moduli])
    top = np.stack([np.full(pr.N, q - 1, dtype=np.uint64) for q in pr.moduli])
    for a in (rnd, top):
        want = np.stack([pr.ntt(a[t], t) for t in range(len(pr.moduli))])
        for path, fwd in ((0, 0), (1, 0), (2, 0), (0, 1), (0, 2), (0, 3), (1, 3)):
            g.set_ntt_path(path)
            g.set_ntt_forward(fwd)
            d = to_dev(a[None])
            g.ntt(d)
            assert np.array_equal(u64(d)[0], want), (path, fwd)
            g.ntt(d, inverse=True)
            assert np.array_equal(u64(d)[0], a), (path, fwd)
        g.set_ntt_forward(0)
    if logN == 16:
        # a key switch transforms converted copies out of place
        keys = ckks.KeySet(pr, 5, rot_steps=[3])
        sk = g.sk_gen(5)
        evk = g.evk_gen(sk, 5, [3])
        z = rng.uniform(-1, 1, pr.N // 2)
        oct_ = ckks.encrypt(pr, keys.sk, ckks.encode(pr, z, pr.L, 2.0 ** 25), 2, 0)
        ct = g.encrypt(sk, torch.from_numpy(z[None]), pr.L, 2.0 ** 25, seed=2)
        want = oracle_ct_array([ckks.rotate(pr, keys, oct_, 3)])
        for path in (0, 1, 2):
            g.set_ntt_path(path)
            assert np.array_equal(u64(g.rotate(evk, ct, pr.L, 3)), want), path
    g.set_ntt_path(0)
    assert g.device_status() == 0


@pytest.mark.parametrize("dh,S,BS", [(1, 1, 1), (2, 1, 1), (2, 2, 2)])
def test_depthwise_rotated_copies_formed_in_the_mac(tiny, dh, S, BS):
    """Depthwise layers under double hoisting: the batched MAC forms each rotated
    copy sigma((P c0, 0) + acc) from the key inner product's accumulators and
    the lifted input (fe_plan_set_lift_fusion(1), default) or reads the copies a
    lift pass wrote (0); both give the oracle's residues, as does the
    per-primitive path."""
    rng = np.random.default_rng(90 + dh + S)
    x = rng.uniform(0, 1, (BS, 4, 8, 8))
    w = rng.normal(0, 1 / 3, (4, 1, 3, 3))
    plan, outs = run_conv_pair(tiny, x, w, S, depthwise=True, double_hoist=dh)
    g = tiny.g
    steps = plan.steps
    sk = g.sk_gen(3)
    evk = g.evk_gen(sk, 3, steps)
    lay = g.layout(8, 8, 4, BS, S)
    ct = g.encrypt(sk, g.pack(lay, torch.from_numpy(x)), tiny.pr.L, 2.0 ** 25, seed=17)
    pt = g.load_weights(plan, w, float(tiny.pr.q[tiny.pr.L]))
    g.plan_set_lift_fusion(plan, 0)
    unfused = u64(g.he_conv(evk, plan, pt, ct, mode=1))
    g.plan_set_lift_fusion(plan, 1)
    fused = u64(g.he_conv(evk, plan, pt, ct, mode=1))
    assert np.array_equal(fused, unfused) and np.array_equal(fused, u64(outs[1]))
    assert g.device_status() == 0
