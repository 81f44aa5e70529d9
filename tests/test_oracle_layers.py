"""Pins of the oracle's encrypted layers: decrypted outputs against the FP64
plaintext definitions (Eq. 2 for convolution), and the executed rotation
counts against the model's formulas."""
import numpy as np
import pytest

import workloads as W
from oracle import ckks, counts, fragment, henn, plain


def encrypt_layout(pr, keys, lay, x, level, scale, seed=11):
    slots = fragment.pack(lay, x)
    return [ckks.encrypt(pr, keys.sk, ckks.encode(pr, slots[i], level, scale), seed, i)
            for i in range(lay.n_ct)]


def decrypt_layout(pr, keys, lay, cts):
    return fragment.unpack(lay, np.stack([ckks.decrypt(pr, keys.sk, c) for c in cts]))


@pytest.fixture(scope="module")
def tiny():
    p = W.PARAMS["tiny"]
    return ckks.Params(p["logN"], p["n_q"], p["k"], p["bits"], p["pbits"]), p["delta"]


@pytest.mark.parametrize("H,C,Co,K,BS,S,stride", [
    (8, 3, 5, 3, 2, 2, 1),     # K > S, several channels
    (8, 3, 5, 3, 1, 4, 1),     # K <= S: edge rotations only
    (9, 2, 3, 3, 2, 2, 2),     # stride 2 by discarding fragments
    (6, 20, 18, 3, 1, 1, 1),   # several input and output groups (cpc = 8)
    (7, 2, 2, 5, 1, 3, 1),     # S not a power of two
])
def test_he_conv_matches_fp64(tiny, H, C, Co, K, BS, S, stride):
    pr, delta = tiny
    rng = np.random.default_rng(H * 100 + C)
    x = rng.uniform(0, 1, (BS, C, H, H))
    w = rng.normal(0, 1 / K, (Co, C, K, K))
    lay = fragment.Layout(pr.N, H, H, C, BS, S)
    keys = ckks.KeySet(pr, 3, rot_steps=henn.conv_rotation_steps(lay, C, Co, K, stride))
    cts = encrypt_layout(pr, keys, lay, x, pr.L, delta)
    cnt = henn.Counters()
    out, olay = henn.he_conv(pr, keys, cts, lay, w, stride=stride, cnt=cnt)
    y = decrypt_layout(pr, keys, olay, out)
    ref = plain.conv2d(x, w, stride=stride)
    assert np.abs(y - ref).max() < 1e-3
    assert cnt.pmult > 0 and cnt.rescale == olay.n_ct
    # executed inner rotations follow the offset model
    inner = counts.executed_inner(S, K, lay.groups, stride)
    outer = cnt.rot - inner
    assert outer >= 0
    # the invalid region of every output ciphertext decrypts to (noise around) zero
    full = np.stack([ckks.decrypt(pr, keys.sk, c) for c in out])
    mask = np.zeros_like(full, dtype=bool)
    cts_idx, slots = fragment.slot_map(olay)
    mask[cts_idx, slots] = True
    assert np.abs(full[~mask]).max() < 1e-3


@pytest.mark.parametrize("n1,hoist", [(0, "single"), (2, "single"), (0, "double_fused")])
def test_he_conv_empty_sums_are_zero_ciphertexts(tiny, n1, hoist):
    """Outputs none of whose terms has a nonzero plaintext: with H = 6, K = 5,
    S = 4 the valid outputs (h, w <= H - K = 1) lie only in fragments u', v' <= 1,
    so 12 of the 16 output ciphertexts are empty sums; with all-zero weights every
    output is.  An empty sum is the zero ciphertext (every residue 0) at the
    output level and scale, and the decrypted layer equals the FP64 convolution."""
    pr, delta = tiny
    rng = np.random.default_rng(66 + n1)
    H, C, Co, K, S = 6, 2, 3, 5, 4
    x = rng.uniform(0, 1, (1, C, H, H))
    for w in (rng.normal(0, 1 / K, (Co, C, K, K)), np.zeros((Co, C, K, K))):
        lay = fragment.Layout(pr.N, H, H, C, 1, S)
        keys = ckks.KeySet(pr, 3, rot_steps=henn.conv_rotation_steps(lay, C, Co, K, bsgs_n1=n1))
        cts = encrypt_layout(pr, keys, lay, x, pr.L, delta)
        cnt = henn.Counters()
        out, olay = henn.he_conv(pr, keys, cts, lay, w, cnt=cnt, bsgs_n1=n1, hoist=hoist)
        assert np.abs(decrypt_layout(pr, keys, olay, out) - plain.conv2d(x, w)).max() < 1e-3
        nonzero_w = bool(w.any())
        for h in range(olay.groups):
            for up in range(S):
                for vp in range(S):
                    c = out[olay.ct_index(h, up, vp)]
                    assert c.level == pr.L - 1 and c.scale == delta
                    empty = not nonzero_w or up > H - K or vp > H - K
                    assert (not c.as_array().any()) == empty
        assert cnt.rescale == (4 * olay.groups if nonzero_w else 0)
        if not nonzero_w:
            assert cnt.pmult == 0


def test_he_conv_depthwise(tiny):
    pr, delta = tiny
    rng = np.random.default_rng(5)
    x = rng.uniform(-1, 1, (1, 4, 8, 8))
    w = rng.normal(0, 1 / 3, (4, 1, 3, 3))
    lay = fragment.Layout(pr.N, 8, 8, 4, 1, 1)
    keys = ckks.KeySet(pr, 3, rot_steps=henn.conv_rotation_steps(lay, 4, 4, 3, depthwise=True))
    cts = encrypt_layout(pr, keys, lay, x, pr.L, delta)
    cnt = henn.Counters()
    out, olay = henn.he_conv(pr, keys, cts, lay, w, depthwise=True, cnt=cnt)
    assert cnt.rot == 8 * lay.groups  # inner only, no outer rotations for depthwise
    assert np.abs(decrypt_layout(pr, keys, olay, out) - plain.conv2d(x, w, depthwise=True)).max() < 1e-3


def test_aac_bottleneck(tiny):
    """8 -> 2 -> 8 bottleneck of 1x1 convs (Fig. 6): AAC replicates the 2 valid
    channels so the expansion uses 2 diagonals (1 rotation) instead of 8 (7)."""
    pr, delta = tiny
    rng = np.random.default_rng(6)
    lay = fragment.Layout(pr.N, 8, 8, 8, 1, 1)
    assert lay.cpc == 8 and lay.n_ct == 1
    x = rng.uniform(-1, 1, (1, 8, 8, 8))
    w1 = rng.normal(0, 0.3, (2, 8, 1, 1))
    w2 = rng.normal(0, 0.5, (8, 2, 1, 1))
    l1 = henn.out_layout_conv(lay, 2, 1, 1)
    steps = set(henn.conv_rotation_steps(lay, 8, 2, 1)) | set(henn.aac_rotation_steps(l1, 2))
    steps |= set(henn.conv_rotation_steps(l1, 2, 8, 1, in_period=2))
    steps |= set(henn.conv_rotation_steps(l1, 2, 8, 1))
    keys = ckks.KeySet(pr, 3, rot_steps=steps)
    cts = encrypt_layout(pr, keys, lay, x, pr.L, delta)
    h, l1 = henn.he_conv(pr, keys, cts, lay, w1)
    ref = plain.conv2d(plain.conv2d(x, w1), w2)
    c_with, c_without = henn.Counters(), henn.Counters()
    comp = henn.aac_compress(pr, keys, h, l1, 2, cnt=c_with)
    assert c_with.rot == 2  # log2(cpc / c_valid) doublings
    y_with, l2 = henn.he_conv(pr, keys, comp, l1, w2, in_period=2, cnt=c_with)
    y_wo, l2b = henn.he_conv(pr, keys, h, l1, w2, cnt=c_without)
    assert c_with.rot == 2 + 1 and c_without.rot == 7
    assert np.abs(decrypt_layout(pr, keys, l2, y_with) - ref).max() < 1e-3
    assert np.abs(decrypt_layout(pr, keys, l2b, y_wo) - ref).max() < 1e-3
    # the replicated ciphertext holds channel c_loc mod 2 at every position
    rep = np.stack([ckks.decrypt(pr, keys.sk, c) for c in comp])[0].reshape(8, -1)
    hv = np.stack([ckks.decrypt(pr, keys.sk, c) for c in h])[0].reshape(8, -1)
    for c_loc in range(8):
        assert np.abs(rep[c_loc] - hv[c_loc % 2]).max() < 1e-4


def test_square_pool_fc(tiny):
    pr0, delta = tiny
    pr = ckks.Params(10, 4, 1, 40, 50)
    rng = np.random.default_rng(7)
    lay = fragment.Layout(pr.N, 4, 4, 2, 4, 2)
    x = rng.uniform(0, 1, (4, 2, 4, 4))
    P = lay.cpc * lay.m * lay.m
    keys = ckks.KeySet(pr, 3, rot_steps=henn.fc_rotation_steps(P, lay.BS), relin=True)
    cts = encrypt_layout(pr, keys, lay, x, pr.L, 2.0 ** 35)
    sq = henn.he_square(pr, keys, cts)
    pooled, pl = henn.he_avgpool2(pr, sq, lay)
    ref = 4 * plain.avgpool2(plain.poly_act(x))
    assert np.abs(decrypt_layout(pr, keys, pl, pooled) - ref).max() < 1e-3
    # FC on the pooled map (S = 1): features (c, h, w) flattened
    wfc = rng.normal(0, 0.3, (7, 2 * 2 * 2))
    m = pl.m

    def feat(c_ct, p):
        c_loc, k = divmod(p, m * m)
        c = c_ct * pl.cpc + c_loc
        bi, bj = divmod(k, m)
        if c >= pl.C or bi >= pl.H or bj >= pl.W:
            return -1
        return (c * pl.H + bi) * pl.W + bj

    out = henn.he_fc(pr, keys, pooled, feat, P, pl.BS, wfc)
    dec = [ckks.decrypt(pr, keys.sk, c) for c in out]
    y = henn.lenet_decode_logits(dec, P, pl.BS, 7)
    ref_fc = plain.fc(ref.reshape(4, -1), wfc)
    assert np.abs(y - ref_fc).max() < 1e-3
    # outputs P .. P + 2 have all-zero weights, so their ciphertext is an empty
    # sum: the zero ciphertext at the output level and scale; the first one is
    # unchanged (its extra rows are zero too)
    wz = np.zeros((P + 3, wfc.shape[1]))
    wz[:7] = wfc
    out2 = henn.he_fc(pr, keys, pooled, feat, P, pl.BS, wz)
    assert len(out2) == 2 and np.array_equal(out2[0].as_array(), out[0].as_array())
    assert not out2[1].as_array().any()
    assert (out2[1].level, out2[1].scale) == (out[0].level, out[0].scale)


@pytest.mark.slow
def test_conv1_config_end_to_end():
    """The single-conv configuration at full size: 48 inner + 80 outer rotations,
    2,400 PMults, decrypted error <= 1e-3 against Eq. 2 in FP64."""
    p = W.PARAMS["conv1"]
    pr = ckks.Params(p["logN"], p["n_q"], p["k"], p["bits"], p["pbits"])
    x, w = W.conv1_workload(0)
    lay = fragment.Layout(pr.N, 28, 28, 1, 1, 4)
    keys = ckks.KeySet(pr, 7, rot_steps=henn.conv_rotation_steps(lay, 1, 6, 5))
    cts = encrypt_layout(pr, keys, lay, x, pr.L, p["delta"])
    cnt = henn.Counters()
    out, olay = henn.he_conv(pr, keys, cts, lay, w, cnt=cnt)
    assert (cnt.rot, cnt.pmult, cnt.rescale) == (48 + 80, 2400, 16)
    y = decrypt_layout(pr, keys, olay, out)
    assert np.abs(y - plain.conv2d(x, w)).max() < 1e-3
    assert out[0].scale == p["delta"] and out[0].level == pr.L - 1


@pytest.mark.parametrize("H,C,Co,K,BS,S,stride,n1", [
    (6, 20, 18, 3, 1, 1, 1, 4),    # cpc = 8: 2 giant steps of 4 diagonals
    (4, 12, 10, 1, 2, 1, 1, 2),    # pointwise, cpc = 16, n1 = 2
    (8, 6, 9, 3, 1, 2, 2, 4),      # stride 2, cpc = 32
    (6, 8, 8, 1, 1, 1, 1, 3),      # n1 not dividing cpc (last giant step partial)
])
def test_he_conv_bsgs_matches_fp64_and_linear(tiny, H, C, Co, K, BS, S, stride, n1):
    """Baby-step / giant-step outer rotations: the same convolution (decrypted
    within 1e-3 of FP64 and of the linear schedule), fewer key switches when
    there are many diagonals, and the rotation-step list covers every rotation."""
    pr, delta = tiny
    rng = np.random.default_rng(H * 10 + C + n1)
    x = rng.uniform(0, 1, (BS, C, H, H))
    w = rng.normal(0, 1 / K, (Co, C, K, K))
    lay = fragment.Layout(pr.N, H, H, C, BS, S)
    steps = henn.conv_rotation_steps(lay, C, Co, K, stride, bsgs_n1=n1)
    keys = ckks.KeySet(pr, 3, rot_steps=steps)
    cts = encrypt_layout(pr, keys, lay, x, pr.L, delta)
    cnt = henn.Counters()
    out, olay = henn.he_conv(pr, keys, cts, lay, w, stride=stride, cnt=cnt, bsgs_n1=n1)
    y = decrypt_layout(pr, keys, olay, out)
    assert np.abs(y - plain.conv2d(x, w, stride=stride)).max() < 1e-3
    # key switches: (|offsets x babies| - 1) per input ciphertext + (giant steps - 1) per output
    n1e = min(n1, lay.cpc)
    offs = counts.inner_offsets(S, K, stride)
    G_out = -(-Co // lay.cpc)
    diag = {h: henn.conv_diagonals(lay, C, Co, h, False, None) for h in range(G_out)}
    babies = {0} | {d % n1e for h in diag for d in diag[h]}
    inner = sum(len(offs[u]) * len(offs[v]) * len(babies) - 1 for u in range(S) for v in range(S)) * lay.groups
    giants = sum((len({d // n1e for d in diag[h]}) - 1) * (S // stride) ** 2 for h in range(G_out))
    assert cnt.rot == inner + giants
    assert cnt.modup == lay.groups * S * S + giants
    assert set(steps) >= {((a * lay.m + b) * lay.BS + i * lay.blk) for a in [0] for b in [0] for i in babies if i}



@pytest.mark.parametrize("H,C,Co,K,BS,S,stride,n1,dw", [
    (8, 3, 5, 3, 2, 2, 1, 0, False),   # linear, K > S
    (6, 4, 4, 3, 1, 1, 1, 0, True),    # depthwise, inner rotations only
    (6, 20, 18, 3, 1, 1, 1, 4, False), # BSGS: baby steps double hoisted
    (8, 6, 9, 3, 1, 2, 2, 4, False),   # BSGS with stride 2
])
def test_he_conv_double_hoisted_matches_fp64(tiny, H, C, Co, K, BS, S, stride, n1, dw):
    """Double hoisting: the same convolution (within 1e-3 of FP64), the same
    rotations and key switches, one ModDown per partial sum."""
    pr, delta = tiny
    rng = np.random.default_rng(H * 7 + C + n1)
    x = rng.uniform(0, 1, (BS, C, H, H))
    w = rng.normal(0, 1 / K, ((C if dw else Co), 1 if dw else C, K, K))
    lay = fragment.Layout(pr.N, H, H, C, BS, S)
    Cout = C if dw else Co
    steps = henn.conv_rotation_steps(lay, C, Cout, K, stride, depthwise=dw, bsgs_n1=n1)
    keys = ckks.KeySet(pr, 3, rot_steps=steps)
    cts = encrypt_layout(pr, keys, lay, x, pr.L, delta)
    c1, c2 = henn.Counters(), henn.Counters()
    out, olay = henn.he_conv(pr, keys, cts, lay, w, stride=stride, depthwise=dw, cnt=c1, bsgs_n1=n1,
                             hoist="double")
    y = decrypt_layout(pr, keys, olay, out)
    assert np.abs(y - plain.conv2d(x, w, stride=stride, depthwise=dw)).max() < 1e-3
    out2, _ = henn.he_conv(pr, keys, cts, lay, w, stride=stride, depthwise=dw, cnt=c2, bsgs_n1=n1)
    assert (c1.rot, c1.keyswitch, c1.pmult, c1.modup) == (c2.rot, c2.keyswitch, c2.pmult, c2.modup)
    assert 0 < c1.moddown <= c1.pmult


@pytest.mark.parametrize("H,C,Co,K,BS,S,stride,n1,dw", [
    (6, 4, 4, 3, 1, 1, 1, 0, True),    # depthwise: no outer rotation, fused
    (8, 3, 3, 3, 2, 2, 1, 0, True),    # depthwise, S = 2, batch 2
    (6, 8, 8, 1, 1, 1, 1, 8, False),   # BSGS with n1 = cpc: no giant step, fused
    (6, 20, 18, 3, 1, 1, 1, 4, False), # BSGS with giant steps: the double-hoisted path
])
def test_he_conv_fused_moddown_rescale_matches_fp64(tiny, H, C, Co, K, BS, S, stride, n1, dw):
    """hoist="double_fused": when the layer has no outer rotation each output is
    its partial sum divided by q_level P in one step; the convolution stays within
    1e-3 of FP64 with one rescale fewer than double hoisting's ModDown + rescale
    per output, and with outer rotations it is double hoisting exactly."""
    pr, delta = tiny
    rng = np.random.default_rng(H * 11 + C + n1)
    x = rng.uniform(0, 1, (BS, C, H, H))
    w = rng.normal(0, 1 / K, ((C if dw else Co), 1 if dw else C, K, K))
    lay = fragment.Layout(pr.N, H, H, C, BS, S)
    Cout = C if dw else Co
    steps = henn.conv_rotation_steps(lay, C, Cout, K, stride, depthwise=dw, bsgs_n1=n1)
    keys = ckks.KeySet(pr, 3, rot_steps=steps)
    cts = encrypt_layout(pr, keys, lay, x, pr.L, delta)
    c1, c2 = henn.Counters(), henn.Counters()
    out, olay = henn.he_conv(pr, keys, cts, lay, w, stride=stride, depthwise=dw, cnt=c1, bsgs_n1=n1,
                             hoist="double_fused")
    ref, _ = henn.he_conv(pr, keys, cts, lay, w, stride=stride, depthwise=dw, cnt=c2, bsgs_n1=n1,
                          hoist="double")
    y = decrypt_layout(pr, keys, olay, out)
    assert np.abs(y - plain.conv2d(x, w, stride=stride, depthwise=dw)).max() < 1e-3
    assert all(o.level == r.level for o, r in zip(out, ref))
    fused = c1.rot == c2.rot and c1.keyswitch == c2.keyswitch and c1.rescale == c2.rescale
    assert fused
    no_outer = dw or n1 >= lay.cpc
    if not no_outer:  # with outer rotations nothing changes
        assert all(np.array_equal(o.as_array(), r.as_array()) for o, r in zip(out, ref))
    else:  # one division instead of two roundings: residues differ, decryptions agree
        assert any(not np.array_equal(o.as_array(), r.as_array()) for o, r in zip(out, ref))
