"""GPU parity of the fragment-size change between layers (Sec. 5,
Implementation paragraph: rot-mask-add re-encoding when a later layer's block
size differs), through the C ABI: residues equal the oracle's he_repack, and
after decryption the target layout unpacks to the input tensor.  Then a
MobileNet-shaped block at a reduced ring that runs its depthwise 3x3 layer at
S = 2 and its pointwise layer at S = 1 with the re-encoding between them,
bit-exact to the oracle's chain and within 1e-3 of the FP64 block."""
import numpy as np
import pytest

import workloads as W
from oracle import ckks, fragment, henn, plain

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2606_16359_b300 as fe  # noqa: E402


def u64(t):
    return t.detach().cpu().numpy().view(np.uint64)


@pytest.mark.parametrize("case", [
    dict(H=8, C=2, BS=1, Sa=1, Sb=2),
    dict(H=8, C=3, BS=1, Sa=2, Sb=1),
    dict(H=6, C=2, BS=2, Sa=2, Sb=1),
    dict(H=8, C=1, BS=2, Sa=4, Sb=2),
])
def test_repack_bit_exact_to_the_oracle(case):
    p = W.PARAMS["tiny"]
    args = (p["logN"], p["n_q"], p["k"], p["bits"], p["pbits"])
    delta = p["delta"]
    pr = ckks.Params(*args)
    la = fragment.Layout(pr.N, case["H"], case["H"], case["C"], case["BS"], case["Sa"])
    lb = fragment.Layout(pr.N, case["H"], case["H"], case["C"], case["BS"], case["Sb"])
    steps = henn.repack_rotation_steps(la, lb)
    x = np.random.default_rng(case["H"] + case["C"]).uniform(-1, 1, (la.BS, la.C, la.H, la.W))
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        g = fe.Context(*args)
        ga = g.layout(case["H"], case["H"], case["C"], case["BS"], case["Sa"])
        gb = g.layout(case["H"], case["H"], case["C"], case["BS"], case["Sb"])
        plan = g.plan_repack(ga, gb, g.L)
        assert sorted(plan.steps) == sorted(steps)
        sk = g.sk_gen(5)
        evk = g.evk_gen(sk, 5, plan.steps)
        pt = g.load_repack_masks(plan)
        ct = g.encrypt(sk, g.pack(ga, torch.from_numpy(x)), g.L, delta, 7, ct_id0=0)
        out = g.he_repack(evk, plan, pt, ct)
        got = u64(out)
        y = g.unpack(gb, g.decrypt(sk, out, g.L - 1, delta)).cpu().numpy()
        assert plan.info.n_out_ct == lb.n_ct and plan.info.n_in_ct == la.n_ct
    keys = ckks.KeySet(pr, 5, rot_steps=steps)
    slots = fragment.pack(la, x)
    cts = [ckks.encrypt(pr, keys.sk, ckks.encode(pr, slots[i], pr.L, delta), 7, i) for i in range(la.n_ct)]
    oout = henn.he_repack(pr, keys, cts, la, lb)
    assert np.array_equal(got, np.stack([o.as_array() for o in oout]))
    assert np.abs(y - x).max() < 1e-3


def test_block_with_depthwise_at_s2_and_pointwise_at_s1():
    """dw 3x3 on 16x16x8 at S = 2 (4 fragment ciphertexts, 3 inner rotations
    each), re-encoded to S = 1 (one ciphertext of 8 channel blocks of 16x16),
    pw 1x1 8 -> 8 at S = 1; N = 2^12 with 36-bit primes."""
    p = W.PARAMS["mobilenet_small"]
    args = (p["logN"], p["n_q"], p["k"], p["bits"], p["pbits"])
    delta = p["delta"]
    H, C = 16, 8
    rng = np.random.default_rng(21)
    x = rng.uniform(-1, 1, (1, C, H, H))
    wd = rng.normal(0, 1 / 3, (C, 1, 3, 3))
    wp = rng.normal(0, 1 / np.sqrt(C), (C, C, 1, 1))
    pr = ckks.Params(*args)
    la = fragment.Layout(pr.N, H, H, C, 1, 2)
    l_dw = henn.out_layout_conv(la, C, 3, 1)
    lb = fragment.Layout(pr.N, l_dw.H, l_dw.W, C, 1, 1)
    steps = sorted(set(henn.conv_rotation_steps(la, C, C, 3, depthwise=True)) |
                   set(henn.repack_rotation_steps(l_dw, lb)) | set(henn.conv_rotation_steps(lb, C, C, 1)))
    s = torch.cuda.Stream()
    times = {}
    with torch.cuda.stream(s):
        g = fe.Context(*args)
        L = g.L
        ga = g.layout(H, H, C, 1, 2)
        pdw = g.plan_conv(ga, C, 3, depthwise=True, level=L)
        gb = g.layout(pdw.out_layout.H, pdw.out_layout.W, C, 1, 1)
        prp = g.plan_repack(pdw.out_layout, gb, L - 1)
        ppw = g.plan_conv(gb, C, 1, level=L - 2)
        sk = g.sk_gen(9)
        evk = g.evk_gen(sk, 9, steps)
        pt_dw = g.load_weights(pdw, wd, float(g.moduli[L]))
        pt_rp = g.load_repack_masks(prp)
        pt_pw = g.load_weights(ppw, wp, float(g.moduli[L - 2]))
        ct = g.encrypt(sk, g.pack(ga, torch.from_numpy(x)), L, delta, 4, ct_id0=0)
        h_dw = g.he_conv(evk, pdw, pt_dw, ct)
        assert h_dw.shape[0] == prp.info.n_in_ct
        h_rp = g.he_repack(evk, prp, pt_rp, h_dw)
        assert h_rp.shape[0] == ppw.info.n_in_ct
        out = g.he_conv(evk, ppw, pt_pw, h_rp)
        got = u64(out)
        y = g.unpack(ppw.out_layout, g.decrypt(sk, out, L - 3, delta)).cpu().numpy()
        # share of the re-encoding in the block (CUDA events, warm); each layer reads
        # the output of the one before it, of the size its plan expects
        for name, fn in (("dw", lambda: g.he_conv(evk, pdw, pt_dw, ct)),
                         ("repack", lambda: g.he_repack(evk, prp, pt_rp, h_dw)),
                         ("pw", lambda: g.he_conv(evk, ppw, pt_pw, h_rp))):
            fn()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            times[name] = e0.elapsed_time(e1)
        assert g.device_status() == 0
    print("block ms", {k: round(v, 3) for k, v in times.items()},
          "repack share %.1f %%" % (100 * times["repack"] / sum(times.values())),
          "repack rotations", prp.info.n_inner_rot + prp.info.n_outer_rot, "masks", prp.info.n_pt)
    keys = ckks.KeySet(pr, 9, rot_steps=steps)
    slots = fragment.pack(la, x)
    cts = [ckks.encrypt(pr, keys.sk, ckks.encode(pr, slots[i], pr.L, delta), 4, i) for i in range(la.n_ct)]
    oh, ol = henn.he_conv(pr, keys, cts, la, wd, depthwise=True)
    oh = henn.he_repack(pr, keys, oh, ol, lb)
    oout, _ = henn.he_conv(pr, keys, oh, lb, wp)
    assert np.array_equal(got, np.stack([o.as_array() for o in oout]))
    ref = plain.conv2d(plain.conv2d(x, wd, depthwise=True), wp)
    assert np.abs(y - ref).max() < 1e-3
