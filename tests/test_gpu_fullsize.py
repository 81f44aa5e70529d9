"""Bit-exact parity at the full parameter sets, on sampled outputs the oracle
can compute in about a minute.

* The benchmark's parameter set (N = 2^16, 24 x 36-bit + 4 special primes,
  dnum = 6) at the pointwise layers' level 22: a 14x14 pointwise layer with 16
  channels in and out at S = 1 (one ciphertext each side, 31 nonzero channel
  diagonals), run with the schedule the tuner picks for the benchmark's
  pointwise layers -- baby-step / giant-step outer rotations (n1 = 4), double
  hoisting on Q_l P, and MAC items of four outputs sharing their ciphertext
  tiles, i.e. the four-output, one-byte-high-plane MAC with the bit-24 split
  sums (every modulus below 2^36) at the N = 2^16 tile geometry.  The output
  ciphertext equals the oracle's (Sec. 3.1 with BSGS; Eq. 4), in both the
  batched path and a captured graph replayed from host buffers.
* The LeNet parameter set (N = 2^14, 8 x 40-bit + 2 special primes, BS = 128,
  S = 4): ciphertext 0 of conv1 (output channel 0, fragment (0, 0), which reads
  all 16 input fragments through the inner rotations of Eq. 3) equals the
  oracle's."""
import numpy as np
import pytest

import workloads as W
from oracle import ckks, fragment, henn

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2606_16359_b300 as fe  # noqa: E402


def u64(t):
    return t.detach().cpu().numpy().view(np.uint64)


def test_pointwise_bsgs_double_hoisted_four_output_mac_at_the_benchmark_parameters():
    p = W.PARAMS["mobilenet"]
    H, C, level, seed = 14, 16, 22, 31
    rng = np.random.default_rng(7)
    x = rng.uniform(-1, 1, (1, C, H, H))
    w = rng.normal(0, 1 / np.sqrt(C), (C, C, 1, 1))
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        ctx = fe.Context(p["logN"], p["n_q"], p["k"], p["bits"], p["pbits"])
        lay = ctx.layout(H, H, C, 1, 1)
        plan = ctx.plan_conv(lay, C, 1, level=level, bsgs_n1=4, double_hoist=True)
        ctx.plan_set_mac_ways(plan, 4)
        info = plan.info
        assert info.bsgs_n1 == 4 and info.double_hoist == 1 and info.n_in_ct == 1 and info.n_out_ct == 1
        sk = ctx.sk_gen(seed)
        evk = ctx.evk_gen(sk, seed, plan.steps)
        w_scale = float(ctx.moduli[level])
        pt = ctx.load_weights(plan, w, w_scale)
        ct = ctx.encrypt(sk, ctx.pack(lay, torch.from_numpy(x)), level, p["delta"], 5, ct_id0=0)
        got = u64(ctx.he_conv(evk, plan, pt, ct, mode=1))
        # the same layer as a captured graph, replayed through host buffers
        ws = ctx.workspace(ctx.graph_workspace_bytes([plan]))
        out = ctx.empty_ct(1, level - 1)
        g = ctx.graph_capture(evk, [plan], [pt], [ct], [out], ws)
        ib, ob = g.io()
        assert ib == [ct.numel() * 8] and ob == [out.numel() * 8]
        h_in = ct.cpu().pin_memory()
        h_out = torch.zeros(out.shape, dtype=out.dtype, pin_memory=True)
        g.launch_host([h_in], [h_out])
        torch.cuda.synchronize()
        assert ctx.device_status() == 0
    assert np.array_equal(h_out.numpy().view(np.uint64), got)
    pr = ckks.Params(p["logN"], p["n_q"], p["k"], p["bits"], p["pbits"])
    olay = fragment.Layout(pr.N, H, H, C, 1, 1)
    steps = henn.conv_rotation_steps(olay, C, C, 1, bsgs_n1=4)
    assert sorted(steps) == sorted(plan.steps)
    keys = ckks.KeySet(pr, seed, rot_steps=steps)
    slots = fragment.pack(olay, x)
    oct0 = ckks.encrypt(pr, keys.sk, ckks.encode(pr, slots[0], level, p["delta"]), 5, 0)
    oout, _ = henn.he_conv(pr, keys, [oct0], olay, w, w_scale=w_scale, bsgs_n1=4, hoist="double")
    assert len(oout) == 1
    assert np.array_equal(got[0], oout[0].as_array())


def test_lenet_conv1_ciphertext0_at_the_full_lenet_parameters():
    p = W.PARAMS["lenet"]
    wts = W.lenet_weights(0)
    seed = 17
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        ctx = fe.Context(p["logN"], p["n_q"], p["k"], p["bits"], p["pbits"])
        BS = ctx.N // 2 // 64
        assert BS == 128
        x = W.lenet_input(0, BS)
        lay = ctx.layout(28, 28, 1, BS, 4)
        plan = ctx.plan_conv(lay, 6, 5, level=ctx.L)
        sk = ctx.sk_gen(seed)
        evk = ctx.evk_gen(sk, seed, plan.steps)
        w_scale = float(ctx.moduli[ctx.L])
        pt = ctx.load_weights(plan, wts["conv1"], w_scale)
        ct = ctx.encrypt(sk, ctx.pack(lay, torch.from_numpy(x)), ctx.L, p["delta"], 3, ct_id0=0)
        got = u64(ctx.he_conv(evk, plan, pt, ct, mode=1)[0:1])
        assert ctx.device_status() == 0
    pr = ckks.Params(p["logN"], p["n_q"], p["k"], p["bits"], p["pbits"])
    olay = fragment.Layout(pr.N, 28, 28, 1, BS, 4)
    keys = ckks.KeySet(pr, seed, rot_steps=henn.conv_rotation_steps(olay, 1, 6, 5))
    slots = fragment.pack(olay, x)
    octs = [ckks.encrypt(pr, keys.sk, ckks.encode(pr, slots[i], pr.L, p["delta"]), 3, i) for i in range(olay.n_ct)]
    # output channel 0 only: ciphertext 0 of the layer is (channel 0, fragment (0, 0))
    oout, _ = henn.he_conv(pr, keys, octs, olay, wts["conv1"][:1], w_scale=w_scale)
    assert np.array_equal(got[0], oout[0].as_array())
