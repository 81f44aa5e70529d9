"""Network-level parity: the LeNet-shaped network (conv, x^2, pool, conv, x^2,
pool, FC x3) on the GPU against the oracle at a reduced ring (bit-exact output
residues), and at the full LeNet parameter set (N = 2^14, 8 x 40-bit primes,
BS = 128) against the FP64 network (decrypted logits within 1e-3).  Also the
MobileNet-shaped blocks at N = 2^16 against FP64, and one sampled output
ciphertext of the smallest block's depthwise layer against the oracle, both in
the default schedule and in the benchmark's own launch configuration."""
import numpy as np
import pytest

import workloads as W
from oracle import ckks, fragment, henn, plain

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2606_16359_b300 as fe  # noqa: E402
from paper_2606_16359_b300.net import LeNet, MobileNetBlocks  # noqa: E402


def u64(t):
    return t.detach().cpu().numpy().view(np.uint64)


def test_lenet_reduced_ring_bit_exact():
    logN, delta = 11, 2.0 ** 35
    wts = W.lenet_weights(0)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        ctx = fe.Context(logN, 8, 2, 40, 40)
        net = LeNet(ctx, delta, wts, key_seed=9)
        x = W.lenet_input(0, net.BS)
        ct = net.encrypt(x, seed=3)
        out = net.forward(ct, mode=1)
        got = u64(out)
        y = net.decode_logits(out)
    pr = ckks.Params(logN, 8, 2, 40, 40)
    lay = henn.lenet_layouts(pr.N, net.BS)
    keys = ckks.KeySet(pr, 9, rot_steps=henn.lenet_rotation_steps(pr.N, net.BS), relin=True)
    slots = fragment.pack(lay, x)
    octs = [ckks.encrypt(pr, keys.sk, ckks.encode(pr, slots[i], pr.L, delta), 3, i) for i in range(lay.n_ct)]
    oout, P = henn.he_lenet(pr, keys, octs, lay, wts, delta)
    assert np.array_equal(got, np.stack([c.as_array() for c in oout]))
    assert oout[0].scale == net.out_scale
    assert np.abs(y - plain.lenet(x, wts)).max() < 1e-3


def test_lenet_full_size_matches_fp64():
    p = W.PARAMS["lenet"]
    wts = W.lenet_weights(0)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        ctx = fe.Context(p["logN"], p["n_q"], p["k"], p["bits"], p["pbits"])
        net = LeNet(ctx, p["delta"], wts)
        assert net.BS == 128
        x = W.lenet_input(0, net.BS)
        ctx.reset_counters()
        out_b = net.forward(net.encrypt(x), mode=1)
        cnt = ctx.counters()
        y = net.decode_logits(out_b)
        out_p = net.forward(net.encrypt(x), mode=0)
        assert np.array_equal(u64(out_b), u64(out_p))
    assert np.abs(y - plain.lenet(x, wts)).max() < 1e-3
    # Table 4 invariant: key switches = rotations + relinearisations (one per x^2 ciphertext)
    assert cnt["keyswitch"] - cnt["rot"] == cnt["cmult"] == 96 + 64


def test_mobilenet_blocks_decrypt_to_fp64_and_sampled_oracle_ct():
    p = W.PARAMS["mobilenet"]
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        ctx = fe.Context(p["logN"], p["n_q"], p["k"], p["bits"], p["pbits"])
        net = MobileNetBlocks(ctx, delta=p["delta"])
        net.run(mode=1)
        torch.cuda.synchronize()
        errs = [float(np.abs(net.decrypt_block(b) - net.reference_block(b)).max()) for b in range(3)]
        dw3 = net.layers[4]
        got = u64(dw3["out"][0:1])
        assert dw3["name"] == "b2_dw"
    assert max(errs) < 1e-3, errs
    # sampled output: ciphertext 0 of block 3's depthwise layer, recomputed by the oracle
    H, Cin, Cout = W.MOBILENET_BLOCKS[2]
    x, wd, wp = W.mobilenet_block(0, H, Cin, Cout, BS=1, block=2)
    pr = ckks.Params(p["logN"], p["n_q"], p["k"], p["bits"], p["pbits"])
    olay = fragment.Layout(pr.N, H, H, Cin, 1, 1)
    steps = henn.conv_rotation_steps(olay, Cin, Cin, 3, depthwise=True)
    keys = ckks.KeySet(pr, 101, rot_steps=steps)
    slots = fragment.pack(olay, x)
    id0 = 16 + 16  # ciphertext ids of the third block's inputs
    oct0 = ckks.encrypt(pr, keys.sk, ckks.encode(pr, slots[0], pr.L, p["delta"]), 202, id0)
    # group 0 only: channels 0..cpc-1 live in input ciphertext 0
    sub = fragment.Layout(pr.N, H, H, olay.cpc, 1, 1)
    oout, _ = henn.he_conv(pr, keys, [oct0], sub, wd[:olay.cpc], depthwise=True)
    assert np.array_equal(got[0], oout[0].as_array())


def test_mobilenet_blocks_in_the_bench_launch_configuration():
    """The benchmark's own configuration at full size (N = 2^16, 24 x 36-bit +
    4 special primes): schedules picked by the autotuner, one captured graph per
    block launched side by side on its own stream with the host copies inside,
    the streams left running ahead across steps.  Every block's output decrypts
    to the FP64 result within 1e-3; the copied-back residues equal the eager
    batched path and the per-op path bit for bit; and ciphertext 0 of the
    smallest block's depthwise layer, in the hoisting the tuner chose, equals
    the oracle's."""
    p = W.PARAMS["mobilenet"]
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        ctx = fe.Context(p["logN"], p["n_q"], p["k"], p["bits"], p["pbits"])
        net = MobileNetBlocks(ctx, delta=p["delta"], schedule="tuned")
        net.run(mode=1)
        torch.cuda.synchronize()
        eager = [u64(o) for o in net.outputs]
        net.run(mode=0)
        torch.cuda.synchronize()
        per_op = [u64(o) for o in net.outputs]
        net.capture(concurrent=True)
        h_in = [t.cpu().pin_memory() for t in net.inputs]
        h_out = [torch.empty(t.shape, dtype=t.dtype, pin_memory=True) for t in net.outputs]
        for t in net.inputs + net.outputs:
            t.zero_()
        for _ in range(2):
            net.launch(h_in, h_out, join=False)
        net.join()
        torch.cuda.synchronize()
        for o, h in zip(net.outputs, h_out):
            o.copy_(h)
        errs = [float(np.abs(net.decrypt_block(b) - net.reference_block(b)).max()) for b in range(3)]
        dw3 = net.layers[4]
        got = u64(dw3["out"][0:1])
        hoist = {0: "single", 1: "double", 2: "double_fused"}[dw3["plan"].info.double_hoist]
        assert ctx.device_status() == 0
    assert max(errs) < 1e-3, errs
    for b in range(3):
        graph_out = h_out[b].numpy().view(np.uint64)
        assert np.array_equal(graph_out, eager[b]) and np.array_equal(graph_out, per_op[b]), b
    H, Cin, Cout = W.MOBILENET_BLOCKS[2]
    x, wd, wp = W.mobilenet_block(0, H, Cin, Cout, BS=1, block=2)
    pr = ckks.Params(p["logN"], p["n_q"], p["k"], p["bits"], p["pbits"])
    olay = fragment.Layout(pr.N, H, H, Cin, 1, 1)
    keys = ckks.KeySet(pr, 101, rot_steps=henn.conv_rotation_steps(olay, Cin, Cin, 3, depthwise=True))
    slots = fragment.pack(olay, x)
    oct0 = ckks.encrypt(pr, keys.sk, ckks.encode(pr, slots[0], pr.L, p["delta"]), 202, 16 + 16)
    sub = fragment.Layout(pr.N, H, H, olay.cpc, 1, 1)
    oout, _ = henn.he_conv(pr, keys, [oct0], sub, wd[:olay.cpc], depthwise=True,
                           hoist=hoist)
    assert np.array_equal(got[0], oout[0].as_array())
