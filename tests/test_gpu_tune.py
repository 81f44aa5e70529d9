"""The schedule autotuner: every candidate is timed, the fastest is chosen and
cached, and a network built with the tuned schedules decrypts to the FP64
result (each schedule's residues are pinned by the BSGS parity tests)."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2606_16359_b300 as fe  # noqa: E402
from paper_2606_16359_b300.net import MobileNetBlocks  # noqa: E402
from paper_2606_16359_b300.tune import Tuner  # noqa: E402


def test_tuner_times_all_candidates_and_tuned_blocks_decrypt():
    p = W.PARAMS["mobilenet_small"]
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        ctx = fe.Context(p["logN"], p["n_q"], p["k"], p["bits"], p["pbits"])
        t = Tuner(ctx, n_keys=4, n_pts=8)
        lay = ctx.layout(8, 8, 64, 1, 1)  # cpc = 32 at N = 2^12
        n1, dh, times = t.conv_schedule(lay, 64, 1, level=ctx.L - 1)
        assert {int(k.split("/")[0]) for k in times} == {0, 2, 4, 8, 16, 32}
        assert times[f"{n1}/{int(dh)}"] == min(times.values()) and all(v > 0 for v in times.values())
        assert t.conv_schedule(lay, 64, 1, level=ctx.L - 1)[2] == times  # cached
        plan = ctx.plan_conv(lay, 64, 1, level=ctx.L - 1, bsgs_n1=n1, double_hoist=dh)
        ways, wt = t.mac_ways(plan)
        assert set(wt) == {1, 2, 4} and wt[ways] == min(wt.values()) and plan.mac_ways == ways
        net = MobileNetBlocks(ctx, blocks=[(8, 64, 64), (6, 32, 48)], delta=p["delta"], schedule="tuned")
        net.run(mode=1)
        torch.cuda.synchronize()
        errs = [float(np.abs(net.decrypt_block(b) - net.reference_block(b)).max()) for b in range(2)]
    assert max(errs) < 1e-3, errs
    assert len(net.schedule) == 2 and len(net.tune_ms) == 2



def test_batched_blocks_graph_decrypt_every_input():
    """Three inputs per block in one graph-captured step: every input decrypts to
    its FP64 result, and equals the same input run alone bit for bit."""
    p = W.PARAMS["mobilenet_small"]
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        ctx = fe.Context(p["logN"], p["n_q"], p["k"], p["bits"], p["pbits"])
        net = MobileNetBlocks(ctx, blocks=[(8, 64, 64)], delta=p["delta"], schedule=4, batch=3)
        net.capture()
        net.graph.launch()
        torch.cuda.synchronize()
        errs = [float(np.abs(net.decrypt_block(0, b) - net.reference_block(0, b)).max()) for b in range(3)]
        out = net.outputs[0].cpu().numpy()
        single = MobileNetBlocks(ctx, blocks=[(8, 64, 64)], delta=p["delta"], schedule=4, batch=1)
        single.run()
        torch.cuda.synchronize()
        one = single.outputs[0].cpu().numpy()
    assert max(errs) < 1e-3, errs
    assert np.array_equal(out[:one.shape[0]], one)


def test_concurrent_block_graphs_equal_sequential():
    """One graph per independent block, launched side by side on their own
    streams with the host copies in and out inside each stream: the outputs
    copied back equal the residues of the layers run one after another."""
    p = W.PARAMS["mobilenet_small"]
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        ctx = fe.Context(p["logN"], p["n_q"], p["k"], p["bits"], p["pbits"])
        net = MobileNetBlocks(ctx, blocks=[(8, 16, 16), (8, 32, 32), (4, 64, 64)], delta=p["delta"], schedule=4)
        net.run(mode=1)
        torch.cuda.synchronize()
        want = [o.cpu().numpy() for o in net.outputs]
        net.capture(concurrent=True)
        assert len(net.graphs) == 3
        h_in = [t.cpu().pin_memory() for t in net.inputs]
        h_out = [torch.empty(t.shape, dtype=t.dtype, pin_memory=True) for t in net.outputs]
        for t in net.inputs + net.outputs:
            t.zero_()
        for _ in range(2):
            net.launch(h_in, h_out)
        torch.cuda.synchronize()
    for w_, h in zip(want, h_out):
        assert np.array_equal(h.numpy(), w_)


def test_request_chunked_graph_equals_one_chunk():
    """Five inputs per block captured with the requests taken two at a time
    (fe_graph_capture_chunked: chunks of 2, 2, 1 over one data region per
    graph, a smaller workspace) give the residues of the unchunked capture,
    and every input decrypts to its FP64 result."""
    p = W.PARAMS["mobilenet_small"]
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        ctx = fe.Context(p["logN"], p["n_q"], p["k"], p["bits"], p["pbits"])
        net = MobileNetBlocks(ctx, blocks=[(8, 32, 32), (4, 64, 64)], delta=p["delta"], schedule=4, batch=5)
        plans = [l_["plan"] for l_ in net.layers[:2]]
        assert ctx.graph_workspace_bytes_chunked(plans, 5, 2) < ctx.graph_workspace_bytes(plans, 5)
        net.capture(concurrent=True)
        net.launch()
        torch.cuda.synchronize()
        want = [o.cpu().numpy() for o in net.outputs]
        for o in net.outputs:
            o.zero_()
        net.capture(concurrent=True, req_chunk=2)
        net.launch()
        torch.cuda.synchronize()
        got = [o.cpu().numpy() for o in net.outputs]
        errs = [float(np.abs(net.decrypt_block(b, r) - net.reference_block(b, r)).max())
                for b in range(2) for r in range(5)]
        assert ctx.device_status() == 0
    for w_, g_ in zip(want, got):
        assert np.array_equal(g_, w_)
    assert max(errs) < 1e-3, errs


def test_graph_host_outputs_at_level_1_are_the_dropped_limbs_and_decrypt():
    """fe_graph_set_host_output_level: the host receives the first two limbs of
    every output polynomial (the same ciphertexts modulo q_0 q_1), which equal
    the device residues' first limbs and decrypt to the FP64 blocks."""
    p = W.PARAMS["mobilenet_small"]
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        ctx = fe.Context(p["logN"], p["n_q"], p["k"], p["bits"], p["pbits"])
        net = MobileNetBlocks(ctx, blocks=[(8, 16, 16), (4, 64, 64)], delta=p["delta"], schedule=4)
        net.capture(concurrent=True)
        h_in = [t.cpu().pin_memory() for t in net.inputs]
        full = net.host_outputs(None)
        net.launch(h_in, full)
        torch.cuda.synchronize()
        low = net.host_outputs(1)
        ib, ob = net.graphs[0].io()
        assert ob == [low[0].numel() * 8]
        net.launch(h_in, low)
        torch.cuda.synchronize()
        errs = []
        for b in range(2):
            assert np.array_equal(low[b].numpy(), full[b].numpy()[:, :, :2, :])
            slots = ctx.decrypt(net.sk, low[b].to("cuda"), 1, net.delta)
            y = ctx.unpack(net.ref_inputs[b][3], slots).cpu().numpy()
            errs.append(float(np.abs(y - net.reference_block(b)).max()))
        with pytest.raises(fe.FencError):
            net.graphs[0].set_host_output_level(ctx.L)  # above the outputs' level
    assert max(errs) < 1e-3, errs


def test_graph_with_every_ntt_form_equals_eager_default():
    """At N = 2^16 (where the cluster form of the NTT exists), a block captured
    in a graph with the single-pass cluster NTT (fe_ctx_set_ntt_path(2)) and
    with the other forward forms (fe_ctx_set_ntt_forward) gives the residues
    of the eager run with the default two-pass transform."""
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        ctx = fe.Context(16, 4, 2, 36, 36)
        net = MobileNetBlocks(ctx, blocks=[(8, 16, 16)], delta=2.0 ** 30, schedule=4)
        net.run(mode=1)
        torch.cuda.synchronize()
        want = net.outputs[0].cpu().numpy()
        err = float(np.abs(net.decrypt_block(0) - net.reference_block(0)).max())
        for path, fwd in ((2, 0), (0, 3), (1, 1)):
            ctx.set_ntt_path(path)
            ctx.set_ntt_forward(fwd)
            net.outputs[0].zero_()
            net.capture()
            net.graph.launch()
            torch.cuda.synchronize()
            assert np.array_equal(net.outputs[0].cpu().numpy(), want), (path, fwd)
        ctx.set_ntt_path(0)
        ctx.set_ntt_forward(0)
        assert ctx.device_status() == 0
    assert err < 1e-3, err
