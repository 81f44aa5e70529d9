"""The request loop (continuous batching over two ring sizes, admission by
device memory) on the GPU: every request's result is the same alone and in the
mix (residues bit-exact, so within any tolerance), decrypted LeNet logits match
the FP64 network, batching and overlap actually happen, and memory admission
serialises or rejects as configured."""
import numpy as np
import pytest

import workloads as W
from oracle import plain

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2606_16359_b300 as fe  # noqa: E402
from paper_2606_16359_b300.net import LeNet, MobileNetBlocks  # noqa: E402


@pytest.fixture(scope="module")
def models():
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        c_small = fe.Context(11, 8, 2, 40, 40)          # LeNet shape at N = 2^11
        wts = W.lenet_weights(0)
        lenet = LeNet(c_small, 2.0 ** 35, wts, key_seed=9)
        xs = [W.lenet_input(i, lenet.BS) for i in range(3)]
        l_in = [lenet.encrypt(x, seed=40 + i).cpu().pin_memory() for i, x in enumerate(xs)]
        p = W.PARAMS["mobilenet_small"]
        # N = 2^14 and 128 channels: a block group keeps the device busy for
        # several milliseconds, longer than the host takes to enqueue a LeNet
        # group, so overlap is observable (a 32-channel block finished before
        # the next group was enqueued once the transforms got faster)
        c_mb = fe.Context(14, p["n_q"], p["k"], p["bits"], p["pbits"])
        mb = MobileNetBlocks(c_mb, blocks=[(32, 128, 128)], delta=p["delta"])
        m_in = [mb.inputs[0].cpu().pin_memory()]
        torch.cuda.synchronize()
    return dict(lenet=lenet, xs=xs, wts=wts, l_in=l_in, mb=mb, m_in=m_in, stream=s)


def _server(M, **kw):
    srv = fe.Server(**kw)
    lenet, mb = M["lenet"], M["mb"]
    ml = srv.add_model(lenet.ctx, lenet.evk, lenet.serve_ops(), lenet.lay0.n_ct, lenet.ctx.L)
    mm = srv.add_model(mb.ctx, mb.evk, mb.serve_ops(0), mb.layers[0]["plan"].info.n_in_ct, mb.ctx.L)
    return srv, ml, mm


def _out_buf(srv, model):
    n_ct, lv, _, ob = srv.model_io(model)
    return torch.empty(ob // 8, dtype=torch.int64).pin_memory()


def _workload(M):
    # 10 requests: LeNet inputs 0, 1, 2 and the MobileNet-shaped block, interleaved;
    # the block's group is formed first, the LeNet groups run beside it
    kinds = ["m", "l0", "l1", "m", "l2", "l0", "m", "l1", "l2", "l0"]
    return kinds


def _inp(M, k):
    return M["m_in"][0] if k == "m" else M["l_in"][int(k[1])]


def test_alone_equals_mix_and_decrypts(models):
    M = models
    kinds = _workload(M)
    # alone: one request at a time, no batching, one stream
    srv, ml, mm = _server(M, max_batch=1, max_inflight=1)
    alone = {}
    for k in ("l0", "l1", "l2", "m"):
        out = _out_buf(srv, mm if k == "m" else ml)
        rid = srv.submit(mm if k == "m" else ml, _inp(M, k), out)
        st, lat = srv.wait(rid)
        assert st == 0 and lat > 0
        alone[k] = out.numpy().copy()
    srv.close()
    # mix: a burst queued while admission is paused, then batched (up to 4 per
    # group) and overlapped (3 streams)
    srv, ml, mm = _server(M, max_batch=4, max_inflight=3)
    srv.pause(True)
    outs, rids = [], []
    for k in kinds:
        out = _out_buf(srv, mm if k == "m" else ml)
        outs.append(out)
        rids.append(srv.submit(mm if k == "m" else ml, _inp(M, k), out))
    srv.pause(False)
    for rid in rids:
        st, _ = srv.wait(rid)
        assert st == 0
    stats = srv.stats()
    srv.close()
    for k, out in zip(kinds, outs):
        assert np.array_equal(out.numpy(), alone[k]), k
    assert stats["completed"] == len(kinds) and stats["rejected"] == 0
    assert stats["max_group"] >= 2, stats        # requests of one model were batched
    assert 2 <= stats["max_inflight"] <= 3, stats  # groups overlapped on the device, at most 3 at once
    assert 0 < stats["p50_ms"] <= stats["p99_ms"]
    # decrypted logits of a served LeNet request against the FP64 network
    lenet = M["lenet"]
    with torch.cuda.stream(M["stream"]):
        ct = torch.from_numpy(alone["l1"]).cuda().view(-1, 2, lenet.ctx.L - 7 + 1, lenet.ctx.N)
        y = lenet.decode_logits(ct)
    assert np.abs(y - plain.lenet(M["xs"][1], M["wts"])).max() < 1e-3


def test_request_larger_than_the_budget_is_rejected(models):
    M = models
    srv, ml, mm = _server(M, max_batch=1, max_inflight=3, hbm_budget_bytes=1)
    out = _out_buf(srv, ml)
    st, _ = srv.wait(srv.submit(ml, M["l_in"][0], out))
    assert st == fe.FE_ENOMEM
    assert srv.stats()["rejected"] == 1 and srv.stats()["completed"] == 0
    srv.close()


def test_admission_serialises_when_memory_is_short(models):
    M = models
    # measure one LeNet group's footprint, then give room for one group only
    srv, ml, mm = _server(M, max_batch=1, max_inflight=3)
    out = _out_buf(srv, ml)
    st, _ = srv.wait(srv.submit(ml, M["l_in"][0], out))
    need = srv.stats()["peak_bytes"]
    srv.close()
    srv, ml, mm = _server(M, max_batch=1, max_inflight=3, hbm_budget_bytes=need + need // 2)
    outs = [_out_buf(srv, ml) for _ in range(4)]
    rids = [srv.submit(ml, M["l_in"][i % 3], outs[i]) for i in range(4)]
    for r in rids:
        st, _ = srv.wait(r)
        assert st == 0
    s = srv.stats()
    srv.close()
    assert s["max_inflight"] == 1 and s["completed"] == 4 and s["peak_bytes"] <= need + need // 2


def test_arrivals_during_running_groups_are_batched(models):
    """Continuous batching: with the only stream busy on a LeNet request, the
    requests that arrive meanwhile queue and are admitted in groups when the
    stream frees up (the MobileNet-shaped one first, as the oldest, then the
    LeNet ones together); equal inputs give equal outputs."""
    M = models
    srv, ml, mm = _server(M, max_batch=8, max_inflight=1)
    first = _out_buf(srv, ml)
    r0 = srv.submit(ml, M["l_in"][0], first)
    mid = _out_buf(srv, mm)
    r1 = srv.submit(mm, M["m_in"][0], mid)
    outs = [_out_buf(srv, ml) for _ in range(6)]
    rids = [srv.submit(ml, M["l_in"][i % 3], outs[i]) for i in range(6)]
    for r in [r0, r1] + rids:
        assert srv.wait(r)[0] == 0
    s = srv.stats()
    srv.close()
    assert s["completed"] == 8 and s["groups"] < 8 and s["max_group"] >= 2, s
    assert np.array_equal(outs[0].numpy(), first.numpy())
    for i in range(6):
        assert np.array_equal(outs[i].numpy(), outs[i % 3].numpy())


def test_served_refresh_chain_equals_the_direct_chain():
    """A model whose operations include activations and a ciphertext refresh
    (block, refresh, block at N = 2^10, 22 primes of 50 bits): every request's
    served result equals the direct chain's residues, alone and batched two at
    a time."""
    from paper_2606_16359_b300.net import RefreshChain
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        ctx = fe.Context(10, 22, 4, 50)
        ch = RefreshChain(ctx, 6, 4, h=32, key_seed=41, seed=5)
        want = ch.forward().cpu().numpy()
        torch.cuda.synchronize()
    srv = fe.Server(max_batch=2, max_inflight=2)
    try:
        mid = srv.add_model(ctx, ch.evk, ch.serve_ops(), ch.lay.n_ct, ctx.L)
        n_ct, lv, ib, ob = srv.model_io(mid)
        assert lv == ch.out_level and ib == ch.ct.numel() * 8
        inp = ch.ct.cpu().pin_memory()
        outs = [torch.empty(ob // 8, dtype=torch.int64).pin_memory() for _ in range(3)]
        srv.pause(True)
        rids = [srv.submit(mid, inp, o) for o in outs]
        srv.pause(False)
        for rid in rids:
            st, _ = srv.wait(rid)
            assert st == 0
        for o in outs:
            assert np.array_equal(o.numpy(), want.reshape(-1))
        assert srv.stats()["max_group"] == 2
    finally:
        srv.close()
