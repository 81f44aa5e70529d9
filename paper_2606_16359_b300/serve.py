"""Serving workload: a Poisson stream of encrypted requests through the request
loop (fe_server_*), mixing LeNet-shaped inferences at N = 2^14 (one request =
one encrypted slot batch of 128 images through the whole network) and
MobileNet-block-shaped inferences at N = 2^16 (one request = one input through
the 56x56x128 -> 128 dw3x3 + pw block).  Keys and plaintexts of both models are
resident; admission is by free device memory; inputs are U[0, 1) (LeNet) and
U[-1, 1) (MobileNet block), encrypted once per distinct input ahead of time
and copied host -> device inside each request.

    python -m paper_2606_16359_b300.serve [--duration 20] [--loads 0.5,0.8,1.0]
        [--mix 0.8] [--deep 0.0] [--max-batch 4] [--max-inflight 3]

--deep F adds a third model, a fraction F of the requests: a deeper network
that refreshes its ciphertexts between blocks (net.RefreshChain: dw3x3 + pw
block, refresh, block on a 14x14x32 map at N = 2^16 with 24 + 4 primes of 50
bits, a dense secret and an encapsulated refresh); the LeNet fraction stays
--mix and the MobileNet block takes the rest.

Capacity is measured first: each model alone, one request at a time; the mix's
capacity is 1 / (f t_lenet + d t_deep + (1 - f - d) t_mobilenet), d the --deep
fraction.  Then, for each load factor,
requests arrive at rate load x capacity for `duration` seconds (exponential
inter-arrival times, seeded) and the loop reports p50 / p99 latency (submit to
result in host memory) and completed requests per second.  One JSON line per
load factor.
"""
import argparse
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def build_models(torch, fe, mb_block=(56, 128, 128), deep=False):
    import workloads as W
    from .net import LeNet, MobileNetBlocks, RefreshChain

    p = W.PARAMS["lenet"]
    c14 = fe.Context(p["logN"], p["n_q"], p["k"], p["bits"], p["pbits"])
    wts = W.lenet_weights(0)
    lenet = LeNet(c14, p["delta"], wts)
    l_in = [lenet.encrypt(W.lenet_input(i, lenet.BS), seed=50 + i).cpu().pin_memory() for i in range(4)]
    q = W.PARAMS["mobilenet"]
    c16 = fe.Context(q["logN"], q["n_q"], q["k"], q["bits"], q["pbits"])
    mb = MobileNetBlocks(c16, blocks=[mb_block], delta=q["delta"])
    m_in = [mb.inputs[0].cpu().pin_memory()]
    M = dict(lenet=lenet, l_in=l_in, mb=mb, m_in=m_in)
    if deep:
        c50 = fe.Context(16, 24, 4, 50)
        ch = RefreshChain(c50, 14, 32, h=64, encapsulate=True)
        M.update(deep=ch, d_in=[ch.ct.cpu().pin_memory()])
    torch.cuda.synchronize()
    return M


def make_server(fe, M, max_batch, max_inflight):
    srv = fe.Server(max_batch=max_batch, max_inflight=max_inflight)
    lenet, mb = M["lenet"], M["mb"]
    ml = srv.add_model(lenet.ctx, lenet.evk, lenet.serve_ops(), lenet.lay0.n_ct, lenet.ctx.L)
    mm = srv.add_model(mb.ctx, mb.evk, mb.serve_ops(0), mb.layers[0]["plan"].info.n_in_ct, mb.ctx.L)
    md = None
    if "deep" in M:
        ch = M["deep"]
        md = srv.add_model(ch.ctx, ch.evk, ch.serve_ops(), ch.lay.n_ct, ch.ctx.L)
    return srv, ml, mm, md


def out_buffers(torch, srv, model, n):
    _, _, _, ob = srv.model_io(model)
    return [torch.empty(ob // 8, dtype=torch.int64).pin_memory() for _ in range(n)]


def service_time(torch, fe, M, which, reps=3):
    srv, ml, mm, md = make_server(fe, M, 1, 1)
    model = {"lenet": ml, "mobilenet_block": mm, "deep_chain": md}[which]
    inp = {"lenet": M["l_in"][0], "mobilenet_block": M["m_in"][0], "deep_chain": M.get("d_in", [None])[0]}[which]
    outs = out_buffers(torch, srv, model, 1)
    srv.wait(srv.submit(model, inp, outs[0]))  # warm-up
    lat = []
    for _ in range(reps):
        st, ms = srv.wait(srv.submit(model, inp, outs[0]))
        assert st == 0
        lat.append(ms)
    srv.close()
    return float(np.median(lat)) / 1e3


def run_load(torch, fe, M, rate, duration, mix, max_batch, max_inflight, seed, pool=(64, 8), deep=0.0):
    """Poisson arrivals for `duration` seconds; a waiter thread collects results
    in submission order and recycles the pinned output buffers (pools of
    pool[0] LeNet and pool[1] MobileNet-block or deep-chain outputs; a
    submission that finds its pool empty waits and is counted as late)."""
    import queue
    import threading

    rng = np.random.default_rng(seed)
    srv, ml, mm, md = make_server(fe, M, max_batch, max_inflight)
    free = {ml: queue.Queue(), mm: queue.Queue()}
    for b in out_buffers(torch, srv, ml, pool[0]):
        free[ml].put(b)
    for b in out_buffers(torch, srv, mm, pool[1]):
        free[mm].put(b)
    if md is not None:
        free[md] = queue.Queue()
        for b in out_buffers(torch, srv, md, pool[1]):
            free[md].put(b)
    todo = queue.Queue()
    lat = {"lenet": [], "mobilenet_block": []}
    if md is not None:
        lat["deep_chain"] = []
    failed = [0]

    def waiter():
        while True:
            item = todo.get()
            if item is None:
                return
            rid, model, buf, kind = item
            st, ms = srv.wait(rid)
            if st == 0:
                lat[kind].append(ms)
            else:
                failed[0] += 1
            free[model].put(buf)

    th = threading.Thread(target=waiter)
    th.start()
    n, late = 0, 0
    t0 = time.perf_counter()
    t_next = t0
    while True:
        t_next += rng.exponential(1.0 / rate)
        if t_next - t0 > duration:
            break
        now = time.perf_counter()
        if t_next > now:
            time.sleep(t_next - now)
        u = rng.uniform()
        if u < mix:
            model, kind, inp = ml, "lenet", M["l_in"][n % len(M["l_in"])]
        elif md is not None and u < mix + deep:
            model, kind, inp = md, "deep_chain", M["d_in"][0]
        else:
            model, kind, inp = mm, "mobilenet_block", M["m_in"][0]
        try:
            buf = free[model].get_nowait()
        except queue.Empty:
            late += 1
            buf = free[model].get()
        todo.put((srv.submit(model, inp, buf), model, buf, kind))
        n += 1
    todo.put(None)
    th.join()
    t_end = time.perf_counter()
    stats = srv.stats()
    srv.close()
    per = {k: {"n": len(v), "p50_ms": float(np.percentile(v, 50)) if v else None,
               "p99_ms": float(np.percentile(v, 99)) if v else None} for k, v in lat.items()}
    return stats, per, n / (t_end - t0), t_end - t0, late, failed[0]


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--duration", type=float, default=20.0)
    ap.add_argument("--loads", default="0.5,0.8,1.0")
    ap.add_argument("--mix", type=float, default=0.8, help="fraction of LeNet-shaped requests")
    ap.add_argument("--deep", type=float, default=0.0,
                    help="fraction of deep-chain requests (block, refresh, block; 0: not built)")
    ap.add_argument("--max-batch", type=int, default=4)
    ap.add_argument("--max-inflight", type=int, default=3)
    ap.add_argument("--seed", type=int, default=0)
    args = ap.parse_args(argv)
    import torch

    sys.path.insert(0, ROOT)
    import paper_2606_16359_b300 as fe

    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        if args.mix < 0 or args.deep < 0 or args.mix + args.deep > 1:
            raise SystemExit("--mix and --deep must be fractions summing to at most 1")
        M = build_models(torch, fe, deep=args.deep > 0)
        t_l = service_time(torch, fe, M, "lenet")
        t_m = service_time(torch, fe, M, "mobilenet_block")
        t_d = service_time(torch, fe, M, "deep_chain") if args.deep > 0 else 0.0
        cap = 1.0 / (args.mix * t_l + args.deep * t_d + (1 - args.mix - args.deep) * t_m)
        for load in (float(x) for x in args.loads.split(",")):
            stats, per, offered, wall, late, failed = run_load(torch, fe, M, load * cap, args.duration, args.mix,
                                                               args.max_batch, args.max_inflight, args.seed,
                                                               deep=args.deep)
            line = {"metric": "serving latency and throughput", "load": load, "offered_req_per_s": offered,
                    "capacity_req_per_s_alone": cap,
                    "service_s_alone": dict({"lenet": t_l, "mobilenet_block": t_m},
                                            **({"deep_chain": t_d} if args.deep > 0 else {})),
                    "completed": stats["completed"], "rejected": stats["rejected"], "failed": failed,
                    "late_submissions": late,
                    "req_per_s": stats["completed"] / wall, "p50_ms": stats["p50_ms"], "p99_ms": stats["p99_ms"],
                    "per_model": per, "groups": stats["groups"], "max_group": stats["max_group"],
                    "max_inflight": stats["max_inflight"], "peak_bytes": stats["peak_bytes"],
                    "config": {"mix_lenet": args.mix, "mix_deep_chain": args.deep,
                               "deep_chain": "N=2^16 24+4 x 50-bit, 14x14x32 dw+pw, refresh, dw+pw, dense secret",
                               "lenet": "N=2^14 L=7 BS=128",
                               "mobilenet_block": "N=2^16 L=23 56x56x128->128", "duration_s": args.duration,
                               "max_batch": args.max_batch, "max_inflight": args.max_inflight,
                               "arrivals": "Poisson, seed %d" % args.seed}}
            print(json.dumps(line), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
