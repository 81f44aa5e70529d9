"""Benchmark of the encrypted-convolution hot path on B300.

Workload (default): the three MobileNet-shaped blocks (depthwise 3x3 then
pointwise) at N = 2^16, 24 x 36-bit + 4 special primes, scale 2^32, inputs
U[-1, 1), weights N(0, 1/fan_in), fragment size S = 1, one encrypted input per
block.  A step runs all six HE convolutions (inner rotations, PMult-MAC,
outer rotations, rescale) with keys, plaintexts and ciphertexts resident.  The
outer rotations of each pointwise layer use the schedule the autotuner times
fastest (linear or baby-step / giant-step); --schedule linear keeps one outer
rotation per channel diagonal.  The blocks are independent, so a step
launches one captured graph per block on its own stream (--one-stream: one
graph over the six layers in order); the end-to-end run copies each block's
input in and output out inside that block's stream.  The per-block streams are
joined only at the end of a timed region: one block's next step queues behind
its own previous step while the other blocks are still busy.

Reported: key switches per second (the metric's throughput form), ms per step
and per layer, beside the batched/graph path two per-op paths (mode 0: one
launch per primitive per ciphertext with the same hoisted schedule; mode 2: the
layer composed from single-ciphertext operations, every rotation a key switch
of its own), the
roofline fraction of the dominant kernel class, the CPU oracle timed on the
host, an end-to-end number through host buffers, and SM clocks sampled during
the timed region.

    python bench.py [--steps K] [--warmup W] [--gpus N] [--impl reference]
"""
import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "he_conv layer ms & key-switches/s on 1 B300, % HBM roofline, vs plain path"
PARAMS = dict(logN=16, n_q=24, k=4, qbits=36, pbits=36)
DELTA = 2.0 ** 32
WORKLOAD = "mobilenet_blocks_3x(dw3x3+pw)_N2^16_L23_k4"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 50 ms while running; the
    sampler has written its first line before the block it wraps starts, so the
    samples cover the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        import tempfile
        fd, self.path = tempfile.mkstemp(prefix="fenc_clocks_", suffix=".csv")
        os.close(fd)

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        if self.proc is not None:
            t0 = time.time()
            while time.time() - t0 < 3.0 and self.proc.poll() is None and os.path.getsize(self.path) == 0:
                time.sleep(0.02)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            self.proc.wait()
            self.f.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        try:
            os.unlink(self.path)
        except OSError:
            pass
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
        return dist, rank, world, local
    return None, 0, 1, local


def reduce_max(dist, v):
    if dist is None:
        return v
    import torch
    t = torch.tensor([v], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(dist):
    if dist is not None:
        dist.barrier()


def profiled_traffic(profile, key, source):
    """A DRAM-traffic figure (ncu dram__bytes_read.sum + dram__bytes_write.sum)
    recorded in a profiles/ summary as `<key> <bytes> <source>_sha256 <hash>`,
    or None when the kernel source changed since that capture."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "paper_2606_16359_b300", "csrc", source), "rb") as f:
            sha = hashlib.sha256(f.read()).hexdigest()
        with open(os.path.join(ROOT, "profiles", profile)) as f:
            for line in f:
                w = line.split()
                if len(w) == 4 and w[0] == key:
                    return float(w[1]) if w[3] == sha else None
    except OSError:
        pass
    return None


def ntt_traffic_per_limb_pass():
    """DRAM bytes of one limb-pass of the NTT (ncu over 532 limbs)."""
    return profiled_traffic("ntt_pass_N65536_532limbs.txt", "traffic_bytes_per_limb_pass", "ntt.cu")


def mac_traffic_ratio():
    """DRAM bytes / algorithmic bytes of the PMult-MAC, from ncu on a small
    pointwise layer (one kernel, two launches, a few GB resident); the MAC
    streams each operand once, so its traffic scales with its algorithmic
    bytes."""
    return profiled_traffic("mac_traffic_pointwise_14x14x128_layer.txt", "traffic_ratio_to_algorithmic", "kernels.cu")


# Warp instructions per lazy Shoup butterfly, counted by ncu on the register-
# resident probe (profiles/ntt_pass_N65536_532limbs.txt).
BUTTERFLY_WARP_INSTRUCTIONS = 23.2


def butterfly_issue_roof(torch):
    """Butterflies per second at the issue limit, Gbutterfly/s: every SM's four
    schedulers issue one warp instruction per clock at the maximum SM clock, and
    a warp completes 32 butterflies per BUTTERFLY_WARP_INSTRUCTIONS."""
    n_sm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    mhz = None
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            mhz = float(json.load(f).get("sm_max_mhz") or 0) or None
    except (OSError, ValueError):
        pass
    if mhz is None:
        mhz = 2032.0  # B300 maximum SM clock
    return n_sm * 4 * mhz * 1e6 * 32 / BUTTERFLY_WARP_INSTRUCTIONS / 1e9, n_sm, mhz


def butterfly_roof(ctx, torch):
    """Integer-pipe roof of the NTT butterfly arithmetic on this GPU, Gbutterfly/s
    (register-resident probe of the transform's own butterflies, one full wave)."""
    n_sm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    buf = torch.empty(n_sm * 8 * 256, dtype=torch.int64, device="cuda")
    ctx.probe_butterflies(buf, 0, 40)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    best = 0.0
    for _ in range(3):
        e0.record()
        n = ctx.probe_butterflies(buf, 0, 400)
        e1.record()
        torch.cuda.synchronize()
        best = max(best, n / (e0.elapsed_time(e1) / 1e3) / 1e9)
    return best


_ORACLE = {}


def _oracle_setup(level=22):
    """Per-process oracle state: the parameter set, one rotation key and a random
    ciphertext at `level` (the level of the pointwise layers)."""
    from oracle import ckks
    pr = ckks.Params(PARAMS["logN"], PARAMS["n_q"], PARAMS["k"], PARAMS["qbits"], PARAMS["pbits"])
    keys = ckks.KeySet(pr, 1, rot_steps=[1])
    rng = np.random.default_rng(os.getpid())
    c = ckks.Ciphertext(np.stack([rng.integers(0, pr.moduli[i], pr.N, dtype=np.uint64) for i in range(level + 1)]),
                        np.stack([rng.integers(0, pr.moduli[i], pr.N, dtype=np.uint64) for i in range(level + 1)]),
                        level, 1.0)
    _ORACLE.update(ckks=ckks, pr=pr, keys=keys, c=c)


def _oracle_rotations(n_rot):
    """n_rot oracle rotations (key switches) in this process; returns seconds."""
    if not _ORACLE:
        _oracle_setup()
    o = _ORACLE
    t0 = time.perf_counter()
    for _ in range(n_rot):
        o["ckks"].rotate(o["pr"], o["keys"], o["c"], 1)
    return time.perf_counter() - t0


def host_cpu():
    """(usable host cores, CPU model)."""
    try:
        n = len(os.sched_getaffinity(0))
    except AttributeError:
        n = os.cpu_count() or 1
    model = "unknown"
    try:
        for line in open("/proc/cpuinfo"):
            if line.startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except OSError:
        pass
    return n, model


class OraclePool:
    """The CPU oracle as it stands, run in `workers` single-threaded processes
    (spawned, so they share no state with a CUDA context of the parent); each
    process holds its own parameter set, key and ciphertext."""

    def __init__(self, workers):
        import multiprocessing as mp
        self.workers = workers
        saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
        for k in saved:
            os.environ[k] = "1"
        try:
            self.pool = mp.get_context("spawn").Pool(workers, initializer=_oracle_setup)
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v

    def run(self, n_rot_each):
        """Every process runs n_rot_each rotations; returns (rotations, wall seconds)."""
        t0 = time.perf_counter()
        self.pool.map(_oracle_rotations, [n_rot_each] * self.workers, chunksize=1)
        return n_rot_each * self.workers, time.perf_counter() - t0

    def close(self):
        self.pool.close()
        self.pool.join()


def cpu_oracle_keyswitch(n_rot):
    """The CPU oracle (as it stands, single-threaded, in this process) on a
    bounded sample: n_rot rotations of one ciphertext at level 22 of the same
    parameter set (set-up and a first rotation untimed)."""
    _oracle_setup()
    _oracle_rotations(1)
    dt = _oracle_rotations(n_rot)
    return n_rot / dt, dt


REFRESH_SMALL = dict(logN=10, n_q=20, k=4, bits=50, h=32, scale_in=2.0 ** 45)


def cpu_oracle_refresh():
    """The CPU oracle's refresh (as it stands, single-threaded) of one level-0
    ciphertext on the small refresh workload (N = 2^10, 20 + 4 primes of 50
    bits, secret weight 32, default schedule); key generation untimed."""
    import time as _t

    from oracle import boot, ckks
    p = REFRESH_SMALL
    pr = ckks.Params(p["logN"], p["n_q"], p["k"], p["bits"])
    bp = boot.BootParams(pr)
    keys = boot.SparseKeySet(pr, 3, p["h"], rot_steps=boot.boot_rotation_steps(pr, bp), relin=True, conj=True)
    tab = boot.cos_table(pr.N)
    z = np.random.default_rng(12).uniform(-1, 1, pr.N // 2)
    ct = ckks.encrypt(pr, keys.sk, ckks.encode(pr, z, 0, p["scale_in"]), 4, 0)
    t0 = _t.perf_counter()
    boot.bootstrap(pr, keys, ct, bp, tab=tab)
    return _t.perf_counter() - t0


def gpu_refresh_small(torch, stream, reps=10):
    """fe_he_bootstrap on the small refresh workload (the oracle's sample above)."""
    import paper_2606_16359_b300 as fe
    p = REFRESH_SMALL
    with torch.cuda.stream(stream):
        ctx = fe.Context(p["logN"], p["n_q"], p["k"], p["bits"])
        sk = ctx.sk_gen_sparse(3, p["h"])
        b = ctx.boot_create(p["scale_in"])
        evk = ctx.evk_gen(sk, 3, b.steps, relin=True)
        z = np.random.default_rng(12).uniform(-1, 1, (1, ctx.N // 2))
        ct = ctx.encrypt(sk, z, 0, p["scale_in"], seed=4)
        ws = ctx.workspace(b.workspace_bytes(1))
        out = ctx.bootstrap(evk, b, ct, ws=ws)
        for _ in range(2):
            ctx.bootstrap(evk, b, ct, ws=ws, out=out)
        torch.cuda.synchronize()
        a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            ctx.bootstrap(evk, b, ct, ws=ws, out=out)
        e.record(stream)
        torch.cuda.synchronize()
    return a.elapsed_time(e) / reps


def cpu_oracle_all_cores(n_rot_each, max_workers=64):
    """The same oracle rotation on every usable host core (one process each, at
    most max_workers, about 0.5 GB of host memory apiece)."""
    cores, model = host_cpu()
    workers = max(1, min(cores, max_workers))
    pool = OraclePool(workers)
    try:
        pool.run(1)  # set-up and one warm rotation per process
        n, dt = pool.run(n_rot_each)
    finally:
        pool.close()
    return n / dt, dt, workers, cores, model


def refresh_bench(torch, stream, steps):
    """Time fe_he_bootstrap at N = 2^16 (24 x 50-bit primes, 4 special primes,
    secret weight 64; CoeffToSlot 3 levels, EvalMod 11, SlotToCoeff 3; stage
    groups with n1^2 >= 4 x their offsets, double-hoisted, complex form) on one level-0
    ciphertext; report ms (direct calls and one captured graph), levels, key
    switches and the decrypted error."""
    import paper_2606_16359_b300 as fe
    with torch.cuda.stream(stream):
        ctx = fe.Context(16, 24, 4, 50)
        sk = ctx.sk_gen_sparse(31, 64)
        s_in = 2.0 ** 45
        b = ctx.boot_create(s_in, 3, 3, 6)
        evk = ctx.evk_gen(sk, 31, b.steps, relin=True)
        z = np.random.default_rng(9).uniform(-1, 1, (1, ctx.N // 2))
        ct = ctx.encrypt(sk, z, 0, s_in, seed=10)
        ws = ctx.workspace(b.workspace_bytes(1))
        out = ctx.bootstrap(evk, b, ct, ws=ws)
        for _ in range(2):
            ctx.bootstrap(evk, b, ct, ws=ws, out=out)
        torch.cuda.synchronize()
        ctx.reset_counters()
        a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(steps):
            ctx.bootstrap(evk, b, ct, ws=ws, out=out)
        e.record(stream)
        torch.cuda.synchronize()
        cnt = ctx.counters()
        ms = a.elapsed_time(e) / steps
        err = float(np.abs(ctx.decrypt(sk, out, b.out_level, b.out_scale).cpu().numpy() - z).max())
        # the same refresh replayed as one captured graph (fe_boot_graph_capture)
        want = out.clone()
        g = ctx.boot_graph_capture(evk, b, ct, out, ws)
        for _ in range(2):
            g.launch()
        torch.cuda.synchronize()
        graph_equal = bool(torch.equal(out, want))
        a.record(stream)
        for _ in range(steps):
            g.launch()
        e.record(stream)
        torch.cuda.synchronize()
        ms_graph = a.elapsed_time(e) / steps
        del g, want
        # kernel classes of one refresh (CUDA events per launch), and the leading
        # class, the transform in its general 64-bit form for 50-bit moduli,
        # against the butterfly probe run on this context's modulus q_0
        by_class = {}
        for kd in ("ntt", "bconv", "keyip", "combine", "mac", "rescale"):
            ctx.profile_begin(kd)
            ctx.bootstrap(evk, b, ct, ws=ws, out=out)
            t, n, byt = ctx.profile_end()
            by_class[kd] = {"ms": round(t, 3), "launches": n, "algorithmic_GB": round(byt / 1e9, 3)}
        t_ntt = by_class["ntt"]["ms"]
        limb_passes = by_class["ntt"]["algorithmic_GB"] * 1e9 / (8.0 * ctx.N)
        bfly_rate = limb_passes * (ctx.N // 2) * (ctx.logN / 2) / (t_ntt / 1e3) / 1e9 if t_ntt else 0.0
        bfly_peak = butterfly_roof(ctx, torch)
    ks = cnt["keyswitch"] / steps
    res = {"ms": round(ms, 3), "ms_graph": round(ms_graph, 3), "graph_equals_direct": graph_equal,
           "steps": steps, "warmup": 3, "params": "N=2^16, 24 x 50-bit q, 4 x 50-bit p, h=64, groups 3/11/3 levels, baby ratio 4, double hoisting, complex form",
           "levels_used": 23 - b.out_level, "out_level": b.out_level, "keyswitches": ks,
           "keyswitch_per_s": ks / (ms / 1e3), "max_abs_err": err,
           "evk_gb": evk.buf.numel() * 8 / 1e9, "workspace_gb": ws.numel() * 8 / 1e9,
           "by_class": by_class,
           "roofline": {"kernel": "ntt", "bound": "alu", "achieved": bfly_rate, "peak": bfly_peak,
                        "unit": "Gbutterfly/s", "frac": bfly_rate / bfly_peak if bfly_peak else None,
                        "peak_source": "measured in this run: the butterfly probe on this context's 50-bit q_0 "
                                       "(general 64-bit Shoup butterflies, register-resident, one full wave)"}}
    del out, ws, ct, evk, b, sk, ctx
    return res


def run_reference(args):
    dist, rank, world, local = dist_setup(args)
    if rank != 0:
        return 0
    cores, model = host_cpu()
    workers = max(1, min(cores, 64))
    pool = OraclePool(workers)
    per_step = []
    try:
        for i in range(args.warmup + args.steps):
            n, dt = pool.run(1)
            if i >= args.warmup:
                per_step.append(dt)
    finally:
        pool.close()
    total = sum(per_step)
    value = args.steps * workers / total
    sample = (f"each step: one oracle rotation of a level-22 ciphertext (N=2^16, 6 digits) in each of {workers} "
              f"single-threaded processes, one per host core ({cores} usable, {model})")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "keyswitch/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "step": f"{workers} CPU-oracle rotations (key switches) at level 22, "
                                                     f"one per process"},
            "cpu_baseline": {"value": value, "unit": "keyswitch/s", "cores": workers, "kind": "oracle",
                             "sample": sample, "cpu_model": model},
            "e2e": {"value": value, "unit": "keyswitch/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--plain-steps", type=int, default=1)
    ap.add_argument("--cpu-rotations", type=int, default=4)
    ap.add_argument("--no-graph", action="store_true")
    ap.add_argument("--one-stream", action="store_true",
                    help="one graph over all layers in order (default: one graph per block, side by side)")
    ap.add_argument("--profile", default="auto", help="kernel class timed for the roofline, or 'auto'")
    ap.add_argument("--batch", type=int, default=1, help="independent encrypted inputs per block per step")
    ap.add_argument("--schedule", default="tuned",
                    help="outer rotations of the pointwise layers: tuned (autotuner), linear, or n1")
    ap.add_argument("--variants", type=int, default=1,
                    help="also time the one-graph form and 4 and 16 inputs per block (context fields)")
    ap.add_argument("--no-refresh", dest="refresh", action="store_false",
                    help="skip the ciphertext-refresh (bootstrapping) measurement")
    ap.add_argument("--ncu-step", action="store_true",
                    help="set up, run one warm step, then one batched step between cudaProfilerStart and "
                         "cudaProfilerStop (for ncu --profile-from-start off), and exit")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    dist, rank, world, local = dist_setup(args)
    torch.cuda.set_device(local)
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        return run_ours(args, dist, rank, world, local)


def run_ours(args, dist, rank, world, local):
    import torch
    import paper_2606_16359_b300 as fe
    from paper_2606_16359_b300.net import MobileNetBlocks

    t_setup = time.perf_counter()
    ctx = fe.Context(**PARAMS)
    net = MobileNetBlocks(ctx, delta=DELTA, schedule=args.schedule, batch=args.batch)
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t_setup
    ks_per_step = net.keyswitches_per_step
    stream = torch.cuda.current_stream()
    if args.ncu_step:
        net.run(mode=1)
        torch.cuda.synchronize()
        ctx.reset_counters()
        torch.cuda.profiler.start()
        net.run(mode=1)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        print(json.dumps({"ncu_step": True, "launches": ctx.counters()["launches"]}), flush=True)
        return 0

    # correctness of one step against FP64 (untimed)
    net.run(mode=1)
    torch.cuda.synchronize()
    errs = [float(np.abs(net.decrypt_block(b, r) - net.reference_block(b, r)).max())
            for b in range(len(net.blocks)) for r in range(net.batch)]

    use_graph = not args.no_graph
    if use_graph:
        net.capture(concurrent=not args.one_stream)

    def step():
        # per-block streams run ahead across steps (each block's next step queues
        # behind its own previous one); the timed region joins them at its end
        if use_graph:
            net.launch(join=args.one_stream)
        else:
            net.run(mode=1)

    def join():
        if use_graph:
            net.join()

    for _ in range(args.warmup):
        step()
    join()
    torch.cuda.synchronize()
    barrier(dist)

    # ---- timed region: K steps, events on the launching stream ----
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        barrier(dist)
        ev0.record(stream)
        for _ in range(args.steps):
            step()
        join()
        ev1.record(stream)
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    if ctx.device_status():
        raise RuntimeError("a bounded device wait expired during the timed steps")
    ms = reduce_max(dist, ms)
    barrier(dist)
    ms_step = ms / args.steps
    value = world * ks_per_step * args.steps / (ms / 1e3)

    # ---- per-layer times (batched path, events around each layer) ----
    layer_ms = []
    for i in range(len(net.layers)):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        net.run_layer(i)
        torch.cuda.synchronize()
        e0.record(stream)
        net.run_layer(i)
        e1.record(stream)
        torch.cuda.synchronize()
        layer_ms.append(e0.elapsed_time(e1))

    # ---- dominant kernel class and its roofline (batched path, same workload) ----
    kinds = ["ntt", "bconv", "keyip", "combine", "mac", "rescale"]
    per_kind = {}
    for kd in kinds:
        ctx.profile_begin(kd)
        net.run(mode=1)
        t, n, b = ctx.profile_end()
        per_kind[kd] = (t, n, b)
    dom = max(per_kind, key=lambda k: per_kind[k][0]) if args.profile == "auto" else args.profile
    ctx.profile_begin(dom)
    for _ in range(args.steps):
        net.run(mode=1)
    t_dom, n_dom, b_dom = ctx.profile_end()
    peak, peak_kind = peaks()
    achieved = (b_dom / n_dom) / (t_dom / n_dom / 1e3) / 1e9 if n_dom else 0.0
    shares = {k: round(v[0] / sum(x[0] for x in per_kind.values()), 4) for k, v in per_kind.items()}
    # every class beside the dominant one: CUDA-event time over one step and its
    # algorithmic bytes per second against the measured HBM copy rate (the NTT
    # and base conversion are bound by the integer pipes, so their fraction is
    # low by construction; the bytes of the key inner product, lift and MAC
    # count operand re-reads that hit L2)
    by_class = {k: {"ms": round(t, 3), "launches": n, "algorithmic_GBps": round(b / (t / 1e3) / 1e9, 1) if t else 0.0,
                    "hbm_frac": round(b / (t / 1e3) / 1e9 / peak, 3) if t else 0.0}
                for k, (t, n, b) in per_kind.items()}
    roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_source": peak_kind, "traffic": None, "launches": n_dom,
                "avg_launch_us": 1e3 * t_dom / max(1, n_dom), "time_share": shares, "by_class": by_class}
    if dom == "mac":
        ratio = mac_traffic_ratio()
        roofline["traffic"] = ratio * (b_dom / n_dom) if ratio and n_dom else None
        roofline["traffic_unit"] = ("bytes per launch: ncu dram read + write over algorithmic bytes on a small "
                                    "pointwise layer (%s), times this launch's algorithmic bytes" % ratio)
    if dom == "ntt":
        # the 64-bit-word transform is bound by the integer pipes: butterflies per
        # second against the live butterfly-probe roof; HBM figures kept beside it
        bfly_peak = butterfly_roof(ctx, torch)
        limb_passes = b_dom / (8.0 * ctx.N)
        bfly = limb_passes * (ctx.N // 2) * (ctx.logN / 2)
        bfly_rate = bfly / (t_dom / 1e3) / 1e9
        tpl = ntt_traffic_per_limb_pass()
        roofline["traffic"] = tpl * limb_passes / n_dom if tpl else None
        roofline["traffic_unit"] = "bytes per launch (ncu dram read + write; algorithmic: %.0f)" % (b_dom / n_dom)
        issue_peak, n_sm, mhz = butterfly_issue_roof(torch)
        roofline.update({"bound": "alu", "achieved": bfly_rate, "peak": bfly_peak, "unit": "Gbutterfly/s",
                         "frac": bfly_rate / bfly_peak,
                         "peak_source": "measured in this run: the butterfly probe (the transform's own lazy Shoup "
                                        "butterflies on register-resident residues, one full wave of CTAs)",
                         "issue_limit_context": issue_peak,
                         "issue_limit_source": "derived, context only: %d SMs x 4 warp instructions per clock x "
                                               "%.0f MHz x 32 lanes / %.1f warp instructions per butterfly"
                                               % (n_sm, mhz, BUTTERFLY_WARP_INSTRUCTIONS),
                         "hbm_GBps": achieved, "hbm_peak_GBps": peak, "hbm_frac": achieved / peak,
                         "hbm_peak_source": peak_kind})

    # ---- plain per-op path (one launch per primitive per ciphertext) ----
    net.run(mode=0)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.plain_steps):
        net.run(mode=0)
    e1.record(stream)
    torch.cuda.synchronize()
    plain_ms = e0.elapsed_time(e1) / args.plain_steps
    # where the per-primitive path spends its time, by kernel class (CUDA events)
    plain_by_class = {}
    for kd in kinds:
        ctx.profile_begin(kd)
        net.run(mode=0)
        t, n, b = ctx.profile_end()
        plain_by_class[kd] = {"ms": round(t, 3), "launches": n, "algorithmic_GB": round(b / 1e9, 2)}

    # ---- the layers composed from single-ciphertext operations (mode 2): every
    # rotation its own key switch, one PMult per term, as a per-op HE library ----
    net.run(mode=2)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.plain_steps):
        net.run(mode=2)
    e1.record(stream)
    torch.cuda.synchronize()
    per_op_ms = e0.elapsed_time(e1) / args.plain_steps

    # ---- end to end through host buffers: H2D inputs, graph step, D2H outputs ----
    def e2e_run(out_level):
        h_in = [t.cpu().pin_memory() for t in net.inputs]
        if use_graph:
            h_out = net.host_outputs(out_level)
        else:
            h_out = [torch.empty(t.shape, dtype=t.dtype, pin_memory=True) for t in net.outputs]
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        for _ in range(args.steps):
            if use_graph:
                # each block's copies in its own stream, beside the other blocks' kernels
                net.launch(h_in, h_out, join=args.one_stream)
            else:
                for d, h in zip(net.inputs, h_in):
                    d.copy_(h, non_blocking=True)
                step()
                for h, d in zip(h_out, net.outputs):
                    h.copy_(d, non_blocking=True)
        join()
        b.record(stream)
        torch.cuda.synchronize()
        ms_ = reduce_max(dist, a.elapsed_time(b)) / args.steps
        return ms_, sum(t.numel() * 8 for t in h_in), sum(t.numel() * 8 for t in h_out), h_out

    # results leave the device modulus-switched to level 1 (the first two limbs of
    # every polynomial: an exact modulus drop, enough to decrypt at the scale)
    out_level = 1 if use_graph else None
    e2e_full_ms, _, d2h_full, _ = e2e_run(None)
    e2e_ms, h2d, d2h, h_out = e2e_run(out_level)
    e2e_value = world * ks_per_step / (e2e_ms / 1e3)
    if use_graph:
        # the level-1 results decrypt to the FP64 blocks like the full ones
        for b in range(len(net.blocks)):
            t = h_out[b].to("cuda")
            slots = ctx.decrypt(net.sk, t[:t.shape[0] // net.batch], out_level, net.delta)
            y = ctx.unpack(net.ref_inputs[b][3], slots).cpu().numpy()
            errs.append(float(np.abs(y - net.reference_block(b, 0)).max()))

    launches_step = None
    ctx.reset_counters()
    net.run(mode=1)
    torch.cuda.synchronize()
    cnt = ctx.counters()
    launches_step = cnt["launches"]

    config = {"workload": WORKLOAD, "blocks": net.blocks, "inputs_per_block": net.batch,
              "ms_per_input": ms_step / net.batch, "keyswitches_per_step": ks_per_step,
              "pmults_per_step": net.pmults_per_step, "rotation_keys": net.n_keys,
              "schedule": net.schedule, "tune_ms": net.tune_ms,
              "path": (("one graph, one stream" if args.one_stream else
                        f"graph per block x{len(net.graphs)} streams") if use_graph else "batched"),
              "e2e_path": ("fe_graph_launch_host per graph (host copies in, replay, host copies out)"
                           if use_graph else "torch copies around the batched layers"),
              "layer_ms": {l_["name"]: round(t, 3) for l_, t in zip(net.layers, layer_ms)},
              "plain_path_ms_per_step": plain_ms, "speedup_vs_plain": plain_ms / ms_step,
              "plain_path_by_class": plain_by_class,
              "batched_path_by_class": {k: {"ms": round(v[0], 3), "launches": v[1], "algorithmic_GB": round(v[2] / 1e9, 2)}
                                        for k, v in per_kind.items()},
              "per_op_library_ms_per_step": per_op_ms, "speedup_vs_per_op_library": per_op_ms / ms_step,
              "max_abs_err_vs_fp64": max(errs), "setup_s": round(t_setup, 1),
              "l2": "inputs (keys, plaintexts) far larger than L2; no flush",
              "parallelism": f"replicas x{world}"}

    # ---- variants (context for the headline, not separate bench lines): the whole
    # step as one graph on one stream, and B independent inputs per block ----
    variants = {}
    if use_graph and args.variants:
        def timed(net_, concurrent, steps, req_chunk=None):
            net_.capture(concurrent=concurrent, req_chunk=req_chunk)
            for _ in range(3):
                net_.launch(join=not concurrent)
            net_.join()
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(steps):
                net_.launch(join=not concurrent)
            net_.join()
            b.record(stream)
            torch.cuda.synchronize()
            if ctx.device_status():
                raise RuntimeError("a bounded device wait expired in a variant")
            t = a.elapsed_time(b) / steps
            return {"ms_per_step": round(t, 3), "keyswitches_per_step": net_.keyswitches_per_step,
                    "keyswitch_per_s": net_.keyswitches_per_step / (t / 1e3),
                    "ms_per_input": round(t / net_.batch, 3), "steps": steps, "warmup": 3}
        if not args.one_stream:
            variants["one_graph_one_stream"] = timed(net, False, args.steps)
        import gc
        schedule = net.schedule
        del net
        gc.collect()
        torch.cuda.empty_cache()
        for B in (4, 16):
            if B == args.batch:
                continue
            nb = MobileNetBlocks(ctx, delta=DELTA, schedule=schedule, batch=B)
            # the hoisted rotated copies of 16 inputs per block are tens of GB: their graphs
            # take the requests 4 at a time over one data region each
            req_chunk = None if B <= 4 else 4
            plans = [l_["plan"] for l_ in nb.layers]
            need = sum((ctx.graph_workspace_bytes(plans[2 * b:2 * b + 2], B) if req_chunk is None else
                        ctx.graph_workspace_bytes_chunked(plans[2 * b:2 * b + 2], B, req_chunk))
                       for b in range(len(nb.blocks)))
            free = torch.cuda.mem_get_info()[0]
            if need > free - (4 << 30):
                variants[f"batch_{B}"] = {"skipped": f"graph workspace {need / 1e9:.1f} GB, {free / 1e9:.1f} GB free"}
            else:
                variants[f"batch_{B}"] = dict(timed(nb, True, max(3, min(args.steps, 5)), req_chunk),
                                              path="graph per block, 3 streams" +
                                                   (f", requests {req_chunk} at a time" if req_chunk else ""))
            del nb, plans
            gc.collect()
            torch.cuda.empty_cache()

    # ---- the ciphertext refresh between blocks (bootstrapping), on its own
    # parameter set: N = 2^16, 24 primes of 50 bits, sparse secret of weight 64 ----
    refresh = None
    if args.refresh:
        import gc
        gc.collect()
        torch.cuda.empty_cache()
        refresh = refresh_bench(torch, stream, max(3, min(args.steps, 10)))
        refresh["small"] = {"ms": round(gpu_refresh_small(torch, stream), 3), "reps": 10, "warmup": 3,
                            "params": "N=2^10, 20 x 50-bit q, 4 x 50-bit p, h=32, default schedule",
                            "cpu_oracle": "cpu_baseline.refresh"}

    cpu = None
    if rank == 0 and args.cpu_rotations > 0:
        v1, dt1 = cpu_oracle_keyswitch(args.cpu_rotations)
        va, dta, workers, cores, model = cpu_oracle_all_cores(max(1, args.cpu_rotations // 2))
        cpu = {"value": va, "unit": "keyswitch/s", "cores": workers, "kind": "oracle",
               "sample": f"{max(1, args.cpu_rotations // 2)} oracle rotations of a level-22 ciphertext (the pointwise "
                         f"layers' level; N=2^16, 6 digits) in each of {workers} single-threaded processes, "
                         f"{dta:.1f} s wall",
               "cpu_model": model, "host_cores": cores,
               "single_thread": {"value": v1, "unit": "keyswitch/s", "cores": 1,
                                 "sample": f"{args.cpu_rotations} oracle rotations of one level-22 ciphertext, "
                                           f"{dt1:.1f} s"}}
        if args.refresh:
            t_ref = cpu_oracle_refresh()
            cpu["refresh"] = {"value": t_ref * 1e3, "unit": "ms per refresh", "cores": 1, "kind": "oracle",
                              "sample": "one refresh of one level-0 ciphertext at N=2^10 (20 x 50-bit q, 4 x 50-bit "
                                        "p, h=32, default schedule), single-threaded; the GPU's time on the same "
                                        "workload is config.refresh.small"}

    if rank == 0:
        clocks = clk.summary()
        line = {
            "metric": METRIC, "value": value, "unit": "keyswitch/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": dict(config, variants=variants, refresh=refresh),
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": "keyswitch/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms,
                    "results": ("output ciphertexts copied at level %s (exact modulus drop)" % out_level
                                if out_level is not None else "output ciphertexts at their own level"),
                    "full_level": {"ms_per_step": e2e_full_ms, "d2h_bytes_per_step": d2h_full}},
            "gpu_launches": launches_step * args.steps,
            "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
