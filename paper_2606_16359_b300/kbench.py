"""Kernel micro-benchmarks through the C ABI (one JSON line each).

    python -m paper_2606_16359_b300.kbench ntt [--logN 16] [--limbs 512] [--reps 10]
    python -m paper_2606_16359_b300.kbench alu [--iters 400]
    python -m paper_2606_16359_b300.kbench keyswitch [--n 8] [--level 22] [--reps 5]
    python -m paper_2606_16359_b300.kbench mac [--reps 5]
    python -m paper_2606_16359_b300.kbench layer [--channels 128] [--hw 14] [--dw] [--reps 5]
    python -m paper_2606_16359_b300.kbench aac [--reps 5]
    python -m paper_2606_16359_b300.kbench configs [--reps 5]
    python -m paper_2606_16359_b300.kbench repack
    python -m paper_2606_16359_b300.kbench refresh [--reps 5] [--graph 1]
    python -m paper_2606_16359_b300.kbench transformer [--tokens 128] [--embed 768] [--reps 3]

ntt: forward and inverse negacyclic NTT over a batch of limbs of the 36-bit
     moduli (N = 2^logN); algorithmic bytes 2 N w per limb transform (read and
     write each word once), butterflies (N / 2) log2 N per limb.
alu: the integer-pipe roof of the transform's butterfly arithmetic, from a
     register-resident probe of the same lazy Shoup butterflies.
refresh: one ciphertext refresh (bootstrapping) at N = 2^16 with 24 + 4 primes of
     50 bits and a secret of weight 64, timed over --reps refreshes; the last
     refresh is bracketed by two one-block butterfly-probe launches, markers for
     a profiler's launch list.  --graph 1 captures the refresh in one CUDA
     graph (fe_boot_graph_capture; checked equal to the direct call) and times
     its replays.
transformer: the Sec. 7 extension at BERT-base shapes (a projection, the
     attention products, an FFN), N = 2^16 with the convolution parameters.
keyswitch: rotations (hybrid key switch + automorphism) of n ciphertexts at one
     level with one key; algorithmic bytes per key switch without key reuse
     [(l+1) + 2 dnum (l+1+k) + 2 (l+1)] N w.

Inputs are larger than L2 (126 MB) unless stated; times are CUDA events on the
launching stream after warm-up.  Used for the ncu captures of single kernels,
which need a small, self-contained case.
"""
import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def hbm_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


def _events(torch):
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def bench_ntt(ctx, torch, args):
    ctx.set_ntt_radix(args.radix)
    ctx.set_ntt_q36(args.q36)
    ctx.set_ntt_path(args.path)
    ctx.set_ntt_forward(args.fwd)
    N, nm = ctx.N, ctx.n_mod
    n_poly = max(1, (args.limbs + nm - 1) // nm)
    limbs = n_poly * nm
    # residues below 2^(bits - 1) are valid for every modulus of `bits` bits
    d = torch.randint(0, 2 ** (args.qbits - 1), (n_poly, nm, N), dtype=torch.int64, device="cuda")
    out = {}
    for inv in (False, True):
        for _ in range(2):
            ctx.ntt(d, inverse=inv)
        torch.cuda.synchronize()
        e0, e1 = _events(torch)
        e0.record()
        for _ in range(args.reps):
            ctx.ntt(d, inverse=inv)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.reps
        us_limb = 1e3 * ms / limbs
        gbs = 2 * N * 8 * limbs / (ms / 1e3) / 1e9
        bfly = (N // 2) * ctx.logN * limbs / (ms / 1e3)
        out["inverse" if inv else "forward"] = {"ms": ms, "us_per_limb": us_limb, "GBps": gbs,
                                                "Gbutterfly_per_s": bfly / 1e9}
    peak, src = hbm_peak()
    for v in out.values():
        v["hbm_frac"] = v["GBps"] / peak
    return {"kernel": "ntt", "qbits": args.qbits, "radix": args.radix, "q36": args.q36, "path": args.path, "fwd": args.fwd, "logN": ctx.logN, "limbs": limbs, "bytes_in": limbs * N * 8,
            "peak_GBps": peak, "peak_source": src, **out}


def bench_alu(ctx, torch, args):
    ctx.set_ntt_q36(args.q36)
    n_sm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    buf = torch.empty(n_sm * 8 * 256, dtype=torch.int64, device="cuda")
    ctx.probe_butterflies(buf, 0, max(1, args.iters // 10))
    torch.cuda.synchronize()
    e0, e1 = _events(torch)
    e0.record()
    n = ctx.probe_butterflies(buf, 0, args.iters)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    return {"kernel": "butterfly_probe", "q36": args.q36, "blocks": n // (256 * 60 * args.iters), "threads": 256,
            "iters": args.iters, "butterflies": n, "ms": ms, "Gbutterfly_per_s": n / (ms / 1e3) / 1e9}


def bench_keyswitch(ctx, torch, args):
    lv = args.level
    sk = ctx.sk_gen(1)
    evk = ctx.evk_gen(sk, 1, [1])
    slots = torch.zeros((args.n, ctx.N // 2), dtype=torch.float64, device="cuda")
    ct = ctx.encrypt(sk, slots, lv, 2.0 ** 32, 3)
    for _ in range(2):
        ctx.rotate(evk, ct, lv, 1)
    torch.cuda.synchronize()
    e0, e1 = _events(torch)
    e0.record()
    for _ in range(args.reps):
        ctx.rotate(evk, ct, lv, 1)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.reps
    k, N = ctx.k, ctx.N
    dnum = (lv + 1 + k - 1) // k
    per_ks = ((lv + 1) + 2 * dnum * (lv + 1 + k) + 2 * (lv + 1)) * N * 8
    peak, src = hbm_peak()
    us = 1e3 * ms / args.n
    return {"kernel": "keyswitch", "level": lv, "n_ct": args.n, "dnum": dnum, "ms": ms, "us_per_keyswitch": us,
            "keyswitch_per_s": 1e6 / us, "bytes_per_keyswitch_no_reuse": per_ks,
            "GBps_no_reuse": per_ks / (us / 1e6) / 1e9, "hbm_frac_no_reuse": per_ks / (us / 1e6) / 1e9 / peak,
            "peak_GBps": peak, "peak_source": src}


def bench_mac(ctx, torch, args):
    """The pointwise layer of the 14x14x512 -> 512 block (cpc = 128, 4 input and
    4 output ciphertexts, level 22) with baby-step / giant-step n1 = 16, run in
    timing mode (plaintexts from a pool of 48, keys aliased, smallest
    workspace); reports the MAC launches' time and their plaintext and
    ciphertext bytes."""
    from paper_2606_16359_b300.tune import Tuner
    lv = ctx.L - 1
    t = Tuner(ctx, n_keys=4, n_pts=48)
    lay = ctx.layout(14, 14, 512, 1, 1)
    plan = ctx.plan_conv(lay, 512, 1, level=lv, bsgs_n1=16)
    i = plan.info
    ctx.evk_alias(t.evk, plan.steps)
    x = torch.randint(0, 2 ** 35, (i.n_in_ct, 2, lv + 1, ctx.N), dtype=torch.int64, device="cuda")
    out = ctx.empty_ct(i.n_out_ct, lv - 1)
    ws = ctx.workspace(ctx.workspace_bytes(plan, 1, minimum=True))
    for _ in range(2):
        ctx.he_layer_timing(t.evk, plan, t.pts, t.n_pool, x, out, ws)
    ctx.profile_begin("mac")
    for _ in range(args.reps):
        ctx.he_layer_timing(t.evk, plan, t.pts, t.n_pool, x, out, ws)
    ms, n, b = ctx.profile_end()
    peak, src = hbm_peak()
    pt_bytes = i.pt_bytes * args.reps
    return {"kernel": "mac", "level": lv, "n_pt": i.n_pt, "launches": n, "ms": ms / args.reps,
            "pt_GBps": pt_bytes / (ms / 1e3) / 1e9, "algorithmic_GBps": b / (ms / 1e3) / 1e9,
            "hbm_frac": b / (ms / 1e3) / 1e9 / peak, "peak_GBps": peak, "peak_source": src,
            "status": ctx.device_status()}


def bench_layer(ctx, torch, args):
    """One real layer on resident operands (no pool, no aliasing) at level 22,
    N = 2^16, double hoisting (fused ModDown and rescale where it applies),
    real keys and encoded weights: pointwise
    HxHxC -> C with baby-step / giant-step n1 = 16, or with --dw the depthwise
    3x3 conv HxHxC (H = --hw, C = --channels; the defaults keep every operand a
    few GB, larger than L2).  For ncu captures of the MAC, key inner product,
    base conversion and lift kernels with DRAM traffic as in the bench step.
    Reports the layer's CUDA-event time and the per-kernel-class times and
    algorithmic bytes."""
    import numpy as np
    lv = ctx.L - 1
    C, H = args.channels, args.hw
    lay = ctx.layout(H, H, C, 1, 1)
    if args.dw:
        plan = ctx.plan_conv(lay, C, 3, depthwise=True, level=lv, double_hoist=2)
        w = np.random.default_rng(0).normal(0, 1 / 3, (C, 1, 3, 3))
    else:
        plan = ctx.plan_conv(lay, C, 1, level=lv, bsgs_n1=16, double_hoist=2)
        w = np.random.default_rng(0).normal(0, 1 / np.sqrt(C), (C, C, 1, 1))
    i = plan.info
    sk = ctx.sk_gen(5)
    evk = ctx.evk_gen(sk, 5, plan.steps)
    pt = ctx.load_weights(plan, w, float(ctx.moduli[lv]))
    x = ctx.encrypt(sk, ctx.pack(lay, torch.from_numpy(np.random.default_rng(1).uniform(-1, 1, (1, C, H, H)))),
                    lv, 2.0 ** 32, seed=3)
    out = ctx.empty_ct(i.n_out_ct, lv - 1)
    ws = ctx.workspace(i.workspace_bytes)
    for _ in range(2):
        ctx.he_conv(evk, plan, pt, x, ws=ws, out=out)
    torch.cuda.synchronize()
    e0, e1 = _events(torch)
    e0.record()
    for _ in range(args.reps):
        ctx.he_conv(evk, plan, pt, x, ws=ws, out=out)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.reps
    kinds = {}
    for kind in ("mac", "keyip", "bconv", "ntt", "combine"):
        ctx.profile_begin(kind)
        ctx.he_conv(evk, plan, pt, x, ws=ws, out=out)
        kms, n, b = ctx.profile_end()
        kinds[kind] = {"ms": kms, "launches": n, "GB": b / 1e9, "GBps": b / (kms / 1e3) / 1e9 if kms else 0.0}
    return {"kernel": "layer", "depthwise": bool(args.dw), "hw": H, "channels": C, "level": lv, "n_pt": i.n_pt, "pt_GB": i.pt_bytes / 1e9,
            "n_inner_rot": i.n_inner_rot, "n_outer_rot": i.n_outer_rot, "ms": ms, "kinds": kinds,
            "status": ctx.device_status()}


def bench_aac(ctx, torch, args):
    """Arch-aware Ciphertext Compression on the residual-shortcut shapes of
    Table 7 (8 valid channels after a channel-reducing layer, N = 2^16, level
    22): the compression (log2(cpc / 8) rotate-and-adds per ciphertext) against
    the next 1x1 conv 8 -> Nout with the replicated input (8 diagonals) and
    without compression (every diagonal of the sparse input).  The convs run
    in timing mode (plaintext pool, aliased keys); the compression with real
    keys.  Overhead = compression / (compression + conv with AAC)."""
    from paper_2606_16359_b300.tune import Tuner
    lv = ctx.L - 1
    t = Tuner(ctx, n_keys=4, n_pts=32)
    sk = ctx.sk_gen(3)
    rows = []
    for nin, nout, H in ((64, 128, 56), (128, 256, 28), (256, 512, 14), (512, 512, 7)):
        lay = ctx.layout(H, H, 8, 1, 1)
        cpc = lay.cpc
        steps = []
        s = 8
        while s < cpc:
            steps.append(-s * lay.m * lay.m * lay.BS)
            s *= 2
        evk = ctx.evk_gen(sk, 3, steps) if steps else None
        ct = torch.randint(0, 2 ** 35, (lay.n_ct, 2, lv + 1, ctx.N), dtype=torch.int64, device="cuda")
        t_cmp = 0.0
        if evk is not None:
            ctx.compress(evk, lay, 8, ct, lv)
            torch.cuda.synchronize()
            e0, e1 = _events(torch)
            e0.record()
            for _ in range(args.reps):
                ctx.compress(evk, lay, 8, ct, lv)
            e1.record()
            torch.cuda.synchronize()
            t_cmp = e0.elapsed_time(e1) / args.reps
        p_aac = ctx.plan_conv(lay, nout, 1, level=lv, in_period=8 if cpc > 8 else 0)
        p_raw = ctx.plan_conv(lay, nout, 1, level=lv)
        t_aac = t.time_plan(p_aac, args.reps)
        t_raw = t.time_plan(p_raw, args.reps)
        rows.append({"shape": [nin, 8, nout, H], "cpc": cpc, "util_without": min(1.0, 8 / cpc), "util_with": 1.0,
                     "compress_ms": t_cmp, "conv_with_aac_ms": t_aac, "conv_without_ms": t_raw,
                     "outer_rot_with": p_aac.info.n_outer_rot, "outer_rot_without": p_raw.info.n_outer_rot,
                     "overhead_pct": 100 * t_cmp / max(1e-9, t_cmp + t_aac),
                     "speedup": t_raw / max(1e-9, t_cmp + t_aac)})
    return {"kernel": "aac", "level": lv, "rows": rows, "status": ctx.device_status()}


def bench_repack(ctx, torch, args):
    """Cost of running each MobileNet-shaped block's depthwise layer at S = 2 and
    its pointwise layer at S = 1 (N = 2^16, level 23): the rotations the
    depthwise layer saves at S = 2, against the rotations, masks and mask bytes
    of the S = 2 -> 1 re-encoding between the layers (plans only; nothing is
    encoded or run at this size)."""
    import workloads as W
    out = []
    L = ctx.L
    for H, Cin, Cout in W.MOBILENET_BLOCKS:
        row = {"block": [H, Cin, Cout]}
        for S in (1, 2):
            lay = ctx.layout(H, H, Cin, 1, S)
            pdw = ctx.plan_conv(lay, Cin, 3, depthwise=True, level=L)
            row[f"dw_S{S}_rotations"] = pdw.info.n_inner_rot
            if S == 2:
                lo = pdw.out_layout
                tgt = ctx.layout(lo.H, lo.W, Cin, 1, 1)
                prp = ctx.plan_repack(lo, tgt, L - 1)
                i = prp.info
                row.update(repack_rotations=i.n_inner_rot + i.n_outer_rot, repack_masks=i.n_pt,
                           repack_mask_GB=round(i.pt_bytes / 1e9, 1), repack_bsgs_n1=i.bsgs_n1)
        row["rotations_saved_by_S2"] = row["dw_S1_rotations"] - row["dw_S2_rotations"]
        out.append(row)
    return {"kernel": "repack_plans", "logN": ctx.logN, "level": L, "blocks": out}


def bench_transformer(ctx, torch, args):
    """The transformer extension (Sec. 7) at N = 2^16, 24 + 4 primes of --qbits
    bits (36: the convolution parameters; 50: the refresh's), scale
    2^(qbits - 4), BERT-base shapes: n = 128
    tokens, E = 768, S from fe_choose_token_fragment (gamma = 6).  Timed (CUDA
    events, one warm-up, --reps runs): a projection E -> E; the attention
    products Q K^T (its n diagonals) and (Q K^T) V with token-wise rotations;
    an FFN E' -> 4 E' -> E' with 0.125 x^2 + 0.5 x + 0.25 between, E' = 256,
    the widest whose hidden layer fits the P = N / (2 n) positions at the same
    S; --hoist 1 runs the linear layers double-hoisted.  Inputs U[-1, 1) (Q
    and K scaled by E^(-1/4) / 2.3 and V by 1/4, so
    that every product stays near unit size); weights N(0, 1 / fan_in).
    Reports ms, key switches and the decryption's max error against FP64."""
    import numpy as np

    import paper_2606_16359_b300 as fe
    n, E, gam, Ef = args.tokens, args.embed, 6.0, 256
    S = fe.choose_token_fragment(E, n, gam)["S"]
    L, delta = ctx.L, 2.0 ** (args.qbits - 4)
    a, b, c = 0.125, 0.5, 0.25
    rng = np.random.default_rng(21)
    lay = ctx.token_layout(n, E, S)
    lay_f = ctx.token_layout(n, Ef, S)
    p_proj = ctx.plan_token_linear(lay, E, L)
    p_f1 = ctx.plan_token_linear(lay_f, 4 * Ef, L)
    p_f2 = ctx.plan_token_linear(p_f1.token_out, Ef, L - 2)
    for p in (p_proj, p_f1, p_f2):
        ctx.plan_set_hoisting(p, args.hoist)
    steps = sorted(set(ctx.attention_rotation_steps(lay)) |
                   {s for p in (p_proj, p_f1, p_f2) for s in p.steps})
    sk = ctx.sk_gen(5)
    evk = ctx.evk_gen(sk, 5, steps, relin=True)
    x = rng.uniform(-1, 1, (n, E))
    wp = rng.normal(0, 1 / np.sqrt(E), (E, E))
    qa = E ** -0.25 / 2.3
    Q, K = (rng.uniform(-qa, qa, (n, E)) for _ in range(2))
    V = rng.uniform(-0.25, 0.25, (n, E))
    xf = rng.uniform(-1, 1, (n, Ef))
    w1 = rng.normal(0, 1 / np.sqrt(Ef), (4 * Ef, Ef))
    w2 = rng.normal(0, 1 / np.sqrt(4 * Ef), (Ef, 4 * Ef))
    enc = lambda X, ly, sd: ctx.encrypt(sk, ctx.token_pack(ly, torch.from_numpy(X)), L, delta, sd)  # noqa: E731
    ct_x, ct_q, ct_k, ct_v, ct_f = enc(x, lay, 1), enc(Q, lay, 2), enc(K, lay, 3), enc(V, lay, 4), enc(xf, lay_f, 6)
    pt_p = ctx.load_weights(p_proj, wp, ctx.weight_scale(L, delta, delta))
    pt_1 = ctx.load_weights(p_f1, w1, ctx.weight_scale(L, delta, delta, a))
    s1 = ctx.plan_out_scale(p_f1, delta)
    s_act = ctx.poly_act_scale(L - 1, s1, a)
    pt_2 = ctx.load_weights(p_f2, w2, ctx.weight_scale(L - 2, s_act, delta))

    def projection():
        return ctx.he_fc(evk, p_proj, pt_p, ct_x)

    def attention():
        D, d_scale = ctx.he_attention_scores(evk, lay, ct_q, ct_k, L, delta, delta)
        return ctx.he_attention_apply(evk, lay, D, L - 2, d_scale, ct_v, L, delta)

    def ffn():
        h = ctx.he_fc(evk, p_f1, pt_1, ct_f)
        h, _ = ctx.he_poly_act(evk, h, L - 1, s1, a, b, c)
        return ctx.he_fc(evk, p_f2, pt_2, h)

    def timed(fn):
        r = fn()
        torch.cuda.synchronize()
        ctx.reset_counters()
        fn()
        torch.cuda.synchronize()
        ks = ctx.counters()["keyswitch"]
        st = torch.cuda.current_stream()
        t0, t1 = _events(torch)
        t0.record(st)
        for _ in range(args.reps):
            fn()
        t1.record(st)
        torch.cuda.synchronize()
        return r, t0.elapsed_time(t1) / args.reps, ks

    res = {"what": "transformer", "logN": ctx.logN, "qbits": args.qbits, "scale_log2": args.qbits - 4,
           "linear_hoisting": args.hoist,
           "level": L, "tokens": n, "embed": E, "S": S,
           "rotation_keys": len(steps), "evk_gb": round(evk.buf.numel() * 8 / 1e9, 1), "reps": args.reps}
    out, ms, ks = timed(projection)
    y = ctx.token_unpack(p_proj.token_out, ctx.decrypt(sk, out, L - 1, ctx.plan_out_scale(p_proj, delta)))
    res["projection"] = {"ms": ms, "keyswitches": ks,
                         "max_abs_err": float(np.abs(y.cpu().numpy() - x @ wp.T).max())}
    (O, o_level, o_scale), ms, ks = timed(attention)
    y = ctx.token_unpack(lay, ctx.decrypt(sk, O, o_level, o_scale))
    res["attention"] = {"ms": ms, "keyswitches": ks, "out_level": o_level,
                        "max_abs_err": float(np.abs(y.cpu().numpy() - (Q @ K.T) @ V).max())}
    if args.classes:
        # CUDA-event time of each kernel class over one attention call (one call per class)
        by = {}
        for kd in ("ntt", "bconv", "keyip", "combine", "mac", "rescale", "encode"):
            ctx.profile_begin(kd)
            attention()
            t, nl, byt = ctx.profile_end()
            by[kd] = {"ms": round(t, 2), "launches": nl}
        res["attention"]["by_class"] = by
    out, ms, ks = timed(ffn)
    y = ctx.token_unpack(p_f2.token_out, ctx.decrypt(sk, out, L - 3, ctx.plan_out_scale(p_f2, s_act)))
    t = xf @ w1.T
    res["ffn"] = {"embed": Ef, "hidden": 4 * Ef, "ms": ms, "keyswitches": ks,
                  "max_abs_err": float(np.abs(y.cpu().numpy() - (a * t * t + b * t + c) @ w2.T).max())}
    assert ctx.device_status() == 0
    return res


def bench_configs(ctx_unused, torch, args):
    """The two small configurations end to end on the GPU: the single 5x5 conv
    1 -> 6 at N = 2^13 (S = 4) and the LeNet-shaped network at N = 2^14
    (128 images), batched and per-op paths, with the max error against FP64."""
    import numpy as np
    import workloads as W
    from paper_2606_16359_b300 import plainref
    from paper_2606_16359_b300.net import LeNet
    import paper_2606_16359_b300 as fe

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        e0, e1 = _events(torch)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    out = {"kernel": "configs"}
    p = W.PARAMS["conv1"]
    c1 = fe.Context(p["logN"], p["n_q"], p["k"], p["bits"], p["pbits"])
    x, w = W.conv1_workload(0)
    lay = c1.layout(28, 28, 1, 1, 4)
    plan = c1.plan_conv(lay, 6, 5, level=c1.L)
    sk = c1.sk_gen(1)
    evk = c1.evk_gen(sk, 1, plan.steps)
    ct = c1.encrypt(sk, c1.pack(lay, torch.from_numpy(x)), c1.L, p["delta"], 2)
    pt = c1.load_weights(plan, w, float(c1.moduli[c1.L]))
    ws = c1.workspace(plan.info.workspace_bytes)
    res = {}
    for mode in (1, 0):
        res[mode] = timed(lambda: c1.he_conv(evk, plan, pt, ct, mode=mode, ws=ws), args.reps)
    y = c1.unpack(plan.out_layout, c1.decrypt(sk, c1.he_conv(evk, plan, pt, ct, ws=ws), c1.L - 1, p["delta"]))
    out["conv1"] = {"batched_ms": res[1], "per_op_ms": res[0], "rotations": plan.info.n_inner_rot + plan.info.n_outer_rot,
                    "pmults": plan.info.n_pt, "max_abs_err": float(np.abs(y.cpu().numpy() - plainref.conv2d(x, w)).max())}
    p = W.PARAMS["lenet"]
    c2 = fe.Context(p["logN"], p["n_q"], p["k"], p["bits"], p["pbits"])
    wts = W.lenet_weights(0)
    net = LeNet(c2, p["delta"], wts)
    xs = W.lenet_input(0, net.BS)
    ct2 = net.encrypt(xs)
    for mode in (1, 0):
        res[mode] = timed(lambda: net.forward(ct2, mode=mode), args.reps)
    yl = net.decode_logits(net.forward(ct2))
    out["lenet"] = {"images": net.BS, "batched_ms": res[1], "per_op_ms": res[0], "ms_per_image": res[1] / net.BS,
                    "max_abs_err": float(np.abs(yl - plainref.lenet(xs, wts)).max())}
    out["status"] = c1.device_status() | c2.device_status()
    return out


def bench_refresh(ctx_unused, torch, args):
    import numpy as np

    import paper_2606_16359_b300 as fe
    ctx = fe.Context(16, 24, 4, 50)
    sk = ctx.sk_gen_sparse(31, 64)
    s_in = 2.0 ** 45
    b = ctx.boot_create(s_in, args.n_cts, args.n_stc, args.double_angles, baby_ratio=args.baby_ratio,
                        double_hoist=args.double_hoist, form=args.form)
    evk = ctx.evk_gen(sk, 31, b.steps, relin=True)
    z = np.random.default_rng(9).uniform(-1, 1, (args.n_ct, ctx.N // 2))
    ct = ctx.encrypt(sk, z, 0, s_in, seed=10)
    ws = ctx.workspace(b.workspace_bytes(args.n_ct))
    out = ctx.bootstrap(evk, b, ct, ws=ws)
    for _ in range(2):
        ctx.bootstrap(evk, b, ct, ws=ws, out=out)
    torch.cuda.synchronize()
    run = lambda: ctx.bootstrap(evk, b, ct, ws=ws, out=out)  # noqa: E731
    if args.graph:
        # one graph of the whole refresh (fe_boot_graph_capture: item tables
        # uploaded first, launches captured), checked against the direct call
        want = out.clone()
        g = ctx.boot_graph_capture(evk, b, ct, out, ws)
        out.zero_()
        g.launch()
        torch.cuda.synchronize()
        if not torch.equal(out, want):
            raise RuntimeError("the replayed refresh differs from the direct call")
        run = g.launch
    st = torch.cuda.current_stream()
    a, e = _events(torch)
    a.record(st)
    for _ in range(args.reps):
        run()
    e.record(st)
    torch.cuda.synchronize()
    ms = a.elapsed_time(e) / args.reps
    probe = torch.empty(256, dtype=torch.int64, device="cuda")
    ctx.probe_butterflies(probe, 1, 1)
    ctx.reset_counters()
    ctx.bootstrap(evk, b, ct, ws=ws, out=out)
    cnt = ctx.counters()
    ctx.probe_butterflies(probe, 1, 1)
    torch.cuda.synchronize()
    err = float(np.abs(ctx.decrypt(sk, out, b.out_level, b.out_scale).cpu().numpy() - z).max())
    return {"what": "refresh", "form": args.form, "graph": bool(args.graph), "n_ct": args.n_ct, "ms_per_ct": ms / args.n_ct,
            "groups": [args.n_cts, args.n_stc], "double_angles": args.double_angles,
            "levels_used": 23 - b.out_level, "baby_ratio": args.baby_ratio, "double_hoist": args.double_hoist, "ms": ms, "reps": args.reps,
            "out_level": b.out_level, "max_abs_err": err, "rotation_keys": len(b.steps),
            "evk_gb": evk.buf.numel() * 8 / 1e9, "counters_per_refresh": cnt}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("what", choices=["ntt", "alu", "keyswitch", "mac", "layer", "aac", "configs", "repack",
                                     "refresh", "transformer"])
    ap.add_argument("--tokens", type=int, default=128, help="transformer: tokens n")
    ap.add_argument("--embed", type=int, default=768, help="transformer: embedding dimension E")
    ap.add_argument("--classes", type=int, default=0, help="transformer: 1 adds the attention's time by kernel class")
    ap.add_argument("--hoist", type=int, default=0,
                    help="transformer: hoisting of the linear layers (0 single, 1 double: baby rotations on Q P)")
    ap.add_argument("--logN", type=int, default=16)
    ap.add_argument("--qbits", type=int, default=36,
                    help="modulus bits of the 24 + 4 primes (36: the convolution parameters; 50: the refresh's)")
    ap.add_argument("--limbs", type=int, default=512)
    ap.add_argument("--reps", type=int, default=10)
    ap.add_argument("--iters", type=int, default=400)
    ap.add_argument("--n", type=int, default=8)
    ap.add_argument("--level", type=int, default=22)
    ap.add_argument("--radix", type=int, default=8, help="NTT elements per thread per round (8 or 16)")
    ap.add_argument("--fwd", type=int, default=0, help="forward NTT form flags: 1 reduce every stage, 2 36-bit Shoup product")
    ap.add_argument("--path", type=int, default=0, help="NTT data path: 0 two passes direct (default), 1 two passes staged, 2 one pass on 8-CTA clusters (N = 2^16)")
    ap.add_argument("--q36", type=int, default=1, help="36-bit Shoup product in the inverse NTT (1, default), nowhere (0), or also in the probe (2)")
    ap.add_argument("--channels", type=int, default=128, help="channels of the layer case")
    ap.add_argument("--hw", type=int, default=14, help="map height = width of the layer case")
    ap.add_argument("--dw", action="store_true", help="layer case: depthwise 3x3 instead of pointwise")
    ap.add_argument("--baby-ratio", type=int, default=4, help="refresh: baby-step rule of the stage groups")
    ap.add_argument("--double-hoist", type=int, default=1, help="refresh: 1 keeps the groups' baby rotations on Q P")
    ap.add_argument("--n-cts", type=int, default=3, help="refresh: CoeffToSlot stage groups (levels)")
    ap.add_argument("--n-stc", type=int, default=3, help="refresh: SlotToCoeff stage groups (levels)")
    ap.add_argument("--double-angles", type=int, default=6, help="refresh: EvalMod double angles")
    ap.add_argument("--n-ct", type=int, default=1, help="refresh: ciphertexts refreshed in one call")
    ap.add_argument("--form", default="complex", choices=["real", "complex"], help="refresh: transform form")
    ap.add_argument("--graph", type=int, default=0, help="refresh: 1 times replays of one captured graph")
    args = ap.parse_args(argv)
    import torch

    sys.path.insert(0, ROOT)
    import paper_2606_16359_b300 as fe

    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        ctx = fe.Context(args.logN, 24, 4, args.qbits, args.qbits)
        fn = {"ntt": bench_ntt, "alu": bench_alu, "keyswitch": bench_keyswitch, "mac": bench_mac,
              "layer": bench_layer, "aac": bench_aac, "configs": bench_configs,
              "repack": bench_repack, "refresh": bench_refresh, "transformer": bench_transformer}[args.what]
        print(json.dumps(fn(ctx, torch, args)), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
