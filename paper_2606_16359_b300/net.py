"""Multi-layer encrypted workloads assembled from the C-ABI layers.

MobileNetBlocks: three depthwise-3x3 + pointwise blocks under the fragment
encoding at S = 1 (the largest maps need S = 1 to fit a ciphertext), each
block an independent encrypted input.  All layers' ciphertexts, plaintexts and
keys stay resident on the device; a step runs the six HE convolutions.

RefreshChain: two such blocks with the activation after each convolution and
a ciphertext refresh (bootstrapping) between them, at the refresh's parameters.

LeNet: conv5x5 1->6, x^2, avgpool2, conv5x5 6->16, x^2, avgpool2, FC 256->120->84->10
at the largest slot batch (Sec. 5, Implementation paragraph: x^2 activation,
pooling by fragment sums, FC by diagonals with baby-step / giant-step).
"""
import numpy as np

import workloads as W

from . import Context, FeLayout  # noqa: F401


def _torch():
    import torch
    return torch


class MobileNetBlocks:
    """schedule: "linear" (one outer rotation per channel diagonal, Eq. 4),
    "tuned" (per layer, the fastest outer-rotation split, hoisting and MAC tile
    timed by the autotuner), an int n1 (baby steps), or the list of per-block
    schedule dicts a tuned instance reports in `.schedule` (reused without
    tuning again).  batch: independent encrypted inputs per block, run
    together (keys shared across them)."""

    def __init__(self, ctx, blocks=None, seed=0, delta=2.0 ** 32, key_seed=101, enc_seed=202, schedule="linear",
                 batch=1):
        torch = _torch()
        self.ctx = ctx
        self.delta = delta
        self.blocks = list(W.MOBILENET_BLOCKS if blocks is None else blocks)
        L = ctx.L
        self.layers = []  # dicts: plan, pt, inp, out, level
        self.inputs, self.ref_inputs = [], []
        self.schedule, self.tune_ms = [], []
        self.batch = B = int(batch)
        tuner = None
        if schedule == "tuned":
            from .tune import Tuner
            tuner = Tuner(ctx)
        plans = []
        given = schedule if isinstance(schedule, (list, tuple)) else None
        for bi, (H, Cin, Cout) in enumerate(self.blocks):
            x, wd, wp = W.mobilenet_block(seed, H, Cin, Cout, BS=1, block=bi)
            lay = ctx.layout(H, H, Cin, 1, 1)
            dh_dw, dh_pw = False, False
            if tuner is not None:
                _, dh_dw, t_dw = tuner.conv_schedule(lay, Cin, 3, depthwise=True, level=L)
            elif given is not None:
                dh_dw = given[bi]["dw_double_hoist"]
            pdw = ctx.plan_conv(lay, Cin, 3, depthwise=True, level=L, double_hoist=dh_dw)
            if tuner is not None:
                n1, dh_pw, times = tuner.conv_schedule(pdw.out_layout, Cout, 1, level=L - 1)
                self.tune_ms.append({"dw": {k: round(v, 3) for k, v in t_dw.items()},
                                     "pw": {k: round(v, 3) for k, v in times.items()}})
            elif given is not None:
                n1, dh_pw = given[bi]["pw_bsgs_n1"], given[bi]["pw_double_hoist"]
            elif schedule == "linear":
                n1 = 0
            else:
                n1 = int(schedule)
            ppw = ctx.plan_conv(pdw.out_layout, Cout, 1, level=L - 1, bsgs_n1=n1, double_hoist=dh_pw)
            if tuner is not None:
                ways, wt = tuner.mac_ways(ppw)
                self.tune_ms[-1]["pw_mac_ways"] = {str(k): round(v, 3) for k, v in wt.items()}
            elif given is not None:
                ctx.plan_set_mac_ways(ppw, given[bi]["pw_mac_ways"])
            self.schedule.append({"dw_double_hoist": int(dh_dw), "pw_bsgs_n1": ppw.info.bsgs_n1,
                                  "pw_double_hoist": int(dh_pw), "pw_mac_ways": getattr(ppw, "mac_ways", 4)})
            plans.append((lay, pdw, ppw, x, wd, wp))
        del tuner
        steps = sorted({s for _, a, b, *_ in plans for s in a.steps + b.steps})
        self.sk = ctx.sk_gen(key_seed)
        self.evk = ctx.evk_gen(self.sk, key_seed, steps)
        self.n_keys = len(steps)
        ct_id = 0
        for bi, (lay, pdw, ppw, x, wd, wp) in enumerate(plans):
            xs = [x] + [W.mobilenet_block(seed + 1000 * b, *self.blocks[bi], BS=1, block=bi)[0] for b in range(1, B)]
            cts = []
            for xb in xs:
                slots = ctx.pack(lay, torch.from_numpy(xb))
                cts.append(ctx.encrypt(self.sk, slots, L, delta, enc_seed, ct_id0=ct_id))
                ct_id += lay.n_ct
            ct = torch.cat(cts, 0).contiguous() if B > 1 else cts[0]
            pt_dw = ctx.load_weights(pdw, wd, float(ctx.moduli[L]))
            pt_pw = ctx.load_weights(ppw, wp, float(ctx.moduli[L - 1]))
            mid = ctx.empty_ct(B * pdw.info.n_out_ct, L - 1)
            out = ctx.empty_ct(B * ppw.info.n_out_ct, L - 2)
            self.layers.append(dict(plan=pdw, pt=pt_dw, inp=ct, out=mid, level=L, name=f"b{bi}_dw"))
            self.layers.append(dict(plan=ppw, pt=pt_pw, inp=mid, out=out, level=L - 1, name=f"b{bi}_pw"))
            self.inputs.append(ct)
            self.ref_inputs.append((xs, wd, wp, ppw.out_layout))
        self.outputs = [self.layers[2 * i + 1]["out"] for i in range(len(self.blocks))]
        self.ws_bytes = max(ctx.workspace_bytes(l_["plan"], B) for l_ in self.layers)
        self._ws = None  # the eager path's workspace, allocated on first use (graphs bring their own)
        self.graph = None

    @property
    def ws(self):
        if self._ws is None:
            self._ws = self.ctx.workspace(self.ws_bytes)
        return self._ws

    @property
    def keyswitches_per_step(self):
        return self.batch * sum(l_["plan"].info.n_inner_rot + l_["plan"].info.n_outer_rot for l_ in self.layers)

    @property
    def pmults_per_step(self):
        return self.batch * sum(l_["plan"].info.n_pt for l_ in self.layers)

    def run(self, mode=1):
        for i in range(len(self.layers)):
            self.run_layer(i, mode)

    def run_layer(self, i, mode=1):
        l_ = self.layers[i]
        if self.batch == 1:
            self.ctx.he_conv(self.evk, l_["plan"], l_["pt"], l_["inp"], mode=mode, ws=self.ws, out=l_["out"])
        else:
            self.ctx.he_layer_batch(self.evk, l_["plan"], l_["pt"], l_["inp"], self.batch, mode=mode, ws=self.ws,
                                    out=l_["out"])

    def capture(self, concurrent=True, req_chunk=None):
        """CUDA graph(s) of one step.  concurrent: the blocks are independent, so
        each gets its own graph, workspace and stream and launch() runs them side
        by side (one block's kernels and copies overlap another's); otherwise one
        graph runs all layers in order in one shared workspace.  req_chunk: take
        the batch's requests that many at a time inside each graph (one data
        region per graph sized for req_chunk requests)."""
        torch = _torch()
        groups = ([self.layers[2 * b:2 * b + 2] for b in range(len(self.blocks))] if concurrent
                  else [self.layers])
        self.graphs, self.graph_ws, self.streams = [], [], []
        for ls in groups:
            plans = [l_["plan"] for l_ in ls]
            if req_chunk is None:
                ws = self.ctx.workspace(self.ctx.graph_workspace_bytes(plans, self.batch))
            else:
                ws = self.ctx.workspace(self.ctx.graph_workspace_bytes_chunked(plans, self.batch, req_chunk))
            s = torch.cuda.Stream()
            s.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(s):
                g = self.ctx.graph_capture(self.evk, plans, [l_["pt"] for l_ in ls], [l_["inp"] for l_ in ls],
                                           [l_["out"] for l_ in ls], ws, n_req=self.batch, req_chunk=req_chunk)
            torch.cuda.current_stream().wait_stream(s)
            self.graphs.append(g)
            self.graph_ws.append(ws)
            self.streams.append(s)
        self.graph = self.graphs[0] if len(self.graphs) == 1 else None
        self._fork = torch.cuda.Event()
        self._join = [torch.cuda.Event() for _ in self.graphs]
        return self.graphs

    def launch(self, h_in=None, h_out=None, join=True):
        """One step through the captured graph(s): fork from the current stream
        to the per-graph streams, optionally copy each block's input from pinned
        host memory first (h_in) and its output back after (h_out), and join
        back.  join=False leaves the per-block streams running ahead: the next
        step's work of one block queues behind its own previous step (same
        stream, same buffers) while the other blocks are still busy; join()
        waits for all of them."""
        torch = _torch()
        main = torch.cuda.current_stream()
        self._fork.record(main)
        per = len(self.blocks) // len(self.graphs)
        for i, (g, s) in enumerate(zip(self.graphs, self.streams)):
            s.wait_event(self._fork)
            with torch.cuda.stream(s):
                blocks = range(i * per, (i + 1) * per)
                if h_in is not None and h_out is not None:
                    # through the C ABI: host copies in, replay, host copies out (fe_graph_launch_host)
                    g.launch_host([h_in[b] for b in blocks], [h_out[b] for b in blocks])
                    continue
                if h_in is not None:
                    for b in blocks:
                        self.inputs[b].copy_(h_in[b], non_blocking=True)
                g.launch()
                if h_out is not None:
                    for b in blocks:
                        h_out[b].copy_(self.outputs[b], non_blocking=True)
        if join:
            self.join()

    def host_outputs(self, level=None):
        """Pinned host buffers for launch(h_in, h_out), with the captured graphs set
        to hand their outputs over at `level` (an exact modulus drop; None: the
        outputs' own level)."""
        torch = _torch()
        for g in self.graphs:
            g.set_host_output_level(level)
        bufs = []
        for o in self.outputs:
            n, two, nl, N = o.shape
            bufs.append(torch.empty((n, two, nl if level is None else level + 1, N), dtype=o.dtype,
                                    pin_memory=True))
        return bufs

    def join(self):
        """Make the current stream wait for every per-block stream."""
        torch = _torch()
        main = torch.cuda.current_stream()
        for i, s in enumerate(self.streams):
            self._join[i].record(s)
            main.wait_event(self._join[i])

    def serve_ops(self, bi):
        """Operation chain of block bi for the request loop (dw then pw)."""
        from . import OP_LAYER
        dw, pw = self.layers[2 * bi], self.layers[2 * bi + 1]
        return [(OP_LAYER, dw["plan"], dw["pt"]), (OP_LAYER, pw["plan"], pw["pt"])]

    def decrypt_block(self, bi, b=0):
        xs, wd, wp, olay = self.ref_inputs[bi]
        n = self.outputs[bi].shape[0] // self.batch
        slots = self.ctx.decrypt(self.sk, self.outputs[bi][b * n:(b + 1) * n], self.ctx.L - 2, self.delta)
        return self.ctx.unpack(olay, slots).cpu().numpy()

    def reference_block(self, bi, b=0):
        """FP64 plaintext result of block bi for input b (valid convolutions)."""
        xs, wd, wp, _ = self.ref_inputs[bi]
        x = xs[b]
        from .plainref import conv2d
        return conv2d(conv2d(x, wd, depthwise=True), wp)


class LeNet:
    """LeNet-5-shaped encrypted network at the largest slot batch for S = 4
    (BS = N / 2 / 64): conv, act, pool, conv, act, pool, FC x3.  The activation
    is a x^2 + b x + c (act = (a, b, c); x^2 by default).  The library fixes
    every scale: each linear layer's weight scale (fe_weight_scale, with the
    next activation's a), the scale after it (fe_plan_out_scale) and after the
    activation (fe_poly_act_scale); this class only passes them along."""

    def __init__(self, ctx, delta, weights, S=4, key_seed=7, act=(1.0, 0.0, 0.0)):
        self.ctx, self.delta, self.S = ctx, delta, S
        self.act = tuple(float(v) for v in act)
        a = self.act[0]
        self.BS = ctx.N // 2 // 64
        L = ctx.L
        if L < 7:
            raise ValueError("the network needs 7 levels")
        self.lay0 = ctx.layout(28, 28, 1, self.BS, S)
        # plans
        self.p1 = ctx.plan_conv(self.lay0, 6, 5, level=L)
        l1 = self.p1.out_layout
        lp1 = ctx.layout(l1.H // 2, l1.W // 2, l1.C, l1.BS, l1.S // 2, l1.m)
        self.p2 = ctx.plan_conv(lp1, 16, 5, level=L - 2)
        l2 = self.p2.out_layout
        lp2 = ctx.layout(l2.H // 2, l2.W // 2, l2.C, l2.BS, l2.S // 2, l2.m)
        self.f1 = ctx.plan_fc_layout(lp2, 120, L - 4)
        self.f2 = ctx.plan_fc_next(self.f1, 84, L - 5)
        self.f3 = ctx.plan_fc_next(self.f2, 10, L - 6)
        self.lp1, self.lp2 = lp1, lp2
        steps = sorted({s for p in (self.p1, self.p2, self.f1, self.f2, self.f3) for s in p.steps})
        self.sk = ctx.sk_gen(key_seed)
        self.evk = ctx.evk_gen(self.sk, key_seed, steps, relin=a != 0)
        # weights and scales (input scale delta at level L)
        s = self.in_scale = delta
        self.pt1 = ctx.load_weights(self.p1, weights["conv1"], ctx.weight_scale(L, s, delta, a))
        s = ctx.plan_out_scale(self.p1, s)
        self.s_act1 = s
        s = ctx.poly_act_scale(L - 1, s, a)
        self.pt2 = ctx.load_weights(self.p2, weights["conv2"], ctx.weight_scale(L - 2, s, delta, a), wmul=0.25)
        s = ctx.plan_out_scale(self.p2, s)
        self.s_act2 = s
        s = ctx.poly_act_scale(L - 3, s, a)
        self.ptf1 = ctx.load_weights(self.f1, weights["fc1"], ctx.weight_scale(L - 4, s, delta), wmul=0.25)
        s = ctx.plan_out_scale(self.f1, s)
        self.ptf2 = ctx.load_weights(self.f2, weights["fc2"], ctx.weight_scale(L - 5, s, delta))
        s = ctx.plan_out_scale(self.f2, s)
        self.ptf3 = ctx.load_weights(self.f3, weights["fc3"], ctx.weight_scale(L - 6, s, delta))
        self.out_scale = ctx.plan_out_scale(self.f3, s)
        self.ws = ctx.workspace(max(p.info.workspace_bytes for p in (self.p1, self.p2, self.f1, self.f2, self.f3)))

    def serve_ops(self):
        """Operation chain of the whole network for the request loop (x^2 activation)."""
        from . import OP_LAYER, OP_POOL, OP_SQUARE
        assert self.act == (1.0, 0.0, 0.0), "the request loop runs the x^2 activation"
        return [(OP_LAYER, self.p1, self.pt1), (OP_SQUARE,), (OP_POOL, self.p1.out_layout),
                (OP_LAYER, self.p2, self.pt2), (OP_SQUARE,), (OP_POOL, self.p2.out_layout),
                (OP_LAYER, self.f1, self.ptf1), (OP_LAYER, self.f2, self.ptf2), (OP_LAYER, self.f3, self.ptf3)]

    def encrypt(self, x, seed=3):
        slots = self.ctx.pack(self.lay0, _torch().from_numpy(np.asarray(x, dtype=np.float64)))
        return self.ctx.encrypt(self.sk, slots, self.ctx.L, self.delta, seed)

    def forward(self, ct, mode=1):
        c, L = self.ctx, self.ctx.L
        h = c.he_conv(self.evk, self.p1, self.pt1, ct, mode=mode, ws=self.ws)
        h, _ = c.he_poly_act(self.evk, h, L - 1, self.s_act1, *self.act)
        h, _ = c.he_avgpool(self.p1.out_layout, h, L - 2)
        h = c.he_conv(self.evk, self.p2, self.pt2, h, mode=mode, ws=self.ws)
        h, _ = c.he_poly_act(self.evk, h, L - 3, self.s_act2, *self.act)
        h, _ = c.he_avgpool(self.p2.out_layout, h, L - 4)
        h = c.he_fc(self.evk, self.f1, self.ptf1, h, mode=mode, ws=self.ws)
        h = c.he_fc(self.evk, self.f2, self.ptf2, h, mode=mode, ws=self.ws)
        return c.he_fc(self.evk, self.f3, self.ptf3, h, mode=mode, ws=self.ws)

    def decode_logits(self, out_ct):
        slots = self.ctx.decrypt(self.sk, out_ct, self.ctx.L - 7, self.out_scale)
        return self.ctx.fc_unpack(self.f3, slots, self.BS, 10).cpu().numpy()


class RefreshChain:
    """n_blocks MobileNet-shaped blocks (depthwise 3x3, a x^2 + b x + c,
    pointwise, the same activation; two by default) with a ciphertext refresh
    between consecutive blocks: the pattern of the paper's deeper networks,
    which refresh their ciphertexts between blocks (Sec. 5, Evaluation
    Methodology).  The context needs the refresh's parameters (levels above the
    refresh's depth, moduli of about 50 bits); the secret is sparse (weight h),
    or, with encapsulate, dense with a sparse secret borrowed by the refresh
    (fe_boot_encapsulate).  Block 1 runs from level L; every block's output is
    brought to level 0 at the refresh's input scale (fe_boot_prepare), the
    refresh returns it at boot.out_level, and the next block runs from there.
    The library fixes every scale (fe_weight_scale, fe_plan_out_scale,
    fe_poly_act_scale, fe_boot_output); this class only passes them along."""

    def __init__(self, ctx, H, C, delta=2.0 ** 40, act=(0.5, 0.5, 0.0), h=64, scale_in=2.0 ** 44, seed=5,
                 key_seed=41, boot_groups=(3, 3), double_angles=6, encapsulate=False, n_blocks=2):
        torch = _torch()
        self.ctx, self.delta, self.act = ctx, delta, tuple(float(v) for v in act)
        a = self.act[0]
        L = ctx.L
        if n_blocks < 1:
            raise ValueError("n_blocks must be positive")
        self.x = W.mobilenet_block(seed, H, C, C, BS=1, block=0)[0]
        self.w = [W.mobilenet_block(seed, H, C, C, BS=1, block=i)[1:] for i in range(n_blocks)]
        self.boot = ctx.boot_create(scale_in, boot_groups[0], boot_groups[1], double_angles)
        lb = self.boot.out_level
        # a block spends 4 levels; a block that a refresh follows must end at level 1 or above
        if n_blocks > 1 and (lb < 4 or (n_blocks > 2 and lb < 5) or L < 5):
            raise ValueError("the refresh leaves too few levels for the blocks after it")
        lay = ctx.layout(H, H, C, 1, 1)
        self.lay = lay
        self.plans = []
        cur = lay
        for i in range(n_blocks):
            lv = L if i == 0 else lb
            pd = ctx.plan_conv(cur, C, 3, depthwise=True, level=lv)
            pp = ctx.plan_conv(pd.out_layout, C, 1, level=lv - 2)
            self.plans.append((pd, pp, lv))
            cur = pp.out_layout
        all_plans = [p for pd, pp, _ in self.plans for p in (pd, pp)]
        steps = sorted({s for p in all_plans for s in p.steps} | set(self.boot.steps))
        if encapsulate:
            # the network under the dense secret; the refresh borrows a sparse one for ModRaise
            self.sk = ctx.sk_gen(key_seed)
            self.sk_sparse = ctx.sk_gen_sparse(key_seed + 1, h)
            ctx.boot_encapsulate(self.boot, self.sk, self.sk_sparse, key_seed)
        else:
            self.sk = ctx.sk_gen_sparse(key_seed, h)
        self.evk = ctx.evk_gen(self.sk, key_seed, steps, relin=True)
        self.n_keys = len(steps)
        self.pts, self.scales = [], []
        self.ws = ctx.workspace(max(p.info.workspace_bytes for p in all_plans))
        self.boot_ws = ctx.workspace(self.boot.workspace_bytes(self.plans[0][1].info.n_out_ct))
        s = delta
        for (pd, pp, lv), (wd, wp) in zip(self.plans, self.w):
            if lv != L:
                s = self.boot.out_scale
            ptd = ctx.load_weights(pd, wd, ctx.weight_scale(lv, s, delta, a))
            s_d = ctx.plan_out_scale(pd, s)
            s_a = ctx.poly_act_scale(lv - 1, s_d, a)
            ptp = ctx.load_weights(pp, wp, ctx.weight_scale(lv - 2, s_a, delta, a))
            s_p = ctx.plan_out_scale(pp, s_a)
            s = ctx.poly_act_scale(lv - 3, s_p, a)
            self.pts.append((ptd, ptp))
            self.scales.append((s_d, s_p, s))
        self.out_layout = self.plans[-1][1].out_layout
        self.out_level = self.plans[-1][2] - 4
        self.out_scale = s
        slots = ctx.pack(lay, torch.from_numpy(self.x))
        self.ct = ctx.encrypt(self.sk, slots, L, delta, seed=7)

    def _block(self, i, h):
        c = self.ctx
        (pd, pp, lv), (ptd, ptp), (s_d, s_p, _) = self.plans[i], self.pts[i], self.scales[i]
        h = c.he_conv(self.evk, pd, ptd, h, ws=self.ws)
        h, _ = c.he_poly_act(self.evk, h, lv - 1, s_d, *self.act)
        h = c.he_conv(self.evk, pp, ptp, h, ws=self.ws)
        h, _ = c.he_poly_act(self.evk, h, lv - 3, s_p, *self.act)
        return h

    def forward(self, trace=None):
        """Block 1, then (prepare, refresh, next block) for each further block;
        returns the output ciphertexts.  trace receives the first block's
        output ("block1") and the first refresh's ("refreshed")."""
        c = self.ctx
        h = self._block(0, self.ct)
        if trace is not None:
            trace["block1"] = h
        for i in range(1, len(self.plans)):
            h = c.boot_prepare(self.boot, h, self.plans[i - 1][2] - 4, self.scales[i - 1][2])
            h = c.bootstrap(self.evk, self.boot, h, ws=self.boot_ws)
            if trace is not None and i == 1:
                trace["refreshed"] = h
            h = self._block(i, h)
        return h

    def decrypt(self, out):
        slots = self.ctx.decrypt(self.sk, out, self.out_level, self.out_scale)
        return self.ctx.unpack(self.out_layout, slots).cpu().numpy()

    def serve_ops(self):
        """The chain as a request-loop model: layers, activations and the refresh."""
        from . import OP_LAYER, OP_POLY_ACT, OP_REFRESH
        ops = []
        for i, ((pd, pp, lv), (ptd, ptp), (s_d, s_p, _)) in enumerate(zip(self.plans, self.pts, self.scales)):
            if i:
                ops.append((OP_REFRESH, self.boot, self.scales[i - 1][2]))
            ops += [(OP_LAYER, pd, ptd), (OP_POLY_ACT, *self.act, s_d), (OP_LAYER, pp, ptp),
                    (OP_POLY_ACT, *self.act, s_p)]
        return ops

    def reference(self):
        """The FP64 network (torch float64) for the decrypted comparison."""
        from . import plainref
        y = self.x
        for wd, wp in self.w:
            y = plainref.conv2d(y, wd, depthwise=True)
            y = plainref.poly_act(y, *self.act)
            y = plainref.conv2d(y, wp)
            y = plainref.poly_act(y, *self.act)
        return y
