"""Multi-layer encrypted workloads assembled from the C-ABI layers.

MobileNetBlocks: three depthwise-3x3 + pointwise blocks under the fragment
encoding at S = 1 (the largest maps need S = 1 to fit a ciphertext), each
block an independent encrypted input.  All layers' ciphertexts, plaintexts and
keys stay resident on the device; a step runs the six HE convolutions.

LeNet: conv5x5 1->6, x^2, avgpool2, conv5x5 6->16, x^2, avgpool2, FC 256->120->84->10
at the largest slot batch (Sec. 4 implementation paragraph: x^2 activation,
pooling by fragment sums, FC by diagonals with baby-step / giant-step).
"""
import numpy as np

import workloads as W

from . import Context, FeLayout  # noqa: F401


def _torch():
    import torch
    return torch


class MobileNetBlocks:
    def __init__(self, ctx, blocks=None, seed=0, delta=2.0 ** 32, key_seed=101, enc_seed=202):
        torch = _torch()
        self.ctx = ctx
        self.delta = delta
        self.blocks = list(W.MOBILENET_BLOCKS if blocks is None else blocks)
        L = ctx.L
        self.layers = []  # dicts: plan, pt, inp, out, level
        self.inputs, self.ref_inputs = [], []
        plans = []
        for bi, (H, Cin, Cout) in enumerate(self.blocks):
            x, wd, wp = W.mobilenet_block(seed, H, Cin, Cout, BS=1, block=bi)
            lay = ctx.layout(H, H, Cin, 1, 1)
            pdw = ctx.plan_conv(lay, Cin, 3, depthwise=True, level=L)
            ppw = ctx.plan_conv(pdw.out_layout, Cout, 1, level=L - 1)
            plans.append((lay, pdw, ppw, x, wd, wp))
        steps = sorted({s for _, a, b, *_ in plans for s in a.steps + b.steps})
        self.sk = ctx.sk_gen(key_seed)
        self.evk = ctx.evk_gen(self.sk, key_seed, steps)
        self.n_keys = len(steps)
        ct_id = 0
        for bi, (lay, pdw, ppw, x, wd, wp) in enumerate(plans):
            slots = ctx.pack(lay, torch.from_numpy(x))
            ct = ctx.encrypt(self.sk, slots, L, delta, enc_seed, ct_id0=ct_id)
            ct_id += lay.n_ct
            pt_dw = ctx.load_weights(pdw, wd, float(ctx.moduli[L]))
            pt_pw = ctx.load_weights(ppw, wp, float(ctx.moduli[L - 1]))
            mid = ctx.empty_ct(pdw.info.n_out_ct, L - 1)
            out = ctx.empty_ct(ppw.info.n_out_ct, L - 2)
            self.layers.append(dict(plan=pdw, pt=pt_dw, inp=ct, out=mid, level=L, name=f"b{bi}_dw"))
            self.layers.append(dict(plan=ppw, pt=pt_pw, inp=mid, out=out, level=L - 1, name=f"b{bi}_pw"))
            self.inputs.append(ct)
            self.ref_inputs.append((x, wd, wp, ppw.out_layout))
        self.outputs = [self.layers[2 * i + 1]["out"] for i in range(len(self.blocks))]
        self.ws_bytes = max(l_["plan"].info.workspace_bytes for l_ in self.layers)
        self.ws = ctx.workspace(self.ws_bytes)
        self.graph = None

    @property
    def keyswitches_per_step(self):
        return sum(l_["plan"].info.n_inner_rot + l_["plan"].info.n_outer_rot for l_ in self.layers)

    @property
    def pmults_per_step(self):
        return sum(l_["plan"].info.n_pt for l_ in self.layers)

    def run(self, mode=1):
        for l_ in self.layers:
            self.ctx.he_conv(self.evk, l_["plan"], l_["pt"], l_["inp"], mode=mode, ws=self.ws, out=l_["out"])

    def run_layer(self, i, mode=1):
        l_ = self.layers[i]
        self.ctx.he_conv(self.evk, l_["plan"], l_["pt"], l_["inp"], mode=mode, ws=self.ws, out=l_["out"])

    def capture(self):
        plans = [l_["plan"] for l_ in self.layers]
        total = sum((p.info.workspace_bytes + 255) // 256 * 256 for p in plans)
        self.graph_ws = self.ctx.workspace(total)
        self.graph = self.ctx.graph_capture(self.evk, plans, [l_["pt"] for l_ in self.layers],
                                            [l_["inp"] for l_ in self.layers], [l_["out"] for l_ in self.layers],
                                            self.graph_ws)
        return self.graph

    def decrypt_block(self, bi):
        x, wd, wp, olay = self.ref_inputs[bi]
        slots = self.ctx.decrypt(self.sk, self.outputs[bi], self.ctx.L - 2, self.delta)
        return self.ctx.unpack(olay, slots).cpu().numpy()

    def reference_block(self, bi):
        """FP64 plaintext result of block bi (valid convolutions)."""
        x, wd, wp, _ = self.ref_inputs[bi]
        from .plainref import conv2d
        return conv2d(conv2d(x, wd, depthwise=True), wp)
