"""Autotuner: picks, per conv layer, the outer-rotation schedule (linear, or
baby-step / giant-step with n1 baby steps), the hoisting of the rotations
(single, or double: kept on Q P with one ModDown per partial sum) and the MAC
tile (how many outputs share one kernel item's ciphertext loads) by timing
every candidate on the GPU, and caches the choice per layer shape.

Candidates are timed through fe_he_layer_timing with plaintexts from a
resident pool of random plaintexts and rotation keys aliased to a few
generated ones (the kernels, launches and memory volume of the real layer,
with a meaningless result), so no candidate needs its own keys or weight
encoding.  The result of the chosen schedule is exact either way: every
candidate computes the same convolution, and the residues of each schedule are
fixed by its plan.

    t = Tuner(ctx)
    n1, hoist, times = t.conv_schedule(lay, Cout, K, level=ctx.L)
"""
import json
import os

_CACHE = {}


def _key(ctx, lay, Cout, K, stride, depthwise, level):
    return json.dumps([ctx.logN, ctx.L, level, lay.H, lay.W, lay.C, lay.BS, lay.S, lay.m, Cout, K, stride,
                       int(depthwise)])


class Tuner:
    """Timing harness bound to one context: a small evk of generated keys that
    keyless steps are aliased to, and a pool of random plaintexts."""

    def __init__(self, ctx, n_keys=8, n_pts=32, cache_file=None):
        import torch
        self.ctx, self.torch = ctx, torch
        sk = ctx.sk_gen(99)
        self.evk = ctx.evk_gen(sk, 99, list(range(1, n_keys + 1)))
        self.n_pool = n_pts
        # room for plaintexts on Q_L * P (double hoisting) at any level
        self.pts = torch.randint(0, 2 ** 35, (n_pts * (ctx.L + 1 + ctx.k) * ctx.N,), dtype=torch.int64,
                                 device="cuda")
        self.cache_file = cache_file
        if cache_file and os.path.exists(cache_file):
            with open(cache_file) as f:
                _CACHE.update(json.load(f))

    def time_plan(self, plan, reps=2):
        """CUDA-event time (ms) of one call of the plan's layer, after a warm-up."""
        torch, ctx = self.torch, self.ctx
        i = plan.info
        ctx.evk_alias(self.evk, plan.steps)
        x = torch.randint(0, 2 ** 35, (i.n_in_ct, 2, plan.level + 1, ctx.N), dtype=torch.int64, device="cuda")
        out = ctx.empty_ct(i.n_out_ct, plan.level - 1)
        ws = ctx.workspace(i.workspace_bytes)
        ctx.he_layer_timing(self.evk, plan, self.pts, self.n_pool, x, out, ws)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            ctx.he_layer_timing(self.evk, plan, self.pts, self.n_pool, x, out, ws)
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    def conv_schedule(self, lay, Cout, K, stride=1, depthwise=False, level=None, reps=2):
        """Fastest schedule of a conv layer: outer rotations (n1 baby steps, 0 =
        linear) and hoisting (0 single; 2 double: rotations and MAC on Q P, with
        ModDown and rescale in one step when there is no outer rotation).
        Returns (n1, hoisting, {"n1/hoisting": ms})."""
        ctx = self.ctx
        level = ctx.L if level is None else level
        key = _key(ctx, lay, Cout, K, stride, depthwise, level)
        if key in _CACHE:
            c = _CACHE[key]
            return c["n1"], c["hoist"], dict(c["ms"])
        n1s = [0]
        if not depthwise and lay.cpc > 1:
            n1 = 2
            while n1 <= lay.cpc:
                n1s.append(n1)
                n1 *= 2
        times = {}
        for n1 in n1s:
            for dh in (0, 2):
                plan = ctx.plan_conv(lay, Cout, K, stride=stride, depthwise=depthwise, level=level, bsgs_n1=n1,
                                     double_hoist=dh)
                if plan.info.n_inner_rot == 0 and dh:
                    continue  # nothing to hoist
                times[f"{n1}/{dh}"] = self.time_plan(plan, reps)
                del plan
        best = min(times, key=times.get)
        n1, dh = (int(v) for v in best.split("/"))
        _CACHE[key] = {"n1": n1, "hoist": dh, "ms": times}
        self._save()
        return n1, dh, times

    def mac_ways(self, plan, reps=2):
        """Fastest MAC tile (outputs sharing one kernel item: 1, 2 or 4) for a
        plan; sets it on the plan and returns (ways, {ways: ms})."""
        ctx = self.ctx
        i = plan.info
        key = json.dumps(["mac_ways", ctx.logN, ctx.L, plan.level, i.n_in_ct, i.n_out_ct, i.n_pt, i.n_inner_rot,
                          i.n_outer_rot, i.bsgs_n1, i.double_hoist])
        if key in _CACHE:
            c = _CACHE[key]
            ctx.plan_set_mac_ways(plan, c["ways"])
            return c["ways"], {int(k): v for k, v in c["ms"].items()}
        times = {}
        for w in (1, 2, 4):
            ctx.plan_set_mac_ways(plan, w)
            times[w] = self.time_plan(plan, reps)
        best = min(times, key=times.get)
        ctx.plan_set_mac_ways(plan, best)
        _CACHE[key] = {"ways": best, "ms": times}
        self._save()
        return best, times

    def _save(self):
        if self.cache_file:
            with open(self.cache_file, "w") as f:
                json.dump(_CACHE, f)
