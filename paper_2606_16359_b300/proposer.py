"""Learned fragment-size and schedule proposer.

A small latency model (fe_mlp_*: 3 hidden layers of 64 ReLU units, fp32, CUDA
training and inference kernels) is trained on per-layer latencies that this
module measures through the library, and proposes for a conv layer the
fragment size S and the outer-rotation schedule (linear, or baby-step /
giant-step with n1 = 2^ceil(log2(cpc) / 2) baby steps) as the argmin of its
predicted latency over the admissible choices.
The paper's analytic choice (Theorem: argmin of Eq. 5, fe_choose_fragment) is
(with the paper's linear outer rotations) is its fallback (no trained model, a
ring degree it was not trained on) and its judge: the proposal stands only if
the model predicts it at least `margin` faster than the analytic choice and
its Eq. 5 rotation count is within `veto` times the analytic choice's;
otherwise the analytic choice is taken.

Measurement of one (layer, S): the full layer is planned on the host (exact
rotation, plaintext and ciphertext counts); a slice of it is run on the GPU,
one input channel group, one output channel group, truncated to its first
output ciphertext, with plaintexts drawn from a resident pool and keyless
rotation steps aliased to generated keys (fe_he_layer_timing, fe_evk_alias:
same kernels and memory volume, meaningless result).  The slice's stage times
(inner rotations, unrotated MAC, outer rotations, rescale, and all MAC
launches) are extrapolated linearly to the full layer by the ratios of the
counts that drive them: inner rotations, plaintext terms, outer rotations and
output ciphertexts.  Layers run at the top level of the parameter set of their
ring degree (N = 2^14: 8 x 40-bit primes; N = 2^16: 24 x 36-bit primes).

    python -m paper_2606_16359_b300.proposer [--layers 200] [--out results.json]
"""
import argparse
import json
import math
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CANDIDATE_S = (1, 2, 4, 8)
PARAM_SET = {14: "lenet", 16: "mobilenet"}
N_FEATURES = 16


def _fe():
    sys.path.insert(0, ROOT)
    import paper_2606_16359_b300 as fe
    return fe


def candidates(layer):
    """Admissible fragment sizes of a layer: the channel block fits a
    ciphertext, Eq. 7 holds (S = 1 always), stride 2 needs an even S.  A
    stride-2 layer whose even sizes all break Eq. 7 (few channels) keeps the
    smallest even size that fits."""
    fe = _fe()
    N = 2 ** layer["logN"]
    out, fitting = [], []
    for S in CANDIDATE_S:
        if layer["stride"] == 2 and S % 2:
            continue
        try:
            r = fe.rotation_model(N, layer["H"], layer["W"], layer["Cin"], layer["Cout"], layer["K"], S, 1,
                                  layer["stride"])
        except fe.FencError:
            continue
        fitting.append((S, r))
        if S > 1 and S > r["s_bound_eq7"]:
            continue
        out.append((S, r))
    return out if out else fitting[:1]


def analytic_choice(layer, cands=None):
    """Argmin of Eq. 5 over the admissible sizes, ties to the smaller S."""
    cands = candidates(layer) if cands is None else cands
    return min(cands, key=lambda c: (c[1]["eq5_total"], c[0]))[0]


def schedules(model):
    """Outer-rotation schedules tried at one fragment size: linear (0), and
    baby-step / giant-step with n1 = 2^ceil(log2(cpc) / 2) when cpc >= 4."""
    cpc = model["cpc"]
    if cpc < 4:
        return [0]
    return [0, 1 << ((cpc.bit_length() - 1 + 1) // 2)]


def choices(layer):
    """All (S, n1, rotation model) the proposer chooses among."""
    return [(S, n1, r) for S, r in candidates(layer) for n1 in schedules(r)]


def features(layer, S, model, counts, n1=0):
    """Feature vector of (layer, S, schedule): shape, ring, fragment geometry,
    baby steps and the exact counts of the planned layer."""
    lg = lambda x: math.log2(1.0 + x)  # noqa: E731
    return [layer["logN"], math.log2(layer["H"]), math.log2(layer["Cin"]), math.log2(layer["Cout"]), layer["K"],
            layer["stride"], math.log2(S), math.log2(model["cpc"]), lg(counts["n_in_ct"]), lg(counts["n_out_ct"]),
            lg(counts["n_inner"]), lg(counts["n_outer"]), lg(counts["n_pt"]), lg(model["eq5_total"]),
            counts["level"] + 1, lg(n1)]


class Measurer:
    """Per ring degree: a context at the parameter set's top level, a pool of
    generated keys to alias, a pool of random plaintexts, random inputs."""

    def __init__(self, logN, n_keys=16, n_pts=48):
        import torch
        import workloads as W
        fe = _fe()
        p = W.PARAMS[PARAM_SET[logN]]
        self.torch, self.fe = torch, fe
        self.ctx = fe.Context(p["logN"], p["n_q"], p["k"], p["bits"], p["pbits"])
        self.level = self.ctx.L
        sk = self.ctx.sk_gen(1)
        self.evk = self.ctx.evk_gen(sk, 1, list(range(1, n_keys + 1)))
        nl = self.level + 1
        self.n_pool = n_pts
        self.pts = torch.randint(0, 2 ** 35, (n_pts * (nl + self.ctx.k) * self.ctx.N,), dtype=torch.int64,
                                 device="cuda")

    def plan(self, layer, S, Cin, Cout, n1=0):
        lay = self.ctx.layout(layer["H"], layer["W"], Cin, 1, S)
        return self.ctx.plan_conv(lay, Cout, layer["K"], stride=layer["stride"], level=self.level, bsgs_n1=n1)

    def counts(self, plan):
        i = plan.info
        return {"n_in_ct": i.n_in_ct, "n_out_ct": i.n_out_ct, "n_inner": i.n_inner_rot, "n_outer": i.n_outer_rot,
                "n_pt": i.n_pt, "level": self.level}

    def time_slice(self, plan, reps=1):
        torch, ctx = self.torch, self.ctx
        i = plan.info
        ctx.evk_alias(self.evk, plan.steps)
        x = torch.randint(0, 2 ** 35, (i.n_in_ct, 2, self.level + 1, ctx.N), dtype=torch.int64, device="cuda")
        out = ctx.empty_ct(i.n_out_ct, self.level - 1)
        ws = ctx.workspace(i.workspace_bytes)
        ctx.he_layer_timing(self.evk, plan, self.pts, self.n_pool, x, out, ws)  # warm-up
        t = {}
        for kind in ("stage_inner", "stage_base", "stage_outer", "stage_rescale", "mac"):
            ctx.profile_begin(kind)
            for _ in range(reps):
                ctx.he_layer_timing(self.evk, plan, self.pts, self.n_pool, x, out, ws)
            ms, n, _ = ctx.profile_end()
            t[kind] = ms / reps
        del x, out, ws
        return t

    def measure(self, layer, S, model, n1=0):
        """Estimated latency (ms) of the full layer at fragment size S with n1
        baby steps (0: linear outer rotations)."""
        full = self.plan(layer, S, layer["Cin"], layer["Cout"], n1)
        cf = self.counts(full)
        cpc = model["cpc"]
        sl = self.plan(layer, S, min(layer["Cin"], cpc), min(layer["Cout"], cpc), n1)
        self.ctx.plan_truncate(sl, 1)
        cs = self.counts(sl)
        t = self.time_slice(sl)
        mac_outer = max(0.0, t["mac"] - t["stage_base"])
        ks_outer = max(0.0, t["stage_outer"] - mac_outer)
        ratio = lambda a, b: (a / b) if b else 0.0  # noqa: E731
        est = (t["stage_inner"] * ratio(cf["n_inner"], cs["n_inner"]) +
               t["mac"] * ratio(cf["n_pt"], cs["n_pt"]) +
               ks_outer * ratio(cf["n_outer"], cs["n_outer"]) +
               t["stage_rescale"] * ratio(cf["n_out_ct"], cs["n_out_ct"]))
        return est, cf, cs, t


class Proposer:
    """Fragment-size proposals from the trained latency model, judged by the
    analytic choice."""

    def __init__(self, mlp=None, trained_logN=(), margin=0.05, veto=8.0):
        self.mlp, self.trained_logN = mlp, set(trained_logN)
        self.margin, self.veto = margin, veto

    def predict(self, layer, counts_of):
        """Predicted latency (ms) of every choice: {(S, n1): ms}; counts_of(S, n1)
        gives the exact counts of the planned layer."""
        ch = choices(layer)
        X = np.array([features(layer, S, r, counts_of(S, n1), n1) for S, n1, r in ch], dtype=np.float32)
        return {(S, n1): float(np.exp(v)) for (S, n1, _), v in zip(ch, self.mlp.predict(X))}

    def propose(self, layer, counts_of):
        """Returns ((S, n1), source), source 'model', 'fallback' or 'judge'."""
        s_an = (analytic_choice(layer), 0)
        if self.mlp is None or layer["logN"] not in self.trained_logN:
            return s_an, "fallback"
        pred = self.predict(layer, counts_of)
        c_m = min(pred, key=pred.get)
        eq5 = {S: r["eq5_total"] for S, r in candidates(layer)}
        if c_m != s_an and (pred[c_m] > (1.0 - self.margin) * pred[s_an] or
                            eq5[c_m[0]] > self.veto * max(eq5[s_an[0]], 1.0)):
            return s_an, "judge"
        return c_m, "model"


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--layers", type=int, default=200)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--out", default="proposer_config4.json",
                    help="report file (JSON), relative to the working directory")
    args = ap.parse_args(argv)
    import torch
    import workloads as W
    fe = _fe()

    layers = W.synthetic_layers(args.seed, args.layers)
    side = torch.cuda.Stream()
    rows = []
    t0 = time.perf_counter()
    with torch.cuda.stream(side):
        meas = {}
        for L in layers:
            if L["logN"] not in meas:
                meas[L["logN"]] = Measurer(L["logN"])
            m = meas[L["logN"]]
            for S, n1, model in choices(L):
                est, cf, cs, t = m.measure(L, S, model, n1)
                rows.append({"layer": L, "S": S, "n1": n1, "ms": est, "counts": cf, "slice": cs, "stage_ms": t,
                             "eq5": model["eq5_total"], "x": features(L, S, model, cf, n1)})
        t_meas = time.perf_counter() - t0
        train = [r for r in rows if r["layer"]["split"] == "train"]
        X = np.array([r["x"] for r in train], dtype=np.float32)
        y = np.log(np.array([r["ms"] for r in train], dtype=np.float32))
        mlp = fe.MLP(N_FEATURES, hidden=64, n_hidden=3, seed=args.seed)
        loss = mlp.train(X, y, steps=args.steps, lr=2e-3, weight_decay=1e-4)
        prop = Proposer(mlp, trained_logN={14, 16})
        summary = {"model": [], "analytic": [], "judged": []}
        hits = {"model": 0, "analytic": 0, "judged": 0}
        sources = {"model": 0, "judge": 0, "fallback": 0}
        per_layer = []
        for L in layers:
            if L["split"] != "test":
                continue
            lr_ = [r for r in rows if r["layer"]["id"] == L["id"]]
            ms = {(r["S"], r["n1"]): r["ms"] for r in lr_}
            cnt = {(r["S"], r["n1"]): r["counts"] for r in lr_}
            best = min(ms, key=ms.get)
            s_an = (analytic_choice(L), 0)
            pred = prop.predict(L, lambda S, n1: cnt[(S, n1)])
            s_model = min(pred, key=pred.get)
            s_j, src = prop.propose(L, lambda S, n1: cnt[(S, n1)])
            sources[src] += 1
            for k, s in (("model", s_model), ("analytic", s_an), ("judged", s_j)):
                summary[k].append(ms[s] / ms[best] - 1.0)
                hits[k] += s == best
            key = lambda c: f"{c[0]}/{c[1]}"  # noqa: E731
            per_layer.append({"id": L["id"], "best": key(best), "model": key(s_model), "analytic": key(s_an),
                              "judged": key(s_j), "source": src, "ms": {key(c): v for c, v in ms.items()},
                              "pred_ms": {key(c): v for c, v in pred.items()}})
        n_test = len(per_layer)
        res = {"metric": "proposer vs analytic fragment-size choice on measured latency",
               "layers": len(layers), "train_samples": len(train), "test_layers": n_test,
               "train_loss_std_mse": loss, "measure_s": t_meas,
               "mean_regret": {k: float(np.mean(v)) for k, v in summary.items()},
               "max_regret": {k: float(np.max(v)) for k, v in summary.items()},
               "best_hit_rate": {k: hits[k] / n_test for k in hits},
               "total_ms_vs_best": {k: float(sum(p["ms"][p[k]] for p in per_layer) /
                                              sum(p["ms"][p["best"]] for p in per_layer)) for k in hits},
               "judged_sources": sources,
               "config": {"candidates_S": CANDIDATE_S, "schedules": "linear, BSGS n1 = 2^ceil(log2(cpc)/2)",
                          "mlp": "16 -> 64x3 ReLU -> 1, fp32, Adam",
                          "steps": args.steps, "seed": args.seed,
                          "timing": "slice (1 in group, 1 out group, first output ct) extrapolated per stage",
                          "judge": {"margin": prop.margin, "veto_eq5_ratio": prop.veto}}}
        print(json.dumps(res), flush=True)
        os.makedirs(os.path.dirname(args.out), exist_ok=True)
        with open(args.out, "w") as f:
            json.dump({"summary": res, "per_layer": per_layer,
                       "rows": [{k: v for k, v in r.items() if k != "layer"} | {"id": r["layer"]["id"]}
                                for r in rows]}, f)
    return 0


if __name__ == "__main__":
    sys.exit(main())
