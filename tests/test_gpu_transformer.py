"""GPU parity of the transformer extension's linear layers (Sec. 7) through
the C ABI: fragmented token packing equals the oracle's, a projection
Y = X W^T on fragmented embeddings equals the oracle's residues, and an FFN
(E -> gamma E, a x^2 + b x + c, gamma E -> E) equals the oracle's chain bit for
bit and the FP64 FFN within 1e-3."""
import numpy as np
import pytest

import workloads as W
from oracle import ckks, fragment, henn

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2606_16359_b300 as fe  # noqa: E402


def u64(t):
    return t.detach().cpu().numpy().view(np.uint64)


@pytest.mark.parametrize("E,E_out,S", [(32, 24, 2), (30, 40, 4)])
def test_token_pack_and_linear_bit_exact(E, E_out, S):
    p = W.PARAMS["tiny"]
    args = (p["logN"], p["n_q"], p["k"], p["bits"], p["pbits"])
    pr = ckks.Params(*args)
    n_tok = 4
    tl = fragment.TokenLayout(pr.N, n_tok, E, S)
    rng = np.random.default_rng(E + S)
    x = rng.uniform(-1, 1, (n_tok, E))
    w = rng.normal(0, 1 / np.sqrt(E), (E_out, E))
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        g = fe.Context(*args)
        lay = g.token_layout(n_tok, E, S)
        assert (lay.P, lay.F, lay.n_ct) == (tl.P, tl.F, tl.n_ct)
        slots = g.token_pack(lay, torch.from_numpy(x))
        assert np.array_equal(slots.cpu().numpy(), fragment.pack_tokens(tl, x))
        assert np.array_equal(g.token_unpack(lay, slots).cpu().numpy(), x)
        plan = g.plan_token_linear(lay, E_out, g.L)
        sk = g.sk_gen(3)
        evk = g.evk_gen(sk, 3, plan.steps)
        pt = g.load_weights(plan, w, float(g.moduli[g.L]))
        ct = g.encrypt(sk, slots, g.L, p["delta"], 5, ct_id0=0)
        out = g.he_fc(evk, plan, pt, ct)
        got = u64(out)
        y = g.token_unpack(plan.token_out, g.decrypt(sk, out, g.L - 1, p["delta"])).cpu().numpy()
    keys = ckks.KeySet(pr, 3, rot_steps=plan.steps)
    cts = [ckks.encrypt(pr, keys.sk, ckks.encode(pr, fragment.pack_tokens(tl, x)[i], pr.L, p["delta"]), 5, i)
           for i in range(tl.n_ct)]
    oout, tlo = henn.he_token_linear(pr, keys, cts, tl, w)
    assert np.array_equal(got, np.stack([o.as_array() for o in oout]))
    assert np.abs(y - x @ w.T).max() < 1e-3


def test_ffn_chain_bit_exact_and_fp64():
    """E = 32 -> 128 -> 32 (gamma = 4) on 8 tokens at S = 4, N = 2^12 with 40-bit
    primes, activation 0.125 x^2 + 0.5 x + 0.25 between the two linear layers;
    every scale from the library's rule."""
    args = (12, 5, 1, 40, 40)
    delta = 2.0 ** 35
    n_tok, E, gam, S = 8, 32, 4, 4
    a, b, c = 0.125, 0.5, 0.25
    rng = np.random.default_rng(11)
    x = rng.uniform(-1, 1, (n_tok, E))
    w1 = rng.normal(0, 1 / np.sqrt(E), (gam * E, E))
    w2 = rng.normal(0, 1 / np.sqrt(gam * E), (E, gam * E))
    pr = ckks.Params(*args)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        g = fe.Context(*args)
        L = g.L
        lay = g.token_layout(n_tok, E, S)
        p1 = g.plan_token_linear(lay, gam * E, L)
        p2 = g.plan_token_linear(p1.token_out, E, L - 2)
        steps = sorted(set(p1.steps) | set(p2.steps))
        sk = g.sk_gen(4)
        evk = g.evk_gen(sk, 4, steps, relin=True)
        pt1 = g.load_weights(p1, w1, g.weight_scale(L, delta, delta, a))
        ct = g.encrypt(sk, g.token_pack(lay, torch.from_numpy(x)), L, delta, 6, ct_id0=0)
        h = g.he_fc(evk, p1, pt1, ct)
        sc = g.plan_out_scale(p1, delta)
        h, sc = g.he_poly_act(evk, h, L - 1, sc, a, b, c)
        pt2 = g.load_weights(p2, w2, g.weight_scale(L - 2, sc, delta))
        out = g.he_fc(evk, p2, pt2, h)
        sc2 = g.plan_out_scale(p2, sc)
        got = u64(out)
        y = g.token_unpack(p2.token_out, g.decrypt(sk, out, L - 3, sc2)).cpu().numpy()
        assert g.device_status() == 0
    keys = ckks.KeySet(pr, 4, rot_steps=steps, relin=True)
    tl = fragment.TokenLayout(pr.N, n_tok, E, S)
    slots = fragment.pack_tokens(tl, x)
    cts = [ckks.encrypt(pr, keys.sk, ckks.encode(pr, slots[i], pr.L, delta), 6, i) for i in range(tl.n_ct)]
    oh, tl1 = henn.he_token_linear(pr, keys, cts, tl, w1, w_scale=henn.weight_scale(pr, pr.L, delta, delta, a))
    oh = henn.he_poly_act(pr, keys, oh, a, b, c)
    oout, tl2 = henn.he_token_linear(pr, keys, oh, tl1, w2,
                                     w_scale=henn.weight_scale(pr, oh[0].level, oh[0].scale, delta, 0))
    assert np.array_equal(got, np.stack([o.as_array() for o in oout]))
    assert sc2 == oout[0].scale
    t = x @ w1.T
    assert np.abs(y - (a * t * t + b * t + c) @ w2.T).max() < 1e-3


def test_attention_products_bit_exact_and_fp64():
    """Q K^T diagonals and (Q K^T) V on fragmented tokens (4 tokens, E = 16,
    S = 2, N = 2^10 with 40-bit primes): residues and scales equal the
    oracle's, decryption equals FP64 within 1e-3."""
    args = (10, 6, 1, 40, 40)
    delta = 2.0 ** 35
    n, E, S = 4, 16, 2
    pr = ckks.Params(*args)
    tl = fragment.TokenLayout(pr.N, n, E, S)
    rng = np.random.default_rng(1)
    Q, K, V = (rng.uniform(-1, 1, (n, E)) for _ in range(3))
    steps = henn.attention_rotation_steps(tl)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        g = fe.Context(*args)
        L = g.L
        lay = g.token_layout(n, E, S)
        assert g.attention_rotation_steps(lay) == steps
        sk = g.sk_gen(2)
        evk = g.evk_gen(sk, 2, steps, relin=True)
        enc = [g.encrypt(sk, g.token_pack(lay, torch.from_numpy(X)), L, delta, sd, ct_id0=0)
               for X, sd in ((Q, 3), (K, 4), (V, 5))]
        D, d_scale = g.he_attention_scores(evk, lay, enc[0], enc[1], L, delta, delta)
        got_d = u64(D)
        O, o_level, o_scale = g.he_attention_apply(evk, lay, D, L - 2, d_scale, enc[2], L, delta)
        got_o = u64(O)
        y = g.token_unpack(lay, g.decrypt(sk, O, o_level, o_scale)).cpu().numpy()
        assert g.device_status() == 0
    keys = ckks.KeySet(pr, 2, rot_steps=steps, relin=True)

    def oenc(X, sd):
        sl = fragment.pack_tokens(tl, X)
        return [ckks.encrypt(pr, keys.sk, ckks.encode(pr, sl[i], pr.L, delta), sd, i) for i in range(S)]
    od = henn.he_attention_scores(pr, keys, oenc(Q, 3), oenc(K, 4), tl)
    assert np.array_equal(got_d, np.stack([d.as_array() for d in od]))
    assert d_scale == od[0].scale
    oo = henn.he_attention_apply(pr, keys, od, oenc(V, 5), tl)
    assert np.array_equal(got_o, np.stack([o.as_array() for o in oo]))
    assert o_scale == oo[0].scale and o_level == oo[0].level
    assert np.abs(y - (Q @ K.T) @ V).max() < 1e-3
