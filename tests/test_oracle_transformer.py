"""Pins of the oracle's transformer extension (Sec. 7): the fragmented token
layout round-trips, the rotation model picks the block size the paper reports
for the BERT-base encoder block (E = 768, n = 128, gamma about 6: minimum at
S = 4), and the linear layer on fragmented embeddings decrypts to X W^T."""
import numpy as np
import pytest

import workloads as W
from oracle import ckks, counts, fragment, henn


def test_token_layout_round_trip_and_positions():
    tl = fragment.TokenLayout(1024, 4, 30, 4)
    assert tl.P == 128 and tl.F == 8 and tl.n_ct == 4
    x = np.random.default_rng(0).normal(size=(4, 30))
    s = fragment.pack_tokens(tl, x)
    assert np.array_equal(fragment.unpack_tokens(tl, s), x)
    # element e = f S + s of token t: ciphertext s, slot f n_tok + t
    assert s[2, 3 * 4 + 1] == x[1, 3 * 4 + 2]
    # every ciphertext holds ceil(E / S) positions of every token at most
    assert (s[:, tl.F * tl.n_tok:] == 0).all()
    with pytest.raises(ValueError):
        fragment.TokenLayout(1024, 4, 600, 4)  # 150 positions > P = 128


def test_rotation_model_picks_s4_for_bert_base():
    """Sec. 7: BERT-base (E = 768, n = 128, gamma about 6) has its minimum
    latency at S = 4; the model gamma E / S + 2 n S has its minimum there too
    (S* = sqrt(18) = 4.24), and it falls then rises in S."""
    S, cost = counts.choose_S_transformer(768, 128, 6)
    assert S == 4 and cost == 6 * 768 / 4 + 2 * 128 * 4
    assert counts.s_star_transformer(768, 128, 6) == pytest.approx(18 ** 0.5)
    costs = [counts.transformer_rotations(768, 128, 6, s) for s in (1, 2, 4, 8, 16)]
    assert costs[0] > costs[1] > costs[2] < costs[3] < costs[4]
    # S = 1 is full-embedding packing: E - 1 aggregation rotations per FFN stage become gamma E
    assert counts.transformer_rotations(768, 128, 6, 1) == 6 * 768 + 256


@pytest.mark.parametrize("E,E_out,S", [(32, 24, 2), (30, 40, 4), (16, 16, 1)])
def test_token_linear_decrypts_to_xwt(E, E_out, S):
    p = W.PARAMS["tiny"]
    pr = ckks.Params(p["logN"], p["n_q"], p["k"], p["bits"], p["pbits"])
    n_tok = 4
    tl = fragment.TokenLayout(pr.N, n_tok, E, S)
    rng = np.random.default_rng(E + S)
    x = rng.uniform(-1, 1, (n_tok, E))
    w = rng.normal(0, 1 / np.sqrt(E), (E_out, E))
    keys = ckks.KeySet(pr, 3, rot_steps=henn.fc_rotation_steps(tl.P, n_tok))
    slots = fragment.pack_tokens(tl, x)
    cts = [ckks.encrypt(pr, keys.sk, ckks.encode(pr, slots[i], pr.L, p["delta"]), 5, i) for i in range(tl.n_ct)]
    out, tlo = henn.he_token_linear(pr, keys, cts, tl, w)
    assert len(out) == S and tlo.E == E_out
    y = fragment.unpack_tokens(tlo, np.stack([ckks.decrypt(pr, keys.sk, c) for c in out]))
    assert np.abs(y - x @ w.T).max() < 1e-3


def _attn_setup(n=4, E=16, S=2, seed=1):
    pr = ckks.Params(10, 6, 1, 40, 40)
    delta = 2.0 ** 35
    tl = fragment.TokenLayout(pr.N, n, E, S)
    rng = np.random.default_rng(seed)
    Q, K, V = (rng.uniform(-1, 1, (n, E)) for _ in range(3))
    keys = ckks.KeySet(pr, 2, rot_steps=henn.attention_rotation_steps(tl), relin=True)

    def enc(X, sd):
        sl = fragment.pack_tokens(tl, X)
        return [ckks.encrypt(pr, keys.sk, ckks.encode(pr, sl[i], pr.L, delta), sd, i) for i in range(S)]
    return pr, keys, tl, Q, K, V, enc(Q, 3), enc(K, 4), enc(V, 5)


def test_drop_level_and_token_rotation():
    """Dropping the last limb keeps the message and the scale; a token-wise
    rotation by r moves token (t + r) mod n into token t in every position."""
    pr, keys, tl, Q, K, V, q, k, v = _attn_setup()
    d = henn.drop_level(q[0])
    assert d.level == pr.L - 1 and d.scale == q[0].scale
    assert np.abs(ckks.decrypt(pr, keys.sk, d) - ckks.decrypt(pr, keys.sk, q[0])).max() < 1e-6
    ms = henn.mask_scale_pow2(pr, pr.L)
    want = fragment.pack_tokens(tl, Q)[1]
    for r in range(tl.n_tok):
        y = ckks.decrypt(pr, keys.sk, henn.token_rotate(pr, keys, q[1], tl, r, ms))
        rolled = np.concatenate([np.roll(want[f * tl.n_tok:(f + 1) * tl.n_tok], -r) for f in range(tl.P)])
        assert np.abs(y - rolled).max() < 1e-4


def test_attention_scores_and_apply_match_fp64():
    """Sec. 7's attention products on fragmented tokens: the n diagonals of
    Q K^T (replicated over positions) and then (Q K^T) V, against FP64."""
    pr, keys, tl, Q, K, V, q, k, v = _attn_setup()
    D = henn.he_attention_scores(pr, keys, q, k, tl)
    A = Q @ K.T
    n = tl.n_tok
    for r, d in enumerate(D):
        z = ckks.decrypt(pr, keys.sk, d).reshape(tl.P, n)
        want = np.array([A[i][(i + r) % n] for i in range(n)])
        assert np.abs(z - want[None, :]).max() < 1e-3
    assert len({d.scale for d in D}) == 1 and D[0].level == pr.L - 2
    O = henn.he_attention_apply(pr, keys, D, v, tl)
    y = fragment.unpack_tokens(tl, np.stack([ckks.decrypt(pr, keys.sk, o) for o in O]))
    assert np.abs(y - A @ V).max() < 1e-3
