"""Host logic of the fragment-size proposer (no GPU): candidate sets, the
analytic choice it falls back on, and its feature vector."""
import pytest

import workloads as W
from oracle import counts

fe = pytest.importorskip("paper_2606_16359_b300")
proposer = pytest.importorskip("paper_2606_16359_b300.proposer")


def _lib_or_skip():
    try:
        fe.load()
    except Exception as e:
        pytest.skip(f"libfenc not built: {e}")


def test_candidates_respect_fit_eq7_and_stride():
    _lib_or_skip()
    for L in W.synthetic_layers(0, 200):
        cands = proposer.candidates(L)
        assert cands, L
        for S, r in cands:
            assert S in proposer.CANDIDATE_S
            assert L["stride"] == 1 or S % 2 == 0
            assert S == 1 or S <= r["s_bound_eq7"] or (L["stride"] == 2 and cands == [(2, r)])
            assert r["m"] ** 2 <= 2 ** L["logN"] // 2


def test_analytic_choice_is_the_oracle_eq5_argmin():
    _lib_or_skip()
    for L in W.synthetic_layers(0, 200):
        if L["stride"] != 1:
            continue
        want = counts.choose_S(2 ** L["logN"], L["H"], L["K"], L["Cin"], L["Cout"], 1,
                               candidates=proposer.CANDIDATE_S)
        assert proposer.analytic_choice(L) == want[0], L


def test_features_and_fallback():
    _lib_or_skip()
    L = W.synthetic_layers(0, 1)[0]
    S, r = proposer.candidates(L)[0]
    c = {"n_in_ct": 4, "n_out_ct": 4, "n_inner": 12, "n_outer": 28, "n_pt": 100, "level": 23}
    x = proposer.features(L, S, r, c, 4)
    assert len(x) == proposer.N_FEATURES and all(v == v for v in x)
    # no trained model: the analytic choice, marked as the fallback
    P = proposer.Proposer(None)
    assert P.propose(L, lambda s, n1: c) == ((proposer.analytic_choice(L), 0), "fallback")
    # schedules: linear always, BSGS with n1 = 2^ceil(log2(cpc)/2) when cpc >= 4
    for S, n1, r in proposer.choices(L):
        assert n1 == 0 or (r["cpc"] >= 4 and n1 * n1 >= r["cpc"] and n1 * n1 < 4 * r["cpc"])
