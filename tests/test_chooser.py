"""The library's rotation-complexity model and analytic fragment-size choice
(host code behind the C ABI, no GPU) against the oracle's Eq. 3 - Eq. 8 and the
printed values of Table 6."""
import math
import os

import pytest

import workloads as W
from oracle import counts

fe = pytest.importorskip("paper_2606_16359_b300")

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _lib_or_skip():
    try:
        fe.load()
    except Exception as e:  # library not built
        pytest.skip(f"libfenc not built: {e}")


def _table6():
    rows = []
    for line in open(os.path.join(GOLD, "table6_rotations.txt")):
        line = line.split("#")[0].strip()
        if line:
            rows.append(line.split())
    return rows


def test_table6_counts_and_bold_choice():
    _lib_or_skip()
    rows = _table6()
    for ni, no, K, BS, H, S, rot in rows:
        r = fe.rotation_model(2 ** 15, int(H), int(H), int(ni), int(no), int(K), int(S.rstrip("*")), int(BS))
        assert r["eq5_total"] == int(rot)
    for i in range(0, len(rows), 3):
        grp = rows[i:i + 3]
        bold = [int(r[5].rstrip("*")) for r in grp if r[5].endswith("*")][0]
        ni, no, K, BS, H = (int(x) for x in grp[0][:5])
        Ss = sorted(int(r[5].rstrip("*")) for r in grp)
        ch = fe.choose_fragment(2 ** 15, H, H, ni, no, K, BS, max_S=Ss[-1])
        # the library searches all powers of two up to the largest listed S; the
        # listed rows are a subset, so its argmin is at least as good
        assert ch["eq5"] <= min(counts.total_eq5(ni, no, K, s, BS, counts.alpha(2 ** 15, H)) for s in Ss)
        if set(Ss) == {Ss[0] * 2 ** j for j in range(len(Ss))} and Ss[0] == 1:
            assert ch["S"] == bold


def test_s_star_worked_value():
    _lib_or_skip()
    r = fe.rotation_model(2 ** 15, 32, 32, 128, 32, 9, 4, 8)
    assert round(r["s_star_eq8"], 2) == 3.57


def test_choice_matches_oracle_on_synthetic_layers():
    _lib_or_skip()
    for L in W.synthetic_layers(0, 200):
        N = 2 ** L["logN"]
        for BS in (1, 4):
            want = counts.choose_S(N, L["H"], L["K"], L["Cin"], L["Cout"], BS)
            try:
                got = fe.choose_fragment(N, L["H"], L["W"], L["Cin"], L["Cout"], L["K"], BS)
            except fe.FencError:
                assert want is None
                continue
            assert want is not None
            assert got["S"] == want[0], (L, BS, got, want)
            assert math.isclose(got["eq5"], want[1], rel_tol=1e-12)


def test_executed_inner_matches_oracle():
    _lib_or_skip()
    for S in (1, 2, 4, 8):
        for K in (1, 3, 5, 7):
            for stride in (1, 2):
                if stride == 2 and S % 2:
                    continue
                M = 8 * S
                r = fe.rotation_model(2 ** 14, M, M, 3, 4, K, S, 1, stride)
                groups = -(-3 // r["cpc"])
                assert r["executed_inner"] == counts.executed_inner(S, K, groups, stride)


def test_rejects_bad_arguments():
    _lib_or_skip()
    with pytest.raises(fe.FencError):
        fe.rotation_model(2 ** 10, 224, 224, 3, 3, 3, 1, 1)   # block does not fit
    with pytest.raises(fe.FencError):
        fe.choose_fragment(1000, 8, 8, 3, 3, 3, 1)            # N not a power of two


def test_token_fragment_choice_matches_the_oracle_and_the_paper():
    """Sec. 7: the block size of fragmented token embeddings minimises
    gamma E / S + 2 n S; for BERT-base (E = 768, n = 128, gamma about 6) the
    paper's encoder block is fastest at S = 4."""
    import paper_2606_16359_b300 as fe
    from oracle import counts
    r = fe.choose_token_fragment(768, 128, 6.0)
    assert r["S"] == 4 and r["rotations"] == counts.transformer_rotations(768, 128, 6, 4)
    assert abs(r["s_star"] - counts.s_star_transformer(768, 128, 6)) < 1e-12
    import random
    rng = random.Random(3)
    for _ in range(200):
        E = rng.choice([64, 96, 128, 192, 256, 384, 512, 768, 1024])
        n = rng.choice([8, 16, 32, 64, 128, 256, 512])
        g = rng.choice([1.0, 2.0, 4.0, 6.0, 8.0])
        assert fe.choose_token_fragment(E, n, g)["S"] == counts.choose_S_transformer(E, n, g)[0]
