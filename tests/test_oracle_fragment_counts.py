"""Pins of the fragment encoding (Algorithm 1) and of the rotation-complexity
model (Eq. 3 - Eq. 8) against the values the paper prints."""
import os

import numpy as np
import pytest

from oracle import counts, fragment

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    rows = []
    for line in open(os.path.join(GOLD, name)):
        line = line.split("#")[0].strip()
        if line:
            rows.append(line.split())
    return rows


def _worked():
    return {r[0]: float(r[1]) for r in _rows("worked_values.txt")}


def test_table6_rotation_counts_exact():
    for ni, no, K, BS, H, S, rot in _rows("table6_rotations.txt"):
        ni, no, K, BS, H, rot = int(ni), int(no), int(K), int(BS), int(H), int(rot)
        S = int(S.rstrip("*"))
        a = counts.alpha(2 ** 15, H)
        assert counts.total_eq5(ni, no, K, S, BS, a) == rot


def test_table6_bold_rows_are_eq5_argmin():
    rows = _rows("table6_rotations.txt")
    for i in range(0, len(rows), 3):
        grp = rows[i:i + 3]
        bold = [int(r[5].rstrip("*")) for r in grp if r[5].endswith("*")][0]
        ni, no, K, BS, H = (int(x) for x in grp[0][:5])
        Ss = [int(r[5].rstrip("*")) for r in grp]
        best = counts.choose_S(2 ** 15, H, K, ni, no, BS, candidates=Ss)
        assert best[0] == bold
        # the closed form rounded to nearest agrees with the argmin on these rows
        s_star = counts.s_star_eq8(K, ni, no, BS, counts.alpha(2 ** 15, H))
        assert min(Ss, key=lambda s: abs(s - s_star)) == bold


def test_s_star_worked_value():
    w = _worked()
    s = counts.s_star_eq8(9, 128, 32, 8, counts.alpha(2 ** 15, 32))
    assert round(s, 2) == w["s_star_conv128_32_9_bs8"]


def test_fig3_toy_counts():
    """Fig. 3: 1x16x4x4 input, conv(16,16,3,1), BS=1, 16-slot ciphertexts (N = 32)."""
    w = _worked()
    a = counts.alpha(32, 4)
    got = [counts.total_eq5(16, 16, 3, S, 1, a) for S in (1, 2, 4)]
    assert got == [w["fig3_rot_S1"], w["fig3_rot_S2"], w["fig3_rot_S4"]]
    assert counts.choose_S(32, 4, 3, 16, 16, 1, candidates=(1, 2, 4))[0] == 2
    # S=1: inner only; S=4 (= M): outer only
    assert counts.outer_eq4(16, 1, 1, a) == 0
    assert counts.inner_eq3(16, 3, 4, a, M=4) == 0


def test_eq7_slot_waste_example():
    w = _worked()
    l2 = fragment.Layout(8, 4, 4, 1, 1, 2)
    l4 = fragment.Layout(8, 4, 4, 1, 1, 4)
    assert l2.n_ct == w["eq7_S2_cts"] and l2.utilisation() == 1.0
    assert l4.n_ct == w["eq7_S4_cts"] and l4.utilisation() == w["eq7_S4_util"]
    a = counts.alpha(8, 4)
    assert 2 <= counts.s_bound_eq7(1, 1, a) < 4


def test_table7_residual_utilisation():
    for ni, nds, no, H, u_wo, u_w in _rows("table7_residual_util.txt"):
        lay = fragment.Layout(2 ** 16, int(H), int(H), int(nds), 1, 1)
        util = int(nds) / lay.cpc
        assert round(min(util, 1.0), 2) == pytest.approx(float(u_wo), abs=0.005)


def test_fragment_pack_unpack_round_trip_and_slot_map():
    rng = np.random.default_rng(0)
    for (N, H, C, BS, S) in [(256, 7, 3, 2, 2), (512, 10, 5, 1, 4), (128, 4, 2, 2, 1), (2048, 12, 6, 4, 3)]:
        lay = fragment.Layout(N, H, H, C, BS, S)
        x = rng.normal(size=(BS, C, H, H))
        slots = fragment.pack(lay, x)
        assert np.array_equal(fragment.unpack(lay, slots), x)
        cts, sl = fragment.slot_map(lay)
        assert np.array_equal(slots[cts, sl], x)
        # every valid element occupies a distinct (ct, slot)
        flat = cts.ravel() * (N // 2) + sl.ravel()
        assert len(np.unique(flat)) == flat.size
        assert lay.cpc * lay.m * lay.m * BS == N // 2


def test_S1_BS1_is_row_major_and_S_M_is_pixelwise():
    """Generality: S=1, BS=1 recovers row-major multi-channel packing; S=M puts
    one pixel position per ciphertext (pixel-wise packing)."""
    N, H, C = 128, 8, 1
    lay = fragment.Layout(N, H, H, C, 1, 1)
    x = np.arange(H * H, dtype=float).reshape(1, 1, H, H)
    assert np.array_equal(fragment.pack(lay, x)[0][:H * H], x.ravel())
    lay = fragment.Layout(32, 4, 4, 16, 1, 4)  # S = M = 4
    assert lay.m == 1 and lay.n_ct == 16
    x = np.arange(16 * 16, dtype=float).reshape(1, 16, 4, 4)
    s = fragment.pack(lay, x)
    for u in range(4):
        for v in range(4):
            assert np.array_equal(s[lay.ct_index(0, u, v)], x[0, :, u, v])


def test_executed_inner_rotation_counts():
    # config "single conv": S=4, K=5 -> 3 per input ciphertext, 16 ciphertexts
    assert counts.executed_inner(4, 5, 1) == 48
    # LeNet conv2 at S=2, K=5: 8 per ciphertext x 24 ciphertexts
    assert counts.executed_inner(2, 5, 6) == 192
    # K > S: (ceil(K/S)^2 - 1) per ciphertext whenever S divides K - 1 ... e.g. S=1
    for K in (3, 5):
        assert counts.executed_inner(1, K, 1) == K * K - 1
    # K <= S: edge rotations only; S=4, K=3 executes 1.25 per ciphertext on average
    assert counts.executed_inner(4, 3, 1) / 16 == 1.25


def _edge_fragments(S):
    """Brute-force count of the fragments of an S x S fragment grid that lie on
    its border (first or last fragment row or column)."""
    return sum(1 for u in range(S) for v in range(S) if u in (0, S - 1) or v in (0, S - 1))


@pytest.mark.parametrize("S", [2, 3, 4, 5, 8, 16])
def test_eq3_case2_is_the_border_of_the_fragment_grid(S):
    """Eq. 3, case K <= S < M (Sec. 4.2, inner-rotation complexity): only the
    edge computations rotate, up to 4(S - 1) rotations per S x S set of fragment
    ciphertexts.  With N_in / alpha = S^2 ciphertexts (one full fragment set),
    the per-layer value must equal the enumerated border fragments."""
    alpha_ = 2.0
    n_in = alpha_ * S * S
    assert counts.inner_eq3_case2(n_in, S, alpha_) == pytest.approx(_edge_fragments(S))
    # linear in the ciphertext count N_in / alpha
    assert counts.inner_eq3_case2(3 * n_in, S, alpha_) == pytest.approx(3 * _edge_fragments(S))


def test_eq6_equals_eq3_per_regime_and_falls_with_S():
    """Eq. 6 (Sec. 4.2, large batch): with no outer rotations left, the cost is
    the inner-rotation cost of Eq. 3 alone, in both regimes, and it does not
    grow as S grows from 2 on (the statement after Eq. 6; at S = 1 the case
    K <= S is the 1x1 kernel, which needs no rotation at all).  Its S < K regime at S = 1 is
    the (K^2 - 1) rotations per ciphertext that the enumerated inner offsets
    give (every tap but the centre needs its own rotation)."""
    for K in (1, 2, 3, 5, 7):
        for n_in, a in ((16, 1.0), (64, 4.0), (512, 8.0)):
            prev = None
            for S in (1, 2, 4, 8, 16, 32):
                v = counts.amortized_eq6(n_in, K, S, a)
                if S < K:
                    assert v == counts.inner_eq3(n_in, K, S, a)
                else:
                    assert v == counts.inner_eq3_case2(n_in, S, a)
                # non-increasing from S = 2 on, and from S = 1 whenever K > 1
                if prev is not None and (S > 2 or K > 1):
                    assert v <= prev + 1e-12
                prev = v
            if K > 1:
                # S = 1: one ciphertext per channel block, K^2 - 1 executed rotations each
                per_ct = counts.executed_inner(1, K, 1)
                assert counts.amortized_eq6(n_in, K, 1, a) == per_ct * n_in / a


def test_eq5_printed_first_case_is_eq3_case2_plus_eq4():
    """The first case of Eq. 5 as printed, (BS/alpha)(4(S-1)/S^2 N_in +
    (alpha S^2/BS - 1) N_out), is BS times Eq. 3 case 2 plus Eq. 4, and both
    cases of Eq. 5 reduce to the Table 6 total (inner term 0 for K <= S)
    minus or plus exactly that edge term."""
    for (ni, no, K, BS, H, S) in [(64, 64, 3, 4, 32, 4), (128, 32, 3, 8, 32, 8), (32, 128, 3, 8, 32, 4)]:
        a = counts.alpha(2 ** 15, H)
        printed = (BS / a) * (4 * (S - 1) / (S * S) * ni + (a * S * S / BS - 1) * no)
        assert printed == pytest.approx(BS * counts.inner_eq3_case2(ni, S, a) + counts.outer_eq4(no, S, BS, a))
        assert printed - counts.total_eq5(ni, no, K, S, BS, a) == pytest.approx(
            BS * counts.inner_eq3_case2(ni, S, a))
