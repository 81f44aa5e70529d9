"""Pins of the oracle's fragment-size change (Sec. 5, Implementation paragraph:
the block size S is adjusted between layers by rot-mask-add): after
decryption, the re-encoded ciphertexts unpack under the target layout to the
original tensor, in both directions and with a batch, and the rotations it
executes are the baby and giant steps its BSGS split counts."""
import numpy as np
import pytest

import workloads as W
from oracle import ckks, fragment, henn


@pytest.fixture(scope="module")
def tiny():
    p = W.PARAMS["tiny"]
    return ckks.Params(p["logN"], p["n_q"], p["k"], p["bits"], p["pbits"]), p["delta"]


def _run(pr, delta, la, lb, seed):
    x = np.random.default_rng(seed).uniform(-1, 1, (la.BS, la.C, la.H, la.W))
    keys = ckks.KeySet(pr, 5, rot_steps=henn.repack_rotation_steps(la, lb))
    slots = fragment.pack(la, x)
    cts = [ckks.encrypt(pr, keys.sk, ckks.encode(pr, slots[i], pr.L, delta), 7, i) for i in range(la.n_ct)]
    cnt = henn.Counters()
    out = henn.he_repack(pr, keys, cts, la, lb, cnt=cnt)
    assert len(out) == lb.n_ct and out[0].level == pr.L - 1 and out[0].scale == pytest.approx(delta)
    y = fragment.unpack(lb, np.stack([ckks.decrypt(pr, keys.sk, c) for c in out]))
    return x, y, cnt


@pytest.mark.parametrize("case", [
    dict(H=8, C=2, BS=1, Sa=1, Sb=2),    # finer fragments: 1 -> 4 ciphertexts per group
    dict(H=8, C=3, BS=1, Sa=2, Sb=1),    # the other way
    dict(H=6, C=2, BS=2, Sa=2, Sb=1),    # a batch of two, a map side that is not a power of two
    dict(H=8, C=1, BS=2, Sa=4, Sb=2),    # S = M to a coarser split
])
def test_repack_unpacks_to_the_tensor_under_the_target_layout(tiny, case):
    pr, delta = tiny
    la = fragment.Layout(pr.N, case["H"], case["H"], case["C"], case["BS"], case["Sa"])
    lb = fragment.Layout(pr.N, case["H"], case["H"], case["C"], case["BS"], case["Sb"])
    x, y, cnt = _run(pr, delta, la, lb, case["H"] + case["C"])
    assert np.abs(y - x).max() < 1e-3
    # the executed rotations are the BSGS split's distinct baby steps per source
    # ciphertext plus its distinct giant steps per target ciphertext
    n1 = henn.repack_bsgs_n1(la, lb)
    baby, giant = set(), set()
    for (ct, cs), ds in henn.repack_shifts(la, lb).items():
        for d in ds:
            if d % n1:
                baby.add((cs, d % n1))
            if d // n1:
                giant.add((ct, d // n1))
    assert cnt.rot == len(baby) + len(giant)


def test_repack_map_is_a_bijection_onto_the_target_positions(tiny):
    pr, _ = tiny
    la = fragment.Layout(pr.N, 7, 7, 5, 1, 2)
    lb = fragment.Layout(pr.N, 7, 7, 5, 1, 1)
    m = henn.repack_map(la, lb)
    assert len({s for s, _ in m}) == len({t for _, t in m}) == len(m) == 5 * 7 * 7
    # every pair agrees with Algorithm 1's slot map of each layout
    cts_a, sl_a = fragment.slot_map(la)
    cts_b, sl_b = fragment.slot_map(lb)
    for c in range(5):
        for h in range(7):
            for w in range(7):
                (sa, pa), (sb, pb) = m[(c * 7 + h) * 7 + w]
                assert (sa, pa * la.BS) == (cts_a[0, c, h, w], sl_a[0, c, h, w])
                assert (sb, pb * lb.BS) == (cts_b[0, c, h, w], sl_b[0, c, h, w])
