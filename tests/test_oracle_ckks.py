"""Pins of the oracle's RNS-CKKS operations: exact CRT identities for the base
conversions, ModDown and rescale (checked with Python big integers), and
decryption identities for key switching and rotation (Eq. 1)."""
from math import prod

import numpy as np
import pytest

from oracle import _core as C
from oracle import ckks


def crt(residues, moduli):
    """Centred integer from residues (Python ints)."""
    Q = prod(moduli)
    x = 0
    for r, q in zip(residues, moduli):
        Qh = Q // q
        x += int(r) * Qh * pow(Qh % q, -1, q)
    x %= Q
    return x - Q if x > Q // 2 else x


@pytest.fixture(scope="module")
def pr():
    return ckks.Params(5, 5, 2, 36)


def test_centred_bconv_identity(pr):
    rng = np.random.default_rng(0)
    src = [1, 2]
    coef = [rng.integers(0, pr.moduli[i], pr.N, dtype=np.uint64) for i in src]
    dst = [0, 3, 4, pr.p_index(0), pr.p_index(1)]
    out = ckks.centred_bconv(pr, coef, src, dst)
    B = prod(pr.moduli[i] for i in src)
    for n in range(pr.N):
        x = crt([coef[0][n], coef[1][n]], [pr.moduli[i] for i in src])
        Y = 0
        for pos, i in enumerate(src):
            bi = pr.moduli[i]
            yi = int(coef[pos][n]) * pow((B // bi) % bi, -1, bi) % bi
            yi = yi - bi if yi > bi // 2 else yi
            Y += yi * (B // bi)
        assert (Y - x) % B == 0 and abs((Y - x) // B) <= 1
        for t in dst:
            assert int(out[t][n]) == Y % pr.moduli[t]


def test_mod_down_is_rounded_division(pr):
    """ModDown(x) = (x - Y) / P with Y = centred conversion of [x]_P (an exact integer identity)."""
    rng = np.random.default_rng(1)
    level = 3
    limbs = pr.ks_limbs(level)
    xc = {t: rng.integers(0, pr.moduli[t], pr.N, dtype=np.uint64) for t in limbs}
    x = {t: pr.ntt(xc[t], t) for t in limbs}
    out = ckks.mod_down(pr, x, level)
    outc = [pr.intt(out[i], i) for i in range(level + 1)]
    ps = [pr.p_index(j) for j in range(pr.k)]
    P = pr.P
    Q = prod(pr.moduli[i] for i in range(level + 1))
    for n in range(pr.N):
        X = crt([xc[t][n] for t in limbs], [pr.moduli[t] for t in limbs])
        Y = 0
        for t in ps:
            pj = pr.moduli[t]
            yj = int(xc[t][n]) * pow((P // pj) % pj, -1, pj) % pj
            yj = yj - pj if yj > pj // 2 else yj
            Y += yj * (P // pj)
        assert (X - Y) % P == 0
        want = (X - Y) // P
        got = crt([outc[i][n] for i in range(level + 1)], [pr.moduli[i] for i in range(level + 1)])
        assert (got - want) % Q == 0
        # and it is round(X / P) up to the conversion error |u| <= k/2
        assert abs(want - (2 * X + P) // (2 * P)) <= pr.k // 2 + 1


def test_rescale_is_rounded_division(pr):
    rng = np.random.default_rng(2)
    lv = 3
    c = [rng.integers(0, pr.moduli[t], pr.N, dtype=np.uint64) for t in range(lv + 1)]
    ct = ckks.Ciphertext(np.stack([pr.ntt(c[t], t) for t in range(lv + 1)]),
                         np.stack([pr.ntt(c[t], t) for t in range(lv + 1)]), lv, 1.0)
    out = ckks.rescale(pr, ct)
    ql = pr.moduli[lv]
    outc = [pr.intt(out.c0[i], i) for i in range(lv)]
    for n in range(pr.N):
        X = crt([c[t][n] for t in range(lv + 1)], pr.moduli[:lv + 1])
        r = int(c[lv][n]) % ql
        r = r - ql if r > ql // 2 else r
        want = (X - r) // ql
        assert (X - r) % ql == 0
        got = crt([outc[i][n] for i in range(lv)], pr.moduli[:lv])
        assert got == want


@pytest.fixture(scope="module")
def keyed():
    pr = ckks.Params(7, 4, 2, 40)
    keys = ckks.KeySet(pr, 5, rot_steps=[1, 2, 5, -3, 32], relin=True)
    return pr, keys


def test_encrypt_decrypt(keyed):
    pr, keys = keyed
    z = np.random.default_rng(3).uniform(-1, 1, pr.N // 2)
    ct = ckks.encrypt(pr, keys.sk, ckks.encode(pr, z, pr.L, 2.0 ** 30), 1, 0)
    assert np.abs(ckks.decrypt(pr, keys.sk, ct) - z).max() < 1e-6
    # b + a s = m + e exactly, with e the centred binomial noise
    m = C.encode(z, pr.logN, 2.0 ** 30)
    e = ckks.decrypt_coef(pr, keys.sk, ct) - m
    assert np.abs(e).max() <= 21


def test_switch_key_decrypts_under_source(keyed):
    """Key switching identity: KS(c) = (d0, d1) with d0 + d1 s_dst ~ c s_src."""
    pr, keys = keyed
    lv = pr.L
    rng = np.random.default_rng(4)
    c = np.stack([rng.integers(0, pr.moduli[t], pr.N, dtype=np.uint64) for t in range(lv + 1)])
    d0, d1 = ckks.key_switch_ext(pr, ckks.mod_up(pr, c, lv), keys.relin, lv)
    for t in range(lv + 1):
        q = pr.moduli[t]
        s2 = C.vec_mul(keys.sk.ntt[t], keys.sk.ntt[t], q)
        lhs = C.vec_add(d0[t], C.vec_mul(d1[t], keys.sk.ntt[t], q), q)
        diff = C.centre(pr.intt(C.vec_sub(lhs, C.vec_mul(c[t], s2, q), q), t), q)
        assert np.abs(diff).max() < 2 ** 14


@pytest.mark.parametrize("r", [1, 2, 5, -3, 32])
def test_rotation_decrypts_to_shifted_slots(keyed, r):
    pr, keys = keyed
    z = np.random.default_rng(6).uniform(-1, 1, pr.N // 2)
    ct = ckks.encrypt(pr, keys.sk, ckks.encode(pr, z, pr.L, 2.0 ** 30), 1, 1)
    out = ckks.decrypt(pr, keys.sk, ckks.rotate(pr, keys, ct, r))
    assert np.abs(out - np.roll(z, -r)).max() < 1e-4


def test_hoisted_rotation_equals_plain_rotation(keyed):
    pr, keys = keyed
    z = np.random.default_rng(7).uniform(-1, 1, pr.N // 2)
    ct = ckks.encrypt(pr, keys.sk, ckks.encode(pr, z, pr.L, 2.0 ** 30), 1, 2)
    ext = ckks.mod_up(pr, ct.c1, ct.level)
    for r in [1, 5]:
        a = ckks.rotate_ext(pr, keys, ct, ext, r)
        b = ckks.rotate(pr, keys, ct, r)
        assert np.array_equal(a.as_array(), b.as_array())


def test_pmult_rescale_and_cmult(keyed):
    pr, keys = keyed
    rng = np.random.default_rng(8)
    z = rng.uniform(-1, 1, pr.N // 2)
    w = rng.uniform(-1, 1, pr.N // 2)
    ct = ckks.encrypt(pr, keys.sk, ckks.encode(pr, z, pr.L, 2.0 ** 30), 1, 3)
    pt = ckks.encode(pr, w, pr.L, float(pr.q[pr.L]))
    out = ckks.rescale(pr, ckks.pmult(pr, ct, pt))
    assert out.level == pr.L - 1 and out.scale == 2.0 ** 30
    assert np.abs(ckks.decrypt(pr, keys.sk, out) - z * w).max() < 1e-5
    sq = ckks.rescale(pr, ckks.cmult_relin(pr, keys, ct, ct))
    assert np.abs(ckks.decrypt(pr, keys.sk, sq) - z * z).max() < 1e-3


def test_tensor_decrypts_to_the_negacyclic_product(keyed):
    """The unrelinearised product: d0 + d1 s + d2 s^2 on q_0, back in the
    coefficient domain, equals the schoolbook negacyclic product (Python
    integers) of the two decrypted polynomials, exactly mod q_0."""
    from oracle import _core as C
    pr, keys = keyed
    rng = np.random.default_rng(21)
    x = ckks.encrypt(pr, keys.sk, ckks.encode(pr, rng.uniform(-1, 1, pr.N // 2), pr.L, 2.0 ** 12), 3, 0)
    y = ckks.encrypt(pr, keys.sk, ckks.encode(pr, rng.uniform(-1, 1, pr.N // 2), pr.L, 2.0 ** 12), 3, 1)
    d0, d1, d2, lv, scale = ckks.tensor(pr, x, y)
    assert lv == pr.L and scale == 2.0 ** 24
    q, N = pr.moduli[0], pr.N
    sv = [int(v) for v in keys.sk.ntt[0]]
    dec = np.array([(int(d0[0][i]) + int(d1[0][i]) * sv[i] + int(d2[0][i]) * sv[i] * sv[i]) % q for i in range(N)],
                   dtype=np.uint64)
    got = [int(v) for v in C.centre(pr.intt(dec, 0), q)]
    mx = [int(v) for v in ckks.decrypt_coef(pr, keys.sk, x)]
    my = [int(v) for v in ckks.decrypt_coef(pr, keys.sk, y)]
    prod = [0] * N
    for i in range(N):
        for j in range(N):
            k = i + j
            if k < N:
                prod[k] += mx[i] * my[j]
            else:
                prod[k - N] -= mx[i] * my[j]
    want = [((v + q // 2) % q) - q // 2 for v in prod]
    assert got == want


def test_products_summed_before_one_relinearisation(keyed):
    """Two products summed in tensor form and relinearised once decrypt to
    z1 w1 + z2 w2, like the sum of two relinearised products."""
    pr, keys = keyed
    rng = np.random.default_rng(22)
    z = rng.uniform(-1, 1, (4, pr.N // 2))
    c = [ckks.encrypt(pr, keys.sk, ckks.encode(pr, z[i], pr.L, 2.0 ** 30), 4, i) for i in range(4)]
    lazy = ckks.relinearize(pr, keys, ckks.tensor_add(pr, ckks.tensor(pr, c[0], c[1]), ckks.tensor(pr, c[2], c[3])))
    eager = ckks.add(pr, ckks.cmult_relin(pr, keys, c[0], c[1]), ckks.cmult_relin(pr, keys, c[2], c[3]))
    want = z[0] * z[1] + z[2] * z[3]
    for ct in (lazy, eager):
        assert np.abs(ckks.decrypt(pr, keys.sk, ckks.rescale(pr, ct)) - want).max() < 1e-3


def test_double_hoisted_rotation_moddown_equals_rotation(keyed):
    """A rotation kept on Q P and brought down alone equals the rotation exactly;
    the lifted ciphertext comes back exactly; a double-hoisted sum decrypts to
    the sum of the products within the noise."""
    pr, keys = keyed
    z = np.random.default_rng(4).uniform(-1, 1, pr.N // 2)
    ct = ckks.encrypt(pr, keys.sk, ckks.encode(pr, z, pr.L, 2.0 ** 30), 2, 0)
    ext = ckks.mod_up(pr, ct.c1, ct.level)
    for r in (1, 5):
        Vb, Va = ckks.rotate_ext_qp(pr, keys, ct, ext, r)
        got = ckks.mod_down_ct(pr, Vb, Va, ct.level, ct.scale)
        want = ckks.rotate_ext(pr, keys, ct, ext, r)
        assert np.array_equal(got.as_array(), want.as_array())
    Lb, La = ckks.lift_qp(pr, ct)
    assert np.array_equal(ckks.mod_down_ct(pr, Lb, La, ct.level, ct.scale).as_array(), ct.as_array())
    # a sum of double-hoisted products brought down once: Rot(ct,1) w1 + ct w2
    w1 = np.random.default_rng(5).uniform(-1, 1, pr.N // 2)
    w2 = np.random.default_rng(6).uniform(-1, 1, pr.N // 2)
    dw = float(pr.moduli[pr.L])
    terms = [(ckks.rotate_ext_qp(pr, keys, ct, ext, 1), ckks.encode_qp(pr, w1, pr.L, dw)),
             (ckks.lift_qp(pr, ct), ckks.encode_qp(pr, w2, pr.L, dw))]
    ab, aa = ckks.mac_qp(pr, pr.L, terms)
    y = ckks.decrypt(pr, keys.sk, ckks.rescale(pr, ckks.mod_down_ct(pr, ab, aa, pr.L, ct.scale * dw)))
    assert np.abs(y - (np.roll(z, -1) * w1 + z * w2)).max() < 1e-5


def test_mod_down_rescale_is_rounded_division(pr):
    """ModDown and rescale in one conversion: the result is (X - Y) / (q_l P) with
    Y the centred conversion of [X]_{q_l P} (an exact integer identity), hence
    round(X / (q_l P)) up to the conversion error (|u| <= (k + 1) / 2)."""
    rng = np.random.default_rng(4)
    level = 3
    limbs = pr.ks_limbs(level)
    xc = {t: rng.integers(0, pr.moduli[t], pr.N, dtype=np.uint64) for t in limbs}
    x = {t: pr.ntt(xc[t], t) for t in limbs}
    out = ckks.mod_down_rescale(pr, x, level)
    outc = [pr.intt(out[i], i) for i in range(level)]
    src = [level] + [pr.p_index(j) for j in range(pr.k)]
    B = prod(pr.moduli[t] for t in src)
    Q = prod(pr.moduli[i] for i in range(level))
    for n in range(pr.N):
        X = crt([xc[t][n] for t in limbs], [pr.moduli[t] for t in limbs])
        Y = 0
        for t in src:
            b = pr.moduli[t]
            y = int(xc[t][n]) * pow((B // b) % b, -1, b) % b
            y = y - b if y > b // 2 else y
            Y += y * (B // b)
        assert (X - Y) % B == 0
        want = (X - Y) // B
        got = crt([outc[i][n] for i in range(level)], [pr.moduli[i] for i in range(level)])
        assert (got - want) % Q == 0
        assert abs(want - (2 * X + B) // (2 * B)) <= (pr.k + 1) // 2 + 1


def test_mod_down_rescale_close_to_the_two_steps(pr):
    """On a ciphertext-sized input the one-step division and ModDown followed by
    rescale differ by at most a few units (two roundings against one)."""
    rng = np.random.default_rng(5)
    level = 3
    limbs = pr.ks_limbs(level)
    xc = {t: rng.integers(0, pr.moduli[t], pr.N, dtype=np.uint64) for t in limbs}
    x = {t: pr.ntt(xc[t], t) for t in limbs}
    one = ckks.mod_down_rescale(pr, x, level)
    md = ckks.mod_down(pr, x, level)
    two = ckks.rescale(pr, ckks.Ciphertext(md, md, level, 1.0)).c0
    Q = prod(pr.moduli[i] for i in range(level))
    for n in range(0, pr.N, 7):
        a = crt([int(pr.intt(one[i], i)[n]) for i in range(level)], pr.moduli[:level])
        b = crt([int(pr.intt(two[i], i)[n]) for i in range(level)], pr.moduli[:level])
        d = (a - b) % Q
        assert min(d, Q - d) <= pr.k + 2
