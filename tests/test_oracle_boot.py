"""CPU pins of the bootstrapping oracle (oracle/boot.py): the refresh that the
paper's deeper networks apply between blocks (Sec. 5, Evaluation Methodology).

Each pin checks the oracle against something other than itself: the direct
definition of the canonical embedding U0[l][j] = zeta^(5^l j) (a dense numpy
matrix), the oracle's own decode (slot convention), mpmath-free float64 sines,
exact integer decryption by CRT with Python integers, and the message that
went in.
"""
import cmath
import math

import numpy as np
import pytest

from oracle import _core as C
from oracle import boot, ckks


def u0_matrix(N):
    n = N // 2
    return np.array([[cmath.exp(1j * math.pi * (pow(5, l, 2 * N) * j) / N) for j in range(n)] for l in range(n)])


def brv(x, bits):
    return int(format(x, f"0{bits}b")[::-1], 2) if bits else 0


def dense_group(N, stages, inverse):
    n = N // 2
    M = np.zeros((n, n), dtype=complex)
    for o in range(n):
        for i in range(n):
            e = boot.group_entry(N, stages, inverse, o, i)
            if e is not None:
                M[o, i] = cmath.exp(1j * math.pi * e[0] / N) / 2 ** e[1]
    return M


def crt_coef(pr, sk, ct):
    """c0 + c1 s over every limb of ct, recombined exactly (centred integers)."""
    lv = ct.level
    qs = [pr.moduli[i] for i in range(lv + 1)]
    Q = math.prod(qs)
    res = [pr.intt(C.vec_add(ct.c0[i], C.vec_mul(ct.c1[i], sk.ntt[i], q), q), i) for i, q in enumerate(qs)]
    out = []
    for j in range(pr.N):
        x = sum(int(res[i][j]) * (Q // q) * pow((Q // q) % q, -1, q) for i, q in enumerate(qs)) % Q
        out.append(x - Q if x > Q // 2 else x)
    return out


def crt_slots(pr, sk, ct):
    """Complex slot values u / scale of ct, decrypted over all its limbs."""
    t = np.array([float(v) for v in crt_coef(pr, sk, ct)])
    n = pr.N // 2
    return u0_matrix(pr.N) @ (t[:n] + 1j * t[n:]) / ct.scale


@pytest.mark.parametrize("logN", [3, 4, 5, 6])
def test_special_fft_stages_factor_the_embedding(logN):
    """S_k ... S_1 R = U0 with R the bit reversal; the inverse stages in the
    CoeffToSlot order give R U0^-1; every grouping gives the same products."""
    N = 1 << logN
    n = N // 2
    k = n.bit_length() - 1
    U0 = u0_matrix(N)
    R = np.zeros((n, n))
    for j in range(n):
        R[brv(j, k), j] = 1
    F = np.eye(n, dtype=complex)
    for s in range(1, k + 1):
        F = dense_group(N, [s], False) @ F
    assert np.abs(F @ R - U0).max() < 1e-12
    G = np.eye(n, dtype=complex)
    for s in range(k, 0, -1):
        G = dense_group(N, [s], True) @ G
    assert np.abs(G - R @ np.linalg.inv(U0)).max() < 1e-12
    for ng in range(1, k + 1):
        groups = boot.stage_groups(k, ng)
        assert sorted(s for g in groups for s in g) == list(range(1, k + 1))
        Gs = np.eye(n, dtype=complex)
        for grp in groups[::-1]:
            Gs = dense_group(N, sorted(grp, reverse=True), True) @ Gs
        Fs = np.eye(n, dtype=complex)
        for grp in groups:
            Fs = dense_group(N, sorted(grp), False) @ Fs
        assert np.abs(Gs - G).max() < 1e-12 and np.abs(Fs - F).max() < 1e-12


def test_slot_convention_matches_decode():
    """The oracle's decode is Re(U0 (t_lo + i t_hi)) / scale: the embedding the
    stages factor is the one the scheme encodes with."""
    for logN in (4, 6):
        N = 1 << logN
        t = np.random.default_rng(logN).integers(-1000, 1000, N)
        z = C.decode(t, logN, 1.0)
        u = u0_matrix(N) @ (t[:N // 2] + 1j * t[N // 2:])
        assert np.abs(z - u.real).max() < 1e-9


def test_cos_table_is_correctly_rounded_and_symmetric():
    N = 1 << 9
    tab = boot.cos_table(N)
    assert tab[0] == 1.0 and tab[N // 2] == 0.0
    for e in range(-3 * N, 3 * N, 7):
        c, s = boot.cos_pi(tab, N, e), boot.sin_pi(tab, N, e)
        a = math.pi * (e % (2 * N)) / N  # libm on the reduced angle: a few ulp of 1
        assert abs(c - math.cos(a)) <= 2.0 ** -50 and abs(s - math.sin(a)) <= 2.0 ** -50
    for e in (0, N // 2, N, 3 * N // 2):
        assert boot.cos_pi(tab, N, e) in (0.0, 1.0, -1.0) and boot.sin_pi(tab, N, e) in (0.0, 1.0, -1.0)


@pytest.mark.parametrize("logN,groups", [(6, 2), (7, 3), (8, 3)])
def test_real_form_diagonals_apply_the_transforms(logN, groups):
    """The CoeffToSlot diagonals, applied with plain rotations (np.roll) to
    (2 Re u, 2 Im u), give (pi / 2^(r-1)) R w with u = U0 w; the SlotToCoeff
    diagonals applied to (Re, Im) of R v give kappa Re(U0 v)."""
    N = 1 << logN
    n = N // 2
    k = n.bit_length() - 1
    pr = ckks.Params(logN, 18, 1, 50)
    bp = boot.BootParams(pr, groups, groups, 6)
    tab = boot.cos_table(N)
    rng = np.random.default_rng(logN)
    u = rng.normal(size=n) + 1j * rng.normal(size=n)

    def apply(d, vecs, n_out):
        outs = [np.zeros(n) for _ in range(n_out)]
        for (o, i, r), v in d.items():
            outs[o] += v * np.roll(vecs[i], -r)
        return outs

    vec = [2 * u.real, 2 * u.imag]
    for d in boot.cts_diagonals(pr, bp, tab):
        vec = apply(d, vec, 2)
    w = np.linalg.solve(u0_matrix(N), u)
    wb = np.array([w[brv(j, k)] for j in range(n)])
    sc = math.pi / 2 ** (bp.r - 1)
    assert np.abs(vec[0] - sc * wb.real).max() < 1e-11
    assert np.abs(vec[1] - sc * wb.imag).max() < 1e-11
    v = rng.normal(size=n) + 1j * rng.normal(size=n)
    vb = np.array([v[brv(j, k)] for j in range(n)])
    s_in = 2.0 ** 40
    vec = [vb.real, vb.imag]
    sds = boot.stc_diagonals(pr, bp, tab, s_in)
    for gi, d in enumerate(sds):
        vec = apply(d, vec, 1 if gi == len(sds) - 1 else 2)
    kappa = boot.stc_kappa(pr.moduli[0], s_in)
    want = kappa * (u0_matrix(N) @ v).real
    assert np.abs(vec[0] - want).max() < 1e-12 * np.abs(want).max() * n


def test_bsgs_decomposition():
    for offs in ([0], [-3, -1, 1, 3], list(range(-15, 16)), [8 * j for j in range(-7, 9)]):
        for n1 in (1, 2, 4, 8):
            dec = boot.bsgs_decompose(offs, n1)
            assert all(g + b == r for r, (g, b) in dec.items())
            assert all(b >= 0 for g, b in dec.values())
            assert len({b for g, b in dec.values()}) <= n1
            assert len({g for g, b in dec.values()}) <= -(-len(offs) // n1) + 1


def test_sparse_ternary_secret():
    for N, h in ((256, 16), (1024, 32), (1024, 1024)):
        s = boot.sparse_ternary(5, N, h)
        assert np.count_nonzero(s) == h and set(np.unique(s)) <= {-1, 0, 1}
        assert np.array_equal(s, boot.sparse_ternary(5, N, h))
        assert not np.array_equal(s, boot.sparse_ternary(6, N, h))
    # positions and signs are spread evenly over many seeds
    hits = np.zeros(64)
    signs = 0
    for seed in range(400):
        s = boot.sparse_ternary(seed, 64, 8)
        hits += s != 0
        signs += int(s.sum())
    assert hits.min() > 25 and hits.max() < 75 and abs(signs) < 150
    with pytest.raises(ValueError):
        boot.sparse_ternary(1, 16, 0)


def test_eval_mod_polynomial_and_double_angles():
    """cos of the Taylor polynomial after r double angles is sin(2 pi y)."""
    r = 6
    y = np.concatenate([np.arange(-16, 17) + e for e in (-0.01, -1e-4, 0.0, 1e-4, 0.01)])
    got = boot.eval_mod_plain(y, r)
    assert np.abs(got - np.sin(2 * np.pi * y)).max() < 1e-8
    I = np.round(y)
    eps = y - I
    assert np.abs(got / (2 * np.pi) - eps).max() < (2 * np.pi) ** 2 * 0.01 ** 3 / 6 + 1e-9


@pytest.fixture(scope="module")
def small():
    logN = 8
    pr = ckks.Params(logN, 19, 4, 50)
    bp = boot.BootParams(pr, 3, 3, 6)
    keys = boot.SparseKeySet(pr, 7, 16, rot_steps=boot.boot_rotation_steps(pr, bp), relin=True, conj=True)
    return pr, bp, keys


def test_mod_raise_decrypts_to_m_plus_q0_I(small):
    pr, bp, keys = small
    z = np.random.default_rng(2).uniform(-1, 1, pr.N // 2)
    ct = ckks.encrypt(pr, keys.sk, ckks.encode(pr, z, 0, 2.0 ** 45), 3, 0)
    x = boot.mod_raise(pr, ct, 4)
    q0 = pr.moduli[0]
    c0 = [int(v) for v in C.centre(pr.intt(ct.c0[0], 0), q0)]
    c1 = [int(v) for v in C.centre(pr.intt(ct.c1[0], 0), q0)]
    s = [int(v) for v in keys.sk.coef]
    t = list(c0)
    for i in range(pr.N):
        for j in range(pr.N):
            if c1[i] and s[j]:
                k = i + j
                if k < pr.N:
                    t[k] += c1[i] * s[j]
                else:
                    t[k - pr.N] -= c1[i] * s[j]
    assert crt_coef(pr, keys.sk, x) == t
    m = ckks.decrypt_coef(pr, keys.sk, ct)
    I = [(t[j] - int(m[j])) // q0 for j in range(pr.N)]
    assert all((t[j] - int(m[j])) % q0 == 0 for j in range(pr.N))
    assert max(abs(v) for v in I) <= (16 + 1) // 2 + 1
    assert x.scale == float(q0) and x.level == 4


def test_conjugation_and_parts(small):
    pr, bp, keys = small
    z = np.random.default_rng(3).uniform(-1, 1, pr.N // 2)
    ct = ckks.encrypt(pr, keys.sk, ckks.encode(pr, z, 0, 2.0 ** 45), 4, 0)
    x = boot.mod_raise(pr, ct, 6)
    u = crt_slots(pr, keys.sk, x)
    cj = boot.conjugate(pr, keys, x)
    assert np.abs(crt_slots(pr, keys.sk, cj) - np.conj(u)).max() < 1e-9
    re = ckks.add(pr, x, cj)
    im = boot.mul_monomial(pr, boot.sub(pr, x, cj), pr.N // 2, -1)
    assert np.abs(crt_slots(pr, keys.sk, re) - 2 * u.real).max() < 1e-9
    assert np.abs(crt_slots(pr, keys.sk, im) - 2 * u.imag).max() < 1e-9


@pytest.mark.parametrize("hoist", ["single", "double"])
def test_he_lintrans_matches_the_plain_product(small, hoist):
    pr, bp, keys = small
    n = pr.N // 2
    rng = np.random.default_rng(4)
    diags = {}
    for (o, i) in ((0, 0), (0, 1), (1, 1)):
        for r in (-6, -2, 0, 2, 4, 6):
            diags[(o, i, r)] = rng.uniform(-1, 1, n)
    n1 = 2
    steps = boot.lintrans_steps(diags, n, n1)
    for st in steps:
        keys.add_rotation(st)
    lv = 5
    zs = [rng.uniform(-1, 1, n) for _ in range(2)]
    cts = [ckks.encrypt(pr, keys.sk, ckks.encode(pr, z, lv, 2.0 ** 40), 5, i) for i, z in enumerate(zs)]
    out = boot.he_lintrans(pr, keys, cts, diags, 2, n1, hoist=hoist)
    for o in range(2):
        want = sum(v * np.roll(zs[i], -r) for (oo, i, r), v in diags.items() if oo == o)
        got = ckks.decrypt(pr, keys.sk, out[o])
        assert out[o].level == lv - 1 and out[o].scale == 2.0 ** 40
        assert np.abs(got - want).max() < 1e-6


def test_eval_mod_homomorphic_matches_plain(small):
    pr, bp, keys = small
    n = pr.N // 2
    rng = np.random.default_rng(5)
    y = rng.integers(-8, 9, n) + rng.uniform(-0.002, 0.002, n)
    lv = 12
    x = (math.pi / 2 ** (bp.r - 1)) * y
    ct = ckks.encrypt(pr, keys.sk, ckks.encode(pr, x, lv, float(pr.moduli[0])), 6, 0)
    out = boot.eval_mod(pr, keys, ct, bp.r)
    assert out.level == lv - 5 - bp.r
    got = crt_slots(pr, keys.sk, out).real
    assert np.abs(got - boot.eval_mod_plain(y, bp.r)).max() < 1e-7
    assert np.abs(got - np.sin(2 * np.pi * y)).max() < 1e-7


def test_bootstrap_refreshes_the_message(small):
    """A level-0 ciphertext comes back at level top - depth holding the same
    slot values (bound: the sine's cubic term for coefficients of this size,
    about 4e-4 at N = 2^8 and scale_in = q_0 / 2^5, plus noise)."""
    pr, bp, keys = small
    z = np.random.default_rng(6).uniform(-1, 1, pr.N // 2)
    ct = ckks.encrypt(pr, keys.sk, ckks.encode(pr, z, 0, 2.0 ** 45), 7, 0)
    out = boot.bootstrap(pr, keys, ct, bp)
    assert out.level == bp.top - bp.depth == pr.L - 17
    assert np.abs(ckks.decrypt(pr, keys.sk, out) - z).max() < 4e-4


def test_bootstrap_single_hoisted_refreshes_the_message(small):
    """The refresh with square-root baby steps (ratio 1) and a ModDown per
    rotation (single hoisting) also returns the message."""
    pr, _, keys = small
    bp = boot.BootParams(pr, 3, 3, 6, baby_ratio=1, double_hoist=False)
    for st in boot.boot_rotation_steps(pr, bp):
        keys.add_rotation(st)
    z = np.random.default_rng(7).uniform(-1, 1, pr.N // 2)
    ct = ckks.encrypt(pr, keys.sk, ckks.encode(pr, z, 0, 2.0 ** 45), 8, 0)
    out = boot.bootstrap(pr, keys, ct, bp)
    assert out.level == pr.L - 17
    assert np.abs(ckks.decrypt(pr, keys.sk, out) - z).max() < 4e-4


def test_bootstrap_in_fourteen_levels(small):
    """Two CoeffToSlot groups, 5 + 5 EvalMod levels and two SlotToCoeff groups:
    a refresh in 14 levels (the budget the paper's refresh spends) that still
    returns the message at N = 2^8."""
    pr, _, keys = small
    bp = boot.BootParams(pr, 2, 2, 5)
    assert bp.depth == 14
    for st in boot.boot_rotation_steps(pr, bp):
        keys.add_rotation(st)
    z = np.random.default_rng(9).uniform(-1, 1, pr.N // 2)
    ct = ckks.encrypt(pr, keys.sk, ckks.encode(pr, z, 0, 2.0 ** 45), 10, 0)
    out = boot.bootstrap(pr, keys, ct, bp)
    assert out.level == pr.L - 14
    assert np.abs(ckks.decrypt(pr, keys.sk, out) - z).max() < 4e-4


def test_prepare_reaches_level_zero_at_the_input_scale(small):
    """prepare keeps the slot values and lands at level 0 with the requested scale."""
    pr, bp, keys = small
    z = np.random.default_rng(11).uniform(-2, 2, pr.N // 2)
    ct = ckks.encrypt(pr, keys.sk, ckks.encode(pr, z, 9, 2.0 ** 48), 12, 0)
    out = boot.prepare(pr, ct, 2.0 ** 44)
    assert out.level == 0 and out.scale == 2.0 ** 44
    assert np.abs(ckks.decrypt(pr, keys.sk, out) - z).max() < 1e-9
    with pytest.raises(ValueError):
        boot.prepare(pr, out, 2.0 ** 44)


def test_encapsulated_refresh_with_a_dense_secret():
    """Sparse-secret encapsulation: the network's secret is the dense ternary one
    (ckks.KeySet); the refresh switches its input to a sparse secret for
    ModRaise and back to the dense secret at level top.  The raised ciphertext
    decrypts (exactly, by CRT) under the dense secret to m + q_0 I with I
    bounded by the sparse secret's weight, and the refresh returns the message."""
    logN = 8
    pr = ckks.Params(logN, 19, 4, 50)
    bp = boot.BootParams(pr, 3, 3, 6)
    keys = ckks.KeySet(pr, 17, rot_steps=boot.boot_rotation_steps(pr, bp), relin=True)
    boot.add_conjugation(keys)
    enc = boot.Encapsulation(keys, 18, 16)
    assert np.count_nonzero(keys.sk.coef) > pr.N // 2  # dense
    z = np.random.default_rng(14).uniform(-1, 1, pr.N // 2)
    ct = ckks.encrypt(pr, keys.sk, ckks.encode(pr, z, 0, 2.0 ** 45), 15, 0)
    # the raise under the sparse secret, switched back: t = m + q_0 I with small I
    x = boot.key_switch(pr, boot.mod_raise(pr, boot.key_switch(pr, ct, enc.to_sparse), 6), enc.to_dense)
    t = crt_coef(pr, keys.sk, x)
    m = ckks.decrypt_coef(pr, keys.sk, ct)
    q0 = pr.moduli[0]
    I = [round((t[j] - int(m[j])) / q0) for j in range(pr.N)]
    assert max(abs(v) for v in I) <= (16 + 1) // 2 + 1
    assert max(abs(t[j] - int(m[j]) - q0 * I[j]) for j in range(pr.N)) < 2 ** 20  # key-switch noise only
    out = boot.bootstrap(pr, keys, ct, bp, encaps=enc)
    assert np.abs(ckks.decrypt(pr, keys.sk, out) - z).max() < 4e-4
    # without encapsulation, ModRaise under the dense secret exceeds the sparse secret's bound
    t2 = crt_coef(pr, keys.sk, boot.mod_raise(pr, ct, 6))
    assert max(abs(round((t2[j] - int(m[j])) / q0)) for j in range(pr.N)) > (16 + 1) // 2 + 1


@pytest.mark.parametrize("logN", [4, 6, 8])
def test_complex_encode_matches_the_embedding(logN):
    """encode_complex(z) is the real polynomial whose slot vector U0 (m_lo + i m_hi)
    is scale z (within rounding), and equals encode for real z."""
    N = 1 << logN
    n = N // 2
    rng = np.random.default_rng(logN)
    z = rng.uniform(-1, 1, n) + 1j * rng.uniform(-1, 1, n)
    m = C.encode_complex(z, logN, 2.0 ** 30)
    u = u0_matrix(N) @ (m[:n] + 1j * m[n:]) / 2.0 ** 30
    assert np.abs(u - z).max() < n * 2.0 ** -30
    zr = rng.uniform(-1, 1, n)
    assert np.array_equal(C.encode_complex(zr + 0j, logN, 2.0 ** 40), C.encode(zr, logN, 2.0 ** 40))


@pytest.mark.parametrize("logN,groups", [(6, 2), (8, 3)])
def test_complex_form_diagonals_apply_the_transforms(logN, groups):
    """The complex-form CoeffToSlot diagonals applied with np.roll to u give
    (pi / 2^r) R U0^-1 u, and the SlotToCoeff diagonals applied to R v give
    kappa U0 v."""
    N = 1 << logN
    n = N // 2
    k = n.bit_length() - 1
    pr = ckks.Params(logN, 18, 1, 50)
    bp = boot.BootParams(pr, groups, groups, 6, form="complex")
    tab = boot.cos_table(N)
    rng = np.random.default_rng(logN + 1)

    def apply(d, v):
        out = np.zeros(n, dtype=complex)
        for (o, i, r), dv in d.items():
            out += dv * np.roll(v, -r)
        return out

    u = rng.normal(size=n) + 1j * rng.normal(size=n)
    v = u
    for d in boot.cts_diagonals_complex(pr, bp, tab):
        v = apply(d, v)
    w = np.linalg.solve(u0_matrix(N), u)
    wb = np.array([w[brv(j, k)] for j in range(n)])
    assert np.abs(v - math.pi / 2 ** bp.r * wb).max() < 1e-11
    y = rng.normal(size=n) + 1j * rng.normal(size=n)
    v = np.array([y[brv(j, k)] for j in range(n)])
    s_in = 2.0 ** 40
    for d in boot.stc_diagonals_complex(pr, bp, tab, s_in):
        v = apply(d, v)
    want = boot.stc_kappa(pr.moduli[0], s_in) * (u0_matrix(N) @ y)
    assert np.abs(v - want).max() < 1e-12 * np.abs(want).max() * n


def test_bootstrap_real_form_refreshes_the_message(small):
    """The real form (transforms on the pair (re, im) of real-slot ciphertexts,
    the split before CoeffToSlot) returns the message at the same level as the
    complex form (the default)."""
    pr, _, keys = small
    bp = boot.BootParams(pr, 3, 3, 6, form="real")
    for st in boot.boot_rotation_steps(pr, bp):
        keys.add_rotation(st)
    z = np.random.default_rng(16).uniform(-1, 1, pr.N // 2)
    ct = ckks.encrypt(pr, keys.sk, ckks.encode(pr, z, 0, 2.0 ** 45), 18, 0)
    out = boot.bootstrap(pr, keys, ct, bp)
    assert out.level == pr.L - 17
    assert np.abs(ckks.decrypt(pr, keys.sk, out) - z).max() < 4e-4
