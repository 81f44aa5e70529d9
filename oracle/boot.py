"""CKKS bootstrapping: the ciphertext refresh that the paper's deeper networks
(SqueezeNet, ResNet18, MobileNet) need between convolution blocks (Sec. 5,
Evaluation Methodology: NEXUS-style bootstrapping, 14 levels per refresh).

Test infrastructure only (see oracle/__init__.py).

The paper adopts an existing bootstrapping and does not print its steps.  This
module writes out the standard CKKS refresh (ModRaise, CoeffToSlot, EvalMod,
SlotToCoeff) for this library's real-slot encoding, in the order below, with
every constant defined so that it is one correctly rounded double or one IEEE
operation on such doubles.

Notation: N ring degree, n = N/2 slots, zeta = exp(i pi / N), slot l is the
evaluation at zeta^(5^l) (the encoding of ckks.py).  A real polynomial t has the
complex slot vector u = U0 (t_lo + i t_hi), U0[l][j] = zeta^(5^l j) (j < n),
t_lo = (t_0 .. t_{n-1}), t_hi = (t_n .. t_{N-1}), because zeta^(5^l n) = i.

 1. ModRaise: a level-0 ciphertext (modulus q_0) is read as centred integers and
    reduced modulo every prime up to `top`; it decrypts to t = m + q_0 I with a
    small integer polynomial I (|I_j| <= (h + 1) / 2 for a secret of weight h).
    Its declared scale is q_0, so its slot values are u / q_0.
 2. Real and imaginary parts: with the conjugation sigma_{-1} (Galois element
    2N - 1, one key switch), ct_re = ct + sigma(ct) holds 2 Re(u / q_0) and
    ct_im = -X^(N/2) (ct - sigma(ct)) holds 2 Im(u / q_0) (X^(N/2) multiplies
    every slot by i).  Both are real-slot ciphertexts.
 3. CoeffToSlot: U0 = S_k ... S_1 R (R the bit reversal of k = log2 n bits,
    S_s the butterfly stages of the decimation-in-time special FFT, see
    stage_entry).  Applying S_1^-1 ... S_k^-1 (S_k^-1 first) to u gives R w,
    w = t_lo + i t_hi, in bit-reversed order, which EvalMod (slot-wise) does not
    mind and SlotToCoeff takes as it is.  The stages are merged into groups of
    consecutive stages; each group is one level: a plaintext-matrix product on
    the pair (re, im) by the diagonal method with baby / giant steps
    (he_lintrans), in real form (re', im') = (Re G re - Im G im, Im G re + Re G im).
    The factor 1/2 of step 2 and the EvalMod pre-scaling pi / 2^(r-1) are
    folded into the first group applied.
 4. EvalMod, on both parts: the slot values y = t_j / q_0 = I_j + eps_j become
    sin(2 pi y) ~ 2 pi eps_j: x = 2 pi (y - 1/4) / 2^r, cos x by its Taylor
    polynomial of degree 16 (terms in w = x^2 up to w^8), then r double angles
    c <- 2 c^2 - 1, which give cos(2 pi (y - 1/4)) = sin(2 pi y).
 5. SlotToCoeff: S_k ... S_1 (S_1 first) on the complex vector re + i im,
    grouped like step 3; the last group keeps only the real part (the message
    has real slots).  The factor q_0 / (2 pi scale_in) is folded into the first
    group applied, so the result decrypts to the input's slot values.

The secret must be sparse (weight h, sparse_ternary) for I to stay within the
range the Taylor polynomial covers.  Levels used: n_cts + 5 + r + n_stc.
"""
import math
from fractions import Fraction

import mpmath
import numpy as np

from . import _core as C
from . import ckks

KIND_SK_SPARSE = 6


# ---------------------------------------------------------------------------
# Sparse ternary secret
# ---------------------------------------------------------------------------

def sparse_ternary(seed, N, h):
    """h distinct nonzero positions with signs, drawn with a partial
    Fisher-Yates shuffle: for i < h, word w_i = word(seed, tag(6), i) gives
    j = i + floor((w_i >> 1) (N - i) / 2^63), positions i and j of the index
    list are swapped, and s[index[i]] = -1 if w_i is odd else +1."""
    if not 0 < h <= N:
        raise ValueError("hamming weight must be in [1, N]")
    idx = list(range(N))
    s = np.zeros(N, dtype=np.int64)
    tg = ckks.tag(KIND_SK_SPARSE)
    for i in range(h):
        w = C.word(seed, tg, i)
        j = i + (((w >> 1) * (N - i)) >> 63)
        idx[i], idx[j] = idx[j], idx[i]
        s[idx[i]] = -1 if (w & 1) else 1
    return s


class SparseKeySet(ckks.KeySet):
    """KeySet whose secret is sparse_ternary(seed, N, h); switching keys as in
    ckks.KeySet (same random streams), plus the conjugation key."""

    def __init__(self, pr, seed, h, rot_steps=(), relin=False, conj=False):
        self.pr = pr
        self.seed = seed
        sk = ckks.SecretKey.__new__(ckks.SecretKey)
        sk.coef = sparse_ternary(seed, pr.N, h)
        sk.ntt = ckks.signed_to_ntt(pr, sk.coef, range(len(pr.moduli)))
        self.sk = sk
        self.rot = {}
        for r in sorted({r % (pr.N // 2) for r in rot_steps} - {0}):
            self.add_rotation(r)
        self.relin = None
        if relin:
            s2 = np.stack([C.vec_mul(sk.ntt[t], sk.ntt[t], m) for t, m in enumerate(pr.moduli)])
            self.relin = ckks.SwitchKey(pr, seed, 0, s2, sk.ntt)
        if conj:
            add_conjugation(self)


# Object tags of the two encapsulation keys (Galois elements are odd and below
# 2N, the relinearisation key is 0, so the even values 2N and 2N + 2 are free).
def swk_obj_to_sparse(pr):
    return 2 * pr.N


def swk_obj_to_dense(pr):
    return 2 * pr.N + 2


class Encapsulation:
    """Sparse-secret encapsulation of a refresh: the network keeps a dense secret
    s (ckks.KeySet) and the refresh borrows a sparse secret s' of weight h only
    for ModRaise.  Keys: s -> s' (object 2N) and s' -> s (object 2N + 2), both
    from the dense key set's seed, in ckks.SwitchKey's form."""

    def __init__(self, keys, sparse_seed, h):
        pr = keys.pr
        coef = sparse_ternary(sparse_seed, pr.N, h)
        self.s_sparse_ntt = ckks.signed_to_ntt(pr, coef, range(len(pr.moduli)))
        self.to_sparse = ckks.SwitchKey(pr, keys.seed, swk_obj_to_sparse(pr), keys.sk.ntt, self.s_sparse_ntt)
        self.to_dense = ckks.SwitchKey(pr, keys.seed, swk_obj_to_dense(pr), self.s_sparse_ntt, keys.sk.ntt)


def key_switch(pr, ct, key):
    """(c0, c1) under the key's source secret -> (c0 + d0, d1) under its
    destination secret, (d0, d1) the hybrid key switch of c1 (Sec. 2)."""
    d0, d1 = ckks.key_switch_ext(pr, ckks.mod_up(pr, ct.c1, ct.level), key, ct.level)
    c0 = np.stack([C.vec_add(ct.c0[t], d0[t], pr.moduli[t]) for t in range(ct.level + 1)])
    return ckks.Ciphertext(c0, d1, ct.level, ct.scale)


def conj_galois(pr):
    return 2 * pr.N - 1


def add_conjugation(keys):
    """Switching key for sigma_{2N-1} (its own inverse), object tag 2N - 1."""
    pr = keys.pr
    g = conj_galois(pr)
    if g in keys.rot:
        return
    perm = pr.automorph_perm(g)
    s_dst = np.stack([C.gather(keys.sk.ntt[t], perm) for t in range(len(pr.moduli))])
    keys.rot[g] = ckks.SwitchKey(pr, keys.seed, g, keys.sk.ntt, s_dst)


def conjugate(pr, keys, ct):
    """sigma_{-1}(ct): the slots' complex conjugate (Eq. 1's form with g = 2N - 1)."""
    g = conj_galois(pr)
    d0, d1 = ckks.key_switch_ext(pr, ckks.mod_up(pr, ct.c1, ct.level), keys.rot[g], ct.level)
    c0 = np.stack([C.vec_add(ct.c0[t], d0[t], pr.moduli[t]) for t in range(ct.level + 1)])
    return ckks.Ciphertext(ckks.automorph_ntt(pr, c0, g, ct.level), ckks.automorph_ntt(pr, d1, g, ct.level),
                           ct.level, ct.scale)


# ---------------------------------------------------------------------------
# Exact helpers
# ---------------------------------------------------------------------------

def mod_raise(pr, ct, top):
    """Level-0 ciphertext -> level `top`: centred residues mod q_0 on every prime."""
    if ct.level != 0:
        raise ValueError("ModRaise takes a level-0 ciphertext")
    q0 = pr.moduli[0]
    polys = []
    for c in (ct.c0, ct.c1):
        coef = C.centre(pr.intt(c[0], 0), q0)
        polys.append(ckks.signed_to_ntt(pr, coef, range(top + 1)))
    return ckks.Ciphertext(polys[0], polys[1], top, float(q0))


def prepare(pr, ct, scale_in):
    """A ciphertext at level >= 1 with declared scale s, brought to the
    refresh's input: level 0 at declared scale scale_in, same slot values.
    The ciphertext is dropped to level 1 (exact), multiplied by the integer
    B = nearest((scale_in / s) q_1) and rescaled by q_1."""
    if ct.level < 1:
        raise ValueError("prepare needs a level to rescale")
    x = drop_level(ct, ct.level - 1)
    B = ckks.nearest_int((scale_in / ct.scale) * float(pr.moduli[1]))
    r = ckks.rescale(pr, ckks.mul_int(pr, x, B))
    r.scale = scale_in
    return r


def mul_monomial(pr, ct, e, sign=1):
    """ct times sign X^e (exact; the scale is unchanged)."""
    m = np.zeros(pr.N, dtype=np.int64)
    m[e] = sign
    mm = ckks.signed_to_ntt(pr, m, range(ct.level + 1))
    c0 = np.stack([C.vec_mul(ct.c0[t], mm[t], pr.moduli[t]) for t in range(ct.level + 1)])
    c1 = np.stack([C.vec_mul(ct.c1[t], mm[t], pr.moduli[t]) for t in range(ct.level + 1)])
    return ckks.Ciphertext(c0, c1, ct.level, ct.scale)


def sub(pr, x, y):
    return ckks.add(pr, x, ckks.mul_int(pr, y, -1))


def drop_level(ct, times=1):
    """The ciphertext modulo Q_{level - times}: its first limbs (exact, same scale)."""
    lv = ct.level - times
    return ckks.Ciphertext(ct.c0[:lv + 1].copy(), ct.c1[:lv + 1].copy(), lv, ct.scale)


# ---------------------------------------------------------------------------
# The special FFT's stages and the twiddles as correctly rounded doubles
# ---------------------------------------------------------------------------

def cos_table(N):
    """cos(pi e / N) for e in [0, N/2], each the double nearest to the exact
    value (mpmath at 200 bits, then rounded once); e = N/2 gives 0 exactly."""
    with mpmath.workprec(200):
        tab = [float(mpmath.cos(mpmath.pi * e / N)) for e in range(N // 2)]
    return tab + [0.0]


def cos_pi(tab, N, e):
    """cos(pi e / N) for any integer e, from the table by the exact symmetries
    cos(-a) = cos(a), cos(a + 2 pi) = cos(a), cos(pi - a) = -cos(a)."""
    e %= 2 * N
    if e > N:
        e = 2 * N - e
    return -tab[N - e] if e > N // 2 else tab[e]


def sin_pi(tab, N, e):
    """sin(pi e / N) = cos(pi (N/2 - e) / N)."""
    return cos_pi(tab, N, N // 2 - e)


def tau(N, s, p):
    """Exponent of zeta in the twiddle of stage s (block m = 2^s) at position
    p < m/2: zeta_(m)^(5^p), zeta_(m) = exp(i pi / (2m)) = zeta^(N / (2m))."""
    m = 1 << s
    return (pow(5, p, 4 * m) * (N // (2 * m))) % (2 * N)


def stage_entry(N, s, inverse, o, i):
    """Entry (o, i) of S_s (or S_s^-1) as (exponent of zeta mod 2N, halvings),
    or None where it is zero.  S_s with m = 2^s, h = m/2, p = o mod m:
      p < h:  out[o] = in[o] + zeta^tau(p) in[o + h]
      p >= h: out[o] = in[o - h] - zeta^tau(p - h) in[o]
    and its inverse
      p < h:  in[o] = (out[o] + out[o + h]) / 2
      p >= h: in[o] = zeta^-tau(p - h) (out[o - h] - out[o]) / 2."""
    m = 1 << s
    h = m >> 1
    if o // m != i // m:
        return None
    p, pi = o % m, i % m
    twoN = 2 * N
    if not inverse:
        if p < h:
            if pi == p:
                return (0, 0)
            if pi == p + h:
                return (tau(N, s, p), 0)
        else:
            if pi == p - h:
                return (0, 0)
            if pi == p:
                return ((tau(N, s, p - h) + N) % twoN, 0)
        return None
    if p < h:
        if pi == p or pi == p + h:
            return (0, 1)
        return None
    t = tau(N, s, p - h)
    if pi == p - h:
        return ((-t) % twoN, 1)
    if pi == p:
        return ((N - t) % twoN, 1)
    return None


def group_entry(N, stages, inverse, o, i):
    """Entry (o, i) of the product of consecutive stages, `stages` in the order
    they are applied (a vector meets stages[0] first): the unique path from
    index i to index o sets, at stage s, bit s - 1 of the running index to o's.
    Returns (exponent mod 2N, halvings) or None."""
    bits = 0
    for s in stages:
        bits |= 1 << (s - 1)
    if (o ^ i) & ~bits:
        return None
    x, e, hv = i, 0, 0
    for s in stages:
        b = 1 << (s - 1)
        y = (x & ~b) | (o & b)
        ent = stage_entry(N, s, inverse, y, x)
        if ent is None:
            return None
        e += ent[0]
        hv += ent[1]
        x = y
    return (e % (2 * N), hv)


def stage_groups(k, n_groups):
    """Stages 1..k split into n_groups consecutive ranges, the larger ranges at
    the top: [[1..a], [a+1..b], ...] in increasing order."""
    if not 1 <= n_groups <= k:
        raise ValueError("need 1 <= groups <= log2(n)")
    base, extra = divmod(k, n_groups)
    sizes = [base + (1 if g >= n_groups - extra else 0) for g in range(n_groups)]
    out, s = [], 1
    for sz in sizes:
        out.append(list(range(s, s + sz)))
        s += sz
    return out


def group_offsets(stages, n):
    """Distinct diagonal offsets of a group modulo n: the residues of
    sum_s e_s 2^(s-1), e_s in {-1, 0, 1}, each taken as its representative in
    (-n/2, n/2] (the group of the top stages wraps around and covers every
    multiple of its lowest stride)."""
    lo = 1 << (min(stages) - 1)
    span = (1 << len(stages)) - 1
    half = n // 2
    return sorted({((j * lo + half - 1) % n) - (half - 1) for j in range(-span, span + 1)})


def group_diagonals(N, tab, stages, inverse, kappa, parts):
    """Real-form diagonals of one group.

    Returns {(out, in, offset): slot vector} for the pair map
      parts = 2: (re', im') = (Re G re - Im G im, Im G re + Re G im)
      parts = 1: re' = Re G re - Im G im
    with d_r[o] = G[o][(o + r) mod n].  Each value is sign * 2^-halvings *
    cos or sin of pi e / N (exact), times kappa in one IEEE product when
    kappa != 1.  Diagonal vectors that are zero everywhere are left out."""
    n = N // 2
    out = {}
    for r in group_offsets(stages, n):
        re = np.zeros(n)
        im = np.zeros(n)
        for o in range(n):
            ent = group_entry(N, stages, inverse, o, (o + r) % n)
            if ent is None:
                continue
            e, hv = ent
            c = math.ldexp(cos_pi(tab, N, e), -hv)
            s = math.ldexp(sin_pi(tab, N, e), -hv)
            if kappa != 1.0:
                c = c * kappa
                s = s * kappa
            re[o] = c
            im[o] = s
        cand = [((0, 0), re), ((0, 1), -im)]
        if parts == 2:
            cand += [((1, 0), im), ((1, 1), re)]
        for (oo, ii), v in cand:
            if np.any(v != 0.0):
                out[(oo, ii, r)] = v + 0.0  # no negative zeros
    return out


def group_diagonals_complex(N, tab, stages, inverse, kappa):
    """Complex diagonals of one group acting on one ciphertext's complex slots:
    {(0, 0, r): d_r}, d_r[o] = G[o][(o + r) mod n] = 2^-halvings (cos + i sin)(pi e / N),
    each part times kappa in one IEEE product when kappa != 1; all-zero diagonals
    are left out."""
    n = N // 2
    out = {}
    for r in group_offsets(stages, n):
        re = np.zeros(n)
        im = np.zeros(n)
        for o in range(n):
            ent = group_entry(N, stages, inverse, o, (o + r) % n)
            if ent is None:
                continue
            e, hv = ent
            c = math.ldexp(cos_pi(tab, N, e), -hv)
            s = math.ldexp(sin_pi(tab, N, e), -hv)
            if kappa != 1.0:
                c = c * kappa
                s = s * kappa
            re[o] = c
            im[o] = s
        if np.any(re != 0.0) or np.any(im != 0.0):
            out[(0, 0, r)] = re + 1j * im
    return out


def encode_c(pr, z, level, scale):
    """Plaintext of complex slot values z on q_0..q_level (NTT form)."""
    m = C.encode_complex(z, pr.logN, scale)
    return ckks.Plaintext(ckks.signed_to_ntt(pr, m, range(level + 1)), level, scale)


def encode_qp_c(pr, z, level, scale):
    """The same on Q_level * P (dict limb -> NTT residues)."""
    m = C.encode_complex(z, pr.logN, scale)
    return {t: pr.ntt(C.from_signed(m, pr.moduli[t]), t) for t in pr.ks_limbs(level)}


# ---------------------------------------------------------------------------
# Plaintext-matrix products by the diagonal method with baby / giant steps
# ---------------------------------------------------------------------------

def bsgs_decompose(offsets, n1):
    """Split every offset r = giant + baby: r_lo = min, delta = gcd of r - r_lo
    (1 when all equal), j = (r - r_lo) / delta, baby = (j mod n1) delta,
    giant = r_lo + (j div n1) n1 delta.  Returns {r: (giant, baby)}."""
    r_lo = min(offsets)
    delta = 0
    for r in offsets:
        delta = math.gcd(delta, r - r_lo)
    delta = delta or 1
    dec = {}
    for r in offsets:
        j = (r - r_lo) // delta
        dec[r] = (r_lo + (j // n1) * n1 * delta, (j % n1) * delta)
    return dec


def default_n1(n_offsets, baby_ratio=1):
    """Baby steps: the smallest power of two n1 with n1^2 >= baby_ratio times the
    number of offsets (baby_ratio > 1 trades giant-step rotations, each with
    its own ModUp, for hoisted baby-step rotations)."""
    n1 = 1
    while n1 * n1 < baby_ratio * n_offsets:
        n1 *= 2
    return n1


def lintrans_steps(diags, n, n1):
    dec = bsgs_decompose(sorted({k[2] for k in diags}), n1)
    return sorted({v % n for g, b in dec.values() for v in (g, b)} - {0})


def he_lintrans(pr, keys, cts, diags, n_out, n1, w_scale=None, hoist="single"):
    """out[o] = rescale(sum_{(o, i, r)} d ⊙ Rot(cts[i], r)) by baby / giant steps:
    for every giant step g, the sum over (i, b) of Rot(d, -g) ⊙ Rot(cts[i], b)
    (the baby rotations of each input hoisted, rotate_ext) is rotated by g (one
    rotation of the sum), the giant sums are added, and the result is rescaled
    once.  Plaintexts are encoded at w_scale (default q_level), so the declared
    output scale equals the input scale.
    hoist="double": the baby rotations stay on Q_level * P (rotate_ext_qp, the
    unrotated inputs lifted by lift_qp), each (output, giant) sum is formed there
    with the plaintexts on Q_level * P and takes one ModDown before its giant
    rotation (the composition of henn.he_conv_bsgs with hoist="double")."""
    double = hoist == "double"
    level = cts[0].level
    n = pr.N // 2
    ws = float(pr.moduli[level]) if w_scale is None else w_scale
    dec = bsgs_decompose(sorted({k[2] for k in diags}), n1)
    baby = {}
    for i, ct in enumerate(cts):
        need = sorted({dec[r][1] for (o, ii, r) in diags if ii == i})
        ext = None
        for b in need:
            if b % n == 0:
                baby[(i, b)] = ckks.lift_qp(pr, ct) if double else ct
            else:
                if ext is None:
                    ext = ckks.mod_up(pr, ct.c1, ct.level)
                rot = ckks.rotate_ext_qp if double else ckks.rotate_ext
                baby[(i, b)] = rot(pr, keys, ct, ext, b)
    out = []
    for o in range(n_out):
        groups = {}
        for (oo, i, r), v in diags.items():
            if oo != o:
                continue
            g, b = dec[r]
            z = np.roll(v, g)  # pt[l] = v[(l - g) mod n]
            cplx = np.iscomplexobj(z)
            if double:
                pt = (encode_qp_c if cplx else ckks.encode_qp)(pr, z, level, ws)
                groups.setdefault(g, []).append((baby[(i, b)], pt))
            else:
                term = ckks.pmult(pr, baby[(i, b)], (encode_c if cplx else ckks.encode)(pr, z, level, ws))
                groups[g] = term if g not in groups else ckks.add(pr, groups[g], term)
        total = None
        for g in sorted(groups):
            acc = groups[g]
            if double:
                ab, aa = ckks.mac_qp(pr, level, acc)
                acc = ckks.mod_down_ct(pr, ab, aa, level, cts[0].scale * ws)
            if g % n:
                acc = ckks.rotate(pr, keys, acc, g)
            total = acc if total is None else ckks.add(pr, total, acc)
        r = ckks.rescale(pr, total)
        r.scale = cts[0].scale
        out.append(r)
    return out


# ---------------------------------------------------------------------------
# EvalMod: scaled-integer steps with declared scales
# ---------------------------------------------------------------------------

def taylor_cos_coeffs(D=8):
    """a_k = (-1)^k / (2k)!, k = 0..D, each the double nearest to the rational."""
    return [float(Fraction((-1) ** k, math.factorial(2 * k))) for k in range(D + 1)]


def ev_mul(pr, keys, a, b):
    """relin(a (x) b), rescaled: scale (s_a s_b) / q_level."""
    ql = float(pr.moduli[a.level])
    r = ckks.rescale(pr, ckks.cmult_relin(pr, keys, a, b))
    r.scale = (a.scale * b.scale) / ql
    return r


def ev_cmul(pr, ct, c, s_t):
    """Value times c at declared scale s_t, one level:
    K = nearest(((c s_t) q_level) / s), ct K rescaled by q_level."""
    ql = float(pr.moduli[ct.level])
    K = ckks.nearest_int(((c * s_t) * ql) / ct.scale)
    r = ckks.rescale(pr, ckks.mul_int(pr, ct, K))
    r.scale = s_t
    return r


def ev_addc(pr, ct, c):
    """Value plus c: K = nearest(c s) added to the constant coefficient."""
    return ckks.add_int(pr, ct, ckks.nearest_int(c * ct.scale))


def eval_mod(pr, keys, ct, r):
    """sin(2 pi y) on slot values x = 2 pi y / 2^r (already scaled by the
    CoeffToSlot constants); uses 5 + r levels:
      x <- x - pi / 2^(r+1)                    (now 2 pi (y - 1/4) / 2^r)
      w = x^2, w2 = w^2, w3 = w2 w, w4 = w2^2
      q1 = a4 + a5 w + a6 w2 + a7 w3 + a8 w4   (declared scale s0, level l0 - 4)
      p  = w4 q1 + a1 w + a2 w2 + a3 w3 + a0   (scale (s4 s0) / q_{l0-4}, level l0 - 5)
      r times: c <- 2 c^2 - 1."""
    a = taylor_cos_coeffs(8)
    s0 = ct.scale
    x = ev_addc(pr, ct, -math.ldexp(math.pi, -(r + 1)))
    w = ev_mul(pr, keys, x, x)
    w2 = ev_mul(pr, keys, w, w)
    w3 = ev_mul(pr, keys, w2, drop_level(w))
    w4 = ev_mul(pr, keys, w2, w2)
    q1 = drop_level(ev_cmul(pr, w, a[5], s0), 2)
    q1 = ckks.add(pr, q1, drop_level(ev_cmul(pr, w2, a[6], s0)))
    q1 = ckks.add(pr, q1, ev_cmul(pr, w3, a[7], s0))
    q1 = ckks.add(pr, q1, ev_cmul(pr, w4, a[8], s0))
    q1 = ev_addc(pr, q1, a[4])
    l4 = q1.level
    sc = (w4.scale * s0) / float(pr.moduli[l4])
    p = ev_mul(pr, keys, drop_level(w4), q1)
    p = ckks.add(pr, p, drop_level(ev_cmul(pr, w, a[1], sc), 3))
    p = ckks.add(pr, p, drop_level(ev_cmul(pr, w2, a[2], sc), 2))
    p = ckks.add(pr, p, drop_level(ev_cmul(pr, w3, a[3], sc), 1))
    c = ev_addc(pr, p, a[0])
    for _ in range(r):
        c = ev_addc(pr, ckks.mul_int(pr, ev_mul(pr, keys, c, c), 2), -1.0)
    return c


def eval_mod_plain(y, r):
    """The same polynomial and double angles on plain float64 slot values y."""
    a = taylor_cos_coeffs(8)
    x = (math.pi / 2 ** (r - 1)) * np.asarray(y, dtype=np.float64) - math.ldexp(math.pi, -(r + 1))
    w = x * x
    c = sum(a[k] * w ** k for k in range(9))
    for _ in range(r):
        c = 2 * c * c - 1
    return c


# ---------------------------------------------------------------------------
# The refresh
# ---------------------------------------------------------------------------

class BootParams:
    """n_cts / n_stc: stage groups (levels) of CoeffToSlot / SlotToCoeff;
    r: double angles; top: level after ModRaise (default L); baby_ratio: the
    baby-step rule of every group (default_n1); double_hoist: the groups'
    products with hoist="double" (he_lintrans); form: "real" (the transforms on
    the pair (re, im) in real form) or "complex" (on one ciphertext with complex
    diagonals, the real and imaginary parts split after CoeffToSlot)."""

    def __init__(self, pr, n_cts=3, n_stc=3, r=6, top=None, baby_ratio=4, double_hoist=True, form="complex"):
        if form not in ("real", "complex"):
            raise ValueError("form must be 'real' or 'complex'")
        self.form = form
        self.baby_ratio = baby_ratio
        self.hoist = "double" if double_hoist else "single"
        self.N = pr.N
        self.k = (pr.N // 2).bit_length() - 1
        self.n_cts, self.n_stc, self.r = n_cts, n_stc, r
        self.top = pr.L if top is None else top
        self.depth = n_cts + 5 + r + n_stc
        if self.depth > self.top:
            raise ValueError(f"the refresh needs {self.depth} levels above 0, top is {self.top}")
        self.cts_groups = stage_groups(self.k, n_cts)[::-1]  # applied from the top stages down
        self.stc_groups = stage_groups(self.k, n_stc)        # applied from stage 1 up


def cts_diagonals(pr, bp, tab):
    """The CoeffToSlot groups' diagonals in the order applied; the first carries
    kappa = (1/2) (2 pi / 2^r) = pi / 2^r (exact)."""
    out = []
    for gi, grp in enumerate(bp.cts_groups):
        kappa = math.ldexp(math.pi, -bp.r) if gi == 0 else 1.0
        stages = sorted(grp, reverse=True)  # S_hi^-1 meets the vector first
        out.append(group_diagonals(pr.N, tab, stages, True, kappa, 2))
    return out


def stc_kappa(q0, scale_in):
    return (float(q0) / (2.0 * math.pi)) / scale_in


def stc_diagonals(pr, bp, tab, scale_in):
    """The SlotToCoeff groups' diagonals in the order applied; the first carries
    kappa = (q_0 / (2 pi)) / scale_in, the last keeps only the real part."""
    out = []
    for gi, grp in enumerate(bp.stc_groups):
        kappa = stc_kappa(pr.moduli[0], scale_in) if gi == 0 else 1.0
        parts = 1 if gi == len(bp.stc_groups) - 1 else 2
        out.append(group_diagonals(pr.N, tab, sorted(grp), False, kappa, parts))
    return out


def cts_diagonals_complex(pr, bp, tab):
    """The CoeffToSlot groups as complex diagonals on one ciphertext, in the order
    applied; the first carries kappa = pi / 2^r (the 1/2 of the later split
    and the EvalMod pre-scaling pi / 2^(r-1))."""
    out = []
    for gi, grp in enumerate(bp.cts_groups):
        kappa = math.ldexp(math.pi, -bp.r) if gi == 0 else 1.0
        out.append(group_diagonals_complex(pr.N, tab, sorted(grp, reverse=True), True, kappa))
    return out


def stc_diagonals_complex(pr, bp, tab, scale_in):
    """The SlotToCoeff groups as complex diagonals, in the order applied; the
    first carries kappa = (q_0 / (2 pi)) / scale_in."""
    out = []
    for gi, grp in enumerate(bp.stc_groups):
        kappa = stc_kappa(pr.moduli[0], scale_in) if gi == 0 else 1.0
        out.append(group_diagonals_complex(pr.N, tab, sorted(grp), False, kappa))
    return out


def boot_rotation_steps(pr, bp):
    """Rotation steps of every group (mod n), the conjugation excluded."""
    n = pr.N // 2
    steps = set()
    for groups in (bp.cts_groups, bp.stc_groups):
        for grp in groups:
            offs = group_offsets(grp, n)
            dec = bsgs_decompose(offs, default_n1(len(offs), bp.baby_ratio))
            steps |= {v % n for g, b in dec.values() for v in (g, b)}
    return sorted(steps - {0})


def bootstrap(pr, keys, ct, bp, tab=None, trace=None, encaps=None):
    """Refresh a level-0 ciphertext (declared scale ct.scale) to level
    bp.top - bp.depth; the result decrypts to the same slot values.
    encaps (an Encapsulation): the input is under the dense secret of `keys`;
    it is switched to the sparse secret at level 0, raised, and switched back
    to the dense secret at level top before CoeffToSlot."""
    tab = cos_table(pr.N) if tab is None else tab
    scale_in = ct.scale
    if encaps is not None:
        ct = key_switch(pr, ct, encaps.to_sparse)
    x = mod_raise(pr, ct, bp.top)
    if encaps is not None:
        x = key_switch(pr, x, encaps.to_dense)
    if bp.form == "complex":
        return _bootstrap_complex(pr, keys, x, bp, tab, scale_in, trace)
    cj = conjugate(pr, keys, x)
    re = ckks.add(pr, x, cj)
    im = mul_monomial(pr, sub(pr, x, cj), pr.N // 2, -1)
    if trace is not None:
        trace["raised"] = x
        trace["parts"] = (re, im)
    pair = [re, im]
    for d in cts_diagonals(pr, bp, tab):
        pair = he_lintrans(pr, keys, pair, d, 2, default_n1(len({k[2] for k in d}), bp.baby_ratio), hoist=bp.hoist)
    if trace is not None:
        trace["cts"] = pair
    pair = [eval_mod(pr, keys, c, bp.r) for c in pair]
    if trace is not None:
        trace["evalmod"] = pair
    sds = stc_diagonals(pr, bp, tab, scale_in)
    for gi, d in enumerate(sds):
        pair = he_lintrans(pr, keys, pair, d, 1 if gi == len(sds) - 1 else 2,
                           default_n1(len({k[2] for k in d}), bp.baby_ratio), hoist=bp.hoist)
    return pair[0]


def _bootstrap_complex(pr, keys, x, bp, tab, scale_in, trace):
    """The complex form from the raised ciphertext x:
      CoeffToSlot on x with complex diagonals (slots: (pi / 2^r) R (t_lo + i t_hi) / q_0),
      re = w + conj(w), im = -X^(N/2) (w - conj(w)) (one conjugation),
      EvalMod on both, v = e_re + X^(N/2) e_im (slots e_re + i e_im),
      SlotToCoeff on v with complex diagonals (its real part is the message;
      the imaginary part is noise)."""
    n = pr.N // 2
    for d in cts_diagonals_complex(pr, bp, tab):
        x = he_lintrans(pr, keys, [x], d, 1, default_n1(len({k[2] for k in d}), bp.baby_ratio), hoist=bp.hoist)[0]
    if trace is not None:
        trace["cts"] = x
    cj = conjugate(pr, keys, x)
    re = ckks.add(pr, x, cj)
    im = mul_monomial(pr, sub(pr, x, cj), n, -1)
    e_re, e_im = eval_mod(pr, keys, re, bp.r), eval_mod(pr, keys, im, bp.r)
    if trace is not None:
        trace["evalmod"] = [e_re, e_im]
    v = ckks.add(pr, e_re, mul_monomial(pr, e_im, n, 1))
    for d in stc_diagonals_complex(pr, bp, tab, scale_in):
        v = he_lintrans(pr, keys, [v], d, 1, default_n1(len({k[2] for k in d}), bp.baby_ratio), hoist=bp.hoist)[0]
    return v
