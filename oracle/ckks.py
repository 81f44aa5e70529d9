"""RNS-CKKS, written out plainly: parameters, keys, encode/encrypt/decrypt,
PMult/Add/CMult, rotation (Eq. 1) and rescale.

Test infrastructure only (see oracle/__init__.py).

Readings of the paper that this file fixes (the paper names the CKKS primitives
in its background section and Eq. 1 but leaves their RNS details open):

* Moduli: q_0 > q_1 > ... > q_L are the largest primes below 2^bits with
  q = 1 (mod 2N); the k special primes p_0.. are the next ones in that sequence.
  psi for each modulus is its smallest primitive 2N-th root of unity.
* Polynomials are kept per limb in NTT form, NTT(a)[i] = a(psi^(2 brv(i) + 1)).
* Slot l is the evaluation at zeta^(5^l), zeta = exp(i pi / N); Rot(v, r)[l] = v[l + r].
* Randomness: SplitMix64 outputs addressed by (master seed, tag, index);
  uniform residues floor(w q / 2^64), ternary secret floor(3 w / 2^64) - 1,
  errors from the centred binomial with eta = 21.
* Secret-key encryption (the client keeps the key): b = -a s + m + e.
* Key switching is the hybrid RNS method with digits of k consecutive primes.
  Every base conversion (ModUp of a digit, ModDown from P) is the approximate
  conversion with centred digits y_i in (-b_i/2, b_i/2]; ModDown therefore
  rounds x / P to nearest up to the conversion's small integer error.
* Rotation by r with g = 5^r mod 2N key-switches c1 from s to
  sigma_{g^-1}(s) first and applies the automorphism sigma_g afterwards:
  Rot(ct) = sigma_g((c0, 0) + KS(c1)).  Eq. 1 applies sigma_g first; both
  decrypt to the rotated message.
* Rescale divides by the last prime with rounding: (c - [c]_{q_l}) / q_l with the
  centred representative.
"""
from math import prod

import numpy as np

from . import _core as C

KIND_SK, KIND_CT_A, KIND_CT_E, KIND_KEY_A, KIND_KEY_E = 1, 2, 3, 4, 5


def tag(kind, obj=0, digit=0, limb=0):
    """Address of one random stream: kind | object | digit | limb."""
    assert obj < (1 << 32) and digit < (1 << 16) and limb < (1 << 8)
    return (kind << 56) | (obj << 24) | (digit << 8) | limb


def brv(x, bits):
    r = 0
    for _ in range(bits):
        r = (r << 1) | (x & 1)
        x >>= 1
    return r


class Params:
    """Ring degree N = 2^logN, n_q ciphertext primes of `bits` bits and k special
    primes of `pbits` bits (default: the next primes of the same sequence)."""

    def __init__(self, logN, n_q, k, bits, pbits=None):
        self.logN = logN
        self.N = 1 << logN
        self.q = C.ntt_primes(logN, bits, 0, n_q)
        pbits = bits if pbits is None else pbits
        skip = 0
        self.p = []
        while len(self.p) < k:
            cand = C.ntt_primes(logN, pbits, skip, 1)[0]
            skip += 1
            if cand not in self.q:
                self.p.append(cand)
        self.moduli = self.q + self.p
        self.L = n_q - 1
        self.k = k
        self.bits = bits
        self.pbits = pbits
        self.psi = [C.min_psi(m, logN) for m in self.moduli]
        self.P = prod(self.p)

    def p_index(self, j):
        """Index of special prime p_j in `moduli`."""
        return self.L + 1 + j

    def digits(self, level):
        """Hybrid key-switching digits at `level`: groups of k consecutive q's."""
        n = level + 1
        return [list(range(j * self.k, min((j + 1) * self.k, n))) for j in range((n + self.k - 1) // self.k)]

    def ks_limbs(self, level):
        """Moduli indices of the extended basis Q_level * P."""
        return list(range(level + 1)) + [self.p_index(j) for j in range(self.k)]

    def galois(self, r):
        """Galois element of a left rotation by r slots: 5^r mod 2N."""
        return pow(5, r % (self.N // 2), 2 * self.N)

    # --- per-limb transforms -------------------------------------------------
    def ntt(self, a, idx):
        return C.ntt(a, self.logN, self.moduli[idx], self.psi[idx])

    def intt(self, a, idx):
        return C.intt(a, self.logN, self.moduli[idx], self.psi[idx])

    def automorph_perm(self, g):
        """perm with NTT(sigma_g a)[i] = NTT(a)[perm[i]]:
        2 brv(perm[i]) + 1 = (2 brv(i) + 1) g (mod 2N)."""
        cache = self.__dict__.setdefault("_perm_cache", {})
        if g not in cache:
            N, logN = self.N, self.logN
            perm = np.empty(N, dtype=np.int64)
            for i in range(N):
                e = ((2 * brv(i, logN) + 1) * g) % (2 * N)
                perm[i] = brv((e - 1) // 2, logN)
            cache[g] = perm
        return cache[g]

    def automorph_coef(self, a, g, q):
        """sigma_g on a coefficient-form limb: X^j -> X^(j g mod 2N), X^N = -1."""
        N = self.N
        out = np.zeros(N, dtype=np.uint64)
        for j in range(N):
            t = (j * g) % (2 * N)
            v = int(a[j])
            if t < N:
                out[t] = v
            else:
                out[t - N] = (q - v) % q
        return out


# ---------------------------------------------------------------------------
# Polynomials over a list of limbs (moduli indices), NTT form unless stated.
# ---------------------------------------------------------------------------

def signed_to_ntt(pr, m, limbs):
    """Signed integer coefficients -> NTT-form residues on the given limbs."""
    return np.stack([pr.ntt(C.from_signed(m, pr.moduli[t]), t) for t in limbs])


class Ciphertext:
    def __init__(self, c0, c1, level, scale):
        self.c0 = c0  # [level+1][N] uint64, NTT form
        self.c1 = c1
        self.level = level
        self.scale = scale

    def copy(self):
        return Ciphertext(self.c0.copy(), self.c1.copy(), self.level, self.scale)

    def as_array(self):
        return np.stack([self.c0, self.c1])


class Plaintext:
    def __init__(self, m, level, scale):
        self.m = m  # [level+1][N] NTT form
        self.level = level
        self.scale = scale


class SecretKey:
    """Ternary secret s, with its NTT form on every modulus."""

    def __init__(self, pr, seed):
        self.coef = C.sample_ternary(seed, tag(KIND_SK), pr.N)
        self.ntt = signed_to_ntt(pr, self.coef, range(len(pr.moduli)))


class SwitchKey:
    """Hybrid key-switching key from s_src to s_dst over Q_L * P, one pair per digit.

    b_j = -a_j s_dst + e_j + [t in digit j] (P mod t) s_src   on every limb t,
    a_j uniform (sampled in NTT form), e_j centred binomial.
    """

    def __init__(self, pr, seed, obj, s_src_ntt, s_dst_ntt):
        all_limbs = range(len(pr.moduli))
        self.b, self.a = [], []
        for j, dig in enumerate(pr.digits(pr.L)):
            a = np.stack([C.sample_uniform(seed, tag(KIND_KEY_A, obj, j, t), pr.moduli[t], pr.N)
                          for t in all_limbs])
            e = C.sample_cbd21(seed, tag(KIND_KEY_E, obj, j, 0), pr.N)
            e_ntt = signed_to_ntt(pr, e, all_limbs)
            b = np.empty_like(a)
            for t in all_limbs:
                mt = pr.moduli[t]
                bt = C.vec_sub(e_ntt[t], C.vec_mul(a[t], s_dst_ntt[t], mt), mt)
                if t in dig:
                    bt = C.vec_add(bt, C.vec_scalar_mul(s_src_ntt[t], pr.P % mt, mt), mt)
                b[t] = bt
            self.b.append(b)
            self.a.append(a)


class KeySet:
    """Secret key plus the switching keys the evaluator needs."""

    def __init__(self, pr, seed, rot_steps=(), relin=False):
        self.pr = pr
        self.seed = seed
        self.sk = SecretKey(pr, seed)
        self.rot = {}
        for r in sorted({r % (pr.N // 2) for r in rot_steps} - {0}):
            self.add_rotation(r)
        self.relin = None
        if relin:
            s2 = np.stack([C.vec_mul(self.sk.ntt[t], self.sk.ntt[t], m) for t, m in enumerate(pr.moduli)])
            self.relin = SwitchKey(pr, seed, 0, s2, self.sk.ntt)

    def add_rotation(self, r):
        pr = self.pr
        g = pr.galois(r)
        if g in self.rot:
            return
        g_inv = pow(g, -1, 2 * pr.N)
        perm = pr.automorph_perm(g_inv)
        s_dst = np.stack([C.gather(self.sk.ntt[t], perm) for t in range(len(pr.moduli))])
        self.rot[g] = SwitchKey(pr, self.seed, g, self.sk.ntt, s_dst)


# ---------------------------------------------------------------------------
# Encode / encrypt / decrypt
# ---------------------------------------------------------------------------

def encode(pr, z, level, scale):
    """Plaintext of the real slot vector z at `scale`, NTT form on q_0..q_level."""
    m = C.encode(np.asarray(z, dtype=np.float64), pr.logN, scale)
    return Plaintext(signed_to_ntt(pr, m, range(level + 1)), level, scale)


def encrypt(pr, sk, pt, seed, ct_id):
    """Secret-key encryption: c1 = a uniform, c0 = -a s + m + e."""
    lv = pt.level
    a = np.stack([C.sample_uniform(seed, tag(KIND_CT_A, ct_id, 0, t), pr.moduli[t], pr.N)
                  for t in range(lv + 1)])
    e = C.sample_cbd21(seed, tag(KIND_CT_E, ct_id), pr.N)
    e_ntt = signed_to_ntt(pr, e, range(lv + 1))
    c0 = np.empty_like(a)
    for t in range(lv + 1):
        q = pr.moduli[t]
        c0[t] = C.vec_add(C.vec_sub(pt.m[t], C.vec_mul(a[t], sk.ntt[t], q), q), e_ntt[t], q)
    return Ciphertext(c0, a, lv, pt.scale)


def decrypt_coef(pr, sk, ct):
    """m = c0 + c1 s on limb q_0, centred: signed coefficients."""
    q = pr.moduli[0]
    m = C.vec_add(ct.c0[0], C.vec_mul(ct.c1[0], sk.ntt[0], q), q)
    return C.centre(pr.intt(m, 0), q)


def decrypt(pr, sk, ct):
    """Decrypt and decode to N/2 real slot values."""
    return C.decode(decrypt_coef(pr, sk, ct), pr.logN, ct.scale)


# ---------------------------------------------------------------------------
# Homomorphic primitives
# ---------------------------------------------------------------------------

def add(pr, x, y):
    assert x.level == y.level
    c0 = np.stack([C.vec_add(x.c0[t], y.c0[t], pr.moduli[t]) for t in range(x.level + 1)])
    c1 = np.stack([C.vec_add(x.c1[t], y.c1[t], pr.moduli[t]) for t in range(x.level + 1)])
    return Ciphertext(c0, c1, x.level, x.scale)


def pmult(pr, ct, pt):
    assert ct.level == pt.level
    c0 = np.stack([C.vec_mul(ct.c0[t], pt.m[t], pr.moduli[t]) for t in range(ct.level + 1)])
    c1 = np.stack([C.vec_mul(ct.c1[t], pt.m[t], pr.moduli[t]) for t in range(ct.level + 1)])
    return Ciphertext(c0, c1, ct.level, ct.scale * pt.scale)


def centred_bconv(pr, coef, src, dst):
    """Approximate base conversion with centred digits.

    coef: coefficient-form residues of x on the source moduli `src`.
    Returns, for each destination modulus index t in `dst`, the residues mod t of
      sum_{i in src} y_i * (B/b_i),  y_i = [x_i * (B/b_i)^-1]_{b_i} in (-b_i/2, b_i/2],
    where B is the product of the source moduli.  This equals x + u B for a small
    integer u (|u| <= |src|/2), and is exact when |src| = 1.
    """
    B = prod(pr.moduli[i] for i in src)
    ys = []
    for pos, i in enumerate(src):
        bi = pr.moduli[i]
        bhat = B // bi
        ys.append(C.centre(C.vec_scalar_mul(coef[pos], pow(bhat % bi, -1, bi), bi), bi))
    out = {}
    for t in dst:
        mt = pr.moduli[t]
        acc = np.zeros(pr.N, dtype=np.uint64)
        for pos, i in enumerate(src):
            C.vec_mac_scalar(acc, C.from_signed(ys[pos], mt), (B // pr.moduli[i]) % mt, mt)
        out[t] = acc
    return out


def mod_up(pr, d, level):
    """Hybrid ModUp of d (NTT form on q_0..q_level).

    Returns one dict per digit D: extended limb index -> NTT-form residues of the
    centred base conversion of [d]_D to every modulus of Q_level * P outside D.
    Limbs of the digit itself keep d's residues.
    """
    coef = [pr.intt(d[i], i) for i in range(level + 1)]
    ext = []
    for dig in pr.digits(level):
        others = [t for t in pr.ks_limbs(level) if t not in dig]
        conv = centred_bconv(pr, [coef[i] for i in dig], dig, others)
        e = {t: d[t].copy() for t in dig}
        for t in others:
            e[t] = pr.ntt(conv[t], t)
        ext.append(e)
    return ext


def mod_down(pr, x, level):
    """ModDown of x (dict limb -> NTT residues over Q_level * P) to Q_level:
    (x - conv_P(x)) * P^-1 with conv_P the centred base conversion of [x]_P, which
    is round(x / P) up to the conversion's small integer error."""
    ps = [pr.p_index(j) for j in range(pr.k)]
    coef = [pr.intt(x[t], t) for t in ps]
    conv = centred_bconv(pr, coef, ps, range(level + 1))
    out = np.empty((level + 1, pr.N), dtype=np.uint64)
    for i in range(level + 1):
        qi = pr.moduli[i]
        y = C.vec_sub(x[i], pr.ntt(conv[i], i), qi)
        out[i] = C.vec_scalar_mul(y, pow(pr.P % qi, -1, qi), qi)
    return out


def key_inner_product(pr, ext, key, level):
    """Inner product of the extended digits with a switching key over
    Q_level * P: (acc_b, acc_a) as dicts limb -> NTT residues."""
    acc_b, acc_a = {}, {}
    for t in pr.ks_limbs(level):
        mt = pr.moduli[t]
        ab = np.zeros(pr.N, dtype=np.uint64)
        aa = np.zeros(pr.N, dtype=np.uint64)
        for j, e in enumerate(ext):
            C.vec_mac(ab, e[t], key.b[j][t], mt)
            C.vec_mac(aa, e[t], key.a[j][t], mt)
        acc_b[t], acc_a[t] = ab, aa
    return acc_b, acc_a


def key_switch_ext(pr, ext, key, level):
    """Inner product of the extended digits with a switching key, then ModDown.
    Returns (d0, d1) on Q_level."""
    acc_b, acc_a = key_inner_product(pr, ext, key, level)
    return mod_down(pr, acc_b, level), mod_down(pr, acc_a, level)


# ---------------------------------------------------------------------------
# Double hoisting: rotations kept on Q_level * P until after the products
# with plaintexts, with one ModDown per sum (instead of one per rotation).
# ---------------------------------------------------------------------------

def rotate_ext_qp(pr, keys, ct, ext, r):
    """Rotation by r left on the key-switching basis: V = sigma_g((P c0, 0) + acc)
    over Q_level * P (dicts limb -> NTT residues), acc the key inner product of
    the hoisted digits.  mod_down(V) is exactly rotate_ext(ct, ext, r)."""
    g = pr.galois(r)
    lv = ct.level
    acc_b, acc_a = key_inner_product(pr, ext, keys.rot[g], lv)
    perm = pr.automorph_perm(g)
    Vb, Va = {}, {}
    for t in pr.ks_limbs(lv):
        mt = pr.moduli[t]
        b = acc_b[t]
        if t <= lv:
            b = C.vec_add(b, C.vec_scalar_mul(ct.c0[t], pr.P % mt, mt), mt)
        Vb[t] = C.gather(b, perm)
        Va[t] = C.gather(acc_a[t], perm)
    return Vb, Va


def lift_qp(pr, ct):
    """(P c0, P c1) on Q_level * P: P times the ciphertext on the q limbs, zero on
    the special limbs, so that mod_down returns ct exactly."""
    Vb, Va = {}, {}
    for t in pr.ks_limbs(ct.level):
        mt = pr.moduli[t]
        if t <= ct.level:
            Vb[t] = C.vec_scalar_mul(ct.c0[t], pr.P % mt, mt)
            Va[t] = C.vec_scalar_mul(ct.c1[t], pr.P % mt, mt)
        else:
            Vb[t] = np.zeros(pr.N, dtype=np.uint64)
            Va[t] = np.zeros(pr.N, dtype=np.uint64)
    return Vb, Va


def encode_qp(pr, z, level, scale):
    """The plaintext of encode(z, level, scale) on Q_level * P: dict limb -> NTT."""
    m = C.encode(np.asarray(z, dtype=np.float64), pr.logN, scale)
    return {t: pr.ntt(C.from_signed(m, pr.moduli[t]), t) for t in pr.ks_limbs(level)}


def mac_qp(pr, level, terms):
    """sum_t V_t (x) pt_t over Q_level * P; terms: list of ((Vb, Va), pt_qp)."""
    ab = {t: np.zeros(pr.N, dtype=np.uint64) for t in pr.ks_limbs(level)}
    aa = {t: np.zeros(pr.N, dtype=np.uint64) for t in pr.ks_limbs(level)}
    for (Vb, Va), pt in terms:
        for t in pr.ks_limbs(level):
            mt = pr.moduli[t]
            C.vec_mac(ab[t], Vb[t], pt[t], mt)
            C.vec_mac(aa[t], Va[t], pt[t], mt)
    return ab, aa


def mod_down_ct(pr, Vb, Va, level, scale):
    """ModDown of a pair on Q_level * P to a ciphertext on Q_level."""
    return Ciphertext(mod_down(pr, Vb, level), mod_down(pr, Va, level), level, scale)


def mod_down_rescale(pr, x, level):
    """ModDown and rescale as one division (x dict limb -> NTT residues over
    Q_level * P, result on Q_{level-1}): the centred base conversion of
    [x]_{q_level P} to q_0..q_{level-1}, then (x - conv) (q_level P)^-1, which is
    round(x / (q_level P)) up to the conversion's small integer error.  It
    replaces ModDown followed by the rescale of Sec. 2 (rounding x / P, then
    the result / q_level) when nothing else is added on Q_level in between."""
    src = [level] + [pr.p_index(j) for j in range(pr.k)]
    coef = [pr.intt(x[t], t) for t in src]
    conv = centred_bconv(pr, coef, src, range(level))
    out = np.empty((level, pr.N), dtype=np.uint64)
    for i in range(level):
        qi = pr.moduli[i]
        y = C.vec_sub(x[i], pr.ntt(conv[i], i), qi)
        out[i] = C.vec_scalar_mul(y, pow(pr.P * pr.moduli[level] % qi, -1, qi), qi)
    return out


def mod_down_rescale_ct(pr, Vb, Va, level, scale):
    """A pair on Q_level * P at `scale` (times P) to a ciphertext on Q_{level-1}
    at scale / q_level."""
    return Ciphertext(mod_down_rescale(pr, Vb, level), mod_down_rescale(pr, Va, level), level - 1,
                      scale / pr.moduli[level])


def automorph_ntt(pr, poly, g, level):
    perm = pr.automorph_perm(g)
    return np.stack([C.gather(poly[t], perm) for t in range(level + 1)])


def rotate_ext(pr, keys, ct, ext, r):
    """Rotation by r slots given the ModUp of ct.c1 (hoisting: ext is shared
    by every rotation of the same ciphertext)."""
    if r % (pr.N // 2) == 0:
        return ct.copy()
    g = pr.galois(r)
    d0, d1 = key_switch_ext(pr, ext, keys.rot[g], ct.level)
    c0 = np.stack([C.vec_add(ct.c0[t], d0[t], pr.moduli[t]) for t in range(ct.level + 1)])
    return Ciphertext(automorph_ntt(pr, c0, g, ct.level), automorph_ntt(pr, d1, g, ct.level),
                      ct.level, ct.scale)


def rotate(pr, keys, ct, r):
    return rotate_ext(pr, keys, ct, mod_up(pr, ct.c1, ct.level), r)


def rescale(pr, ct):
    """Divide by q_level with rounding, (c - [c]_{q_level}) * q_level^-1 with the
    centred representative; drops one limb and divides the scale by q_level."""
    lv = ct.level
    ql = pr.moduli[lv]

    def one(c):
        r = C.centre(pr.intt(c[lv], lv), ql)
        out = np.empty((lv, pr.N), dtype=np.uint64)
        for i in range(lv):
            qi = pr.moduli[i]
            y = C.vec_sub(c[i], pr.ntt(C.from_signed(r, qi), i), qi)
            out[i] = C.vec_scalar_mul(y, pow(ql % qi, -1, qi), qi)
        return out

    return Ciphertext(one(ct.c0), one(ct.c1), lv - 1, ct.scale / ql)


def tensor(pr, x, y):
    """Ciphertext product before relinearisation: (d0, d1, d2) = (x0 y0,
    x0 y1 + x1 y0, x1 y1) per limb, with level and scale; decrypts under
    (1, s, s^2) to the product of the messages."""
    assert x.level == y.level
    lv = x.level
    d0 = np.empty_like(x.c0)
    d1 = np.empty_like(x.c0)
    d2 = np.empty_like(x.c0)
    for t in range(lv + 1):
        q = pr.moduli[t]
        d0[t] = C.vec_mul(x.c0[t], y.c0[t], q)
        d1[t] = C.vec_add(C.vec_mul(x.c0[t], y.c1[t], q), C.vec_mul(x.c1[t], y.c0[t], q), q)
        d2[t] = C.vec_mul(x.c1[t], y.c1[t], q)
    return (d0, d1, d2, lv, x.scale * y.scale)


def tensor_add(pr, a, b):
    """Sum of two products of tensor() at one level and scale (per limb mod q)."""
    assert a[3] == b[3] and a[4] == b[4]
    lv = a[3]
    parts = tuple(np.stack([C.vec_add(a[k][t], b[k][t], pr.moduli[t]) for t in range(lv + 1)]) for k in range(3))
    return parts + (lv, a[4])


def relinearize(pr, keys, d):
    """(d0, d1, d2) -> (d0, d1) + KS_{s^2 -> s}(d2) with the relinearisation key."""
    d0, d1, d2, lv, scale = d
    e0, e1 = key_switch_ext(pr, mod_up(pr, d2, lv), keys.relin, lv)
    c0 = np.stack([C.vec_add(d0[t], e0[t], pr.moduli[t]) for t in range(lv + 1)])
    c1 = np.stack([C.vec_add(d1[t], e1[t], pr.moduli[t]) for t in range(lv + 1)])
    return Ciphertext(c0, c1, lv, scale)


def cmult_relin(pr, keys, x, y):
    """Ciphertext product (d0, d1, d2) followed by relinearisation of d2."""
    return relinearize(pr, keys, tensor(pr, x, y))


# ---------------------------------------------------------------------------
# Constants and integer scalars (the affine parts of a polynomial activation)
# ---------------------------------------------------------------------------

def nearest_int(x):
    """The integer nearest to the IEEE double x, ties away from zero (exact)."""
    from fractions import Fraction
    f = Fraction(float(x))
    n = abs(f.numerator) // f.denominator
    if abs(f) - n >= Fraction(1, 2):
        n += 1
    return n if f >= 0 else -n


def add_int(pr, ct, K):
    """Add the integer K to the constant coefficient of the message: the constant
    polynomial K has the value K at every NTT position, so K mod q_t is added to
    every residue of c0.  The scale is unchanged."""
    c0 = np.stack([C.vec_add(ct.c0[t], np.full(pr.N, K % pr.moduli[t], dtype=np.uint64), pr.moduli[t])
                   for t in range(ct.level + 1)])
    return Ciphertext(c0, ct.c1.copy(), ct.level, ct.scale)


def mul_int(pr, ct, K):
    """Multiply both polynomials by the integer K (mod each q_t).  The message is
    multiplied by K; the caller decides what that does to the scale."""
    c0 = np.stack([C.vec_scalar_mul(ct.c0[t], K % pr.moduli[t], pr.moduli[t]) for t in range(ct.level + 1)])
    c1 = np.stack([C.vec_scalar_mul(ct.c1[t], K % pr.moduli[t], pr.moduli[t]) for t in range(ct.level + 1)])
    return Ciphertext(c0, c1, ct.level, ct.scale)
