"""Exact-integer restatement of the NTT's Shoup product for moduli below 2^36
(shoup36 in csrc/ntt.cu): the 32-bit word steps it takes, with Python
integers reduced modulo 2^32 / 2^64 exactly where the kernel's registers wrap,
must give a result congruent to a w mod q and in [0, 2q), for every input the
transforms feed it (a < 2^42), at the extreme operands and on random ones.
The lemma behind it is Harvey's (lazy Shoup multiplication, 2014): with
wq = floor(w 2^63 / q) and a < 2^63, a w - floor(a wq / 2^63) q lies in [0, 2q)."""
import random

M32 = (1 << 32) - 1
M64 = (1 << 64) - 1


def shoup36(a, w, q):
    """The kernel's steps (twiddle companion wq = floor(w 2^64 / q) as stored)."""
    wq = (w << 64) // q
    nq = (-q) & M64
    a0, a1 = a & M32, a >> 32
    w0, w1 = w & M32, w >> 32
    W63 = wq >> 1
    l, h = W63 & M32, W63 >> 32
    h2 = (h << 1) & M32
    n0, n1 = nq & M32, nq >> 32
    t = (a0 * l) >> 32
    Z = t
    Z = a0 * h + Z
    assert Z <= M64
    Z = a1 * l + Z
    assert Z <= M64, "64-bit sum overflows"
    Z >>= 31
    Z = a1 * h2 + Z
    assert Z <= M64
    q0, q1 = Z & M32, Z >> 32
    T = (a0 * w0) & M64
    T = (q0 * n0 + T) & M64
    tl, th = T & M32, T >> 32
    th = (a0 * w1 + th) & M32
    th = (a1 * w0 + th) & M32
    th = (q0 * n1 + th) & M32
    th = (q1 * n0 + th) & M32
    return (th << 32) | tl, Z


def _check(a, w, q):
    T, Q = shoup36(a, w, q)
    assert Q == (a * ((w << 63) // q)) >> 63  # the quotient is the exact floor
    assert 0 <= T < 2 * q
    assert T % q == (a * w) % q


def test_shoup36_extremes():
    for q in ((1 << 36) - 5, (1 << 35) + 1, 68719476731, 34359738421, (1 << 25) + 1):
        for a in (0, 1, q - 1, 2 * q - 1, 4 * q - 1, 35 * q, (1 << 42) - 1, (1 << 32) - 1, 1 << 32):
            for w in (0, 1, q - 1, q // 2, (1 << 32) - 1 if q > 1 << 32 else q - 2):
                _check(a, w, q)


def test_shoup36_random():
    rng = random.Random(5)
    for _ in range(20000):
        q = rng.randrange(1 << 25, 1 << 36) | 1
        _check(rng.randrange(0, 1 << 42), rng.randrange(0, q), q)


def fin32(x, q):
    """The forward transform's final reduction for 2^25 <= q < 2^36 (csrc/ntt.cu):
    Q' = floor((x >> 20) mu / 2^32) with mu = floor(2^64 / q) >> 12, one 32 x 32
    product; the result x - Q' q before the last conditional subtraction."""
    mu = ((1 << 64) // q) >> 12
    t = x >> 20
    assert t <= M32 and mu <= M32
    Qp = (t * mu) >> 32
    return x - Qp * q


def test_fin32_quotient_is_exact_or_one_short():
    """x below 35 q (the forward transform's values without inner reductions)
    reduces to [0, 2q): Q' is floor(x / q) or one less, since the dropped low
    20 bits of x add less than 2^20 / q <= 2^-5 and the truncation of mu less
    than 2^22 / 2^32 to the quotient."""
    rng = random.Random(11)
    qs = [(1 << 36) - 5, 68719476731, 34359738421, (1 << 25) + 1, (1 << 25) + 3, 50331653]
    for q in qs:
        xs = [0, 1, q - 1, q, 2 * q - 1, 35 * q - 1, 34 * q, (35 * q) & ~((1 << 20) - 1)]
        xs += [rng.randrange(35 * q) for _ in range(5000)]
        for x in xs:
            r = fin32(x, q)
            assert 0 <= r < 2 * q, (q, x)
            assert r % q == x % q
