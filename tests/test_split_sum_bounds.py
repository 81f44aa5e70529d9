"""Exact-integer checks of the bounds behind the kernels' split sums.

The MAC, base conversion and key inner product never reduce between terms:
they accumulate exact sums of products of residues and reduce once.  With
every modulus below 2^40 the MAC keeps three 32-bit words fed by 32-bit
multiply-adds (Acc40); below 2^36 it splits one factor at bit 24 and keeps
a + b 2^24 (Acc36), folding a into b every 16 terms and reducing modulo q every
2^14 terms.  These tests restate each form with Python integers at the
extreme operands and check the identities and the headroom the kernels assume.
"""
import random

M64 = (1 << 64) - 1
M32 = (1 << 32) - 1


def acc40_term(w, x, y):
    """One Acc40 term on the words (w0, w1, w2), returning the new words and
    the largest value w2 reached (it must stay below 2^32)."""
    x0, x1, y0, y1 = x & M32, x >> 32, y & M32, y >> 32
    lo = w[0] + ((x0 * y0) & M32)
    c = lo >> 32
    mid = w[1] + ((x0 * y0) >> 32) + c
    c = mid >> 32
    top = w[2] + x1 * y1 + c
    mid &= M32
    mid2 = mid + ((x0 * y1) & M32)
    top += ((x0 * y1) >> 32) + (mid2 >> 32)
    mid3 = (mid2 & M32) + ((x1 * y0) & M32)
    top += ((x1 * y0) >> 32) + (mid3 >> 32)
    return (lo & M32, mid3 & M32, top), top


def test_acc40_is_exact_and_w2_fits_2_15_terms():
    q = (1 << 40) - 87  # any residue is below 2^40
    xs = [q - 1] * (1 << 15)
    w, peak = (0, 0, 0), 0
    for x in xs:
        w, top = acc40_term(w, x, q - 1)
        peak = max(peak, top)
    assert peak < 1 << 32
    assert w[0] + (w[1] << 32) + (w[2] << 64) == sum(x * (q - 1) for x in xs)
    rng = random.Random(40)
    for _ in range(200):
        pairs = [(rng.randrange(1 << 40), rng.randrange(1 << 40)) for _ in range(rng.randrange(1, 40))]
        w = (0, 0, 0)
        for x, y in pairs:
            w, _ = acc40_term(w, x, y)
        assert w[0] + (w[1] << 32) + (w[2] << 64) == sum(x * y for x, y in pairs)


def acc36_mad(a, b, x, y):
    """One Acc36 term: a += x yl, b += x yh (y = yl + yh 2^24), each as a
    widening 32x32 product plus a 32-bit product added to the high word."""
    x0, x1 = x & M32, x >> 32
    yl, yh = y & ((1 << 24) - 1), y >> 24
    a_new = a + x0 * yl + ((x1 * yl) << 32)
    b_new = b + x0 * yh + ((x1 * yh) << 32)
    return a_new, b_new


def test_acc36_terms_and_folds_fit_64_bits():
    top = (1 << 36) - 1  # the largest residue below 2^36
    # per term: x yl < 2^60 and x yh < 2^48
    assert top * ((1 << 24) - 1) < 1 << 60 and top * ((1 << 12) - 1) < 1 << 48
    # sixteen terms after a fold (a below 2^24) stay below 2^64
    a, b = (1 << 24) - 1, 0
    for _ in range(16):
        a, b = acc36_mad(a, b, top, top)
    assert a <= M64
    # 2^14 terms between reductions modulo q: b keeps headroom, including the
    # high parts moved in by the folds
    a, b = 0, 0
    for t in range(1 << 14):
        a, b = acc36_mad(a, b, top, top)
        assert a <= M64 and b <= M64
        if t % 16 == 15:
            b += a >> 24
            a &= (1 << 24) - 1
    assert a + (b << 24) == (1 << 14) * top * top


def test_acc36_value_is_the_exact_sum():
    rng = random.Random(36)
    for _ in range(200):
        pairs = [(rng.randrange(1 << 36), rng.randrange(1 << 36)) for _ in range(rng.randrange(1, 60))]
        a = b = 0
        for t, (x, y) in enumerate(pairs):
            a, b = acc36_mad(a, b, x, y)
            assert a <= M64 and b <= M64
            if t % 16 == 15:
                b += a >> 24
                a &= (1 << 24) - 1
        assert a + (b << 24) == sum(x * y for x, y in pairs)


def test_narrow_barrett_input_bound():
    """Base conversion sums at most 9 products of residues below 2^40 (8
    sources and the -B term) and the key inner product at most 8 digits; both
    stay below the 2^84 that the one-product Barrett reduction accepts."""
    assert 9 * ((1 << 40) - 1) ** 2 < 1 << 84
    assert 16 * ((1 << 40) - 1) ** 2 < 1 << 84
