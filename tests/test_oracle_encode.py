"""Pins of the oracle's canonical-embedding encode/decode."""
import numpy as np
import pytest

from oracle import _core as C


def test_constant_vector_encodes_to_constant_polynomial():
    logN = 6
    for c in [0.5, -1.25, 3.0]:
        z = np.full(32, c)
        m = C.encode(z, logN, 2.0 ** 30)
        assert m[0] == round(c * 2 ** 30) and not m[1:].any()


@pytest.mark.parametrize("logN", [3, 4, 5])
def test_encode_matches_definition_quad(logN):
    """Round(Delta * tau^-1(z)) against the definition summed in quad precision."""
    z = np.random.default_rng(logN).uniform(-1, 1, (1 << logN) // 2)
    exact = C.encode_direct_real(z, logN, 2.0 ** 40)
    m = C.encode(z, logN, 2.0 ** 40)
    assert np.array_equal(m, np.round(exact).astype(np.int64))


def test_encode_decode_round_trip():
    logN = 10
    z = np.random.default_rng(1).uniform(-2, 2, 512)
    m = C.encode(z, logN, 2.0 ** 30)
    err = np.abs(C.decode(m, logN, 2.0 ** 30) - z).max()
    # each of the N coefficients is off by at most 1/2: |error| <= N / 2 / Delta
    assert err <= 1024 / 2 / 2 ** 30


def test_rotation_of_slots_is_the_galois_automorphism_exactly():
    """encode(z shifted left by r) == sigma_{5^r}(encode(z)) coefficient by coefficient:
    slot l is the evaluation at zeta^(5^l)."""
    logN = 6
    N = 1 << logN
    z = np.random.default_rng(2).uniform(-1, 1, N // 2)
    m = C.encode(z, logN, 2.0 ** 30)
    for r in [1, 3, 7]:
        g = pow(5, r, 2 * N)
        mr = C.encode(np.roll(z, -r), logN, 2.0 ** 30)
        expect = np.zeros(N, dtype=np.int64)
        for j in range(N):
            t = j * g % (2 * N)
            if t < N:
                expect[t] = m[j]
            else:
                expect[t - N] = -m[j]
        assert np.array_equal(mr, expect)


def test_encode_guard_band_recomputes_near_ties():
    """A coefficient whose exact value is near a half-integer goes through the
    quad-precision recomputation and still rounds like the definition."""
    logN = 4
    z = np.zeros(8)
    z[0] = 1.0
    scale = 8.0 * (0.5 + 1e-9)   # m_0 = (2/N) * scale * sum z = scale/8 * ... near 0.5
    m = C.encode(z, logN, scale)
    exact = C.encode_direct_real(z, logN, scale)
    assert np.array_equal(m, np.round(exact).astype(np.int64))
