"""Pins of the oracle's modular arithmetic and negacyclic NTT against the
definitions they implement (textbook facts, no paper value needed)."""
import numpy as np
import pytest

from oracle import _core as C
from oracle import ckks


@pytest.mark.parametrize("logN,bits", [(3, 20), (4, 30), (5, 36), (6, 40), (5, 50), (6, 60)])
def test_primes_and_psi(logN, bits):
    N = 1 << logN
    ps = C.ntt_primes(logN, bits, 0, 4)
    assert ps == sorted(ps, reverse=True) and len(set(ps)) == 4
    for q in ps:
        assert q < (1 << bits) and q % (2 * N) == 1 and C.is_prime(q)
        # no prime of the sequence was skipped between consecutive entries
        psi = C.min_psi(q, logN)
        assert pow(psi, N, q) == q - 1
    # brute-force minimality of psi on a small prime
    q = C.ntt_primes(3, 12, 0, 1)[0]
    psi = C.min_psi(q, 3)
    roots = [x for x in range(2, q) if pow(x, 8, q) == q - 1]
    assert psi == min(roots)


def test_prime_sequence_is_dense():
    """Every q = 1 mod 2N between consecutive primes of the sequence is composite."""
    logN, bits = 5, 30
    ps = C.ntt_primes(logN, bits, 0, 3)
    for hi, lo in zip(ps, ps[1:]):
        for cand in range(lo + 64, hi, 64):
            assert not C.is_prime(cand)
    top = (1 << bits) - 64 + 1
    for cand in range(ps[0] + 64, top + 1, 64):
        assert not C.is_prime(cand)


@pytest.mark.parametrize("logN", [3, 4, 5, 6])
@pytest.mark.parametrize("bits", [30, 40, 60])
def test_ntt_matches_direct_definition(logN, bits):
    q = C.ntt_primes(logN, bits, 0, 1)[0]
    psi = C.min_psi(q, logN)
    rng = np.random.default_rng(logN * 100 + bits)
    a = rng.integers(0, q, 1 << logN, dtype=np.uint64)
    A = C.ntt(a, logN, q, psi)
    assert np.array_equal(A, C.ntt_direct(a, logN, q, psi))
    assert np.array_equal(C.intt(A, logN, q, psi), a)


@pytest.mark.parametrize("logN,bits", [(3, 30), (5, 40), (6, 60)])
def test_ntt_product_is_negacyclic_schoolbook(logN, bits):
    q = C.ntt_primes(logN, bits, 0, 1)[0]
    psi = C.min_psi(q, logN)
    rng = np.random.default_rng(logN)
    a = rng.integers(0, q, 1 << logN, dtype=np.uint64)
    b = rng.integers(0, q, 1 << logN, dtype=np.uint64)
    prod = C.intt(C.vec_mul(C.ntt(a, logN, q, psi), C.ntt(b, logN, q, psi), q), logN, q, psi)
    assert np.array_equal(prod, C.negacyclic_schoolbook(a, b, q))
    # X * X^(N-1) = -1
    x1 = np.zeros(1 << logN, dtype=np.uint64); x1[1] = 1
    xn = np.zeros(1 << logN, dtype=np.uint64); xn[-1] = 1
    minus_one = np.zeros(1 << logN, dtype=np.uint64); minus_one[0] = q - 1
    assert np.array_equal(C.negacyclic_schoolbook(x1, xn, q), minus_one)


def test_automorphism_permutation_matches_coefficient_map():
    pr = ckks.Params(5, 2, 1, 30)
    rng = np.random.default_rng(3)
    q = pr.q[0]
    a = rng.integers(0, q, pr.N, dtype=np.uint64)
    for r in [1, 2, 5, 15, -1]:
        g = pr.galois(r)
        lhs = C.gather(pr.ntt(a, 0), pr.automorph_perm(g))
        rhs = pr.ntt(pr.automorph_coef(a, g, q), 0)
        assert np.array_equal(lhs, rhs)


def test_modmul_against_python_ints():
    rng = np.random.default_rng(5)
    for bits in [30, 40, 50, 60]:
        q = C.ntt_primes(4, bits, 0, 1)[0]
        for _ in range(50):
            a, b = (int(x) for x in rng.integers(0, q, 2, dtype=np.uint64))
            assert C.mulmod(a, b, q) == a * b % q
            assert C.invmod(a, q) * a % q == (1 if a else 0) or a == 0


def test_splitmix64_reference_values():
    # SplitMix64 seeded with 0 (published reference outputs of the generator)
    s = 0
    outs = []
    for _ in range(3):
        s = (s + 0x9E3779B97F4A7C15) % (1 << 64)
        outs.append(C.mix64(s))
    assert outs == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_samplers_distributions():
    n = 1 << 15
    t = C.sample_ternary(1, 2, n)
    assert set(np.unique(t)) == {-1, 0, 1}
    assert abs(np.mean(t == 0) - 1 / 3) < 0.02
    e = C.sample_cbd21(1, 3, n)
    assert abs(e.mean()) < 0.1 and abs(e.var() - 10.5) < 0.5 and np.abs(e).max() <= 21
    q = C.ntt_primes(10, 36, 0, 1)[0]
    u = C.sample_uniform(1, 4, q, n)
    assert u.max() < q and abs(u.astype(np.float64).mean() / q - 0.5) < 0.01
