"""The oracle's ChaCha20 generator (RFC 8439), the samplers' option besides
SplitMix64: pinned to the RFC's known-answer vectors (tests/golden/), then the
word mapping and the samplers' distributions on top of it."""
import os

import numpy as np
import pytest

from oracle import _core

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "chacha20_rfc8439.txt")


def _golden():
    vals = {}
    with open(GOLDEN) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                name, *words = line.split()
                vals[name] = [int(w, 16) for w in words]
    return vals


@pytest.fixture
def chacha():
    key6 = np.array([0x01234567, 0x89abcdef, 0x0badf00d, 0xdeadbeef, 0x13579bdf, 0x2468ace0], dtype=np.uint32)
    _core.set_generator("chacha20", key6)
    yield key6
    _core.set_generator("splitmix64")


def test_quarter_round_rfc8439_vector():
    g = _golden()
    assert list(_core.chacha_quarter(*g["quarter_in"])) == g["quarter_out"]


def test_block_function_rfc8439_vector():
    g = _golden()
    out = _core.chacha20_block(g["block_key"], g["block_counter"][0], g["block_nonce"])
    assert [int(v) for v in out] == g["block_out"]


def test_word_is_the_keyed_block_output(chacha):
    master, tag = 0x1122334455667788, (4 << 56) | (3 << 24) | (2 << 8) | 5
    key8 = [master & 0xFFFFFFFF, master >> 32] + [int(v) for v in chacha]
    for n in (0, 1, 7, 8, 15, 1000, 65535):
        blk = _core.chacha20_block(key8, n >> 3, [tag & 0xFFFFFFFF, tag >> 32, 0])
        j = 2 * (n & 7)
        assert _core.word(master, tag, n) == int(blk[j]) | (int(blk[j + 1]) << 32)


def test_generator_switch_changes_and_restores_words(chacha):
    w_chacha = [_core.word(9, 17, n) for n in range(16)]
    _core.set_generator("splitmix64")
    w_split = [_core.word(9, 17, n) for n in range(16)]
    assert w_split != w_chacha
    _core.set_generator("chacha20", chacha)
    assert [_core.word(9, 17, n) for n in range(16)] == w_chacha


def test_samplers_on_chacha20_have_their_distributions(chacha):
    n = 1 << 16
    q = (1 << 36) - 5 * (1 << 20) + 1
    u = _core.sample_uniform(3, 11, q, n).astype(np.float64)
    assert u.max() < q and abs(u.mean() / q - 0.5) < 0.01 and abs(u.std() / q - (1 / 12) ** 0.5) < 0.01
    t = _core.sample_ternary(3, 12, n)
    assert set(np.unique(t)) == {-1, 0, 1}
    assert all(abs(np.mean(t == v) - 1 / 3) < 0.01 for v in (-1, 0, 1))
    e = _core.sample_cbd21(3, 13, n).astype(np.float64)
    # centred binomial with eta = 21: mean 0, variance eta / 2
    assert abs(e.max()) <= 21 and abs(e.mean()) < 0.05 and abs(e.var() - 10.5) < 0.3
