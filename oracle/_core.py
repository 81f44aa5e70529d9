"""ctypes bindings to the oracle's C primitives (oracle/ckks_core.c).

Test infrastructure only.  Each wrapper takes and returns numpy arrays; the
arithmetic itself lives in the C file.
"""
import ctypes
import numpy as np

from . import build as _build

_lib = ctypes.CDLL(_build.build())

u64 = ctypes.c_uint64
i64 = ctypes.c_int64
P = ctypes.c_void_p

_sig = {
    "or_mulmod": (u64, [u64, u64, u64]),
    "or_powmod": (u64, [u64, u64, u64]),
    "or_invmod": (u64, [u64, u64]),
    "or_is_prime": (ctypes.c_int, [u64]),
    "or_ntt_primes": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, P]),
    "or_min_psi": (u64, [u64, ctypes.c_int]),
    "or_ntt_direct": (None, [P, P, ctypes.c_int, u64, u64]),
    "or_ntt": (None, [P, ctypes.c_int, u64, u64]),
    "or_intt": (None, [P, ctypes.c_int, u64, u64]),
    "or_negacyclic_schoolbook": (None, [P, P, P, ctypes.c_int, u64]),
    "or_vec_add": (None, [P, P, P, ctypes.c_int, u64]),
    "or_vec_sub": (None, [P, P, P, ctypes.c_int, u64]),
    "or_vec_mul": (None, [P, P, P, ctypes.c_int, u64]),
    "or_vec_scalar_mul": (None, [P, u64, P, ctypes.c_int, u64]),
    "or_vec_mac_scalar": (None, [P, u64, P, ctypes.c_int, u64]),
    "or_vec_mac": (None, [P, P, P, ctypes.c_int, u64]),
    "or_vec_from_signed": (None, [P, P, ctypes.c_int, u64]),
    "or_vec_centre": (None, [P, P, ctypes.c_int, u64]),
    "or_vec_reduce": (None, [P, P, ctypes.c_int, u64]),
    "or_vec_gather": (None, [P, P, P, ctypes.c_int]),
    "or_mix64": (u64, [u64]),
    "or_word": (u64, [u64, u64, u64]),
    "or_chacha_quarter": (None, [P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "or_chacha20_block": (None, [P, ctypes.c_uint32, P, P]),
    "or_set_generator": (None, [ctypes.c_int, P]),
    "or_sample_uniform": (None, [u64, u64, u64, P, ctypes.c_int]),
    "or_sample_ternary": (None, [u64, u64, P, ctypes.c_int]),
    "or_sample_cbd21": (None, [u64, u64, P, ctypes.c_int]),
    "or_encode": (ctypes.c_int, [P, ctypes.c_int, ctypes.c_double, P]),
    "or_encode_complex": (ctypes.c_int, [P, P, ctypes.c_int, ctypes.c_double, P]),
    "or_decode": (None, [P, ctypes.c_int, ctypes.c_double, P]),
    "or_encode_direct_real": (None, [P, ctypes.c_int, ctypes.c_double, P]),
}
for _name, (_res, _args) in _sig.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _u(a):
    return np.ascontiguousarray(a, dtype=np.uint64)


def mulmod(a, b, q):
    return int(_lib.or_mulmod(a, b, q))


def powmod(a, e, q):
    return int(_lib.or_powmod(a, e, q))


def invmod(a, q):
    return int(_lib.or_invmod(a % q, q))


def is_prime(n):
    return bool(_lib.or_is_prime(n))


def ntt_primes(logN, bits, skip, count):
    out = np.zeros(count, dtype=np.uint64)
    if _lib.or_ntt_primes(logN, bits, skip, count, _p(out)) != 0:
        raise ValueError("not enough NTT-friendly primes")
    return [int(x) for x in out]


def min_psi(q, logN):
    return int(_lib.or_min_psi(q, logN))


def ntt(a, logN, q, psi):
    a = _u(a).copy()
    _lib.or_ntt(_p(a), logN, q, psi)
    return a


def intt(a, logN, q, psi):
    a = _u(a).copy()
    _lib.or_intt(_p(a), logN, q, psi)
    return a


def ntt_direct(a, logN, q, psi):
    a = _u(a)
    out = np.zeros_like(a)
    _lib.or_ntt_direct(_p(a), _p(out), logN, q, psi)
    return out


def negacyclic_schoolbook(a, b, q):
    a, b = _u(a), _u(b)
    out = np.zeros_like(a)
    _lib.or_negacyclic_schoolbook(_p(a), _p(b), _p(out), a.size, q)
    return out


def _binop(name):
    f = getattr(_lib, name)

    def op(a, b, q):
        a, b = _u(a), _u(b)
        out = np.empty_like(a)
        f(_p(a), _p(b), _p(out), a.size, q)
        return out
    return op


vec_add = _binop("or_vec_add")
vec_sub = _binop("or_vec_sub")
vec_mul = _binop("or_vec_mul")


def vec_scalar_mul(a, c, q):
    a = _u(a)
    out = np.empty_like(a)
    _lib.or_vec_scalar_mul(_p(a), c % q, _p(out), a.size, q)
    return out


def vec_mac_scalar(acc, a, c, q):
    """acc += a * c (mod q), in place."""
    a = _u(a)
    _lib.or_vec_mac_scalar(_p(a), c % q, _p(acc), a.size, q)


def vec_mac(acc, a, b, q):
    """acc += a * b (mod q), in place."""
    a, b = _u(a), _u(b)
    _lib.or_vec_mac(_p(a), _p(b), _p(acc), a.size, q)


def from_signed(a, q):
    a = np.ascontiguousarray(a, dtype=np.int64)
    out = np.empty(a.size, dtype=np.uint64)
    _lib.or_vec_from_signed(_p(a), _p(out), a.size, q)
    return out


def centre(a, q):
    a = _u(a)
    out = np.empty(a.size, dtype=np.int64)
    _lib.or_vec_centre(_p(a), _p(out), a.size, q)
    return out


def reduce(a, q):
    a = _u(a)
    out = np.empty_like(a)
    _lib.or_vec_reduce(_p(a), _p(out), a.size, q)
    return out


def gather(a, perm):
    a = _u(a)
    perm = np.ascontiguousarray(perm, dtype=np.int64)
    out = np.empty_like(a)
    _lib.or_vec_gather(_p(a), _p(perm), _p(out), a.size)
    return out


def mix64(z):
    return int(_lib.or_mix64(z))


def word(master, tag, n):
    return int(_lib.or_word(master, tag, n))


def chacha_quarter(a, b, c, d):
    s = np.array([a, b, c, d], dtype=np.uint32)
    _lib.or_chacha_quarter(_p(s), 0, 1, 2, 3)
    return tuple(int(v) for v in s)


def chacha20_block(key8, counter, nonce3):
    k = np.ascontiguousarray(key8, dtype=np.uint32)
    nc = np.ascontiguousarray(nonce3, dtype=np.uint32)
    out = np.empty(16, dtype=np.uint32)
    _lib.or_chacha20_block(_p(k), counter, _p(nc), _p(out))
    return out


def set_generator(kind, key6=None):
    """Generator of every sampler: "splitmix64" (default) or "chacha20" keyed by
    (master seed, key6: six 32-bit words of key material)."""
    k = np.ascontiguousarray(key6 if key6 is not None else np.zeros(6), dtype=np.uint32)
    _lib.or_set_generator({"splitmix64": 0, "chacha20": 1}[kind], _p(k))


def sample_uniform(master, tag, q, n):
    out = np.empty(n, dtype=np.uint64)
    _lib.or_sample_uniform(master, tag, q, _p(out), n)
    return out


def sample_ternary(master, tag, n):
    out = np.empty(n, dtype=np.int64)
    _lib.or_sample_ternary(master, tag, _p(out), n)
    return out


def sample_cbd21(master, tag, n):
    out = np.empty(n, dtype=np.int64)
    _lib.or_sample_cbd21(master, tag, _p(out), n)
    return out


class EncodeError(RuntimeError):
    pass


def encode(z, logN, scale):
    """Round(scale * tau^-1(z)) as N signed 64-bit coefficients (z real, N/2 slots)."""
    z = np.ascontiguousarray(z, dtype=np.float64)
    assert z.size == (1 << logN) // 2
    out = np.empty(1 << logN, dtype=np.int64)
    rc = _lib.or_encode(_p(z), logN, float(scale), _p(out))
    if rc < 0:
        raise EncodeError(f"encode failed with status {rc}")
    return out


def encode_complex(z, logN, scale):
    """Round(scale * tau^-1(z)) for complex slot values z (N/2 of them)."""
    z = np.asarray(z, dtype=np.complex128)
    assert z.size == (1 << logN) // 2
    zr = np.ascontiguousarray(z.real)
    zi = np.ascontiguousarray(z.imag)
    out = np.empty(1 << logN, dtype=np.int64)
    rc = _lib.or_encode_complex(_p(zr), _p(zi), logN, float(scale), _p(out))
    if rc < 0:
        raise EncodeError(f"encode failed with status {rc}")
    return out


def decode(m, logN, scale):
    m = np.ascontiguousarray(m, dtype=np.int64)
    out = np.empty((1 << logN) // 2, dtype=np.float64)
    _lib.or_decode(_p(m), logN, float(scale), _p(out))
    return out


def encode_direct_real(z, logN, scale):
    """Unrounded scale * tau^-1(z) from the definition in quad precision (tiny N only)."""
    z = np.ascontiguousarray(z, dtype=np.float64)
    out = np.empty(1 << logN, dtype=np.float64)
    _lib.or_encode_direct_real(_p(z), logN, float(scale), _p(out))
    return out
