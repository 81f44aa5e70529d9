/*
 * CPU oracle: scalar modular-arithmetic and transform primitives.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is part of the plain, slow reference
 * that the CUDA library is checked against.  Only tests/, the smoke check and
 * the CPU-baseline leg of bench.py may load it.  It shares no code, header,
 * table or constant generator with the CUDA path.
 *
 * Everything here is written for obviousness, not speed: products use
 * unsigned __int128 followed by `%`, transforms are textbook recursions.
 *
 * What each function follows:
 *   - CKKS over Z_q[X]/(X^N+1) with RNS limbs: Sec. 2 (CKKS background), the
 *     primitives Add / PMult / CMult / Rot / Rescale.
 *   - Rotation = automorphism + key switch: Eq. 1.
 *   - Canonical-embedding encode/decode: the slot encoding that the CKKS
 *     background section names (N/2 slots, scale Delta).
 */
#include <math.h>
#include <quadmath.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef uint64_t u64;
typedef int64_t i64;
typedef unsigned __int128 u128;
typedef __int128 i128;

/* ------------------------------------------------------------------ */
/* Modular basics                                                      */
/* ------------------------------------------------------------------ */

u64 or_mulmod(u64 a, u64 b, u64 q) { return (u64)(((u128)a * b) % q); }

u64 or_powmod(u64 a, u64 e, u64 q) {
    u64 r = 1 % q;
    a %= q;
    while (e) {
        if (e & 1) r = or_mulmod(r, a, q);
        a = or_mulmod(a, a, q);
        e >>= 1;
    }
    return r;
}

/* inverse by Fermat (q prime) */
u64 or_invmod(u64 a, u64 q) { return or_powmod(a, q - 2, q); }

/* Deterministic Miller-Rabin for 64-bit n (bases 2..37 are sufficient). */
int or_is_prime(u64 n) {
    static const u64 bases[12] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    if (n < 2) return 0;
    for (int i = 0; i < 12; i++) {
        if (n == bases[i]) return 1;
        if (n % bases[i] == 0) return 0;
    }
    u64 d = n - 1;
    int s = 0;
    while ((d & 1) == 0) { d >>= 1; s++; }
    for (int i = 0; i < 12; i++) {
        u64 x = or_powmod(bases[i], d, n);
        if (x == 1 || x == n - 1) continue;
        int composite = 1;
        for (int r = 1; r < s; r++) {
            x = or_mulmod(x, x, n);
            if (x == n - 1) { composite = 0; break; }
        }
        if (composite) return 0;
    }
    return 1;
}

/*
 * The primes q with q = 1 (mod 2N) and q < 2^bits, taken in descending order;
 * entries [skip, skip+count) of that sequence are written to out.
 * Returns 0 on success, -1 if the sequence runs out.
 */
int or_ntt_primes(int logN, int bits, int skip, int count, u64 *out) {
    u64 twoN = (u64)2 << logN;
    u64 q = ((u64)1 << bits) - twoN + 1;
    int found = 0;
    while (found < skip + count) {
        if (q < twoN) return -1;
        if (or_is_prime(q)) {
            if (found >= skip) out[found - skip] = q;
            found++;
        }
        q -= twoN;
    }
    return 0;
}

/* The smallest primitive 2N-th root of unity mod q (the minimum over all N of them). */
u64 or_min_psi(u64 q, int logN) {
    u64 N = (u64)1 << logN;
    u64 twoN = 2 * N;
    u64 c = 0;
    for (u64 x = 2; x < q; x++) {
        u64 t = or_powmod(x, (q - 1) / twoN, q);
        if (or_powmod(t, N, q) == q - 1) { c = t; break; }
    }
    /* all primitive 2N-th roots are c^(odd) */
    u64 best = c, c2 = or_mulmod(c, c, q), cur = c;
    for (u64 t = 0; t < N; t++) {
        if (cur < best) best = cur;
        cur = or_mulmod(cur, c2, q);
    }
    return best;
}

static u64 brv(u64 x, int bits) {
    u64 r = 0;
    for (int i = 0; i < bits; i++) { r = (r << 1) | (x & 1); x >>= 1; }
    return r;
}

/* ------------------------------------------------------------------ */
/* Negacyclic NTT, defined as NTT(a)[i] = a(psi^(2*brv(i)+1)) mod q     */
/* ------------------------------------------------------------------ */

/* O(N^2) direct evaluation of the definition (used for small N). */
void or_ntt_direct(const u64 *a, u64 *out, int logN, u64 q, u64 psi) {
    u64 N = (u64)1 << logN;
    for (u64 i = 0; i < N; i++) {
        u64 x = or_powmod(psi, 2 * brv(i, logN) + 1, q);
        u64 acc = 0, xp = 1;
        for (u64 j = 0; j < N; j++) {
            acc = (u64)(((u128)acc + (u128)a[j] * xp) % q);
            xp = or_mulmod(xp, x, q);
        }
        out[i] = acc;
    }
}

/* textbook recursive radix-2 cyclic DFT over Z_q:  B[k] = sum_j b[j] w^(j k) */
static void dft_rec(u64 *b, u64 n, u64 w, u64 q) {
    if (n == 1) return;
    u64 h = n / 2;
    u64 *ev = malloc(h * sizeof(u64)), *od = malloc(h * sizeof(u64));
    for (u64 j = 0; j < h; j++) { ev[j] = b[2 * j]; od[j] = b[2 * j + 1]; }
    u64 w2 = or_mulmod(w, w, q);
    dft_rec(ev, h, w2, q);
    dft_rec(od, h, w2, q);
    u64 wk = 1;
    for (u64 k = 0; k < h; k++) {
        u64 t = or_mulmod(wk, od[k], q);
        b[k] = (ev[k] + t) % q;
        b[k + h] = (ev[k] + q - t) % q;
        wk = or_mulmod(wk, w, q);
    }
    free(ev);
    free(od);
}

/*
 * a(psi^(2k+1)) = sum_j (a_j psi^j) (psi^2)^(jk): twist by psi^j, cyclic DFT
 * with omega = psi^2, then store entry k at position brv(k).
 */
void or_ntt(u64 *a, int logN, u64 q, u64 psi) {
    u64 N = (u64)1 << logN;
    u64 *b = malloc(N * sizeof(u64));
    u64 pj = 1;
    for (u64 j = 0; j < N; j++) { b[j] = or_mulmod(a[j], pj, q); pj = or_mulmod(pj, psi, q); }
    dft_rec(b, N, or_mulmod(psi, psi, q), q);
    for (u64 k = 0; k < N; k++) a[brv(k, logN)] = b[k];
    free(b);
}

/* inverse of or_ntt: undo the reorder, inverse DFT (omega^-1, 1/N), untwist by psi^-j */
void or_intt(u64 *a, int logN, u64 q, u64 psi) {
    u64 N = (u64)1 << logN;
    u64 *b = malloc(N * sizeof(u64));
    for (u64 k = 0; k < N; k++) b[k] = a[brv(k, logN)];
    u64 psi_inv = or_invmod(psi, q);
    dft_rec(b, N, or_mulmod(psi_inv, psi_inv, q), q);
    u64 n_inv = or_invmod(N % q, q), pj = n_inv;
    for (u64 j = 0; j < N; j++) { a[j] = or_mulmod(b[j], pj, q); pj = or_mulmod(pj, psi_inv, q); }
    free(b);
}

/* schoolbook product in Z_q[X]/(X^N+1) */
void or_negacyclic_schoolbook(const u64 *a, const u64 *b, u64 *out, int N, u64 q) {
    for (int k = 0; k < N; k++) out[k] = 0;
    for (int i = 0; i < N; i++)
        for (int j = 0; j < N; j++) {
            u64 p = or_mulmod(a[i], b[j], q);
            int k = i + j;
            if (k < N) out[k] = (out[k] + p) % q;
            else out[k - N] = (out[k - N] + q - p) % q;
        }
}

/* ------------------------------------------------------------------ */
/* Vector helpers over one limb                                        */
/* ------------------------------------------------------------------ */

void or_vec_add(const u64 *a, const u64 *b, u64 *o, int n, u64 q) {
    for (int i = 0; i < n; i++) o[i] = (a[i] + b[i]) % q;
}
void or_vec_sub(const u64 *a, const u64 *b, u64 *o, int n, u64 q) {
    for (int i = 0; i < n; i++) o[i] = (a[i] + q - b[i]) % q;
}
void or_vec_mul(const u64 *a, const u64 *b, u64 *o, int n, u64 q) {
    for (int i = 0; i < n; i++) o[i] = or_mulmod(a[i], b[i], q);
}
void or_vec_scalar_mul(const u64 *a, u64 c, u64 *o, int n, u64 q) {
    for (int i = 0; i < n; i++) o[i] = or_mulmod(a[i], c % q, q);
}
/* o += a * c (mod q) */
void or_vec_mac_scalar(const u64 *a, u64 c, u64 *o, int n, u64 q) {
    for (int i = 0; i < n; i++) o[i] = (o[i] + or_mulmod(a[i], c % q, q)) % q;
}
/* o += a * b (mod q) */
void or_vec_mac(const u64 *a, const u64 *b, u64 *o, int n, u64 q) {
    for (int i = 0; i < n; i++) o[i] = (o[i] + or_mulmod(a[i], b[i], q)) % q;
}
/* signed 64-bit integers -> residues mod q */
void or_vec_from_signed(const i64 *a, u64 *o, int n, u64 q) {
    for (int i = 0; i < n; i++) {
        i64 r = a[i] % (i64)q;
        o[i] = (u64)(r < 0 ? r + (i64)q : r);
    }
}
/* residues mod q -> centred representative in (-q/2, q/2] */
void or_vec_centre(const u64 *a, i64 *o, int n, u64 q) {
    for (int i = 0; i < n; i++) o[i] = (a[i] > q / 2) ? (i64)a[i] - (i64)q : (i64)a[i];
}
/* o[i] = a[i] mod q for values already in [0, 2^64) */
void or_vec_reduce(const u64 *a, u64 *o, int n, u64 q) {
    for (int i = 0; i < n; i++) o[i] = a[i] % q;
}
/* o[i] = a[perm[i]] */
void or_vec_gather(const u64 *a, const i64 *perm, u64 *o, int n) {
    for (int i = 0; i < n; i++) o[i] = a[perm[i]];
}

/* ------------------------------------------------------------------ */
/* Counter-based generator: SplitMix64 (Steele, Lea & Flood 2014)      */
/* ------------------------------------------------------------------ */

#define GOLDEN_GAMMA 0x9E3779B97F4A7C15ULL

u64 or_mix64(u64 z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* ChaCha20 (RFC 8439, Sec. 2.1-2.3).  The quarter round on four 32-bit
 * words: add, xor, rotate left by 16, 12, 8 and 7. */
static uint32_t rotl32(uint32_t x, int r) { return (x << r) | (x >> (32 - r)); }

void or_chacha_quarter(uint32_t *s, int a, int b, int c, int d) {
    s[a] += s[b]; s[d] ^= s[a]; s[d] = rotl32(s[d], 16);
    s[c] += s[d]; s[b] ^= s[c]; s[b] = rotl32(s[b], 12);
    s[a] += s[b]; s[d] ^= s[a]; s[d] = rotl32(s[d], 8);
    s[c] += s[d]; s[b] ^= s[c]; s[b] = rotl32(s[b], 7);
}

/* Block function: state = the four constants "expand 32-byte k", the eight
 * key words, the block counter and the three nonce words; ten double rounds
 * (four column quarter rounds, then four diagonal ones); the output is the
 * final state plus the initial state, word by word. */
void or_chacha20_block(const uint32_t key[8], uint32_t counter, const uint32_t nonce[3], uint32_t out[16]) {
    uint32_t init[16] = {0x61707865u, 0x3320646eu, 0x79622d32u, 0x6b206574u};
    for (int i = 0; i < 8; i++) init[4 + i] = key[i];
    init[12] = counter;
    for (int i = 0; i < 3; i++) init[13 + i] = nonce[i];
    uint32_t x[16];
    memcpy(x, init, sizeof x);
    for (int round = 0; round < 10; round++) {
        or_chacha_quarter(x, 0, 4, 8, 12);
        or_chacha_quarter(x, 1, 5, 9, 13);
        or_chacha_quarter(x, 2, 6, 10, 14);
        or_chacha_quarter(x, 3, 7, 11, 15);
        or_chacha_quarter(x, 0, 5, 10, 15);
        or_chacha_quarter(x, 1, 6, 11, 12);
        or_chacha_quarter(x, 2, 7, 8, 13);
        or_chacha_quarter(x, 3, 4, 9, 14);
    }
    for (int i = 0; i < 16; i++) out[i] = x[i] + init[i];
}

/* Generator of the samplers: 0 = SplitMix64 (default), 1 = ChaCha20 keyed by
 * (master seed, 192 bits of key material). */
static int g_gen = 0;
static uint32_t g_key6[6];

void or_set_generator(int kind, const uint32_t *key6) {
    g_gen = kind;
    for (int i = 0; i < 6; i++) g_key6[i] = key6 ? key6[i] : 0;
}

/* Word n of stream `tag`:
 *   SplitMix64: output number (n+1) of the stream whose seed is output number
 *   (tag+1) of the generator seeded with `master`;
 *   ChaCha20: key = (master low, master high, key material), nonce = (tag low,
 *   tag high, 0), block counter n / 8; the word is output words 2 (n mod 8) and
 *   2 (n mod 8) + 1 of that block, low word first. */
u64 or_word(u64 master, u64 tag, u64 n) {
    if (g_gen == 1) {
        uint32_t key[8] = {(uint32_t)master, (uint32_t)(master >> 32)};
        for (int i = 0; i < 6; i++) key[2 + i] = g_key6[i];
        const uint32_t nonce[3] = {(uint32_t)tag, (uint32_t)(tag >> 32), 0};
        uint32_t blk[16];
        or_chacha20_block(key, (uint32_t)(n >> 3), nonce, blk);
        const int j = 2 * (int)(n & 7);
        return (u64)blk[j] | ((u64)blk[j + 1] << 32);
    }
    u64 s = or_mix64(master + (tag + 1) * GOLDEN_GAMMA);
    return or_mix64(s + (n + 1) * GOLDEN_GAMMA);
}

/* uniform residue mod q: floor(w * q / 2^64) */
void or_sample_uniform(u64 master, u64 tag, u64 q, u64 *out, int n) {
    for (int i = 0; i < n; i++) out[i] = (u64)(((u128)or_word(master, tag, i) * q) >> 64);
}

/* ternary in {-1, 0, 1}: floor(w * 3 / 2^64) - 1 */
void or_sample_ternary(u64 master, u64 tag, i64 *out, int n) {
    for (int i = 0; i < n; i++) out[i] = (i64)(((u128)or_word(master, tag, i) * 3) >> 64) - 1;
}

/* centred binomial, eta = 21: popcount of the low 21 bits minus popcount of the next 21 */
void or_sample_cbd21(u64 master, u64 tag, i64 *out, int n) {
    for (int i = 0; i < n; i++) {
        u64 w = or_word(master, tag, i);
        int a = 0, b = 0;
        for (int k = 0; k < 21; k++) a += (int)((w >> k) & 1);
        for (int k = 21; k < 42; k++) b += (int)((w >> k) & 1);
        out[i] = a - b;
    }
}

/* ------------------------------------------------------------------ */
/* Canonical-embedding encode / decode                                 */
/*                                                                     */
/* Slot l <-> the root zeta^(5^l mod 2N), zeta = exp(i*pi/N).  For a real */
/* slot vector z the encoded polynomial has coefficients                */
/*   m_j = round( Delta * (2/N) * sum_l z_l cos(pi * (5^l * j mod 2N) / N) ) */
/* Rounding is to the nearest integer.                                 */
/* ------------------------------------------------------------------ */

typedef long double ld;

/* iterative radix-2 complex FFT of length M (a power of two), sign -1 or +1,
 * in long double, twiddles exp(sign * 2 pi i k / M) from cosl/sinl. */
static void fft_ld(ld *re, ld *im, u64 M, int sign) {
    int bits = 0;
    while (((u64)1 << bits) < M) bits++;
    for (u64 i = 0; i < M; i++) {
        u64 j = brv(i, bits);
        if (j > i) {
            ld t = re[i]; re[i] = re[j]; re[j] = t;
            t = im[i]; im[i] = im[j]; im[j] = t;
        }
    }
    const ld PI = 3.141592653589793238462643383279502884L;
    for (u64 len = 2; len <= M; len <<= 1) {
        u64 h = len / 2;
        for (u64 k = 0; k < h; k++) {
            ld ang = sign * 2.0L * PI * (ld)k / (ld)len;
            ld wr = cosl(ang), wi = sinl(ang);
            for (u64 s = 0; s < M; s += len) {
                u64 a = s + k, b = s + k + h;
                ld tr = re[b] * wr - im[b] * wi;
                ld ti = re[b] * wi + im[b] * wr;
                re[b] = re[a] - tr; im[b] = im[a] - ti;
                re[a] += tr; im[a] += ti;
            }
        }
    }
}

/* quad-precision value of Delta * (2/N) * sum_l z_l cos(pi * t_l / N), t_l = 5^l j mod 2N.
 * cq (optional): cq[t] = cosq(pi t / N) for t in [0, 2N), the same quad values the
 * loop would compute term by term. */
static __float128 encode_coef_quad(const double *z, int logN, double scale, u64 j, const __float128 *cq) {
    u64 N = (u64)1 << logN, twoN = 2 * N;
    __float128 acc = 0;
    u64 e = 1;
    for (u64 l = 0; l < N / 2; l++) {
        u64 t = (e * j) % twoN;
        acc += (__float128)z[l] * (cq ? cq[t] : cosq(M_PIq * (__float128)t / (__float128)N));
        e = (e * 5) % twoN;
    }
    return acc * (__float128)scale * 2 / (__float128)N;
}

/*
 * Encode N/2 real slot values at scale `scale` into N signed coefficients.
 * Path: long-double FFT of length 2N over the array A with A[5^l] = A[2N-5^l] = z_l;
 * m_j = Delta * Re(DFT(A)[j]) / N.  Coefficients whose long-double value lies
 * within a guard band of a rounding boundary are recomputed from the definition
 * in quad precision.
 * Returns the number of recomputed coefficients, or -1 if a coefficient is
 * still within 2^-40 of a half-integer after recomputation (ambiguous rounding),
 * or -2 if a coefficient does not fit in 62 bits.
 */
int or_encode(const double *z, int logN, double scale, i64 *out) {
    u64 N = (u64)1 << logN, M = 2 * N;
    ld *re = calloc(M, sizeof(ld)), *im = calloc(M, sizeof(ld));
    u64 e = 1;
    ld l1 = 0;
    for (u64 l = 0; l < N / 2; l++) {
        re[e] += z[l];
        re[M - e] += z[l];
        l1 += fabsl((ld)z[l]);
        e = (e * 5) % M;
    }
    fft_ld(re, im, M, -1);
    /* error of the long-double FFT is far below this band for the sizes used */
    ld bound = (ld)scale * 2.0L * l1 / (ld)N;
    ld guard = bound * (ld)logN * 0x1p-52L;
    if (guard < 0x1p-30L) guard = 0x1p-30L;
    int fallbacks = 0;
    __float128 *cq = NULL;
    for (u64 j = 0; j < N; j++) {
        ld v = (ld)scale * re[j] / (ld)N;
        ld fl = floorl(v);
        ld frac = v - fl;
        if (fabsl(frac - 0.5L) < guard) {
            if (!cq) { /* first fallback of this call: the cosines of every angle pi t / N */
                cq = malloc(M * sizeof(__float128));
                for (u64 t = 0; t < M; t++) cq[t] = cosq(M_PIq * (__float128)t / (__float128)N);
            }
            __float128 vq = encode_coef_quad(z, logN, scale, j, cq);
            __float128 fq = floorq(vq);
            __float128 fracq = vq - fq;
            if (fabsq(fracq - 0.5Q) < 0x1p-40Q) { free(re); free(im); free(cq); return -1; }
            fl = (ld)fq;
            frac = (ld)fracq;
            fallbacks++;
        }
        ld r = frac > 0.5L ? fl + 1 : fl;
        if (fabsl(r) > 0x1p62L) { free(re); free(im); free(cq); return -2; }
        out[j] = (i64)r;
    }
    free(re);
    free(im);
    free(cq);
    return fallbacks;
}

/* quad-precision value of Delta * (2/N) * sum_l (re_l cos(pi t_l / N) + im_l sin(pi t_l / N)),
 * t_l = 5^l j mod 2N: the coefficient of the complex slot vector re + i im.  cq as above;
 * sin(pi t / N) is read as cq[(t + 3N/2) mod 2N] = cos(pi (t - N/2) / N). */
static __float128 encode_coef_quad_complex(const double *re, const double *im, int logN, double scale, u64 j,
                                           const __float128 *cq) {
    u64 N = (u64)1 << logN, twoN = 2 * N;
    __float128 acc = 0;
    u64 e = 1;
    for (u64 l = 0; l < N / 2; l++) {
        u64 t = (e * j) % twoN;
        acc += (__float128)re[l] * cq[t] + (__float128)im[l] * cq[(t + 3 * N / 2) % twoN];
        e = (e * 5) % twoN;
    }
    return acc * (__float128)scale * 2 / (__float128)N;
}

/*
 * Encode N/2 complex slot values re + i im at scale `scale` into N signed
 * coefficients: the real polynomial whose value at zeta^(5^l) is scale (re_l + i im_l)
 * and at the conjugate root its conjugate.  Path: long-double FFT of length 2N
 * over A with A[5^l] = z_l, A[2N - 5^l] = conj(z_l) (a conjugate-symmetric
 * sequence, so the transform is real); m_j = scale DFT(A)[j] / N.  The guard band
 * and the quad fallback are those of or_encode (with |z_l| in the bound).
 * Returns as or_encode.
 */
int or_encode_complex(const double *zr, const double *zi, int logN, double scale, i64 *out) {
    u64 N = (u64)1 << logN, M = 2 * N;
    ld *re = calloc(M, sizeof(ld)), *im = calloc(M, sizeof(ld));
    u64 e = 1;
    ld l1 = 0;
    for (u64 l = 0; l < N / 2; l++) {
        re[e] += zr[l];
        im[e] += zi[l];
        re[M - e] += zr[l];
        im[M - e] -= zi[l];
        l1 += sqrtl((ld)zr[l] * zr[l] + (ld)zi[l] * zi[l]);
        e = (e * 5) % M;
    }
    fft_ld(re, im, M, -1);
    ld bound = (ld)scale * 2.0L * l1 / (ld)N;
    ld guard = bound * (ld)logN * 0x1p-52L;
    if (guard < 0x1p-30L) guard = 0x1p-30L;
    int fallbacks = 0;
    __float128 *cq = NULL;
    for (u64 j = 0; j < N; j++) {
        ld v = (ld)scale * re[j] / (ld)N;
        ld fl = floorl(v);
        ld frac = v - fl;
        if (fabsl(frac - 0.5L) < guard) {
            if (!cq) {
                cq = malloc(M * sizeof(__float128));
                for (u64 t = 0; t < M; t++) cq[t] = cosq(M_PIq * (__float128)t / (__float128)N);
            }
            __float128 vq = encode_coef_quad_complex(zr, zi, logN, scale, j, cq);
            __float128 fq = floorq(vq);
            __float128 fracq = vq - fq;
            if (fabsq(fracq - 0.5Q) < 0x1p-40Q) { free(re); free(im); free(cq); return -1; }
            fl = (ld)fq;
            frac = (ld)fracq;
            fallbacks++;
        }
        ld r = frac > 0.5L ? fl + 1 : fl;
        if (fabsl(r) > 0x1p62L) { free(re); free(im); free(cq); return -2; }
        out[j] = (i64)r;
    }
    free(re);
    free(im);
    free(cq);
    return fallbacks;
}

/* Decode N signed coefficients into N/2 slot values:
 * z_l = Re( sum_j m_j zeta^(5^l j) ) / Delta. */
void or_decode(const i64 *m, int logN, double scale, double *z) {
    u64 N = (u64)1 << logN, M = 2 * N;
    ld *re = calloc(M, sizeof(ld)), *im = calloc(M, sizeof(ld));
    for (u64 j = 0; j < N; j++) re[j] = (ld)m[j];
    fft_ld(re, im, M, +1);
    u64 e = 1;
    for (u64 l = 0; l < N / 2; l++) {
        z[l] = (double)(re[e] / (ld)scale);
        e = (e * 5) % M;
    }
    free(re);
    free(im);
}

/* Direct O(N^2) reference for encode without rounding (used by tests on tiny N). */
void or_encode_direct_real(const double *z, int logN, double scale, double *out) {
    u64 N = (u64)1 << logN;
    for (u64 j = 0; j < N; j++) out[j] = (double)encode_coef_quad(z, logN, scale, j, NULL);
}
