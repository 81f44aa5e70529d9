// Counter-based generators of the samplers: word n of stream `tag` under the
// master seed, computed independently by every thread.
//   SplitMix64 (Steele, Lea, Flood 2014), the default:
//     word = mix(mix(seed + (tag + 1) g) + (n + 1) g), g = 0x9E3779B97F4A7C15.
//   ChaCha20 (RFC 8439, Sec. 2.3), the cryptographic option: key = (seed low,
//     seed high, six 32-bit words of key material set on the context), nonce =
//     (tag low, tag high, 0), block counter n / 8; the word is output words
//     2 (n mod 8) and 2 (n mod 8) + 1 of that block, low word first.
#pragma once

#include "common.h"  // GenKey

namespace fe {

__device__ __forceinline__ u64 splitmix_mix(u64 z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// quarter round of RFC 8439 Sec. 2.1 on words a, b, c, d
__device__ __forceinline__ void chacha_qr(uint32_t& a, uint32_t& b, uint32_t& c, uint32_t& d) {
    a += b; d ^= a; d = __funnelshift_l(d, d, 16);
    c += d; b ^= c; b = __funnelshift_l(b, b, 12);
    a += b; d ^= a; d = __funnelshift_l(d, d, 8);
    c += d; b ^= c; b = __funnelshift_l(b, b, 7);
}

__device__ __forceinline__ u64 chacha_word(const GenKey& g, u64 seed, u64 tag, u64 n) {
    const uint32_t init[16] = {0x61707865u, 0x3320646eu, 0x79622d32u, 0x6b206574u,
                               (uint32_t)seed, (uint32_t)(seed >> 32), g.k[0], g.k[1], g.k[2], g.k[3], g.k[4],
                               g.k[5], (uint32_t)(n >> 3), (uint32_t)tag, (uint32_t)(tag >> 32), 0u};
    uint32_t x[16];
#pragma unroll
    for (int i = 0; i < 16; i++) x[i] = init[i];
#pragma unroll 1
    for (int r = 0; r < 10; r++) {
        chacha_qr(x[0], x[4], x[8], x[12]);
        chacha_qr(x[1], x[5], x[9], x[13]);
        chacha_qr(x[2], x[6], x[10], x[14]);
        chacha_qr(x[3], x[7], x[11], x[15]);
        chacha_qr(x[0], x[5], x[10], x[15]);
        chacha_qr(x[1], x[6], x[11], x[12]);
        chacha_qr(x[2], x[7], x[8], x[13]);
        chacha_qr(x[3], x[4], x[9], x[14]);
    }
    // words 2 (n mod 8) and 2 (n mod 8) + 1 of the block, selected without
    // dynamic register indexing
    const int j = 2 * (int)(n & 7);
    uint32_t lo = 0, hi = 0;
#pragma unroll
    for (int i = 0; i < 16; i += 2) {
        if (i == j) {
            lo = x[i] + init[i];
            hi = x[i + 1] + init[i + 1];
        }
    }
    return (u64)lo | ((u64)hi << 32);
}

__device__ __forceinline__ u64 gen_word(const GenKey& g, u64 seed, u64 tag, u64 n) {
    if (g.kind == kGenChaCha20) return chacha_word(g, seed, tag, n);
    const u64 gamma = 0x9E3779B97F4A7C15ull;
    return splitmix_mix(splitmix_mix(seed + (tag + 1) * gamma) + (n + 1) * gamma);
}

}  // namespace fe
