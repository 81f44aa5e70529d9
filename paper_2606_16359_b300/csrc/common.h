// Internal definitions shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/fenc.h"

typedef uint64_t u64;
typedef int64_t i64;
typedef unsigned __int128 u128;
typedef __int128 i128;

namespace fe {

// ---------------------------------------------------------------------------
// error reporting (thread-local message, integer status codes)
// ---------------------------------------------------------------------------
void set_error(const std::string& msg);
int fail(int code, const std::string& msg);

// A failed call is reported once: its error (if not sticky, e.g. a failed
// allocation) is cleared so that a later call's cudaGetLastError() check does
// not report it again.
#define FE_CUDA_TRY(expr)                                                                  \
    do {                                                                                   \
        cudaError_t _e = (expr);                                                           \
        if (_e != cudaSuccess) {                                                           \
            (void)cudaGetLastError();                                                      \
            return ::fe::fail(FE_ECUDA, std::string(#expr) + ": " + cudaGetErrorString(_e)); \
        }                                                                                  \
    } while (0)

// device buffers must start on a 16-byte boundary (the kernels use 16-byte accesses)
#define FE_ALIGNED(p)                                                                      \
    do {                                                                                   \
        if (((uintptr_t)(p)) & 15) return ::fe::fail(FE_EINVAL, #p " is not 16-byte aligned"); \
    } while (0)

#define FE_TRY(expr)                  \
    do {                              \
        int _rc = (expr);             \
        if (_rc != FE_OK) return _rc; \
    } while (0)

// ---------------------------------------------------------------------------
// A modulus with the constants its reductions need.
//   ratio = floor(2^128 / q) as (hi, lo) words, for 128-bit Barrett reduction.
// ---------------------------------------------------------------------------
// Generator of the samplers (see prng.cuh): kind and ChaCha20 key material.
enum : int { kGenSplitMix64 = 0, kGenChaCha20 = 1 };
struct GenKey {
    int kind;
    uint32_t k[6];
};

struct Modulus {
    u64 q;
    u64 ratio_hi, ratio_lo;  // floor(2^128 / q)
    u64 mu88;                // floor(2^88 / q) (q > 2^24), for reduce_narrow
};

#if defined(__CUDACC__)
// ---------------------------------------------------------------------------
// Device modular arithmetic.  All moduli are odd primes below 2^61, inputs to
// the *_mod helpers are fully reduced (< q) unless stated.
// ---------------------------------------------------------------------------
__device__ __forceinline__ u64 add_mod(u64 a, u64 b, u64 q) {
    u64 s = a + b;
    return s >= q ? s - q : s;
}
__device__ __forceinline__ u64 sub_mod(u64 a, u64 b, u64 q) { return a >= b ? a - b : a + q - b; }
// Shoup multiplication by a constant w with wq = floor(w 2^64 / q); any a < 2^64.
__device__ __forceinline__ u64 mul_shoup(u64 a, u64 w, u64 wq, u64 q) {
    u64 hi = __umul64hi(a, wq);
    u64 r = a * w - hi * q;
    return r >= q ? r - q : r;
}
// 128-bit Barrett reduction of x = (hi, lo) modulo m.q (< 2^62).  The quotient
// estimate floor(x * ratio / 2^128) drops the low word of lo * ratio_lo and is at
// most 2 below floor(x / q), so two conditional subtractions finish the job.
__device__ __forceinline__ u64 reduce128(u64 hi, u64 lo, const Modulus& m) {
    u64 c0 = __umul64hi(lo, m.ratio_lo);
    u128 p1 = (u128)lo * m.ratio_hi;
    u128 p2 = (u128)hi * m.ratio_lo;
    u128 mid = (u128)c0 + (u64)p1 + (u64)p2;
    u64 qhat = hi * m.ratio_hi + (u64)(p1 >> 64) + (u64)(p2 >> 64) + (u64)(mid >> 64);
    u64 r = lo - qhat * m.q;
    if (r >= m.q) r -= m.q;
    if (r >= m.q) r -= m.q;
    return r;
}
__device__ __forceinline__ u64 reduce128(u128 x, const Modulus& m) {
    return reduce128((u64)(x >> 64), (u64)x, m);
}
// x mod q for x < 2^84 and 2^25 <= q < 2^62 (sums of up to 16 products of
// residues below 2^40).  qhat = floor(floor(x / 2^24) mu88 / 2^64) is at most
// x / q and misses it by less than x / 2^88 + 2^24 / q < 1 (the two floors), so
// it is floor(x / q) or one less and one conditional subtraction finishes: one
// 64x64 high product and one low product instead of reduce128's four and one.
__device__ __forceinline__ u64 reduce_narrow(u128 x, const Modulus& m) {
    const u64 qhat = __umul64hi((u64)(x >> 24), m.mu88);
    const u64 r = (u64)x - qhat * m.q;
    return r >= m.q ? r - m.q : r;
}
// Exact sum of products x y of operands below 2^40, in three 32-bit words
// (w2, w1, w0).  With the halves x = x1 2^32 + x0, y = y1 2^32 + y0 (x1, y1 <
// 2^8), x y = x0 y0 + (x0 y1 + x1 y0) 2^32 + x1 y1 2^64; each partial product
// is added to its words by 32-bit multiply-adds with carries: seven per term,
// against the 64x64-bit high and low products and the 128-bit addition of a
// u128 sum.  A term adds at most 2^16 + 2^9 + 3 to w2 (x1 y1 < 2^16, the high
// words of the cross products below 2^8, three carries), so 2^15 terms fit.
struct Acc40 {
    uint32_t w0, w1, w2;
};
__device__ __forceinline__ void acc40_zero(Acc40& a) { a.w0 = a.w1 = a.w2 = 0; }
__device__ __forceinline__ void acc40_mad(Acc40& a, u64 x, u64 y) {
    const uint32_t x0 = (uint32_t)x, x1 = (uint32_t)(x >> 32), y0 = (uint32_t)y, y1 = (uint32_t)(y >> 32);
    asm("mad.lo.cc.u32 %0, %3, %4, %0;\n\t"
        "madc.hi.cc.u32 %1, %3, %4, %1;\n\t"
        "madc.lo.u32 %2, %5, %6, %2;\n\t"
        "mad.lo.cc.u32 %1, %3, %6, %1;\n\t"
        "madc.hi.u32 %2, %3, %6, %2;\n\t"
        "mad.lo.cc.u32 %1, %5, %4, %1;\n\t"
        "madc.hi.u32 %2, %5, %4, %2;"
        : "+r"(a.w0), "+r"(a.w1), "+r"(a.w2)
        : "r"(x0), "r"(y0), "r"(x1), "r"(y1));
}
__device__ __forceinline__ u128 acc40_value(const Acc40& a) {
    return ((u128)a.w2 << 64) | ((u64)a.w1 << 32) | a.w0;
}
// Exact sum of products x y of operands below 2^36, as a + b 2^24.  With
// x = x0 + x1 2^32 (x1 < 2^4) and y = yl + yh 2^24 (yl < 2^24, yh < 2^12):
//   a += x yl = x0 yl + (x1 yl) 2^32   (below 2^60: one widening and one 32-bit multiply-add)
//   b += x yh = x0 yh + (x1 yh) 2^32   (below 2^48: the same)
// so a product costs two widening and two 32-bit multiply-adds with no carry
// chain.  Sixteen terms fit a; acc36_fold moves a's high part into b (every 16
// terms), after which 2^15 more terms fit b.
struct Acc36 {
    u64 a, b;
};
__device__ __forceinline__ void acc36_zero(Acc36& s) { s.a = s.b = 0; }
__device__ __forceinline__ void acc36_mad(Acc36& s, u64 x, uint32_t yl, uint32_t yh) {
    const uint32_t x0 = (uint32_t)x, x1 = (uint32_t)(x >> 32);
    asm("{ .reg .u32 lo, hi;\n\t"
        "mad.wide.u32 %0, %2, %3, %0;\n\t"
        "mov.b64 {lo, hi}, %0;\n\t"
        "mad.lo.u32 hi, %4, %3, hi;\n\t"
        "mov.b64 %0, {lo, hi};\n\t"
        "mad.wide.u32 %1, %2, %5, %1;\n\t"
        "mov.b64 {lo, hi}, %1;\n\t"
        "mad.lo.u32 hi, %4, %5, hi;\n\t"
        "mov.b64 %1, {lo, hi}; }"
        : "+l"(s.a), "+l"(s.b)
        : "r"(x0), "r"(yl), "r"(x1), "r"(yh));
}
__device__ __forceinline__ void acc36_fold(Acc36& s) {
    s.b += s.a >> 24;
    s.a &= (1ull << 24) - 1;
}
__device__ __forceinline__ u128 acc36_value(const Acc36& s) { return ((u128)s.b << 24) + s.a; }
__device__ __forceinline__ uint32_t split24_lo(u64 y) { return (uint32_t)y & ((1u << 24) - 1); }
__device__ __forceinline__ uint32_t split24_hi(u64 y) { return (uint32_t)(y >> 24); }
__device__ __forceinline__ u64 mul_mod(u64 a, u64 b, const Modulus& m) {
    return reduce128((u128)a * b, m);
}
// signed value (|v| < 2^63) to its residue mod q
__device__ __forceinline__ u64 from_signed(i64 v, u64 q) {
    i64 r = v % (i64)q;
    return (u64)(r < 0 ? r + (i64)q : r);
}
// centred representative of a residue: (-q/2, q/2]
__device__ __forceinline__ i64 centre(u64 a, u64 q) { return a > (q >> 1) ? (i64)a - (i64)q : (i64)a; }
#endif

// ---------------------------------------------------------------------------
// Host helpers
// ---------------------------------------------------------------------------
u64 h_mulmod(u64 a, u64 b, u64 q);
u64 h_powmod(u64 a, u64 e, u64 q);
u64 h_invmod(u64 a, u64 q);
Modulus make_modulus(u64 q);
u64 shoup_of(u64 w, u64 q);  // floor(w 2^64 / q)

}  // namespace fe
