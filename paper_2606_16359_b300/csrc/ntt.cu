// Negacyclic NTT / inverse NTT over RNS limbs, batched.
//
// Forward: Cooley-Tukey butterflies with twiddles psi^brv(m + i) (natural order
// in, bit-reversed order out), which computes NTT(a)[i] = a(psi^(2 brv(i) + 1)).
// Inverse: Gentleman-Sande butterflies with psi^-brv(h + i), then N^-1.
//
// One limb (N = N1 * N2) is transformed in two passes.  The stages whose
// butterfly distance is a multiple of N2 act on the N2 columns {x N2 + r}
// independently ("column pass", lines of length N1); the remaining stages act
// on the N1 rows of N2 contiguous elements ("row pass", lines of length N2).
// Stage t of a line of length n with line id `lid` out of `ltot` lines uses
// the twiddle at index (ltot + lid) * (n / 2t) + floor(x / 2t); for the column
// pass ltot = 1, lid = 0, for the row pass ltot = N1, lid = row.
//
// A CTA transforms a tile of lines.  The stages are processed in rounds of up
// to three: each thread keeps 8 elements of a line (stride s = the round's
// smallest distance) in registers and runs the round's butterflies there, so a
// 256-point line takes three rounds instead of eight stages.  The first round
// reads its elements straight from global memory and the last one writes them
// straight back (a warp's accesses cover whole 32-byte sectors); only the
// rounds in between go through the tile in shared memory.  The staged form
// (fe_ctx_set_ntt_path 1) instead loads the whole tile into shared memory with
// coalesced 16-byte accesses first and stores it from there after the last
// round.  Butterflies are Harvey's
// lazy forms with Shoup multiplication: forward values stay in [0, 4q),
// inverse values in [0, 2q), and only the final stage reduces to [0, q)
// (4q < 2^64 since q < 2^62); with all moduli below 2^58 the forward
// transform skips reductions until its last stage (see round_stages).  The first pass may read a separate source
// buffer (out-of-place); the second pass works in place.
#include <algorithm>

#include <cooperative_groups.h>

#include "context.h"

namespace fe {

namespace {

constexpr int kTile = 1024;  // elements per CTA tile (8 KiB)
constexpr int kE = 8;        // elements per thread per round (radix 8; radix 16: 2 kE)

struct NttArgs {
    const u64* src;      // first-pass source (may equal dst)
    size_t src_stride;   // poly stride of src
    u64* dst;
    size_t poly_stride;
    int per_poly;
    const int* mod_map;
    const int* pos_map;
    const Modulus* mods;
    const ulonglong2* tw;  // [n_mod][N] (w, floor(w 2^64 / q))
    const u64* ninv;
    const u64* ninv_sh;
    const u64* ninvw;     // N^-1 times the inverse's last-stage twiddle
    const u64* ninvw_sh;
    int logN, logN2;
};

__device__ __forceinline__ u64 shoup_lazy(u64 a, u64 w, u64 wq, u64 q) {
    return a * w - __umul64hi(a, wq) * q;  // in [0, 2q)
}

// Shoup's product (Shoup; lazy form of Harvey, "Faster arithmetic for
// number-theoretic transforms", 2014) for moduli below 2^36 and inputs
// a < 2^42, from 32-bit multiply-adds only:
//   quotient  Q = floor(a wq63 / 2^63), wq63 = floor(w 2^63 / q) = wq >> 1;
//   result    T = a w - Q q  (mod 2^64), in [0, 2q) since a < 2^63.
// With a = a1 2^32 + a0 (a1 < 2^10) and wq63 = h 2^32 + l (h < 2^31):
//   Z = a0 h + a1 l + floor(a0 l / 2^32) < 2^63 + 2^43 (no 64-bit overflow),
//   Q = 2 a1 h + floor(Z / 2^31)   (exact: the dropped a0 l mod 2^32 term
//   cannot carry past a multiple of 2^31 in Z 2^32 + (a0 l mod 2^32)),
// and T = a w + Q (2^64 - q) mod 2^64 takes two widening multiply-adds for its
// low 64 bits and four 32-bit multiply-adds for the cross terms of its high
// word.  Ten integer multiply instructions against the general form's
// 64 x 64 high product and two 64-bit low products.
__device__ __forceinline__ u64 shoup36(u64 a, u64 w, u64 wq, u64 nq) {
    u64 T;
    asm("{\n\t"
        ".reg .u32 a0, a1, l, h, h2, t, w0, w1, n0, n1, q0, q1, tl, th;\n\t"
        ".reg .u64 Z, W63;\n\t"
        "mov.b64 {a0, a1}, %1;\n\t"
        "mov.b64 {w0, w1}, %2;\n\t"
        "shr.u64 W63, %3, 1;\n\t"
        "mov.b64 {l, h}, W63;\n\t"
        "shl.b32 h2, h, 1;\n\t"
        "mov.b64 {n0, n1}, %4;\n\t"
        "mul.hi.u32 t, a0, l;\n\t"
        "cvt.u64.u32 Z, t;\n\t"
        "mad.wide.u32 Z, a0, h, Z;\n\t"
        "mad.wide.u32 Z, a1, l, Z;\n\t"
        "shr.u64 Z, Z, 31;\n\t"
        "mad.wide.u32 Z, a1, h2, Z;\n\t"
        "mov.b64 {q0, q1}, Z;\n\t"
        "mul.wide.u32 %0, a0, w0;\n\t"
        "mad.wide.u32 %0, q0, n0, %0;\n\t"
        "mov.b64 {tl, th}, %0;\n\t"
        "mad.lo.u32 th, a0, w1, th;\n\t"
        "mad.lo.u32 th, a1, w0, th;\n\t"
        "mad.lo.u32 th, q0, n1, th;\n\t"
        "mad.lo.u32 th, q1, n0, th;\n\t"
        "mov.b64 %0, {tl, th};\n\t"
        "}"
        : "=l"(T)
        : "l"(a), "l"(w), "l"(wq), "l"(nq));
    return T;
}

// One line transform round: `lo` = log2 of the round's smallest distance (s),
// `nst` = number of stages (distances s * 2^(nst-1) .. s), thread holds
// v[r] = line[base + r s] for r < E (E = min(8, line length)), base = blk 8 s + off.
// Stage t = s 2^st needs twiddle index (tw_line << (logn-1-lt)) + (x >> (lt+1)) with
// lt = lo + st; for x = base + r s this is K + (r >> (st+1)), K = (tw_line << (logn-1-lt))
// + (blk << (2-st)), so each stage loads its 8 >> (st+1) distinct twiddles once.
// The three stage slots are unrolled so every register index is a compile-time constant.
// kNoRed (forward only, all moduli < 2^58): no reduction inside the transform;
// each stage adds less than 2q, so values stay below (1 + 2 * 17) q < 2^64.
// kLE = log2 of the elements a thread holds per round (3: radix 8, 4: radix 16).
// fold (inverse only): this round ends the transform; its last stage multiplies its
// sums by N^-1 (fni) and its differences by N^-1 times the stage's twiddle (fwn), so
// that the N^-1 scaling costs no product of its own.
// kPre: load every stage's twiddles before the first stage (row passes, whose
// twiddles differ per row and come from L2), so that their latency overlaps.
template <bool kInv, bool kNoRed, int kLE, bool kQ36 = false, bool kPre = false>
__device__ __forceinline__ void round_stages(u64 (&v)[1 << kLE], int blk, int lo, int nst, int E, int logn,
                                             int tw_line, const ulonglong2* __restrict__ tw, u64 q,
                                             bool fold = false, ulonglong2 fni = {}, ulonglong2 fwn = {}) {
    constexpr int kEE = 1 << kLE, kHalf = kEE / 2;
    const u64 q2 = 2 * q, nq = 0 - q;
    auto mulw = [&](u64 a, const ulonglong2& ww) -> u64 {
        if constexpr (kQ36) return shoup36(a, ww.x, ww.y, nq);
        else return shoup_lazy(a, ww.x, ww.y, q);
    };
    auto load_tw = [&](int si, ulonglong2 (&w)[kHalf]) {
        const int st = kInv ? si : kLE - 1 - si;
        if (st >= nst) return;
        const int lt = lo + st;
        const int K = (tw_line << (logn - 1 - lt)) + (blk << (kLE - 1 - st));
        const int cnt = max(1, E >> (st + 1));
#pragma unroll
        for (int i = 0; i < kHalf; i++)
            if (i < (kHalf >> st) && i < cnt) w[i] = tw[K + i];
    };
    ulonglong2 wpre[kPre ? kLE : 1][kHalf];
    if constexpr (kPre) {
#pragma unroll
        for (int si = 0; si < kLE; si++) load_tw(si, wpre[si]);
    }
#pragma unroll
    for (int si = 0; si < kLE; si++) {
        const int st = kInv ? si : kLE - 1 - si;  // forward: large distances first
        if (st >= nst) continue;
        const int d = 1 << st;
        ulonglong2 w[kHalf];
        if constexpr (kPre) {
#pragma unroll
            for (int i = 0; i < kHalf; i++) w[i] = wpre[si][i];
        } else {
            load_tw(si, w);
        }
#pragma unroll
        for (int r = 0; r < kEE; r++) {
            if ((r & d) || r + d >= E) continue;
            const ulonglong2 ww = w[r >> (st + 1)];
            if (!kInv) {
                u64 X = v[r];
                if (!kNoRed) X = X >= q2 ? X - q2 : X;
                const u64 T = mulw(v[r + d], ww);
                v[r] = X + T;
                v[r + d] = X - T + q2;
            } else if (fold && st == nst - 1) {
                const u64 X = v[r], Y = v[r + d];  // both in [0, 2q): X + Y below 4q
                v[r] = mulw(X + Y, fni);
                v[r + d] = mulw(X - Y + q2, fwn);
            } else {
                const u64 X = v[r], Y = v[r + d];
                u64 S = X + Y;
                v[r] = S >= q2 ? S - q2 : S;
                v[r + d] = mulw(X - Y + q2, ww);
            }
        }
    }
}

// kCol: column pass (lines = columns of length N1) else row pass (lines = rows of length N2).
// kLogN > 0 fixes the ring degree at compile time so that the tile geometry, the
// round structure and every shift fold into constants; kLogN = 0 reads it at run time.
// CTAs of kTile / 2^kLE threads; the bound lets 9 radix-8 CTAs (36 warps) share an SM
// kStaged: the whole tile passes through shared memory before the first round and
// after the last one; otherwise those two rounds access global memory directly.
template <int kLogN, bool kInv, bool kCol, bool kNoRed, int kLE, bool kQ36, bool kStaged>
__global__ void __launch_bounds__(kTile >> kLE, kLE == 3 ? 9 : (kLE == 4 ? 8 : 6)) ntt_pass(NttArgs a, int first) {
    constexpr int kEE = 1 << kLE;
    extern __shared__ u64 tile[];
    const int logN = kLogN ? kLogN : a.logN;
    const int logN2 = kLogN ? kLogN / 2 : a.logN2;
    const int N2 = 1 << logN2, N1 = 1 << (logN - logN2);
    const int logn = kCol ? logN - logN2 : logN2;
    const int n = 1 << logn;
    const int lines = kCol ? min(kTile / N1, N2) : min(kTile / N2, N1);
    const int tiles_per_limb = (kCol ? N2 : N1) / lines;
    const int E = min(kEE, n);
    const int tpl = n / E;  // threads per line
    const int nthr = lines * tpl;
    const int nthreads = kLogN ? (nthr > 32 ? nthr : 32) : (int)blockDim.x;
    const int limb = blockIdx.x / tiles_per_limb;
    const int l0 = (blockIdx.x % tiles_per_limb) * lines;
    const int poly = limb / a.per_poly, jl = limb % a.per_poly;
    const int mi = a.mod_map[jl];
    const int pos = a.pos_map ? a.pos_map[jl] : jl;
    const u64 q = a.mods[mi].q;
    const ulonglong2* tw = a.tw + ((size_t)mi << logN);
    u64* d = a.dst + (size_t)poly * a.poly_stride + ((size_t)pos << logN);
    const u64* s = first ? a.src + (size_t)poly * a.src_stride + ((size_t)pos << logN) : d;
    const int total = lines * n;
    // column pass tile[CIDX(x, c)]: element x of the `lines` columns side by side,
    // with a pad row after every 8 rows; row pass tile[RIDX(row, x)] with one pad
    // word per 8.  The pads spread the strided rounds over the banks: without the
    // column pass's, its unit-stride round put 8 threads of a warp on one bank.
    const int rs = N2 + (N2 >> 3);
#define RIDX(ln, x) ((ln) * rs + (x) + ((x) >> 3))
#define CIDX(x, c) (((x) + ((x) >> 3)) * lines + (c))
    // global offset of element x of line ln of the tile
#define GOFF(ln, x) (kCol ? (size_t)(x) * N2 + l0 + (ln) : (size_t)(l0 + (ln)) * N2 + (x))
    // staged load: each thread issues all of its 16-byte loads before storing to shared memory
    if (kStaged) {
        const int pairs = total >> 1;
#pragma unroll 1
        for (int e0 = 0; e0 < pairs; e0 += 4 * nthreads) {
            ulonglong2 buf[4];
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const int e = e0 + (int)threadIdx.x + k * nthreads;
                if (e < pairs) {
                    const int el = 2 * e;
                    if (kCol) {
                        const int x = el / lines, c = el - x * lines;
                        buf[k] = *reinterpret_cast<const ulonglong2*>(s + (size_t)x * N2 + l0 + c);
                    } else {
                        buf[k] = *reinterpret_cast<const ulonglong2*>(s + (size_t)l0 * N2 + el);
                    }
                }
            }
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const int e = e0 + (int)threadIdx.x + k * nthreads;
                if (e < pairs) {
                    const int el = 2 * e;
                    if (kCol) {
                        const int x = el / lines, c = el - x * lines;
                        const int x1 = (el + 1) / lines, c1 = el + 1 - x1 * lines;
                        tile[CIDX(x, c)] = buf[k].x;
                        tile[CIDX(x1, c1)] = buf[k].y;
                    } else {
                        const int ln = el >> logN2, x = el & (N2 - 1);
                        tile[RIDX(ln, x)] = buf[k].x;
                        tile[RIDX(ln, x + 1)] = buf[k].y;
                    }
                }
            }
        }
    }
    if (kStaged) __syncthreads();
    // the pass that completes the transform reduces to [0, q), fused into the store
    const bool last_pass = kInv ? kCol : !kCol;
    const u64 q2 = 2 * q;
    const u64 ni = a.ninv[mi], nis = a.ninv_sh[mi];
    const u64 qinv64 = a.mods[mi].ratio_hi;  // floor(2^64 / q)
    // forward, no reductions inside the transform (values below 35 q < 2^42 when q < 2^36):
    // quotient from one 32 x 32 product, Q' = floor((x >> 20) mu / 2^32) with
    // mu = floor(2^52 / q) = floor(2^64 / q) >> 12, which is floor(x / q) or one less
    // for 2^25 <= q < 2^36, so x - Q' q lies in [0, 2q)
    auto fin = [&](u64 x, bool folded) -> u64 {
        if (!last_pass) return x;
        if (kInv) {
            if (!folded) x = kQ36 ? shoup36(x, ni, nis, 0 - q) : shoup_lazy(x, ni, nis, q);  // [0, 2q)
        } else if (kNoRed) {
            if ((q >> 36) == 0 && (q >> 25) != 0) {
                const uint32_t mu52 = (uint32_t)(qinv64 >> 12);
                const uint32_t Qp = (uint32_t)(((u64)(uint32_t)(x >> 20) * mu52) >> 32);
                x -= (u64)Qp * q;
            } else {
                x -= __umul64hi(x, qinv64) * q;
            }  // [0, 2q)
        } else {
            x = x >= q2 ? x - q2 : x;
        }
        return x >= q ? x - q : x;
    };
    const int tid = threadIdx.x;
    const int line = kCol ? tid % lines : tid / tpl;
    const int j = kCol ? tid / lines : tid % tpl;
    const int tw_line = kCol ? 1 : (N1 + l0 + line);
    // rounds: exponent chunks of kLE from the top, remainder at the bottom
    const int nr = (logn + kLE - 1) / kLE;
#pragma unroll
    for (int rr = 0; rr < nr; rr++) {
        const int k = kInv ? nr - 1 - rr : rr;  // chunk index from the top
        const int hi = logn - 1 - kLE * k;      // largest exponent of the chunk
        const int lo = max(0, hi - (kLE - 1));
        const int nst = hi - lo + 1;
        const bool from_global = !kStaged && rr == 0, to_global = !kStaged && rr == nr - 1;
        // a row-pass round of unit stride holds consecutive elements: 16-byte global accesses
        const bool vec = !kCol && lo == 0 && E == kEE;
        if (tid < nthr) {
            u64 v[kEE];
            // thread j of the line: block (j >> lo), offset (j & (s - 1)), block size kEE s
            int blk = j >> lo;
            int base = (blk << (lo + kLE)) + (j & ((1 << lo) - 1));
            if (E < kEE) base = blk = 0;
            if (from_global && vec) {
#pragma unroll
                for (int r = 0; r < kEE; r += 2) {
                    const ulonglong2 p = *reinterpret_cast<const ulonglong2*>(s + GOFF(line, base + r));
                    v[r] = p.x;
                    v[r + 1] = p.y;
                }
            } else {
#pragma unroll
                for (int r = 0; r < kEE; r++) {
                    const int x = base + (r << lo);
                    v[r] = (r < E) ? (from_global ? s[GOFF(line, x)] : (kCol ? tile[CIDX(x, line)] : tile[RIDX(line, x)]))
                                   : 0;
                }
            }
            // the inverse's last round applies N^-1 in its last stage
            const bool fold = kInv && kCol && to_global;
            round_stages<kInv, kNoRed, kLE, kQ36, !kCol>(v, blk, lo, nst, E, logn, tw_line, tw, q, fold,
                                                  make_ulonglong2(ni, nis),
                                                  make_ulonglong2(a.ninvw[mi], a.ninvw_sh[mi]));
            // each thread writes back exactly the positions it read: no barrier in between
            if (to_global && vec) {
#pragma unroll
                for (int r = 0; r < kEE; r += 2)
                    *reinterpret_cast<ulonglong2*>(d + GOFF(line, base + r)) =
                        make_ulonglong2(fin(v[r], fold), fin(v[r + 1], fold));
            } else {
#pragma unroll
                for (int r = 0; r < kEE; r++) {
                    if (r >= E) break;
                    const int x = base + (r << lo);
                    if (to_global) d[GOFF(line, x)] = fin(v[r], fold);
                    else if (kCol) tile[CIDX(x, line)] = v[r];
                    else tile[RIDX(line, x)] = v[r];
                }
            }
        }
        if (!to_global) __syncthreads();
    }
    if (kStaged) {
        const int pairs = total >> 1;
#pragma unroll 4
        for (int e = threadIdx.x; e < pairs; e += nthreads) {
            const int el = 2 * e;
            ulonglong2 o;
            if (kCol) {
                const int x = el / lines, c = el - x * lines;
                const int x1 = (el + 1) / lines, c1 = el + 1 - x1 * lines;
                o.x = fin(tile[CIDX(x, c)], false);
                o.y = fin(tile[CIDX(x1, c1)], false);
                *reinterpret_cast<ulonglong2*>(d + (size_t)x * N2 + l0 + c) = o;
            } else {
                const int ln = el >> logN2, x = el & (N2 - 1);
                o.x = fin(tile[RIDX(ln, x)], false);
                o.y = fin(tile[RIDX(ln, x + 1)], false);
                *reinterpret_cast<ulonglong2*>(d + (size_t)l0 * N2 + el) = o;
            }
        }
    }
#undef GOFF
#undef RIDX
#undef CIDX
}

// Integer-pipe roof of the forward transform's arithmetic.  Every thread keeps 8
// residues in registers and runs `iters` groups of five radix-8 rounds (15 stages,
// 60 butterflies, the same lazy Shoup butterflies as the transform, twiddles 1..7
// of modulus 0, which stay in L1) followed by the reduction the transform applies
// once per element; no tile traffic.  One word per thread is written so that the
// work is kept.  Butterflies executed = blocks * 256 * iters * 60.
template <bool kQ36>
__global__ void __launch_bounds__(256) k_butterfly_probe(const ulonglong2* __restrict__ tw, u64 q, u64 qinv64,
                                                         int iters, u64* out) {
    u64 v[kE];
    const u64 seed = blockIdx.x * 256 + threadIdx.x;
#pragma unroll
    for (int r = 0; r < kE; r++) v[r] = (seed * 8 + r) % q;
#pragma unroll 1
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int k = 0; k < 5; k++) round_stages<false, true, 3, kQ36>(v, 0, 0, 3, kE, 3, 1, tw, q);
#pragma unroll
        for (int r = 0; r < kE; r++) v[r] -= __umul64hi(v[r], qinv64) * q;
    }
    u64 acc = 0;
#pragma unroll
    for (int r = 0; r < kE; r++) acc ^= v[r];
    out[(size_t)blockIdx.x * 256 + threadIdx.x] = acc;
}

// Single-pass transform of N = 2^16 = 256 x 256 on a cluster of 8 CTAs, one limb
// per cluster, so that a limb crosses DRAM once each way instead of twice.
// CTA c first owns the column block c (columns 32c .. 32c+31 of all 256 rows),
// runs the column stages on it, then exchanges data with the other seven CTAs
// through distributed shared memory so that it owns the row block c (rows 32c ..
// 32c+31, all columns), and runs the row stages there (the inverse runs the row
// stages first).  The CTA's shared memory is 8 slots of 32 x 32 elements, row
// stride 33, slot stride 1060 words:
//   column-block view: slot s, entry (a, b) = element (row 32 s + a, column 32 c + b)
//   row-block view:    slot s, entry (a, b) = element (row 32 c + a, column 32 s + b)
// so the exchange swaps CTA c's slot k with CTA k's slot c entry by entry (the
// diagonal slot stays), with no permutation inside a slot: each entry is moved
// by exactly one thread of the cluster, CTA min(c, k) taking the first half of
// the pair's entries and CTA max(c, k) the second.  The row stride (1 mod 16
// words) and the slot stride (4 mod 16) keep every round's 32 lanes at two
// accesses per bank pair, the minimum for 8-byte words: column rounds put the
// lanes on the 32 columns; row rounds of distance >= 4 put them on one row's 32
// groups, and the unit-distance round on 8 rows x 4 groups.  Rounds, butterflies,
// twiddles and the final reduction are those of ntt_pass; the first round reads
// global memory and the last one writes it, as in its direct form.
constexpr int kClB = 32, kClR = 33, kClSW = 1060;
constexpr size_t kClSmem = (size_t)8 * kClSW * sizeof(u64);

// kT threads per CTA, kMinB CTAs per SM (three fit by shared memory).  Measured on
// B300 (N = 2^16, 532 limbs, forward / inverse us per limb): 256 threads x 3 CTAs
// (80 registers) 0.90 / 1.06; 384 x 3 (56 registers, spills) 0.96 / 1.06;
// 512 x 2 (64 registers, spills) 1.03 / 1.10; the two-pass form 0.76 / 0.84.
constexpr int kClT = 256;
template <bool kInv, bool kNoRed, bool kQ36, int kT, int kMinB>
__global__ void __launch_bounds__(kT, kMinB) ntt_cluster16(NttArgs a) {
    constexpr int kClThreads = kT;
    namespace cg = cooperative_groups;
    constexpr int logn = 8, n = 256, N1 = 256;
    constexpr int kGroups = (n / 8) * kClB;  // groups of 8 elements per round and CTA
    extern __shared__ __align__(16) u64 sm[];
    cg::cluster_group cluster = cg::this_cluster();
    uint32_t cid, c;
    asm("mov.u32 %0, %%clusterid.x;" : "=r"(cid));
    asm("mov.u32 %0, %%cluster_ctarank;" : "=r"(c));
    const int limb = (int)cid;
    const int poly = limb / a.per_poly, jl = limb % a.per_poly;
    const int mi = a.mod_map[jl];
    const int pos = a.pos_map ? a.pos_map[jl] : jl;
    const u64 q = a.mods[mi].q;
    const ulonglong2* tw = a.tw + ((size_t)mi << 16);
    u64* d = a.dst + (size_t)poly * a.poly_stride + ((size_t)pos << 16);
    const u64* s = a.src + (size_t)poly * a.src_stride + ((size_t)pos << 16);
    const int tid = threadIdx.x, cB = (int)c * kClB;
    const u64 q2 = 2 * q;
    const u64 ni = a.ninv[mi], nis = a.ninv_sh[mi];
    const u64 qinv64 = a.mods[mi].ratio_hi;
    auto fin = [&](u64 x) -> u64 {
        if (kInv) x = kQ36 ? shoup36(x, ni, nis, 0 - q) : shoup_lazy(x, ni, nis, q);  // [0, 2q)
        else if (kNoRed) x -= __umul64hi(x, qinv64) * q;                              // [0, 2q)
        else x = x >= q2 ? x - q2 : x;
        return x >= q ? x - q : x;
    };
    // column stages on the column block: line = column j (lanes), element x = row
    auto col_round = [&](int rr, bool from_global, bool to_global) {
        const int k = kInv ? 2 - rr : rr;
        const int hi = logn - 1 - 3 * k, lo = max(0, hi - 2), nst = hi - lo + 1;
#pragma unroll 1
        for (int gi = tid; gi < kGroups; gi += kClThreads) {
            const int j = gi & 31, jj = gi >> 5;
            const int blk = jj >> lo, base = (blk << (lo + 3)) + (jj & ((1 << lo) - 1));
            u64 v[8];
#pragma unroll
            for (int r = 0; r < 8; r++) {
                const int x = base + (r << lo);
                v[r] = from_global ? s[(size_t)x * n + cB + j] : sm[kClSW * (x >> 5) + (x & 31) * kClR + j];
            }
            round_stages<kInv, kNoRed, 3, kQ36>(v, blk, lo, nst, 8, logn, 1, tw, q);
#pragma unroll
            for (int r = 0; r < 8; r++) {
                const int x = base + (r << lo);
                if (to_global) d[(size_t)x * n + cB + j] = fin(v[r]);
                else sm[kClSW * (x >> 5) + (x & 31) * kClR + j] = v[r];
            }
        }
    };
    // row stages on the row block: line = local row xl, element x = column
    auto row_round = [&](int rr, bool from_global, bool to_global) {
        const int k = kInv ? 2 - rr : rr;
        const int hi = logn - 1 - 3 * k, lo = max(0, hi - 2), nst = hi - lo + 1;
#pragma unroll 1
        for (int gi = tid; gi < kGroups; gi += kClThreads) {
            const int lane = gi & 31, w = gi >> 5;
            // unit distance: lanes on 8 rows x 4 groups; otherwise on one row's 32 groups
            const int xl = lo == 0 ? (lane >> 2) + 8 * (w >> 3) : w;
            const int jj = lo == 0 ? 4 * (w & 7) + (lane & 3) : lane;
            const int blk = jj >> lo, base = (blk << (lo + 3)) + (jj & ((1 << lo) - 1));
            const size_t grow = (size_t)(cB + xl) * n;
            u64 v[8];
            if (from_global && lo == 0) {
#pragma unroll
                for (int r = 0; r < 8; r += 2) {
                    const ulonglong2 p = *reinterpret_cast<const ulonglong2*>(s + grow + base + r);
                    v[r] = p.x;
                    v[r + 1] = p.y;
                }
            } else {
#pragma unroll
                for (int r = 0; r < 8; r++) {
                    const int x = base + (r << lo);
                    v[r] = from_global ? s[grow + x] : sm[kClSW * (x >> 5) + xl * kClR + (x & 31)];
                }
            }
            round_stages<kInv, kNoRed, 3, kQ36>(v, blk, lo, nst, 8, logn, N1 + cB + xl, tw, q);
            if (to_global && lo == 0) {
#pragma unroll
                for (int r = 0; r < 8; r += 2)
                    *reinterpret_cast<ulonglong2*>(d + grow + base + r) = make_ulonglong2(fin(v[r]), fin(v[r + 1]));
            } else {
#pragma unroll
                for (int r = 0; r < 8; r++) {
                    const int x = base + (r << lo);
                    if (to_global) d[grow + x] = fin(v[r]);
                    else sm[kClSW * (x >> 5) + xl * kClR + (x & 31)] = v[r];
                }
            }
        }
    };
    // exchange: CTA c's slot k <-> CTA k's slot c, 16 bytes per access; of each
    // pair's 32 x 33 entries the lower rank moves the first half, the higher the second
    auto exchange = [&]() {
        constexpr int kHalf = kClB * kClR / 2;  // 528 entries
        constexpr int kVec = kHalf / 2;         // 264 16-byte pairs per half
#pragma unroll 2
        for (int idx = tid; idx < 7 * kVec; idx += kClThreads) {
            const int kk = ((int)c + 1 + idx / kVec) & 7;
            const int p = 2 * (idx % kVec) + ((int)c < kk ? 0 : kHalf);
            ulonglong2* mine = reinterpret_cast<ulonglong2*>(sm + kClSW * kk + p);
            ulonglong2* theirs = reinterpret_cast<ulonglong2*>(cluster.map_shared_rank(sm + kClSW * c + p, kk));
            const ulonglong2 x = *mine, y = *theirs;
            *mine = y;
            *theirs = x;
        }
    };
    if (!kInv) {
        col_round(0, true, false);
        __syncthreads();
        col_round(1, false, false);
        __syncthreads();
        col_round(2, false, false);
        cluster.sync();  // every column block complete and visible to the cluster
        exchange();
        cluster.sync();  // every row block assembled; no remote access after this
        row_round(0, false, false);
        __syncthreads();
        row_round(1, false, false);
        __syncthreads();
        row_round(2, false, true);
    } else {
        row_round(0, true, false);
        __syncthreads();
        row_round(1, false, false);
        __syncthreads();
        row_round(2, false, false);
        cluster.sync();
        exchange();
        cluster.sync();
        col_round(0, false, false);
        __syncthreads();
        col_round(1, false, false);
        __syncthreads();
        col_round(2, false, true);
    }
}

NttArgs make_args(fe_ctx* c, const LimbSet& s, const u64* src, size_t src_stride, bool inverse) {
    NttArgs a;
    a.src = src ? src : s.base;
    a.src_stride = src ? src_stride : s.poly_stride;
    a.dst = s.base;
    a.poly_stride = s.poly_stride;
    a.per_poly = s.per_poly;
    a.mod_map = s.mod_map;
    a.pos_map = s.pos_map;
    a.mods = c->d_mod;
    a.tw = (const ulonglong2*)(inverse ? c->d_itw2 : c->d_tw2);
    a.ninv = c->d_ninv;
    a.ninv_sh = c->d_ninv_sh;
    a.ninvw = c->d_ninvw;
    a.ninvw_sh = c->d_ninvw_sh;
    a.logN = c->logN;
    a.logN2 = c->logN / 2;
    return a;
}

int threads_for(int lines, int n, int E) { return std::max(32, lines * (n / std::min(E, n))); }

template <int kLogN, bool kInv, bool kCol, int kLE = 3, bool kStaged = false>
void launch_one(bool nored, bool q36, dim3 g, int t, size_t sm, cudaStream_t st, const NttArgs& a, int first) {
    if (q36) {
        if (nored && !kInv)
            ntt_pass<kLogN, kInv, kCol, true, kLE, true, kStaged><<<g, t, sm, st>>>(a, first);
        else
            ntt_pass<kLogN, kInv, kCol, false, kLE, true, kStaged><<<g, t, sm, st>>>(a, first);
    } else if (nored && !kInv) {
        ntt_pass<kLogN, kInv, kCol, true, kLE, false, kStaged><<<g, t, sm, st>>>(a, first);
    } else {
        ntt_pass<kLogN, kInv, kCol, false, kLE, false, kStaged><<<g, t, sm, st>>>(a, first);
    }
}

// compile-time ring degrees for the production sizes, run-time geometry otherwise
// radix 16 (le = 4) and radix 4 (le = 2), and the staged form, are compiled for the
// production ring degrees 2^14 and 2^16
template <bool kInv, bool kCol>
void launch_pass(int logN, bool nored, bool q36, dim3 g, int t, size_t sm, cudaStream_t st, const NttArgs& a,
                 int first, int le, bool staged) {
    if (staged && le == 3 && logN == 16) return launch_one<16, kInv, kCol, 3, true>(nored, q36, g, t, sm, st, a, first);
    if (staged && le == 3 && logN == 14) return launch_one<14, kInv, kCol, 3, true>(nored, q36, g, t, sm, st, a, first);
    if (le == 4 && logN == 16) return launch_one<16, kInv, kCol, 4>(nored, q36, g, t, sm, st, a, first);
    if (le == 4 && logN == 14) return launch_one<14, kInv, kCol, 4>(nored, q36, g, t, sm, st, a, first);
    if (le == 2 && logN == 16) return launch_one<16, kInv, kCol, 2>(nored, q36, g, t, sm, st, a, first);
    if (le == 2 && logN == 14) return launch_one<14, kInv, kCol, 2>(nored, q36, g, t, sm, st, a, first);
    switch (logN) {
        case 10: launch_one<10, kInv, kCol>(nored, q36, g, t, sm, st, a, first); break;
        case 11: launch_one<11, kInv, kCol>(nored, q36, g, t, sm, st, a, first); break;
        case 12: launch_one<12, kInv, kCol>(nored, q36, g, t, sm, st, a, first); break;
        case 13: launch_one<13, kInv, kCol>(nored, q36, g, t, sm, st, a, first); break;
        case 14: launch_one<14, kInv, kCol>(nored, q36, g, t, sm, st, a, first); break;
        case 15: launch_one<15, kInv, kCol>(nored, q36, g, t, sm, st, a, first); break;
        case 16: launch_one<16, kInv, kCol>(nored, q36, g, t, sm, st, a, first); break;
        case 17: launch_one<17, kInv, kCol>(nored, q36, g, t, sm, st, a, first); break;
        default: launch_one<0, kInv, kCol>(nored, q36, g, t, sm, st, a, first); break;
    }
}

template <bool kInv, bool kNoRed, bool kQ36, int kT, int kMinB>
cudaError_t launch_cluster(int limbs, cudaStream_t st, const NttArgs& a) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(8 * limbs);
    cfg.blockDim = dim3(kT);
    cfg.dynamicSmemBytes = kClSmem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 8;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, ntt_cluster16<kInv, kNoRed, kQ36, kT, kMinB>, a);
}

// Whether the cluster form can run here: its shared-memory size is accepted and at
// least one cluster of 8 CTAs fits on the device.  Decided once per context.
template <bool kInv, bool kNoRed, bool kQ36, int kT, int kMinB>
bool cluster_fits() {
    auto kern = ntt_cluster16<kInv, kNoRed, kQ36, kT, kMinB>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kClSmem) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(8);
    cfg.blockDim = dim3(kT);
    cfg.dynamicSmemBytes = kClSmem;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 8;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return n > 0;
}

template <int kT, int kMinB>
bool fits_all() {
    return cluster_fits<false, true, false, kT, kMinB>() && cluster_fits<false, false, false, kT, kMinB>() &&
           cluster_fits<true, false, false, kT, kMinB>() && cluster_fits<true, false, true, kT, kMinB>();
}

bool cluster_usable(fe_ctx* c) {
    if (c->ntt_cluster_ok < 0) {
        // every instance the context can launch must fit (their shared memory is identical)
        const bool ok = fits_all<kClT, 3>();
        c->ntt_cluster_ok = ok ? 1 : 0;
    }
    return c->ntt_cluster_ok == 1;
}

template <bool kInv>
void run_ntt(fe_ctx* c, const LimbSet& s, const u64* src, size_t src_stride, cudaStream_t st) {
    int limbs = s.per_poly * s.n_poly;
    if (limbs == 0) return;
    NttArgs a = make_args(c, s, src, src_stride, kInv);
    if (c->ntt_path == 2 && c->logN == 16 && cluster_usable(c)) {
        // single pass on clusters of 8 CTAs, one limb per cluster
        const bool nored = !kInv && c->max_mod_bits <= 58;
        const bool q36 = kInv && c->max_mod_bits <= 36 && c->ntt_q36;
        ProfScope ps(c, PK_NTT, st, 16.0 * limbs * c->N);
        if (q36) launch_cluster<kInv, false, true, kClT, 3>(limbs, st, a);
        else if (nored) launch_cluster<false, true, false, kClT, 3>(limbs, st, a);
        else launch_cluster<kInv, false, false, kClT, 3>(limbs, st, a);
        c->cnt.ntt += limbs;
        c->cnt.launches += 1;
        return;
    }
    const int N = c->N, N2 = 1 << a.logN2, N1 = N / N2;
    const int C = std::min(kTile / N1, N2), R = std::min(kTile / N2, N1);
    const size_t smc = (size_t)(N1 + (N1 >> 3) + 1) * C * 8, smr = (size_t)R * (N2 + (N2 >> 3)) * 8;
    // algorithmic bytes of a limb transform, 2 N w, split over its two passes
    const double bytes = 8.0 * limbs * N;
    const bool big = c->logN == 14 || c->logN == 16;
    const int le = big && c->ntt_radix == 16 ? 4 : (big && c->ntt_radix == 4 ? 2 : 3);
    const int tc = threads_for(C, N1, 1 << le), tr = threads_for(R, N2, 1 << le);
    // forward: no reduction inside the transform when every modulus is below 2^58, unless
    // fe_ctx_set_ntt_forward asks for Harvey's reduction to [0, 4q) at every stage (an ALU
    // compare per butterfly in place of a 64-bit Barrett step per element at the end)
    const bool nored = c->max_mod_bits <= 58 && !(c->ntt_fwd & 1);
    // every modulus below 2^36: the 36-bit Shoup product in the inverse passes (inputs below
    // 4 q, within its 2^42 bound).  Measured on B300 (N = 2^16, 532 limbs): inverse 0.932 ->
    // 0.908 us per limb; the forward passes were 1.6 % slower with it and keep the general form.
    const bool q36 = c->max_mod_bits <= 36 && (kInv ? c->ntt_q36 != 0 : (c->ntt_fwd & 2) != 0);
    const dim3 gc(limbs * (N2 / C)), gr(limbs * (N1 / R));
    if (!kInv) {
        {
            ProfScope ps(c, PK_NTT, st, bytes);
            launch_pass<false, true>(c->logN, nored, q36, gc, tc, smc, st, a, 1, le, c->ntt_path == 1);
        }
        {
            ProfScope ps(c, PK_NTT, st, bytes);
            launch_pass<false, false>(c->logN, nored, q36, gr, tr, smr, st, a, 0, le, c->ntt_path == 1);
        }
    } else {
        {
            ProfScope ps(c, PK_NTT, st, bytes);
            launch_pass<true, false>(c->logN, false, q36, gr, tr, smr, st, a, 1, le, c->ntt_path == 1);
        }
        {
            ProfScope ps(c, PK_NTT, st, bytes);
            launch_pass<true, true>(c->logN, false, q36, gc, tc, smc, st, a, 0, le, c->ntt_path == 1);
        }
    }
    c->cnt.ntt += limbs;
    c->cnt.launches += 2;
}

}  // namespace

int butterfly_probe(fe_ctx* c, uint32_t* blocks, uint32_t iters, u64* out, cudaStream_t st) {
    const Modulus m = make_modulus(c->mod[0]);
    if (*blocks == 0) {  // one full wave: every SM holds as many CTAs as fit
        int per_sm = 0;
        FE_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_butterfly_probe<false>, 256, 0));
        *blocks = (uint32_t)(std::min(per_sm, 8) * c->n_sm);
    }
    // the forward transform's butterfly (the general form; fe_ctx_set_ntt_q36(ctx, 2) probes
    // the 36-bit form the inverse passes use)
    if (c->max_mod_bits <= 36 && c->ntt_q36 == 2)
        k_butterfly_probe<true><<<*blocks, 256, 0, st>>>((const ulonglong2*)c->d_tw2, m.q, m.ratio_hi, (int)iters, out);
    else
        k_butterfly_probe<false><<<*blocks, 256, 0, st>>>((const ulonglong2*)c->d_tw2, m.q, m.ratio_hi, (int)iters, out);
    c->cnt.launches += 1;
    return cudaGetLastError() == cudaSuccess ? FE_OK : fail(FE_ECUDA, "butterfly probe launch");
}

void ntt_prepare(fe_ctx* c) {
    if (c->logN == 16) cluster_usable(c);
}

void ntt_forward(fe_ctx* c, const LimbSet& s, cudaStream_t st) { run_ntt<false>(c, s, nullptr, 0, st); }
void ntt_inverse(fe_ctx* c, const LimbSet& s, cudaStream_t st) { run_ntt<true>(c, s, nullptr, 0, st); }
void ntt_forward_from(fe_ctx* c, const u64* src, size_t src_stride, const LimbSet& dst, cudaStream_t st) {
    run_ntt<false>(c, dst, src, src_stride, st);
}
void ntt_inverse_from(fe_ctx* c, const u64* src, size_t src_stride, const LimbSet& dst, cudaStream_t st) {
    run_ntt<true>(c, dst, src, src_stride, st);
}

}  // namespace fe

extern "C" int fe_ctx_set_ntt_forward(fe_ctx* c, int flags) {
    if (!c) return fe::fail(FE_EINVAL, "null argument");
    if (flags < 0 || flags > 3) return fe::fail(FE_EINVAL, "forward NTT flags must be in [0, 3]");
    c->ntt_fwd = flags;
    return FE_OK;
}

extern "C" int fe_ctx_set_ntt_q36(fe_ctx* c, int enable) {
    if (!c) return fe::fail(FE_EINVAL, "null argument");
    if (enable < 0 || enable > 2) return fe::fail(FE_EINVAL, "enable must be 0, 1 or 2");
    c->ntt_q36 = enable;
    return FE_OK;
}

extern "C" int fe_ctx_set_ntt_path(fe_ctx* c, int path) {
    if (!c) return fe::fail(FE_EINVAL, "null argument");
    if (path < 0 || path > 2) return fe::fail(FE_EINVAL, "NTT path must be 0, 1 or 2");
    c->ntt_path = path;
    return FE_OK;
}

extern "C" int fe_ctx_set_ntt_radix(fe_ctx* c, int radix) {
    if (!c) return fe::fail(FE_EINVAL, "null argument");
    if (radix != 4 && radix != 8 && radix != 16) return fe::fail(FE_EINVAL, "NTT radix must be 4, 8 or 16");
    c->ntt_radix = radix;
    return FE_OK;
}
