// Element-wise and key-switching kernels.
//
// All kernels stream limb-major data with one thread per coefficient and
// coalesced 8-byte accesses; products of two residues are accumulated in
// 128 bits and reduced once (Barrett, 2^128 / q) per output word.  The MAC,
// with every modulus below 2^40, keeps its sums in three 32-bit words instead
// (Acc40): sixteen independent sums per thread hide the carry chain's latency,
// which the one to four sums of base conversion and the key inner product do
// not (there the split form measured 7 % and 1.5 % slower).
#include <algorithm>
#include <type_traits>

#include "kernels.cuh"

namespace fe {

namespace {
constexpr int kB = 256;

inline dim3 grid_for(int N, int y, int z = 1) { return dim3((N + kB - 1) / kB, y, z); }

// ------------------------------------------------------------------------
// Base conversion with centred digits (see BConvTab).
// One thread per (coefficient, polynomial).
// ------------------------------------------------------------------------
// kS = number of source moduli (compile time, so that the digits stay in registers)
template <int kS, bool kNarrow>
__global__ void k_bconv(BConvTab t, const Modulus* mods, int L, int level, int logN,
                        const u64* in, size_t in_stride, int in_pos_base, u64* out,
                        size_t out_stride, int copy_src) {
    const int N = 1 << logN;
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const u64* ip = in + blockIdx.y * in_stride;
    u64* op = out + blockIdx.y * out_stride;
    u64 y[kS];
    int neg = 0;
#pragma unroll
    for (int i = 0; i < kS; i++) {
        int mi = t.src[i];
        u64 b = mods[mi].q;
        u64 x = ip[((size_t)(ext_pos(mi, L, level) - in_pos_base) << logN) + n];
        if (copy_src) op[((size_t)ext_pos(mi, L, level) << logN) + n] = x;
        u64 v = mul_shoup(x, t.inv[i], t.inv_sh[i], b);
        y[i] = v;
        neg += v > (b >> 1);
    }
    for (int d = 0; d < t.n_dst; d++) {
        int mt = t.dst[d];
        u128 acc = (u128)t.negB[d] * (u64)neg;
        const u64* row = t.mat + d * kS;
#pragma unroll
        for (int i = 0; i < kS; i++) acc += (u128)y[i] * row[i];
        op[((size_t)ext_pos(mt, L, level) << logN) + n] = kNarrow ? reduce_narrow(acc, mods[mt]) : reduce128(acc, mods[mt]);
    }
}

// Two coefficients per thread (n, n + 1) with 16-byte accesses: the table
// words are read once for both, and with every modulus below 2^40 each
// destination keeps two independent three-word sums (Acc40).  Needs 16-byte
// aligned bases and even strides (checked by the launcher).
template <int kS, bool kNarrow, bool kM36>
__global__ void k_bconv2(BConvTab t, const Modulus* mods, int L, int level, int logN,
                         const u64* in, size_t in_stride, int in_pos_base, u64* out,
                         size_t out_stride, int copy_src) {
    const int N = 1 << logN;
    const int n = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    if (n >= N) return;
    const u64* ip = in + blockIdx.y * in_stride;
    u64* op = out + blockIdx.y * out_stride;
    u64 y0[kS], y1[kS];
    int neg0 = 0, neg1 = 0;
#pragma unroll
    for (int i = 0; i < kS; i++) {
        const int mi = t.src[i];
        const u64 b = mods[mi].q;
        const ulonglong2 x =
            *reinterpret_cast<const ulonglong2*>(ip + ((size_t)(ext_pos(mi, L, level) - in_pos_base) << logN) + n);
        if (copy_src) *reinterpret_cast<ulonglong2*>(op + ((size_t)ext_pos(mi, L, level) << logN) + n) = x;
        y0[i] = mul_shoup(x.x, t.inv[i], t.inv_sh[i], b);
        y1[i] = mul_shoup(x.y, t.inv[i], t.inv_sh[i], b);
        neg0 += y0[i] > (b >> 1);
        neg1 += y1[i] > (b >> 1);
    }
    for (int d = 0; d < t.n_dst; d++) {
        const int mt = t.dst[d];
        const u64* row = t.mat + d * kS;
        const u64 nb = t.negB[d];
        ulonglong2 r;
        if constexpr (kM36) {  // every modulus below 2^36; at most 9 terms
            Acc36 a0, a1;
            acc36_zero(a0);
            acc36_zero(a1);
            const uint32_t nl = split24_lo(nb), nh = split24_hi(nb);
            acc36_mad(a0, (u64)neg0, nl, nh);
            acc36_mad(a1, (u64)neg1, nl, nh);
#pragma unroll
            for (int i = 0; i < kS; i++) {
                const u64 w = row[i];
                const uint32_t wl = split24_lo(w), wh = split24_hi(w);
                acc36_mad(a0, y0[i], wl, wh);
                acc36_mad(a1, y1[i], wl, wh);
            }
            r.x = reduce_narrow(acc36_value(a0), mods[mt]);
            r.y = reduce_narrow(acc36_value(a1), mods[mt]);
        } else if constexpr (kNarrow) {
            Acc40 a0, a1;
            acc40_zero(a0);
            acc40_zero(a1);
            acc40_mad(a0, nb, (u64)neg0);
            acc40_mad(a1, nb, (u64)neg1);
#pragma unroll
            for (int i = 0; i < kS; i++) {
                const u64 w = row[i];
                acc40_mad(a0, y0[i], w);
                acc40_mad(a1, y1[i], w);
            }
            r.x = reduce_narrow(acc40_value(a0), mods[mt]);
            r.y = reduce_narrow(acc40_value(a1), mods[mt]);
        } else {
            u128 a0 = (u128)nb * (u64)neg0, a1 = (u128)nb * (u64)neg1;
#pragma unroll
            for (int i = 0; i < kS; i++) {
                const u64 w = row[i];
                a0 += (u128)y0[i] * w;
                a1 += (u128)y1[i] * w;
            }
            r.x = reduce128(a0, mods[mt]);
            r.y = reduce128(a1, mods[mt]);
        }
        *reinterpret_cast<ulonglong2*>(op + ((size_t)ext_pos(mt, L, level) << logN) + n) = r;
    }
}

// ------------------------------------------------------------------------
// Evaluation-key inner product:
//   acc_b[p][n] = sum_j ext_j[p][n] * key_j.b[kl(p)][n],  acc_a likewise,
// over the positions p of Q_level * P.  blockIdx.y = position, z = item.
// ------------------------------------------------------------------------
__global__ void k_keyip(const KsItem* items, const Modulus* mods, int L, int level, int k,
                        int logN, int n_mod, int narrow) {
    const int N = 1 << logN;
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const KsItem it = items[blockIdx.z];
    const int p = blockIdx.y;
    const int np = level + 1 + k;
    const int mi = p <= level ? p : L + 1 + (p - level - 1);
    const int dnum = (level + 1 + k - 1) / k;
    const Modulus m = mods[mi];
    u128 ab = 0, aa = 0;
    for (int j = 0; j < dnum; j++) {
        u64 e = it.ext[((size_t)(j * np + p) << logN) + n];
        const u64* kb = it.key + ((size_t)(j * 2 * n_mod + mi) << logN);
        const u64* ka = kb + ((size_t)n_mod << logN);
        ab += (u128)e * kb[n];
        aa += (u128)e * ka[n];
    }
    it.acc[((size_t)p << logN) + n] = narrow ? reduce_narrow(ab, m) : reduce128(ab, m);
    it.acc[((size_t)(np + p) << logN) + n] = narrow ? reduce_narrow(aa, m) : reduce128(aa, m);
}

// key-stationary form: blockIdx.x = group of items that share one key; kD =
// number of digits (compile time, so that the key words stay in registers).
// Each thread handles two consecutive coefficients with 16-byte accesses.  The
// digits of the next item are fetched into shared memory by cp.async while
// the current item is computed (double buffer); every thread copies and reads
// only its own slots, so waiting on its own copies is enough (no barrier).
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(smem_dst)),
                 "l"(gmem_src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int kPending>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(kPending) : "memory");
}

template <int kD, bool kNarrow>
__global__ void __launch_bounds__(256, 2) k_keyip_grouped(const KsGroup* groups, const KsItem* items,
                                                          const Modulus* mods, int L, int level, int k,
                                                          int logN, int n_mod) {
    extern __shared__ ulonglong2 ext_sm[];  // [2 buffers][kD][blockDim.x]
    const int N = 1 << logN;
    // blockIdx.x = group (fastest), so that the CTAs of all keys of one
    // (coefficient tile, limb) run together and the digits they share hit L2
    const int n = 2 * (blockIdx.y * blockDim.x + threadIdx.x);
    if (n >= N) return;
    const KsGroup gr = groups[blockIdx.x];
    const int p = blockIdx.z;
    const int np = level + 1 + k;
    const int mi = p <= level ? p : L + 1 + (p - level - 1);
    const Modulus m = mods[mi];
    const int tid = threadIdx.x, nt = blockDim.x;
    // the item pointers are loaded one item ahead of their use (item t + 2's
    // digits while item t is computed), so their global loads stay off the
    // path between two items
    const KsItem* its = items + gr.item0;
    auto fetch = [&](const u64* ext, int buf) {
#pragma unroll
        for (int j = 0; j < kD; j++)
            cp_async16(&ext_sm[(buf * kD + j) * nt + tid], ext + ((size_t)(j * np + p) << logN) + n);
        cp_async_commit();
    };
    fetch(its[0].ext, 0);
    const u64* ext_next = gr.n_items > 1 ? its[1].ext : nullptr;
    ulonglong2 kb[kD], ka[kD];
#pragma unroll
    for (int j = 0; j < kD; j++) {
        const u64* b = gr.key + ((size_t)(j * 2 * n_mod + mi) << logN);
        kb[j] = *reinterpret_cast<const ulonglong2*>(b + n);
        ka[j] = *reinterpret_cast<const ulonglong2*>(b + ((size_t)n_mod << logN) + n);
    }
    const size_t ob = ((size_t)p << logN) + n, oa = ((size_t)(np + p) << logN) + n;
    for (int t = 0; t < gr.n_items; t++) {
        const int buf = t & 1;
        u64* acc = its[t].acc;
        if (t + 1 < gr.n_items) {
            fetch(ext_next, buf ^ 1);
            ext_next = t + 2 < gr.n_items ? its[t + 2].ext : nullptr;
            cp_async_wait<1>();  // item t's copies are complete, item t + 1's may be in flight
        } else {
            cp_async_wait<0>();
        }
        u128 bx = 0, by = 0, ax = 0, ay = 0;
#pragma unroll
        for (int j = 0; j < kD; j++) {
            const ulonglong2 e = ext_sm[(buf * kD + j) * nt + tid];
            bx += (u128)e.x * kb[j].x;
            by += (u128)e.y * kb[j].y;
            ax += (u128)e.x * ka[j].x;
            ay += (u128)e.y * ka[j].y;
        }
        if (kNarrow) {
            *reinterpret_cast<ulonglong2*>(acc + ob) = make_ulonglong2(reduce_narrow(bx, m), reduce_narrow(by, m));
            *reinterpret_cast<ulonglong2*>(acc + oa) = make_ulonglong2(reduce_narrow(ax, m), reduce_narrow(ay, m));
        } else {
            *reinterpret_cast<ulonglong2*>(acc + ob) = make_ulonglong2(reduce128(bx, m), reduce128(by, m));
            *reinterpret_cast<ulonglong2*>(acc + oa) = make_ulonglong2(reduce128(ax, m), reduce128(ay, m));
        }
    }
}

// ------------------------------------------------------------------------
// ModDown combine + automorphism + optional add / accumulate (see CombineItem).
// blockIdx.y = limb i of Q_level, z = item.
// ------------------------------------------------------------------------
// Two coefficients per thread (n even, n + 1), 16-byte accesses: the
// automorphism maps the pair onto a pair (see k_lift).
__global__ void k_combine(const CombineItem* items, const Modulus* mods, const u64* pinv,
                          const u64* pinv_sh, int level, int k, int logN) {
    const int N = 1 << logN;
    const int n = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    if (n >= N) return;
    const CombineItem it = items[blockIdx.z];
    const int i = blockIdx.y;
    const int np = level + 1 + k, nq = level + 1;
    const u64 q = mods[i].q;
    const uint32_t src = it.galois == 1 ? (uint32_t)n : galois_perm(n, it.galois, logN);
    const size_t so = ((size_t)i << logN) + (src & ~1u);
    const bool swap = src & 1u;
    auto load2 = [&](const u64* p) -> ulonglong2 {
        ulonglong2 v = *reinterpret_cast<const ulonglong2*>(p);
        if (swap) {
            const u64 t = v.x;
            v.x = v.y;
            v.y = t;
        }
        return v;
    };
    const ulonglong2 ab = load2(it.acc + so), cb = load2(it.conv + so);
    const ulonglong2 aa = load2(it.acc + ((size_t)np << logN) + so), ca = load2(it.conv + ((size_t)nq << logN) + so);
    ulonglong2 vb, va;
    vb.x = mul_shoup(sub_mod(ab.x, cb.x, q), pinv[i], pinv_sh[i], q);
    vb.y = mul_shoup(sub_mod(ab.y, cb.y, q), pinv[i], pinv_sh[i], q);
    va.x = mul_shoup(sub_mod(aa.x, ca.x, q), pinv[i], pinv_sh[i], q);
    va.y = mul_shoup(sub_mod(aa.y, ca.y, q), pinv[i], pinv_sh[i], q);
    if (it.add0) {
        const ulonglong2 a0 = load2(it.add0 + so);
        vb.x = add_mod(vb.x, a0.x, q);
        vb.y = add_mod(vb.y, a0.y, q);
    }
    if (it.add1) {
        const ulonglong2 a1 = load2(it.add1 + so);
        va.x = add_mod(va.x, a1.x, q);
        va.y = add_mod(va.y, a1.y, q);
    }
    const size_t oo = ((size_t)i << logN) + n;
    ulonglong2* o0 = reinterpret_cast<ulonglong2*>(it.out + oo);
    ulonglong2* o1 = reinterpret_cast<ulonglong2*>(it.out + ((size_t)nq << logN) + oo);
    if (it.accumulate) {
        const ulonglong2 p0 = *o0, p1 = *o1;
        vb.x = add_mod(p0.x, vb.x, q);
        vb.y = add_mod(p0.y, vb.y, q);
        va.x = add_mod(p1.x, va.x, q);
        va.y = add_mod(p1.y, va.y, q);
    }
    *o0 = vb;
    *o1 = va;
}

// Two coefficients per thread (n even, n + 1): the automorphism maps the pair
// onto the pair perm(n) & ~1 (perm(n + 1) = perm(n) ^ 1, since 2 brv(n + 1) + 1
// = 2 brv(n) + 1 + N and N g = N mod 2N flips only the top bit), so every
// access is a 16-byte load or store.
__global__ void k_lift(const LiftItem* items, const Modulus* mods, const int* ks_limbs, const u64* pmod,
                       const u64* pmod_sh, int level, int k, int logN) {
    const int N = 1 << logN;
    const int n = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    if (n >= N) return;
    const LiftItem it = items[blockIdx.z];
    const int p = blockIdx.y, np = level + 1 + k, nq = level + 1;
    const int mi = ks_limbs[p];
    const u64 q = mods[mi].q;
    const uint32_t src = it.galois == 1 ? (uint32_t)n : galois_perm(n, it.galois, logN);
    const uint32_t pair = src & ~1u;
    const bool swap = src & 1u;
    auto load2 = [&](const u64* base) -> ulonglong2 {
        ulonglong2 v = *reinterpret_cast<const ulonglong2*>(base + pair);
        if (swap) {
            const u64 t = v.x;
            v.x = v.y;
            v.y = t;
        }
        return v;
    };
    ulonglong2 vb = make_ulonglong2(0, 0), va = make_ulonglong2(0, 0);
    if (it.acc) {
        vb = load2(it.acc + ((size_t)p << logN));
        va = load2(it.acc + ((size_t)(np + p) << logN));
    }
    if (p < nq) {
        const ulonglong2 c0 = load2(it.ct + ((size_t)p << logN));
        vb.x = add_mod(vb.x, mul_shoup(c0.x, pmod[p], pmod_sh[p], q), q);
        vb.y = add_mod(vb.y, mul_shoup(c0.y, pmod[p], pmod_sh[p], q), q);
        if (!it.acc) {
            const ulonglong2 c1 = load2(it.ct + ((size_t)(nq + p) << logN));
            va.x = mul_shoup(c1.x, pmod[p], pmod_sh[p], q);
            va.y = mul_shoup(c1.y, pmod[p], pmod_sh[p], q);
        }
    }
    *reinterpret_cast<ulonglong2*>(it.out + ((size_t)p << logN) + n) = vb;
    *reinterpret_cast<ulonglong2*>(it.out + ((size_t)(np + p) << logN) + n) = va;
}

__global__ void k_combine_sum(const SumItem* items, const SumEntry* entries, const Modulus* mods,
                              const u64* pinv, const u64* pinv_sh, int level, int k, int logN) {
    const int N = 1 << logN;
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const SumItem it = items[blockIdx.z];
    const int i = blockIdx.y;
    const int np = level + 1 + k, nq = level + 1;
    const u64 q = mods[i].q;
    const size_t oo = ((size_t)i << logN) + n, oo1 = ((size_t)nq << logN) + oo;
    u64 c0 = 0, ab = 0, aa = 0;  // sums of perm(c0), perm(acc_b - conv_b), perm(acc_a - conv_a)
    for (int e = 0; e < it.n_e; e++) {
        const SumEntry en = entries[it.e0 + e];
        const uint32_t src = galois_perm(n, en.galois, logN);
        const size_t so = ((size_t)i << logN) + src;
        u64 vb = en.acc[so], va = en.acc[((size_t)np << logN) + so];
        if (!it.convsum) {
            vb = sub_mod(vb, en.conv[so], q);
            va = sub_mod(va, en.conv[((size_t)nq << logN) + so], q);
        }
        c0 = add_mod(c0, en.add0[so], q);
        ab = add_mod(ab, vb, q);
        aa = add_mod(aa, va, q);
    }
    if (it.convsum) {
        ab = sub_mod(ab, it.convsum[oo], q);
        aa = sub_mod(aa, it.convsum[oo1], q);
    }
    u64 v0 = add_mod(c0, mul_shoup(ab, pinv[i], pinv_sh[i], q), q);
    u64 v1 = mul_shoup(aa, pinv[i], pinv_sh[i], q);
    if (it.base) {
        v0 = add_mod(v0, it.base[oo], q);
        v1 = add_mod(v1, it.base[oo1], q);
    }
    if (it.accumulate) {
        v0 = add_mod(v0, it.out[oo], q);
        v1 = add_mod(v1, it.out[oo1], q);
    }
    it.out[oo] = v0;
    it.out[oo1] = v1;
}

// coefficient-domain automorphism sum: (sigma_g a)[i] = a[j] if j = i g^-1 mod 2N < N,
// else -a[j - N]
__global__ void k_autosum(const SumItem* items, const SumEntry* entries, u64* out, const Modulus* mods,
                          int level, int logN) {
    const int N = 1 << logN;
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const SumItem it = items[blockIdx.z];
    const int nq = level + 1;
    const int pl = blockIdx.y;  // poly * nq + limb
    const int i = pl % nq;
    const u64 q = mods[i].q;
    const size_t lo = (size_t)pl << logN;
    u64 acc = 0;
    for (int e = 0; e < it.n_e; e++) {
        const SumEntry en = entries[it.e0 + e];
        const uint32_t j = (uint32_t)(((uint64_t)n * en.galois_inv) & ((2ull << logN) - 1));
        if (j < (uint32_t)N)
            acc = add_mod(acc, en.conv[lo + j], q);
        else
            acc = sub_mod(acc, en.conv[lo + j - N], q);
    }
    out[(size_t)blockIdx.z * 2 * nq * N + lo + n] = acc;
}

// ------------------------------------------------------------------------
// PMult-MAC: out[poly][i][n] = sum_terms ct[poly][i][n] * pt[i][n]
// blockIdx.x = item, y = coefficient tile, z = limb i.  Partial sums stay in
// 128 bits; with moduli below 2^48 (HB <= 2) a product is below 2^96 and the
// sums are reduced once at the end, wider moduli fold every 16 terms
// (products below 2^122).
// ------------------------------------------------------------------------
// PMult-MAC with the operand tiles streamed through shared memory by the bulk
// async-copy engine.  One CTA = one item (up to W outputs sharing their
// ciphertext terms), one limb, a tile of T coefficients (T = min(512, N)):
// T / 2 consumer threads (two coefficients each) and one producer warp.  For
// term t the CTA needs the tiles of c0 and c1 of the term's ciphertext (2 T 8
// bytes) and of each output's compact plaintext (T low words and T high parts
// of HB bytes, (4 + HB) T contiguous bytes), copied with cp.async.bulk into
// stage t mod S and signalled on the stage's "full" mbarrier (arrive.expect_tx
// by the producer, complete_tx by the copies).  Each consumer warp arrives on
// the stage's "empty" mbarrier when it has read the stage; the producer waits
// for that before refilling it, so consumers never wait on one another.  Every
// wait is bounded (`limit` ns of %globaltimer, 2 s unless fe_ctx_set_mac_wait
// changed it): on expiry the thread sets bit 0 of *status and stops without
// writing its outputs.  Before it exits, the producer waits (bounded) until the
// copies of the last S terms it issued have landed, on the normal path as on
// expiry, so no copy is still writing into the CTA's shared memory when it
// ends.  unfed_term >= 0 (tests of the expiry path only) makes the producer
// announce that term's bytes without issuing its copies: its stage never fills
// and the consumers' wait runs out.
constexpr int kMacTile = 512;
constexpr int kMacStageBytes = 98304;  // shared memory for the stages of one CTA

template <int W, int HB>
__host__ __device__ constexpr int mac_stage_bytes() { return (16 + W * (4 + HB)) * kMacTile; }
template <int W, int HB>
__host__ __device__ constexpr int mac_stages() { return kMacStageBytes / mac_stage_bytes<W, HB>(); }

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0;
}
// bounded wait for phase `parity` of the barrier; false when the limit expired.
// The clock is read only once the first attempt finds the phase incomplete, so
// a wait on a stage that is already full costs one try_wait.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint64_t limit_ns) {
    if (mbar_try(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (;;) {
        if (mbar_try(bar, parity)) return true;
        if (global_ns() - t0 > limit_ns) return false;
    }
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

template <int W, int HB, bool kM36>
__global__ void __launch_bounds__(kMacTile / 2 + 32, 2) k_mac(const MacItem* items, const MacTerm* terms,
                                                          const Modulus* mods, const int* mod_map, int nl,
                                                          int logN, int T, uint32_t* status, uint64_t limit,
                                                          int unfed_term) {
    constexpr int S = mac_stages<W, HB>();
    extern __shared__ __align__(128) unsigned char mac_smem[];
    uint64_t* full = (uint64_t*)mac_smem;  // [S]
    uint64_t* empty = full + S;            // [S]
    unsigned char* stage0 = mac_smem + 256;  // [S] x (c0 | c1 | W x (low | high))
    const size_t stage_stride = (size_t)(16 + W * (4 + HB)) * T;
    // blockIdx.x = item (fastest): the items of one (tile, limb) run together and
    // the ciphertext tiles they share are read from L2
    // the item stays in global memory (cached): its counts are kept in
    // registers, its pointers and term indices are read where they are used
    const MacItem* itp = items + blockIdx.x;
    const int n_terms = itp->n_terms, n_out = itp->n_out;
    const int i = blockIdx.z;
    const Modulus m = mods[mod_map ? mod_map[i] : i];
    const size_t base = (size_t)blockIdx.y * T;
    const size_t off0 = ((size_t)i << logN) + base, off1 = ((size_t)(nl + i) << logN) + base;
    // compact plaintext limb i, tile blockIdx.y: T low words then T high parts,
    // (4 + HB) T contiguous bytes
    const size_t pt_off = ((size_t)i << logN) * (4 + HB) + base * (4 + HB);
    const uint32_t ct_tile = (uint32_t)T * 8u, lo_tile = (uint32_t)T * 4u, hi_tile = (uint32_t)T * HB;
    const int tid = threadIdx.x;
    const int n_cons = T / 2;                  // consumer threads
    const int n_cons_warps = (n_cons + 31) / 32;
    if (tid == 0) {
        for (int s = 0; s < S; s++) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], n_cons_warps);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (tid >= n_cons) {
        // producer warp: lane 0 keeps up to S terms in flight.  The operand
        // pointers of the next term are loaded as soon as the current term's
        // copies are issued, so their global loads complete during the wait
        // for a free stage; the loops over the outputs are unrolled over W so
        // that the item stays in registers.
        if (tid != n_cons) return;
        const uint32_t stage_bytes = 2 * ct_tile + (uint32_t)n_out * (lo_tile + hi_tile);
        const u64* ct = nullptr;
        const uint8_t* pt[W];
        auto load_pointers = [&](int t) {
            ct = terms[itp->term0[0] + t].ct;
#pragma unroll
            for (int k = 0; k < W; k++) pt[k] = k < n_out ? terms[itp->term0[k] + t].pt : nullptr;
        };
        if (n_terms > 0) load_pointers(0);
        int issued = 0;
        bool ok = true;
        for (; issued < n_terms; issued++) {
            const int s = issued % S;
            if (issued >= S && !mbar_wait(&empty[s], (uint32_t)((issued / S - 1) & 1), limit)) {
                ok = false;
                break;
            }
            unsigned char* st = stage0 + (size_t)s * stage_stride;
            mbar_expect_tx(&full[s], stage_bytes);
            if (issued != unfed_term) {  // an unfed term (expiry tests only) never fills its stage
                bulk_g2s(st, ct + off0, ct_tile, &full[s]);
                bulk_g2s(st + ct_tile, ct + off1, ct_tile, &full[s]);
#pragma unroll
                for (int k = 0; k < W; k++)
                    if (k < n_out)
                        bulk_g2s(st + 2 * ct_tile + (size_t)k * (lo_tile + hi_tile), pt[k] + pt_off,
                                 lo_tile + hi_tile, &full[s]);
            }
            if (issued + 1 < n_terms) load_pointers(issued + 1);
        }
        if (!ok) atomicOr(status, 1u);
        // Before this thread exits, the copies of the last S issued terms must have
        // landed: consumers that gave up early no longer keep the CTA (and its
        // shared memory) alive.  On the normal path these phases complete as the
        // copies arrive, independently of the consumers.  Bounded like every wait.
        for (int t = issued - S < 0 ? 0 : issued - S; t < issued; t++)
            if (t != unfed_term && !mbar_wait(&full[t % S], (uint32_t)((t / S) & 1), limit)) atomicOr(status, 1u);
        return;
    }
    // (coefficient 2 tid, 2 tid + 1) x (c0, c1 part); with 1-byte high planes
    // (every modulus below 2^40) the sums are kept as Acc40, else in 128 bits
    // (every modulus below 2^36: Acc36, two widening and two 32-bit
    // multiply-adds per product, folded every 16 terms)
    constexpr bool kSplit = HB == 1;
    using Acc = typename std::conditional<kM36, Acc36, typename std::conditional<kSplit, Acc40, u128>::type>::type;
    Acc a0[W], a1[W], b0[W], b1[W];
    auto zero = [](Acc& a) {
        if constexpr (kM36) acc36_zero(a); else if constexpr (kSplit) acc40_zero(a); else a = 0;
    };
    auto mad = [](Acc& a, u64 x, u64 y) {
        if constexpr (kM36) acc36_mad(a, x, split24_lo(y), split24_hi(y));
        else if constexpr (kSplit) acc40_mad(a, x, y);
        else a += (u128)x * y;
    };
    auto value = [](const Acc& a) -> u128 {
        if constexpr (kM36) return acc36_value(a); else if constexpr (kSplit) return acc40_value(a); else return a;
    };
#pragma unroll
    for (int k = 0; k < W; k++) {
        zero(a0[k]);
        zero(a1[k]);
        zero(b0[k]);
        zero(b1[k]);
    }
    for (int t = 0; t < n_terms; t++) {
        const int s = t % S;
        if (!mbar_wait(&full[s], (uint32_t)((t / S) & 1), limit)) {
            atomicOr(status, 1u);
            return;
        }
        const unsigned char* st = stage0 + (size_t)s * stage_stride;
        const ulonglong2 x0 = reinterpret_cast<const ulonglong2*>(st)[tid];
        const ulonglong2 x1 = reinterpret_cast<const ulonglong2*>(st + ct_tile)[tid];
#pragma unroll
        for (int k = 0; k < W; k++) {
            if (k >= n_out) break;
            const unsigned char* pk = st + 2 * ct_tile + (size_t)k * (lo_tile + hi_tile);
            const uint2 lo = reinterpret_cast<const uint2*>(pk)[tid];
            u64 hx, hy;
            if (HB == 1) {
                const uchar2 h = reinterpret_cast<const uchar2*>(pk + lo_tile)[tid];
                hx = h.x, hy = h.y;
            } else if (HB == 2) {
                const ushort2 h = reinterpret_cast<const ushort2*>(pk + lo_tile)[tid];
                hx = h.x, hy = h.y;
            } else {
                const uint2 h = reinterpret_cast<const uint2*>(pk + lo_tile)[tid];
                hx = h.x, hy = h.y;
            }
            const u64 px = (u64)lo.x | (hx << 32), py = (u64)lo.y | (hy << 32);
            if constexpr (kM36) {
                const uint32_t lx = split24_lo(px), hx = split24_hi(px), ly = split24_lo(py), hy = split24_hi(py);
                acc36_mad(a0[k], x0.x, lx, hx);
                acc36_mad(a1[k], x0.y, ly, hy);
                acc36_mad(b0[k], x1.x, lx, hx);
                acc36_mad(b1[k], x1.y, ly, hy);
            } else {
                mad(a0[k], x0.x, px);
                mad(a1[k], x0.y, py);
                mad(b0[k], x1.x, px);
                mad(b1[k], x1.y, py);
            }
        }
        __syncwarp();
        if ((tid & 31) == 0) mbar_arrive(&empty[s]);
        // the Acc40 sums hold 2^15 terms (HB = 1); a product is below 2^96 when
        // every modulus is below 2^48 (HB = 2), so 2^31 terms fit the 128-bit
        // sums; wider moduli (products below 2^120) fold every 16 terms.  A fold
        // replaces a sum by its residue, which leaves the final residue unchanged.
        if constexpr (kM36) {
            if ((t & 15) == 15) {
#pragma unroll
                for (int k = 0; k < W; k++) {
                    if (k >= n_out) break;
                    acc36_fold(a0[k]);
                    acc36_fold(a1[k]);
                    acc36_fold(b0[k]);
                    acc36_fold(b1[k]);
                }
            }
        }
        if ((kSplit && (t & 0x3FFF) == 0x3FFF) || (HB == 4 && (t & 15) == 15)) {
            auto fold = [&](Acc& a) {
                const u64 r = reduce128(value(a), m);
                zero(a);
                mad(a, r, 1);
            };
#pragma unroll
            for (int k = 0; k < W; k++) {
                if (k >= n_out) break;
                fold(a0[k]);
                fold(a1[k]);
                fold(b0[k]);
                fold(b1[k]);
            }
        }
    }
#pragma unroll
    for (int k = 0; k < W; k++) {
        if (k >= n_out) break;
        ulonglong2 r0, r1;
        r0.x = reduce128(value(a0[k]), m);
        r0.y = reduce128(value(a1[k]), m);
        r1.x = reduce128(value(b0[k]), m);
        r1.y = reduce128(value(b1[k]), m);
        reinterpret_cast<ulonglong2*>(itp->out[k] + off0)[tid] = r0;
        reinterpret_cast<ulonglong2*>(itp->out[k] + off1)[tid] = r1;
    }
}

// byte offset of the tile holding residue n inside a compact limb, and n's index in it
__device__ __forceinline__ size_t pt_tile_at(int n, int T, int hb, int& r) {
    r = n % T;
    return (size_t)(n / T) * (4 + hb) * T;
}

// 64-bit limbs -> compact limbs (tiles of T residues: T low words, then T high parts)
__global__ void k_pt_compact(const u64* in, uint8_t* out, int hb, int T, int logN) {
    const int N = 1 << logN;
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const size_t j = blockIdx.y;
    const u64 v = in[(j << logN) + n];
    int r;
    uint8_t* tile = out + j * (4 + hb) * (size_t)N + pt_tile_at(n, T, hb, r);
    reinterpret_cast<uint32_t*>(tile)[r] = (uint32_t)v;
    uint8_t* hi = tile + 4 * (size_t)T;
    if (hb == 1) hi[r] = (uint8_t)(v >> 32);
    else if (hb == 2) reinterpret_cast<uint16_t*>(hi)[r] = (uint16_t)(v >> 32);
    else reinterpret_cast<uint32_t*>(hi)[r] = (uint32_t)(v >> 32);
}

__global__ void k_pmult_compact(const u64* ct, const uint8_t* pt, u64* out, const Modulus* mods, int nl, int hb,
                                int T, int logN, int accumulate) {
    const int N = 1 << logN;
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const int i = blockIdx.y;  // limb
    const Modulus m = mods[i];
    int r;
    const uint8_t* tile = pt + (size_t)i * (4 + hb) * N + pt_tile_at(n, T, hb, r);
    const uint8_t* hi = tile + 4 * (size_t)T;
    const u64 h = hb == 1 ? (u64)hi[r] : (hb == 2 ? (u64)reinterpret_cast<const uint16_t*>(hi)[r]
                                                  : (u64)reinterpret_cast<const uint32_t*>(hi)[r]);
    const u64 p = (u64)reinterpret_cast<const uint32_t*>(tile)[r] | (h << 32);
    for (int poly = 0; poly < 2; poly++) {
        const size_t o = ((size_t)poly * nl + i) * N + n;
        u64 v = mul_mod(ct[o], p, m);
        out[o] = accumulate ? add_mod(out[o], v, m.q) : v;
    }
}

// ModDown and rescale in one division by q_l P: out_i = (acc_i - conv_i)
// (q_l P)^-1 mod q_i for i < l.  acc: [n][2][l+1+k][N] (NTT form), conv:
// [n][2][l][N] (NTT form of the centred conversion of [acc]_{q_l P}), outs[j]:
// item j's output [2][l][N].  blockIdx.y = limb i, z = polynomial over 2n.
__global__ void k_mdrs_combine(const u64* acc, const u64* conv, u64* const* outs, const Modulus* mods,
                               const u64* qpinv, const u64* qpinv_sh, int level, int k, int L, int logN) {
    const int N = 1 << logN;
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const int i = blockIdx.y, z = blockIdx.z, item = z >> 1, poly = z & 1;
    const int np = level + 1 + k;
    const u64 q = mods[i].q;
    const u64 a = acc[((((size_t)item * 2 + poly) * np + i) << logN) + n];
    const u64 c = conv[((((size_t)item * 2 + poly) * level + i) << logN) + n];
    const size_t ti = (size_t)level * (L + 1) + i;
    outs[item][(((size_t)poly * level + i) << logN) + n] = mul_shoup(sub_mod(a, c, q), qpinv[ti], qpinv_sh[ti], q);
}

__global__ void k_rescale_combine(const u64* in, const u64* lift, u64* out, const Modulus* mods,
                                  const u64* qlinv, const u64* qlinv_sh, int level, int L,
                                  int logN) {
    const int N = 1 << logN;
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const int i = blockIdx.y, poly = blockIdx.z;  // poly over n_ct * 2
    const u64 q = mods[i].q;
    const u64* ip = in + (size_t)poly * (level + 1) * N;
    const u64* lp = lift + (size_t)poly * level * N;
    u64* op = out + (size_t)poly * level * N;
    u64 v = sub_mod(ip[((size_t)i << logN) + n], lp[((size_t)i << logN) + n], q);
    const size_t ti = (size_t)level * (L + 1) + i;
    op[((size_t)i << logN) + n] = mul_shoup(v, qlinv[ti], qlinv_sh[ti], q);
}

__global__ void k_add(const u64* a, const u64* b, u64* out, const Modulus* mods, int nl, int logN) {
    const int N = 1 << logN;
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const int limb = blockIdx.y;  // over the 2 (l+1) limbs of one ciphertext
    const u64 q = mods[limb % nl].q;
    const size_t o = ((size_t)blockIdx.z * gridDim.y + limb) * N + n;
    out[o] = add_mod(a[o], b[o], q);
}

__global__ void k_pmult(const u64* ct, const u64* pt, u64* out, const Modulus* mods, int nl,
                        int logN, int accumulate) {
    const int N = 1 << logN;
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const int i = blockIdx.y, ci = blockIdx.z;  // limb, ciphertext
    const Modulus m = mods[i];
    const u64 p = pt[((size_t)ci * nl + i) * N + n];
    for (int poly = 0; poly < 2; poly++) {
        const size_t o = (((size_t)ci * 2 + poly) * nl + i) * N + n;
        u64 v = mul_mod(ct[o], p, m);
        out[o] = accumulate ? add_mod(out[o], v, m.q) : v;
    }
}

// (x0, x1) (x) (y0, y1) -> d0 = x0 y0, d1 = x0 y1 + x1 y0, d2 = x1 y1 ([3][l+1][N] per ct)
__global__ void k_tensor(const u64* x, const u64* y, u64* d, const Modulus* mods, int nl, int logN) {
    const int N = 1 << logN;
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const int i = blockIdx.y, ci = blockIdx.z;
    const Modulus m = mods[i];
    const size_t b = (size_t)ci * 2 * nl * N, o = (size_t)i * N + n, s = (size_t)nl * N;
    u64 x0 = x[b + o], x1 = x[b + s + o], y0 = y[b + o], y1 = y[b + s + o];
    const size_t db = (size_t)ci * 3 * nl * N;
    d[db + o] = mul_mod(x0, y0, m);
    d[db + s + o] = reduce128((u128)reduce128((u128)x0 * y1, m) + (u128)x1 * y0, m);
    d[db + 2 * s + o] = mul_mod(x1, y1, m);
}

__global__ void k_sample_uniform(GenKey gk, u64 seed, u64 tag_base, u64* out, const int* mod_idx,
                                 const Modulus* mods, int logN) {
    const int N = 1 << logN;
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const int l = blockIdx.y;
    const int mi = mod_idx[l];
    const u64 w = gen_word(gk, seed, tag_base + (u64)mi, (u64)n);
    out[((size_t)l << logN) + n] = (u64)(((u128)w * mods[mi].q) >> 64);
}

// kind 0: ternary floor(3 w / 2^64) - 1; kind 1: centred binomial eta = 21
__global__ void k_sample_signed(GenKey gk, u64 seed, u64 tag, int kind, i64* out, int logN) {
    const int N = 1 << logN;
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const u64 w = gen_word(gk, seed, tag, (u64)n);
    if (kind == 0)
        out[n] = (i64)(((u128)w * 3u) >> 64) - 1;
    else
        out[n] = (i64)__popcll(w & 0x1FFFFFull) - (i64)__popcll((w >> 21) & 0x1FFFFFull);
}

__global__ void k_signed_to_limbs(const i64* v, u64* out, const Modulus* mods, int first_mod,
                                  size_t stride, int logN) {
    const int N = 1 << logN;
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const int l = blockIdx.y;
    out[(size_t)l * stride + n] = from_signed(v[n], mods[first_mod + l].q);
}

}  // namespace

void launch_bconv(fe_ctx* c, const BConvTab& t, int level, const u64* in, size_t in_stride,
                  int in_pos_base, u64* out, size_t out_stride, int n_poly, bool copy_src,
                  cudaStream_t st) {
    if (n_poly == 0) return;
    ProfScope ps(c, PK_BCONV, st, 8.0 * c->N * n_poly * (t.n_src * (copy_src ? 2 : 1) + t.n_dst));
    const int cs = copy_src ? 1 : 0;
    // two coefficients per thread when every 16-byte access is aligned
    const bool pair = c->N >= 2 && !(((uintptr_t)in | (uintptr_t)out) & 15) && !(in_stride & 1) &&
                      !(out_stride & 1) && !(c->N & 1);
    const dim3 g = pair ? grid_for(c->N / 2, n_poly) : grid_for(c->N, n_poly);
#define FE_BCONV(S)                                                                                   \
    case S:                                                                                           \
        if (pair && c->narrow && c->max_mod_bits <= 36)                                               \
            k_bconv2<S, true, true><<<g, kB, 0, st>>>(t, c->d_mod, c->L, level, c->logN, in, in_stride, \
                                                      in_pos_base, out, out_stride, cs);              \
        else if (pair && c->narrow)                                                                   \
            k_bconv2<S, true, false><<<g, kB, 0, st>>>(t, c->d_mod, c->L, level, c->logN, in,         \
                                                       in_stride, in_pos_base, out, out_stride, cs);  \
        else if (pair)                                                                                \
            k_bconv2<S, false, false><<<g, kB, 0, st>>>(t, c->d_mod, c->L, level, c->logN, in,        \
                                                        in_stride, in_pos_base, out, out_stride, cs); \
        else if (c->narrow)                                                                           \
            k_bconv<S, true><<<g, kB, 0, st>>>(t, c->d_mod, c->L, level, c->logN, in, in_stride,      \
                                               in_pos_base, out, out_stride, cs);                     \
        else                                                                                          \
            k_bconv<S, false><<<g, kB, 0, st>>>(t, c->d_mod, c->L, level, c->logN, in, in_stride,     \
                                                in_pos_base, out, out_stride, cs);                    \
        break;
    switch (t.n_src) {
        FE_BCONV(1) FE_BCONV(2) FE_BCONV(3) FE_BCONV(4) FE_BCONV(5) FE_BCONV(6) FE_BCONV(7) FE_BCONV(8)
        default: break;  // n_src <= k <= 8 (checked at context creation)
    }
#undef FE_BCONV
    c->cnt.launches++;
}

void launch_keyip(fe_ctx* c, const KsItem* items, int n_items, int level, cudaStream_t st) {
    if (!n_items) return;
    const int np = level + 1 + c->k, dn = (level + c->k) / c->k;
    ProfScope ps(c, PK_KEYIP, st, 8.0 * c->N * np * n_items * (3.0 * dn + 2));
    k_keyip<<<grid_for(c->N, level + 1 + c->k, n_items), kB, 0, st>>>(items, c->d_mod, c->L, level,
                                                                     c->k, c->logN, c->n_mod, c->narrow);
    c->cnt.launches++;
}

template <int D, bool kNarrow>
static void keyip_launch(dim3 g, size_t esm, cudaStream_t st, const KsGroup* groups, const KsItem* items, fe_ctx* c,
                         int level) {
    static bool set = false;  // more than 48 KiB of digit buffers when D > 6
    if (!set && esm > (48u << 10))
        set = cudaFuncSetAttribute(k_keyip_grouped<D, kNarrow>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)esm) == cudaSuccess;
    k_keyip_grouped<D, kNarrow><<<g, kB, esm, st>>>(groups, items, c->d_mod, c->L, level, c->k, c->logN, c->n_mod);
}

void launch_keyip_grouped(fe_ctx* c, const KsGroup* groups, const KsItem* items, int n_groups,
                          int n_items, int level, cudaStream_t st, int n_sources) {
    if (!n_groups) return;
    const int np = level + 1 + c->k, dn = (level + c->k) / c->k;
    // algorithmic bytes: every key once, every distinct source's digits once,
    // every item's two accumulators written
    const double src = n_sources > 0 ? n_sources : n_items;
    ProfScope ps(c, PK_KEYIP, st, 8.0 * c->N * np * (2.0 * dn * n_groups + src * dn + 2.0 * n_items));
    const dim3 g(n_groups, (c->N / 2 + kB - 1) / kB, level + 1 + c->k);  // two coefficients per thread
    const size_t esm = (size_t)2 * dn * kB * 16;                          // double-buffered digits
    // narrow reductions for up to 8 digits (the sums stay below 2^84)
#define FE_KEYIP_N(D)                                                                                 \
    case D:                                                                                           \
        if (c->narrow)                                                                                \
            keyip_launch<D, true>(g, esm, st, groups, items, c, level);                              \
        else                                                                                          \
            keyip_launch<D, false>(g, esm, st, groups, items, c, level);                             \
        break;
#define FE_KEYIP(D)                                                                                   \
    case D:                                                                                           \
        keyip_launch<D, false>(g, esm, st, groups, items, c, level);                                 \
        break;
    switch (dn) {
        FE_KEYIP_N(1) FE_KEYIP_N(2) FE_KEYIP_N(3) FE_KEYIP_N(4) FE_KEYIP_N(5) FE_KEYIP_N(6) FE_KEYIP_N(7)
        FE_KEYIP_N(8) FE_KEYIP(9) FE_KEYIP(10) FE_KEYIP(11) FE_KEYIP(12) FE_KEYIP(13) FE_KEYIP(14)
        FE_KEYIP(15) FE_KEYIP(16)
        default: break;  // dnum <= 16 (checked at context creation)
    }
#undef FE_KEYIP_N
#undef FE_KEYIP
    c->cnt.launches++;
}

void launch_combine(fe_ctx* c, const CombineItem* items, int n_items, int level, cudaStream_t st) {
    if (!n_items) return;
    ProfScope ps(c, PK_COMBINE, st, 8.0 * c->N * (level + 1) * 7.0 * n_items);
    k_combine<<<grid_for(c->N / 2, level + 1, n_items), kB, 0, st>>>(items, c->d_mod, c->d_pinv,
                                                                c->d_pinv_sh, level, c->k, c->logN);
    c->cnt.launches++;
}

void launch_lift(fe_ctx* c, const LiftItem* items, int n_items, int level, cudaStream_t st, int n_acc, int n_sources) {
    if (!n_items) return;
    const int np = level + 1 + c->k;
    // algorithmic bytes: each accumulator read (2 np limbs), each distinct
    // source ciphertext read once (2 (l+1)), every output written (2 np)
    const double acc = n_acc >= 0 ? n_acc : n_items, src = n_sources > 0 ? n_sources : n_items;
    ProfScope ps(c, PK_COMBINE, st, 8.0 * c->N * (2.0 * np * acc + 2.0 * (level + 1) * src + 2.0 * np * n_items));
    k_lift<<<grid_for(c->N / 2, np, n_items), kB, 0, st>>>(items, c->d_mod, c->lv[level].d_ks_limbs, c->d_pmod,
                                                           c->d_pmod_sh, level, c->k, c->logN);
    c->cnt.launches++;
}

void launch_combine_sum(fe_ctx* c, const SumItem* items, const SumEntry* entries, int n_items,
                        int n_entries, int level, cudaStream_t st) {
    if (!n_items) return;
    ProfScope ps(c, PK_COMBINE, st, 8.0 * c->N * (level + 1) * (4.0 * n_items + 5.0 * n_entries));
    k_combine_sum<<<grid_for(c->N, level + 1, n_items), kB, 0, st>>>(
        items, entries, c->d_mod, c->d_pinv, c->d_pinv_sh, level, c->k, c->logN);
    c->cnt.launches++;
}

void launch_autosum(fe_ctx* c, const SumItem* items, const SumEntry* entries, int n_items, int n_entries, u64* out,
                    int level, cudaStream_t st) {
    if (!n_items) return;
    ProfScope ps(c, PK_COMBINE, st, 8.0 * c->N * 2 * (level + 1) * ((double)n_entries + n_items));
    k_autosum<<<grid_for(c->N, 2 * (level + 1), n_items), kB, 0, st>>>(items, entries, out, c->d_mod, level, c->logN);
    c->cnt.launches++;
}

template <int W, int HB, bool kM36>
static void mac_launch(dim3 g, int threads, size_t smem, cudaStream_t st, const MacItem* items, const MacTerm* terms,
                       const Modulus* mods, const int* mm, int nl, int logN, int T, uint32_t* status,
                       uint64_t limit, int unfed_term) {
    static bool set = false;
    if (!set)
        set = cudaFuncSetAttribute(k_mac<W, HB, kM36>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) ==
              cudaSuccess;
    k_mac<W, HB, kM36><<<g, threads, smem, st>>>(items, terms, mods, mm, nl, logN, T, status, limit, unfed_term);
}

void launch_mac(fe_ctx* c, const MacItem* items, const MacTerm* terms, int n_items, int n_ct_terms,
                int n_pt_terms, int n_outputs, int ways, int level, cudaStream_t st, bool qp, int n_ct_distinct) {
    if (!n_items) return;
    const int nl = qp ? level + 1 + c->k : level + 1;
    // algorithmic bytes: every plaintext as stored, every distinct ciphertext once
    // (loads of one ciphertext by several items come from L2), every output written
    const double cts = n_ct_distinct > 0 ? n_ct_distinct : n_ct_terms;
    ProfScope ps(c, PK_MAC, st, (double)c->N * nl * (8.0 * (2.0 * cts + 2.0 * n_outputs) +
                                                     (4.0 + c->pt_hb) * n_pt_terms));
    const int T = pt_tile(c);
    const dim3 g(n_items, c->N / T, nl);
    const int threads = T / 2 + 32;
    const int w = ways <= 1 ? 1 : (ways == 2 ? 2 : 4);
    const size_t smem = 256 + (size_t)kMacStageBytes;
    const int* mm = nl == level + 1 ? nullptr : c->lv[level].d_ks_limbs;
#define FE_MAC(W, HB)                                                                                    \
    mac_launch<W, HB, false>(g, threads, smem, st, items, terms, c->d_mod, mm, nl, c->logN, T, c->d_status, \
                             c->mac_wait_ns, c->mac_unfed_term)
#define FE_MAC36(W)                                                                                    \
    mac_launch<W, 1, true>(g, threads, smem, st, items, terms, c->d_mod, mm, nl, c->logN, T, c->d_status, \
                           c->mac_wait_ns, c->mac_unfed_term)
    if (c->pt_hb == 1 && c->max_mod_bits <= 36) {
        if (w == 1) FE_MAC36(1);
        else if (w == 2) FE_MAC36(2);
        else FE_MAC36(4);
    } else if (c->pt_hb == 1) {
        if (w == 1) FE_MAC(1, 1);
        else if (w == 2) FE_MAC(2, 1);
        else FE_MAC(4, 1);
    } else if (c->pt_hb == 2) {
        if (w == 1) FE_MAC(1, 2);
        else if (w == 2) FE_MAC(2, 2);
        else FE_MAC(4, 2);
    } else {
        if (w == 1) FE_MAC(1, 4);
        else if (w == 2) FE_MAC(2, 4);
        else FE_MAC(4, 4);
    }
#undef FE_MAC
#undef FE_MAC36
    c->cnt.launches++;
}

// Rotated-term MAC (see RotTerm): one coefficient pair per thread, grid (pairs,
// limb, item).  The automorphism maps the pair onto a pair (k_lift), so each
// operand is one 16-byte gather; the rotated copy's value is formed exactly as
// k_lift forms it (acc + P c0 on the q limbs, acc alone on the p limbs; acc for
// the second polynomial) and multiplied into the sums as k_mac does, so the
// residues equal the lift followed by the MAC.  The copies are never written:
// the lift's store and the MAC's reload of every rotated copy are saved.
template <int HB, bool kM36>
__global__ void __launch_bounds__(256) k_mac_rot(const RotItem* items, const RotTerm* terms, const Modulus* mods,
                                                 const int* ks_limbs, int nq, int np, int logN, int T) {
    const int N = 1 << logN;
    const int n = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    if (n >= N) return;
    const RotItem it = items[blockIdx.z];
    const int p = blockIdx.y;
    const Modulus m = mods[ks_limbs[p]];
    const u64 q = m.q;
    const size_t o0 = (size_t)p << logN, o1 = (size_t)(np + p) << logN;
    // compact plaintext limb p: tile n / T holds T low words then T high parts
    const size_t pt_tile_off = o0 * (4 + HB) + (size_t)(n / T) * (4 + HB) * T;
    const int r = n % T;
    constexpr bool kSplit = HB == 1;
    using Acc = typename std::conditional<kM36, Acc36, typename std::conditional<kSplit, Acc40, u128>::type>::type;
    auto zero = [](Acc& a) {
        if constexpr (kM36) acc36_zero(a); else if constexpr (kSplit) acc40_zero(a); else a = 0;
    };
    auto mad = [](Acc& a, u64 x, u64 y) {
        if constexpr (kM36) acc36_mad(a, x, split24_lo(y), split24_hi(y));
        else if constexpr (kSplit) acc40_mad(a, x, y);
        else a += (u128)x * y;
    };
    auto value = [](const Acc& a) -> u128 {
        if constexpr (kM36) return acc36_value(a); else if constexpr (kSplit) return acc40_value(a); else return a;
    };
    Acc a0, a1, b0, b1;
    zero(a0);
    zero(a1);
    zero(b0);
    zero(b1);
    for (int t = 0; t < it.n_terms; t++) {
        const RotTerm tm = terms[it.term0 + t];
        ulonglong2 v0, v1;
        if (tm.acc) {
            const uint32_t src = galois_perm(n, tm.galois, logN);
            const uint32_t pair = src & ~1u;
            const bool swap = src & 1u;
            auto load2 = [&](const u64* base) -> ulonglong2 {
                ulonglong2 v = *reinterpret_cast<const ulonglong2*>(base + pair);
                if (swap) {
                    const u64 x = v.x;
                    v.x = v.y;
                    v.y = x;
                }
                return v;
            };
            v0 = load2(tm.acc + o0);
            v1 = load2(tm.acc + o1);
            if (p < nq) {
                const ulonglong2 pc = load2(tm.xp + o0);  // P c0 at the source pair
                v0.x = add_mod(v0.x, pc.x, q);
                v0.y = add_mod(v0.y, pc.y, q);
            }
        } else {
            v0 = *reinterpret_cast<const ulonglong2*>(tm.xp + o0 + n);
            v1 = *reinterpret_cast<const ulonglong2*>(tm.xp + o1 + n);
        }
        const uint8_t* pk = tm.pt + pt_tile_off;
        const uint2 lo = *reinterpret_cast<const uint2*>(pk + (size_t)r * 4);
        u64 hx, hy;
        if (HB == 1) {
            const uchar2 h = *reinterpret_cast<const uchar2*>(pk + (size_t)4 * T + r);
            hx = h.x, hy = h.y;
        } else if (HB == 2) {
            const ushort2 h = *reinterpret_cast<const ushort2*>(pk + (size_t)4 * T + (size_t)r * 2);
            hx = h.x, hy = h.y;
        } else {
            const uint2 h = *reinterpret_cast<const uint2*>(pk + (size_t)4 * T + (size_t)r * 4);
            hx = h.x, hy = h.y;
        }
        const u64 px = (u64)lo.x | (hx << 32), py = (u64)lo.y | (hy << 32);
        mad(a0, v0.x, px);
        mad(a1, v0.y, py);
        mad(b0, v1.x, px);
        mad(b1, v1.y, py);
        // the same folds as k_mac (a fold replaces a sum by its residue)
        if constexpr (kM36) {
            if ((t & 15) == 15) {
                acc36_fold(a0);
                acc36_fold(a1);
                acc36_fold(b0);
                acc36_fold(b1);
            }
        }
        if ((kSplit && (t & 0x3FFF) == 0x3FFF) || (HB == 4 && (t & 15) == 15)) {
            auto fold = [&](Acc& a) {
                const u64 v = reduce128(value(a), m);
                zero(a);
                mad(a, v, 1);
            };
            fold(a0);
            fold(a1);
            fold(b0);
            fold(b1);
        }
    }
    *reinterpret_cast<ulonglong2*>(it.out + o0 + n) = make_ulonglong2(reduce128(value(a0), m), reduce128(value(a1), m));
    *reinterpret_cast<ulonglong2*>(it.out + o1 + n) = make_ulonglong2(reduce128(value(b0), m), reduce128(value(b1), m));
}

void launch_mac_rot(fe_ctx* c, const RotItem* items, const RotTerm* terms, int n_items, int n_terms, int n_acc_terms,
                    int level, cudaStream_t st) {
    if (!n_items) return;
    const int np = level + 1 + c->k, nq = level + 1;
    // algorithmic bytes: each rotated term's accumulators (2 np limbs) and the P c0
    // limbs (nq) it adds, each unrotated term's lifted copy (2 np), every plaintext
    // as stored, every output written
    ProfScope ps(c, PK_MAC, st, (double)c->N * (8.0 * ((2.0 * np + nq) * n_acc_terms + 2.0 * np * (n_terms - n_acc_terms) +
                                                       2.0 * np * n_items) +
                                                (4.0 + c->pt_hb) * np * n_terms));
    const dim3 g((c->N / 2 + 255) / 256, np, n_items);
    const int T = pt_tile(c);
    const int* ks = c->lv[level].d_ks_limbs;
    if (c->pt_hb == 1 && c->max_mod_bits <= 36)
        k_mac_rot<1, true><<<g, 256, 0, st>>>(items, terms, c->d_mod, ks, nq, np, c->logN, T);
    else if (c->pt_hb == 1)
        k_mac_rot<1, false><<<g, 256, 0, st>>>(items, terms, c->d_mod, ks, nq, np, c->logN, T);
    else if (c->pt_hb == 2)
        k_mac_rot<2, false><<<g, 256, 0, st>>>(items, terms, c->d_mod, ks, nq, np, c->logN, T);
    else
        k_mac_rot<4, false><<<g, 256, 0, st>>>(items, terms, c->d_mod, ks, nq, np, c->logN, T);
    c->cnt.launches++;
}

void launch_pt_compact(fe_ctx* c, const u64* in, uint8_t* out, int n_limbs, cudaStream_t st) {
    if (n_limbs <= 0) return;
    k_pt_compact<<<grid_for(c->N, n_limbs), kB, 0, st>>>(in, out, c->pt_hb, pt_tile(c), c->logN);
    c->cnt.launches++;
}

void launch_pmult_compact(fe_ctx* c, const u64* ct, const uint8_t* pt, u64* out, int level, bool accumulate,
                          cudaStream_t st) {
    k_pmult_compact<<<grid_for(c->N, level + 1), kB, 0, st>>>(ct, pt, out, c->d_mod, level + 1, c->pt_hb,
                                                             pt_tile(c), c->logN, accumulate ? 1 : 0);
    c->cnt.launches++;
}

void launch_mdrs_combine(fe_ctx* c, const u64* acc, const u64* conv, u64* const* outs, int n, int level,
                         cudaStream_t st) {
    if (!n) return;
    ProfScope ps(c, PK_RESCALE, st, 8.0 * c->N * 2 * n * (3.0 * level));
    k_mdrs_combine<<<grid_for(c->N, level, 2 * n), kB, 0, st>>>(acc, conv, outs, c->d_mod, c->d_qpinv, c->d_qpinv_sh,
                                                               level, c->k, c->L, c->logN);
    c->cnt.launches++;
}

void launch_rescale_combine(fe_ctx* c, const u64* in, const u64* lift, u64* out, int n_ct,
                            int level, cudaStream_t st) {
    ProfScope ps(c, PK_RESCALE, st, 8.0 * c->N * 2 * n_ct * (level + 1 + 2.0 * level));
    k_rescale_combine<<<grid_for(c->N, level, 2 * n_ct), kB, 0, st>>>(
        in, lift, out, c->d_mod, c->d_qlinv, c->d_qlinv_sh, level, c->L, c->logN);
    c->cnt.launches++;
}

void launch_add(fe_ctx* c, const u64* a, const u64* b, u64* out, int n_ct, int level,
                cudaStream_t st) {
    if (!n_ct) return;
    k_add<<<grid_for(c->N, 2 * (level + 1), n_ct), kB, 0, st>>>(a, b, out, c->d_mod, level + 1, c->logN);
    c->cnt.launches++;
}

void launch_pmult(fe_ctx* c, const u64* ct, const u64* pt, u64* out, int n_ct, int level,
                  bool accumulate, cudaStream_t st) {
    if (!n_ct) return;
    k_pmult<<<grid_for(c->N, level + 1, n_ct), kB, 0, st>>>(ct, pt, out, c->d_mod, level + 1, c->logN,
                                                           accumulate ? 1 : 0);
    c->cnt.launches++;
}

void launch_tensor(fe_ctx* c, const u64* x, const u64* y, u64* d012, int n_ct, int level,
                   cudaStream_t st) {
    if (!n_ct) return;
    k_tensor<<<grid_for(c->N, level + 1, n_ct), kB, 0, st>>>(x, y, d012, c->d_mod, level + 1, c->logN);
    c->cnt.launches++;
}

void launch_sample_uniform_limbs(fe_ctx* c, uint64_t seed, uint64_t tag_base, u64* out, int n_limbs,
                                 const int* mod_idx_dev, cudaStream_t st) {
    k_sample_uniform<<<grid_for(c->N, n_limbs), kB, 0, st>>>(c->gen, seed, tag_base, out, mod_idx_dev, c->d_mod,
                                                            c->logN);
    c->cnt.launches++;
}

void launch_sample_signed(fe_ctx* c, uint64_t seed, uint64_t tag, int kind, i64* out, cudaStream_t st) {
    k_sample_signed<<<grid_for(c->N, 1), kB, 0, st>>>(c->gen, seed, tag, kind, out, c->logN);
    c->cnt.launches++;
}

void launch_signed_to_limbs(fe_ctx* c, const i64* v, u64* out, int first_mod, int n_limbs,
                            size_t out_stride_words, cudaStream_t st) {
    k_signed_to_limbs<<<grid_for(c->N, n_limbs), kB, 0, st>>>(v, out, c->d_mod, first_mod,
                                                             out_stride_words, c->logN);
    c->cnt.launches++;
}

}  // namespace fe
