// Element-wise and key-switching kernels (declarations shared by the op files).
#pragma once

#include "context.h"
#include "prng.cuh"

namespace fe {

// position of modulus `mi` inside a polynomial over Q_level * P
__host__ __device__ __forceinline__ int ext_pos(int mi, int L, int level) {
    return mi <= L ? mi : mi - (L - level);
}

// NTT-domain index of the automorphism sigma_g: NTT(sigma_g a)[n] = NTT(a)[perm(n)]
// with 2 brv(perm(n)) + 1 = (2 brv(n) + 1) g mod 2N.
__device__ __forceinline__ uint32_t galois_perm(uint32_t n, uint32_t g, int logN) {
    uint32_t br = __brev(n) >> (32 - logN);
    uint64_t e = ((2ull * br + 1ull) * g) & ((2ull << logN) - 1ull);
    uint32_t j = (uint32_t)((e - 1) >> 1);
    return __brev(j) >> (32 - logN);
}

// One key-switch work item: ext digits -> accumulators over Q_l * P.
struct KsItem {
    const u64* ext;  // [dnum_l][l+1+k][N]
    const u64* key;  // [dnum_L][2][n_mod][N]
    u64* acc;        // [2][l+1+k][N]
};
// Items sharing one key: each thread reads the key once and applies it to all of them.
struct KsGroup {
    const u64* key;
    int item0, n_items;
};

// One ModDown/combine item: acc (NTT, [2][l+1+k][N]) and its converted P part
// (conv, NTT form on Q_l, [2][l+1][N]) ->
//   out0[n] (+)= add0[perm(n)] + (acc_b - conv_b)[perm(n)] P^-1
//   out1[n] (+)= add1[perm(n)] + (acc_a - conv_a)[perm(n)] P^-1
struct CombineItem {
    const u64* acc;
    const u64* conv;
    const u64* add0;  // [l+1][N] or null
    const u64* add1;  // [l+1][N] or null
    u64* out;         // [2][l+1][N]
    uint32_t galois;  // 1 = no automorphism
    int accumulate;   // 1: out += result
};

// Summed combine (rotate-and-sum over diagonals): for one output ciphertext,
//   out0[n] (+)= base0[n] + sum_e ( add0_e[perm_e(n)] + (acc_b - conv_b)_e[perm_e(n)] P^-1 )
//   out1[n] (+)= base1[n] + sum_e (acc_a - conv_a)_e[perm_e(n)] P^-1
// With convsum set, the entries' converted parts are not subtracted one by one:
// convsum = NTT(sum_e sigma_e(conv_e)) (conv_e in coefficient form, sigma_e the
// coefficient-domain automorphism) is subtracted once, which equals
// sum_e perm_e(NTT(conv_e)) because the NTT and the automorphism are linear.
struct SumEntry {
    const u64* acc;   // [2][l+1+k][N]
    const u64* conv;  // [2][l+1][N]: NTT form (per-entry path) or coefficient form (convsum path)
    const u64* add0;  // [l+1][N] (c0 of the rotated ciphertext)
    uint32_t galois;
    uint32_t galois_inv;  // g^-1 mod 2N
};
struct SumItem {
    u64* out;            // [2][l+1][N]
    const u64* base;     // [2][l+1][N] or null
    int e0, n_e;
    int accumulate;
    const u64* convsum;  // [2][l+1][N] NTT form, or null
};

// Double hoisting: a rotated copy kept on the key-switching basis Q_l * P,
//   out = sigma_g((P c0, 0) + acc)   (acc: key inner product [2][l+1+k][N], ct: [2][l+1][N]),
// or, with acc = null and galois = 1, the lift (P c0, P c1) of ct (zero on the
// special limbs).  out: [2][l+1+k][N], NTT form.
struct LiftItem {
    const u64* acc;
    const u64* ct;
    u64* out;
    uint32_t galois;
};
// n_acc: items with an accumulator (-1 = all), n_sources: distinct source
// ciphertexts (0 = every item its own); both for the profiler's byte count
void launch_lift(fe_ctx* c, const LiftItem* items_dev, int n_items, int level, cudaStream_t st, int n_acc = -1,
                 int n_sources = 0);

// PMult-MAC item: up to kMacWays outputs whose term lists read the same
// ciphertexts in the same order, out[k] = sum_t ct_t (x) pt_{k,t} with
// ct_t = terms[term0[0] + t].ct and pt_{k,t} = terms[term0[k] + t].pt, so each
// ciphertext word is loaded once for all of them.
constexpr int kMacWays = 4;
struct MacItem {
    u64* out[kMacWays];  // [2][l+1][N] each
    int term0[kMacWays];
    int n_terms, n_out;
};
// Plan plaintexts are stored compactly, limb by limb, each limb as N / T tiles
// of T = pt_tile(c) residues: the T low 32-bit words, then the T high parts of
// c->pt_hb bytes each, so one limb takes (4 + pt_hb) N bytes and the PMult-MAC
// fetches a tile with one bulk copy.
struct MacTerm {
    const u64* ct;      // [2][l+1][N]
    const uint8_t* pt;  // compact plaintext, l+1 limbs
};
// PMult-MAC whose terms are rotated copies made on the fly (double hoisting with
// one output per item: depthwise layers).  A rotated term is sigma_g((P c0, 0) +
// acc) read straight from the key inner product's accumulators and the input's
// lifted copy (P c0, P c1); an unrotated term is the lifted copy itself.
struct RotTerm {
    const u64* acc;     // [2][l+1+k][N] key inner product of the rotation, or nullptr
    const u64* xp;      // [2][l+1+k][N] lifted input (P c0, P c1)
    const uint8_t* pt;  // compact plaintext, l+1+k limbs
    uint32_t galois;    // 1 for an unrotated term
};
struct RotItem {
    u64* out;  // [2][l+1+k][N]
    int term0, n_terms;
};
// n_acc_terms: terms with an accumulator (the profiler's byte count)
void launch_mac_rot(fe_ctx* c, const RotItem* items_dev, const RotTerm* terms_dev, int n_items, int n_terms,
                    int n_acc_terms, int level, cudaStream_t st);
inline size_t pt_limb_bytes(const fe_ctx* c) { return (size_t)(4 + c->pt_hb) * c->N; }
inline int pt_tile(const fe_ctx* c) { return c->N < 512 ? c->N : 512; }
// n_limbs 64-bit limbs [n_limbs][N] -> compact limbs
void launch_pt_compact(fe_ctx* c, const u64* in, uint8_t* out, int n_limbs, cudaStream_t st);
// out (+)= ct (x) pt for one ciphertext at `level` and a compact plaintext
void launch_pmult_compact(fe_ctx* c, const u64* ct, const uint8_t* pt, u64* out, int level, bool accumulate,
                          cudaStream_t st);

// Base conversion of n_poly polynomials: source modulus src[i] is read at position
// ext_pos(src[i]) - in_pos_base of an input polynomial (stride in_stride words),
// destination dst[d] is written at position ext_pos(dst[d]) of an output polynomial;
// copy_src also copies the source limbs to their output positions.
void launch_bconv(fe_ctx* c, const BConvTab& t, int level, const u64* in, size_t in_stride,
                  int in_pos_base, u64* out, size_t out_stride, int n_poly, bool copy_src,
                  cudaStream_t st);
void launch_keyip(fe_ctx* c, const KsItem* items_dev, int n_items, int level, cudaStream_t st);
// n_sources: distinct digit arrays among the items (for the profiler's byte
// count; 0 = every item its own)
void launch_keyip_grouped(fe_ctx* c, const KsGroup* groups_dev, const KsItem* items_dev,
                          int n_groups, int n_items, int level, cudaStream_t st, int n_sources = 0);
void launch_combine(fe_ctx* c, const CombineItem* items_dev, int n_items, int level,
                    cudaStream_t st);
void launch_combine_sum(fe_ctx* c, const SumItem* items_dev, const SumEntry* entries_dev,
                        int n_items, int n_entries, int level, cudaStream_t st);
// convsum_i = sum over item i's entries of sigma_e(conv_e) in the coefficient domain
// (out + i * 2 (l+1) N words)
void launch_autosum(fe_ctx* c, const SumItem* items_dev, const SumEntry* entries_dev, int n_items,
                    int n_entries, u64* out, int level, cudaStream_t st);
// n_ct_terms: ciphertext loads (sum of n_terms over items); n_pt_terms: plaintext
// loads (sum of n_terms x n_out); n_outputs: outputs written; ways: the largest
// n_out of the items (1, 2 or 4 selects the kernel)
// qp: operands on the key-switching basis Q_level * P (l+1+k limbs, ciphertext
// polynomials [2][l+1+k][N], plaintexts [l+1+k][N]) instead of Q_level
// n_ct_distinct: distinct ciphertexts among the terms (for the profiler's byte
// count; 0 = every ciphertext load counted)
void launch_mac(fe_ctx* c, const MacItem* items_dev, const MacTerm* terms_dev, int n_items,
                int n_ct_terms, int n_pt_terms, int n_outputs, int ways, int level, cudaStream_t st,
                bool qp = false, int n_ct_distinct = 0);
void launch_rescale_combine(fe_ctx* c, const u64* in, const u64* lift, u64* out, int n_ct,
                            int level, cudaStream_t st);
// out_j = (acc_j - conv_j) (q_l P)^-1 on q_0..q_{l-1} for n items (see moddown_rescale)
void launch_mdrs_combine(fe_ctx* c, const u64* acc, const u64* conv, u64* const* outs_dev, int n, int level,
                         cudaStream_t st);
void launch_add(fe_ctx* c, const u64* a, const u64* b, u64* out, int n_ct, int level,
                cudaStream_t st);
void launch_pmult(fe_ctx* c, const u64* ct, const u64* pt, u64* out, int n_ct, int level,
                  bool accumulate, cudaStream_t st);
void launch_tensor(fe_ctx* c, const u64* x, const u64* y, u64* d012, int n_ct, int level,
                   cudaStream_t st);

// sampling (counter-based SplitMix64 words)
void launch_sample_uniform_limbs(fe_ctx* c, uint64_t seed, uint64_t tag_base, u64* out,
                                 int n_limbs, const int* mod_idx_dev, cudaStream_t st);
void launch_sample_signed(fe_ctx* c, uint64_t seed, uint64_t tag, int kind, i64* out,
                          cudaStream_t st);
void launch_signed_to_limbs(fe_ctx* c, const i64* v, u64* out, int first_mod, int n_limbs,
                            size_t out_stride_words, cudaStream_t st);

}  // namespace fe
