// Batched scheme operations used by the layer code.
#pragma once

#include "kernels.cuh"

namespace fe {

// random-stream addresses of the generator: tag = kind << 56 | object << 24 | digit << 8 | limb
enum : uint64_t { kTagSk = 1, kTagCtA = 2, kTagCtE = 3, kTagKeyA = 4, kTagKeyE = 5 };
inline uint64_t make_tag(uint64_t kind, uint64_t obj, uint64_t digit, uint64_t limb) {
    return (kind << 56) | (obj << 24) | (digit << 8) | limb;
}

inline int dnum_at(const fe_ctx* c, int level) { return (level + 1 + c->k - 1) / c->k; }
inline size_t ext_words(const fe_ctx* c, int level) {
    return (size_t)dnum_at(c, level) * (level + 1 + c->k) * c->N;
}
inline size_t acc_words(const fe_ctx* c, int level) { return 2 * (size_t)(level + 1 + c->k) * c->N; }
inline size_t ct_words(const fe_ctx* c, int level) { return 2 * (size_t)(level + 1) * c->N; }

// ModUp of n polynomials at `level` (each l+1 limbs, NTT form, poly stride src_stride words):
// coef receives their inverse NTTs ([n][l+1][N]); ext receives the extended digits
// ([n][dnum][l+1+k][N], NTT form).
void modup(fe_ctx* c, const u64* src, size_t src_stride, int n, int level, u64* coef, u64* ext,
           cudaStream_t st);
// Rotations of n_ct ciphertexts at `level` by each of n_steps steps with one
// ModUp per ciphertext for all steps: out holds [n_steps][n_ct] ciphertexts,
// each the residues fe_rotate gives (the key switch precedes the
// automorphism, so the extended digits of c1 serve every step).  Scratch from
// the stream-ordered allocator; steps are taken in chunks whose accumulators
// fit 4 GB.  Errors: FE_EKEY (a missing key), FE_ENOMEM, FE_ECUDA.
int rotate_many(fe_ctx* c, const fe_evk* evk, const u64* in, int n_ct, int level, const int32_t* steps,
                int n_steps, u64* out, cudaStream_t st);
// ModDown preparation for n accumulators acc [n][2][l+1+k][N] (NTT form): the P limbs are
// inverse-transformed in place, converted to Q_level into conv [n][2][l+1][N] and transformed.
void moddown_prepare(fe_ctx* c, u64* acc, int n, int level, u64* conv, cudaStream_t st);
// the same without the final NTT: conv receives the conversion in coefficient form
void moddown_to_coef(fe_ctx* c, u64* acc, int n, int level, u64* conv, cudaStream_t st);
// ModDown and rescale in one division by q_l P for n accumulators acc
// [n][2][l+1+k][N] (NTT form; the q_l and P limbs are inverse-transformed in
// place): the centred conversion of [acc]_{q_l P} to q_0..q_{l-1} into conv
// [n][2][l][N], then outs_dev[j] = (acc_j - conv_j) (q_l P)^-1 ([2][l][N]).
void moddown_rescale(fe_ctx* c, u64* acc, int n, int level, u64* conv, u64* const* outs_dev, cudaStream_t st);
// Rescale n ciphertexts in -> out (level -> level - 1); tmp: [2n][N], lift: [2n][level][N].
void rescale_batch(fe_ctx* c, const u64* in, int n, int level, u64* out, u64* tmp, u64* lift,
                   cudaStream_t st);
size_t rescale_tmp_words(const fe_ctx* c, int n, int level);

const u64* evk_key(const fe_evk* evk, uint32_t galois);

// d = relin(x (x) y) for n pairs of ciphertexts at `level` (CMult with
// relinearisation, no rescale); scratch carved from cv (cmult_relin_bytes).
int cmult_relin(fe_ctx* c, const fe_evk* evk, const u64* x, const u64* y, int n, int level, u64* d, Carver& cv,
                cudaStream_t st);
size_t cmult_relin_bytes(const fe_ctx* c, int n, int level);
// d = relin of n ciphertext products (d0, d1, d2) [n][3][level+1][N] (as
// launch_tensor leaves them, or sums of them): (d0, d1) + KS(d2); scratch
// carved from cv (relin_tensors_bytes)
int relin_tensors(fe_ctx* c, const fe_evk* evk, const u64* d012, int n, int level, u64* d, Carver& cv,
                  cudaStream_t st);
size_t relin_tensors_bytes(const fe_ctx* c, int n, int level);

// Per-limb constants of an affine map of ciphertexts (polynomial activation,
// integer products and constants of the bootstrapping's EvalMod).
constexpr int kMaxAffineLimbs = 64;
struct AffineConsts {
    u64 mul[kMaxAffineLimbs];  // factor per limb (both polynomials)
    u64 add[kMaxAffineLimbs];  // constant per limb (c0 only: a constant message term)
};
// out = in * mul_i (+ add_i on c0) for n ciphertexts at `level` (do_mul false: add only)
int launch_affine(fe_ctx* c, const u64* in, u64* out, int n, int level, const AffineConsts& k, bool do_mul,
                  cudaStream_t st);
// the integer nearest to x, ties away from zero, reduced mod q (any finite x)
u64 nearest_mod(double x, u64 q);

// the bytes of a host table carried to dst by kernel parameters (pieces of
// 2 KB, one launch each)
int copy_by_params(void* dst, const void* src, size_t bytes, cudaStream_t st);

// copy a per-call host table into device memory on `st`.  The source is
// ordinary (pageable) host memory that the caller frees on return, so a
// stream capture must not record it as a copy: the replay would read freed
// memory.  Under capture the table goes by kernel parameters instead, which
// the graph keeps by value.
inline int copy_host_table(void* dst, const void* src, size_t bytes, cudaStream_t st) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    FE_CUDA_TRY(cudaStreamIsCapturing(st, &cs));
    if (cs != cudaStreamCaptureStatusNone) return copy_by_params(dst, src, bytes, st);
    FE_CUDA_TRY(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st));
    return FE_OK;
}

// upload a host vector into a device region carved from a workspace
template <class T>
int upload(const std::vector<T>& v, T* dst, cudaStream_t st) {
    if (v.empty()) return FE_OK;
    return copy_host_table(dst, v.data(), v.size() * sizeof(T), st);
}

}  // namespace fe
