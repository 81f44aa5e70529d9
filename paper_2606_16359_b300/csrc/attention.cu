// Attention products of the transformer extension (Sec. 7) on fragmented
// token embeddings (fe_token_layout: element f S + s of token t in ciphertext s,
// slot f n + t).  The token-wise aggregation the paper names for Q K^T and A V
// is done with token-wise rotations: every position block of n token slots is
// rotated by r tokens as M_lo (x) Rot(x, r) + M_hi (x) Rot(x, r - n), the masks
// selecting the tokens t < n - r and t >= n - r, encoded at a power of two
// (their coefficients are rationals with denominators dividing N: at 2^k >= N
// none falls on a rounding tie, as one can at a prime scale).
//
// These layers are composed from the library's primitives (rotation, PMult,
// addition, CMult with relinearisation, rescale) in a fixed order, so that
// their residues equal the oracle's step for step.  Each call encodes the
// 2 (n - 1) token masks once, runs every token rotation, product and rescale
// on the S ciphertexts together and the position sums on all n score
// diagonals together; per ciphertext the steps are those of the oracle.
// Scratch comes from the stream-ordered allocator.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "ops.h"

extern "C" int fe_rotate(fe_ctx* c, const fe_evk* evk, const void* ct_dev, uint32_t n_ct, uint32_t level,
                         int32_t r, void* out_dev, void* stream);
extern "C" int fe_encode(fe_ctx* c, const double* slots_dev, uint32_t n, uint32_t level, double scale, void* pt_dev,
                         void* stream);
extern "C" int fe_pmult(fe_ctx* c, const void* ct_dev, const void* pt_dev, uint32_t n_ct, uint32_t level,
                        void* out_dev, void* stream);
extern "C" int fe_add(fe_ctx* c, const void* a_dev, const void* b_dev, uint32_t n_ct, uint32_t level, void* out_dev,
                      void* stream);
extern "C" int fe_rescale(fe_ctx* c, const void* ct_dev, uint32_t n_ct, uint32_t level, void* out_dev,
                          void* stream);
extern "C" int fe_token_layout_make(const fe_ctx* c, fe_token_layout* t);

namespace fe {
namespace {
constexpr int kB = 256;

// slot l -> 1 when its token (l mod n) is below n - r (lo) / at or above it (hi)
__global__ void k_token_mask(double* lo, double* hi, int n, int r, int half) {
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= half) return;
    const bool below = (l % n) < n - r;
    lo[l] = below ? 1.0 : 0.0;
    hi[l] = below ? 0.0 : 1.0;
}

// out = in times the per-limb constant k[i] (both polynomials), n ciphertexts at `level`
__global__ void k_mul_const(const u64* in, u64* out, const Modulus* mods, const u64* k, int nl, int logN) {
    const int N = 1 << logN;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= N) return;
    const int limb = blockIdx.y, ci = blockIdx.z;  // limb over 2 nl
    const int i = limb % nl;
    const size_t o = ((size_t)ci * 2 * nl + limb) * N + x;
    out[o] = mul_mod(in[o], k[i], mods[i]);
}

// first l limbs of each polynomial of n ciphertexts at level l (modulus dropped to Q_{l-1})
__global__ void k_drop_limb(const u64* in, u64* out, int nl_in, int logN) {
    const int N = 1 << logN;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= N) return;
    const int nl_out = nl_in - 1;
    const int limb = blockIdx.y, ci = blockIdx.z;  // limb over 2 nl_out
    const int poly = limb / nl_out, i = limb % nl_out;
    out[(((size_t)ci * 2 + poly) * nl_out + i) * N + x] = in[(((size_t)ci * 2 + poly) * nl_in + i) * N + x];
}

struct Dev {
    void* p = nullptr;
    cudaStream_t st;
    explicit Dev(cudaStream_t s) : st(s) {}
    ~Dev() {
        if (p) cudaFreeAsync(p, st);
    }
    template <class T>
    T* get(size_t count) {
        if (cudaMallocAsync(&p, std::max<size_t>(count * sizeof(T), 16), st) != cudaSuccess) {
            p = nullptr;
            (void)cudaGetLastError();  // the caller reports FE_ENOMEM; nothing stays pending
            return nullptr;
        }
        return (T*)p;
    }
};

double mask_scale_pow2(const fe_ctx* c, int level) {
    return std::ldexp(1.0, 63 - __builtin_clzll(c->mod[level]));
}

// out = x with its last limb dropped (n ciphertexts at `level`)
int drop_limb(fe_ctx* c, const u64* x, int n, int level, u64* out, cudaStream_t st) {
    k_drop_limb<<<dim3((c->N + kB - 1) / kB, 2 * level, n), kB, 0, st>>>(x, out, level + 1, c->logN);
    c->cnt.launches++;
    FE_CUDA_TRY(cudaGetLastError());
    return FE_OK;
}

// out = a + b over rows of N residues, row r modulo q_(r mod nl) (products
// (d0, d1, d2) of level nl - 1 laid out [..][3][nl][N], summed before one
// relinearisation)
__global__ void k_add_rows(const u64* a, const u64* b, u64* out, const Modulus* mods, int nl, int logN) {
    const int N = 1 << logN;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= N) return;
    const size_t o = (size_t)blockIdx.y * N + x;
    out[o] = add_mod(a[o], b[o], mods[blockIdx.y % nl].q);
}
int add_rows(fe_ctx* c, const u64* a, const u64* b, u64* out, int rows, int nl, cudaStream_t st) {
    k_add_rows<<<dim3((c->N + kB - 1) / kB, rows), kB, 0, st>>>(a, b, out, c->d_mod, nl, c->logN);
    c->cnt.launches++;
    FE_CUDA_TRY(cudaGetLastError());
    return FE_OK;
}

// out = M_lo (x) a + M_hi (x) b per limb for n ciphertexts (both masks shared):
// the two PMults and the addition of a token rotation in one pass
__global__ void k_mask_pair(const u64* a, const u64* b, const u64* mlo, const u64* mhi, u64* out,
                            const Modulus* mods, int nl, int logN) {
    const int N = 1 << logN;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= N) return;
    const int limb = blockIdx.y, ci = blockIdx.z;  // limb over 2 nl
    const int i = limb % nl;
    const Modulus m = mods[i];
    const size_t o = ((size_t)ci * 2 * nl + limb) * N + x, mo = (size_t)i * N + x;
    out[o] = add_mod(mul_mod(a[o], mlo[mo], m), mul_mod(b[o], mhi[mo], m), m.q);
}

// The token masks of every r = 1 .. n - 1 at `level`, encoded once per call:
// plaintext 2 (r - 1) selects the tokens t < n - r, 2 (r - 1) + 1 the others.
struct TokenMasks {
    Dev buf;
    u64* pts = nullptr;
    size_t pt_words = 0;
    explicit TokenMasks(cudaStream_t st) : buf(st) {}
    const u64* lo(int r) const { return pts + (size_t)(2 * (r - 1)) * pt_words; }
    const u64* hi(int r) const { return pts + (size_t)(2 * (r - 1) + 1) * pt_words; }
};
int make_token_masks(fe_ctx* c, const fe_token_layout& T, int level, double ms, TokenMasks& M, cudaStream_t st) {
    const int half = c->N / 2, n = (int)T.n_tok;
    if (n < 2) return FE_OK;
    const size_t n_pt = 2 * (size_t)(n - 1);
    M.pt_words = (size_t)(level + 1) * c->N;
    M.pts = M.buf.get<u64>(n_pt * M.pt_words);
    Dev sb(st);
    double* slots = sb.get<double>(n_pt * half);
    if (!M.pts || !slots) return fail(FE_ENOMEM, "token mask scratch");
    for (int r = 1; r < n; r++) {
        double* lo = slots + (size_t)(2 * (r - 1)) * half;
        k_token_mask<<<(half + kB - 1) / kB, kB, 0, st>>>(lo, lo + half, n, r, half);
        c->cnt.launches++;
    }
    FE_CUDA_TRY(cudaGetLastError());
    return fe_encode(c, slots, (uint32_t)n_pt, (uint32_t)level, ms, M.pts, st);
}

// Token-wise rotation of n ciphertexts at `level` by r tokens (one level):
// out (level - 1) = rescale(M_lo (x) Rot(x, r) + M_hi (x) Rot(x, r - n)).
// r = 0: rescale(x times the integer ms), token_rotate0 (tmp: n ciphertexts at
// `level` plus level + 1 words); r > 0: token_rotations below.
int token_rotate0(fe_ctx* c, const u64* x, int n_ct, int level, double ms, u64* tmp, u64* out, cudaStream_t st) {
    const dim3 grid((c->N + kB - 1) / kB, 2 * (level + 1), n_ct);
    std::vector<u64> kh(level + 1);
    const u64 m = (u64)ms;  // a power of two below the modulus
    for (int i = 0; i <= level; i++) kh[i] = m % c->mod[i];
    u64* k = tmp + n_ct * ct_words(c, level);  // the per-limb constants
    FE_TRY(copy_host_table(k, kh.data(), kh.size() * 8, st));
    k_mul_const<<<grid, kB, 0, st>>>(x, tmp, c->d_mod, k, level + 1, c->logN);
    c->cnt.launches++;
    FE_CUDA_TRY(cudaGetLastError());
    return fe_rescale(c, tmp, n_ct, level, out, st);
}

// Every token rotation of n_ct ciphertexts x at `level`, r = 0 .. n - 1, in
// order, a chunk of r values at a time: the rotations by r and r - n hoisted
// together into rb (2 chunk n_ct ciphertexts), each r's masks applied with the
// result compacted in place to the front of rb (result i overwrites rotated
// copies that results before it already consumed), and one rescale of the
// chunk into kr (chunk n_ct ciphertexts at level - 1, [r][ct]); then
// use(r0, rn, kr) for r = r0 .. r0 + rn - 1.  r = 0 comes alone.
template <class Use>
int token_rotations(fe_ctx* c, const fe_evk* evk, const fe_token_layout& T, const u64* x, int n_ct, int level,
                    double ms, const TokenMasks& M, int chunk, u64* rb, u64* tmp, u64* kr, Use&& use,
                    cudaStream_t st) {
    const int n = (int)T.n_tok;
    const size_t ctw = ct_words(c, level);
    FE_TRY(token_rotate0(c, x, n_ct, level, ms, tmp, kr, st));
    FE_TRY(use(0, 1, kr));
    std::vector<int32_t> steps;
    const dim3 grid((c->N + kB - 1) / kB, 2 * (level + 1), n_ct);
    for (int r0 = 1; r0 < n; r0 += chunk) {
        const int rn = std::min(chunk, n - r0);
        steps.clear();
        for (int r = r0; r < r0 + rn; r++) {
            steps.push_back(r);
            steps.push_back(r - n);
        }
        FE_TRY(rotate_many(c, evk, x, n_ct, level, steps.data(), 2 * rn, rb, st));
        for (int i = 0; i < rn; i++) {
            const u64* a = rb + (size_t)(2 * i) * n_ct * ctw;
            k_mask_pair<<<grid, kB, 0, st>>>(a, a + n_ct * ctw, M.lo(r0 + i), M.hi(r0 + i), rb + (size_t)i * n_ct * ctw,
                                            c->d_mod, level + 1, c->logN);
            c->cnt.launches++;
            c->cnt.pmult += 2 * n_ct;
        }
        FE_CUDA_TRY(cudaGetLastError());
        FE_TRY(fe_rescale(c, rb, (uint32_t)(rn * n_ct), level, kr, st));
        FE_TRY(use(r0, rn, kr));
    }
    return FE_OK;
}

// r values per hoisted chunk: the rotated copies (2 chunk n_ct ciphertexts) within 2 GB
int rotation_chunk(const fe_ctx* c, int n_tok, int n_ct, int level) {
    const size_t per_r = 2 * (size_t)n_ct * ct_words(c, level) * 8;
    return (int)std::max<size_t>(1, std::min<size_t>(std::max(1, n_tok - 1), (2ull << 30) / per_r));
}

// acc += Rot(acc, 2^k n) for k = 0 .. log2(P) - 1, n_ct ciphertexts at `level`
// (rot: n_ct ciphertexts of scratch)
int position_sum(fe_ctx* c, const fe_evk* evk, const fe_token_layout& T, u64* acc, int n_ct, int level, u64* rot,
                 cudaStream_t st) {
    for (uint32_t step = T.n_tok; step < (uint32_t)c->N / 2; step *= 2) {
        FE_TRY(fe_rotate(c, evk, acc, n_ct, level, (int32_t)step, rot, st));
        FE_TRY(fe_add(c, acc, rot, n_ct, level, acc, st));
    }
    return FE_OK;
}

int check_common(fe_ctx* c, const fe_evk* evk, const fe_token_layout* lay, fe_token_layout* T) {
    if (!c || !evk || !lay) return fail(FE_EINVAL, "null argument");
    if (!evk->relin) return fail(FE_EKEY, "no relinearisation key");
    *T = *lay;
    FE_TRY(fe_token_layout_make(c, T));
    for (uint32_t r = 1; r < T->n_tok; r++)
        for (int32_t s : {(int32_t)r, (int32_t)r - (int32_t)T->n_tok})
            if (!evk_key(evk, c->galois(s))) return fail(FE_EKEY, "missing rotation key for step " + std::to_string(s));
    for (uint32_t step = T->n_tok; step < (uint32_t)c->N / 2; step *= 2)
        if (!evk_key(evk, c->galois((int32_t)step)))
            return fail(FE_EKEY, "missing rotation key for step " + std::to_string(step));
    return FE_OK;
}
}  // namespace
}  // namespace fe

using namespace fe;

extern "C" int fe_attention_rotation_steps(const fe_ctx* c, const fe_token_layout* lay, int32_t* steps, uint32_t max,
                                           uint32_t* n_steps) {
    if (!c || !lay || !n_steps) return fail(FE_EINVAL, "null argument");
    fe_token_layout T = *lay;
    FE_TRY(fe_token_layout_make(c, &T));
    std::vector<int32_t> v;
    for (int32_t r = 1; r < (int32_t)T.n_tok; r++) {
        v.push_back(r - (int32_t)T.n_tok);
        v.push_back(r);
    }
    for (uint32_t step = T.n_tok; step < (uint32_t)c->N / 2; step *= 2) v.push_back((int32_t)step);
    std::sort(v.begin(), v.end());
    v.erase(std::unique(v.begin(), v.end()), v.end());
    *n_steps = (uint32_t)v.size();
    if (steps)
        for (size_t i = 0; i < v.size() && i < max; i++) steps[i] = v[i];
    return FE_OK;
}

extern "C" int fe_he_attention_scores(fe_ctx* c, const fe_evk* evk, const fe_token_layout* lay, const void* q_dev,
                                      const void* k_dev, uint32_t level, double q_scale, double k_scale,
                                      void* out_dev, double* out_scale, void* stream) {
    fe_token_layout T;
    FE_TRY(check_common(c, evk, lay, &T));
    if (!q_dev || !k_dev || !out_dev) return fail(FE_EINVAL, "null argument");
    FE_ALIGNED(q_dev);
    FE_ALIGNED(k_dev);
    FE_ALIGNED(out_dev);
    if (level < 2 || (int)level > c->L) return fail(FE_ELEVEL, "the attention scores need two levels");
    cudaStream_t st = (cudaStream_t)stream;
    const int lv = (int)level, n = (int)T.n_tok, S = (int)T.n_ct;
    const double ms = mask_scale_pow2(c, lv);
    const size_t ctw = ct_words(c, lv), ctw1 = ct_words(c, lv - 1), ctw2 = ct_words(c, lv - 2);
    TokenMasks M(st);
    FE_TRY(make_token_masks(c, T, lv, ms, M, st));
    const int chunk = rotation_chunk(c, n, S, lv);
    const size_t cw = (size_t)chunk * S * ctw1;             // one chunk's ciphertexts at lv - 1
    const size_t tw = 3 * (size_t)lv * c->N;                 // one product (d0, d1, d2) at lv - 1
    const size_t rl_bytes = relin_tensors_bytes(c, chunk, lv - 1);
    Dev wb(st), tb(st), cb(st), rb(st), hb(st), pb(st);
    u64* work = wb.get<u64>(2 * cw + (size_t)chunk * ctw1);  // Q copies, rotated K, relinearised sums
    u64* tmp = tb.get<u64>(S * ctw + 2 * c->N);              // token rotation scratch (r = 0)
    char* rl = cb.get<char>(rl_bytes);                       // relinearisation scratch
    u64* rot = rb.get<u64>((size_t)n * ctw2);                // position-sum scratch
    u64* hoist = hb.get<u64>(2 * (size_t)chunk * S * ctw);   // hoisted rotations of K
    u64* prods = pb.get<u64>(((size_t)chunk * S + chunk) * tw);  // products, their sums per r
    if (!work || !tmp || !rl || !rot || !hoist || !prods) return fail(FE_ENOMEM, "attention scratch");
    u64 *qrep = work, *kr = work + cw, *rel = work + 2 * cw;
    u64 *t3 = prods, *sum3 = prods + (size_t)chunk * S * tw;
    // Q with one limb dropped, once per r of a chunk
    FE_TRY(drop_limb(c, (const u64*)q_dev, S, lv, qrep, st));
    for (int i = 1; i < chunk; i++)
        FE_CUDA_TRY(cudaMemcpyAsync(qrep + (size_t)i * S * ctw1, qrep, (size_t)S * ctw1 * 8, cudaMemcpyDeviceToDevice,
                                    st));
    // diagonal r: the S products Q_s (x) K_s rotated by r tokens, summed, one
    // relinearisation, rescaled (a chunk of r values at once); then every
    // diagonal's position sums
    auto diagonals = [&](int r0, int rn, const u64* krr) -> int {
        launch_tensor(c, qrep, krr, t3, rn * S, lv - 1, st);
        const u64* sums = t3;
        if (S > 1) {
            for (int i = 0; i < rn; i++) {
                const u64* p = t3 + (size_t)i * S * tw;
                u64* a = sum3 + (size_t)i * tw;
                FE_TRY(add_rows(c, p, p + tw, a, 3 * lv, lv, st));
                for (int q = 2; q < S; q++) FE_TRY(add_rows(c, a, p + q * tw, a, 3 * lv, lv, st));
            }
            sums = sum3;
        }
        Carver cv(rl, rl_bytes);
        FE_TRY(relin_tensors(c, evk, sums, rn, lv - 1, rel, cv, st));
        c->cnt.cmult += rn * S;
        return fe_rescale(c, rel, (uint32_t)rn, lv - 1, (u64*)out_dev + (size_t)r0 * ctw2, st);
    };
    FE_TRY(token_rotations(c, evk, T, (const u64*)k_dev, S, lv, ms, M, chunk, hoist, tmp, kr, diagonals, st));
    FE_TRY(position_sum(c, evk, T, (u64*)out_dev, n, lv - 2, rot, st));
    // scales as the operations change them: K rotated (k ms) / q_l, product q (.),
    // rescale by q_{l-1}
    const double kr_scale = (k_scale * ms) / (double)c->mod[lv];
    if (out_scale) *out_scale = (q_scale * kr_scale) / (double)c->mod[lv - 1];
    FE_CUDA_TRY(cudaGetLastError());
    return FE_OK;
}

extern "C" int fe_he_attention_apply(fe_ctx* c, const fe_evk* evk, const fe_token_layout* lay, const void* d_dev,
                                     uint32_t d_level, double d_scale, const void* v_dev, uint32_t v_level,
                                     double v_scale, void* out_dev, uint32_t* out_level, double* out_scale,
                                     void* stream) {
    fe_token_layout T;
    FE_TRY(check_common(c, evk, lay, &T));
    if (!d_dev || !v_dev || !out_dev) return fail(FE_EINVAL, "null argument");
    FE_ALIGNED(d_dev);
    FE_ALIGNED(v_dev);
    FE_ALIGNED(out_dev);
    if (v_level < 1 || (int)v_level > c->L || d_level < 1 || (int)d_level > c->L)
        return fail(FE_ELEVEL, "level out of range");
    cudaStream_t st = (cudaStream_t)stream;
    const int vl = (int)v_level, dl = (int)d_level, n = (int)T.n_tok, S = (int)T.n_ct;
    const int ml = std::min(vl - 1, dl);  // level of the products
    if (ml < 1) return fail(FE_ELEVEL, "the attention output needs a level to rescale");
    const double ms = mask_scale_pow2(c, vl);
    const size_t ctwv = ct_words(c, vl), ctwv1 = ct_words(c, vl - 1), ctwd = ct_words(c, dl),
                 ctwm = ct_words(c, ml);
    TokenMasks M(st);
    FE_TRY(make_token_masks(c, T, vl, ms, M, st));
    const size_t wide = std::max(ctwv1, ctwd);
    const int chunk = rotation_chunk(c, n, S, vl);
    const size_t cs = (size_t)chunk * S;      // ciphertexts of one chunk
    const size_t tw = 3 * (size_t)(ml + 1) * c->N;  // one product (d0, d1, d2) at ml
    const size_t rl_bytes = relin_tensors_bytes(c, S, ml);
    Dev wb(st), tb(st), db(st), cb(st), hb(st), pb(st);
    u64* work = wb.get<u64>(cs * ctwv1 + S * ctwm);               // rotated V, relinearised sums
    u64* tmp = tb.get<u64>(S * ctwv + 2 * c->N);                  // token rotation scratch (r = 0)
    u64* drop = db.get<u64>(2 * cs * wide + cs * ctwm);           // level drops, D_r for every s
    char* rl = cb.get<char>(rl_bytes);                            // relinearisation scratch
    u64* hoist = hb.get<u64>(2 * cs * ctwv);                      // hoisted rotations of V
    u64* prods = pb.get<u64>((cs + S) * tw);                      // products, their sums per s
    if (!work || !tmp || !drop || !rl || !hoist || !prods) return fail(FE_ENOMEM, "attention scratch");
    u64 *vr = work, *rel = work + cs * ctwv1;
    u64 *bx = drop, *by = drop + cs * wide, *drep = drop + 2 * cs * wide;
    u64 *t3 = prods, *acc3 = prods + cs * tw;
    // output s: the n products D_r (x) V_s rotated by r tokens summed over r
    // (a chunk of r values at once), one relinearisation, rescaled once
    auto terms = [&](int r0, int rn, const u64* vrr) -> int {
        // D_r dropped to the products' level (one limb at a time), one copy per s
        for (int i = 0; i < rn; i++) {
            const u64* x = (const u64*)d_dev + (size_t)(r0 + i) * ctwd;
            for (int l = dl; l > ml; l--) {
                u64* dst = (x == bx) ? by : bx;
                FE_TRY(drop_limb(c, x, 1, l, dst, st));
                x = dst;
            }
            for (int q = 0; q < S; q++)
                FE_CUDA_TRY(cudaMemcpyAsync(drep + ((size_t)i * S + q) * ctwm, x, ctwm * 8, cudaMemcpyDeviceToDevice,
                                            st));
        }
        // the rotated V of the chunk dropped the same way
        const u64* y = vrr;
        for (int l = vl - 1; l > ml; l--) {
            u64* dst = (y == bx) ? by : bx;
            FE_TRY(drop_limb(c, y, rn * S, l, dst, st));
            y = dst;
        }
        launch_tensor(c, drep, y, t3, rn * S, ml, st);
        for (int i = 0; i < rn; i++) {
            const u64* p = t3 + (size_t)i * S * tw;
            if (r0 + i == 0)
                FE_CUDA_TRY(cudaMemcpyAsync(acc3, p, (size_t)S * tw * 8, cudaMemcpyDeviceToDevice, st));
            else
                FE_TRY(add_rows(c, acc3, p, acc3, (int)(3 * S * (ml + 1)), ml + 1, st));
        }
        return FE_OK;
    };
    FE_TRY(token_rotations(c, evk, T, (const u64*)v_dev, S, vl, ms, M, chunk, hoist, tmp, vr, terms, st));
    {
        Carver cv(rl, rl_bytes);
        FE_TRY(relin_tensors(c, evk, acc3, S, ml, rel, cv, st));
        c->cnt.cmult += n * S;
    }
    FE_TRY(fe_rescale(c, rel, S, ml, (u64*)out_dev, st));
    const double vr_scale = (v_scale * ms) / (double)c->mod[vl];
    if (out_level) *out_level = (uint32_t)(ml - 1);
    if (out_scale) *out_scale = (d_scale * vr_scale) / (double)c->mod[ml];
    FE_CUDA_TRY(cudaGetLastError());
    return FE_OK;
}
