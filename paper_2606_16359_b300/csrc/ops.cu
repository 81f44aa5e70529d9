// Scheme operations: key generation, encryption, decryption, ModUp / ModDown,
// rotation (Eq. 1), rescale, and the primitive entry points of the C ABI.
#include <algorithm>
#include <cstring>
#include <memory>
#include <set>

#include "ops.h"

namespace fe {

namespace {
constexpr int kB = 256;
inline dim3 grid_for(int N, int y, int z = 1) { return dim3((N + kB - 1) / kB, y, z); }

__device__ __forceinline__ i64 cbd21(u64 w) {
    return (i64)__popcll(w & 0x1FFFFFull) - (i64)__popcll((w >> 21) & 0x1FFFFFull);
}

// b = e - a s_dst + [t in digit] (P mod t) s_src, all NTT form, one digit of one key;
// s_dst[n] = s[perm_{gal_dst}(n)]
__global__ void k_key_b(u64* b, const u64* a, const u64* e, const u64* s_src, const u64* s,
                        uint32_t gal_dst, const u64* pmod, int dig_lo, int dig_hi,
                        const Modulus* mods, int logN) {
    const int N = 1 << logN;
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const int t = blockIdx.y;
    const Modulus m = mods[t];
    const size_t o = ((size_t)t << logN) + n;
    const uint32_t sn = gal_dst == 1 ? (uint32_t)n : galois_perm(n, gal_dst, logN);
    u64 v = sub_mod(e[o], mul_mod(a[o], s[((size_t)t << logN) + sn], m), m.q);
    if (t >= dig_lo && t < dig_hi) v = add_mod(v, mul_mod(pmod[t], s_src[o], m), m.q);
    b[o] = v;
}

__global__ void k_square_limbs(const u64* s, u64* out, const Modulus* mods, int logN) {
    const int N = 1 << logN;
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const size_t o = ((size_t)blockIdx.y << logN) + n;
    out[o] = mul_mod(s[o], s[o], mods[blockIdx.y]);
}

// ciphertext z: c1[t] = uniform (tag CtA(id0 + z, limb t)); e (tag CtE(id0 + z)) signed
__global__ void k_enc_sample(GenKey gk, u64 seed, u64 id0, u64* ct, i64* e, const Modulus* mods, int nl,
                             int logN) {
    const int N = 1 << logN;
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const u64 id = id0 + blockIdx.z;
    const int t = blockIdx.y;
    u64* c1 = ct + ((size_t)blockIdx.z * 2 + 1) * nl * N;
    const u64 w = gen_word(gk, seed, (kTagCtA << 56) | (id << 24) | (u64)t, (u64)n);
    c1[((size_t)t << logN) + n] = (u64)(((u128)w * mods[t].q) >> 64);
    if (t == 0) e[(size_t)blockIdx.z * N + n] = cbd21(gen_word(gk, seed, (kTagCtE << 56) | (id << 24), (u64)n));
}

// c0 = m + e - a s  (m, e NTT form)
__global__ void k_enc_c0(u64* ct, const u64* m, const u64* e, const u64* s, const Modulus* mods, int nl,
                         int logN) {
    const int N = 1 << logN;
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const int t = blockIdx.y, z = blockIdx.z;
    const Modulus md = mods[t];
    const size_t o = ((size_t)t << logN) + n;
    u64* c0 = ct + (size_t)z * 2 * nl * N;
    const u64* c1 = c0 + (size_t)nl * N;
    const size_t mo = (size_t)z * nl * N + o;
    u64 v = add_mod(m[mo], e[mo], md.q);
    c0[o] = sub_mod(v, mul_mod(c1[o], s[o], md), md.q);
}

__global__ void k_signed_rows_to_limbs(const i64* e, u64* out, const Modulus* mods, int nl, int logN) {
    const int N = 1 << logN;
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const int t = blockIdx.y, z = blockIdx.z;
    out[((size_t)z * nl + t) * N + n] = from_signed(e[(size_t)z * N + n], mods[t].q);
}

// m = c0 + c1 s on the first nl2 limbs
__global__ void k_dec_mul(const u64* ct, const u64* s, u64* out, const Modulus* mods, int nl, int nl2,
                          int logN) {
    const int N = 1 << logN;
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const int t = blockIdx.y, z = blockIdx.z;
    const Modulus md = mods[t];
    const size_t o = ((size_t)t << logN) + n;
    const u64* c0 = ct + (size_t)z * 2 * nl * N;
    const u64* c1 = c0 + (size_t)nl * N;
    out[((size_t)z * nl2 + t) * N + n] = add_mod(c0[o], mul_mod(c1[o], s[o], md), md.q);
}

// centred CRT of one or two limbs -> double-double
__global__ void k_crt_dd(const u64* x, double* mdd, u64 q0, u64 q1, u64 q0inv_q1, int nl2, int logN) {
    const int N = 1 << logN;
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const int z = blockIdx.y;
    const u64 x0 = x[((size_t)z * nl2) * N + n];
    i128 v;
    if (nl2 == 1) {
        v = (i128)centre(x0, q0);
    } else {
        const u64 x1 = x[((size_t)z * nl2 + 1) * N + n];
        const u64 x0m = x0 % q1;
        const u64 d = x1 >= x0m ? x1 - x0m : x1 + q1 - x0m;
        const u64 kk = (u64)(((u128)d * q0inv_q1) % q1);
        const u128 Q = (u128)q0 * q1;
        u128 u = (u128)x0 + (u128)q0 * kk;
        v = u > Q / 2 ? (i128)u - (i128)Q : (i128)u;
    }
    const double hi = (double)v;
    const double lo = (double)(v - (i128)hi);
    mdd[2 * ((size_t)z * N + n)] = hi;
    mdd[2 * ((size_t)z * N + n) + 1] = lo;
}

}  // namespace

const u64* evk_key(const fe_evk* evk, uint32_t galois) {
    auto it = evk->rot.find(galois);
    return it == evk->rot.end() ? nullptr : it->second;
}

void modup(fe_ctx* c, const u64* src, size_t src_stride, int n, int level, u64* coef, u64* ext,
           cudaStream_t st) {
    if (n == 0) return;
    const int N = c->N, nl = level + 1, np = level + 1 + c->k, dn = dnum_at(c, level);
    ntt_inverse_from(c, src, src_stride, LimbSet{coef, (size_t)nl * N, nl, n, c->d_identity_map}, st);
    // the converted limbs of every digit, then their forward NTT
    for (int j = 0; j < dn; j++)
        launch_bconv(c, c->lv[level].modup[j], level, coef, (size_t)nl * N, 0, ext + (size_t)j * np * N,
                     (size_t)dn * np * N, n, false, st);
    const LevelTabs& lt = c->lv[level];
    LimbSet others{ext, (size_t)dn * np * N, lt.n_up_ntt, n, lt.d_up_mod, lt.d_up_pos};
    ntt_forward(c, others, st);
    // a digit's own limbs keep the input's NTT-form residues
    for (int j = 0; j < dn; j++) {
        const int lo = j * c->k, cnt = std::min(c->k, nl - lo);
        cudaMemcpy2DAsync(ext + ((size_t)j * np + lo) * N, (size_t)dn * np * N * 8, src + (size_t)lo * N,
                          src_stride * 8, (size_t)cnt * N * 8, n, cudaMemcpyDeviceToDevice, st);
    }
}

void moddown_prepare(fe_ctx* c, u64* acc, int n, int level, u64* conv, cudaStream_t st) {
    if (n == 0) return;
    const int N = c->N, nl = level + 1, np = level + 1 + c->k;
    ntt_inverse(c, LimbSet{acc + (size_t)nl * N, (size_t)np * N, c->k, 2 * n, c->lv[level].d_ks_limbs + nl},
                st);
    BConvTab t = c->moddown;
    t.n_dst = nl;  // destination-major table: the first l+1 destinations
    launch_bconv(c, t, level, acc, (size_t)np * N, 0, conv, (size_t)nl * N, 2 * n, false, st);
    ntt_forward(c, LimbSet{conv, (size_t)nl * N, nl, 2 * n, c->d_identity_map}, st);
}

void moddown_to_coef(fe_ctx* c, u64* acc, int n, int level, u64* conv, cudaStream_t st) {
    if (n == 0) return;
    const int N = c->N, nl = level + 1, np = level + 1 + c->k;
    ntt_inverse(c, LimbSet{acc + (size_t)nl * N, (size_t)np * N, c->k, 2 * n, c->lv[level].d_ks_limbs + nl},
                st);
    BConvTab t = c->moddown;
    t.n_dst = nl;
    launch_bconv(c, t, level, acc, (size_t)np * N, 0, conv, (size_t)nl * N, 2 * n, false, st);
}

void moddown_rescale(fe_ctx* c, u64* acc, int n, int level, u64* conv, u64* const* outs_dev, cudaStream_t st) {
    if (n == 0) return;
    const int N = c->N, np = level + 1 + c->k;
    ntt_inverse(c, LimbSet{acc + (size_t)level * N, (size_t)np * N, c->k + 1, 2 * n, c->lv[level].d_ks_limbs + level},
                st);
    launch_bconv(c, c->lv[level].mdrs, level, acc, (size_t)np * N, 0, conv, (size_t)level * N, 2 * n, false, st);
    ntt_forward(c, LimbSet{conv, (size_t)level * N, level, 2 * n, c->d_identity_map}, st);
    launch_mdrs_combine(c, acc, conv, outs_dev, n, level, st);
    c->cnt.rescale += n;
}

size_t rescale_tmp_words(const fe_ctx* c, int n, int level) {
    return 2 * (size_t)n * c->N + 2 * (size_t)n * level * c->N;
}

void rescale_batch(fe_ctx* c, const u64* in, int n, int level, u64* out, u64* tmp, u64* lift,
                   cudaStream_t st) {
    if (n == 0) return;
    const int N = c->N, nl = level + 1;
    ntt_inverse_from(c, in + (size_t)level * N, (size_t)nl * N, LimbSet{tmp, (size_t)N, 1, 2 * n, c->d_identity_map + level},
                     st);
    launch_bconv(c, c->lv[level].rescale, level, tmp, (size_t)N, level, lift, (size_t)level * N, 2 * n,
                 false, st);
    ntt_forward(c, LimbSet{lift, (size_t)level * N, level, 2 * n, c->d_identity_map}, st);
    launch_rescale_combine(c, in, lift, out, n, level, st);
    c->cnt.rescale += n;
}

int sk_gen(fe_ctx* c, uint64_t seed, u64* sk, cudaStream_t st) {
    i64* s;
    FE_CUDA_TRY(cudaMallocAsync(&s, (size_t)c->N * 8, st));
    launch_sample_signed(c, seed, make_tag(kTagSk, 0, 0, 0), 0, s, st);
    launch_signed_to_limbs(c, s, sk, 0, c->n_mod, (size_t)c->N, st);
    ntt_forward(c, LimbSet{sk, (size_t)c->n_mod * c->N, c->n_mod, 1, c->d_identity_map}, st);
    FE_CUDA_TRY(cudaFreeAsync(s, st));
    FE_CUDA_TRY(cudaGetLastError());
    return FE_OK;
}

// Copies of per-call host tables inside a stream capture: each piece of the
// table travels as a kernel parameter (copied by value when the launch is
// captured), so the graph rewrites the table from its own copy on every replay.
namespace {
constexpr int kParamBytes = 2048;
struct ParamBlock {
    unsigned char b[kParamBytes];
};
__global__ void k_copy_param(unsigned char* dst, ParamBlock p, int n) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = p.b[i];
}
}  // namespace

int copy_by_params(void* dst, const void* src, size_t bytes, cudaStream_t st) {
    const unsigned char* s = (const unsigned char*)src;
    for (size_t off = 0; off < bytes; off += kParamBytes) {
        ParamBlock p;
        const int n = (int)std::min<size_t>(kParamBytes, bytes - off);
        std::memcpy(p.b, s + off, (size_t)n);
        k_copy_param<<<1, 256, 0, st>>>((unsigned char*)dst + off, p, n);
        FE_CUDA_TRY(cudaGetLastError());
    }
    return FE_OK;
}

}  // namespace fe

using namespace fe;

// ---------------------------------------------------------------------------
// C ABI: keys
// ---------------------------------------------------------------------------

extern "C" int fe_sk_gen(fe_ctx* c, uint64_t seed, void* sk_dev, void* stream) {
    FE_ALIGNED(sk_dev);
    if (!c || !sk_dev) return fail(FE_EINVAL, "null argument");
    return sk_gen(c, seed, (u64*)sk_dev, (cudaStream_t)stream);
}

extern "C" size_t fe_evk_bytes(const fe_ctx* c, uint32_t n_steps, int relin) {
    if (!c) return 0;
    return (size_t)(n_steps + (relin ? 1 : 0)) * c->dnum * 2 * c->n_mod * c->N * 8;
}

extern "C" int fe_evk_gen(fe_ctx* c, const void* sk_dev, uint64_t seed, const int32_t* steps,
                          uint32_t n_steps, int relin, void* evk_dev, size_t evk_bytes, void* stream,
                          fe_evk** out) {
    FE_ALIGNED(evk_dev); FE_ALIGNED(sk_dev);
    if (!c || !sk_dev || !evk_dev || !out || (n_steps && !steps)) return fail(FE_EINVAL, "null argument");
    if (evk_bytes < fe_evk_bytes(c, n_steps, relin)) return fail(FE_ENOMEM, "evk buffer too small");
    cudaStream_t st = (cudaStream_t)stream;
    const int N = c->N, nm = c->n_mod;
    std::set<uint32_t> seen;
    for (uint32_t i = 0; i < n_steps; i++) {
        if (steps[i] != FE_STEP_CONJ && steps[i] % (N / 2) == 0)
            return fail(FE_EINVAL, "rotation step is a multiple of N/2");
        if (!seen.insert(c->galois(steps[i])).second) return fail(FE_EINVAL, "duplicate rotation step");
    }
    std::unique_ptr<fe_evk> h(new fe_evk());
    h->ctx = c;
    h->base = (u64*)evk_dev;
    h->relin = nullptr;
    const size_t key_words = (size_t)c->dnum * 2 * nm * N;
    const u64* s = (const u64*)sk_dev;
    std::vector<u64> pmod(nm);
    for (int t = 0; t < nm; t++) {
        u64 P = 1;
        for (int j = 0; j < c->k; j++) P = h_mulmod(P, c->mod[c->L + 1 + j] % c->mod[t], c->mod[t]);
        pmod[t] = P;
    }
    u64 *e_ntt, *s2, *d_pmod;
    i64* e;
    FE_CUDA_TRY(cudaMallocAsync(&e_ntt, (size_t)nm * N * 8, st));
    FE_CUDA_TRY(cudaMallocAsync(&s2, (size_t)nm * N * 8, st));
    FE_CUDA_TRY(cudaMallocAsync(&e, (size_t)N * 8, st));
    FE_CUDA_TRY(cudaMallocAsync(&d_pmod, nm * 8, st));
    FE_CUDA_TRY(cudaMemcpyAsync(d_pmod, pmod.data(), nm * 8, cudaMemcpyHostToDevice, st));
    auto gen = [&](u64* key, uint32_t obj, const u64* s_src, uint32_t gal_dst) {
        for (int j = 0; j < c->dnum; j++) {
            u64* b = key + (size_t)j * 2 * nm * N;
            u64* a = b + (size_t)nm * N;
            launch_sample_uniform_limbs(c, seed, make_tag(kTagKeyA, obj, j, 0), a, nm, c->d_identity_map, st);
            launch_sample_signed(c, seed, make_tag(kTagKeyE, obj, j, 0), 1, e, st);
            launch_signed_to_limbs(c, e, e_ntt, 0, nm, (size_t)N, st);
            ntt_forward(c, LimbSet{e_ntt, (size_t)nm * N, nm, 1, c->d_identity_map}, st);
            int lo = j * c->k, hi = std::min((j + 1) * c->k, c->L + 1);
            k_key_b<<<grid_for(N, nm), kB, 0, st>>>(b, a, e_ntt, s_src, s, gal_dst, d_pmod, lo, hi, c->d_mod,
                                                    c->logN);
            c->cnt.launches++;
        }
    };
    for (uint32_t i = 0; i < n_steps; i++) {
        uint32_t g = c->galois(steps[i]);
        uint32_t g_inv = (uint32_t)h_invmod(g, (u64)2 * N);
        u64* key = h->base + (size_t)i * key_words;
        gen(key, g, s, g_inv);  // switches from s to sigma_{g^-1}(s)
        h->rot[g] = key;
        h->steps.push_back(steps[i]);
    }
    if (relin) {
        k_square_limbs<<<grid_for(N, nm), kB, 0, st>>>(s, s2, c->d_mod, c->logN);
        u64* key = h->base + (size_t)n_steps * key_words;
        gen(key, 0, s2, 1);  // switches from s^2 to s
        h->relin = key;
    }
    cudaFreeAsync(e_ntt, st);
    cudaFreeAsync(s2, st);
    cudaFreeAsync(e, st);
    cudaFreeAsync(d_pmod, st);
    FE_CUDA_TRY(cudaStreamSynchronize(st));
    FE_CUDA_TRY(cudaGetLastError());
    *out = h.release();
    return FE_OK;
}

extern "C" int fe_swk_gen(fe_ctx* c, const void* sk_src, const void* sk_dst, uint64_t seed, uint32_t obj,
                          void* key_dev, size_t key_bytes, void* stream) {
    FE_ALIGNED(sk_src); FE_ALIGNED(sk_dst); FE_ALIGNED(key_dev);
    if (!c || !sk_src || !sk_dst || !key_dev) return fail(FE_EINVAL, "null argument");
    if (key_bytes < fe_evk_bytes(c, 1, 0)) return fail(FE_ENOMEM, "key buffer too small");
    cudaStream_t st = (cudaStream_t)stream;
    const int N = c->N, nm = c->n_mod;
    std::vector<u64> pmod(nm);
    for (int t = 0; t < nm; t++) {
        u64 P = 1;
        for (int j = 0; j < c->k; j++) P = h_mulmod(P, c->mod[c->L + 1 + j] % c->mod[t], c->mod[t]);
        pmod[t] = P;
    }
    u64 *e_ntt, *d_pmod;
    i64* e;
    FE_CUDA_TRY(cudaMallocAsync(&e_ntt, (size_t)nm * N * 8, st));
    FE_CUDA_TRY(cudaMallocAsync(&e, (size_t)N * 8, st));
    FE_CUDA_TRY(cudaMallocAsync(&d_pmod, nm * 8, st));
    FE_CUDA_TRY(cudaMemcpyAsync(d_pmod, pmod.data(), nm * 8, cudaMemcpyHostToDevice, st));
    // b_j = e_j - a_j s_dst + [t in digit j] (P mod t) s_src, the layout of one rotation key
    u64* key = (u64*)key_dev;
    for (int j = 0; j < c->dnum; j++) {
        u64* b = key + (size_t)j * 2 * nm * N;
        u64* a = b + (size_t)nm * N;
        launch_sample_uniform_limbs(c, seed, make_tag(kTagKeyA, obj, j, 0), a, nm, c->d_identity_map, st);
        launch_sample_signed(c, seed, make_tag(kTagKeyE, obj, j, 0), 1, e, st);
        launch_signed_to_limbs(c, e, e_ntt, 0, nm, (size_t)N, st);
        ntt_forward(c, LimbSet{e_ntt, (size_t)nm * N, nm, 1, c->d_identity_map}, st);
        const int lo = j * c->k, hi = std::min((j + 1) * c->k, c->L + 1);
        k_key_b<<<grid_for(N, nm), kB, 0, st>>>(b, a, e_ntt, (const u64*)sk_src, (const u64*)sk_dst, 1, d_pmod, lo,
                                                hi, c->d_mod, c->logN);
        c->cnt.launches++;
    }
    cudaFreeAsync(e_ntt, st);
    cudaFreeAsync(e, st);
    cudaFreeAsync(d_pmod, st);
    FE_CUDA_TRY(cudaStreamSynchronize(st));
    FE_CUDA_TRY(cudaGetLastError());
    return FE_OK;
}

extern "C" int fe_evk_upload(fe_ctx* c, const void* evk_host, size_t evk_host_bytes, const int32_t* steps,
                             uint32_t n_steps, int relin, void* evk_dev, size_t evk_dev_bytes, void* stream,
                             fe_evk** out) {
    FE_ALIGNED(evk_dev);
    if (!c || !evk_host || !evk_dev || !out || (n_steps && !steps)) return fail(FE_EINVAL, "null argument");
    const size_t need = fe_evk_bytes(c, n_steps, relin);
    if (evk_host_bytes < need) return fail(FE_EINVAL, "host key bytes shorter than the keys of the steps");
    if (evk_dev_bytes < need) return fail(FE_ENOMEM, "evk buffer too small");
    const int N = c->N;
    std::set<uint32_t> seen;
    for (uint32_t i = 0; i < n_steps; i++) {
        if (steps[i] != FE_STEP_CONJ && steps[i] % (N / 2) == 0)
            return fail(FE_EINVAL, "rotation step is a multiple of N/2");
        if (!seen.insert(c->galois(steps[i])).second) return fail(FE_EINVAL, "duplicate rotation step");
    }
    cudaStream_t st = (cudaStream_t)stream;
    FE_CUDA_TRY(cudaMemcpyAsync(evk_dev, evk_host, need, cudaMemcpyHostToDevice, st));
    FE_CUDA_TRY(cudaStreamSynchronize(st));
    std::unique_ptr<fe_evk> h(new fe_evk());
    h->ctx = c;
    h->base = (u64*)evk_dev;
    const size_t key_words = (size_t)c->dnum * 2 * c->n_mod * N;
    for (uint32_t i = 0; i < n_steps; i++) {
        h->rot[c->galois(steps[i])] = h->base + (size_t)i * key_words;
        h->steps.push_back(steps[i]);
    }
    h->relin = relin ? h->base + (size_t)n_steps * key_words : nullptr;
    *out = h.release();
    return FE_OK;
}

extern "C" void fe_evk_destroy(fe_evk* evk) { delete evk; }

extern "C" int fe_evk_alias(fe_ctx* c, fe_evk* evk, const int32_t* steps, uint32_t n_steps, uint32_t* n_aliased) {
    if (!c || !evk || (n_steps && !steps)) return fail(FE_EINVAL, "null argument");
    std::vector<u64*> pool;
    for (auto& kv : evk->rot) pool.push_back(kv.second);
    if (pool.empty() && evk->relin) pool.push_back(evk->relin);
    if (pool.empty()) return fail(FE_EKEY, "fe_evk_alias needs at least one generated key");
    uint32_t added = 0;
    for (uint32_t i = 0; i < n_steps; i++) {
        if (steps[i] != FE_STEP_CONJ && steps[i] % (c->N / 2) == 0) continue;
        const uint32_t g = c->galois(steps[i]);
        if (evk->rot.count(g)) continue;
        evk->rot[g] = pool[added % pool.size()];
        added++;
    }
    if (n_aliased) *n_aliased = added;
    return FE_OK;
}

// ---------------------------------------------------------------------------
// C ABI: encode / encrypt / decrypt
// ---------------------------------------------------------------------------

extern "C" int fe_encode(fe_ctx* c, const double* slots, uint32_t n, uint32_t level, double scale,
                         void* pt_dev, void* stream) {
    FE_ALIGNED(slots);
    FE_ALIGNED(pt_dev);
    if (!c || !slots || !pt_dev) return fail(FE_EINVAL, "null argument");
    if ((int)level > c->L) return fail(FE_ELEVEL, "level above L");
    return encode_batch(c, slots, (int)n, (int)level, scale, (u64*)pt_dev, (cudaStream_t)stream);
}

extern "C" int fe_encode_encrypt(fe_ctx* c, const void* sk_dev, const double* slots, uint32_t n_ct,
                                 uint32_t level, double scale, uint64_t seed, uint64_t ct_id0, void* ct_dev,
                                 void* stream) {
    FE_ALIGNED(slots);
    FE_ALIGNED(ct_dev); FE_ALIGNED(sk_dev);
    if (!c || !sk_dev || !slots || !ct_dev) return fail(FE_EINVAL, "null argument");
    if ((int)level > c->L) return fail(FE_ELEVEL, "level above L");
    if (ct_id0 + n_ct >= (1ull << 32)) return fail(FE_EINVAL, "ciphertext ids must stay below 2^32");
    if (n_ct == 0) return FE_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const int N = c->N, nl = level + 1;
    u64 *m, *en;
    i64* e;
    FE_CUDA_TRY(cudaMallocAsync(&m, (size_t)n_ct * nl * N * 8, st));
    FE_CUDA_TRY(cudaMallocAsync(&en, (size_t)n_ct * nl * N * 8, st));
    FE_CUDA_TRY(cudaMallocAsync(&e, (size_t)n_ct * N * 8, st));
    int rc = encode_batch(c, slots, (int)n_ct, (int)level, scale, m, st);
    if (rc == FE_OK) {
        u64* ct = (u64*)ct_dev;
        k_enc_sample<<<grid_for(N, nl, n_ct), kB, 0, st>>>(c->gen, seed, ct_id0, ct, e, c->d_mod, nl, c->logN);
        k_signed_rows_to_limbs<<<grid_for(N, nl, n_ct), kB, 0, st>>>(e, en, c->d_mod, nl, c->logN);
        ntt_forward(c, LimbSet{en, (size_t)nl * N, nl, (int)n_ct, c->d_identity_map}, st);
        k_enc_c0<<<grid_for(N, nl, n_ct), kB, 0, st>>>(ct, m, en, (const u64*)sk_dev, c->d_mod, nl, c->logN);
        c->cnt.launches += 3;
    }
    cudaFreeAsync(m, st);
    cudaFreeAsync(en, st);
    cudaFreeAsync(e, st);
    FE_CUDA_TRY(cudaStreamSynchronize(st));
    FE_CUDA_TRY(cudaGetLastError());
    return rc;
}

extern "C" int fe_decrypt_decode(fe_ctx* c, const void* sk_dev, const void* ct_dev, uint32_t n_ct,
                                 uint32_t level, double scale, double* slots, void* stream) {
    FE_ALIGNED(slots);
    FE_ALIGNED(ct_dev); FE_ALIGNED(sk_dev);
    if (!c || !sk_dev || !ct_dev || !slots) return fail(FE_EINVAL, "null argument");
    if ((int)level > c->L) return fail(FE_ELEVEL, "level above L");
    if (n_ct == 0) return FE_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const int N = c->N, nl = level + 1, nl2 = std::min(2, nl);
    u64* x;
    double* mdd;
    FE_CUDA_TRY(cudaMallocAsync(&x, (size_t)n_ct * nl2 * N * 8, st));
    FE_CUDA_TRY(cudaMallocAsync(&mdd, (size_t)n_ct * N * 16, st));
    k_dec_mul<<<grid_for(N, nl2, n_ct), kB, 0, st>>>((const u64*)ct_dev, (const u64*)sk_dev, x, c->d_mod,
                                                     nl, nl2, c->logN);
    ntt_inverse(c, LimbSet{x, (size_t)nl2 * N, nl2, (int)n_ct, c->d_identity_map}, st);
    k_crt_dd<<<grid_for(N, n_ct), kB, 0, st>>>(x, mdd, c->mod[0], c->L >= 1 ? c->mod[1] : 1, c->q0inv_q1,
                                               nl2, c->logN);
    c->cnt.launches += 2;
    int rc = decode_batch(c, mdd, (int)n_ct, scale, slots, st);
    cudaFreeAsync(x, st);
    cudaFreeAsync(mdd, st);
    FE_CUDA_TRY(cudaStreamSynchronize(st));
    FE_CUDA_TRY(cudaGetLastError());
    return rc;
}

// ---------------------------------------------------------------------------
// C ABI: primitives
// ---------------------------------------------------------------------------

extern "C" int fe_ntt(fe_ctx* c, void* data, uint32_t n_poly, uint32_t n_limbs, uint32_t first_mod,
                      int inverse, void* stream) {
    FE_ALIGNED(data);
    if (!c || !data) return fail(FE_EINVAL, "null argument");
    if ((int)(first_mod + n_limbs) > c->n_mod) return fail(FE_EINVAL, "limb range outside the moduli");
    LimbSet s{(u64*)data, (size_t)n_limbs * c->N, (int)n_limbs, (int)n_poly, c->d_identity_map + first_mod};
    if (inverse)
        ntt_inverse(c, s, (cudaStream_t)stream);
    else
        ntt_forward(c, s, (cudaStream_t)stream);
    FE_CUDA_TRY(cudaGetLastError());
    return FE_OK;
}

extern "C" int fe_probe_butterflies(fe_ctx* c, uint32_t blocks, uint32_t iters, void* out_dev,
                                    uint64_t* butterflies, void* stream) {
    if (!c || !out_dev) return fail(FE_EINVAL, "null argument");
    FE_ALIGNED(out_dev);
    if (iters == 0) return fail(FE_EINVAL, "iters must be positive");
    FE_TRY(butterfly_probe(c, &blocks, iters, (u64*)out_dev, (cudaStream_t)stream));
    if (butterflies) *butterflies = (uint64_t)blocks * 256 * iters * 60;
    return FE_OK;
}

namespace fe {
int rotate_many(fe_ctx* c, const fe_evk* evk, const u64* in, int n_ct, int level, const int32_t* steps,
                int n_steps, u64* out, cudaStream_t st) {
    if (n_ct <= 0 || n_steps <= 0) return FE_OK;
    const int N = c->N, nl = level + 1;
    const size_t ctw = ct_words(c, level), aw = acc_words(c, level), ew = ext_words(c, level);
    std::vector<const u64*> key(n_steps, nullptr);
    std::vector<uint32_t> gal(n_steps, 1);
    for (int j = 0; j < n_steps; j++) {
        if (steps[j] != FE_STEP_CONJ && steps[j] % (N / 2) == 0) continue;  // the identity
        gal[j] = c->galois(steps[j]);
        key[j] = evk_key(evk, gal[j]);
        if (!key[j]) return fail(FE_EKEY, "missing rotation key for step " + std::to_string(steps[j]));
    }
    const size_t per_step = (size_t)n_ct * (aw + ctw) * 8;
    const int chunk = (int)std::max<size_t>(1, std::min<size_t>(n_steps, (4ull << 30) / per_step));
    u64 *coef = nullptr, *ext = nullptr, *acc = nullptr, *conv = nullptr;
    void* items = nullptr;
    const size_t item_bytes = (size_t)chunk * n_ct * (sizeof(KsItem) + sizeof(CombineItem)) + (size_t)chunk * sizeof(KsGroup);
    int rc = FE_OK;
    if (cudaMallocAsync(&coef, (size_t)n_ct * nl * N * 8, st) != cudaSuccess ||
        cudaMallocAsync(&ext, (size_t)n_ct * ew * 8, st) != cudaSuccess ||
        cudaMallocAsync(&acc, (size_t)chunk * n_ct * aw * 8, st) != cudaSuccess ||
        cudaMallocAsync(&conv, (size_t)chunk * n_ct * ctw * 8, st) != cudaSuccess ||
        cudaMallocAsync(&items, item_bytes, st) != cudaSuccess) {
        (void)cudaGetLastError();  // an allocation failure is reported as FE_ENOMEM, not left pending
        rc = fail(FE_ENOMEM, "hoisted rotation scratch");
    }
    if (rc == FE_OK) modup(c, in + (size_t)nl * N, ctw, n_ct, level, coef, ext, st);
    KsItem* dks = (KsItem*)items;
    CombineItem* dcb = (CombineItem*)(dks + (size_t)chunk * n_ct);
    KsGroup* dkg = (KsGroup*)(dcb + (size_t)chunk * n_ct);
    for (int j0 = 0; rc == FE_OK && j0 < n_steps; j0 += chunk) {
        const int jn = std::min(chunk, n_steps - j0);
        std::vector<KsItem> ks;
        std::vector<CombineItem> cb;
        std::vector<KsGroup> kg;
        for (int j = j0; j < j0 + jn; j++) {
            u64* o = out + (size_t)j * n_ct * ctw;
            if (!key[j]) {
                if (cudaMemcpyAsync(o, in, (size_t)n_ct * ctw * 8, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
                    rc = fail(FE_ECUDA, "hoisted rotation copy");
                continue;
            }
            kg.push_back(KsGroup{key[j], (int)ks.size(), n_ct});
            for (int i = 0; i < n_ct; i++) {
                const size_t k = ks.size();
                ks.push_back(KsItem{ext + i * ew, key[j], acc + k * aw});
                cb.push_back(CombineItem{acc + k * aw, conv + k * ctw, in + i * ctw, nullptr, o + i * ctw, gal[j], 0});
            }
        }
        if (ks.empty() || rc != FE_OK) continue;
        const int m = (int)ks.size();
        rc = upload(ks, dks, st);
        if (rc == FE_OK) rc = upload(cb, dcb, st);
        if (rc == FE_OK) rc = upload(kg, dkg, st);
        if (rc != FE_OK) break;
        launch_keyip_grouped(c, dkg, dks, (int)kg.size(), m, level, st, n_ct);
        moddown_prepare(c, acc, m, level, conv, st);
        launch_combine(c, dcb, m, level, st);
        c->cnt.rot += m;
        c->cnt.keyswitch += m;
    }
    if (coef) cudaFreeAsync(coef, st);
    if (ext) cudaFreeAsync(ext, st);
    if (acc) cudaFreeAsync(acc, st);
    if (conv) cudaFreeAsync(conv, st);
    if (items) cudaFreeAsync(items, st);
    FE_TRY(rc);
    FE_CUDA_TRY(cudaGetLastError());
    return FE_OK;
}
}  // namespace fe

extern "C" int fe_rotate_many(fe_ctx* c, const fe_evk* evk, const void* ct_dev, uint32_t n_ct, uint32_t level,
                              const int32_t* steps, uint32_t n_steps, void* out_dev, void* stream) {
    FE_ALIGNED(ct_dev); FE_ALIGNED(out_dev);
    if (!c || !evk || !ct_dev || !out_dev || (n_steps && !steps)) return fail(FE_EINVAL, "null argument");
    if ((int)level > c->L) return fail(FE_ELEVEL, "level above L");
    if (n_ct == 0 || n_steps == 0) return FE_OK;
    if (n_ct > (1u << 20) || n_steps > (1u << 20)) return fail(FE_EINVAL, "n_ct and n_steps must be below 2^20");
    const size_t in_b = (size_t)n_ct * ct_words(c, (int)level) * 8, out_b = in_b * n_steps;
    const char *i0 = (const char*)ct_dev, *o0 = (const char*)out_dev;
    if (o0 < i0 + in_b && i0 < o0 + out_b) return fail(FE_EINVAL, "the outputs overlap the inputs");
    return rotate_many(c, evk, (const u64*)ct_dev, (int)n_ct, (int)level, steps, (int)n_steps, (u64*)out_dev,
                       (cudaStream_t)stream);
}

extern "C" int fe_rotate(fe_ctx* c, const fe_evk* evk, const void* ct_dev, uint32_t n_ct, uint32_t level,
                         int32_t r, void* out_dev, void* stream) {
    FE_ALIGNED(ct_dev); FE_ALIGNED(out_dev);
    if (!c || !evk || !ct_dev || !out_dev) return fail(FE_EINVAL, "null argument");
    if ((int)level > c->L) return fail(FE_ELEVEL, "level above L");
    if (n_ct == 0) return FE_OK;
    if (n_ct > (1u << 20)) return fail(FE_EINVAL, "n_ct must be below 2^20");
    const size_t bytes = (size_t)n_ct * ct_words(c, (int)level) * 8;
    const char *i0 = (const char*)ct_dev, *o0 = (const char*)out_dev;
    if (o0 < i0 + bytes && i0 < o0 + bytes) return fail(FE_EINVAL, "a rotation cannot run in place");
    // one step of the hoisted form: ModUp, the key inner product with the key
    // read once for all n_ct ciphertexts, ModDown, automorphism
    return rotate_many(c, evk, (const u64*)ct_dev, (int)n_ct, (int)level, &r, 1, (u64*)out_dev,
                       (cudaStream_t)stream);
}

extern "C" int fe_rescale(fe_ctx* c, const void* ct_dev, uint32_t n_ct, uint32_t level, void* out_dev,
                          void* stream) {
    FE_ALIGNED(ct_dev); FE_ALIGNED(out_dev);
    if (!c || !ct_dev || !out_dev) return fail(FE_EINVAL, "null argument");
    if (level == 0) return fail(FE_ELEVEL, "rescale at level 0");
    if ((int)level > c->L) return fail(FE_ELEVEL, "level above L");
    if (n_ct == 0) return FE_OK;
    cudaStream_t st = (cudaStream_t)stream;
    u64* tmp;
    FE_CUDA_TRY(cudaMallocAsync(&tmp, rescale_tmp_words(c, n_ct, level) * 8, st));
    rescale_batch(c, (const u64*)ct_dev, n_ct, level, (u64*)out_dev, tmp, tmp + 2 * (size_t)n_ct * c->N, st);
    cudaFreeAsync(tmp, st);
    FE_CUDA_TRY(cudaGetLastError());
    return FE_OK;
}

extern "C" int fe_pmult(fe_ctx* c, const void* ct_dev, const void* pt_dev, uint32_t n_ct, uint32_t level,
                        void* out_dev, void* stream) {
    if (!c || !ct_dev || !pt_dev || !out_dev) return fail(FE_EINVAL, "null argument");
    FE_ALIGNED(ct_dev);
    FE_ALIGNED(pt_dev);
    FE_ALIGNED(out_dev);
    if ((int)level > c->L) return fail(FE_ELEVEL, "level above L");
    launch_pmult(c, (const u64*)ct_dev, (const u64*)pt_dev, (u64*)out_dev, n_ct, level, false,
                 (cudaStream_t)stream);
    c->cnt.pmult += n_ct;
    FE_CUDA_TRY(cudaGetLastError());
    return FE_OK;
}

extern "C" int fe_add(fe_ctx* c, const void* a, const void* b, uint32_t n_ct, uint32_t level, void* out,
                      void* stream) {
    if (!c || !a || !b || !out) return fail(FE_EINVAL, "null argument");
    FE_ALIGNED(a);
    FE_ALIGNED(b);
    FE_ALIGNED(out);
    if ((int)level > c->L) return fail(FE_ELEVEL, "level above L");
    launch_add(c, (const u64*)a, (const u64*)b, (u64*)out, n_ct, level, (cudaStream_t)stream);
    FE_CUDA_TRY(cudaGetLastError());
    return FE_OK;
}
