// Layers around the convolution: x^2 activation (CMult + relinearisation +
// rescale), 2x2 average pooling by fragment sums, Arch-aware Ciphertext
// Compression (rotate-and-add replication), and CUDA-graph capture of a
// sequence of planned layers.
#include <algorithm>
#include <climits>
#include <cstdint>
#include <cmath>
#include <memory>

#include "graph.h"
#include "plan.h"

namespace fe {
namespace {
constexpr int kB = 256;

// out[(g S' + u) S' + v] = sum_{di, dj} in[(g S + 2u + di) S + 2v + dj], S' = S / 2
__global__ void k_pool(const u64* in, u64* out, const Modulus* mods, int S, int nl, int logN) {
    const int N = 1 << logN;
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const int limb = blockIdx.y, o = blockIdx.z;  // limb over 2 nl
    const int So = S / 2;
    const int g = o / (So * So), u = (o / So) % So, v = o % So;
    const u64 q = mods[limb % nl].q;
    const size_t per = 2 * (size_t)nl * N, off = (size_t)limb * N + n;
    u64 acc = 0;
    for (int di = 0; di < 2; di++)
        for (int dj = 0; dj < 2; dj++) {
            const int ci = (g * S + 2 * u + di) * S + 2 * v + dj;
            acc = add_mod(acc, in[(size_t)ci * per + off], q);
        }
    out[(size_t)o * per + off] = acc;
}

struct KsScratch {
    u64 *coef, *ext, *acc, *conv;
    KsItem* ks;
    KsGroup* kg;
};

size_t ks_scratch_bytes(const fe_ctx* c, int n, int level) {
    return (size_t)n * ((level + 1) * (size_t)c->N + ext_words(c, level) + acc_words(c, level) + ct_words(c, level)) * 8 +
           (size_t)n * (sizeof(KsItem) + sizeof(SumItem) + sizeof(SumEntry) + sizeof(CombineItem)) + 16 * 256;
}

bool carve_ks(Carver& cv, const fe_ctx* c, int n, int level, KsScratch* s) {
    s->coef = cv.take<u64>((size_t)n * (level + 1) * c->N);
    s->ext = cv.take<u64>((size_t)n * ext_words(c, level));
    s->acc = cv.take<u64>((size_t)n * acc_words(c, level));
    s->conv = cv.take<u64>((size_t)n * ct_words(c, level));
    s->ks = cv.take<KsItem>(n);
    s->kg = cv.take<KsGroup>(1);
    return cv.ok;
}

// out = in * mul_i (+ add_i on c0), limb i of each of n ciphertexts [2][nl][N]
__global__ void k_affine(const u64* in, u64* out, const Modulus* mods, AffineConsts k, int nl, int logN,
                         int do_mul) {
    const int N = 1 << logN;
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const int limb = blockIdx.y, ci = blockIdx.z;  // limb over 2 nl
    const int i = limb % nl;
    const Modulus m = mods[i];
    const size_t o = ((size_t)ci * 2 * nl + limb) * N + n;
    u64 v = in[o];
    if (do_mul) v = mul_mod(v, k.mul[i], m);
    if (limb < nl) v = add_mod(v, k.add[i], m.q);
    out[o] = v;
}

}  // namespace

// the integer nearest to x, ties away from zero, reduced mod q (any finite x)
u64 nearest_mod(double x, u64 q) {
    double t = std::trunc(x);
    if (std::fabs(x - t) >= 0.5) t += x > 0 ? 1.0 : -1.0;
    const bool neg = t < 0;
    const double mag = std::fabs(t);
    int e = 0;
    const double fr = std::frexp(mag, &e);  // mag = fr 2^e, fr in [1/2, 1)
    u64 r;
    if (e <= 63) {
        r = (u64)mag % q;
    } else {  // mag = M 2^(e - 53) with the 53-bit integer M
        const u64 M = (u64)std::ldexp(fr, 53);
        r = h_mulmod(M % q, h_powmod(2, (u64)(e - 53), q), q);
    }
    return neg && r ? q - r : r;
}

int launch_affine(fe_ctx* c, const u64* in, u64* out, int n, int level, const AffineConsts& k, bool do_mul,
                  cudaStream_t st) {
    if (level + 1 > kMaxAffineLimbs) return fail(FE_EINVAL, "more limbs than the affine kernel holds");
    if (!n) return FE_OK;
    k_affine<<<dim3((c->N + kB - 1) / kB, 2 * (level + 1), n), kB, 0, st>>>(in, out, c->d_mod, k, level + 1, c->logN,
                                                                           do_mul ? 1 : 0);
    c->cnt.launches++;
    return FE_OK;
}

// d = relin of n products (d0, d1, d2) [n][3][nl][N] on Q_level: (d0, d1) + KS(d2)
int relin_tensors(fe_ctx* c, const fe_evk* evk, const u64* d012, int n, int level, u64* d, Carver& cv,
                  cudaStream_t st) {
    const int N = c->N, nl = level + 1;
    KsScratch s;
    carve_ks(cv, c, n, level, &s);
    CombineItem* dcb = cv.take<CombineItem>(n);
    if (!cv.ok) return fail(FE_ENOMEM, "workspace too small");
    std::vector<KsItem> ks(n);
    std::vector<CombineItem> cb(n);
    for (int i = 0; i < n; i++) {
        ks[i] = KsItem{s.ext + i * ext_words(c, level), evk->relin, s.acc + i * acc_words(c, level)};
        const u64* dd = d012 + (size_t)i * 3 * nl * N;
        cb[i] = CombineItem{s.acc + i * acc_words(c, level), s.conv + i * ct_words(c, level), dd, dd + (size_t)nl * N,
                            d + i * ct_words(c, level), 1, 0};
    }
    std::vector<KsGroup> kg{KsGroup{evk->relin, 0, n}};
    FE_TRY(upload(ks, s.ks, st));
    FE_TRY(upload(kg, s.kg, st));
    FE_TRY(upload(cb, dcb, st));
    modup(c, d012 + 2 * (size_t)nl * N, 3 * (size_t)nl * N, n, level, s.coef, s.ext, st);
    launch_keyip_grouped(c, s.kg, s.ks, 1, n, level, st);
    moddown_prepare(c, s.acc, n, level, s.conv, st);
    launch_combine(c, dcb, n, level, st);
    c->cnt.keyswitch += n;
    return FE_OK;
}

size_t relin_tensors_bytes(const fe_ctx* c, int n, int level) {
    return ks_scratch_bytes(c, n, level) + (size_t)n * sizeof(CombineItem) + 2 * 256;
}

// d = relin(x (x) y) on Q_level for n pairs of ciphertexts, no rescale (CMult + relinearisation)
int cmult_relin(fe_ctx* c, const fe_evk* evk, const u64* x, const u64* y, int n, int level, u64* d, Carver& cv,
                cudaStream_t st) {
    u64* d012 = cv.take<u64>((size_t)n * 3 * (level + 1) * c->N);
    if (!cv.ok) return fail(FE_ENOMEM, "workspace too small");
    launch_tensor(c, x, y, d012, n, level, st);
    FE_TRY(relin_tensors(c, evk, d012, n, level, d, cv, st));
    c->cnt.cmult += n;
    return FE_OK;
}

size_t cmult_relin_bytes(const fe_ctx* c, int n, int level) {
    return ks_scratch_bytes(c, n, level) + (size_t)n * (3 * (level + 1)) * c->N * 8 +
           (size_t)n * sizeof(CombineItem) + 4 * 256;
}

namespace {
int square_relin(fe_ctx* c, const fe_evk* evk, const u64* in, int n, int level, u64* d, Carver& cv,
                 cudaStream_t st) {
    return cmult_relin(c, evk, in, in, n, level, d, cv, st);
}

}  // namespace
}  // namespace fe

using namespace fe;

extern "C" size_t fe_square_workspace_bytes(const fe_ctx* c, uint32_t n, uint32_t level) {
    if (!c) return 0;
    return ks_scratch_bytes(c, n, level) + (size_t)n * (3 * (level + 1) + 2 * (level + 1)) * c->N * 8 +
           rescale_tmp_words(c, n, level) * 8 + 8 * 256;
}

extern "C" int fe_he_square(fe_ctx* c, const fe_evk* evk, const void* in_dev, uint32_t n, uint32_t level,
                            void* out_dev, void* ws, size_t ws_bytes, void* stream) {
    FE_ALIGNED(in_dev); FE_ALIGNED(out_dev); FE_ALIGNED(ws);
    if (!c || !evk || !in_dev || !out_dev || !ws) return fail(FE_EINVAL, "null argument");
    if (level == 0 || (int)level > c->L) return fail(FE_ELEVEL, "x^2 needs a level to rescale");
    if (!evk->relin) return fail(FE_EKEY, "no relinearisation key");
    if (ws_bytes < fe_square_workspace_bytes(c, n, level)) return fail(FE_ENOMEM, "workspace too small");
    if (n == 0) return FE_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const int N = c->N;
    Carver cv(ws, ws_bytes);
    u64* tmp = cv.take<u64>((size_t)n * ct_words(c, level));
    u64* rs = cv.take<u64>(rescale_tmp_words(c, n, level));
    if (!cv.ok) return fail(FE_ENOMEM, "workspace too small");
    FE_TRY(square_relin(c, evk, (const u64*)in_dev, (int)n, (int)level, tmp, cv, st));
    rescale_batch(c, tmp, n, level, (u64*)out_dev, rs, rs + 2 * (size_t)n * N, st);
    FE_CUDA_TRY(cudaGetLastError());
    return FE_OK;
}

extern "C" size_t fe_poly_act_workspace_bytes(const fe_ctx* c, uint32_t n, uint32_t level) {
    if (!c) return 0;
    return fe_square_workspace_bytes(c, n, level) + (size_t)n * ct_words(c, level) * 8 + 256;
}

extern "C" int fe_poly_act_scale(const fe_ctx* c, uint32_t level, double in_scale, double a, double* out_scale) {
    if (!c || !out_scale) return fail(FE_EINVAL, "null argument");
    if (level == 0 || (int)level > c->L) return fail(FE_ELEVEL, "the activation needs a level to rescale");
    if (!(in_scale > 0) || !std::isfinite(a)) return fail(FE_EINVAL, "bad scale or coefficient");
    const double ql = (double)c->mod[level];
    *out_scale = a != 0 ? (in_scale * in_scale) / (ql * std::fabs(a)) : in_scale;
    return FE_OK;
}

extern "C" int fe_he_poly_act(fe_ctx* c, const fe_evk* evk, double a, double b, double cc, const void* in_dev,
                              uint32_t n, uint32_t level, double in_scale, void* out_dev, double* out_scale, void* ws,
                              size_t ws_bytes, void* stream) {
    FE_ALIGNED(in_dev); FE_ALIGNED(out_dev); FE_ALIGNED(ws);
    if (!c || !in_dev || !out_dev || !ws) return fail(FE_EINVAL, "null argument");
    if (!std::isfinite(a) || !std::isfinite(b) || !std::isfinite(cc)) return fail(FE_EINVAL, "coefficient not finite");
    double sc = 0;
    FE_TRY(fe_poly_act_scale(c, level, in_scale, a, &sc));
    if (a != 0 && (!evk || !evk->relin)) return fail(FE_EKEY, "no relinearisation key");
    if (ws_bytes < fe_poly_act_workspace_bytes(c, n, level)) return fail(FE_ENOMEM, "workspace too small");
    if (out_scale) *out_scale = sc;
    if (n == 0) return FE_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const int nl = level + 1;
    const double s = in_scale, ql = (double)c->mod[level];
    Carver cv(ws, ws_bytes);
    u64* u = cv.take<u64>((size_t)n * ct_words(c, level));
    u64* v = cv.take<u64>((size_t)n * ct_words(c, level));
    u64* rs = cv.take<u64>(rescale_tmp_words(c, n, level));
    if (!cv.ok) return fail(FE_ENOMEM, "workspace too small");
    AffineConsts k{};
    if (a != 0) {
        // a x^2 + b x + c = a [(x + beta)^2 + gamma]: shift, square, scale by sign(a) and add
        const double beta = b / (2.0 * a);
        const double gamma = cc / a - beta * beta;
        const bool neg = a < 0;
        for (int i = 0; i < nl; i++) {
            k.mul[i] = 1;
            k.add[i] = nearest_mod(beta * s, c->mod[i]);
        }
        FE_TRY(launch_affine(c, (const u64*)in_dev, u, n, level, k, false, st));
        FE_TRY(square_relin(c, evk, u, (int)n, (int)level, v, cv, st));
        for (int i = 0; i < nl; i++) {
            const u64 q = c->mod[i], g = nearest_mod(gamma * (s * s), q);
            k.mul[i] = neg ? q - 1 : 1;
            k.add[i] = neg && g ? q - g : g;
        }
        FE_TRY(launch_affine(c, v, v, n, level, k, neg, st));
    } else {
        // b x + c: times the integer nearest b q_l, plus the integer nearest c s q_l
        for (int i = 0; i < nl; i++) {
            k.mul[i] = nearest_mod(b * ql, c->mod[i]);
            k.add[i] = nearest_mod(cc * (s * ql), c->mod[i]);
        }
        FE_TRY(launch_affine(c, (const u64*)in_dev, v, n, level, k, true, st));
    }
    rescale_batch(c, v, n, level, (u64*)out_dev, rs, rs + 2 * (size_t)n * c->N, st);
    FE_CUDA_TRY(cudaGetLastError());
    return FE_OK;
}

extern "C" int fe_weight_scale(const fe_ctx* c, uint32_t level, double s_in, double delta, double act_a,
                               double* w_scale) {
    if (!c || !w_scale) return fail(FE_EINVAL, "null argument");
    if (level == 0 || (int)level > c->L) return fail(FE_ELEVEL, "a linear layer needs a level to rescale");
    if (!(s_in > 0) || !(delta > 0) || !std::isfinite(act_a)) return fail(FE_EINVAL, "bad scale");
    const double t = act_a != 0 ? std::sqrt(delta * (double)c->mod[level - 1] * std::fabs(act_a)) : delta;
    *w_scale = (t / s_in) * (double)c->mod[level];
    return FE_OK;
}

extern "C" int fe_he_avgpool(fe_ctx* c, const fe_layout* lay, const void* in_dev, uint32_t level, void* out_dev,
                             fe_layout* out_lay, void* stream) {
    if (!c || !lay || !in_dev || !out_dev) return fail(FE_EINVAL, "null argument");
    FE_ALIGNED(in_dev);
    FE_ALIGNED(out_dev);
    if ((int)level > c->L) return fail(FE_ELEVEL, "level above L");
    fe_layout L = *lay;
    FE_TRY(layout_fill(c->N, &L));
    if (L.S % 2) return fail(FE_EINVAL, "pooling by fragment sums needs an even S");
    fe_layout O{};
    O.H = L.H / 2;
    O.W = L.W / 2;
    O.C = L.C;
    O.BS = L.BS;
    O.S = L.S / 2;
    O.m = L.m;
    FE_TRY(layout_fill(c->N, &O));
    const int nl = level + 1;
    k_pool<<<dim3((c->N + kB - 1) / kB, 2 * nl, O.n_ct), kB, 0, (cudaStream_t)stream>>>(
        (const u64*)in_dev, (u64*)out_dev, c->d_mod, L.S, nl, c->logN);
    c->cnt.launches++;
    if (out_lay) *out_lay = O;
    FE_CUDA_TRY(cudaGetLastError());
    return FE_OK;
}

extern "C" size_t fe_compress_workspace_bytes(const fe_ctx* c, uint32_t n, uint32_t level) {
    if (!c) return 0;
    return ks_scratch_bytes(c, n, level) + 2 * (size_t)n * ct_words(c, level) * 8 + 8 * 256;
}

namespace fe {
namespace {
// rotate-and-add replication of the c_valid valid channel blocks (Fig. 6) on n
// ciphertexts at `level`; the layout L is filled and validated by the caller
int compress_core(fe_ctx* c, const fe_evk* evk, const fe_layout& L, uint32_t c_valid, const void* in_dev, uint32_t n,
                  uint32_t level, void* out_dev, void* ws, size_t ws_bytes, cudaStream_t st) {
    const size_t ctw = ct_words(c, level);
    if (n == 0) return FE_OK;
    std::vector<int32_t> steps;
    for (uint32_t s = c_valid; s < L.cpc; s *= 2) steps.push_back(-(int32_t)(s * L.m * L.m * L.BS));
    if (steps.empty()) {
        FE_CUDA_TRY(cudaMemcpyAsync(out_dev, in_dev, n * ctw * 8, cudaMemcpyDeviceToDevice, st));
        return FE_OK;
    }
    for (int32_t s : steps)
        if (!evk_key(evk, c->galois(s))) return fail(FE_EKEY, "missing rotation key for step " + std::to_string(s));
    Carver cv(ws, ws_bytes);
    KsScratch ksc;
    carve_ks(cv, c, n, level, &ksc);
    SumItem* dsum = cv.take<SumItem>(n);
    SumEntry* dent = cv.take<SumEntry>(n);
    u64* buf[2] = {cv.take<u64>(n * ctw), cv.take<u64>(n * ctw)};
    if (!cv.ok) return fail(FE_ENOMEM, "workspace too small");
    const u64* cur = (const u64*)in_dev;
    for (size_t si = 0; si < steps.size(); si++) {
        u64* next = si + 1 == steps.size() ? (u64*)out_dev : buf[si % 2];
        const u64* key = evk_key(evk, c->galois(steps[si]));
        std::vector<KsItem> ks(n);
        std::vector<SumItem> sums(n);
        std::vector<SumEntry> ents(n);
        for (uint32_t i = 0; i < n; i++) {
            ks[i] = KsItem{ksc.ext + i * ext_words(c, level), key, ksc.acc + i * acc_words(c, level)};
            const uint32_t gal = c->galois(steps[si]);
            ents[i] = SumEntry{ksc.acc + i * acc_words(c, level), ksc.conv + i * ctw, cur + i * ctw, gal,
                               (uint32_t)h_invmod(gal, 2 * (u64)c->N)};
            sums[i] = SumItem{next + i * ctw, cur + i * ctw, (int)i, 1, 0, nullptr};
        }
        std::vector<KsGroup> kg{KsGroup{key, 0, (int)n}};
        FE_TRY(upload(ks, ksc.ks, st));
        FE_TRY(upload(kg, ksc.kg, st));
        FE_TRY(upload(ents, dent, st));
        FE_TRY(upload(sums, dsum, st));
        modup(c, cur + (size_t)(level + 1) * c->N, ctw, n, level, ksc.coef, ksc.ext, st);
        launch_keyip_grouped(c, ksc.kg, ksc.ks, 1, (int)n, level, st);
        moddown_prepare(c, ksc.acc, n, level, ksc.conv, st);
        launch_combine_sum(c, dsum, dent, n, n, level, st);
        c->cnt.rot += n;
        c->cnt.keyswitch += n;
        cur = next;
        // the item tables are rewritten by the next step: keep the stream ordered
        FE_CUDA_TRY(cudaStreamSynchronize(st));
    }
    FE_CUDA_TRY(cudaGetLastError());
    return FE_OK;
}
}  // namespace
}  // namespace fe

extern "C" int fe_compress(fe_ctx* c, const fe_evk* evk, const fe_layout* lay, uint32_t c_valid, const void* in_dev,
                           uint32_t n, uint32_t level, void* out_dev, void* ws, size_t ws_bytes, void* stream) {
    FE_ALIGNED(in_dev); FE_ALIGNED(out_dev); FE_ALIGNED(ws);
    if (!c || !evk || !lay || !in_dev || !out_dev || !ws) return fail(FE_EINVAL, "null argument");
    if ((int)level > c->L) return fail(FE_ELEVEL, "level above L");
    fe_layout L = *lay;
    FE_TRY(layout_fill(c->N, &L));
    if (c_valid == 0 || L.cpc % c_valid) return fail(FE_EINVAL, "c_valid must divide cpc");
    if (ws_bytes < fe_compress_workspace_bytes(c, n, level)) return fail(FE_ENOMEM, "workspace too small");
    return compress_core(c, evk, L, c_valid, in_dev, n, level, out_dev, ws, ws_bytes, (cudaStream_t)stream);
}

namespace fe {
namespace {
// 0/1 slot vector of the valid channel blocks: slot < c_valid m^2 BS
__global__ void k_aac_mask(double* slots, int n_one, int half) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < half) slots[i] = i < n_one ? 1.0 : 0.0;
}
}  // namespace
}  // namespace fe

extern "C" size_t fe_compress_masked_workspace_bytes(const fe_ctx* c, uint32_t n, uint32_t level) {
    if (!c) return 0;
    return fe_compress_workspace_bytes(c, n, level) + (size_t)n * ct_words(c, level) * 8 +
           (size_t)(level + 1) * c->N * 8 + (size_t)c->N / 2 * 8 + 4 * 256;
}

extern "C" int fe_compress_masked(fe_ctx* c, const fe_evk* evk, const fe_layout* lay, uint32_t c_valid,
                                  double mask_scale, const void* in_dev, uint32_t n, uint32_t level, double in_scale,
                                  void* out_dev, double* out_scale, void* ws, size_t ws_bytes, void* stream) {
    FE_ALIGNED(in_dev); FE_ALIGNED(out_dev); FE_ALIGNED(ws);
    if (!c || !evk || !lay || !in_dev || !out_dev || !ws) return fail(FE_EINVAL, "null argument");
    if ((int)level > c->L) return fail(FE_ELEVEL, "level above L");
    if (!(mask_scale >= 1) || !(in_scale > 0)) return fail(FE_EINVAL, "bad scale");
    fe_layout L = *lay;
    FE_TRY(layout_fill(c->N, &L));
    if (c_valid == 0 || L.cpc % c_valid) return fail(FE_EINVAL, "c_valid must divide cpc");
    if (ws_bytes < fe_compress_masked_workspace_bytes(c, n, level)) return fail(FE_ENOMEM, "workspace too small");
    if (out_scale) *out_scale = in_scale * mask_scale;
    if (n == 0) return FE_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t ctw = ct_words(c, level);
    Carver cv(ws, ws_bytes);
    u64* masked = cv.take<u64>((size_t)n * ctw);
    u64* pt = cv.take<u64>((size_t)(level + 1) * c->N);
    double* slots = cv.take<double>((size_t)c->N / 2);
    if (!cv.ok) return fail(FE_ENOMEM, "workspace too small");
    const int half = c->N / 2;
    k_aac_mask<<<(half + kB - 1) / kB, kB, 0, st>>>(slots, (int)(c_valid * L.m * L.m * L.BS), half);
    c->cnt.launches++;
    FE_TRY(encode_batch(c, slots, 1, (int)level, mask_scale, pt, st));
    for (uint32_t i = 0; i < n; i++)
        launch_pmult(c, (const u64*)in_dev + i * ctw, pt, masked + i * ctw, 1, (int)level, false, st);
    c->cnt.pmult += n;
    return compress_core(c, evk, L, c_valid, masked, n, level, out_dev, (char*)ws + (ws_bytes - cv.left),
                         cv.left, st);
}


namespace {
// shared data region of a captured sequence: the largest default data region
// of its layers
size_t graph_data_bytes(const fe_plan* const* plans, uint32_t n, uint32_t n_req) {
    size_t data = 0;
    for (uint32_t i = 0; i < n; i++) {
        const size_t def = fe_plan_workspace_bytes(plans[i], n_req, 0);
        const size_t ch = plan_chunk(plans[i], n_req, 1, def, false);
        data = std::max(data, plan_data_bytes(plans[i], ch, n_req));
    }
    return (data + 255) & ~(size_t)255;
}
}  // namespace

extern "C" size_t fe_graph_workspace_bytes(const fe_plan* const* plans, uint32_t n, uint32_t n_req) {
    if (!plans || n_req == 0) return 0;
    for (uint32_t i = 0; i < n; i++)
        if (!plans[i]) return 0;
    const size_t data = graph_data_bytes(plans, n, n_req);
    size_t tables = 0;
    for (uint32_t i = 0; i < n; i++)
        tables += (plan_table_bytes(plans[i], plan_chunk(plans[i], n_req, 1, data, true), n_req) + 255) & ~(size_t)255;
    return tables + data;
}

extern "C" int fe_graph_capture_batch(fe_ctx* c, const fe_evk* evk, const fe_plan* const* plans,
                                      const void* const* pts, const void* const* ins, void* const* outs, uint32_t n,
                                      uint32_t n_req, void* ws, size_t ws_bytes, void* stream, fe_graph** out) {
    if (!c || !evk || !plans || !pts || !ins || !outs || !ws || !out) return fail(FE_EINVAL, "null argument");
    if (n_req == 0) return fail(FE_EINVAL, "n_req must be positive");
    cudaStream_t st = (cudaStream_t)stream;
    if (!st) return fail(FE_EINVAL, "graph capture needs a non-default stream");
    FE_ALIGNED(ws);
    for (uint32_t i = 0; i < n; i++) {
        if (!plans[i]) return fail(FE_EINVAL, "null plan");
        FE_ALIGNED(pts[i]);
        FE_ALIGNED(ins[i]);
        FE_ALIGNED(outs[i]);
    }
    // every layer keeps its own item tables (they must survive until replay);
    // the data region (rotated copies, sums, scratch) is shared, layers run in order
    const size_t data = graph_data_bytes(plans, n, n_req);
    std::vector<size_t> off(n + 1, 0);
    for (uint32_t i = 0; i < n; i++) {
        const size_t ch = plan_chunk(plans[i], n_req, 1, data, true);
        off[i + 1] = off[i] + ((plan_table_bytes(plans[i], ch, n_req) + 255) & ~(size_t)255);
    }
    if (off[n] + data > ws_bytes) return fail(FE_ENOMEM, "workspace too small for the captured layers");
    char* shared = (char*)ws + off[n];
    for (uint32_t i = 0; i < n; i++)
        FE_TRY(run_plan(c, evk, plans[i], (const u64*)ins[i], (const u64*)pts[i], (u64*)outs[i], (char*)ws + off[i],
                        off[i + 1] - off[i], 1, st, 1, (int)n_req, 0, shared, data));
    FE_CUDA_TRY(cudaStreamSynchronize(st));
    std::unique_ptr<fe_graph> g(new fe_graph());
    FE_CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    int rc = FE_OK;
    for (uint32_t i = 0; i < n && rc == FE_OK; i++)
        rc = run_plan(c, evk, plans[i], (const u64*)ins[i], (const u64*)pts[i], (u64*)outs[i], (char*)ws + off[i],
                      off[i + 1] - off[i], 1, st, 2, (int)n_req, 0, shared, data);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(st, &graph);
    if (rc != FE_OK) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    if (e != cudaSuccess) return fail(FE_ECUDA, std::string("capture: ") + cudaGetErrorString(e));
    g->graph = graph;
    FE_CUDA_TRY(cudaGraphInstantiate(&g->exec, graph, 0));
    for (uint32_t i = 0; i < n; i++) {
        const fe_plan* p = plans[i];
        bool external = true;
        for (uint32_t j = 0; j < i; j++) external = external && outs[j] != ins[i];
        bool dup = false;
        for (const auto& e : g->in) dup = dup || e.dev == ins[i];
        if (external && !dup)
            g->in.push_back({const_cast<void*>(ins[i]), (size_t)n_req * p->n_in * 2 * (p->level + 1) * c->limb_bytes()});
    }
    for (uint32_t j = 0; j < n; j++) {
        bool read_later = false;
        for (uint32_t i = j + 1; i < n; i++) read_later = read_later || ins[i] == outs[j];
        if (!read_later) {
            g->out.push_back({outs[j], (size_t)n_req * plans[j]->n_out * 2 * plans[j]->level * c->limb_bytes()});
            g->out_level.push_back((uint32_t)plans[j]->level - 1);
        }
    }
    g->N = (size_t)c->N;
    *out = g.release();
    return FE_OK;
}

extern "C" size_t fe_graph_workspace_bytes_chunked(const fe_plan* const* plans, uint32_t n, uint32_t n_req,
                                                   uint32_t req_chunk) {
    if (!plans || n_req == 0 || req_chunk == 0) return 0;
    for (uint32_t i = 0; i < n; i++)
        if (!plans[i]) return 0;
    const uint32_t rc = std::min(req_chunk, n_req);
    const size_t data = graph_data_bytes(plans, n, rc);
    size_t tables = 0;
    for (uint32_t i = 0; i < n; i++)
        for (uint32_t r0 = 0; r0 < n_req; r0 += rc) {
            const uint32_t nr = std::min(rc, n_req - r0);
            tables += (plan_table_bytes(plans[i], plan_chunk(plans[i], nr, 1, data, true), nr) + 255) & ~(size_t)255;
        }
    return tables + data;
}

extern "C" int fe_graph_capture_chunked(fe_ctx* c, const fe_evk* evk, const fe_plan* const* plans,
                                        const void* const* pts, const void* const* ins, void* const* outs, uint32_t n,
                                        uint32_t n_req, uint32_t req_chunk, void* ws, size_t ws_bytes, void* stream,
                                        fe_graph** out) {
    if (!c || !evk || !plans || !pts || !ins || !outs || !ws || !out) return fail(FE_EINVAL, "null argument");
    if (n_req == 0 || req_chunk == 0) return fail(FE_EINVAL, "n_req and req_chunk must be positive");
    cudaStream_t st = (cudaStream_t)stream;
    if (!st) return fail(FE_EINVAL, "graph capture needs a non-default stream");
    FE_ALIGNED(ws);
    for (uint32_t i = 0; i < n; i++) {
        if (!plans[i]) return fail(FE_EINVAL, "null plan");
        FE_ALIGNED(pts[i]);
        FE_ALIGNED(ins[i]);
        FE_ALIGNED(outs[i]);
    }
    const uint32_t rc = std::min(req_chunk, n_req);
    const size_t data = graph_data_bytes(plans, n, rc);
    // item tables per (layer, request chunk), in capture order; one shared data region
    struct Piece {
        uint32_t layer, r0, nr;
        size_t off, bytes;
    };
    std::vector<Piece> pieces;
    size_t off = 0;
    for (uint32_t i = 0; i < n; i++)
        for (uint32_t r0 = 0; r0 < n_req; r0 += rc) {
            const uint32_t nr = std::min(rc, n_req - r0);
            const size_t b = (plan_table_bytes(plans[i], plan_chunk(plans[i], nr, 1, data, true), nr) + 255) &
                             ~(size_t)255;
            pieces.push_back({i, r0, nr, off, b});
            off += b;
        }
    if (off + data > ws_bytes) return fail(FE_ENOMEM, "workspace too small for the captured layers");
    char* shared = (char*)ws + off;
    auto in_at = [&](const Piece& q) {
        return (const u64*)ins[q.layer] + (size_t)q.r0 * plans[q.layer]->n_in * ct_words(c, plans[q.layer]->level);
    };
    auto out_at = [&](const Piece& q) {
        return (u64*)outs[q.layer] + (size_t)q.r0 * plans[q.layer]->n_out * ct_words(c, plans[q.layer]->level - 1);
    };
    for (const Piece& q : pieces)
        FE_TRY(run_plan(c, evk, plans[q.layer], in_at(q), (const u64*)pts[q.layer], out_at(q), (char*)ws + q.off,
                        q.bytes, 1, st, 1, (int)q.nr, 0, shared, data));
    FE_CUDA_TRY(cudaStreamSynchronize(st));
    std::unique_ptr<fe_graph> g(new fe_graph());
    FE_CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    int rc_ = FE_OK;
    for (size_t k = 0; k < pieces.size() && rc_ == FE_OK; k++) {
        const Piece& q = pieces[k];
        rc_ = run_plan(c, evk, plans[q.layer], in_at(q), (const u64*)pts[q.layer], out_at(q), (char*)ws + q.off,
                       q.bytes, 1, st, 2, (int)q.nr, 0, shared, data);
    }
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(st, &graph);
    if (rc_ != FE_OK) {
        if (graph) cudaGraphDestroy(graph);
        return rc_;
    }
    if (e != cudaSuccess) return fail(FE_ECUDA, std::string("capture: ") + cudaGetErrorString(e));
    g->graph = graph;
    FE_CUDA_TRY(cudaGraphInstantiate(&g->exec, graph, 0));
    for (uint32_t i = 0; i < n; i++) {
        bool external = true;
        for (uint32_t j = 0; j < i; j++) external = external && outs[j] != ins[i];
        bool dup = false;
        for (const auto& e2 : g->in) dup = dup || e2.dev == ins[i];
        if (external && !dup)
            g->in.push_back({const_cast<void*>(ins[i]),
                             (size_t)n_req * plans[i]->n_in * 2 * (plans[i]->level + 1) * c->limb_bytes()});
    }
    for (uint32_t j = 0; j < n; j++) {
        bool read_later = false;
        for (uint32_t i = j + 1; i < n; i++) read_later = read_later || ins[i] == outs[j];
        if (!read_later) {
            g->out.push_back({outs[j], (size_t)n_req * plans[j]->n_out * 2 * plans[j]->level * c->limb_bytes()});
            g->out_level.push_back((uint32_t)plans[j]->level - 1);
        }
    }
    g->N = (size_t)c->N;
    *out = g.release();
    return FE_OK;
}

extern "C" int fe_graph_capture(fe_ctx* c, const fe_evk* evk, const fe_plan* const* plans, const void* const* pts,
                                const void* const* ins, void* const* outs, uint32_t n, void* ws, size_t ws_bytes,
                                void* stream, fe_graph** out) {
    return fe_graph_capture_batch(c, evk, plans, pts, ins, outs, n, 1, ws, ws_bytes, stream, out);
}

extern "C" int fe_graph_launch(fe_graph* g, void* stream) {
    if (!g) return fail(FE_EINVAL, "null argument");
    FE_CUDA_TRY(cudaGraphLaunch(g->exec, (cudaStream_t)stream));
    return FE_OK;
}

namespace {
// host-side bytes of final output i: its ciphertexts at the host output level
size_t host_out_bytes(const fe_graph* g, size_t i) {
    const uint32_t lv = g->out_level[i];
    if (g->host_out_level >= lv) return g->out[i].bytes;
    const size_t per_ct_full = 2 * (size_t)(lv + 1) * g->N * 8;
    return g->out[i].bytes / per_ct_full * 2 * (size_t)(g->host_out_level + 1) * g->N * 8;
}
}  // namespace

extern "C" int fe_graph_set_host_output_level(fe_graph* g, uint32_t level) {
    if (!g) return fail(FE_EINVAL, "null argument");
    if (level != UINT32_MAX)
        for (uint32_t lv : g->out_level)
            if (level > lv) return fail(FE_ELEVEL, "host output level above an output's level");
    g->host_out_level = level;
    return FE_OK;
}

extern "C" int fe_graph_io(const fe_graph* g, uint32_t* n_in, size_t* in_bytes, uint32_t* n_out,
                           size_t* out_bytes) {
    if (!g || !n_in || !n_out) return fail(FE_EINVAL, "null argument");
    if (in_bytes)
        for (size_t i = 0; i < g->in.size(); i++) in_bytes[i] = g->in[i].bytes;
    if (out_bytes)
        for (size_t i = 0; i < g->out.size(); i++) out_bytes[i] = host_out_bytes(g, i);
    *n_in = (uint32_t)g->in.size();
    *n_out = (uint32_t)g->out.size();
    return FE_OK;
}

extern "C" int fe_graph_launch_host(fe_graph* g, const void* const* in_host, void* const* out_host, void* stream) {
    if (!g || (!g->in.empty() && !in_host) || (!g->out.empty() && !out_host)) return fail(FE_EINVAL, "null argument");
    for (size_t i = 0; i < g->in.size(); i++)
        if (!in_host[i]) return fail(FE_EINVAL, "null host input buffer");
    for (size_t i = 0; i < g->out.size(); i++)
        if (!out_host[i]) return fail(FE_EINVAL, "null host output buffer");
    cudaStream_t st = (cudaStream_t)stream;
    for (size_t i = 0; i < g->in.size(); i++)
        FE_CUDA_TRY(cudaMemcpyAsync(g->in[i].dev, in_host[i], g->in[i].bytes, cudaMemcpyHostToDevice, st));
    FE_CUDA_TRY(cudaGraphLaunch(g->exec, st));
    for (size_t i = 0; i < g->out.size(); i++) {
        const uint32_t lv = g->out_level[i];
        if (g->host_out_level >= lv) {
            FE_CUDA_TRY(cudaMemcpyAsync(out_host[i], g->out[i].dev, g->out[i].bytes, cudaMemcpyDeviceToHost, st));
        } else {
            // the first host_out_level + 1 limbs of every polynomial: the same ciphertexts
            // modulo q_0 .. q_{host_out_level} (an exact modulus drop)
            const size_t full = (size_t)(lv + 1) * g->N * 8, part = (size_t)(g->host_out_level + 1) * g->N * 8;
            FE_CUDA_TRY(cudaMemcpy2DAsync(out_host[i], part, g->out[i].dev, full, part, g->out[i].bytes / full,
                                          cudaMemcpyDeviceToHost, st));
        }
    }
    return FE_OK;
}

extern "C" void fe_graph_destroy(fe_graph* g) {
    if (!g) return;
    cudaGraphExecDestroy(g->exec);
    cudaGraphDestroy(g->graph);
    delete g;
}
