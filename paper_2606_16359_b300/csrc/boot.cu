// CKKS bootstrapping: the ciphertext refresh that deeper networks apply between
// convolution blocks (Sec. 5, Evaluation Methodology: each refresh of the
// paper's networks uses NEXUS's bootstrapping and consumes 14 levels).
//
// The paper adopts an existing bootstrapping without printing its steps; this
// file implements the standard CKKS refresh for the library's real-slot
// encoding (slot l at zeta^(5^l), zeta = exp(i pi / N), n = N/2 slots):
//  1. ModRaise: a level-0 ciphertext read as centred integers mod q_0 and
//     reduced modulo q_0..q_top; it decrypts to t = m + q_0 I, I small for a
//     sparse secret (fe_sk_gen_sparse).  Declared scale q_0.
//  2. re = ct + conj(ct) and im = -X^(N/2) (ct - conj(ct)) hold 2 Re(u) and
//     2 Im(u) of the slot vector u = U0 (t_lo + i t_hi) / q_0,
//     U0[l][j] = zeta^(5^l j).
//  3. CoeffToSlot: U0 = S_k ... S_1 R (butterfly stages of the special FFT,
//     R the bit reversal); S_1^-1 ... S_k^-1 applied to u, in groups of
//     consecutive stages, one level each, as real-form plaintext-matrix
//     products on the pair (re, im) by the diagonal method with baby / giant
//     steps (a planned FC-kind layer, run_plan).  Result: t / q_0 in
//     bit-reversed coefficient order, scaled by pi / 2^(r-1).
//  4. EvalMod on both parts: x - pi / 2^(r+1), the Taylor polynomial of cos to
//     degree 16, r double angles: sin(2 pi t / q_0) = sin(2 pi eps).
//  5. SlotToCoeff: S_k ... S_1 on re + i im in groups, the last keeping the
//     real part; the factor q_0 / (2 pi scale_in) folded into the first group.
// Every constant is a correctly rounded double (twiddles from a quad-precision
// cosine, Taylor coefficients as 1 / (2k)!) or one IEEE operation on such
// doubles, so that the plaintexts and integer constants are reproducible.
#include <algorithm>
#include <cmath>
#include <map>
#include <memory>
#include <numeric>
#include <set>
#include <vector>

#include "graph.h"
#include "plan.h"
#include "prng.cuh"

double boot_cos_pi_table_entry(int N, int e);  // boot_tables.cpp

struct fe_boot {
    fe_ctx* c = nullptr;
    int n_cts = 0, n_stc = 0, r = 0, top = 0, depth = 0;
    int form = 0;  // 0: transforms on the pair (re, im) in real form; 1: on one ciphertext, complex diagonals
    double scale_in = 0, out_scale = 0;
    std::vector<std::unique_ptr<fe_plan>> plans;  // CoeffToSlot groups, then SlotToCoeff groups (order applied)
    std::vector<u64*> pts;                        // their compact plaintexts (owned)
    u64* mono = nullptr;                          // NTT(-X^(N/2)) on q_0..q_top (owned)
    std::vector<int32_t> steps;                   // rotation steps (mod n) and FE_STEP_CONJ
    // sparse-secret encapsulation (caller-owned keys, or null): dense -> sparse at
    // level 0 before ModRaise, sparse -> dense at level top after it
    const u64* key_to_sparse = nullptr;
    const u64* key_to_dense = nullptr;
    ~fe_boot() {
        for (u64* p : pts) cudaFree(p);
        if (mono) cudaFree(mono);
    }
};

namespace fe {
namespace {
constexpr int kB = 256;

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------

// Sparse ternary secret of weight h (one block): partial Fisher-Yates over the
// index list, word w_i = gen_word(seed, tag, i): j = i + floor((w_i >> 1)(N - i) / 2^63),
// swap, s[idx[i]] = w_i odd ? -1 : +1.
__global__ void k_sparse_ternary(GenKey gk, u64 seed, u64 tag, int h, int N, int* idx, i64* s) {
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
        idx[j] = j;
        s[j] = 0;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    for (int i = 0; i < h; i++) {
        const u64 w = gen_word(gk, seed, tag, (u64)i);
        const int j = i + (int)(((u128)(w >> 1) * (u64)(N - i)) >> 63);
        const int t = idx[i];
        idx[i] = idx[j];
        idx[j] = t;
        s[idx[i]] = (w & 1) ? -1 : 1;
    }
}

// out[z][limb i] = centred(coef0[z]) mod q_i, i < nl (z over 2 n polynomials)
__global__ void k_mod_raise(const u64* coef0, u64* out, const Modulus* mods, u64 q0, int nl, int logN) {
    const int N = 1 << logN;
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const int i = blockIdx.y, z = blockIdx.z;
    const i64 v = centre(coef0[(size_t)z * N + n], q0);
    out[((size_t)z * nl + i) * N + n] = from_signed(v, mods[i].q);
}

// pair[z] = (x + cj, (x - cj) mono), z over n ciphertexts at nl limbs
__global__ void k_boot_parts(const u64* x, const u64* cj, const u64* mono, u64* pair, const Modulus* mods, int nl,
                             int logN) {
    const int N = 1 << logN;
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const int limb = blockIdx.y, z = blockIdx.z;  // limb over 2 nl
    const int i = limb % nl;
    const Modulus m = mods[i];
    const size_t o = ((size_t)z * 2 * nl + limb) * N + n;
    const u64 a = x[o], b = cj[o];
    pair[((size_t)(2 * z) * 2 * nl + limb) * N + n] = add_mod(a, b, m.q);
    pair[((size_t)(2 * z + 1) * 2 * nl + limb) * N + n] = mul_mod(sub_mod(a, b, m.q), mono[(size_t)i * N + n], m);
}

// complex form: v[z] = e[2z] + X^(N/2) e[2z+1] = e[2z] - mono e[2z+1] (slots e_re + i e_im),
// z over n ciphertexts at nl limbs, mono = NTT(-X^(N/2))
__global__ void k_boot_join(const u64* e, const u64* mono, u64* v, const Modulus* mods, int nl, int logN) {
    const int N = 1 << logN;
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const int limb = blockIdx.y, z = blockIdx.z;  // limb over 2 nl
    const int i = limb % nl;
    const Modulus m = mods[i];
    const u64 a = e[((size_t)(2 * z) * 2 * nl + limb) * N + n];
    const u64 b = e[((size_t)(2 * z + 1) * 2 * nl + limb) * N + n];
    v[((size_t)z * 2 * nl + limb) * N + n] = sub_mod(a, mul_mod(b, mono[(size_t)i * N + n], m), m.q);
}

// ---------------------------------------------------------------------------
// host helpers
// ---------------------------------------------------------------------------

int sk_gen_sparse(fe_ctx* c, uint64_t seed, uint32_t h, u64* sk, cudaStream_t st) {
    const int N = c->N;
    i64* s;
    int* idx;
    FE_CUDA_TRY(cudaMallocAsync(&s, (size_t)N * 8, st));
    FE_CUDA_TRY(cudaMallocAsync(&idx, (size_t)N * 4, st));
    k_sparse_ternary<<<1, 1024, 0, st>>>(c->gen, seed, make_tag(6, 0, 0, 0), (int)h, N, idx, s);
    c->cnt.launches++;
    launch_signed_to_limbs(c, s, sk, 0, c->n_mod, (size_t)N, st);
    ntt_forward(c, LimbSet{sk, (size_t)c->n_mod * N, c->n_mod, 1, c->d_identity_map}, st);
    FE_CUDA_TRY(cudaFreeAsync(s, st));
    FE_CUDA_TRY(cudaFreeAsync(idx, st));
    FE_CUDA_TRY(cudaGetLastError());
    return FE_OK;
}

// n level-0 ciphertexts [n][2][1][N] -> [n][2][top+1][N]; tmp: [2n][N]
void mod_raise(fe_ctx* c, const u64* in, int n, int top, u64* out, u64* tmp, cudaStream_t st) {
    const int N = c->N;
    ntt_inverse_from(c, in, (size_t)N, LimbSet{tmp, (size_t)N, 1, 2 * n, c->d_identity_map}, st);
    k_mod_raise<<<dim3((N + kB - 1) / kB, top + 1, 2 * n), kB, 0, st>>>(tmp, out, c->d_mod, c->mod[0], top + 1,
                                                                        c->logN);
    c->cnt.launches++;
    ntt_forward(c, LimbSet{out, (size_t)(top + 1) * N, top + 1, 2 * n, c->d_identity_map}, st);
}

struct ConjScratch {
    u64 *coef, *ext, *acc, *conv;
    KsItem* ks;
    CombineItem* cb;
};
void carve_conj(Carver& cv, const fe_ctx* c, int n, int level, ConjScratch* s) {
    s->coef = cv.take<u64>((size_t)n * (level + 1) * c->N);
    s->ext = cv.take<u64>((size_t)n * ext_words(c, level));
    s->acc = cv.take<u64>((size_t)n * acc_words(c, level));
    s->conv = cv.take<u64>((size_t)n * ct_words(c, level));
    s->ks = cv.take<KsItem>(n);
    s->cb = cv.take<CombineItem>(n);
}

// out = sigma_g((c0, 0) + KS_key(c1)) for n ciphertexts at `level` (g = 1: a plain
// key switch from the key's source secret to its destination secret)
int ks_batch(fe_ctx* c, const u64* key, uint32_t g, const u64* in, int n, int level, u64* out, const ConjScratch& s,
             cudaStream_t st) {
    const int N = c->N, nl = level + 1;
    std::vector<KsItem> ks(n);
    std::vector<CombineItem> cb(n);
    for (int i = 0; i < n; i++) {
        ks[i] = KsItem{s.ext + i * ext_words(c, level), key, s.acc + i * acc_words(c, level)};
        cb[i] = CombineItem{s.acc + i * acc_words(c, level), s.conv + i * ct_words(c, level),
                            in + i * ct_words(c, level), nullptr, out + i * ct_words(c, level), g, 0};
    }
    FE_TRY(upload(ks, s.ks, st));
    FE_TRY(upload(cb, s.cb, st));
    modup(c, in + (size_t)nl * N, ct_words(c, level), n, level, s.coef, s.ext, st);
    launch_keyip(c, s.ks, n, level, st);
    moddown_prepare(c, s.acc, n, level, s.conv, st);
    launch_combine(c, s.cb, n, level, st);
    c->cnt.keyswitch += n;
    return FE_OK;
}

// out = sigma_{2N-1}(in) with its key switch, n ciphertexts at `level` (the
// rotation of Eq. 1 with the conjugation's Galois element)
int conjugate_batch(fe_ctx* c, const fe_evk* evk, const u64* in, int n, int level, u64* out, const ConjScratch& s,
                    cudaStream_t st) {
    const uint32_t g = c->galois(FE_STEP_CONJ);
    const u64* key = evk_key(evk, g);
    if (!key) return fail(FE_EKEY, "missing conjugation key (step FE_STEP_CONJ)");
    FE_TRY(ks_batch(c, key, g, in, n, level, out, s, st));
    c->cnt.rot += n;
    return FE_OK;
}

// ---------------------------------------------------------------------------
// plaintext-matrix products by the diagonal method with baby / giant steps
// ---------------------------------------------------------------------------

struct LtDiag {
    int out, in;
    int32_t off;
};

// Every offset r = giant + baby: r_lo = min, delta = gcd of r - r_lo (1 when
// all are equal), j = (r - r_lo) / delta, baby = (j mod n1) delta,
// giant = r_lo + (j div n1) n1 delta.
void bsgs_split(const std::vector<int32_t>& offs, int n1, std::map<int32_t, std::pair<int32_t, int32_t>>& dec) {
    const int32_t lo = *std::min_element(offs.begin(), offs.end());
    int64_t delta = 0;
    for (int32_t r : offs) delta = std::gcd(delta, (int64_t)r - lo);
    if (!delta) delta = 1;
    for (int32_t r : offs) {
        const int64_t j = ((int64_t)r - lo) / delta;
        dec[r] = {(int32_t)(lo + (j / n1) * n1 * delta), (int32_t)((j % n1) * delta)};
    }
}

// An FC-kind plan computing out[o] = rescale(sum_{(o, i, r)} d ⊙ Rot(in[i], r)):
// inner rotations = baby steps of each input, one group per (output, giant
// step) whose plaintexts are the diagonals rotated by -giant.  pt_src[k] =
// (diagonal index, giant step) of the plan's k-th plaintext.
int plan_lintrans(fe_ctx* c, int n_in, int n_out, const std::vector<LtDiag>& d, int n1, int level,
                  std::unique_ptr<fe_plan>& p, std::vector<std::pair<int, int32_t>>& pt_src) {
    const int n = c->N / 2;
    if (level < 1 || level > c->L) return fail(FE_ELEVEL, "a plaintext-matrix product needs a level to rescale");
    if (n_in < 1 || n_out < 1 || d.empty() || n1 < 1) return fail(FE_EINVAL, "empty plaintext-matrix product");
    std::set<std::tuple<int, int, int32_t>> seen;
    std::vector<int32_t> offs;
    std::vector<int> has_out(n_out, 0);
    for (const LtDiag& x : d) {
        if (x.out < 0 || x.out >= n_out || x.in < 0 || x.in >= n_in) return fail(FE_EINVAL, "diagonal index out of range");
        if (x.off <= -n || x.off >= n) return fail(FE_EINVAL, "diagonal offset outside (-N/2, N/2)");
        if (!seen.insert({x.out, x.in, x.off}).second) return fail(FE_EINVAL, "duplicate diagonal");
        offs.push_back(x.off);
        has_out[x.out] = 1;
    }
    for (int o = 0; o < n_out; o++)
        if (!has_out[o]) return fail(FE_EINVAL, "an output with no diagonal");
    std::map<int32_t, std::pair<int32_t, int32_t>> dec;
    bsgs_split(offs, n1, dec);
    p.reset(new fe_plan());
    p->c = c;
    p->kind = 1;
    p->level = level;
    p->n_in = n_in;
    p->n_out = n_out;
    p->P = n;
    p->BS = 1;
    p->n1 = n1;
    p->lintrans = 1;
    auto mod_n = [n](int64_t v) { return (int32_t)(((v % n) + n) % n); };
    std::map<std::pair<int, int32_t>, int> rslot;
    for (int i = 0; i < n_in; i++) {
        std::set<int32_t> babies;
        for (const LtDiag& x : d)
            if (x.in == i && mod_n(dec[x.off].second)) babies.insert(dec[x.off].second);
        for (int32_t b : babies) {
            rslot[{i, b}] = (int)p->inner.size();
            p->inner.push_back({i, b});
        }
    }
    p->outs.resize(n_out);
    pt_src.clear();
    for (int o = 0; o < n_out; o++) {
        std::map<int32_t, std::vector<int>> by_giant;
        for (int k = 0; k < (int)d.size(); k++)
            if (d[k].out == o) by_giant[dec[d[k].off].first].push_back(k);
        for (auto& kv : by_giant) {
            fe_plan::Group grp{mod_n(kv.first) ? kv.first : 0, (int)p->terms.size(), 0};
            for (int k : kv.second) {
                const int32_t b = dec[d[k].off].second;
                const int src = mod_n(b) ? rslot.at({d[k].in, b}) : -(d[k].in + 1);
                p->terms.push_back({src, p->n_pt++});
                pt_src.push_back({k, kv.first});
                grp.nt++;
            }
            p->outs[o].groups.push_back(grp);
        }
    }
    finish_plan(p.get());
    return FE_OK;
}

// plaintext k = diagonal pt_src[k].first rotated by -giant, encoded at w_scale
// on q_0..q_level (and p_0..p_{k-1} when the plan is double-hoisted) and stored
// compact at pt_dev
// (diag_im: imaginary parts of complex diagonals, or null for real ones)
int load_lintrans(fe_ctx* c, const fe_plan* p, const std::vector<std::pair<int, int32_t>>& pt_src,
                  const std::vector<const double*>& diag_vals, double w_scale, void* pt_dev, cudaStream_t st,
                  const std::vector<const double*>* diag_im = nullptr) {
    const int N = c->N, n = N / 2, nl = p->level + 1 + (p->dhoist ? c->k : 0);
    const int chunk = std::max(1, std::min({p->n_pt, (int)((64ull << 20) / ((size_t)n * 8)),
                                            (int)((1ull << 30) / ((size_t)nl * N * 8))}));
    double *z, *zi = nullptr;
    u64* limbs;
    FE_CUDA_TRY(cudaMallocAsync(&z, (size_t)chunk * n * 8, st));
    if (diag_im) FE_CUDA_TRY(cudaMallocAsync(&zi, (size_t)chunk * n * 8, st));
    FE_CUDA_TRY(cudaMallocAsync(&limbs, (size_t)chunk * nl * N * 8, st));
    std::vector<double> host((size_t)chunk * n), host_im(diag_im ? (size_t)chunk * n : 0);
    int rc = FE_OK;
    for (int s0 = 0; s0 < p->n_pt && rc == FE_OK; s0 += chunk) {
        const int cn = std::min(chunk, p->n_pt - s0);
        for (int k = 0; k < cn; k++) {
            const double* v = diag_vals[pt_src[s0 + k].first];
            const int64_t g = pt_src[s0 + k].second;
            double* dst = host.data() + (size_t)k * n;
            for (int l = 0; l < n; l++) dst[l] = v[(((l - g) % n) + n) % n];  // Rot(d, -g)
            if (diag_im) {
                const double* vi = (*diag_im)[pt_src[s0 + k].first];
                double* di = host_im.data() + (size_t)k * n;
                for (int l = 0; l < n; l++) di[l] = vi[(((l - g) % n) + n) % n];
            }
        }
        FE_CUDA_TRY(cudaMemcpyAsync(z, host.data(), (size_t)cn * n * 8, cudaMemcpyHostToDevice, st));
        if (diag_im) FE_CUDA_TRY(cudaMemcpyAsync(zi, host_im.data(), (size_t)cn * n * 8, cudaMemcpyHostToDevice, st));
        rc = encode_batch(c, z, cn, p->level, w_scale, limbs, st, p->dhoist != 0, zi);
        if (rc == FE_OK) launch_pt_compact(c, limbs, (uint8_t*)pt_dev + (size_t)s0 * nl * pt_limb_bytes(c), cn * nl, st);
        FE_CUDA_TRY(cudaStreamSynchronize(st));  // the host staging buffer is refilled next
    }
    cudaFreeAsync(z, st);
    if (zi) cudaFreeAsync(zi, st);
    cudaFreeAsync(limbs, st);
    FE_CUDA_TRY(cudaStreamSynchronize(st));
    return rc;
}

// ---------------------------------------------------------------------------
// the special FFT's stages (correctly rounded twiddles)
// ---------------------------------------------------------------------------

struct Trig {
    int N;
    std::vector<double> tab;  // cos(pi e / N), e in [0, N/2]
    explicit Trig(int N_) : N(N_), tab(N_ / 2 + 1) {
        for (int e = 0; e <= N / 2; e++) tab[e] = boot_cos_pi_table_entry(N, e);
    }
    // cos(pi e / N) by cos(-a) = cos(a), cos(a + 2 pi) = cos(a), cos(pi - a) = -cos(a)
    double cos_pi(int64_t e) const {
        e = ((e % (2 * N)) + 2 * N) % (2 * N);
        if (e > N) e = 2 * N - e;
        return e > N / 2 ? -tab[N - e] : tab[e];
    }
    double sin_pi(int64_t e) const { return cos_pi((int64_t)N / 2 - e); }
};

// exponents of zeta in the twiddles of stage s at positions p < 2^(s-1):
// zeta_(m)^(5^p), m = 2^s, zeta_(m) = zeta^(N / (2m))
std::vector<int64_t> stage_taus(int N, int s) {
    const int64_t m = 1ll << s, h = m >> 1;
    std::vector<int64_t> t(h);
    int64_t e = 1;  // 5^p mod 4m
    for (int64_t p = 0; p < h; p++) {
        t[p] = (e * (N / (2 * m))) % (2 * (int64_t)N);
        e = (e * 5) % (4 * m);
    }
    return t;
}

// entry (o, i) of S_s or S_s^-1 as (exponent mod 2N, halvings); false where zero
//   S_s, p = o mod m, h = m/2:  p < h: out[o] = in[o] + zeta^tau(p) in[o + h];
//                               p >= h: out[o] = in[o - h] - zeta^tau(p - h) in[o]
//   S_s^-1:  p < h: in[o] = (out[o] + out[o + h]) / 2;
//            p >= h: in[o] = zeta^-tau(p - h) (out[o - h] - out[o]) / 2
bool stage_entry(int N, int s, bool inverse, int64_t o, int64_t i, const std::vector<int64_t>& tau, int64_t* e,
                 int* hv) {
    const int64_t m = 1ll << s, h = m >> 1;
    if (o / m != i / m) return false;
    const int64_t p = o % m, pi = i % m, twoN = 2 * (int64_t)N;
    if (!inverse) {
        *hv = 0;
        if (p < h) {
            if (pi == p) { *e = 0; return true; }
            if (pi == p + h) { *e = tau[p]; return true; }
        } else {
            if (pi == p - h) { *e = 0; return true; }
            if (pi == p) { *e = (tau[p - h] + N) % twoN; return true; }
        }
        return false;
    }
    *hv = 1;
    if (p < h) {
        if (pi == p || pi == p + h) { *e = 0; return true; }
        return false;
    }
    const int64_t t = tau[p - h];
    if (pi == p - h) { *e = (twoN - t) % twoN; return true; }
    if (pi == p) { *e = ((N - t) % twoN + twoN) % twoN; return true; }
    return false;
}

// stages 1..k in n_groups consecutive ranges, the larger ranges at the top
std::vector<std::vector<int>> stage_groups(int k, int n_groups) {
    std::vector<std::vector<int>> out;
    const int base = k / n_groups, extra = k % n_groups;
    int s = 1;
    for (int g = 0; g < n_groups; g++) {
        const int sz = base + (g >= n_groups - extra ? 1 : 0);
        std::vector<int> grp;
        for (int j = 0; j < sz; j++) grp.push_back(s + j);
        s += sz;
        out.push_back(grp);
    }
    return out;
}

// distinct offsets of a group mod n, as representatives in (-n/2, n/2]
std::vector<int32_t> group_offsets(const std::vector<int>& stages, int n) {
    const int64_t lo = 1ll << (*std::min_element(stages.begin(), stages.end()) - 1);
    const int64_t span = (1ll << stages.size()) - 1, half = n / 2;
    std::set<int32_t> out;
    for (int64_t j = -span; j <= span; j++) out.insert((int32_t)((((j * lo + half - 1) % n) + n) % n - (half - 1)));
    return std::vector<int32_t>(out.begin(), out.end());
}

// baby steps: the smallest power of two n1 with n1^2 >= ratio x the number of offsets
int default_n1(size_t n_offsets, uint32_t ratio = 1) {
    int n1 = 1;
    while ((size_t)n1 * n1 < (size_t)std::max<uint32_t>(1, ratio) * n_offsets) n1 *= 2;
    return n1;
}

// Real-form diagonals of one group (stages in the order applied): for parts = 2
// (re', im') = (Re G re - Im G im, Im G re + Re G im), for parts = 1 re' only;
// d_r[o] = G[o][(o + r) mod n] = sign 2^-halvings cis(pi e / N), times kappa in
// one IEEE product when kappa != 1; all-zero vectors are left out.
// parts = 0: the complex form, one diagonal (0, 0, r) per offset with its real
// parts in vals and imaginary parts in vals_im (left out when both are zero).
void group_diagonals(int N, const Trig& tr, const std::vector<int>& stages, bool inverse, double kappa, int parts,
                     std::vector<LtDiag>& diags, std::vector<std::vector<double>>& vals,
                     std::vector<std::vector<double>>* vals_im = nullptr) {
    const int n = N / 2;
    int bits = 0;
    for (int s : stages) bits |= 1 << (s - 1);
    std::vector<std::vector<int64_t>> taus(stages.size());
    for (size_t a = 0; a < stages.size(); a++) taus[a] = stage_taus(N, stages[a]);
    for (int32_t r : group_offsets(stages, n)) {
        std::vector<double> re(n, 0.0), im(n, 0.0);
        for (int64_t o = 0; o < n; o++) {
            const int64_t i0 = ((o + r) % n + n) % n;
            if ((o ^ i0) & ~(int64_t)bits) continue;
            int64_t x = i0, e = 0;
            int hv = 0;
            bool ok = true;
            for (size_t a = 0; a < stages.size() && ok; a++) {
                const int64_t b = 1ll << (stages[a] - 1);
                const int64_t y = (x & ~b) | (o & b);
                int64_t ee;
                int hh;
                ok = stage_entry(N, stages[a], inverse, y, x, taus[a], &ee, &hh);
                e += ee;
                hv += hh;
                x = y;
            }
            if (!ok) continue;
            e %= 2 * (int64_t)N;
            double cv = std::ldexp(tr.cos_pi(e), -hv), sv = std::ldexp(tr.sin_pi(e), -hv);
            if (kappa != 1.0) {
                cv = cv * kappa;
                sv = sv * kappa;
            }
            re[o] = cv;
            im[o] = sv;
        }
        auto nonzero = [](const std::vector<double>& v) {
            for (double a : v)
                if (a != 0.0) return true;
            return false;
        };
        if (parts == 0) {
            if (nonzero(re) || nonzero(im)) {
                diags.push_back({0, 0, r});
                vals.push_back(re);
                vals_im->push_back(im);
            }
            continue;
        }
        std::vector<double> nim(n);
        for (int o = 0; o < n; o++) nim[o] = -im[o];
        const std::vector<std::pair<std::pair<int, int>, const std::vector<double>*>> cand =
            parts == 2 ? std::vector<std::pair<std::pair<int, int>, const std::vector<double>*>>{
                             {{0, 0}, &re}, {{0, 1}, &nim}, {{1, 0}, &im}, {{1, 1}, &re}}
                       : std::vector<std::pair<std::pair<int, int>, const std::vector<double>*>>{{{0, 0}, &re},
                                                                                                {{0, 1}, &nim}};
        for (auto& cd : cand)
            if (nonzero(*cd.second)) {
                diags.push_back({cd.first.first, cd.first.second, r});
                vals.push_back(*cd.second);
            }
    }
}

// Taylor coefficients of cos in w = x^2: a_k = (-1)^k / (2k)!, correctly rounded
// ((2k)! <= 16! is exact in a double, so the quotient is one rounding)
double taylor_a(int k) {
    double f = 1.0;
    for (int i = 2; i <= 2 * k; i++) f *= (double)i;
    return (k & 1 ? -1.0 : 1.0) / f;
}

// ---------------------------------------------------------------------------
// EvalMod on ciphertexts with declared scales
// ---------------------------------------------------------------------------

struct Ev {
    u64* p;
    int level;
    double scale;
};

struct EvCtx {
    fe_ctx* c;
    const fe_evk* evk;
    int n;  // ciphertexts per operand
    cudaStream_t st;
    Carver* scratch;  // per-operation scratch (reset after each operation)
    char* scratch_base;
    size_t scratch_bytes;
    bool launch = true;  // false: levels, scales and buffers only (no launch)
};

size_t ct_bytes(const fe_ctx* c, int n, int level) { return (size_t)n * ct_words(c, level) * 8; }

// relin(a (x) b) rescaled: scale (s_a s_b) / q_level
int ev_mul(EvCtx& e, const Ev& a, const Ev& b, Ev& out) {
    fe_ctx* c = e.c;
    const int lv = a.level;
    Carver cv(e.scratch_base, e.scratch_bytes);
    u64* d = cv.take<u64>((size_t)e.n * ct_words(c, lv));
    u64* tmp = cv.take<u64>(rescale_tmp_words(c, e.n, lv));
    if (!cv.ok) return fail(FE_ENOMEM, "bootstrap workspace too small");
    if (e.launch) {
        FE_TRY(cmult_relin(c, e.evk, a.p, b.p, e.n, lv, d, cv, e.st));
        rescale_batch(c, d, e.n, lv, out.p, tmp, tmp + 2 * (size_t)e.n * c->N, e.st);
    }
    out.level = lv - 1;
    out.scale = (a.scale * b.scale) / (double)c->mod[lv];
    return FE_OK;
}

// value times coef at declared scale s_t: K = nearest(((coef s_t) q_level) / s), ct K rescaled
int ev_cmul(EvCtx& e, const Ev& a, double coef, double s_t, Ev& out) {
    fe_ctx* c = e.c;
    const int lv = a.level;
    Carver cv(e.scratch_base, e.scratch_bytes);
    u64* d = cv.take<u64>((size_t)e.n * ct_words(c, lv));
    u64* tmp = cv.take<u64>(rescale_tmp_words(c, e.n, lv));
    if (!cv.ok) return fail(FE_ENOMEM, "bootstrap workspace too small");
    const double x = ((coef * s_t) * (double)c->mod[lv]) / a.scale;
    AffineConsts k{};
    for (int i = 0; i <= lv; i++) k.mul[i] = nearest_mod(x, c->mod[i]);
    if (e.launch) {
        FE_TRY(launch_affine(c, a.p, d, e.n, lv, k, true, e.st));
        rescale_batch(c, d, e.n, lv, out.p, tmp, tmp + 2 * (size_t)e.n * c->N, e.st);
    }
    out.level = lv - 1;
    out.scale = s_t;
    return FE_OK;
}

// in place: value times mul (an integer, 1 for none) plus coef: K = nearest(coef s)
int ev_affine(EvCtx& e, Ev& a, int64_t mul, double coef) {
    fe_ctx* c = e.c;
    AffineConsts k{};
    const double x = coef * a.scale;
    for (int i = 0; i <= a.level; i++) {
        const u64 q = c->mod[i];
        k.mul[i] = mul >= 0 ? (u64)mul % q : q - (u64)(-mul) % q;
        k.add[i] = nearest_mod(x, q);
    }
    return e.launch ? launch_affine(c, a.p, a.p, e.n, a.level, k, mul != 1, e.st) : FE_OK;
}

// the first (level + 1 - times) limbs of each polynomial
int ev_drop(EvCtx& e, const Ev& a, int times, Ev& out) {
    const fe_ctx* c = e.c;
    const int nl = a.level + 1 - times;
    if (e.launch && (out.p != a.p || times)) {
        FE_CUDA_TRY(cudaMemcpy2DAsync(out.p, (size_t)nl * c->N * 8, a.p, (size_t)(a.level + 1) * c->N * 8,
                                      (size_t)nl * c->N * 8, 2 * (size_t)e.n, cudaMemcpyDeviceToDevice, e.st));
    }
    out.level = a.level - times;
    out.scale = a.scale;
    return FE_OK;
}

int ev_add(EvCtx& e, Ev& acc, const Ev& b) {
    if (e.launch) launch_add(e.c, acc.p, b.p, acc.p, e.n, acc.level, e.st);
    return FE_OK;
}

// sin(2 pi y) from x = (pi / 2^(r-1)) y, 5 + r levels (same steps and constants as
// the oracle's eval_mod); bufs: 8 ciphertext arrays of n ciphertexts at x's level
int eval_mod(EvCtx& e, Ev x, int r, u64* const* bufs, Ev& result) {
    double a[9];
    for (int k = 0; k <= 8; k++) a[k] = taylor_a(k);
    const double s0 = x.scale;
    FE_TRY(ev_affine(e, x, 1, -std::ldexp(M_PI, -(r + 1))));
    Ev w{bufs[0]}, w2{bufs[1]}, w3{bufs[2]}, w4{bufs[3]}, q1{bufs[4]}, t{bufs[5]}, t2{bufs[6]}, p{bufs[7]};
    FE_TRY(ev_mul(e, x, x, w));
    FE_TRY(ev_mul(e, w, w, w2));
    FE_TRY(ev_drop(e, w, 1, t));
    FE_TRY(ev_mul(e, w2, t, w3));
    FE_TRY(ev_mul(e, w2, w2, w4));
    // q1 = a4 + a5 w + a6 w2 + a7 w3 + a8 w4 at declared scale s0
    FE_TRY(ev_cmul(e, w, a[5], s0, t));
    FE_TRY(ev_drop(e, t, 2, q1));
    FE_TRY(ev_cmul(e, w2, a[6], s0, t));
    FE_TRY(ev_drop(e, t, 1, t2));
    FE_TRY(ev_add(e, q1, t2));
    FE_TRY(ev_cmul(e, w3, a[7], s0, t));
    FE_TRY(ev_add(e, q1, t));
    FE_TRY(ev_cmul(e, w4, a[8], s0, t));
    FE_TRY(ev_add(e, q1, t));
    FE_TRY(ev_affine(e, q1, 1, a[4]));
    const double sc = (w4.scale * s0) / (double)e.c->mod[q1.level];
    FE_TRY(ev_drop(e, w4, 1, t2));
    FE_TRY(ev_mul(e, t2, q1, p));
    FE_TRY(ev_cmul(e, w, a[1], sc, t));
    FE_TRY(ev_drop(e, t, 3, t2));
    FE_TRY(ev_add(e, p, t2));
    FE_TRY(ev_cmul(e, w2, a[2], sc, t));
    FE_TRY(ev_drop(e, t, 2, t2));
    FE_TRY(ev_add(e, p, t2));
    FE_TRY(ev_cmul(e, w3, a[3], sc, t));
    FE_TRY(ev_drop(e, t, 1, t2));
    FE_TRY(ev_add(e, p, t2));
    FE_TRY(ev_affine(e, p, 1, a[0]));
    // r double angles c <- 2 c^2 - 1, alternating between p and t
    Ev cur = p, nxt = t;
    for (int i = 0; i < r; i++) {
        FE_TRY(ev_mul(e, cur, cur, nxt));
        FE_TRY(ev_affine(e, nxt, 2, -1.0));
        std::swap(cur, nxt);
    }
    result = cur;
    return FE_OK;
}

// ---------------------------------------------------------------------------
// the refresh: buffers carved in one pass (dry: sizes only).  phase bit 1
// uploads the transforms' item tables, bit 2 launches; every transform keeps
// its tables in a region of its own, so that the launches of phase 2 alone can
// be captured in a graph after phase 1 (fe_boot_graph_capture).
// ---------------------------------------------------------------------------

int boot_run(fe_ctx* c, const fe_evk* evk, const fe_boot* b, const u64* in, int R, u64* out, void* ws,
             size_t ws_bytes, cudaStream_t st, bool dry, size_t* need, int phase = 3) {
    const int N = c->N, top = b->top;
    const bool L = (phase & 2) != 0;
    Carver cv(dry ? nullptr : ws, dry ? SIZE_MAX : ws_bytes);
    u64* raised = cv.take<u64>((size_t)R * ct_words(c, top));
    u64* cj = cv.take<u64>((size_t)R * ct_words(c, top));
    u64* pa = cv.take<u64>(2 * (size_t)R * ct_words(c, top));
    u64* pb = cv.take<u64>(2 * (size_t)R * ct_words(c, top));
    u64* tmp = cv.take<u64>(2 * (size_t)R * N);
    ConjScratch cs;
    carve_conj(cv, c, R, top, &cs);
    const int lv0 = top - b->n_cts;
    u64* bufs[8];
    for (int i = 0; i < 8; i++) bufs[i] = cv.take<u64>(2 * (size_t)R * ct_words(c, lv0));
    // the transforms' data region (rotated copies, sums, scratch), shared with
    // EvalMod, and one item-table region per transform
    size_t data = 0;
    for (auto& p : b->plans) {
        const size_t def = fe_plan_workspace_bytes(p.get(), (uint32_t)R, 0);
        data = std::max(data, plan_data_bytes(p.get(), plan_chunk(p.get(), R, 1, def, false), R));
    }
    data = (data + 255) & ~(size_t)255;
    const size_t ev_ws = cmult_relin_bytes(c, 2 * R, lv0) + ct_bytes(c, 2 * R, lv0) +
                         rescale_tmp_words(c, 2 * R, lv0) * 8 + 8 * 256;
    const size_t shared_bytes = std::max(data, ev_ws);
    char* shared = cv.take<char>(shared_bytes);
    std::vector<char*> tab(b->plans.size());
    std::vector<size_t> tab_bytes(b->plans.size());
    for (size_t i = 0; i < b->plans.size(); i++) {
        const fe_plan* p = b->plans[i].get();
        tab_bytes[i] = (plan_table_bytes(p, plan_chunk(p, R, 1, data, true), R) + 255) & ~(size_t)255;
        tab[i] = cv.take<char>(tab_bytes[i]);
    }
    if (dry) {
        *need = SIZE_MAX - cv.left;
        return FE_OK;
    }
    if (!cv.ok) return fail(FE_ENOMEM, "bootstrap workspace too small (fe_boot_workspace_bytes)");
    auto transform = [&](size_t pi, const u64* src, u64* dst) {
        return run_plan(c, evk, b->plans[pi].get(), src, b->pts[pi], dst, tab[pi], tab_bytes[pi], 1, st, phase, R, 0,
                        shared, data);
    };
    if (L) {
        if (b->key_to_sparse) {
            // the level-0 inputs (dense secret) switched to the sparse secret (into pb), raised
            // (into cj), switched back to the dense secret at level top (into raised)
            FE_TRY(ks_batch(c, b->key_to_sparse, 1, in, R, 0, pb, cs, st));
            mod_raise(c, pb, R, top, cj, tmp, st);
            FE_TRY(ks_batch(c, b->key_to_dense, 1, cj, R, top, raised, cs, st));
        } else {
            mod_raise(c, in, R, top, raised, tmp, st);
        }
    }
    EvCtx e{c, evk, 2 * R, st, nullptr, shared, shared_bytes};
    e.launch = L;
    if (b->form == 1) {
        // complex form: CoeffToSlot on the raised ciphertexts, the split at lv0,
        // EvalMod, the join, SlotToCoeff (every transform one in, one out)
        u64* x = raised;
        size_t pi = 0;
        for (; pi < (size_t)b->n_cts; pi++) {
            u64* dst = x == pa ? pb : pa;
            FE_TRY(transform(pi, x, dst));
            x = dst;
        }
        u64* pair = x == pa ? pb : pa;
        if (L) {
            FE_TRY(conjugate_batch(c, evk, x, R, lv0, cj, cs, st));
            k_boot_parts<<<dim3((N + kB - 1) / kB, 2 * (lv0 + 1), R), kB, 0, st>>>(x, cj, b->mono, pair, c->d_mod,
                                                                                  lv0 + 1, c->logN);
            c->cnt.launches++;
            FE_CUDA_TRY(cudaGetLastError());
        }
        Ev xe{pair, lv0, (double)c->mod[0]}, y{};
        FE_TRY(eval_mod(e, xe, b->r, bufs, y));
        if (y.scale != b->out_scale || y.level != top - b->n_cts - 5 - b->r)
            return fail(FE_EINVAL, "bootstrap: EvalMod scale bookkeeping disagrees with the plan");
        u64* v = x;  // the CoeffToSlot output is no longer needed
        if (L) {
            k_boot_join<<<dim3((N + kB - 1) / kB, 2 * (y.level + 1), R), kB, 0, st>>>(y.p, b->mono, v, c->d_mod,
                                                                                     y.level + 1, c->logN);
            c->cnt.launches++;
            FE_CUDA_TRY(cudaGetLastError());
        }
        u64* cur = v;
        for (; pi < b->plans.size(); pi++) {
            const bool last = pi + 1 == b->plans.size();
            u64* dst = last ? out : (cur == pa ? pb : pa);
            FE_TRY(transform(pi, cur, dst));
            cur = dst;
        }
        return FE_OK;
    }
    if (L) {
        FE_TRY(conjugate_batch(c, evk, raised, R, top, cj, cs, st));
        k_boot_parts<<<dim3((N + kB - 1) / kB, 2 * (top + 1), R), kB, 0, st>>>(raised, cj, b->mono, pa, c->d_mod,
                                                                              top + 1, c->logN);
        c->cnt.launches++;
        FE_CUDA_TRY(cudaGetLastError());
    }
    size_t pi = 0;
    for (; pi < (size_t)b->n_cts; pi++) {
        FE_TRY(transform(pi, pa, pb));
        std::swap(pa, pb);
    }
    // EvalMod on the 2R parts (pa holds [R][2] ciphertexts at lv0, i.e. 2R in a row)
    Ev x{pa, lv0, (double)c->mod[0]}, y{};
    FE_TRY(eval_mod(e, x, b->r, bufs, y));
    if (y.scale != b->out_scale || y.level != top - b->n_cts - 5 - b->r)
        return fail(FE_EINVAL, "bootstrap: EvalMod scale bookkeeping disagrees with the plan");
    const u64* cur = y.p;
    for (; pi < b->plans.size(); pi++) {
        const bool last = pi + 1 == b->plans.size();
        u64* dst = last ? out : (cur == pa ? pb : pa);
        FE_TRY(transform(pi, cur, dst));
        cur = dst;
    }
    return FE_OK;
}

}  // namespace
}  // namespace fe

using namespace fe;

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------

extern "C" int fe_sk_gen_sparse(fe_ctx* c, uint64_t seed, uint32_t h, void* sk_dev, void* stream) {
    FE_ALIGNED(sk_dev);
    if (!c || !sk_dev) return fail(FE_EINVAL, "null argument");
    if (h == 0 || h > (uint32_t)c->N) return fail(FE_EINVAL, "hamming weight must be in [1, N]");
    return sk_gen_sparse(c, seed, h, (u64*)sk_dev, (cudaStream_t)stream);
}

extern "C" int fe_conjugate(fe_ctx* c, const fe_evk* evk, const void* ct_dev, uint32_t n_ct, uint32_t level,
                            void* out_dev, void* stream) {
    return fe_rotate(c, evk, ct_dev, n_ct, level, FE_STEP_CONJ, out_dev, stream);
}

extern "C" int fe_mod_drop(fe_ctx* c, const void* ct_dev, uint32_t n_ct, uint32_t level, uint32_t to_level,
                           void* out_dev, void* stream) {
    FE_ALIGNED(ct_dev);
    FE_ALIGNED(out_dev);
    if (!c || !ct_dev || !out_dev) return fail(FE_EINVAL, "null argument");
    if ((int)level > c->L || to_level > level) return fail(FE_ELEVEL, "levels must satisfy to_level <= level <= L");
    if (n_ct == 0) return FE_OK;
    if (ct_dev == out_dev && to_level != level) return fail(FE_EINVAL, "a level drop cannot run in place");
    const size_t N = (size_t)c->N, nl = (size_t)to_level + 1;
    // each polynomial keeps its first to_level + 1 limbs (rows of 2 n_ct polynomials)
    FE_CUDA_TRY(cudaMemcpy2DAsync(out_dev, nl * N * 8, ct_dev, ((size_t)level + 1) * N * 8, nl * N * 8, 2 * (size_t)n_ct,
                                  cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
    return FE_OK;
}

extern "C" int fe_mod_raise(fe_ctx* c, const void* ct_dev, uint32_t n_ct, uint32_t top, void* out_dev, void* stream) {
    FE_ALIGNED(ct_dev);
    FE_ALIGNED(out_dev);
    if (!c || !ct_dev || !out_dev) return fail(FE_EINVAL, "null argument");
    if ((int)top > c->L) return fail(FE_ELEVEL, "level above L");
    if (n_ct == 0) return FE_OK;
    cudaStream_t st = (cudaStream_t)stream;
    u64* tmp;
    FE_CUDA_TRY(cudaMallocAsync(&tmp, 2 * (size_t)n_ct * c->N * 8, st));
    mod_raise(c, (const u64*)ct_dev, (int)n_ct, (int)top, (u64*)out_dev, tmp, st);
    cudaFreeAsync(tmp, st);
    FE_CUDA_TRY(cudaGetLastError());
    return FE_OK;
}

extern "C" int fe_plan_lintrans(fe_ctx* c, uint32_t n_in, uint32_t n_out, uint32_t n_diag, const uint32_t* diag_out,
                                const uint32_t* diag_in, const int32_t* diag_offset, uint32_t n1, uint32_t level,
                                fe_plan** out) {
    if (!c || !out || (n_diag && (!diag_out || !diag_in || !diag_offset))) return fail(FE_EINVAL, "null argument");
    std::vector<LtDiag> d(n_diag);
    std::set<int32_t> offs;
    for (uint32_t k = 0; k < n_diag; k++) {
        d[k] = LtDiag{(int)diag_out[k], (int)diag_in[k], diag_offset[k]};
        offs.insert(diag_offset[k]);
    }
    std::unique_ptr<fe_plan> p;
    std::vector<std::pair<int, int32_t>> src;
    FE_TRY(plan_lintrans(c, (int)n_in, (int)n_out, d, n1 ? (int)n1 : default_n1(offs.size()), (int)level, p, src));
    p->lt_src = src;
    p->lt_ndiag = n_diag;
    *out = p.release();
    return FE_OK;
}

extern "C" int fe_plan_lintrans_load(fe_ctx* c, fe_plan* p, const double* values_host, double w_scale, void* pt_dev,
                                     void* stream) {
    FE_ALIGNED(pt_dev);
    if (!c || !p || !values_host || !pt_dev) return fail(FE_EINVAL, "null argument");
    if (!p->lintrans) return fail(FE_EINVAL, "not a plaintext-matrix plan");
    if (p->c != c) return fail(FE_EINVAL, "the plan belongs to another context");
    const size_t n = (size_t)c->N / 2;
    std::vector<const double*> vals(p->lt_ndiag);
    for (size_t k = 0; k < vals.size(); k++) vals[k] = values_host + k * n;
    FE_TRY(load_lintrans(c, p, p->lt_src, vals, w_scale, pt_dev, (cudaStream_t)stream));
    p->w_scale = w_scale;
    return FE_OK;
}

extern "C" int fe_he_lintrans(fe_ctx* c, const fe_evk* evk, const fe_plan* p, const void* pt_dev, const void* in_dev,
                              void* out_dev, uint32_t n_req, void* ws, size_t ws_bytes, void* stream) {
    FE_ALIGNED(pt_dev); FE_ALIGNED(in_dev); FE_ALIGNED(out_dev); FE_ALIGNED(ws);
    if (!c || !evk || !p || !pt_dev || !in_dev || !out_dev || !ws) return fail(FE_EINVAL, "null argument");
    if (!p->lintrans) return fail(FE_EINVAL, "not a plaintext-matrix plan");
    if (n_req == 0) return FE_OK;
    return run_plan(c, evk, p, (const u64*)in_dev, (const u64*)pt_dev, (u64*)out_dev, ws, ws_bytes, 1,
                    (cudaStream_t)stream, 3, (int)n_req);
}

extern "C" int fe_boot_create(fe_ctx* c, const fe_boot_params* prm, double scale_in, void* stream, fe_boot** out) {
    if (!c || !prm || !out) return fail(FE_EINVAL, "null argument");
    const int N = c->N, n = N / 2;
    int k = 0;
    while ((1 << k) < n) k++;
    const int n_cts = (int)prm->n_cts, n_stc = (int)prm->n_stc, r = (int)prm->r;
    const int top = prm->top ? (int)prm->top : c->L;
    if (n_cts < 1 || n_cts > k || n_stc < 1 || n_stc > k || r < 1 || r > 16)
        return fail(FE_EINVAL, "bootstrap parameters: 1 <= groups <= log2(N/2), 1 <= r <= 16");
    if (top > c->L) return fail(FE_ELEVEL, "top level above L");
    if (n_cts + 5 + r + n_stc > top) return fail(FE_ELEVEL, "the refresh needs n_cts + 5 + r + n_stc levels below top");
    if (!(scale_in > 0)) return fail(FE_EINVAL, "scale_in must be positive");
    if (top + 1 > kMaxAffineLimbs) return fail(FE_EINVAL, "more limbs than the EvalMod kernels hold");
    cudaStream_t st = (cudaStream_t)stream;
    std::unique_ptr<fe_boot> b(new fe_boot());
    b->c = c;
    b->n_cts = n_cts;
    b->n_stc = n_stc;
    b->r = r;
    b->top = top;
    b->depth = n_cts + 5 + r + n_stc;
    b->scale_in = scale_in;
    if (prm->form > 1) return fail(FE_EINVAL, "bootstrap form must be 0 (real) or 1 (complex)");
    b->form = (int)prm->form;
    const Trig tr(N);
    auto groups_cts = stage_groups(k, n_cts);
    std::reverse(groups_cts.begin(), groups_cts.end());  // applied from the top stages down
    const auto groups_stc = stage_groups(k, n_stc);      // applied from stage 1 up
    std::set<int32_t> steps;
    auto add_group = [&](const std::vector<int>& grp, bool inverse, double kappa, int parts, int level) -> int {
        std::vector<int> stages = grp;
        std::sort(stages.begin(), stages.end());
        if (inverse) std::reverse(stages.begin(), stages.end());  // S_hi^-1 meets the vector first
        std::vector<LtDiag> d;
        std::vector<std::vector<double>> vals, vals_im;
        group_diagonals(N, tr, stages, inverse, kappa, parts, d, vals, &vals_im);
        std::unique_ptr<fe_plan> p;
        std::vector<std::pair<int, int32_t>> src;
        // real form: the pair (re, im) in, parts out; complex form (parts 0): one in, one out
        FE_TRY(plan_lintrans(c, parts ? 2 : 1, parts ? parts : 1, d,
                             default_n1(group_offsets(stages, n).size(), prm->baby_ratio), level, p, src));
        for (int32_t s : p->steps) steps.insert(((s % n) + n) % n);
        p->dhoist = prm->double_hoist ? 1 : 0;
        std::vector<const double*> vp(vals.size()), vpi(vals_im.size());
        for (size_t i = 0; i < vals.size(); i++) vp[i] = vals[i].data();
        for (size_t i = 0; i < vals_im.size(); i++) vpi[i] = vals_im[i].data();
        const size_t nl = (size_t)level + 1 + (p->dhoist ? c->k : 0);
        u64* pt;
        FE_CUDA_TRY(cudaMalloc(&pt, std::max<size_t>(16, (size_t)p->n_pt * nl * pt_limb_bytes(c))));
        b->pts.push_back(pt);
        FE_TRY(load_lintrans(c, p.get(), src, vp, (double)c->mod[level], pt, st, parts ? nullptr : &vpi));
        p->w_scale = (double)c->mod[level];
        b->plans.push_back(std::move(p));
        return FE_OK;
    };
    int level = top;
    for (size_t gi = 0; gi < groups_cts.size(); gi++, level--)
        FE_TRY(add_group(groups_cts[gi], true, gi == 0 ? std::ldexp(M_PI, -r) : 1.0, b->form ? 0 : 2, level));
    // EvalMod: 5 + r levels; its output scale follows from the declared scales
    {
        const int lv0 = level;
        const double s0 = (double)c->mod[0];
        const double s1 = (s0 * s0) / (double)c->mod[lv0];
        const double s2 = (s1 * s1) / (double)c->mod[lv0 - 1];
        const double s4 = (s2 * s2) / (double)c->mod[lv0 - 2];
        const double sc = (s4 * s0) / (double)c->mod[lv0 - 4];
        double s = sc;
        int l = lv0 - 5;
        for (int i = 0; i < r; i++, l--) s = (s * s) / (double)c->mod[l];
        level = l;
        b->out_scale = s;
    }
    const double kappa_stc = ((double)c->mod[0] / (2.0 * M_PI)) / scale_in;
    for (size_t gi = 0; gi < groups_stc.size(); gi++, level--)
        FE_TRY(add_group(groups_stc[gi], false, gi == 0 ? kappa_stc : 1.0,
                         b->form ? 0 : (gi + 1 == groups_stc.size() ? 1 : 2), level));
    // -X^(N/2) on q_0..q_top, NTT form
    {
        i64* v;
        FE_CUDA_TRY(cudaMallocAsync(&v, (size_t)N * 8, st));
        FE_CUDA_TRY(cudaMemsetAsync(v, 0, (size_t)N * 8, st));
        const i64 minus_one = -1;
        FE_CUDA_TRY(cudaMemcpyAsync(v + N / 2, &minus_one, 8, cudaMemcpyHostToDevice, st));
        FE_CUDA_TRY(cudaMalloc(&b->mono, (size_t)(top + 1) * N * 8));
        launch_signed_to_limbs(c, v, b->mono, 0, top + 1, (size_t)N, st);
        ntt_forward(c, LimbSet{b->mono, (size_t)(top + 1) * N, top + 1, 1, c->d_identity_map}, st);
        FE_CUDA_TRY(cudaFreeAsync(v, st));
        FE_CUDA_TRY(cudaStreamSynchronize(st));
    }
    steps.erase(0);
    b->steps.assign(steps.begin(), steps.end());
    b->steps.push_back(FE_STEP_CONJ);
    FE_CUDA_TRY(cudaGetLastError());
    *out = b.release();
    return FE_OK;
}

extern "C" int fe_boot_rotation_steps(const fe_boot* b, int32_t* steps, uint32_t max, uint32_t* n) {
    if (!b || !n) return fail(FE_EINVAL, "null argument");
    *n = (uint32_t)b->steps.size();
    if (steps)
        for (uint32_t i = 0; i < std::min<uint32_t>(max, *n); i++) steps[i] = b->steps[i];
    return FE_OK;
}

extern "C" int fe_boot_output(const fe_boot* b, uint32_t* level, double* scale) {
    if (!b) return fail(FE_EINVAL, "null argument");
    if (level) *level = (uint32_t)(b->top - b->depth);
    if (scale) *scale = b->out_scale;
    return FE_OK;
}

extern "C" size_t fe_boot_workspace_bytes(const fe_boot* b, uint32_t n_ct) {
    if (!b || n_ct == 0) return 0;
    size_t need = 0;
    boot_run(b->c, nullptr, b, nullptr, (int)n_ct, nullptr, nullptr, 0, nullptr, true, &need);
    return need;
}

extern "C" int fe_he_bootstrap(fe_ctx* c, const fe_evk* evk, const fe_boot* b, const void* ct_dev, uint32_t n_ct,
                               void* out_dev, void* ws, size_t ws_bytes, void* stream) {
    FE_ALIGNED(ct_dev); FE_ALIGNED(out_dev); FE_ALIGNED(ws);
    if (!c || !evk || !b || !ct_dev || !out_dev || !ws) return fail(FE_EINVAL, "null argument");
    if (b->c != c) return fail(FE_EINVAL, "the bootstrap belongs to another context");
    if (!evk->relin) return fail(FE_EKEY, "the refresh needs the relinearisation key");
    if (n_ct == 0) return FE_OK;
    return boot_run(c, evk, b, (const u64*)ct_dev, (int)n_ct, (u64*)out_dev, ws, ws_bytes, (cudaStream_t)stream,
                    false, nullptr);
}

extern "C" int fe_boot_graph_capture(fe_ctx* c, const fe_evk* evk, const fe_boot* b, const void* ct_dev,
                                     uint32_t n_ct, void* out_dev, void* ws, size_t ws_bytes, void* stream,
                                     fe_graph** out) {
    FE_ALIGNED(ct_dev); FE_ALIGNED(out_dev); FE_ALIGNED(ws);
    if (!c || !evk || !b || !ct_dev || !out_dev || !ws || !out) return fail(FE_EINVAL, "null argument");
    if (b->c != c) return fail(FE_EINVAL, "the bootstrap belongs to another context");
    if (!evk->relin) return fail(FE_EKEY, "the refresh needs the relinearisation key");
    if (n_ct == 0) return fail(FE_EINVAL, "n_ct must be positive");
    cudaStream_t st = (cudaStream_t)stream;
    if (!st) return fail(FE_EINVAL, "graph capture needs a non-default stream");
    // the transforms' item tables go to their regions of ws first; then the
    // launches alone are captured (they read the tables when the graph runs)
    FE_TRY(boot_run(c, evk, b, (const u64*)ct_dev, (int)n_ct, (u64*)out_dev, ws, ws_bytes, st, false, nullptr, 1));
    FE_CUDA_TRY(cudaStreamSynchronize(st));
    FE_CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    const int rc =
        boot_run(c, evk, b, (const u64*)ct_dev, (int)n_ct, (u64*)out_dev, ws, ws_bytes, st, false, nullptr, 2);
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(st, &graph);
    if (rc != FE_OK) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    if (e != cudaSuccess) return fail(FE_ECUDA, std::string("capture: ") + cudaGetErrorString(e));
    std::unique_ptr<fe_graph> g(new fe_graph());
    g->graph = graph;
    const cudaError_t ie = cudaGraphInstantiate(&g->exec, graph, 0);
    if (ie != cudaSuccess) {
        cudaGraphDestroy(graph);
        return fail(FE_ECUDA, std::string("graph instantiation: ") + cudaGetErrorString(ie));
    }
    const uint32_t out_level = (uint32_t)(b->top - b->depth);
    g->in.push_back({const_cast<void*>(ct_dev), (size_t)n_ct * ct_words(c, 0) * 8});
    g->out.push_back({out_dev, (size_t)n_ct * ct_words(c, (int)out_level) * 8});
    g->out_level.push_back(out_level);
    g->N = (size_t)c->N;
    *out = g.release();
    return FE_OK;
}

extern "C" int fe_key_switch(fe_ctx* c, const void* key_dev, const void* ct_dev, uint32_t n_ct, uint32_t level,
                             void* out_dev, void* stream) {
    FE_ALIGNED(key_dev); FE_ALIGNED(ct_dev); FE_ALIGNED(out_dev);
    if (!c || !key_dev || !ct_dev || !out_dev) return fail(FE_EINVAL, "null argument");
    if ((int)level > c->L) return fail(FE_ELEVEL, "level above L");
    if (n_ct == 0) return FE_OK;
    if (ct_dev == out_dev) return fail(FE_EINVAL, "a key switch cannot run in place");
    cudaStream_t st = (cudaStream_t)stream;
    size_t need = 0;
    {
        Carver dry(nullptr, SIZE_MAX);
        ConjScratch cs;
        carve_conj(dry, c, (int)n_ct, (int)level, &cs);
        need = SIZE_MAX - dry.left;
    }
    void* ws;
    FE_CUDA_TRY(cudaMallocAsync(&ws, need, st));
    Carver cv(ws, need);
    ConjScratch cs;
    carve_conj(cv, c, (int)n_ct, (int)level, &cs);
    const int rc = ks_batch(c, (const u64*)key_dev, 1, (const u64*)ct_dev, (int)n_ct, (int)level, (u64*)out_dev, cs,
                            st);
    cudaFreeAsync(ws, st);
    FE_TRY(rc);
    FE_CUDA_TRY(cudaGetLastError());
    return FE_OK;
}

extern "C" int fe_boot_encapsulate(fe_ctx* c, fe_boot* b, const void* sk_dense, const void* sk_sparse, uint64_t seed,
                                   void* keys_dev, size_t keys_bytes, void* stream) {
    FE_ALIGNED(keys_dev);
    if (!c || !b || !sk_dense || !sk_sparse || !keys_dev) return fail(FE_EINVAL, "null argument");
    if (b->c != c) return fail(FE_EINVAL, "the bootstrap belongs to another context");
    const size_t one = fe_evk_bytes(c, 1, 0);
    if (keys_bytes < 2 * one) return fail(FE_ENOMEM, "encapsulation key buffer too small (2 keys)");
    u64* k0 = (u64*)keys_dev;
    u64* k1 = k0 + one / 8;
    // object tags 2N and 2N + 2: Galois elements are odd and the relinearisation key is 0
    FE_TRY(fe_swk_gen(c, sk_dense, sk_sparse, seed, (uint32_t)(2 * c->N), k0, one, stream));
    FE_TRY(fe_swk_gen(c, sk_sparse, sk_dense, seed, (uint32_t)(2 * c->N + 2), k1, one, stream));
    b->key_to_sparse = k0;
    b->key_to_dense = k1;
    return FE_OK;
}

extern "C" size_t fe_boot_prepare_workspace_bytes(const fe_ctx* c, uint32_t n_ct) {
    if (!c || n_ct == 0) return 0;
    return 2 * (size_t)n_ct * ct_words(c, 1) * 8 + rescale_tmp_words(c, (int)n_ct, 1) * 8 + 3 * 256;
}

extern "C" int fe_boot_prepare(fe_ctx* c, const fe_boot* b, const void* ct_dev, uint32_t n_ct, uint32_t level,
                               double in_scale, void* out_dev, void* ws, size_t ws_bytes, void* stream) {
    FE_ALIGNED(ct_dev); FE_ALIGNED(out_dev); FE_ALIGNED(ws);
    if (!c || !b || !ct_dev || !out_dev || !ws) return fail(FE_EINVAL, "null argument");
    if (b->c != c) return fail(FE_EINVAL, "the bootstrap belongs to another context");
    if (level < 1 || (int)level > c->L) return fail(FE_ELEVEL, "prepare needs 1 <= level <= L");
    if (!(in_scale > 0)) return fail(FE_EINVAL, "in_scale must be positive");
    if (n_ct == 0) return FE_OK;
    cudaStream_t st = (cudaStream_t)stream;
    Carver cv(ws, ws_bytes);
    u64* x = cv.take<u64>((size_t)n_ct * ct_words(c, 1));
    u64* y = cv.take<u64>((size_t)n_ct * ct_words(c, 1));
    u64* tmp = cv.take<u64>(rescale_tmp_words(c, (int)n_ct, 1));
    if (!cv.ok) return fail(FE_ENOMEM, "workspace too small (fe_boot_prepare_workspace_bytes)");
    FE_TRY(fe_mod_drop(c, ct_dev, n_ct, level, 1, x, stream));
    // B = nearest((scale_in / s) q_1): the value is unchanged at the declared scale scale_in
    const double bq = (b->scale_in / in_scale) * (double)c->mod[1];
    AffineConsts k{};
    for (int i = 0; i <= 1; i++) k.mul[i] = nearest_mod(bq, c->mod[i]);
    FE_TRY(launch_affine(c, x, y, (int)n_ct, 1, k, true, st));
    rescale_batch(c, y, (int)n_ct, 1, (u64*)out_dev, tmp, tmp + 2 * (size_t)n_ct * c->N, st);
    FE_CUDA_TRY(cudaGetLastError());
    return FE_OK;
}

extern "C" void fe_boot_destroy(fe_boot* b) { delete b; }
