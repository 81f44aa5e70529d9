// Host-side parameter generation: NTT-friendly primes, psi, NTT twiddle tables,
// base-conversion tables, the encoder's slot maps and its double-double roots.
#include <quadmath.h>
#include <string.h>

#include <algorithm>
#include <thread>

#include "context.h"

namespace fe {

static thread_local std::string g_err = "no error";

void set_error(const std::string& msg) { g_err = msg; }
int fail(int code, const std::string& msg) {
    g_err = msg;
    return code;
}
const char* last_error() { return g_err.c_str(); }

u64 h_mulmod(u64 a, u64 b, u64 q) { return (u64)((u128)a * b % q); }
u64 h_powmod(u64 a, u64 e, u64 q) {
    u64 acc = 1 % q, base = a % q;
    for (; e; e >>= 1, base = h_mulmod(base, base, q))
        if (e & 1) acc = h_mulmod(acc, base, q);
    return acc;
}
// extended Euclid on signed 128-bit integers
u64 h_invmod(u64 a, u64 q) {
    i128 t = 0, nt = 1, r = q, nr = a % q;
    while (nr) {
        i128 qq = r / nr, tmp;
        tmp = t - qq * nt;
        t = nt;
        nt = tmp;
        tmp = r - qq * nr;
        r = nr;
        nr = tmp;
    }
    if (t < 0) t += q;
    return (u64)t;
}
u64 shoup_of(u64 w, u64 q) { return (u64)(((u128)w << 64) / q); }

Modulus make_modulus(u64 q) {
    // floor(2^128 / q) = floor((2^128 - 1) / q) for q not a power of two
    u128 r = (~(u128)0) / q;
    Modulus m;
    m.q = q;
    m.ratio_hi = (u64)(r >> 64);
    m.ratio_lo = (u64)r;
    m.mu88 = q > (1ull << 24) ? (u64)(((u128)1 << 88) / q) : 0;
    return m;
}

// Miller-Rabin with the first twelve primes as witnesses (exact for 64-bit n).
static bool probably_prime(u64 n) {
    if (n < 4) return n >= 2;
    if (!(n & 1)) return false;
    u64 d = n - 1;
    int r = __builtin_ctzll(d);
    d >>= r;
    for (u64 a : {2ULL, 3ULL, 5ULL, 7ULL, 11ULL, 13ULL, 17ULL, 19ULL, 23ULL, 29ULL, 31ULL, 37ULL}) {
        if (a % n == 0) continue;
        u64 x = h_powmod(a, d, n);
        if (x == 1 || x == n - 1) continue;
        bool witness = true;
        for (int i = 1; i < r && witness; i++) {
            x = h_mulmod(x, x, n);
            if (x == n - 1) witness = false;
        }
        if (witness) return false;
    }
    return true;
}

// primes p = 1 mod 2N below 2^bits, descending, skipping the given ones
static std::vector<u64> prime_run(int logN, int bits, int count, const std::vector<u64>& skip) {
    std::vector<u64> out;
    u64 step = (u64)2 << logN;
    for (u64 c = ((u64)1 << bits) + 1 - step; (int)out.size() < count && c > step; c -= step) {
        if (std::find(skip.begin(), skip.end(), c) != skip.end()) continue;
        if (probably_prime(c)) out.push_back(c);
    }
    return out;
}

// smallest primitive 2N-th root of unity: take a generator g of Z_q^*, set
// w = g^((q-1)/2N) (a primitive 2N-th root), and minimise over its odd powers.
static u64 min_primitive_root_2N(u64 q, int logN) {
    u64 m = q - 1;
    std::vector<u64> fac;
    u64 t = m;
    for (u64 f = 2; f * f <= t; f += (f == 2 ? 1 : 2)) {
        if (t % f == 0) {
            fac.push_back(f);
            while (t % f == 0) t /= f;
        }
    }
    if (t > 1) fac.push_back(t);
    u64 g = 2;
    for (;; g++) {
        bool gen = true;
        for (u64 f : fac)
            if (h_powmod(g, m / f, q) == 1) {
                gen = false;
                break;
            }
        if (gen) break;
    }
    u64 twoN = (u64)2 << logN;
    u64 w = h_powmod(g, m / twoN, q), w2 = h_mulmod(w, w, q), cur = w, best = w;
    for (u64 i = 0; i < twoN / 2; i++) {
        best = std::min(best, cur);
        cur = h_mulmod(cur, w2, q);
    }
    return best;
}

static u64 bitrev(u64 x, int bits) {
    u64 r = 0;
    for (int i = 0; i < bits; i++) r |= ((x >> i) & 1) << (bits - 1 - i);
    return r;
}

}  // namespace fe

using namespace fe;

uint32_t fe_ctx::galois(int32_t r) const {
    if (r == FE_STEP_CONJ) return (uint32_t)(2 * N - 1);  // sigma_{-1}: complex conjugation of the slots
    int64_t half = N / 2;
    int64_t rr = ((int64_t)r % half + half) % half;
    return (uint32_t)h_powmod(5, (u64)rr, (u64)2 * N);
}

namespace {

struct PoolBuilder {
    std::vector<char> host;
    size_t put(const void* src, size_t bytes) {
        size_t off = (host.size() + 255) & ~(size_t)255;
        host.resize(off + bytes);
        if (bytes) memcpy(host.data() + off, src, bytes);
        return off;
    }
};

struct TabOffsets {
    size_t src, dst, inv, inv_sh, mat, negB;
    int n_src, n_dst;
};

TabOffsets build_tab(PoolBuilder& pb, const std::vector<u64>& mod, const std::vector<int>& src,
                     const std::vector<int>& dst) {
    TabOffsets o;
    o.n_src = (int)src.size();
    o.n_dst = (int)dst.size();
    std::vector<u64> inv, inv_sh, mat, negB;
    for (int i : src) {
        u64 b = mod[i], bhat = 1;  // (B / b_i) mod b_i
        for (int i2 : src)
            if (i2 != i) bhat = h_mulmod(bhat, mod[i2] % b, b);
        u64 iv = h_invmod(bhat, b);
        inv.push_back(iv);
        inv_sh.push_back(shoup_of(iv, b));
    }
    for (int t : dst)  // destination-major, so a table truncates to its first destinations
        for (int i : src) {
            u64 mt = mod[t], v = 1;
            for (int i2 : src)
                if (i2 != i) v = h_mulmod(v, mod[i2] % mt, mt);
            mat.push_back(v);
        }
    for (int t : dst) {
        u64 mt = mod[t], B = 1;
        for (int i : src) B = h_mulmod(B, mod[i] % mt, mt);
        negB.push_back((mt - B) % mt);
    }
    o.src = pb.put(src.data(), src.size() * sizeof(int));
    o.dst = pb.put(dst.data(), dst.size() * sizeof(int));
    o.inv = pb.put(inv.data(), inv.size() * 8);
    o.inv_sh = pb.put(inv_sh.data(), inv_sh.size() * 8);
    o.mat = pb.put(mat.data(), mat.size() * 8);
    o.negB = pb.put(negB.data(), negB.size() * 8);
    return o;
}

BConvTab resolve(const TabOffsets& o, char* base) {
    BConvTab t;
    t.n_src = o.n_src;
    t.n_dst = o.n_dst;
    t.src = (const int*)(base + o.src);
    t.dst = (const int*)(base + o.dst);
    t.inv = (const u64*)(base + o.inv);
    t.inv_sh = (const u64*)(base + o.inv_sh);
    t.mat = (const u64*)(base + o.mat);
    t.negB = (const u64*)(base + o.negB);
    return t;
}

}  // namespace

extern "C" const char* fe_last_error(void) { return fe::last_error(); }

extern "C" int fe_ctx_create(const fe_params* p, fe_ctx** out) {
    if (!p || !out) return fail(FE_EINVAL, "null argument");
    if (p->logN < 4 || p->logN > 17 || p->n_q < 1 || p->k < 1 || p->k > 8 || p->qbits > 61 ||
        p->pbits > 61 || p->qbits < p->logN + 2 || p->pbits < p->logN + 2)
        return fail(FE_EINVAL, "parameter set out of range");
    std::unique_ptr<fe_ctx> c(new fe_ctx());
    c->prm = *p;
    c->logN = p->logN;
    c->N = 1 << p->logN;
    c->L = p->n_q - 1;
    c->k = p->k;
    c->n_mod = p->n_q + p->k;
    c->dnum = (p->n_q + p->k - 1) / p->k;
    if (c->dnum > 16) return fail(FE_EINVAL, "more than 16 key-switching digits (raise k)");
    memset(&c->cnt, 0, sizeof(c->cnt));
    c->mod = prime_run(c->logN, p->qbits, p->n_q, {});
    if ((int)c->mod.size() != (int)p->n_q) return fail(FE_EINVAL, "not enough ciphertext primes");
    std::vector<u64> sp = prime_run(c->logN, p->pbits, p->k, c->mod);
    if ((int)sp.size() != (int)p->k) return fail(FE_EINVAL, "not enough special primes");
    c->mod.insert(c->mod.end(), sp.begin(), sp.end());
    c->max_mod_bits = 0;
    for (u64 m : c->mod) c->max_mod_bits = std::max(c->max_mod_bits, 64 - __builtin_clzll(m));
    c->pt_hb = c->max_mod_bits <= 40 ? 1 : (c->max_mod_bits <= 48 ? 2 : 4);
    {
        int min_bits = 64;
        for (u64 m : c->mod) min_bits = std::min(min_bits, 64 - __builtin_clzll(m));
        // sums of up to 16 products of residues below 2^40 stay below 2^84
        c->narrow = c->max_mod_bits <= 40 && min_bits >= 26 && c->dnum <= 15 && c->k <= 15 ? 1 : 0;
    }

    int dev;
    FE_CUDA_TRY(cudaGetDevice(&dev));
    FE_CUDA_TRY(cudaGetDeviceProperties(&c->prop, dev));
    c->n_sm = c->prop.multiProcessorCount;
    c->device = dev;

    const int N = c->N, nm = c->n_mod;
    c->psi.resize(nm);
    {
        std::vector<std::thread> th;
        for (int i = 0; i < nm; i++)
            th.emplace_back([&, i] { c->psi[i] = min_primitive_root_2N(c->mod[i], c->logN); });
        for (auto& t : th) t.join();
    }
    std::vector<u64> tw2((size_t)nm * N * 2), itw2((size_t)nm * N * 2);
    std::vector<u64> ninv(nm), ninv_sh(nm), pinv(nm, 0), pinv_sh(nm, 0), pmod(nm, 0), pmod_sh(nm, 0);
    std::vector<u64> ninvw(nm), ninvw_sh(nm);
    {
        std::vector<std::thread> th;
        for (int i = 0; i < nm; i++)
            th.emplace_back([&, i] {
                u64 q = c->mod[i], w = c->psi[i], wi = h_invmod(w, q);
                std::vector<u64> pw(N), pwi(N);
                pw[0] = 1;
                pwi[0] = 1;
                for (int j = 1; j < N; j++) {
                    pw[j] = h_mulmod(pw[j - 1], w, q);
                    pwi[j] = h_mulmod(pwi[j - 1], wi, q);
                }
                for (int j = 0; j < N; j++) {
                    u64 a = pw[bitrev(j, c->logN)], b = pwi[bitrev(j, c->logN)];
                    tw2[2 * ((size_t)i * N + j)] = a;
                    tw2[2 * ((size_t)i * N + j) + 1] = shoup_of(a, q);
                    itw2[2 * ((size_t)i * N + j)] = b;
                    itw2[2 * ((size_t)i * N + j) + 1] = shoup_of(b, q);
                }
                ninv[i] = h_invmod((u64)N % q, q);
                ninv_sh[i] = shoup_of(ninv[i], q);
                // the inverse transform's last stage has the single twiddle at index 1;
                // its product with N^-1 lets that stage apply the final scaling
                ninvw[i] = h_mulmod(itw2[2 * ((size_t)i * N + (N > 1 ? 1 : 0))], ninv[i], q);
                ninvw_sh[i] = shoup_of(ninvw[i], q);
            });
        for (auto& t : th) t.join();
    }
    for (int i = 0; i <= c->L; i++) {
        u64 q = c->mod[i], P = 1;
        for (int j = 0; j < c->k; j++) P = h_mulmod(P, c->mod[c->L + 1 + j] % q, q);
        pinv[i] = h_invmod(P, q);
        pinv_sh[i] = shoup_of(pinv[i], q);
        pmod[i] = P;
        pmod_sh[i] = shoup_of(P, q);
    }
    std::vector<u64> qlinv((size_t)(c->L + 1) * (c->L + 1), 0), qlinv_sh(qlinv.size(), 0);
    std::vector<u64> qpinv(qlinv.size(), 0), qpinv_sh(qlinv.size(), 0);
    for (int l = 1; l <= c->L; l++)
        for (int i = 0; i < l; i++) {
            u64 v = h_invmod(c->mod[l] % c->mod[i], c->mod[i]);
            qlinv[(size_t)l * (c->L + 1) + i] = v;
            qlinv_sh[(size_t)l * (c->L + 1) + i] = shoup_of(v, c->mod[i]);
            u64 w = h_mulmod(v, pinv[i], c->mod[i]);  // (q_l P)^-1
            qpinv[(size_t)l * (c->L + 1) + i] = w;
            qpinv_sh[(size_t)l * (c->L + 1) + i] = shoup_of(w, c->mod[i]);
        }
    // double-double table exp(-2 pi i j / 2N), j in [0, N), rounded from quad precision
    std::vector<double> ddw((size_t)N * 4);
    for (int j = 0; j < N; j++) {
        __float128 ang = -4 * atanq((__float128)1) * (__float128)j / (__float128)N;
        __float128 cr = cosq(ang), ci = sinq(ang);
        double rh = (double)cr, ih = (double)ci;
        ddw[4 * j + 0] = rh;
        ddw[4 * j + 1] = (double)(cr - (__float128)rh);
        ddw[4 * j + 2] = ih;
        ddw[4 * j + 3] = (double)(ci - (__float128)ih);
    }

    PoolBuilder pb;
    std::vector<Modulus> mods(nm);
    for (int i = 0; i < nm; i++) mods[i] = make_modulus(c->mod[i]);
    size_t o_mod = pb.put(mods.data(), nm * sizeof(Modulus));
    size_t o_ninv = pb.put(ninv.data(), nm * 8), o_ninv_sh = pb.put(ninv_sh.data(), nm * 8);
    size_t o_ninvw = pb.put(ninvw.data(), nm * 8), o_ninvw_sh = pb.put(ninvw_sh.data(), nm * 8);
    size_t o_pinv = pb.put(pinv.data(), nm * 8), o_pinv_sh = pb.put(pinv_sh.data(), nm * 8);
    size_t o_pmod = pb.put(pmod.data(), nm * 8), o_pmod_sh = pb.put(pmod_sh.data(), nm * 8);
    size_t o_ql = pb.put(qlinv.data(), qlinv.size() * 8);
    size_t o_ql_sh = pb.put(qlinv_sh.data(), qlinv_sh.size() * 8);
    size_t o_qp = pb.put(qpinv.data(), qpinv.size() * 8);
    size_t o_qp_sh = pb.put(qpinv_sh.data(), qpinv_sh.size() * 8);
    std::vector<int> ident(nm);
    for (int i = 0; i < nm; i++) ident[i] = i;
    size_t o_ident = pb.put(ident.data(), nm * sizeof(int));
    std::vector<int> t2slot(N), slot2t(N / 2);
    {
        u64 e = 1, twoN = 2 * (u64)N;
        for (int l = 0; l < N / 2; l++) {
            t2slot[(e - 1) / 2] = l;
            t2slot[(twoN - e - 1) / 2] = l;
            slot2t[l] = (int)((e - 1) / 2);
            e = e * 5 % twoN;
        }
    }
    size_t o_t2s = pb.put(t2slot.data(), N * sizeof(int));
    size_t o_s2t = pb.put(slot2t.data(), (N / 2) * sizeof(int));
    std::vector<int> qs(c->L + 1), ps(c->k);
    for (int i = 0; i <= c->L; i++) qs[i] = i;
    for (int j = 0; j < c->k; j++) ps[j] = c->L + 1 + j;
    TabOffsets md = build_tab(pb, c->mod, ps, qs);
    struct LvOff {
        std::vector<TabOffsets> up;
        TabOffsets rs, mdrs;
        size_t ks, up_pos, up_mod;
        int n_up;
        std::vector<int> ks_limbs;
    };
    std::vector<LvOff> lvo(c->L + 1);
    for (int l = 0; l <= c->L; l++) {
        std::vector<int> ks;
        for (int i = 0; i <= l; i++) ks.push_back(i);
        for (int j = 0; j < c->k; j++) ks.push_back(c->L + 1 + j);
        lvo[l].ks_limbs = ks;
        lvo[l].ks = pb.put(ks.data(), ks.size() * sizeof(int));
        int nd = (l + 1 + c->k - 1) / c->k;
        std::vector<int> up_pos, up_mod;
        const int np = l + 1 + c->k;
        for (int j = 0; j < nd; j++) {
            std::vector<int> dig, oth;
            for (int i = j * c->k; i < std::min((j + 1) * c->k, l + 1); i++) dig.push_back(i);
            for (int t : ks)
                if (std::find(dig.begin(), dig.end(), t) == dig.end()) oth.push_back(t);
            lvo[l].up.push_back(build_tab(pb, c->mod, dig, oth));
            for (int pos = 0; pos < np; pos++)
                if (std::find(dig.begin(), dig.end(), pos) == dig.end()) {  // positions of q's equal their index
                    up_pos.push_back(j * np + pos);
                    up_mod.push_back(ks[pos]);
                }
        }
        lvo[l].n_up = (int)up_pos.size();
        lvo[l].up_pos = pb.put(up_pos.data(), up_pos.size() * sizeof(int));
        lvo[l].up_mod = pb.put(up_mod.data(), up_mod.size() * sizeof(int));
        if (l >= 1) {
            std::vector<int> lower;
            for (int i = 0; i < l; i++) lower.push_back(i);
            lvo[l].rs = build_tab(pb, c->mod, {l}, lower);
            std::vector<int> qp{l};
            for (int j = 0; j < c->k; j++) qp.push_back(c->L + 1 + j);
            lvo[l].mdrs = build_tab(pb, c->mod, qp, lower);
        }
    }

    const uint32_t zero_status[4] = {0, 0, 0, 0};
    const size_t o_status = pb.put(zero_status, sizeof(zero_status));
    char* dpool = nullptr;
    FE_CUDA_TRY(cudaMalloc(&dpool, pb.host.size()));
    c->pool = dpool;
    FE_CUDA_TRY(cudaMemcpy(dpool, pb.host.data(), pb.host.size(), cudaMemcpyHostToDevice));
    c->d_mod = (Modulus*)(dpool + o_mod);
    c->d_ninv = (u64*)(dpool + o_ninv);
    c->d_ninv_sh = (u64*)(dpool + o_ninv_sh);
    c->d_ninvw = (u64*)(dpool + o_ninvw);
    c->d_ninvw_sh = (u64*)(dpool + o_ninvw_sh);
    c->d_pinv = (u64*)(dpool + o_pinv);
    c->d_pinv_sh = (u64*)(dpool + o_pinv_sh);
    c->d_pmod = (u64*)(dpool + o_pmod);
    c->d_pmod_sh = (u64*)(dpool + o_pmod_sh);
    c->d_qlinv = (u64*)(dpool + o_ql);
    c->d_qlinv_sh = (u64*)(dpool + o_ql_sh);
    c->d_qpinv = (u64*)(dpool + o_qp);
    c->d_qpinv_sh = (u64*)(dpool + o_qp_sh);
    c->d_identity_map = (int*)(dpool + o_ident);
    c->d_status = (uint32_t*)(dpool + o_status);
    c->d_t2slot = (int*)(dpool + o_t2s);
    c->d_slot2t = (int*)(dpool + o_s2t);
    c->q0inv_q1 = c->L >= 1 ? h_invmod(c->mod[0] % c->mod[1], c->mod[1]) : 0;
    c->moddown = resolve(md, dpool);
    c->lv.resize(c->L + 1);
    for (int l = 0; l <= c->L; l++) {
        for (auto& o : lvo[l].up) c->lv[l].modup.push_back(resolve(o, dpool));
        if (l >= 1) c->lv[l].rescale = resolve(lvo[l].rs, dpool);
        if (l >= 1) c->lv[l].mdrs = resolve(lvo[l].mdrs, dpool);
        c->lv[l].ks_limbs = lvo[l].ks_limbs;
        c->lv[l].d_ks_limbs = (const int*)(dpool + lvo[l].ks);
        c->lv[l].n_up_ntt = lvo[l].n_up;
        c->lv[l].d_up_pos = (const int*)(dpool + lvo[l].up_pos);
        c->lv[l].d_up_mod = (const int*)(dpool + lvo[l].up_mod);
    }
    auto up = [&](u64** dst, const std::vector<u64>& v) -> int {
        FE_CUDA_TRY(cudaMalloc(dst, v.size() * 8));
        c->allocs.push_back(*dst);
        FE_CUDA_TRY(cudaMemcpy(*dst, v.data(), v.size() * 8, cudaMemcpyHostToDevice));
        return FE_OK;
    };
    FE_TRY(up(&c->d_tw2, tw2));
    FE_TRY(up(&c->d_itw2, itw2));
    FE_CUDA_TRY(cudaMalloc(&c->d_dd_w, ddw.size() * sizeof(double)));
    c->allocs.push_back(c->d_dd_w);
    FE_CUDA_TRY(cudaMemcpy(c->d_dd_w, ddw.data(), ddw.size() * sizeof(double), cudaMemcpyHostToDevice));
    fe::ntt_prepare(c.get());
    *out = c.release();
    return FE_OK;
}

extern "C" void fe_ctx_destroy(fe_ctx* c) {
    if (!c) return;
    for (void* p : c->allocs) cudaFree(p);
    for (cudaEvent_t e : c->prof.ev) cudaEventDestroy(e);
    cudaFree(c->pool);
    delete c;
}

extern "C" int fe_ctx_moduli(const fe_ctx* c, uint64_t* out) {
    if (!c || !out) return fail(FE_EINVAL, "null argument");
    for (int i = 0; i < c->n_mod; i++) out[i] = c->mod[i];
    return FE_OK;
}

extern "C" int fe_get_counters(const fe_ctx* c, fe_counters* out) {
    if (!c || !out) return fail(FE_EINVAL, "null argument");
    *out = c->cnt;
    return FE_OK;
}

namespace fe {
ProfScope::ProfScope(fe_ctx* ctx, int kind, cudaStream_t s, double bytes)
    : c(ctx), st(s), on(ctx->prof.kind == kind) {
    if (!on) return;
    fe_profiler& p = c->prof;
    while (p.used + 2 > p.ev.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) {
            on = false;
            return;
        }
        p.ev.push_back(e);
    }
    cudaEventRecord(p.ev[p.used], st);
    p.bytes += bytes;
    p.launches++;
}
ProfScope::~ProfScope() {
    if (!on) return;
    cudaEventRecord(c->prof.ev[c->prof.used + 1], st);
    c->prof.used += 2;
}
}  // namespace fe

extern "C" int fe_profile_begin(fe_ctx* c, const char* kind) {
    if (!c || !kind) return fail(FE_EINVAL, "null argument");
    static const char* names[PK_COUNT] = {"ntt", "bconv", "keyip", "combine", "mac", "rescale", "encode",
                                          "stage_inner", "stage_base", "stage_outer", "stage_rescale"};
    int k = -1;
    for (int i = 0; i < PK_COUNT; i++)
        if (!strcmp(kind, names[i])) k = i;
    if (k < 0) return fail(FE_EINVAL, std::string("unknown kernel class ") + kind);
    c->prof.kind = k;
    c->prof.used = 0;
    c->prof.bytes = 0;
    c->prof.launches = 0;
    return FE_OK;
}

extern "C" int fe_profile_end(fe_ctx* c, double* total_ms, uint64_t* launches, double* bytes) {
    if (!c || !total_ms || !launches || !bytes) return fail(FE_EINVAL, "null argument");
    double t = 0;
    for (size_t i = 0; i + 1 < c->prof.used; i += 2) {
        FE_CUDA_TRY(cudaEventSynchronize(c->prof.ev[i + 1]));
        float ms = 0;
        FE_CUDA_TRY(cudaEventElapsedTime(&ms, c->prof.ev[i], c->prof.ev[i + 1]));
        t += ms;
    }
    *total_ms = t;
    *launches = c->prof.launches;
    *bytes = c->prof.bytes;
    c->prof.kind = -1;
    c->prof.used = 0;
    return FE_OK;
}

extern "C" int fe_counters_reset(fe_ctx* c) {
    if (!c) return fail(FE_EINVAL, "null argument");
    memset(&c->cnt, 0, sizeof(c->cnt));
    return FE_OK;
}

extern "C" int fe_device_status(fe_ctx* c, uint32_t* status, int reset) {
    if (!c || !status) return fail(FE_EINVAL, "null argument");
    FE_CUDA_TRY(cudaDeviceSynchronize());
    FE_CUDA_TRY(cudaMemcpy(status, c->d_status, sizeof(uint32_t), cudaMemcpyDeviceToHost));
    if (reset) FE_CUDA_TRY(cudaMemset(c->d_status, 0, sizeof(uint32_t)));
    return FE_OK;
}

extern "C" int fe_ctx_set_mac_wait(fe_ctx* c, uint64_t limit_ns, int32_t unfed_term) {
    if (!c) return fe::fail(FE_EINVAL, "null argument");
    if (limit_ns == 0 || limit_ns > 60000000000ull) return fe::fail(FE_EINVAL, "wait limit outside (0, 60 s]");
    if (unfed_term < -1) return fe::fail(FE_EINVAL, "unfed_term must be -1 or a term index");
    c->mac_wait_ns = limit_ns;
    c->mac_unfed_term = unfed_term;
    return FE_OK;
}

extern "C" int fe_ctx_set_generator(fe_ctx* c, int kind, const uint32_t* key_material) {
    if (!c) return fe::fail(FE_EINVAL, "null argument");
    if (kind != FE_GEN_SPLITMIX64 && kind != FE_GEN_CHACHA20) return fe::fail(FE_EINVAL, "unknown generator");
    if (kind == FE_GEN_CHACHA20 && !key_material) return fe::fail(FE_EINVAL, "ChaCha20 needs key material");
    c->gen.kind = kind == FE_GEN_CHACHA20 ? fe::kGenChaCha20 : fe::kGenSplitMix64;
    for (int i = 0; i < 6; i++) c->gen.k[i] = kind == FE_GEN_CHACHA20 ? key_material[i] : 0;
    return FE_OK;
}
