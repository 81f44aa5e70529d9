// Context: moduli, device tables, counters, and the internal launch helpers.
#pragma once

#include <map>
#include <memory>
#include <vector>

#include "common.h"

namespace fe {

// Approximate base conversion with centred digits from `src` moduli to `dst`
// moduli (device pointers into the context's constant pool):
//   y_i = [x_i * (B/b_i)^-1]_{b_i}, taken in (-b_i/2, b_i/2];
//   out_t = sum_i y_i (B/b_i)  mod m_t
// evaluated as sum_i y'_i mat[t][i] + negB[t] * #{i : y'_i > b_i/2} with the
// unsigned y'_i and negB[t] = -B mod m_t.
struct BConvTab {
    int n_src, n_dst;
    const int* src;     // [n_src] modulus indices
    const int* dst;     // [n_dst]
    const u64* inv;     // [n_src] (B/b_i)^-1 mod b_i
    const u64* inv_sh;  // Shoup companions
    const u64* mat;     // [n_dst][n_src] (B/b_i) mod m_t (destination-major: truncatable)
    const u64* negB;    // [n_dst]
};

struct LevelTabs {
    std::vector<BConvTab> modup;  // one per digit
    BConvTab rescale;             // {q_l} -> q_0..q_{l-1}
    BConvTab mdrs;                // {q_l, p_0..p_{k-1}} -> q_0..q_{l-1} (ModDown and rescale in one)
    std::vector<int> ks_limbs;    // q_0..q_l, p_0..p_{k-1}
    const int* d_ks_limbs;        // device copy
    // extended limbs of one ciphertext's ModUp that need a forward NTT (every digit's
    // block minus the digit's own limbs): position in the [dnum][l+1+k] block and modulus
    int n_up_ntt;
    const int* d_up_pos;
    const int* d_up_mod;
};

enum ProfKind {
    PK_NTT = 0, PK_BCONV, PK_KEYIP, PK_COMBINE, PK_MAC, PK_RESCALE, PK_ENCODE,
    // stages of a planned layer: inner rotations, unrotated MAC, outer rotations, rescale
    PK_STAGE_INNER, PK_STAGE_BASE, PK_STAGE_OUTER, PK_STAGE_RESCALE, PK_COUNT
};

}  // namespace fe

// per-context kernel timing state (see fe_profile_begin)
struct fe_profiler {
    int kind = -1;
    std::vector<cudaEvent_t> ev;
    size_t used = 0;
    double bytes = 0;
    uint64_t launches = 0;
};

struct fe_evk {
    fe_ctx* ctx;
    u64* base;                     // caller buffer
    std::map<uint32_t, u64*> rot;  // galois element -> key [dnum][2][n_mod][N]
    u64* relin;                    // or nullptr
    std::vector<int32_t> steps;
};

struct fe_ctx {
    fe_params prm;
    int logN, N, L, k, n_mod, dnum;
    int max_mod_bits;  // bit length of the largest modulus
    // compact plan plaintexts: bytes of the high-bit plane per residue (1 when
    // every modulus is below 2^40, 2 below 2^48, else 4)
    int pt_hb;
    fe::GenKey gen{};  // generator of the samplers (SplitMix64 unless set to ChaCha20)
    // every modulus in [2^25, 2^40], dnum <= 15 and k <= 15: the base conversion
    // and key inner product sums (< 16 products) reduce with reduce_narrow
    int narrow;
    int ntt_radix = 8;  // elements per thread per NTT round (8 or 16; 16 compiled for N = 2^14, 2^16)
    int ntt_q36 = 1;    // use the 36-bit Shoup product in the transform when every modulus is below 2^36
    int ntt_fwd = 0;    // forward NTT form: bit 0 reduce to [0, 4q) every stage, bit 1 36-bit Shoup product
    // NTT data path: 0 two passes, first and last rounds on global memory; 1 two passes
    // staged through shared memory; 2 one pass on clusters of 8 CTAs (N = 2^16)
    int ntt_path = 0;
    int ntt_cluster_ok = -1;  // whether the cluster form fits on the device (-1: not yet asked)
    std::vector<u64> mod;  // q_0..q_L, p_0..p_{k-1}
    std::vector<u64> psi;
    fe::Modulus* d_mod;             // [n_mod]
    u64* d_tw2;                     // [n_mod][N][2]  (psi^brv(j), Shoup companion)
    u64* d_itw2;                    // [n_mod][N][2]  (psi^-brv(j), Shoup companion)
    u64 *d_ninv, *d_ninv_sh;        // [n_mod] N^-1
    u64 *d_ninvw, *d_ninvw_sh;      // [n_mod] N^-1 times the inverse twiddle at index 1
    u64 *d_pinv, *d_pinv_sh;        // [n_mod] P^-1 mod q_i (i <= L)
    u64 *d_pmod, *d_pmod_sh;        // [n_mod] P mod q_i (i <= L)
    u64 *d_qpinv, *d_qpinv_sh;      // [L+1][L+1] (q_l P)^-1 mod q_i, i < l
    u64 *d_qlinv, *d_qlinv_sh;      // [L+1][L+1]: q_l^-1 mod q_i at [l][i]
    double* d_dd_w;                 // [N][4]: exp(-2 pi i j / 2N) as (re_hi, re_lo, im_hi, im_lo)
    int* d_identity_map;            // [n_mod] j -> j
    uint32_t* d_status;             // bit 0: a bounded device wait gave up (kernels skip their work)
    int* d_t2slot;                  // [N]   slot whose root is zeta^(2t+1) or its conjugate
    int* d_slot2t;                  // [N/2] (5^l mod 2N - 1) / 2
    u64 q0inv_q1;                   // q_0^-1 mod q_1 (CRT of two limbs at decryption)
    fe::BConvTab moddown;           // P -> q_0..q_L
    std::vector<fe::LevelTabs> lv;  // per level 0..L
    void* pool;                     // all small device tables live here
    std::vector<void*> allocs;
    fe_counters cnt;
    fe_profiler prof;
    cudaDeviceProp prop;
    int n_sm;
    int device;  // CUDA device the context was created on (its tables live there)
    // bounded waits of the PMult-MAC's mbarriers: the limit, and (for tests of the
    // expiry path only; -1 otherwise) a term whose copies the producer never issues
    uint64_t mac_wait_ns = 2000000000ull;
    int mac_unfed_term = -1;

    int slot_count() const { return N / 2; }
    size_t limb_bytes() const { return (size_t)N * sizeof(u64); }
    uint32_t galois(int32_t r) const;
};

namespace fe {

// NTT over a set of limbs: limb b lives at base + (b / per_poly) * poly_stride
// + (b % per_poly) * N and uses modulus mod_map[b % per_poly].
struct LimbSet {
    u64* base;
    size_t poly_stride;  // in words
    int per_poly;
    int n_poly;
    const int* mod_map;            // device [per_poly]
    const int* pos_map = nullptr;  // device [per_poly]: limb position inside a poly (default j)
};
void ntt_forward(fe_ctx* c, const LimbSet& s, cudaStream_t st);
void ntt_inverse(fe_ctx* c, const LimbSet& s, cudaStream_t st);
// throughput probe of the transform's butterfly arithmetic (blocks x 256 threads)
// (*blocks = 0: one full wave, set on return)
int butterfly_probe(fe_ctx* c, uint32_t* blocks, uint32_t iters, u64* out, cudaStream_t st);
// Decides, outside any stream capture, whether the cluster form of the NTT fits on the device.
void ntt_prepare(fe_ctx* c);
// out-of-place: the first pass reads polynomials from src (poly stride src_stride words)
void ntt_forward_from(fe_ctx* c, const u64* src, size_t src_stride, const LimbSet& dst, cudaStream_t st);
void ntt_inverse_from(fe_ctx* c, const u64* src, size_t src_stride, const LimbSet& dst, cudaStream_t st);

int sk_gen(fe_ctx* c, uint64_t seed, u64* sk, cudaStream_t st);
// qp: the plaintexts on Q_level * P (l+1+k limbs in key-switching order) instead of Q_level
// slots_im (optional): imaginary parts of complex slot values ([n][N/2])
int encode_batch(fe_ctx* c, const double* slots, int n, int level, double scale, u64* pt,
                 cudaStream_t st, bool qp = false, const double* slots_im = nullptr);
int decode_batch(fe_ctx* c, const double* mdd, int n, double scale, double* slots, cudaStream_t st);

// Records CUDA events around one launch when its kernel class is being profiled,
// and adds the launch's algorithmic bytes.
struct ProfScope {
    fe_ctx* c;
    cudaStream_t st;
    bool on;
    ProfScope(fe_ctx* ctx, int kind, cudaStream_t s, double bytes);
    ~ProfScope();
};

// scratch allocation helper: carve 256-byte aligned chunks out of a caller workspace
struct Carver {
    char* p;
    size_t left;
    bool ok = true;
    Carver(void* base, size_t bytes) : p((char*)base), left(bytes) {}
    template <class T>
    T* take(size_t count) {
        size_t b = (count * sizeof(T) + 255) & ~(size_t)255;
        if (b > left) {
            ok = false;
            return nullptr;
        }
        T* r = (T*)p;
        p += b;
        left -= b;
        return r;
    }
};

}  // namespace fe
