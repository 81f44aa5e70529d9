// Negacyclic NTT / inverse NTT over RNS limbs, batched.
//
// Forward: Cooley-Tukey butterflies with twiddles psi^brv(m + i) (natural order
// in, bit-reversed order out), which computes NTT(a)[i] = a(psi^(2 brv(i) + 1)).
// Inverse: Gentleman-Sande butterflies with psi^-brv(h + i), then N^-1.
//
// The transform of one limb (N = N1 * N2) runs in two passes, each staged in
// shared memory: the stages whose butterfly distance is a multiple of N2 act
// on the N2 columns {r + c N2} independently ("column pass"), the remaining
// stages act on contiguous rows of N2 elements ("row pass").  A CTA loads a
// tile of several columns (or rows) with coalesced 8-byte loads, runs its
// stages with __syncthreads between them, and writes the tile back.
#include <algorithm>

#include "context.h"

namespace fe {

namespace {

constexpr int kTile = 4096;  // elements per CTA tile (32 KiB)
constexpr int kThreads = 512;

struct NttArgs {
    u64* base;
    size_t poly_stride;
    int per_poly;
    const int* mod_map;
    const Modulus* mods;
    const u64* tw;  // [n_mod][N]
    const u64* tw_sh;
    const u64* ninv;
    const u64* ninv_sh;
    int logN, logN2;
};

__device__ __forceinline__ u64* limb_ptr(const NttArgs& a, int limb, int& mod_idx) {
    int poly = limb / a.per_poly, j = limb % a.per_poly;
    mod_idx = a.mod_map[j];
    return a.base + (size_t)poly * a.poly_stride + ((size_t)j << a.logN);
}

// Column pass: stages with distance t = tr * N2, tr = N1/2 .. 1 (forward) or
// 1 .. N1/2 (inverse).  Tile = C columns x N1 rows, stored tile[c * C + r].
template <bool kInverse>
__global__ void __launch_bounds__(kThreads) ntt_col_pass(NttArgs a) {
    extern __shared__ u64 tile[];
    const int N = 1 << a.logN, N2 = 1 << a.logN2, N1 = N >> a.logN2;
    const int C = min(kTile / N1, N2);
    const int tiles_per_limb = N2 / C;
    const int limb = blockIdx.x / tiles_per_limb;
    const int r0 = (blockIdx.x % tiles_per_limb) * C;
    int mi;
    u64* d = limb_ptr(a, limb, mi);
    const u64 q = a.mods[mi].q;
    const u64* tw = a.tw + ((size_t)mi << a.logN);
    const u64* tws = a.tw_sh + ((size_t)mi << a.logN);
    const int n = N1 * C;
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
        int c = e / C, r = e % C;
        tile[e] = d[(size_t)c * N2 + r0 + r];
    }
    __syncthreads();
    const int nb = n / 2;
    if (!kInverse) {
        for (int tr = N1 / 2; tr >= 1; tr >>= 1) {
            const int m = N1 / (2 * tr);
            for (int b = threadIdx.x; b < nb; b += blockDim.x) {
                int r = b % C, bb = b / C;
                int grp = bb / tr, pos = bb % tr;
                int c = grp * 2 * tr + pos;
                u64 w = tw[m + grp], ws = tws[m + grp];
                u64 U = tile[c * C + r];
                u64 V = mul_shoup(tile[(c + tr) * C + r], w, ws, q);
                tile[c * C + r] = add_mod(U, V, q);
                tile[(c + tr) * C + r] = sub_mod(U, V, q);
            }
            __syncthreads();
        }
    } else {
        const u64 ni = a.ninv[mi], nis = a.ninv_sh[mi];
        for (int tr = 1; tr <= N1 / 2; tr <<= 1) {
            const int h = N1 / (2 * tr);
            const bool last = (tr == N1 / 2);
            for (int b = threadIdx.x; b < nb; b += blockDim.x) {
                int r = b % C, bb = b / C;
                int grp = bb / tr, pos = bb % tr;
                int c = grp * 2 * tr + pos;
                u64 w = tw[h + grp], ws = tws[h + grp];
                u64 U = tile[c * C + r], V = tile[(c + tr) * C + r];
                u64 s = add_mod(U, V, q);
                u64 t = mul_shoup(sub_mod(U, V, q), w, ws, q);
                if (last) {
                    s = mul_shoup(s, ni, nis, q);
                    t = mul_shoup(t, ni, nis, q);
                }
                tile[c * C + r] = s;
                tile[(c + tr) * C + r] = t;
            }
            __syncthreads();
        }
    }
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
        int c = e / C, r = e % C;
        d[(size_t)c * N2 + r0 + r] = tile[e];
    }
}

// Row pass: stages with distance t = N2/2 .. 1 (forward) or 1 .. N2/2 (inverse),
// within rows of N2 contiguous elements.  Tile = R rows.
template <bool kInverse>
__global__ void __launch_bounds__(kThreads) ntt_row_pass(NttArgs a) {
    extern __shared__ u64 tile[];
    const int N = 1 << a.logN, N2 = 1 << a.logN2, N1 = N >> a.logN2;
    const int R = min(kTile / N2, N1);
    const int tiles_per_limb = N1 / R;
    const int limb = blockIdx.x / tiles_per_limb;
    const int row0 = (blockIdx.x % tiles_per_limb) * R;
    int mi;
    u64* d = limb_ptr(a, limb, mi);
    const u64 q = a.mods[mi].q;
    const u64* tw = a.tw + ((size_t)mi << a.logN);
    const u64* tws = a.tw_sh + ((size_t)mi << a.logN);
    const int n = R * N2;
    u64* g = d + (size_t)row0 * N2;
    for (int e = threadIdx.x; e < n; e += blockDim.x) tile[e] = g[e];
    __syncthreads();
    const int nb = n / 2, half = N2 / 2;
    if (!kInverse) {
        for (int t = N2 / 2; t >= 1; t >>= 1) {
            const int gpr = N2 / (2 * t);  // groups per row
            const int m = N / (2 * t);
            for (int b = threadIdx.x; b < nb; b += blockDim.x) {
                int rho = b / half, bb = b % half;
                int grp = bb / t, pos = bb % t;
                int x = grp * 2 * t + pos;
                int i = (row0 + rho) * gpr + grp;
                u64 w = tw[m + i], ws = tws[m + i];
                int o = rho * N2 + x;
                u64 U = tile[o];
                u64 V = mul_shoup(tile[o + t], w, ws, q);
                tile[o] = add_mod(U, V, q);
                tile[o + t] = sub_mod(U, V, q);
            }
            __syncthreads();
        }
    } else {
        for (int t = 1; t <= N2 / 2; t <<= 1) {
            const int gpr = N2 / (2 * t);
            const int h = N / (2 * t);
            for (int b = threadIdx.x; b < nb; b += blockDim.x) {
                int rho = b / half, bb = b % half;
                int grp = bb / t, pos = bb % t;
                int x = grp * 2 * t + pos;
                int i = (row0 + rho) * gpr + grp;
                u64 w = tw[h + i], ws = tws[h + i];
                int o = rho * N2 + x;
                u64 U = tile[o], V = tile[o + t];
                tile[o] = add_mod(U, V, q);
                tile[o + t] = mul_shoup(sub_mod(U, V, q), w, ws, q);
            }
            __syncthreads();
        }
    }
    for (int e = threadIdx.x; e < n; e += blockDim.x) g[e] = tile[e];
}

NttArgs make_args(fe_ctx* c, const LimbSet& s, bool inverse) {
    NttArgs a;
    a.base = s.base;
    a.poly_stride = s.poly_stride;
    a.per_poly = s.per_poly;
    a.mod_map = s.mod_map;
    a.mods = c->d_mod;
    a.tw = inverse ? c->d_itw : c->d_tw;
    a.tw_sh = inverse ? c->d_itw_sh : c->d_tw_sh;
    a.ninv = c->d_ninv;
    a.ninv_sh = c->d_ninv_sh;
    a.logN = c->logN;
    a.logN2 = c->logN / 2;
    return a;
}

}  // namespace

void ntt_forward(fe_ctx* c, const LimbSet& s, cudaStream_t st) {
    int limbs = s.per_poly * s.n_poly;
    if (limbs == 0) return;
    NttArgs a = make_args(c, s, false);
    const int N = c->N, N2 = 1 << a.logN2, N1 = N / N2;
    int C = std::min(kTile / N1, N2), R = std::min(kTile / N2, N1);
    size_t smc = (size_t)N1 * C * 8, smr = (size_t)R * N2 * 8;
    const double bytes = 16.0 * limbs * N;
    {
        ProfScope ps(c, PK_NTT, st, bytes);
        ntt_col_pass<false><<<limbs * (N2 / C), kThreads, smc, st>>>(a);
    }
    {
        ProfScope ps(c, PK_NTT, st, bytes);
        ntt_row_pass<false><<<limbs * (N1 / R), kThreads, smr, st>>>(a);
    }
    c->cnt.ntt += limbs;
    c->cnt.launches += 2;
}

void ntt_inverse(fe_ctx* c, const LimbSet& s, cudaStream_t st) {
    int limbs = s.per_poly * s.n_poly;
    if (limbs == 0) return;
    NttArgs a = make_args(c, s, true);
    const int N = c->N, N2 = 1 << a.logN2, N1 = N / N2;
    int C = std::min(kTile / N1, N2), R = std::min(kTile / N2, N1);
    size_t smc = (size_t)N1 * C * 8, smr = (size_t)R * N2 * 8;
    const double bytes = 16.0 * limbs * N;
    {
        ProfScope ps(c, PK_NTT, st, bytes);
        ntt_row_pass<true><<<limbs * (N1 / R), kThreads, smr, st>>>(a);
    }
    {
        ProfScope ps(c, PK_NTT, st, bytes);
        ntt_col_pass<true><<<limbs * (N2 / C), kThreads, smc, st>>>(a);
    }
    c->cnt.ntt += limbs;
    c->cnt.launches += 2;
}

}  // namespace fe
