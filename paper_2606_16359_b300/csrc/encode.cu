// Canonical-embedding encode / decode in double-double arithmetic.
//
// For real slot values z_l (slot l <-> root zeta^(e_l), e_l = 5^l mod 2N,
// complex values: z_l at e_l and its conjugate at 2N - e_l in G below;
// zeta = exp(i pi / N)) the encoded coefficients are
//   m_j = round( Delta * (2/N) * sum_l z_l cos(pi e_l j / N) ).
// Written over the odd exponents e = 2t + 1 (each slot appears at e_l and at
// its conjugate 2N - e_l), with G[t] = z_{slot(2t+1)}:
//   m_j = (Delta / N) * Re( exp(-i pi j / N) * sum_t G[t] exp(-2 pi i t j / N) ),
// i.e. one length-N complex DFT of a real sequence followed by a twist.  The
// DFT runs as a radix-2 decimation-in-time FFT with one kernel per stage, in
// double-double (about 106 significant bits) with twiddles rounded from quad
// precision.  A coefficient whose value lies within 2^-40 of a half-integer
// is reported (FE_EENCODE) instead of being rounded.
//
// Decode evaluates z_l = Re( sum_j m_j zeta^(e_l j) ) / Delta with the same
// FFT (opposite sign) after the twist m_j exp(+i pi j / N).
#include <algorithm>

#include "kernels.cuh"

namespace fe {

namespace {

struct dd {
    double hi, lo;
};

__device__ __forceinline__ dd two_sum(double a, double b) {
    double s = a + b, bb = s - a;
    return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ dd quick_two_sum(double a, double b) {
    double s = a + b;
    return {s, b - (s - a)};
}
__device__ __forceinline__ dd dd_add(dd a, dd b) {
    dd s = two_sum(a.hi, b.hi), t = two_sum(a.lo, b.lo);
    s.lo += t.hi;
    s = quick_two_sum(s.hi, s.lo);
    s.lo += t.lo;
    return quick_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ dd dd_neg(dd a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ dd dd_mul(dd a, dd b) {
    double p = a.hi * b.hi;
    double e = fma(a.hi, b.hi, -p);
    e += a.hi * b.lo + a.lo * b.hi;
    return quick_two_sum(p, e);
}
__device__ __forceinline__ dd dd_mul_d(dd a, double b) {
    double p = a.hi * b;
    double e = fma(a.hi, b, -p);
    e += a.lo * b;
    return quick_two_sum(p, e);
}

struct cdd {
    dd re, im;
};
__device__ __forceinline__ cdd cmul(cdd a, cdd b) {
    return {dd_add(dd_mul(a.re, b.re), dd_neg(dd_mul(a.im, b.im))),
            dd_add(dd_mul(a.re, b.im), dd_mul(a.im, b.re))};
}
__device__ __forceinline__ cdd cadd(cdd a, cdd b) { return {dd_add(a.re, b.re), dd_add(a.im, b.im)}; }
__device__ __forceinline__ cdd csub(cdd a, cdd b) {
    return {dd_add(a.re, dd_neg(b.re)), dd_add(a.im, dd_neg(b.im))};
}
// w_j = exp(-2 pi i j / 2N), conjugated if sign > 0
__device__ __forceinline__ cdd root(const double* w, int j, int sign) {
    cdd r = {{w[4 * j], w[4 * j + 1]}, {w[4 * j + 2], w[4 * j + 3]}};
    if (sign > 0) r.im = dd_neg(r.im);
    return r;
}

__device__ __forceinline__ int brv(int x, int logN) { return (int)(__brev((unsigned)x) >> (32 - logN)); }

// X[n][brv(t)] = G[t] = z[n][slot(2t+1)], and with imaginary parts zi the
// complex slot value, conjugated where 2t + 1 is the conjugate root 2N - 5^l
// (t odd: 5^l = 1 mod 4 while 2N - 5^l = 3 mod 4)
__global__ void k_enc_scatter(const double* z, const double* zi, const int* t2slot, cdd* X, int logN) {
    const int N = 1 << logN;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= N) return;
    const size_t si = (size_t)blockIdx.y * (N / 2) + t2slot[t];
    const double v = z[si];
    const double vi = zi ? ((t & 1) ? -zi[si] : zi[si]) : 0.0;
    X[(size_t)blockIdx.y * N + brv(t, logN)] = {{v, 0.0}, {vi, 0.0}};
}

// one radix-2 DIT stage of span 2^s: X[a] +- w^k X[b], w = exp(sign 2 pi i / 2^s)
__global__ void k_fft_stage(cdd* X, const double* w, int logN, int s, int sign) {
    const int N = 1 << logN;
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= N / 2) return;
    const int half = 1 << (s - 1);
    const int kk = b & (half - 1);
    const int i0 = ((b >> (s - 1)) << s) + kk, i1 = i0 + half;
    cdd* x = X + (size_t)blockIdx.y * N;
    const cdd tw = root(w, kk << (logN + 1 - s), sign);
    cdd u = x[i0], v = cmul(x[i1], tw);
    x[i0] = cadd(u, v);
    x[i1] = csub(u, v);
}

// m_j = round(Delta / N * Re(exp(-i pi j / N) F[j])), written as residues on
// limbs 0..level (coefficient form) of pt[n][level+1][N].
__global__ void k_enc_round(const cdd* F, const double* w, double scale, int logN,
                            const Modulus* mods, const int* mod_map, int nl, u64* pt, unsigned* flags) {
    const int N = 1 << logN;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    const cdd f = F[(size_t)blockIdx.y * N + j];
    const cdd r = root(w, j, -1);
    dd v = dd_add(dd_mul(r.re, f.re), dd_neg(dd_mul(r.im, f.im)));
    v = dd_mul_d(v, scale);
    v = {ldexp(v.hi, -logN), ldexp(v.lo, -logN)};
    double ri = rint(v.hi);
    double d = (v.hi - ri) + v.lo;
    if (d > 0.5) {
        ri += 1.0;
        d -= 1.0;
    }
    if (d < -0.5) {
        ri -= 1.0;
        d += 1.0;
    }
    if (fabs(d) > 0.5 - 0x1p-40 || fabs(ri) >= 0x1p62) atomicAdd(flags, 1u);
    const i64 m = (i64)ri;
    u64* o = pt + (size_t)blockIdx.y * nl * N + j;
    for (int i = 0; i < nl; i++) o[(size_t)i * N] = from_signed(m, mods[mod_map ? mod_map[i] : i].q);
}

// decode input: X[n][brv(j)] = m_j exp(+i pi j / N), m_j given as double-double
__global__ void k_dec_twist(const double* mdd, const double* w, cdd* X, int logN) {
    const int N = 1 << logN;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    const size_t o = (size_t)blockIdx.y * N + j;
    const dd mv = {mdd[2 * o], mdd[2 * o + 1]};
    const cdd r = root(w, j, +1);
    X[(size_t)blockIdx.y * N + brv(j, logN)] = {dd_mul(r.re, mv), dd_mul(r.im, mv)};
}

__global__ void k_dec_gather(const cdd* F, const int* slot2t, double inv_scale, double* z, int logN) {
    const int N = 1 << logN;
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= N / 2) return;
    const cdd f = F[(size_t)blockIdx.y * N + slot2t[l]];
    z[(size_t)blockIdx.y * (N / 2) + l] = (f.re.hi + f.re.lo) * inv_scale;
}

}  // namespace

int encode_batch(fe_ctx* c, const double* slots, int n, int level, double scale, u64* pt,
                 cudaStream_t st, bool qp, const double* slots_im) {
    if (n <= 0) return FE_OK;
    const int N = c->N, logN = c->logN;
    // process in chunks so that the complex double-double scratch stays bounded
    const int chunk = std::max(1, std::min(n, (int)((256ull << 20) / ((size_t)N * sizeof(cdd)))));
    cdd* X;
    unsigned* flags;
    FE_CUDA_TRY(cudaMallocAsync(&X, (size_t)chunk * N * sizeof(cdd), st));
    FE_CUDA_TRY(cudaMallocAsync(&flags, sizeof(unsigned), st));
    FE_CUDA_TRY(cudaMemsetAsync(flags, 0, sizeof(unsigned), st));
    const int nl = qp ? level + 1 + c->k : level + 1;
    const int* mod_map = qp ? c->lv[level].d_ks_limbs : c->d_identity_map;
    for (int s0 = 0; s0 < n; s0 += chunk) {
        int cn = std::min(chunk, n - s0);
        k_enc_scatter<<<dim3((N + 255) / 256, cn), 256, 0, st>>>(
            slots + (size_t)s0 * (N / 2), slots_im ? slots_im + (size_t)s0 * (N / 2) : nullptr, c->d_t2slot, X, logN);
        for (int s = 1; s <= logN; s++)
            k_fft_stage<<<dim3((N / 2 + 255) / 256, cn), 256, 0, st>>>(X, c->d_dd_w, logN, s, -1);
        k_enc_round<<<dim3((N + 255) / 256, cn), 256, 0, st>>>(X, c->d_dd_w, scale, logN, c->d_mod, mod_map,
                                                               nl, pt + (size_t)s0 * nl * N, flags);
        c->cnt.launches += 2 + logN;
    }
    ntt_forward(c, LimbSet{pt, (size_t)nl * N, nl, n, mod_map}, st);
    unsigned hflag = 0;
    FE_CUDA_TRY(cudaMemcpyAsync(&hflag, flags, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    FE_CUDA_TRY(cudaFreeAsync(X, st));
    FE_CUDA_TRY(cudaFreeAsync(flags, st));
    FE_CUDA_TRY(cudaStreamSynchronize(st));
    if (hflag) return fail(FE_EENCODE, "encode: coefficient within 2^-40 of a rounding tie");
    return FE_OK;
}

// mdd: [n][N][2] double-double centred coefficients of the decrypted messages
int decode_batch(fe_ctx* c, const double* mdd, int n, double scale, double* slots, cudaStream_t st) {
    const int N = c->N, logN = c->logN;
    cdd* X;
    FE_CUDA_TRY(cudaMallocAsync(&X, (size_t)n * N * sizeof(cdd), st));
    k_dec_twist<<<dim3((N + 255) / 256, n), 256, 0, st>>>(mdd, c->d_dd_w, X, logN);
    for (int s = 1; s <= logN; s++)
        k_fft_stage<<<dim3((N / 2 + 255) / 256, n), 256, 0, st>>>(X, c->d_dd_w, logN, s, +1);
    k_dec_gather<<<dim3((N / 2 + 255) / 256, n), 256, 0, st>>>(X, c->d_slot2t, 1.0 / scale, slots, logN);
    c->cnt.launches += 2 + logN;
    FE_CUDA_TRY(cudaFreeAsync(X, st));
    return FE_OK;
}

}  // namespace fe
