/*
 * fenc.h - C ABI of the B300 (sm_103a) encrypted-convolution library.
 *
 * The library evaluates the hot path of FEnc^2's encrypted CNN inference: the
 * homomorphic convolution under the conv-aware fragment encoding (Algorithm 1,
 * Sec. 4.2; the convolution of Sec. 3.1), with hoisted inner rotations, PMult multiply-accumulate over
 * fragment masks, outer rotations (Eq. 1 rotations, counted by Eq. 3 - Eq. 5),
 * one rescale, and the layers around it: x^2 activation, 2x2 average pooling,
 * fully connected layers, and Arch-aware Ciphertext Compression (Sec. 4.3, Fig. 6).
 * The calls follow the usage flow of the problem statement (Sec. 4.1): the client
 * sends shape metadata, receives the slot mapping, encodes and encrypts; the
 * server evaluates; the client decrypts.
 *
 * Conventions (apply to every entry point):
 *  - Return value: FE_OK (0) on success, a negative FE_E* code otherwise; the
 *    message of the last error on the calling thread is fe_last_error().
 *    Arguments are validated before any launch; no kernel traps or spins
 *    without a bound.
 *  - Pointers named *_dev are device pointers (cudaMalloc / torch CUDA tensors);
 *    *_host are host pointers.  Device buffers passed in are owned by the
 *    caller; the library never frees them.  Every device buffer must start on a
 *    16-byte boundary (cudaMalloc and torch allocations do; kernels use 16-byte
 *    accesses); a misaligned one is rejected with FE_EINVAL before any launch.  Library objects (fe_ctx, fe_evk,
 *    fe_plan, fe_graph) are opaque handles released with their *_destroy call.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Calls enqueue work and return without synchronising unless stated.
 *  - Ring degree N = 2^logN.  Moduli are indexed q_0..q_L (L = n_q - 1, largest
 *    first) followed by the special primes p_0..p_{k-1}.
 *  - Polynomials are uint64 residues in NTT form, limb-major: a polynomial at
 *    level l is [l+1][N]; a ciphertext at level l is [2][l+1][N] (c0, c1);
 *    an array of n ciphertexts is [n][2][l+1][N], contiguous.
 *  - NTT form: NTT(a)[i] = a(psi^(2 brv(i) + 1)) mod q with psi the smallest
 *    primitive 2N-th root of unity mod q.  Slot l is the evaluation at
 *    zeta^(5^l), zeta = exp(i pi / N); a left rotation by r slots uses the
 *    Galois element 5^r mod 2N.
 */
#ifndef FENC_H
#define FENC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FE_OK 0
#define FE_EINVAL (-1)   /* bad argument or shape */
#define FE_ENOMEM (-2)   /* buffer too small / allocation failed */
#define FE_ELEVEL (-3)   /* no level left for the operation */
#define FE_ESCALE (-4)   /* scale mismatch */
#define FE_EKEY (-5)     /* a needed rotation key is missing */
#define FE_ETIMEOUT (-6) /* a bounded device wait gave up */
#define FE_ECUDA (-7)    /* CUDA runtime error */
#define FE_EENCODE (-8)  /* a coefficient lies within 2^-40 of a rounding tie */

/* Rotation-step value that stands for the complex conjugation of the slots
 * (the automorphism X -> X^(2N-1), Galois element 2N - 1) wherever a rotation
 * step is taken: fe_evk_gen, fe_evk_upload, fe_evk_alias, fe_rotate. */
#define FE_STEP_CONJ (-2147483647 - 1)

typedef struct fe_ctx fe_ctx;
typedef struct fe_evk fe_evk;
typedef struct fe_plan fe_plan;
typedef struct fe_graph fe_graph;
typedef struct fe_server fe_server;
typedef struct fe_boot fe_boot;

/* Parameter set.  q primes: the n_q largest primes below 2^qbits with
 * q = 1 (mod 2N); special primes: the k largest primes below 2^pbits with the
 * same congruence that are not among the q's. */
typedef struct {
    uint32_t logN, n_q, k, qbits, pbits;
} fe_params;

/* Fragment layout of a BS x C x H x W activation (Algorithm 1).
 * Inputs: H, W, C, BS, S, m (m = 0: derive m = 2^ceil(log2(ceil(max(H,W)/S)))).
 * Outputs filled by fe_layout_make: m, M = S m, cpc = N / (2 m^2 BS) channels per
 * ciphertext, groups = ceil(C / cpc), n_ct = groups S^2.
 * Slot of element (b, c, h, w): ciphertext (g S + u) S + v with g = c / cpc,
 * u = h mod S, v = w mod S; slot ((c mod cpc) m^2 + (h / S) m + w / S) BS + b. */
typedef struct {
    uint32_t H, W, C, BS, S, m;
    uint32_t M, cpc, groups, n_ct;
} fe_layout;

/* Operation counters (the columns of the paper's Table 4): rotations,
 * key switches, forward+inverse limb NTTs, plaintext mults, ciphertext mults,
 * rescales, and kernel launches issued by the library. */
typedef struct {
    uint64_t rot, keyswitch, ntt, pmult, cmult, rescale, launches;
} fe_counters;

/* ---- rotation-complexity model and fragment-size choice (host only) ------ */

/* The rotation counts of the fragment encoding for one conv layer at fragment
 * size S (Sec. 4.2): alpha = N / (2 M^2) with the padded side M = S m,
 * Eq. 3 inner rotations (ceil(K/S)^2 - 1) Cin / alpha (0 when K <= S or S = M,
 * the convention of Table 6), Eq. 4 outer rotations
 * (BS/alpha)(alpha S^2/BS - 1) Cout (0 for depthwise layers), the Eq. 5 total
 * (BS/alpha)[inner(S) Cin + (alpha S^2/BS - 1) Cout], the Eq. 7 bound
 * sqrt(BS Cin / alpha), the Eq. 8 closed form (K^2 Cin BS / (alpha Cout))^(1/4),
 * and the inner rotations a layer executes (every needed block offset of every
 * input ciphertext, stride 1 or 2). */
typedef struct {
    uint32_t m, M, cpc;
    double alpha, eq3_inner, eq4_outer, eq5_total, s_bound_eq7, s_star_eq8;
    uint64_t executed_inner;
} fe_rotation_model_t;
/* Pure host computation (no device, no context).  Errors: FE_EINVAL (zero
 * extent, N not a power of two, stride not 1 or 2, channel block larger than a
 * ciphertext). */
int fe_rotation_model(uint32_t N, uint32_t H, uint32_t W, uint32_t Cin, uint32_t Cout, uint32_t K,
                      uint32_t S, uint32_t BS, uint32_t stride, int depthwise, fe_rotation_model_t* out);

/* Analytic fragment-size choice (Theorem, Eq. 5, Eq. 7): the argmin of the
 * Eq. 5 total over the power-of-two S <= max_S (0: 32) whose channel block fits
 * a ciphertext (m^2 BS <= N/2) and that satisfy Eq. 7 (S = 1 always does); ties
 * go to the smaller S.  out receives S, its layout geometry, alpha, the Eq. 5
 * value, the Eq. 8 closed form at that alpha, and the number of admissible
 * sizes examined.  Pure host computation.  Errors: FE_EINVAL (bad extents or no
 * admissible S). */
typedef struct {
    uint32_t S, m, M, cpc, n_admissible;
    double alpha, eq5, s_star;
} fe_fragment_choice;
int fe_choose_fragment(uint32_t N, uint32_t H, uint32_t W, uint32_t Cin, uint32_t Cout, uint32_t K,
                       uint32_t BS, int depthwise, uint32_t max_S, fe_fragment_choice* out);

/* ---- context ------------------------------------------------------------ */

/* Create a context on the current CUDA device: generates the moduli and the
 * NTT / base-conversion tables and uploads them (library-owned, freed by
 * fe_ctx_destroy).  Errors: FE_EINVAL (logN outside [4,17], n_q < 1, k outside
 * [1,8], primes above 61 bits), FE_ECUDA. */
int fe_ctx_create(const fe_params* params, fe_ctx** out);
void fe_ctx_destroy(fe_ctx* ctx);
/* Tile choice of the NTT: elements a thread holds per round, 8 (default), 16
 * (fewer shared-memory round trips, more registers) or 4 (more rounds, fewer
 * registers, more resident warps); 4 and 16 are compiled for N = 2^14 and
 * 2^16, other ring degrees stay at 8.  Results do not depend on it.
 * Errors: FE_EINVAL. */
int fe_ctx_set_ntt_radix(fe_ctx* ctx, int radix);
/* Butterfly product of the inverse NTT when every modulus is below 2^36:
 * enable = 1 (default) takes Shoup's product in 32-bit pieces with the quotient
 * against floor(w 2^63 / q) (ten 32-bit multiply instructions, exact for inputs
 * below 2^42); 0 takes the general 64-bit form everywhere.  The forward
 * transform keeps the general form (it measured faster there).  Results do not
 * depend on it; other moduli always take the general form.  enable = 2 is as 1
 * and makes the butterfly probe (fe_probe_butterflies) run the 32-bit-piece
 * form instead of the forward transform's.  Errors: FE_EINVAL. */
int fe_ctx_set_ntt_q36(fe_ctx* ctx, int enable);
/* Form of the forward NTT's butterflies (two-pass paths).  flags bit 0: reduce
 * every stage's sums to [0, 4q) with a compare (Harvey's lazy form) instead of
 * letting them grow to below 35 q and reducing once at the end with a 64-bit
 * Barrett step (the default whenever every modulus is below 2^58); bit 1: take
 * the 36-bit Shoup product of fe_ctx_set_ntt_q36 in the forward transform too
 * (moduli below 2^36 only).  Default 0.  Results do not depend on it.
 * Errors: FE_EINVAL. */
int fe_ctx_set_ntt_forward(fe_ctx* ctx, int flags);
/* Data path of the NTT.  path = 0 (default): two passes (column stages, then
 * row stages of N = N1 x N2), whose first round reads its elements straight
 * from global memory and whose last round writes them straight back, with
 * only the rounds in between going through shared memory.  path = 1: the same
 * two passes with the whole tile loaded into shared memory first and stored
 * from there (compiled for N = 2^14 and 2^16 at radix 8; other shapes take
 * path 0).  path = 2: one pass per limb on a cluster of 8 CTAs that exchange
 * the limb through distributed shared memory between the column and the row
 * stages, so that each limb crosses DRAM once each way (N = 2^16 only, radix
 * 8; other ring degrees, and a device on which such a cluster does not fit,
 * take path 0).  Results do not depend on it.  Errors: FE_EINVAL. */
int fe_ctx_set_ntt_path(fe_ctx* ctx, int path);
/* Generator behind every sampler of the context (secret key, encryption
 * randomness and errors, evaluation keys).  Each sample is drawn from word n of
 * a stream addressed by (seed, tag):
 *   FE_GEN_SPLITMIX64 (default): SplitMix64 (Steele, Lea, Flood 2014),
 *     word = mix(mix(seed + (tag + 1) g) + (n + 1) g), g = 0x9E3779B97F4A7C15;
 *   FE_GEN_CHACHA20: the ChaCha20 block function of RFC 8439 with key =
 *     (seed low, seed high, key_material[0..5]) as eight 32-bit words, nonce =
 *     (tag low, tag high, 0) and block counter n / 8; the word is output words
 *     2 (n mod 8) and 2 (n mod 8) + 1 of that block, low word first.
 * key_material: six 32-bit words (host), required for ChaCha20, ignored for
 * SplitMix64.  Samplers: uniform mod q = floor(word q / 2^64); ternary =
 * floor(3 word / 2^64) - 1; error = popcount(word bits 0..20) - popcount(bits
 * 21..41).  Errors: FE_EINVAL. */
#define FE_GEN_SPLITMIX64 0
#define FE_GEN_CHACHA20 1
int fe_ctx_set_generator(fe_ctx* ctx, int kind, const uint32_t* key_material);
/* Copy the n_q + k moduli (q_0..q_L, p_0..p_{k-1}) to moduli_host. */
int fe_ctx_moduli(const fe_ctx* ctx, uint64_t* moduli_host);
/* Read / reset the operation counters of the context. */
int fe_get_counters(const fe_ctx* ctx, fe_counters* out);
int fe_counters_reset(fe_ctx* ctx);
/* Message of the last error on this thread (never NULL). */
const char* fe_last_error(void);

/* ---- keys (client) ------------------------------------------------------- */

/* Secret key: ternary s sampled from the context's counter-based generator
 * (fe_ctx_set_generator; words addressed by seed and stream), written in NTT
 * form on every modulus: sk_dev holds [n_q + k][N] uint64. */
int fe_sk_gen(fe_ctx* ctx, uint64_t seed, void* sk_dev, void* stream);

/* Bytes of the switching keys for n_steps rotations (+1 relinearisation key if
 * relin != 0): per key dnum = ceil(n_q / k) digits x [2][n_q + k][N] uint64. */
size_t fe_evk_bytes(const fe_ctx* ctx, uint32_t n_steps, int relin);

/* Hybrid key-switching keys (Eq. 1's evk^k_rot, with the special primes as the
 * "large modulus" P), written into the caller buffer evk_dev of at least
 * fe_evk_bytes bytes.  A rotation key for step r switches from s to
 * sigma_{g^-1}(s), g = 5^r mod 2N, so that a rotation key-switches first and
 * applies sigma_g afterwards.  steps_host: n_steps slot offsets (negative =
 * right rotation; duplicates and multiples of N/2 are rejected).  The handle
 * keeps pointers into evk_dev; the buffer must outlive it.
 * Errors: FE_EINVAL, FE_ENOMEM (buffer too small). */
int fe_evk_gen(fe_ctx* ctx, const void* sk_dev, uint64_t seed, const int32_t* steps_host,
               uint32_t n_steps, int relin, void* evk_dev, size_t evk_bytes, void* stream,
               fe_evk** out);
/* Server side: index switching keys that a client generated (fe_evk_gen on
 * its own device, then copied to host memory), so that the secret key never
 * reaches the evaluating party.  evk_host holds fe_evk_bytes(ctx, n_steps,
 * relin) bytes in fe_evk_gen's layout for the same steps in the same order
 * (the relinearisation key last); they are copied into the device buffer
 * evk_dev (caller-owned, at least that size), which must outlive the handle.
 * Errors: FE_EINVAL (short host bytes, bad or duplicate steps), FE_ENOMEM. */
int fe_evk_upload(fe_ctx* ctx, const void* evk_host, size_t evk_host_bytes, const int32_t* steps_host,
                  uint32_t n_steps, int relin, void* evk_dev, size_t evk_dev_bytes, void* stream,
                  fe_evk** out);
void fe_evk_destroy(fe_evk* evk);

/* For latency measurement only: make every step in steps[] that has no key
 * use one of the evk's generated keys (round robin).  Rotations by those steps
 * then compute with the wrong key (their results do not decrypt), but read
 * and write exactly the memory a real key would, so layer timings are
 * representative without generating and storing every key.  *n_aliased
 * (optional) receives the number of steps added.  Errors: FE_EINVAL, FE_EKEY
 * (the evk holds no key). */
int fe_evk_alias(fe_ctx* ctx, fe_evk* evk, const int32_t* steps, uint32_t n_steps, uint32_t* n_aliased);

/* ---- layout, packing, encode / encrypt / decrypt (client) ----------------- */

/* Fill the derived fields of a layout (Algorithm 1 steps 1-2) for the
 * context's ring degree.  Errors: FE_EINVAL when one channel block does not fit
 * a ciphertext (m^2 BS > N/2). */
int fe_layout_make(const fe_ctx* ctx, fe_layout* lay);

/* Algorithm 1 step 3 on the device: x_dev float64 (BS, C, H, W) -> slots_dev
 * float64 [n_ct][N/2], zero padded. */
int fe_fragment_pack(const fe_ctx* ctx, const fe_layout* lay, const double* x_dev,
                     double* slots_dev, void* stream);
/* Inverse of fe_fragment_pack on the valid region. */
int fe_fragment_unpack(const fe_ctx* ctx, const fe_layout* lay, const double* slots_dev,
                       double* y_dev, void* stream);

/* Encode n slot vectors (slots_dev, [n][N/2] float64) at `scale` into
 * plaintexts [n][level+1][N] (NTT form): m = round(scale * tau^-1(z)),
 * evaluated in double-double.  Errors: FE_EENCODE (a coefficient within 2^-40
 * of a rounding tie). */
int fe_encode(fe_ctx* ctx, const double* slots_dev, uint32_t n, uint32_t level, double scale,
              void* pt_dev, void* stream);

/* Encode n_ct slot vectors and encrypt them with the secret key at `level`:
 * c1 = a uniform, c0 = -a s + m + e, e centred binomial (eta = 21).
 * Ciphertext j uses random streams (seed, ct_id0 + j).
 * Output ct_dev: [n_ct][2][level+1][N].  Errors: FE_EENCODE, FE_EINVAL. */
int fe_encode_encrypt(fe_ctx* ctx, const void* sk_dev, const double* slots_dev, uint32_t n_ct,
                      uint32_t level, double scale, uint64_t seed, uint64_t ct_id0, void* ct_dev,
                      void* stream);

/* Decrypt and decode n_ct ciphertexts at `level` and `scale`:
 * m = c0 + c1 s, centred mod q_0 (q_0 q_1 when level >= 1), slots
 * z_l = Re(sum_j m_j zeta^(5^l j)) / scale -> slots_dev [n_ct][N/2] float64. */
int fe_decrypt_decode(fe_ctx* ctx, const void* sk_dev, const void* ct_dev, uint32_t n_ct,
                      uint32_t level, double scale, double* slots_dev, void* stream);

/* ---- CKKS primitives (server) --------------------------------------------- */

/* Forward (inverse != 0: inverse) NTT of n_poly polynomials [n_poly][n_limbs][N]
 * in place; limb j of every polynomial uses modulus index first_mod + j. */
int fe_ntt(fe_ctx* ctx, void* data_dev, uint32_t n_poly, uint32_t n_limbs, uint32_t first_mod,
           int inverse, void* stream);
/* Throughput probe of the forward NTT's butterfly arithmetic (no counterpart in
 * the paper; a measurement aid for the integer-pipe roofline of the transform).
 * Launches `blocks` CTAs of 256 threads (blocks = 0: one full wave, i.e. the
 * SM count times the CTAs that fit on one SM, at most 8); each thread runs
 * `iters` x 60 lazy Shoup butterflies on register-resident residues of modulus
 * q_0 and writes one word to out_dev (caller-owned device buffer of
 * blocks * 256 uint64, or SMs * 8 * 256 when blocks = 0; 16-byte aligned).
 * *butterflies (optional) receives blocks * 256 * iters * 60.  The caller
 * times the launch on `stream`.  Errors: FE_EINVAL, FE_ECUDA. */
int fe_probe_butterflies(fe_ctx* ctx, uint32_t blocks, uint32_t iters, void* out_dev,
                         uint64_t* butterflies, void* stream);
/* Left rotation of n_ct ciphertexts by r slots (Eq. 1): out = sigma_g((c0,0) + KS(c1)),
 * the key read once for all n_ct.  Errors: FE_EKEY when the key for r is missing,
 * FE_EINVAL (null pointer, out overlapping the input). */
int fe_rotate(fe_ctx* ctx, const fe_evk* evk, const void* ct_dev, uint32_t n_ct, uint32_t level,
              int32_t r, void* out_dev, void* stream);
/* Hoisted rotations (Eq. 1 for several steps of one input): n_ct ciphertexts
 * at `level`, each rotated by every steps_host[j] (j < n_steps, host array;
 * FE_STEP_CONJ allowed), out_dev [n_steps][n_ct] ciphertexts at `level`.
 * One ModUp per input ciphertext serves all steps, and each step's key is
 * read once for all n_ct; every output equals fe_rotate's residues.  Scratch
 * from the stream-ordered allocator.  Errors: FE_EINVAL (null pointer, outputs
 * overlapping the inputs), FE_ELEVEL, FE_EKEY (a step without its key),
 * FE_ENOMEM. */
int fe_rotate_many(fe_ctx* ctx, const fe_evk* evk, const void* ct_dev, uint32_t n_ct, uint32_t level,
                   const int32_t* steps_host, uint32_t n_steps, void* out_dev, void* stream);
/* Rescale n_ct ciphertexts from `level` to level-1: (c - [c]_{q_l}) q_l^-1 with
 * the centred representative.  Errors: FE_ELEVEL at level 0. */
int fe_rescale(fe_ctx* ctx, const void* ct_dev, uint32_t n_ct, uint32_t level, void* out_dev,
               void* stream);
/* Rescale without allocating: same result as fe_rescale, but the scratch comes
 * from one fixed 32 MiB array of device memory (a static device variable of the
 * library), so the call never allocates or frees device memory.  The array is
 * reserved on a device when the library's module holding it loads there: under
 * CUDA's lazy module loading (the default) that is the first fe_rescale_noalloc
 * call on that device, so a caller planning a fixed footprint should make one
 * call at start-up; the 32 MiB then stay reserved until the process exits.  For
 * callers that cannot allocate: a serving process whose device footprint is
 * fixed after start-up, a host framework that owns all device memory through its
 * own pool, or latency-critical code that cannot afford an allocation's possible
 * device synchronisation.  There is no counterpart in the paper.
 *  - Size limit: 16 (n_ct N + n_ct level N) bytes of scratch must fit in 32 MiB
 *    (e.g. one ciphertext at N = 2^16 and level 23); larger requests fail with
 *    FE_ENOMEM and a message, before any launch.
 *  - The current device must be the context's device (else FE_EINVAL).  The
 *    first call on a device looks up the array's device address (once per
 *    device); make that first call before any stream capture on the device.
 *  - Every call uses the same array.  Nothing in it needs to start at zero, and
 *    it keeps the last call's contents.  Calls whose work overlaps on the GPU
 *    (different streams, or host threads without ordering) race on the array;
 *    order them on one stream.
 *  - Kernel timing (fe_profile_begin) does not record this call.
 * Errors: FE_EINVAL, FE_ELEVEL, FE_ENOMEM, FE_ECUDA. */
int fe_rescale_noalloc(fe_ctx* ctx, const void* ct_dev, uint32_t n_ct, uint32_t level,
                       void* out_dev, void* stream);
/* out = ct (x) pt per limb (PMult), n_ct ciphertexts times one plaintext each. */
int fe_pmult(fe_ctx* ctx, const void* ct_dev, const void* pt_dev, uint32_t n_ct, uint32_t level,
             void* out_dev, void* stream);
/* out = a + b (Add), n_ct pairs. */
int fe_add(fe_ctx* ctx, const void* a_dev, const void* b_dev, uint32_t n_ct, uint32_t level,
           void* out_dev, void* stream);

/* ---- encrypted layers (server) -------------------------------------------- */

/* Plan one HE convolution layer under the fragment encoding (Sec. 3.1, Sec. 4.2):
 *   in: input layout, Cout, K, stride (1, or 2 with S even), depthwise (Cout = C,
 *   one filter per channel), in_period (0, or c_v when the input was replicated
 *   by fe_compress so that channel position c holds channel c mod c_v), level of
 *   the input ciphertexts.
 *   bsgs_n1: 0 for linear outer rotations (one per nonzero channel diagonal d,
 *   Rot(P_d, d m^2 BS), Eq. 4); n1 > 0 for the baby-step / giant-step schedule
 *   the paper assumes (Sec. 3.1): diagonal d = j n1 + i; every input ciphertext
 *   is rotated by tap offset + i m^2 BS from its one hoisted ModUp, the
 *   plaintexts of diagonal d are rotated left by i m^2 BS, and one giant
 *   rotation by j n1 m^2 BS per output and j > 0 (n1 is clipped to cpc;
 *   depthwise and replicated-input layers stay linear).
 * The plan records the inner rotation offsets, the nonzero diagonals, the
 * multiply-accumulate term lists and the output layout (out_lay).
 * Errors: FE_EINVAL (shape), FE_ELEVEL (level 0). */
int fe_plan_conv(fe_ctx* ctx, const fe_layout* in_lay, uint32_t Cout, uint32_t K, uint32_t stride,
                 int depthwise, uint32_t in_period, uint32_t level, uint32_t bsgs_n1, fe_layout* out_lay,
                 fe_plan** out);
/* Plan a fully connected layer y = W x on ciphertexts whose positions
 * (P = cpc m^2 per ciphertext, BS slots each) hold features:
 *   feat_host[c * P + p] = feature index of position p of input ciphertext c, or -1.
 * Output neuron n sits in ciphertext n / P at position n mod P.  Baby-step /
 * giant-step split n1 = 2^ceil(log2(P)/2), n2 = P / n1. */
int fe_plan_fc(fe_ctx* ctx, uint32_t n_in_ct, uint32_t P, uint32_t BS, const int32_t* feat_host,
               uint32_t F_in, uint32_t F_out, uint32_t level, fe_plan** out);
/* Plan the first fully connected layer on a fragment-packed map (the flatten
 * step of a CNN, Sec. 5 Implementation: FC by diagonals with baby-step /
 * giant-step): feature (c, h, w) of the (C, H, W) map in layout in_lay is input
 * feature (c H + h) W + w (row-major flattening), read from the slot that
 * Algorithm 1 gives it; F_in = C H W.  Same plan as fe_plan_fc with that table.
 * Errors as fe_plan_fc. */
int fe_plan_fc_layout(fe_ctx* ctx, const fe_layout* in_lay, uint32_t F_out, uint32_t level, fe_plan** out);
/* Plan a fully connected layer that reads the output of the fully connected plan
 * `prev` (neuron n of prev at position n mod P of ciphertext n / P), with
 * F_in = prev's F_out.  Errors as fe_plan_fc; FE_EINVAL when prev is not FC. */
int fe_plan_fc_next(fe_ctx* ctx, const fe_plan* prev, uint32_t F_out, uint32_t level, fe_plan** out);
/* Fragment-size change between layers (Sec. 5, Implementation: a later layer
 * whose best block size S differs gets its input re-encoded by rot-mask-add).
 * Plans the re-encoding of ciphertexts in layout `from` into layout `to`
 * (the same BS x C x H x W map; any S and block grid m on either side) at
 * `level`: target ciphertext t = sum over source ciphertexts s and position
 * shifts d of Rot(ct_s, d BS) (x) M_{t,s,d}, M the 0/1 mask of the target
 * positions whose element sits d positions further in s -- the diagonal method
 * of the permutation matrix, with baby-step / giant-step rotations whose n1 (a
 * power of two) minimises the distinct nonzero baby steps per source plus giant
 * steps per target.  It is an FC-kind plan: fe_plan_load_weights with
 * weights_host = NULL writes the masks (at w_scale, normally q_level so the
 * scale is kept), and fe_he_repack (or fe_he_fc, fe_he_layer_batch, graph
 * capture) runs it; one level is consumed.  Cost grows with the distinct
 * shifts, i.e. with how far elements move: cheap for small maps and large
 * batches, costly for large maps at BS = 1.  Errors: FE_EINVAL (layouts of
 * different maps), FE_ELEVEL. */
int fe_plan_repack(fe_ctx* ctx, const fe_layout* from, const fe_layout* to, uint32_t level, fe_plan** out);
int fe_he_repack(fe_ctx* ctx, const fe_evk* evk, const fe_plan* plan, const void* pt_dev, const void* in_dev,
                 void* out_dev, void* workspace_dev, size_t workspace_bytes, int mode, void* stream);
/* ---- transformer extension (Sec. 7): fragmented token embeddings ---------- */

/* n_tok tokens with embedding dimension E, split into fragments of size S:
 * element e = f S + s of token t sits in ciphertext s at position f, slot
 * f n_tok + t, so each of the S ciphertexts holds ceil(E / S) = F elements of
 * every token and an embedding-wise sum spans F positions instead of E.
 * Filled by fe_token_layout_make: P = N / (2 n_tok) positions per ciphertext,
 * F, n_ct = S.  Errors: FE_EINVAL (n_tok does not divide N/2, F > P). */
typedef struct {
    uint32_t n_tok, E, S;
    uint32_t P, F, n_ct;
} fe_token_layout;
int fe_token_layout_make(const fe_ctx* ctx, fe_token_layout* lay);
/* x_dev float64 (n_tok, E) -> slots_dev float64 [S][N/2] (zero padded), and back. */
int fe_token_pack(const fe_ctx* ctx, const fe_token_layout* lay, const double* x_dev, double* slots_dev,
                  void* stream);
int fe_token_unpack(const fe_ctx* ctx, const fe_token_layout* lay, const double* slots_dev, double* x_dev,
                    void* stream);
/* Plan Y = X W^T (W: E_out x E, row-major) on fragmented tokens (the
 * projections and FFN layers of an encoder block): the FC plan of Sec. 5
 * (diagonals with baby-step / giant-step over the P positions, tokens in the
 * batch slots) on the fragment feature table, with output element
 * k = f' S + s' at ciphertext s' position f' (out_lay: the same S and n_tok,
 * E = E_out).  Weights through fe_plan_load_weights (weights_host: W), run by
 * fe_he_fc (the attention products: fe_he_attention_scores / _apply).
 * Errors as fe_plan_fc, FE_EINVAL (layouts). */
int fe_plan_token_linear(fe_ctx* ctx, const fe_token_layout* in_lay, uint32_t E_out, uint32_t level,
                         fe_token_layout* out_lay, fe_plan** out);
/* Attention products on fragmented tokens (Sec. 7: the token-wise aggregation
 * of Q K^T and A V).  A token-wise rotation by r rotates every position block
 * of n_tok slots by r tokens: M_lo (x) Rot(x, r) + M_hi (x) Rot(x, r - n), the
 * 0/1 masks of the tokens t < n - r and t >= n - r encoded at the power of two
 * ms = 2^floor(log2 q_level), then one rescale (r = 0: x times the integer ms,
 * rescaled); scale (s ms) / q_level.  Keys: fe_attention_rotation_steps, plus
 * the relinearisation key.
 * fe_he_attention_scores: Q and K ([S][2][level+1][N] each, scales q_scale,
 * k_scale) -> the n_tok diagonals D_r[i] = A[i][(i + r) mod n] of A = Q K^T
 * (out_dev: [n_tok][2][level-1][N] at level - 2): for each r, the S fragment
 * products Q' (x) K_r (Q' = Q with one limb dropped, K_r K rotated token-wise
 * by r) summed before one relinearisation, rescaled, then summed over the P
 * positions (acc +=
 * Rot(acc, 2^k n)), so D_r holds A[i][(i + r) mod n] at slot f n + i of every
 * position f.  *out_scale = (q_scale ((k_scale ms) / q_l)) / q_{l-1}.
 * fe_he_attention_apply: D (n_tok ciphertexts at d_level, scale d_scale) and V
 * ([S] at v_level) -> O = A V in V's layout: for each fragment of V, the n
 * products D_r (x) V_r (V_r V rotated token-wise by r, the higher of the two
 * with limbs dropped to meet the other, level m = min(v_level - 1, d_level))
 * summed before one relinearisation, rescaled once: *out_level = m - 1,
 * *out_scale = (d_scale
 * ((v_scale ms) / q_{v_level})) / q_m.  Softmax and other non-linear parts of
 * attention are not included.  Composed from the library's primitives with
 * stream-ordered scratch.  Each call encodes its 2 (n_tok - 1) masks once
 * (2 (n_tok - 1) (level + 1) N 8 bytes: 3.2 GB at n_tok = 128, level 23,
 * N = 2^16) and hoists the token rotations of a chunk of offsets (about 2 GB
 * of rotated copies, plus the chunk's CMult scratch); synchronises `stream`
 * once, after the mask encode.  Errors: FE_EKEY, FE_ELEVEL, FE_EINVAL,
 * FE_ENOMEM, FE_EENCODE. */
int fe_attention_rotation_steps(const fe_ctx* ctx, const fe_token_layout* lay, int32_t* steps, uint32_t max,
                                uint32_t* n_steps);
int fe_he_attention_scores(fe_ctx* ctx, const fe_evk* evk, const fe_token_layout* lay, const void* q_dev,
                           const void* k_dev, uint32_t level, double q_scale, double k_scale, void* out_dev,
                           double* out_scale, void* stream);
int fe_he_attention_apply(fe_ctx* ctx, const fe_evk* evk, const fe_token_layout* lay, const void* d_dev,
                          uint32_t d_level, double d_scale, const void* v_dev, uint32_t v_level, double v_scale,
                          void* out_dev, uint32_t* out_level, double* out_scale, void* stream);
/* The block-size choice of Sec. 7: the rotation complexity gamma E / S + 2 n S
 * (FFN and projections: embedding aggregation over E / S positions, gamma the
 * FFN's expansion; attention: token-wise aggregation over S times more tokens
 * per ciphertext) taken as a count, minimised over the power-of-two S <= max_S
 * (0: 64) that divide E, ties to the smaller S; *rotations (optional) receives
 * its value, *s_star (optional) the continuous optimum sqrt(gamma E / (2 n)).
 * Pure host computation.  Errors: FE_EINVAL. */
int fe_choose_token_fragment(uint32_t E, uint32_t n_tok, double gamma, uint32_t max_S, uint32_t* S,
                             double* rotations, double* s_star);

/* Read a fully connected plan's decrypted output slots back as outputs:
 * y_dev[b][n] (BS x F_out, float64) = slots_dev[n / P][(n mod P) BS + b]
 * (slots_dev: the plan's n_out_ct decoded slot vectors of N/2 doubles).
 * Errors: FE_EINVAL. */
int fe_fc_unpack(const fe_ctx* ctx, const fe_plan* plan, const double* slots_dev, double* y_dev, void* stream);
void fe_plan_destroy(fe_plan* plan);

/* Sizes of a plan's buffers: encoded weight plaintexts, input / output
 * ciphertext arrays, and the default device workspace for fe_he_conv /
 * fe_he_fc (a larger workspace lets the batched path take larger chunks). */
typedef struct {
    size_t pt_bytes, in_bytes, out_bytes, workspace_bytes, workspace_min_bytes;
    uint32_t n_in_ct, n_out_ct, n_pt, n_inner_rot, n_outer_rot;
    uint32_t bsgs_n1;  /* baby steps of the outer rotations actually used (0: linear) */
    uint32_t double_hoist;  /* 1: rotations and MAC on Q_l * P; 2: the same with ModDown and
                               rescale fused when there is no outer rotation (fe_plan_set_hoisting) */
} fe_plan_info;
int fe_plan_query(const fe_plan* plan, fe_plan_info* info);
/* Rotation steps the plan needs keys for (steps_host has room for max entries;
 * *n_steps receives the count). */
int fe_plan_rotation_steps(const fe_plan* plan, int32_t* steps_host, uint32_t max,
                           uint32_t* n_steps);

/* Encode the layer's weights into plaintexts (pt_dev, plan pt_bytes) at
 * `w_scale` (the scale the layer multiplies in; q_level keeps the ciphertext
 * scale unchanged across the layer).  weights_host: float64, conv
 * (Cout, Cin, K, K) or (C, 1, K, K) when depthwise; FC (F_out, F_in).  Every
 * weight is multiplied by wmul first (a folded 1/4 of a preceding pooling).
 * Zero weights at invalid output positions make the plaintexts the fragment
 * masks of Fig. 2.
 * Layout (opaque to callers, but fixed): plaintexts one after another, each
 * [level+1] limbs (level+1+k under double hoisting) in NTT form; a limb is
 * N / T tiles of T = min(512, N) consecutive residues, and a tile is the low 32
 * bits of its T residues (uint32) followed by their high bits, hb bytes each
 * (hb = 1 when every modulus of the context is below 2^40, 2 below 2^48, else
 * 4), (4 + hb) T bytes in all.  The residues are the same
 * as those of fe_encode; only their storage is narrower, so the PMult-MAC reads
 * (4 + hb) / 8 of the bytes. */
int fe_plan_load_weights(fe_ctx* ctx, fe_plan* plan, const double* weights_host, double wmul,
                         double w_scale, void* pt_dev, void* stream);
/* The scale rule for a chain of layers (the weights' scale of Sec. 4.3 / Sec. 5):
 * a linear layer at `level` with input scale s_in encodes its weights at
 *   *w_scale = (t / s_in) q_level,
 * so that its output after the rescale by q_level has scale t: t = delta, or,
 * when an activation with leading coefficient act_a != 0 follows (x^2: 1),
 * t = sqrt(delta q_{level-1} |act_a|), which that activation's rescale brings
 * back to delta (fe_poly_act_scale).  IEEE double, in the order written.
 * Errors: FE_ELEVEL (level 0 or above L), FE_EINVAL. */
int fe_weight_scale(const fe_ctx* ctx, uint32_t level, double s_in, double delta, double act_a, double* w_scale);
/* Output scale of a conv or FC plan whose weights were loaded at w_scale:
 * (in_scale w_scale) / q_level.  Errors: FE_EINVAL (weights not loaded). */
int fe_plan_out_scale(const fe_plan* plan, double in_scale, double* out_scale);

/* Run a planned HE convolution: in_dev [n_in_ct][2][level+1][N] -> out_dev
 * [n_out_ct][2][level][N] (rescaled once).  mode 0 = plain path (one launch per
 * primitive per ciphertext), mode 1 = batched path (all ciphertexts of a stage
 * in one launch per primitive, key-stationary inner products, summed
 * rotate-and-add).  Both produce identical residues.  mode 2 = the layer
 * composed from single-ciphertext operations as a per-operation HE library
 * runs it: every rotation a full key switch of its own (no hoisting), one
 * PMult per term, one rotation and addition per partial sum, one rescale per
 * output; it gives the residues of single hoisting (also for a plan set to
 * double hoisting, whose Q*P plaintexts it reads on Q) and is not captured.
 * Errors: FE_EKEY, FE_ENOMEM (workspace too small). */
int fe_he_conv(fe_ctx* ctx, const fe_evk* evk, const fe_plan* plan, const void* pt_dev,
               const void* in_dev, void* out_dev, void* workspace_dev, size_t workspace_bytes,
               int mode, void* stream);
/* Run a planned FC layer (same buffer conventions as fe_he_conv). */
int fe_he_fc(fe_ctx* ctx, const fe_evk* evk, const fe_plan* plan, const void* pt_dev,
             const void* in_dev, void* out_dev, void* workspace_dev, size_t workspace_bytes,
             int mode, void* stream);

/* Workspace bytes for running `plan` on n_req requests at once
 * (fe_he_layer_batch); minimum = 1 gives the smallest workspace that works
 * (outer rotations one at a time), 0 the default (all outer rotations in one
 * chunk unless that needs more than 8 GiB of scratch).  0 on a null plan. */
size_t fe_plan_workspace_bytes(const fe_plan* plan, uint32_t n_req, int minimum);
/* One planned conv or FC layer (Sec. 3.1 / Sec. 5) for n_req independent
 * requests that share the plan, its plaintexts and the keys: in_dev holds
 * [n_req][n_in_ct] ciphertexts at the plan's level, out_dev receives
 * [n_req][n_out_ct] at level - 1.  Items that use the same rotation key are
 * grouped across requests, so each key is streamed once for all of them.  Each
 * request's output residues are identical to running it alone (fe_he_conv /
 * fe_he_fc).  ws: at least fe_plan_workspace_bytes(plan, n_req, 1) bytes.
 * Errors as fe_he_conv. */
int fe_he_layer_batch(fe_ctx* ctx, const fe_evk* evk, const fe_plan* plan, const void* pt_dev,
                      const void* in_dev, void* out_dev, uint32_t n_req, void* ws, size_t ws_bytes,
                      int mode, void* stream);

/* For latency measurement only: run one conv / FC plan with its plaintexts
 * taken cyclically from a pool (term t uses pool plaintext t mod n_pool;
 * pt_pool_dev holds n_pool plaintexts in the layout of fe_plan_load_weights,
 * pt_bytes / n_pt bytes each; any bytes will do).  The kernels,
 * launches and memory volume are those of fe_he_conv; the result is not the
 * layer's.  Errors as fe_he_conv. */
int fe_he_layer_timing(fe_ctx* ctx, const fe_evk* evk, const fe_plan* plan, const void* pt_pool_dev,
                       uint32_t n_pool, const void* in_dev, void* out_dev, void* ws, size_t ws_bytes,
                       void* stream);
/* Hoisting of a plan's inner (and baby-step) rotations.  double_hoist = 0: each
 * rotated copy is brought back to Q_l by its own ModDown (the rotation of
 * Eq. 1).  double_hoist = 1: the rotated copies stay on the key-switching
 * basis Q_l * P as sigma_g((P c0, 0) + key inner product), unrotated inputs
 * are lifted to (P c0, P c1), plaintexts are encoded on Q_l * P, and every
 * partial sum of the MAC takes one ModDown (double hoisting; same convolution,
 * fewer ModDowns, different rounding, its own oracle schedule).
 * double_hoist = 2: as 1, and when the plan has no outer rotation (depthwise
 * layers; baby-step / giant-step with n1 = cpc) every output's one partial sum
 * on Q_l * P is divided by q_l P in a single centred conversion instead of a
 * ModDown followed by the rescale (one transform of the output's limbs saved;
 * one rounding instead of two, its own oracle schedule); with outer rotations
 * it is 1.  Must be set before fe_plan_load_weights: it changes the plaintext
 * size (pt_bytes).  Errors: FE_EINVAL. */
int fe_plan_set_hoisting(fe_plan* plan, int double_hoist);
/* Tile choice of the batched MAC: how many outputs whose terms read the same
 * ciphertexts share one kernel item (1, 2 or 4; default 4).  Results do not
 * depend on it; the autotuner picks the fastest.  Errors: FE_EINVAL. */
int fe_plan_set_mac_ways(fe_plan* plan, uint32_t ways);
/* Depthwise plans under double hoisting, batched path: with enable = 1
 * (default) the MAC forms every rotated copy sigma_g((P c0, 0) + acc) on the
 * fly from the key inner product's accumulators and the lifted input, instead
 * of a lift pass writing the copies for the MAC to read back (the copies'
 * store and reload are saved; same residues).  0 keeps the separate lift.
 * Other plans and the per-primitive path always lift first.  Changes the
 * plan's workspace layout only within fe_plan_workspace_bytes.
 * Errors: FE_EINVAL. */
int fe_plan_set_lift_fusion(fe_plan* plan, int enable);
/* Keep only the first max_out_ct output ciphertexts of a plan (with the terms,
 * plaintexts and inner rotations they use); their results are unchanged.  Used
 * to time a slice of a large layer.  Errors: FE_EINVAL. */
int fe_plan_truncate(fe_plan* plan, uint32_t max_out_ct);

/* x^2 activation (fe_he_poly_act with a = 1, b = c = 0; same residues):
 * CMult with relinearisation, then rescale.  in: [n_ct][2][level+1][N],
 * out: [n_ct][2][level][N].  Workspace: fe_square_workspace_bytes. */
size_t fe_square_workspace_bytes(const fe_ctx* ctx, uint32_t n_ct, uint32_t level);
int fe_he_square(fe_ctx* ctx, const fe_evk* evk, const void* in_dev, uint32_t n_ct, uint32_t level,
                 void* out_dev, void* workspace_dev, size_t workspace_bytes, void* stream);

/* The activation a x^2 + b x + c that replaces ReLU (Sec. 5, Implementation),
 * on n_ct ciphertexts at `level` with scale in_scale, in one level:
 *   a != 0: a x^2 + b x + c = a [(x + beta)^2 + gamma], beta = b / (2a),
 *     gamma = c / a - beta^2: add K1 = nearest(beta s) to the constant term,
 *     CMult with relinearisation, multiply by sign(a) and add
 *     K2 = sign(a) nearest(gamma s s), rescale by q_level; the output decrypts
 *     to a x^2 + b x + c at scale (s s) / (q_level |a|);
 *   a == 0: multiply by nearest(b q_level), add nearest(c (s q_level)), rescale:
 *     scale s.
 * nearest() is the nearest integer of the IEEE double, ties away from zero.
 * With a = 1, b = c = 0 the residues are fe_he_square's.  out: [n_ct][2][level][N];
 * *out_scale (optional) receives the output scale.  Workspace:
 * fe_poly_act_workspace_bytes.  Errors: FE_ELEVEL, FE_EKEY (no relinearisation
 * key when a != 0), FE_ENOMEM, FE_EINVAL (non-finite coefficient or scale). */
size_t fe_poly_act_workspace_bytes(const fe_ctx* ctx, uint32_t n_ct, uint32_t level);
int fe_poly_act_scale(const fe_ctx* ctx, uint32_t level, double in_scale, double a, double* out_scale);
int fe_he_poly_act(fe_ctx* ctx, const fe_evk* evk, double a, double b, double c, const void* in_dev, uint32_t n_ct,
                   uint32_t level, double in_scale, void* out_dev, double* out_scale, void* workspace_dev,
                   size_t workspace_bytes, void* stream);

/* 2x2 average pooling by summing fragment ciphertexts (S even; Sec. 5, Implementation): output
 * fragment (u, v) = sum of input fragments (2u + di, 2v + dj); the 1/4 is left
 * to the next layer's weights.  out_lay receives the output layout (S / 2). */
int fe_he_avgpool(fe_ctx* ctx, const fe_layout* lay, const void* in_dev, uint32_t level,
                  void* out_dev, fe_layout* out_lay, void* stream);

/* Arch-aware Ciphertext Compression (Sec. 4.3, Fig. 6): ciphertexts whose first
 * c_valid channel positions hold data and whose other positions are zero are
 * filled by rotate-and-add doubling, ct += Rot(ct, -s m^2 BS) for
 * s = c_valid, 2 c_valid, ..., cpc / 2; position c then holds channel c mod c_valid.
 * Consumes no level.  Needs rotation keys for -s m^2 BS.  Workspace:
 * fe_compress_workspace_bytes. */
size_t fe_compress_workspace_bytes(const fe_ctx* ctx, uint32_t n_ct, uint32_t level);
int fe_compress(fe_ctx* ctx, const fe_evk* evk, const fe_layout* lay, uint32_t c_valid,
                const void* in_dev, uint32_t n_ct, uint32_t level, void* out_dev,
                void* workspace_dev, size_t workspace_bytes, void* stream);

/* AAC with its plaintext mask (Sec. 4.3, last paragraph), for inputs whose empty
 * channel blocks are not zero (e.g. after an activation with c != 0): every
 * ciphertext is multiplied by the 0/1 mask of the valid blocks (slots below
 * c_valid m^2 BS), encoded at scale mask_scale (Delta_2), and then replicated
 * as by fe_compress.  No rescale: the output stays at `level` with scale
 * in_scale mask_scale (*out_scale, optional), and the next layer's weights take
 * Delta_1 = q_level t / (in_scale Delta_2) from fe_weight_scale, so one rescale
 * follows both multiplications.  The mask's encoding error is about
 * sqrt(N / 12) / Delta_2 of the values: choose Delta_2 well above sqrt(N).
 * Workspace: fe_compress_masked_workspace_bytes.  Errors as fe_compress,
 * FE_EINVAL (mask_scale below 1). */
size_t fe_compress_masked_workspace_bytes(const fe_ctx* ctx, uint32_t n_ct, uint32_t level);
int fe_compress_masked(fe_ctx* ctx, const fe_evk* evk, const fe_layout* lay, uint32_t c_valid, double mask_scale,
                       const void* in_dev, uint32_t n_ct, uint32_t level, double in_scale, void* out_dev,
                       double* out_scale, void* workspace_dev, size_t workspace_bytes, void* stream);

/* ---- batched, graph-captured execution ------------------------------------- */

/* Capture the batched path of n planned layers (conv or FC) into one CUDA graph
 * (stream capture on `stream`, which must not be the legacy default stream).
 * Layer i reads ins_host[i], writes outs_host[i] and uses plaintexts pts_host[i];
 * layers run in the order given, so a layer may read an earlier layer's output.
 * Every layer's item tables are uploaded into workspace_dev before capture (its
 * size: fe_graph_workspace_bytes(plans, n, 1)), so the graph replays kernels
 * only.  Counters are not advanced by graph launches.  The calls that run a
 * plan or a key switch directly (fe_he_conv, fe_he_fc, fe_he_layer_batch,
 * fe_he_lintrans, fe_he_repack, fe_rotate, fe_he_bootstrap and the like) copy
 * such tables from host memory on every call; when their stream is being
 * captured by the caller, the tables travel as kernel parameters instead (one
 * small copy kernel per 2 KB, kept by value in the graph), so the caller's
 * graph replays them correctly, with those extra launches. */
int fe_graph_capture(fe_ctx* ctx, const fe_evk* evk, const fe_plan* const* plans_host,
                     const void* const* pts_host, const void* const* ins_host,
                     void* const* outs_host, uint32_t n, void* workspace_dev,
                     size_t workspace_bytes, void* stream, fe_graph** out);
/* The same for n_req requests per layer (fe_he_layer_batch layout: layer i reads
 * [n_req][n_in_ct] ciphertexts at ins_host[i] and writes [n_req][n_out_ct] at
 * outs_host[i]).  The workspace holds every layer's item tables and one data
 * region (rotated copies, partial sums, scratch) that the layers share, since
 * they run in order; its size is fe_graph_workspace_bytes(plans, n, n_req). */
size_t fe_graph_workspace_bytes(const fe_plan* const* plans_host, uint32_t n, uint32_t n_req);
int fe_graph_capture_batch(fe_ctx* ctx, const fe_evk* evk, const fe_plan* const* plans_host,
                           const void* const* pts_host, const void* const* ins_host,
                           void* const* outs_host, uint32_t n, uint32_t n_req, void* workspace_dev,
                           size_t workspace_bytes, void* stream, fe_graph** out);
/* As fe_graph_capture_batch, with the requests of every layer taken req_chunk
 * at a time (the last chunk may be smaller): each chunk's kernels run in
 * order over one data region sized for req_chunk requests, so the workspace
 * (fe_graph_workspace_bytes_chunked) grows with n_req only through the item
 * tables.  Residues are the same as with one chunk.  For request counts whose
 * hoisted rotated copies do not fit the device at once.  Errors as
 * fe_graph_capture_batch. */
size_t fe_graph_workspace_bytes_chunked(const fe_plan* const* plans_host, uint32_t n, uint32_t n_req,
                                        uint32_t req_chunk);
int fe_graph_capture_chunked(fe_ctx* ctx, const fe_evk* evk, const fe_plan* const* plans_host,
                             const void* const* pts_host, const void* const* ins_host, void* const* outs_host,
                             uint32_t n, uint32_t n_req, uint32_t req_chunk, void* workspace_dev,
                             size_t workspace_bytes, void* stream, fe_graph** out);
int fe_graph_launch(fe_graph* graph, void* stream);
/* The captured sequence's host-visible ends: its external inputs (layer inputs
 * that no earlier layer of the graph writes) and final outputs (layer outputs
 * that no later layer reads), each counted once, in layer order, with their
 * sizes in bytes (n_req x ciphertexts x [2][level+1][N] uint64).  in_bytes /
 * out_bytes may be NULL (counts only); otherwise they have room for the counts.
 * Errors: FE_EINVAL. */
int fe_graph_io(const fe_graph* graph, uint32_t* n_in, size_t* in_bytes, uint32_t* n_out, size_t* out_bytes);
/* One end-to-end step of a captured graph through host memory: on `stream`,
 * copy in_host[i] (fe_graph_io's in_bytes[i] bytes) into external input i,
 * replay the graph, and copy final output j into out_host[j].  Enqueued only:
 * the host buffers must stay valid until the stream reaches the copies (page-
 * locked buffers make the copies asynchronous; pageable ones are staged by the
 * driver).  The caller owns the host buffers.  Errors: FE_EINVAL, FE_ECUDA. */
int fe_graph_launch_host(fe_graph* graph, const void* const* in_host, void* const* out_host, void* stream);
/* Level at which fe_graph_launch_host hands the final outputs to the host:
 * the first level + 1 limbs of every polynomial, i.e. the same ciphertexts
 * modulo q_0 .. q_level (an exact modulus drop, the usual step before a
 * result leaves the server; the client decrypts them at that level and the
 * same scale).  fe_graph_io's out_bytes follow it.  UINT32_MAX (the default)
 * copies the outputs at their own level.  Errors: FE_EINVAL, FE_ELEVEL (above
 * an output's level). */
int fe_graph_set_host_output_level(fe_graph* graph, uint32_t level);
void fe_graph_destroy(fe_graph* graph);

/* ---- latency model (learned fragment / schedule proposer) ------------------- */

/* A small fully connected regression model in fp32 (no counterpart in the
 * paper; it proposes a fragment size and schedule per layer from measured
 * latencies, with the analytic choice of fe_choose_fragment as its fallback
 * and judge): in_dim -> hidden x n_hidden (ReLU) -> 1.  Weights He-uniform
 * from SplitMix64(seed), biases zero.  Parameters are laid out per layer as
 * W [out][in] then b [out].  Training is full-batch Adam (beta 0.9 / 0.999,
 * eps 1e-8, decoupled weight decay) on the mean squared error of the
 * standardised target; features and target are standardised with the
 * training set's statistics, which prediction reuses.  All arithmetic runs in
 * the library's CUDA kernels. */
typedef struct fe_mlp fe_mlp;
int fe_mlp_create(uint32_t in_dim, uint32_t hidden, uint32_t n_hidden, uint64_t seed, fe_mlp** out);
void fe_mlp_destroy(fe_mlp* m);
size_t fe_mlp_param_count(const fe_mlp* m);
/* Copy all parameters to / from host memory (fe_mlp_param_count floats). */
int fe_mlp_get_params(const fe_mlp* m, float* host);
int fe_mlp_set_params(fe_mlp* m, const float* host);
/* Feature means / standard deviations (in_dim each) and the target's mean and
 * standard deviation, as fixed by the last training call. */
int fe_mlp_get_scaling(const fe_mlp* m, float* x_mean, float* x_std, float* y_mean_std);
/* `steps` Adam steps on X_dev [n][in_dim], y_dev [n] (device, fp32, 16-byte
 * aligned); *final_loss (optional) receives the standardised MSE after
 * training.  Needs a non-default stream (one step is graph-captured).
 * Errors: FE_EINVAL, FE_ECUDA. */
int fe_mlp_train(fe_mlp* m, const float* X_dev, const float* y_dev, uint32_t n, uint32_t steps, float lr,
                 float weight_decay, float* final_loss, void* stream);
/* y_dev [n] = model(X_dev [n][in_dim]) in the target's original units. */
int fe_mlp_predict(fe_mlp* m, const float* X_dev, uint32_t n, float* y_dev, void* stream);

/* ---- request loop (serving) --------------------------------------------------- */

/* A serving loop over registered models (no counterpart in the paper, which
 * evaluates one request at a time; the usage flow of Sec. 4.1 per request):
 * requests are batched continuously, admitted by device memory, and run with
 * keys and plaintexts resident.  One scheduler thread per server forms launch
 * groups of up to max_batch pending requests of one model (the model of the
 * oldest pending request), shrunk until the group's device memory fits the
 * budget beside the groups in flight, and runs each group on its own stream
 * (max_inflight streams), so that groups of different models and ring sizes
 * overlap on the device.  A request that cannot fit alone into the whole
 * budget finishes with FE_ENOMEM.  A request's residues do not depend on the
 * group it ran in.  The caller must not use a registered context from other
 * threads while the server runs (its counters are not synchronised). */
typedef struct {
    uint32_t max_batch;        /* requests per launch group, >= 1 */
    uint32_t max_inflight;     /* launch groups (streams) on the device at once, 1..64 */
    size_t hbm_budget_bytes;   /* device bytes for request data; 0: free memory at creation - reserve */
    size_t hbm_reserve_bytes;  /* kept free when hbm_budget_bytes = 0 */
} fe_server_config;

enum { FE_OP_LAYER = 0, FE_OP_SQUARE = 1, FE_OP_POOL = 2, FE_OP_POLY_ACT = 3, FE_OP_REFRESH = 4 };
/* One operation of a model, applied to the output of the previous one:
 * FE_OP_LAYER: a conv or FC plan with its plaintexts (fe_he_layer_batch);
 * FE_OP_SQUARE: x^2 (fe_he_square); FE_OP_POOL: 2x2 average pooling of the
 * fragment layout `layout` (fe_he_avgpool); FE_OP_POLY_ACT: a x^2 + b x + c on
 * inputs of declared scale in_scale (fe_he_poly_act, one level); FE_OP_REFRESH:
 * the ciphertext refresh `boot` of inputs of declared scale in_scale
 * (fe_boot_prepare then fe_he_bootstrap; the level becomes the boot's output
 * level), which lets a served model go deeper than its levels.  Plans,
 * plaintexts and refreshes are owned by the caller and must outlive the server. */
typedef struct {
    int kind;
    const fe_plan* plan;
    const void* pt_dev;
    fe_layout layout;
    double a, b, c;      /* FE_OP_POLY_ACT */
    double in_scale;     /* FE_OP_POLY_ACT, FE_OP_REFRESH */
    const fe_boot* boot; /* FE_OP_REFRESH */
} fe_op;

typedef struct {
    uint64_t submitted, completed, rejected, groups, max_group;
    uint64_t max_inflight;  /* peak concurrency: the most groups whose device intervals (each
                               from the moment its stream starts the input copies to its
                               completion, timed with CUDA events) held one instant; at most
                               the configured max_inflight */
    size_t peak_bytes, budget_bytes;
    double p50_ms, p99_ms, mean_ms, wall_s;  /* latency: submit -> result in the host buffer */
} fe_server_stats_t;

/* Start a server (and its scheduler thread) on the current device.
 * Errors: FE_EINVAL, FE_ECUDA. */
int fe_server_create(const fe_server_config* cfg, fe_server** out);
/* Register a model: ops[0..n_ops) on context ctx with keys evk; requests carry
 * in_ct ciphertexts at in_level ([in_ct][2][in_level+1][N] uint64).  Checks
 * that the levels and ciphertext counts chain.  Errors: FE_EINVAL, FE_ELEVEL,
 * FE_EKEY. */
int fe_server_add_model(fe_server* s, fe_ctx* ctx, const fe_evk* evk, const fe_op* ops, uint32_t n_ops,
                        uint32_t in_ct, uint32_t in_level, uint32_t* model_id);
/* Output shape of a model: ciphertext count, level and the byte sizes of a
 * request's input and output buffers. */
int fe_server_model_io(fe_server* s, uint32_t model, uint32_t* out_ct, uint32_t* out_level,
                       size_t* in_bytes, size_t* out_bytes);
/* Queue a request.  in_host / out_host are caller-owned host buffers of the
 * model's input / output size and must stay valid until the request finishes
 * (pinned memory gives asynchronous copies).  Returns at once with the id. */
int fe_server_submit(fe_server* s, uint32_t model, const void* in_host, void* out_host, uint64_t* req_id);
/* Pause (paused = 1) or resume (0) admission: queued requests wait, groups in
 * flight continue (draining, maintenance, or queueing a burst to run as one
 * batch). */
int fe_server_pause(fe_server* s, int paused);
/* Wait at most timeout_ms for a request; *status receives FE_OK or the
 * request's error, *latency_ms its submit-to-result time.  Errors: FE_ETIMEOUT
 * (not finished within the limit), FE_EINVAL (unknown id). */
int fe_server_wait(fe_server* s, uint64_t req_id, uint32_t timeout_ms, int* status, double* latency_ms);
/* Counters and nearest-rank latency percentiles of the completed requests. */
int fe_server_stats(fe_server* s, fe_server_stats_t* out);
/* Stop the scheduler, wait for the groups in flight, release the streams. */
void fe_server_destroy(fe_server* s);

/* ---- device status ------------------------------------------------------------ */

/* Bounded waits of the PMult-MAC kernel (its mbarrier waits on the bulk copies
 * that stage its operands, and on the consumers that free a stage): limit_ns is
 * the longest a thread waits (default 2 s) before it sets bit 0 of the status
 * word (fe_device_status) and stops.  unfed_term >= 0 exists to test that expiry
 * path: every MAC item then announces the bytes of its term `unfed_term` but
 * issues no copy for it, so that stage never fills, its consumers give up after
 * limit_ns, and the launch's results are invalid; -1 (the default) turns it
 * off.  Applies to launches (and graph captures) made after the call.  No
 * counterpart in the paper.  Errors: FE_EINVAL (limit 0 or above 60 s,
 * unfed_term below -1). */
int fe_ctx_set_mac_wait(fe_ctx* ctx, uint64_t limit_ns, int32_t unfed_term);

/* Synchronise the device and read the context's device status word: bit 0 is
 * set when a kernel's bounded wait on its own asynchronous copies expired (the
 * kernel then skipped its work, so the results of that call are invalid and
 * the caller should treat it as FE_ETIMEOUT).  reset = 1 clears the word. */
int fe_device_status(fe_ctx* ctx, uint32_t* status, int reset);

/* ---- kernel timing ---------------------------------------------------------- */

/* Time every launch of one kernel class with CUDA events recorded on the
 * launching stream: kind is one of "ntt" (forward and inverse NTT passes),
 * "bconv", "keyip", "combine" (ModDown combine, single and summed), "mac",
 * "rescale", "encode".  While active, each launch of that class also adds its
 * algorithmic bytes (words each launch must read and write once) to a total.
 * Kinds: "ntt", "bconv", "keyip", "combine", "mac", "rescale", "encode", and
 * the stages of a planned layer "stage_inner", "stage_base", "stage_outer",
 * "stage_rescale" (one interval per stage and layer call).
 * fe_profile_end synchronises the recorded streams and returns the summed
 * duration in ms, the launch count and the algorithmic bytes.  Not for use
 * inside stream capture. */
int fe_profile_begin(fe_ctx* ctx, const char* kind);
int fe_profile_end(fe_ctx* ctx, double* total_ms, uint64_t* launches, double* bytes);

/* ---- ciphertext refresh (bootstrapping) ----------------------------------- */
/* The paper's deeper networks (SqueezeNet, ResNet18, MobileNet) refresh their
 * ciphertexts between blocks with an existing CKKS bootstrapping (Sec. 5,
 * Evaluation Methodology: NEXUS's, 14 levels per refresh); the paper does not
 * print its steps.  The library implements the standard CKKS refresh for its
 * real-slot encoding: ModRaise, CoeffToSlot (the special FFT's inverse stages
 * in n_cts groups, one level each), EvalMod (a degree-16 Taylor cosine and r
 * double angles, 5 + r levels) and SlotToCoeff (n_stc groups).  ModRaise needs
 * a sparse secret (fe_sk_gen_sparse): either the context's secret, or one the
 * refresh borrows from a network with a dense secret (fe_boot_encapsulate).
 * All buffers are device memory in the ciphertext layout [n][2][level+1][N]
 * unless stated; the library never frees caller buffers. */

/* n_cts / n_stc: stage groups of CoeffToSlot / SlotToCoeff (1..log2(N/2));
 * r: double angles (1..16); top: level after ModRaise (0: L); baby_ratio: every
 * group takes n1 baby steps, the smallest power of two with n1^2 >= baby_ratio
 * x its number of diagonal offsets (0 or 1: about the square root; larger
 * values trade giant-step rotations, each with its own ModUp, for hoisted
 * baby steps); double_hoist: 1 keeps every group's baby rotations on Q * P
 * and takes one ModDown per (output, giant step) sum (fe_plan_set_hoisting 1),
 * 0 a ModDown per rotation; form: 0 runs the transforms on the pair (re, im)
 * of real-slot ciphertexts with real diagonals (the output has real slots), 1 on
 * one ciphertext with complex diagonals (half the rotations; the real and
 * imaginary parts are split after CoeffToSlot by one conjugation and joined
 * before SlotToCoeff; the output's imaginary parts are noise).  The refresh
 * needs n_cts + 5 + r + n_stc <= top and returns at level top - that depth. */
typedef struct {
    uint32_t n_cts, n_stc, r, top, baby_ratio, double_hoist, form;
} fe_boot_params;

/* Sparse ternary secret of Hamming weight h (h distinct positions with signs
 * +-1, by a partial Fisher-Yates shuffle on the generator's words of tag
 * kind 6), written like fe_sk_gen's ([n_mod][N], NTT form).  A refresh needs a
 * sparse secret so that the multiples of q_0 that ModRaise adds stay small
 * (|I| <= (h + 1) / 2).  Errors: FE_EINVAL (h = 0 or h > N). */
int fe_sk_gen_sparse(fe_ctx* ctx, uint64_t seed, uint32_t h, void* sk_dev, void* stream);
/* Complex conjugation of the slots of n_ct ciphertexts (automorphism X -> X^(2N-1)
 * with its key switch, Eq. 1's form); the evk must hold the step FE_STEP_CONJ.
 * Errors: FE_EKEY. */
int fe_conjugate(fe_ctx* ctx, const fe_evk* evk, const void* ct_dev, uint32_t n_ct, uint32_t level,
                 void* out_dev, void* stream);
/* Level drop: n_ct ciphertexts at `level` modulo the smaller modulus
 * Q_to_level = q_0 ... q_to_level (each polynomial keeps its first to_level + 1
 * limbs); exact, the message and its scale are unchanged.  This is how a
 * ciphertext reaches level 0 before a refresh without spending rescales.
 * Errors: FE_ELEVEL (to_level > level or level > L), FE_EINVAL (in place). */
int fe_mod_drop(fe_ctx* ctx, const void* ct_dev, uint32_t n_ct, uint32_t level, uint32_t to_level, void* out_dev,
                void* stream);
/* ModRaise: n_ct level-0 ciphertexts, read as centred integers mod q_0, reduced
 * modulo q_0..q_top (out: level `top`).  The result decrypts to m + q_0 I.
 * Errors: FE_ELEVEL (top > L). */
int fe_mod_raise(fe_ctx* ctx, const void* ct_dev, uint32_t n_ct, uint32_t top, void* out_dev, void* stream);

/* Plaintext-matrix product by the diagonal method with baby / giant steps (the
 * linear transforms of the refresh; any real slot-linear map):
 *   out[o] = rescale( sum over diagonals (o, i, r) of d ⊙ Rot(in[i], r) ),
 * d the diagonal's slot vector, Rot(v, r)[l] = v[l + r].  Offsets are split as
 * r = giant + baby: r_lo = min offset, delta = gcd of (r - r_lo) (1 if all are
 * equal), j = (r - r_lo) / delta, baby = (j mod n1) delta, giant = r_lo +
 * (j div n1) n1 delta; the baby rotations of each input share one ModUp, each
 * (output, giant) sum is rotated once.  Diagonals: n_diag triples (diag_out,
 * diag_in, diag_offset), offsets in (-N/2, N/2), no duplicates, every output
 * with at least one diagonal; n1 = 0 picks the power of two at or above
 * sqrt(#distinct offsets).  The plan runs through fe_plan_query,
 * fe_plan_rotation_steps, fe_plan_workspace_bytes and fe_plan_destroy like
 * the layer plans.  Errors: FE_EINVAL, FE_ELEVEL (level 0 or above L). */
int fe_plan_lintrans(fe_ctx* ctx, uint32_t n_in, uint32_t n_out, uint32_t n_diag, const uint32_t* diag_out,
                     const uint32_t* diag_in, const int32_t* diag_offset, uint32_t n1, uint32_t level,
                     fe_plan** out);
/* Encode the diagonals (values_host: [n_diag][N/2] doubles, in planning order)
 * at w_scale on q_0..q_level into pt_dev (fe_plan_query's pt_bytes).  Output
 * scale = input scale * w_scale / q_level.  Synchronises `stream`. */
int fe_plan_lintrans_load(fe_ctx* ctx, fe_plan* plan, const double* values_host, double w_scale, void* pt_dev,
                          void* stream);
/* Run the product for n_req requests (inputs [n_req][n_in], outputs
 * [n_req][n_out] at level - 1); ws: fe_plan_workspace_bytes(plan, n_req, 0). */
int fe_he_lintrans(fe_ctx* ctx, const fe_evk* evk, const fe_plan* plan, const void* pt_dev, const void* in_dev,
                   void* out_dev, uint32_t n_req, void* ws, size_t ws_bytes, void* stream);

/* Build a refresh: every stage group's diagonals (twiddles cos / sin(pi e / N)
 * rounded once from quad precision; 1/2 and pi / 2^r folded into the first
 * CoeffToSlot group, q_0 / (2 pi scale_in) into the first SlotToCoeff group)
 * encoded on device memory the object owns, and the -X^(N/2) factor of the
 * imaginary part.  scale_in: the declared scale of the level-0 inputs (slot
 * values |z| <= 1 want scale_in well below q_0, e.g. q_0 / 32).  Synchronises
 * `stream`.  Errors: FE_EINVAL, FE_ELEVEL, FE_ENOMEM, FE_ECUDA. */
int fe_boot_create(fe_ctx* ctx, const fe_boot_params* params, double scale_in, void* stream, fe_boot** out);
/* Rotation steps the refresh needs (mod N/2, and FE_STEP_CONJ); *n receives the
 * count, at most `max` are written.  The evk also needs the relinearisation key. */
int fe_boot_rotation_steps(const fe_boot* boot, int32_t* steps, uint32_t max, uint32_t* n);
/* Level and declared scale of the refresh's outputs. */
int fe_boot_output(const fe_boot* boot, uint32_t* level, double* scale);
/* Device workspace of fe_he_bootstrap for n_ct ciphertexts (0 for n_ct = 0). */
size_t fe_boot_workspace_bytes(const fe_boot* boot, uint32_t n_ct);
/* Refresh n_ct level-0 ciphertexts (declared scale scale_in) into out_dev at
 * fe_boot_output's level; the outputs decrypt to the inputs' slot values.
 * ws: fe_boot_workspace_bytes(boot, n_ct).  Errors: FE_EKEY, FE_ENOMEM. */
int fe_he_bootstrap(fe_ctx* ctx, const fe_evk* evk, const fe_boot* boot, const void* ct_dev, uint32_t n_ct,
                    void* out_dev, void* ws, size_t ws_bytes, void* stream);
/* Capture the refresh of n_ct >= 1 ciphertexts from ct_dev into out_dev as one
 * CUDA graph (stream capture on `stream`, not the legacy default stream): the
 * transforms' item tables are uploaded into ws first (fe_boot_workspace_bytes
 * (boot, n_ct); ws must stay untouched while the graph lives), then the
 * launches alone are captured, so that fe_graph_launch replays the whole
 * refresh and gives the residues of fe_he_bootstrap on the same buffers.
 * fe_graph_io reports ct_dev as the input and out_dev as the output (level
 * fe_boot_output), so fe_graph_launch_host applies; release with
 * fe_graph_destroy.  Synchronises `stream` before the capture.  (A caller's
 * own capture of fe_he_bootstrap also replays correctly, but carries every
 * table in copy kernels.)  Errors: FE_EINVAL, FE_EKEY, FE_ENOMEM, FE_ECUDA. */
int fe_boot_graph_capture(fe_ctx* ctx, const fe_evk* evk, const fe_boot* boot, const void* ct_dev, uint32_t n_ct,
                          void* out_dev, void* ws, size_t ws_bytes, void* stream, fe_graph** out);
/* Switching key from secret sk_src to secret sk_dst (both [n_mod][N], NTT
 * form) for the hybrid key switch that rotations use (Eq. 1's KS), random
 * streams of object tag `obj` (rotation keys use their Galois element, the
 * relinearisation key 0), in the layout of one rotation key into caller-owned
 * key_dev: key_bytes >= fe_evk_bytes(ctx, 1, 0).  Synchronises `stream`.
 * Errors: FE_EINVAL (null or misaligned pointer), FE_ENOMEM (key_bytes). */
int fe_swk_gen(fe_ctx* ctx, const void* sk_src, const void* sk_dst, uint64_t seed, uint32_t obj, void* key_dev,
               size_t key_bytes, void* stream);
/* Hybrid key switch (Eq. 1's KS without the automorphism) of n_ct ciphertexts
 * at `level` from the key's source secret to its destination secret:
 * (c0 + d0, d1), (d0, d1) = KS(c1).  Scratch from the stream-ordered allocator.
 * Errors: FE_EINVAL (null pointer, in place), FE_ELEVEL (level > L). */
int fe_key_switch(fe_ctx* ctx, const void* key_dev, const void* ct_dev, uint32_t n_ct, uint32_t level,
                  void* out_dev, void* stream);
/* Sparse-secret encapsulation: the network keeps its dense secret sk_dense (the
 * evk of fe_he_bootstrap is sk_dense's) and the refresh borrows the sparse
 * secret sk_sparse (fe_sk_gen_sparse) for ModRaise only.  Generates the keys
 * dense -> sparse (object 2N) and sparse -> dense (object 2N + 2) into keys_dev
 * (2 x fe_evk_bytes(ctx, 1, 0) bytes, caller-owned, must outlive the boot) and
 * makes fe_he_bootstrap switch its level-0 inputs to the sparse secret, raise
 * them and switch them back at level top (two key switches more).
 * Synchronises `stream`.  Errors: FE_EINVAL (null pointer, another context's
 * boot), FE_ENOMEM (keys_bytes). */
int fe_boot_encapsulate(fe_ctx* ctx, fe_boot* boot, const void* sk_dense, const void* sk_sparse, uint64_t seed,
                        void* keys_dev, size_t keys_bytes, void* stream);
/* Bring n_ct ciphertexts at `level` >= 1 with declared scale in_scale to the
 * refresh's input: level 0 at the boot's scale_in, same slot values.  They are
 * dropped to level 1 (exact), multiplied by B = nearest((scale_in / in_scale)
 * q_1) and rescaled by q_1 (out: level 0).  ws: fe_boot_prepare_workspace_bytes.
 * The slot values must stay within the range the refresh was built for
 * (|z| <= about q_0 / (32 scale_in)).  Errors: FE_ELEVEL, FE_EINVAL, FE_ENOMEM. */
size_t fe_boot_prepare_workspace_bytes(const fe_ctx* ctx, uint32_t n_ct);
int fe_boot_prepare(fe_ctx* ctx, const fe_boot* boot, const void* ct_dev, uint32_t n_ct, uint32_t level,
                    double in_scale, void* out_dev, void* ws, size_t ws_bytes, void* stream);
void fe_boot_destroy(fe_boot* boot);

#ifdef __cplusplus
}
#endif

#endif /* FENC_H */
