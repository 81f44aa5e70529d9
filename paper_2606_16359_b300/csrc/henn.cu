// Encrypted layers under the fragment encoding: planning and execution of the
// HE convolution (Sec. 3.1) and of the fully connected layers, and fragment
// pack / unpack.
//
// A conv plan follows the algorithm order of Sec. 3.1:
//  1. inner rotations: input ciphertext (g, u, v) is rotated by (a m + b) BS
//     for every block offset (a, b) != (0, 0) that some tap needs; one ModUp of
//     its c1 serves all of its rotations (hoisting);
//  2. PMult-MAC over fragment masks: for output (h, u', v') and diagonal d,
//     P_d = sum_g sum_taps R(g, u, v, a, b) (x) pt(h, u', v', d, g, i, j) with
//     u = (u' + i) mod S, a = (u' + i) div S (same for columns);
//  3. outer rotations before rescale: out = P_0 + sum_{d != 0} Rot(P_d, d m^2 BS);
//  4. one rescale.
// An FC plan has the same shape: baby-step rotations of the inputs (1), MAC of
// the rotated diagonals (2), giant-step rotate-and-sum (3), rescale (4).
#include <algorithm>
#include <functional>
#include <map>
#include <memory>
#include <set>
#include <tuple>

#include "plan.h"

namespace fe {

namespace {
constexpr int kB = 256;

// block offsets a of source fragment row u needed by kept output rows u' (u' % stride == 0)
std::vector<std::vector<int>> inner_offsets(int S, int K, int stride) {
    std::vector<std::vector<int>> r(S);
    for (int u = 0; u < S; u++) {
        std::set<int> offs;
        for (int up = 0; up < S; up += stride)
            for (int i = 0; i < K; i++)
                if ((up + i) % S == u) offs.insert((up + i) / S);
        r[u].assign(offs.begin(), offs.end());
    }
    return r;
}

// ---- weight slot vectors -------------------------------------------------
struct ConvPtArgs {
    const fe_plan::ConvPt* pts;
    const double* W;
    double wmul;
    int S, m, BS, cpc, H, Wd, K, stride, Cin, Cout, depthwise, in_period;
};

__global__ void k_conv_pt_slots(ConvPtArgs a, double* z, int slots) {
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= slots) return;
    const fe_plan::ConvPt p = a.pts[blockIdx.y];
    const int blk = a.m * a.m * a.BS;
    // a baby-step plaintext is the diagonal's slot vector rotated left by p.rot
    const int ls = (l + p.rot) % slots;
    const int c_loc = ls / blk, rem = ls % blk;
    const int kblk = rem / a.BS;
    const int bi = kblk / a.m, bj = kblk % a.m;
    double v = 0.0;
    const int c = a.in_period ? c_loc % a.in_period : p.g * a.cpc + c_loc;
    const int o_loc = ((c_loc - p.d) % a.cpc + a.cpc) % a.cpc;
    const int o = p.h * a.cpc + o_loc;
    const int hp = bi * a.S + p.up, wp = bj * a.S + p.vp;
    bool ok = (a.in_period || c < a.Cin) && o < a.Cout && hp <= a.H - a.K && wp <= a.Wd - a.K &&
              hp % a.stride == 0 && wp % a.stride == 0;
    if (ok && a.depthwise && o != c) ok = false;
    if (ok) {
        const int K = a.K;
        const double w = a.depthwise ? a.W[((size_t)c * K + p.i) * K + p.j]
                                     : a.W[(((size_t)o * a.Cin + c) * K + p.i) * K + p.j];
        v = w * a.wmul;
    }
    z[(size_t)blockIdx.y * slots + l] = v;
}

struct FcPtArgs {
    const fe_plan::FcPt* pts;
    const double* W;
    const int* feat;    // [n_in][P]
    const int* rowmap;  // [F_out] neuron -> row of W (-1: zero), or null (row = neuron)
    double wmul;
    int P, BS, n1, F_in, F_out;
};

// rotated diagonal: z[p BS + b] = W[t P + ((p - n1 gam) mod P)][feat(c, (p + beta) mod P)]
__global__ void k_fc_pt_slots(FcPtArgs a, double* z, int slots) {
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= slots) return;
    const fe_plan::FcPt q = a.pts[blockIdx.y];
    const int p = l / a.BS;
    const int p0 = ((p - a.n1 * q.gam) % a.P + a.P) % a.P;
    const int n = q.t * a.P + p0;
    const int f = a.feat[(size_t)q.c * a.P + (p + q.beta) % a.P];
    double v = 0.0;
    const int row = n < a.F_out ? (a.rowmap ? a.rowmap[n] : n) : -1;
    if (row >= 0 && f >= 0) v = a.W[(size_t)row * a.F_in + f] * a.wmul;
    z[(size_t)blockIdx.y * slots + l] = v;
}

// repack mask, rotated for the giant step: z[p BS + b] = 1 when the element at
// source position (p + beta) mod P of ciphertext c has target (t, (p - n1 gam) mod P)
struct RepackPtArgs {
    const fe_plan::FcPt* pts;
    const int* feat;  // [n_in][P] source element ids
    fe_layout B;      // target layout
    int P, BS, n1;
};
__global__ void k_repack_pt_slots(RepackPtArgs a, double* z, int slots) {
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= slots) return;
    const fe_plan::FcPt q = a.pts[blockIdx.y];
    const int p = l / a.BS;
    const int p0 = ((p - a.n1 * q.gam) % a.P + a.P) % a.P;
    const int f = a.feat[(size_t)q.c * a.P + (p + q.beta) % a.P];
    double v = 0.0;
    if (f >= 0) {
        const fe_layout& B = a.B;
        const int w = f % (int)B.W, h = (f / (int)B.W) % (int)B.H, ch = f / ((int)B.W * (int)B.H);
        const int g = ch / (int)B.cpc, c_loc = ch % (int)B.cpc;
        const int ct = (g * (int)B.S + h % (int)B.S) * (int)B.S + w % (int)B.S;
        const int pos = (c_loc * (int)B.m + h / (int)B.S) * (int)B.m + w / (int)B.S;
        if (ct == q.t && pos == p0) v = 1.0;
    }
    z[(size_t)blockIdx.y * slots + l] = v;
}

// ---- fragment pack / unpack ------------------------------------------------
__global__ void k_pack(const double* x, double* slots, fe_layout L, int N) {
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    const int half = N / 2;
    if (l >= half) return;
    const int ci = blockIdx.y;
    const int S = L.S, m = L.m, BS = L.BS;
    const int g = ci / (S * S), u = (ci / S) % S, v = ci % S;
    const int blk = m * m * BS;
    const int c_loc = l / blk, rem = l % blk, kk = rem / BS, b = rem % BS;
    const int bi = kk / m, bj = kk % m;
    const int c = g * L.cpc + c_loc, h = bi * S + u, w = bj * S + v;
    double val = 0.0;
    if (c < (int)L.C && h < (int)L.H && w < (int)L.W) val = x[(((size_t)b * L.C + c) * L.H + h) * L.W + w];
    slots[(size_t)ci * half + l] = val;
}

__global__ void k_unpack(const double* slots, double* y, fe_layout L, int N) {
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t total = (size_t)L.BS * L.C * L.H * L.W;
    if (idx >= total) return;
    const int w = idx % L.W, h = (idx / L.W) % L.H, c = (idx / ((size_t)L.W * L.H)) % L.C,
              b = idx / ((size_t)L.W * L.H * L.C);
    const int S = L.S, m = L.m;
    const int g = c / L.cpc, c_loc = c % L.cpc, u = h % S, v = w % S, bi = h / S, bj = w / S;
    const int ci = (g * S + u) * S + v;
    const size_t slot = ((size_t)c_loc * m * m + bi * m + bj) * L.BS + b;
    y[idx] = slots[(size_t)ci * (N / 2) + slot];
}

struct Sizes {
    size_t ctw, nlN, extw, accw;
};
Sizes sizes_of(const fe_ctx* c, int level) {
    return {ct_words(c, level), (size_t)(level + 1) * c->N, ext_words(c, level), acc_words(c, level)};
}

// rotated groups (output, group index), sorted by step so that groups sharing a key are adjacent
std::vector<std::pair<int, int>> outer_order(const fe_plan* p) {
    std::vector<std::pair<int, int>> v;
    for (int o = 0; o < p->n_out; o++)
        for (int gi = 0; gi < (int)p->outs[o].groups.size(); gi++)
            if (p->outs[o].groups[gi].step) v.push_back({o, gi});
    std::stable_sort(v.begin(), v.end(), [&](const std::pair<int, int>& a, const std::pair<int, int>& b) {
        return p->outs[a.first].groups[a.second].step < p->outs[b.first].groups[b.second].step;
    });
    return v;
}

// Batched path, double hoisting, depthwise (one output per MAC item, no outer
// rotation): the MAC reads the key inner product's accumulators and the lifted
// inputs and forms each rotated copy on the fly (k_mac_rot) instead of the lift
// writing the copies first.  Same residues.
bool lift_in_mac(const fe_plan* p, int mode) {
    return mode == 1 && p->kind == 0 && p->dhoist && p->n_outer == 0 && p->depthwise && p->lift_mac;
}

size_t item_bytes(const fe_plan* p, size_t chunk, size_t R) {
    size_t groups = 0;
    for (auto& o : p->outs) groups += o.groups.size();
    const size_t n_outer = R * p->n_outer;
    size_t n_chunks = n_outer ? (n_outer + chunk - 1) / chunk : 0;
    size_t n = R * p->inner.size() * (sizeof(KsItem) + sizeof(KsGroup) + sizeof(CombineItem));
    n += n_outer * (sizeof(KsItem) + sizeof(KsGroup) + sizeof(SumEntry));
    n += n_chunks * R * p->n_out * sizeof(SumItem);
    n += R * (groups * sizeof(MacItem) + p->terms.size() * sizeof(MacTerm));
    if (p->dhoist) n += R * ((p->inner.size() + p->n_in) * sizeof(LiftItem) + groups * sizeof(CombineItem));
    if (p->dhoist == 2) n += R * p->n_out * sizeof(u64*);
    if (p->dhoist) n += R * (groups * sizeof(RotItem) + p->terms.size() * sizeof(RotTerm));
    return n + 23 * 256;
}

}  // namespace

int layout_fill(int N, fe_layout* l) {
    if (!l->H || !l->W || !l->C || !l->BS || !l->S) return fail(FE_EINVAL, "layout has a zero extent");
    uint32_t m = l->m;
    if (m == 0) {
        uint32_t side = (std::max(l->H, l->W) + l->S - 1) / l->S;
        m = 1;
        while (m < side) m *= 2;
    } else if (l->S * m < std::max(l->H, l->W)) {
        return fail(FE_EINVAL, "block grid too small for the map");
    }
    uint64_t slots = (uint64_t)N / 2, blk = (uint64_t)m * m * l->BS;
    if (blk > slots || slots % blk) return fail(FE_EINVAL, "one channel block does not fit a ciphertext");
    l->m = m;
    l->M = l->S * m;
    l->cpc = (uint32_t)(slots / blk);
    l->groups = (l->C + l->cpc - 1) / l->cpc;
    l->n_ct = l->groups * l->S * l->S;
    return FE_OK;
}

size_t plan_data_bytes(const fe_plan* p, size_t chunk, size_t R) {
    const fe_ctx* c = p->c;
    Sizes z = sizes_of(c, p->level);
    size_t n_mu = p->modup_cts.size(), n_in_rot = p->inner.size();
    const bool dh = p->dhoist;
    // double hoisting keeps the rotated copies and the lifted inputs on Q_l * P
    size_t persist = R * (n_in_rot * (dh ? z.accw : z.ctw) + p->n_out * z.ctw + (dh ? p->n_in * z.accw : 0));
    size_t inner = R * (n_mu * (z.nlN + z.extw) + n_in_rot * (z.accw + (dh ? 0 : z.ctw)));
    size_t base = dh ? R * p->n_out * (z.accw + z.ctw) : 0;
    size_t outer = chunk * (z.ctw + z.nlN + z.extw + z.accw + z.ctw + (dh ? z.accw + z.ctw : 0)) +
                   R * p->n_out * z.ctw;
    size_t rs = rescale_tmp_words(c, (int)(R * p->n_out), p->level);
    size_t words = persist + std::max(std::max(std::max(inner, outer), rs), base);
    // rotated copies formed in the MAC: the accumulators of stage 1 stay live while
    // stage 2 writes its sums after them
    if (lift_in_mac(p, 1)) words = std::max(words, persist + inner + base);
    return words * 8 + 24 * 256;
}

size_t plan_table_bytes(const fe_plan* p, size_t chunk, size_t R) { return item_bytes(p, chunk, R); }

size_t plan_workspace(const fe_plan* p, size_t chunk, size_t R) {
    return plan_data_bytes(p, chunk, R) + plan_table_bytes(p, chunk, R);
}

// the outer-rotation chunk run_plan takes: as large as the data region allows
size_t plan_chunk(const fe_plan* p, size_t R, int mode, size_t data_bytes, bool data_only) {
    size_t chunk = mode == 0 ? 1 : std::max<size_t>(1, R * p->n_outer);
    auto need = [&](size_t ch) { return data_only ? plan_data_bytes(p, ch, R) : plan_workspace(p, ch, R); };
    while (chunk > 1 && need(chunk) > data_bytes) chunk = (chunk + 1) / 2;
    return chunk;
}

// The layer composed from single-ciphertext operations, as a client of a
// per-operation HE library writes it (mode 2): every rotation, inner or outer,
// is a full key switch of its own (ModUp, key inner product, ModDown,
// automorphism: no hoisting, no key reuse across ciphertexts); every term is one
// PMult accumulated into its sum; each rotated partial sum is added to its
// output; each output is rescaled alone.  Same plan, rotations and plaintexts
// (the Q limbs of Q*P plaintexts under double hoisting); the residues are those
// of single hoisting.  One request at a time; nothing is captured.
int run_plan_per_op(fe_ctx* c, const fe_evk* evk, const fe_plan* p, const u64* b_in, const u64* b_pt, u64* b_out,
                    void* ws, size_t ws_bytes, cudaStream_t st) {
    const int lv = p->level;
    const Sizes z = sizes_of(c, lv);
    const size_t ctw_out = ct_words(c, lv - 1);
    const size_t ptb = (size_t)(p->dhoist ? lv + 1 + c->k : lv + 1) * pt_limb_bytes(c);
    std::map<int32_t, const u64*> keys;
    for (int32_t s : p->steps) {
        const u64* k = evk_key(evk, c->galois(s));
        if (!k) return fail(FE_EKEY, "missing rotation key for step " + std::to_string(s));
        keys[s] = k;
    }
    size_t n_rot = p->inner.size();
    for (const auto& o : p->outs)
        for (const auto& g : o.groups) n_rot += g.step != 0;
    Carver cv(ws, ws_bytes);
    KsItem* d_ks = cv.take<KsItem>(std::max<size_t>(1, n_rot));
    CombineItem* d_cb = cv.take<CombineItem>(std::max<size_t>(1, n_rot));
    u64* Rb = cv.take<u64>(p->inner.size() * z.ctw);
    u64* total = cv.take<u64>((size_t)p->n_out * z.ctw);
    u64* Pd = cv.take<u64>(z.ctw);
    u64* T = cv.take<u64>(z.ctw);
    u64* coef = cv.take<u64>(z.nlN);
    u64* ext = cv.take<u64>(z.extw);
    u64* acc = cv.take<u64>(z.accw);
    u64* conv = cv.take<u64>(z.ctw);
    u64* rs = cv.take<u64>(rescale_tmp_words(c, 1, lv));
    if (!cv.ok) return fail(FE_ENOMEM, "workspace too small for the plan");
    // one key-switch item and one combine item per rotation, in execution order
    std::vector<KsItem> ks;
    std::vector<CombineItem> cb;
    for (size_t i = 0; i < p->inner.size(); i++) {
        const auto& in = p->inner[i];
        ks.push_back(KsItem{ext, keys[in.step], acc});
        cb.push_back(CombineItem{acc, conv, b_in + (size_t)in.ci * z.ctw, nullptr, Rb + i * z.ctw,
                                 c->galois(in.step), 0});
    }
    for (const auto& o : p->outs)
        for (const auto& g : o.groups)
            if (g.step) {
                ks.push_back(KsItem{ext, keys[g.step], acc});
                cb.push_back(CombineItem{acc, conv, Pd, nullptr, T, c->galois(g.step), 0});
            }
    FE_TRY(upload(ks, d_ks, st));
    FE_TRY(upload(cb, d_cb, st));
    auto rotate = [&](const u64* src, size_t item) {
        modup(c, src + z.nlN, z.ctw, 1, lv, coef, ext, st);
        launch_keyip(c, d_ks + item, 1, lv, st);
        moddown_prepare(c, acc, 1, lv, conv, st);
        launch_combine(c, d_cb + item, 1, lv, st);
    };
    auto pmults = [&](const fe_plan::Group& g, u64* dst) {
        for (int t = 0; t < g.nt; t++) {
            const fe_plan::Term& tm = p->terms[g.t0 + t];
            const u64* src = tm.src >= 0 ? Rb + (size_t)tm.src * z.ctw : b_in + (size_t)(-tm.src - 1) * z.ctw;
            launch_pmult_compact(c, src, (const uint8_t*)b_pt + (size_t)tm.pt * ptb, dst, lv, t > 0, st);
        }
    };
    for (size_t i = 0; i < p->inner.size(); i++) rotate(b_in + (size_t)p->inner[i].ci * z.ctw, i);
    size_t item = p->inner.size();
    for (int o = 0; o < p->n_out; o++) {
        u64* out = total + (size_t)o * z.ctw;
        bool started = false;
        for (const auto& g : p->outs[o].groups)
            if (!g.step) {
                pmults(g, out);
                started = g.nt > 0;
            }
        if (!started) FE_CUDA_TRY(cudaMemsetAsync(out, 0, z.ctw * 8, st));
        for (const auto& g : p->outs[o].groups)
            if (g.step) {
                pmults(g, Pd);
                rotate(Pd, item++);
                launch_add(c, out, T, out, 1, lv, st);
            }
        rescale_batch(c, out, 1, lv, b_out + (size_t)o * ctw_out, rs, rs + 2 * (size_t)c->N, st);
    }
    c->cnt.rot += n_rot;
    c->cnt.keyswitch += n_rot;
    c->cnt.pmult += p->terms.size();
    FE_CUDA_TRY(cudaGetLastError());
    return FE_OK;
}

// Both phases derive every pointer from (plan, buffers, workspace) alone, so a
// graph can be captured from the launch phase after an upload phase.
// n_req requests share the plan, its plaintexts and keys: request r reads its
// inputs at b_in + r n_in ct words and writes its outputs at b_out + r n_out
// (level - 1) ct words.  Items that use one key are grouped across requests,
// so a key is streamed once per launch for all of them; every request's
// arithmetic is the same as when it runs alone.
int run_plan(fe_ctx* c, const fe_evk* evk, const fe_plan* p, const u64* b_in, const u64* b_pt, u64* b_out,
             void* ws, size_t ws_bytes, int mode, cudaStream_t st, int phase, int n_req, int pt_pool,
             void* data_ws, size_t data_ws_bytes) {
    if (mode == 2) {  // the per-operation composition, request by request
        if (!(phase & 2)) return FE_OK;
        if (pt_pool || data_ws) return fail(FE_EINVAL, "mode 2 runs only real plaintexts, uncaptured");
        for (int r = 0; r < n_req; r++)
            FE_TRY(run_plan_per_op(c, evk, p, b_in + (size_t)r * p->n_in * ct_words(c, p->level), b_pt,
                                   b_out + (size_t)r * p->n_out * ct_words(c, p->level - 1), ws, ws_bytes, st));
        return FE_OK;
    }
    if (mode != 0 && mode != 1) return fail(FE_EINVAL, "mode must be 0, 1 or 2");
    const int N = c->N, lv = p->level;
    Sizes z = sizes_of(c, lv);
    if (n_req < 1) return fail(FE_EINVAL, "n_req must be positive");
    const size_t R = (size_t)n_req;
    const size_t ctw_out = ct_words(c, lv - 1);
    const size_t n_in_rot = p->inner.size(), n_mu = p->modup_cts.size(), n_terms = p->terms.size();
    // double hoisting: rotated copies, lifted inputs and plaintexts on Q_l * P
    const bool dh = p->dhoist != 0;
    // double hoisting without outer rotations: every output is its one partial sum
    // on Q_l * P, divided by q_l P in one step (ModDown and rescale together)
    const bool fuse = p->dhoist == 2 && p->n_outer == 0;
    const size_t rw = dh ? z.accw : z.ctw;                         // words of one rotated copy
    const size_t ptb = (size_t)(dh ? lv + 1 + c->k : lv + 1) * pt_limb_bytes(c);  // bytes of one plaintext
    // item tables in ws; data (rotated copies, sums, scratch) after them, or in
    // data_ws when given (graph capture: one data region shared by all layers)
    const size_t chunk = data_ws ? plan_chunk(p, R, mode, data_ws_bytes, true) : plan_chunk(p, R, mode, ws_bytes, false);
    if (data_ws ? (plan_data_bytes(p, chunk, R) > data_ws_bytes || plan_table_bytes(p, chunk, R) > ws_bytes)
                : plan_workspace(p, chunk, R) > ws_bytes)
        return fail(FE_ENOMEM, "workspace too small for the plan");
    std::map<int32_t, const u64*> keys;
    for (int32_t s : p->steps) {
        const u64* k = evk_key(evk, c->galois(s));
        if (!k) return fail(FE_EKEY, "missing rotation key for step " + std::to_string(s));
        keys[s] = k;
    }
    // ---- carve the workspace: item tables first ----
    Carver cv(ws, ws_bytes);
    size_t n_groups_all = 0;
    for (auto& o : p->outs) n_groups_all += o.groups.size();
    // rotated groups of all requests: (request, output, group), sorted by step
    struct OuterRef {
        int r, o, gi;
    };
    // within one step: request-major, so that consecutive groups of one request
    // (same step, other outputs) can share their ciphertext loads in the MAC
    std::vector<OuterRef> order;
    {
        const auto oo = outer_order(p);
        for (size_t a = 0; a < oo.size();) {
            const int32_t st0 = p->outs[oo[a].first].groups[oo[a].second].step;
            size_t b = a;
            while (b < oo.size() && p->outs[oo[b].first].groups[oo[b].second].step == st0) b++;
            for (size_t r = 0; r < R; r++)
                for (size_t k = a; k < b; k++) order.push_back({(int)r, oo[k].first, oo[k].second});
            a = b;
        }
    }
    const size_t n_chunks = order.empty() ? 0 : (order.size() + chunk - 1) / chunk;
    KsItem* d_in_ks = cv.take<KsItem>(std::max<size_t>(1, R * n_in_rot));
    KsGroup* d_in_kg = cv.take<KsGroup>(std::max<size_t>(1, R * n_in_rot));
    CombineItem* d_in_cb = cv.take<CombineItem>(std::max<size_t>(1, R * n_in_rot));
    MacItem* d_mac = cv.take<MacItem>(std::max<size_t>(1, R * n_groups_all));
    MacTerm* d_terms = cv.take<MacTerm>(std::max<size_t>(1, R * n_terms));
    KsItem* d_out_ks = cv.take<KsItem>(std::max<size_t>(1, order.size()));
    KsGroup* d_out_kg = cv.take<KsGroup>(std::max<size_t>(1, order.size()));
    SumEntry* d_ent = cv.take<SumEntry>(std::max<size_t>(1, order.size()));
    SumItem* d_sum = cv.take<SumItem>(std::max<size_t>(1, n_chunks * R * p->n_out));
    LiftItem* d_lift = cv.take<LiftItem>(dh ? std::max<size_t>(1, R * (n_in_rot + p->n_in)) : 1);
    CombineItem* d_dcb = cv.take<CombineItem>(dh ? std::max<size_t>(1, R * n_groups_all) : 1);
    u64** d_fout = cv.take<u64*>(fuse ? std::max<size_t>(1, R * p->n_out) : 1);
    const bool lm = lift_in_mac(p, mode);
    RotItem* d_ritems = cv.take<RotItem>(lm ? std::max<size_t>(1, R * n_groups_all) : 1);
    RotTerm* d_rterms = cv.take<RotTerm>(lm ? std::max<size_t>(1, R * n_terms) : 1);
    if (!cv.ok) return fail(FE_ENOMEM, "workspace too small for the plan");
    Carver cd(data_ws ? (char*)data_ws : cv.p, data_ws ? data_ws_bytes : cv.left);
    u64* Rb = cd.take<u64>(R * n_in_rot * rw);
    u64* total = cd.take<u64>(R * p->n_out * z.ctw);
    u64* XP = dh ? cd.take<u64>(R * p->n_in * z.accw) : nullptr;
    if (!cd.ok) return fail(FE_ENOMEM, "workspace too small for the plan");
    char* scratch = cd.p;
    const size_t scratch_bytes = cd.left;
    Carver s1(scratch, scratch_bytes);  // stage 1
    u64* coef1 = s1.take<u64>(R * n_mu * z.nlN);
    u64* ext1 = s1.take<u64>(R * n_mu * z.extw);
    u64* acc1 = s1.take<u64>(R * n_in_rot * z.accw);
    u64* conv1 = s1.take<u64>(dh ? 0 : R * n_in_rot * z.ctw);
    // stage 2 under double hoisting: the same region, or after stage 1's accumulators
    // when the MAC still reads them
    Carver s2(lm ? s1.p : scratch, lm ? s1.left : scratch_bytes);
    u64* accB = s2.take<u64>(dh ? R * p->n_out * z.accw : 0);
    u64* convB = s2.take<u64>(dh ? R * p->n_out * z.ctw : 0);
    Carver s3(scratch, scratch_bytes);  // stage 3 (same region)
    u64* Pd = s3.take<u64>(chunk * z.ctw);
    u64* coef3 = s3.take<u64>(chunk * z.nlN);
    u64* ext3 = s3.take<u64>(chunk * z.extw);
    u64* acc3 = s3.take<u64>(chunk * z.accw);
    u64* conv3 = s3.take<u64>(chunk * z.ctw);
    u64* csum3 = s3.take<u64>(R * p->n_out * z.ctw);  // per-output sums of the converted parts
    u64* accO = s3.take<u64>(dh ? chunk * z.accw : 0);
    u64* convO = s3.take<u64>(dh ? chunk * z.ctw : 0);
    Carver s4(scratch, scratch_bytes);  // stage 4 (same region)
    u64* rs_tmp = s4.take<u64>(2 * R * p->n_out * N);
    u64* rs_lift = s4.take<u64>(2 * R * p->n_out * lv * N);
    if (!s1.ok || !s2.ok || !s3.ok || !s4.ok) return fail(FE_ENOMEM, "workspace too small for the plan");

    auto src_ptr = [&](size_t r, int src) -> const u64* {
        if (src >= 0) return Rb + (r * n_in_rot + src) * rw;
        const size_t ci = r * p->n_in + (size_t)(-src - 1);
        return dh ? XP + ci * z.accw : b_in + ci * z.ctw;
    };
    // global index of the s-th converted input (request-major) and its source ciphertext
    auto mu_ct = [&](size_t s) -> size_t { return (s / n_mu) * p->n_in + p->modup_cts[s % n_mu]; };

    // ---- host item tables ----
    std::vector<std::pair<int, int>> iorder;  // (request, R slot), sorted by step
    for (size_t r = 0; r < R; r++)
        for (size_t i = 0; i < n_in_rot; i++) iorder.push_back({(int)r, (int)i});
    std::stable_sort(iorder.begin(), iorder.end(), [&](const std::pair<int, int>& x, const std::pair<int, int>& y) {
        return p->inner[x.second].step < p->inner[y.second].step;
    });
    std::vector<KsItem> iks(iorder.size());
    std::vector<KsGroup> ikg;
    std::vector<CombineItem> icb(R * n_in_rot);
    for (size_t q = 0; q < iorder.size(); q++) {
        const size_t r = iorder[q].first, i = iorder[q].second;
        const auto& in = p->inner[i];
        iks[q] = KsItem{ext1 + (r * n_mu + p->modup_slot[in.ci]) * z.extw, keys[in.step], acc1 + (r * n_in_rot + i) * z.accw};
        if (q == 0 || in.step != p->inner[iorder[q - 1].second].step) ikg.push_back(KsGroup{keys[in.step], (int)q, 0});
        ikg.back().n_items++;
    }
    for (size_t r = 0; r < R; r++)
        for (size_t i = 0; i < n_in_rot; i++) {
            const auto& in = p->inner[i];
            const size_t x = r * n_in_rot + i;
            icb[x] = CombineItem{acc1 + x * z.accw, conv1 + x * z.ctw, b_in + (r * p->n_in + in.ci) * z.ctw, nullptr,
                                 Rb + x * rw, c->galois(in.step), 0};
        }
    // double hoisting: rotated copies sigma((P c0, 0) + acc) and lifted inputs (P c0, P c1)
    std::vector<LiftItem> lifts;
    if (dh) {
        for (size_t r = 0; r < R; r++)
            for (size_t i = 0; i < n_in_rot; i++) {
                const size_t x = r * n_in_rot + i;
                lifts.push_back(LiftItem{acc1 + x * z.accw, b_in + (r * p->n_in + p->inner[i].ci) * z.ctw,
                                         Rb + x * rw, c->galois(p->inner[i].step)});
            }
        for (size_t r = 0; r < R; r++)
            for (int ci = 0; ci < p->n_in; ci++)
                lifts.push_back(LiftItem{nullptr, b_in + (r * p->n_in + ci) * z.ctw, XP + (r * p->n_in + ci) * z.accw, 1});
    }
    std::vector<MacTerm> mterms;
    mterms.reserve(R * n_terms);
    for (size_t r = 0; r < R; r++)
        for (const auto& t : p->terms)
            mterms.push_back(MacTerm{src_ptr(r, t.src),
                                     (const uint8_t*)b_pt + (size_t)(pt_pool ? t.pt % pt_pool : t.pt) * ptb});
    struct OneMac {
        u64* out;
        int term0, n_terms;
    };
    std::vector<OneMac> macs;
    std::vector<size_t> no_base;  // request-major output index
    std::vector<CombineItem> dcb;  // double hoisting: ModDown of every MAC output (base, then outer)
    std::vector<u64*> fout;        // fused: output ciphertext of every base MAC
    for (size_t r = 0; r < R; r++)
        for (int o = 0; o < p->n_out; o++) {
            bool base = false;
            for (const auto& g : p->outs[o].groups)
                if (g.step == 0) {
                    u64* dst = total + (r * p->n_out + o) * z.ctw;
                    if (fuse) fout.push_back(b_out + (r * p->n_out + o) * ctw_out);
                    if (dh) {
                        const size_t b = macs.size();
                        dcb.push_back(CombineItem{accB + b * z.accw, convB + b * z.ctw, nullptr, nullptr, dst, 1, 0});
                        dst = accB + b * z.accw;
                    }
                    macs.push_back(OneMac{dst, (int)(r * n_terms) + g.t0, g.nt});
                    base = true;
                }
            if (!base) no_base.push_back(r * p->n_out + o);
        }
    const size_t n_base = macs.size();
    auto group_of = [&](const OuterRef& x) -> const fe_plan::Group& { return p->outs[x.o].groups[x.gi]; };
    for (size_t k = 0; k < order.size(); k++) {
        const auto& g = group_of(order[k]);
        const size_t sl = k % chunk;
        if (dh) {
            dcb.push_back(CombineItem{accO + sl * z.accw, convO + sl * z.ctw, nullptr, nullptr, Pd + sl * z.ctw, 1, 0});
            macs.push_back(OneMac{accO + sl * z.accw, (int)(order[k].r * n_terms) + g.t0, g.nt});
        } else {
            macs.push_back(OneMac{Pd + sl * z.ctw, (int)(order[k].r * n_terms) + g.t0, g.nt});
        }
    }
    // device MAC items: consecutive outputs whose terms read the same ciphertexts
    // in the same order share one item (up to kMacWays), so each ciphertext word
    // is loaded once for all of them
    struct MacRange {
        int first, count, ct_terms, pt_terms, outputs, ways;
        int ct_distinct;  // distinct ciphertexts among the terms (the profiler's byte count)
    };
    const int ways = mode == 0 ? 1 : std::max(1, std::min(kMacWays, p->mac_ways));
    std::vector<MacItem> dmacs;
    auto same_sources = [&](const OneMac& a, const OneMac& b) {
        if (a.n_terms != b.n_terms) return false;
        for (int t = 0; t < a.n_terms; t++)
            if (mterms[a.term0 + t].ct != mterms[b.term0 + t].ct) return false;
        return true;
    };
    auto merge = [&](size_t b, size_t e) {
        MacRange rg{(int)dmacs.size(), 0, 0, 0, 0, 1, 0};
        std::set<const u64*> cts;
        for (size_t i = b; i < e; i++)
            for (int t = 0; t < macs[i].n_terms; t++) cts.insert(mterms[macs[i].term0 + t].ct);
        rg.ct_distinct = (int)cts.size();
        for (size_t i = b; i < e;) {
            MacItem it{};
            it.n_terms = macs[i].n_terms;
            it.n_out = 0;
            size_t j = i;
            while (j < e && it.n_out < ways && (j == i || same_sources(macs[i], macs[j]))) {
                it.out[it.n_out] = macs[j].out;
                it.term0[it.n_out] = macs[j].term0;
                it.n_out++;
                j++;
            }
            dmacs.push_back(it);
            rg.count++;
            rg.ct_terms += it.n_terms;
            rg.pt_terms += it.n_terms * it.n_out;
            rg.outputs += it.n_out;
            rg.ways = std::max(rg.ways, it.n_out);
            i = j;
        }
        return rg;
    };
    const MacRange base_rg = merge(0, n_base);
    // rotated copies formed in the MAC (lift_in_mac): the base items' terms as
    // (accumulator, lifted input, plaintext, automorphism); every item has one output
    std::vector<RotItem> ritems;
    std::vector<RotTerm> rterms;
    int n_acc_terms = 0;
    bool lm_ok = lm;
    for (int i = 0; lm_ok && i < base_rg.count; i++) lm_ok = dmacs[base_rg.first + i].n_out == 1;
    if (lm_ok) {
        rterms.reserve(R * n_terms);
        for (size_t r = 0; r < R; r++)
            for (const auto& t : p->terms) {
                const uint8_t* ptp = (const uint8_t*)b_pt + (size_t)(pt_pool ? t.pt % pt_pool : t.pt) * ptb;
                if (t.src >= 0) {
                    const auto& in = p->inner[t.src];
                    rterms.push_back(RotTerm{acc1 + (r * n_in_rot + t.src) * z.accw,
                                             XP + (r * p->n_in + in.ci) * z.accw, ptp, c->galois(in.step)});
                    n_acc_terms++;
                } else {
                    rterms.push_back(RotTerm{nullptr, XP + (r * p->n_in + (size_t)(-t.src - 1)) * z.accw, ptp, 1});
                }
            }
        for (int i = 0; i < base_rg.count; i++) {
            const MacItem& it = dmacs[base_rg.first + i];
            ritems.push_back(RotItem{it.out[0], it.term0[0], it.n_terms});
        }
    }
    std::vector<MacRange> chunk_rg;
    for (size_t c0 = 0; c0 < order.size(); c0 += chunk)
        chunk_rg.push_back(merge(n_base + c0, n_base + std::min(order.size(), c0 + chunk)));

    std::vector<KsItem> oks(order.size());
    std::vector<KsGroup> okg;
    std::vector<SumEntry> ents;
    std::vector<SumItem> sums;
    std::vector<std::pair<int, int>> kg_range, sum_range;
    for (size_t c0 = 0; c0 < order.size(); c0 += chunk) {
        size_t c1 = std::min(order.size(), c0 + chunk);
        int kg0 = (int)okg.size();
        std::map<size_t, std::vector<int>> by_out;  // request-major output -> items
        for (size_t k = c0; k < c1; k++) {
            const auto& g = group_of(order[k]);
            size_t s = k - c0;
            oks[k] = KsItem{ext3 + s * z.extw, keys[g.step], acc3 + s * z.accw};
            if (k == c0 || g.step != group_of(order[k - 1]).step) okg.push_back(KsGroup{keys[g.step], (int)k, 0});
            okg.back().n_items++;
            by_out[(size_t)order[k].r * p->n_out + order[k].o].push_back((int)k);
        }
        kg_range.push_back({kg0, (int)okg.size() - kg0});
        int s0 = (int)sums.size();
        for (auto& kv : by_out) {
            // batched path: one NTT of the summed converted parts per output (convsum);
            // plain path: each rotation's converted part is transformed and subtracted alone
            const u64* cs = mode == 0 ? nullptr : csum3 + (size_t)(sums.size() - s0) * z.ctw;
            SumItem si{total + kv.first * z.ctw, nullptr, (int)ents.size(), (int)kv.second.size(), 1, cs};
            for (int k : kv.second) {
                size_t s = k - c0;
                const auto& g = group_of(order[k]);
                const uint32_t gal = c->galois(g.step);
                ents.push_back(SumEntry{acc3 + s * z.accw, conv3 + s * z.ctw, Pd + s * z.ctw, gal,
                                        (uint32_t)h_invmod(gal, 2 * (u64)c->N)});
            }
            sums.push_back(si);
        }
        sum_range.push_back({s0, (int)sums.size() - s0});
    }

    if (phase & 1) {
        FE_TRY(upload(iks, d_in_ks, st));
        FE_TRY(upload(ikg, d_in_kg, st));
        FE_TRY(upload(icb, d_in_cb, st));
        FE_TRY(upload(mterms, d_terms, st));
        FE_TRY(upload(dmacs, d_mac, st));
        FE_TRY(upload(oks, d_out_ks, st));
        FE_TRY(upload(okg, d_out_kg, st));
        FE_TRY(upload(ents, d_ent, st));
        FE_TRY(upload(sums, d_sum, st));
        if (dh) {
            FE_TRY(upload(lifts, d_lift, st));
            FE_TRY(upload(dcb, d_dcb, st));
        }
        if (lm_ok) {
            FE_TRY(upload(ritems, d_ritems, st));
            FE_TRY(upload(rterms, d_rterms, st));
        }
        if (fuse) FE_TRY(upload(fout, d_fout, st));
    }
    if (!(phase & 2)) return FE_OK;

    // ---- stage 1: inner rotations (hoisted ModUp per input ciphertext) ----
    const size_t n_mu_all = R * n_mu;
    {
    ProfScope stage(c, PK_STAGE_INNER, st, 0.0);
    if (mode == 0) {
        for (size_t s = 0; s < n_mu_all; s++)
            modup(c, b_in + mu_ct(s) * z.ctw + z.nlN, z.ctw, 1, lv, coef1 + s * z.nlN, ext1 + s * z.extw, st);
        for (size_t q = 0; q < iorder.size(); q++) {
            const size_t x = (size_t)iorder[q].first * n_in_rot + iorder[q].second;
            launch_keyip(c, d_in_ks + q, 1, lv, st);
            if (dh) launch_lift(c, d_lift + x, 1, lv, st);
            else moddown_prepare(c, acc1 + x * z.accw, 1, lv, conv1 + x * z.ctw, st);
        }
        if (dh)
            for (size_t x = 0; x < R * p->n_in; x++) launch_lift(c, d_lift + R * n_in_rot + x, 1, lv, st);
        else
            for (size_t x = 0; x < R * n_in_rot; x++) launch_combine(c, d_in_cb + x, 1, lv, st);
    } else {
        size_t i = 0;
        while (i < n_mu_all) {  // consecutive runs of rotated inputs are converted together
            size_t j = i + 1;
            while (j < n_mu_all && mu_ct(j) == mu_ct(j - 1) + 1) j++;
            modup(c, b_in + mu_ct(i) * z.ctw + z.nlN, z.ctw, (int)(j - i), lv, coef1 + i * z.nlN, ext1 + i * z.extw, st);
            i = j;
        }
        launch_keyip_grouped(c, d_in_kg, d_in_ks, (int)ikg.size(), (int)iorder.size(), lv, st, (int)n_mu_all);
        if (lm_ok) {  // only the lifted inputs: the MAC forms the rotated copies
            launch_lift(c, d_lift + R * n_in_rot, (int)(R * p->n_in), lv, st, 0, (int)(R * p->n_in));
        } else if (dh) {
            launch_lift(c, d_lift, (int)(R * (n_in_rot + p->n_in)), lv, st, (int)(R * n_in_rot),
                        (int)(R * p->n_in));
        } else {
            moddown_prepare(c, acc1, (int)(R * n_in_rot), lv, conv1, st);
            launch_combine(c, d_in_cb, (int)(R * n_in_rot), lv, st);
        }
    }
    }
    c->cnt.rot += R * n_in_rot;
    c->cnt.keyswitch += R * n_in_rot;

    // ---- stage 2: groups without rotation, straight into the totals ----
    {
    ProfScope stage(c, PK_STAGE_BASE, st, 0.0);
    if (fuse)
        for (size_t o : no_base) FE_CUDA_TRY(cudaMemsetAsync(b_out + o * ctw_out, 0, ctw_out * 8, st));
    else
        for (size_t o : no_base) FE_CUDA_TRY(cudaMemsetAsync(total + o * z.ctw, 0, z.ctw * 8, st));
    if (mode == 0 && fuse) {
        for (size_t i = 0; i < n_base; i++) {
            const int nt = macs[i].n_terms;
            launch_mac(c, d_mac + base_rg.first + i, d_terms, 1, nt, nt, 1, 1, lv, st, true);
            moddown_rescale(c, accB + i * z.accw, 1, lv, convB + i * z.ctw, d_fout + i, st);
        }
    } else if (mode == 0 && dh) {
        for (size_t i = 0; i < n_base; i++) {
            const int nt = macs[i].n_terms;
            launch_mac(c, d_mac + base_rg.first + i, d_terms, 1, nt, nt, 1, 1, lv, st, true);
            moddown_prepare(c, accB + i * z.accw, 1, lv, convB + i * z.ctw, st);
            launch_combine(c, d_dcb + i, 1, lv, st);
        }
    } else if (mode == 0) {
        for (size_t i = 0; i < n_base; i++)
            for (int t = 0; t < macs[i].n_terms; t++) {
                const MacTerm& tm = mterms[macs[i].term0 + t];
                launch_pmult_compact(c, tm.ct, tm.pt, macs[i].out, lv, t > 0, st);
            }
    } else {
        if (lm_ok)
            launch_mac_rot(c, d_ritems, d_rterms, base_rg.count, base_rg.ct_terms, n_acc_terms, lv, st);
        else
            launch_mac(c, d_mac + base_rg.first, d_terms, base_rg.count, base_rg.ct_terms, base_rg.pt_terms,
                       base_rg.outputs, base_rg.ways, lv, st, dh, base_rg.ct_distinct);
        if (fuse) {
            moddown_rescale(c, accB, (int)n_base, lv, convB, d_fout, st);
        } else if (dh) {
            moddown_prepare(c, accB, (int)n_base, lv, convB, st);
            launch_combine(c, d_dcb, (int)n_base, lv, st);
        }
    }
    }

    // ---- stage 3: outer rotations in chunks, summed into the totals ----
    {
    ProfScope stage(c, PK_STAGE_OUTER, st, 0.0);
    for (size_t c0 = 0, ch = 0; c0 < order.size(); c0 += chunk, ch++) {
        size_t c1 = std::min(order.size(), c0 + chunk);
        int cn = (int)(c1 - c0);
        if (mode == 0) {
            for (size_t k = c0; k < c1; k++) {
                const OneMac& m = macs[n_base + k];
                size_t s = k - c0;
                if (dh) {
                    launch_mac(c, d_mac + chunk_rg[ch].first + (k - c0), d_terms, 1, m.n_terms, m.n_terms, 1, 1, lv,
                               st, true);
                    moddown_prepare(c, accO + s * z.accw, 1, lv, convO + s * z.ctw, st);
                    launch_combine(c, d_dcb + n_base + k, 1, lv, st);
                } else {
                    for (int t = 0; t < m.n_terms; t++) {
                        const MacTerm& tm = mterms[m.term0 + t];
                        launch_pmult_compact(c, tm.ct, tm.pt, m.out, lv, t > 0, st);
                    }
                }
                modup(c, Pd + s * z.ctw + z.nlN, z.ctw, 1, lv, coef3 + s * z.nlN, ext3 + s * z.extw, st);
                launch_keyip(c, d_out_ks + k, 1, lv, st);
                moddown_prepare(c, acc3 + s * z.accw, 1, lv, conv3 + s * z.ctw, st);
            }
            for (int si = 0; si < sum_range[ch].second; si++)
                launch_combine_sum(c, d_sum + sum_range[ch].first + si, d_ent, 1, sums[sum_range[ch].first + si].n_e, lv, st);
        } else {
            const MacRange& rg = chunk_rg[ch];
            launch_mac(c, d_mac + rg.first, d_terms, rg.count, rg.ct_terms, rg.pt_terms, rg.outputs, rg.ways, lv,
                       st, dh, rg.ct_distinct);
            if (dh) {
                moddown_prepare(c, accO, cn, lv, convO, st);
                launch_combine(c, d_dcb + n_base + c0, cn, lv, st);
            }
            modup(c, Pd + z.nlN, z.ctw, cn, lv, coef3, ext3, st);
            launch_keyip_grouped(c, d_out_kg + kg_range[ch].first, d_out_ks, kg_range[ch].second, cn, lv, st);
            moddown_to_coef(c, acc3, cn, lv, conv3, st);
            const int ns = sum_range[ch].second;
            launch_autosum(c, d_sum + sum_range[ch].first, d_ent, ns, cn, csum3, lv, st);
            ntt_forward(c, LimbSet{csum3, (size_t)z.nlN, lv + 1, 2 * ns, c->d_identity_map}, st);
            launch_combine_sum(c, d_sum + sum_range[ch].first, d_ent, ns, cn, lv, st);
        }
    }
    }
    c->cnt.rot += order.size();
    c->cnt.keyswitch += order.size();
    c->cnt.pmult += R * n_terms;

    // ---- stage 4: rescale (done with the ModDown when fused) ----
    if (!fuse) {
    ProfScope stage(c, PK_STAGE_RESCALE, st, 0.0);
    if (mode == 0) {
        for (size_t o = 0; o < R * p->n_out; o++)
            rescale_batch(c, total + o * z.ctw, 1, lv, b_out + o * ctw_out, rs_tmp, rs_lift, st);
    } else {
        rescale_batch(c, total, (int)(R * p->n_out), lv, b_out, rs_tmp, rs_lift, st);
    }
    }
    FE_CUDA_TRY(cudaGetLastError());
    return FE_OK;
}

}  // namespace fe

using namespace fe;

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------

extern "C" int fe_layout_make(const fe_ctx* c, fe_layout* l) {
    if (!c || !l) return fail(FE_EINVAL, "null argument");
    return layout_fill(c->N, l);
}

extern "C" int fe_fragment_pack(const fe_ctx* c, const fe_layout* lay, const double* x, double* slots,
                                void* stream) {
    if (!c || !lay || !x || !slots) return fail(FE_EINVAL, "null argument");
    FE_ALIGNED(x);
    FE_ALIGNED(slots);
    fe_layout L = *lay;
    FE_TRY(layout_fill(c->N, &L));
    k_pack<<<dim3((c->N / 2 + kB - 1) / kB, L.n_ct), kB, 0, (cudaStream_t)stream>>>(x, slots, L, c->N);
    FE_CUDA_TRY(cudaGetLastError());
    return FE_OK;
}

extern "C" int fe_fragment_unpack(const fe_ctx* c, const fe_layout* lay, const double* slots, double* y,
                                  void* stream) {
    if (!c || !lay || !slots || !y) return fail(FE_EINVAL, "null argument");
    FE_ALIGNED(slots);
    FE_ALIGNED(y);
    fe_layout L = *lay;
    FE_TRY(layout_fill(c->N, &L));
    size_t total = (size_t)L.BS * L.C * L.H * L.W;
    k_unpack<<<(unsigned)((total + kB - 1) / kB), kB, 0, (cudaStream_t)stream>>>(slots, y, L, c->N);
    FE_CUDA_TRY(cudaGetLastError());
    return FE_OK;
}

void fe::finish_plan(fe_plan* p) {
    std::set<int32_t> st;
    for (auto& in : p->inner) st.insert(in.step);
    p->n_outer = 0;
    for (auto& o : p->outs)
        for (auto& g : o.groups)
            if (g.step) {
                st.insert(g.step);
                p->n_outer++;
            }
    p->steps.assign(st.begin(), st.end());
    p->modup_slot.assign(p->n_in, -1);
    std::set<int> mu;
    for (auto& in : p->inner) mu.insert(in.ci);
    p->modup_cts.assign(mu.begin(), mu.end());
    for (size_t i = 0; i < p->modup_cts.size(); i++) p->modup_slot[p->modup_cts[i]] = (int)i;
}

extern "C" int fe_plan_conv(fe_ctx* c, const fe_layout* in_lay, uint32_t Cout, uint32_t K, uint32_t stride,
                            int depthwise, uint32_t in_period, uint32_t level, uint32_t bsgs_n1, fe_layout* out_lay,
                            fe_plan** out) {
    if (!c || !in_lay || !out) return fail(FE_EINVAL, "null argument");
    if (level == 0 || (int)level > c->L) return fail(FE_ELEVEL, "conv needs a level to rescale");
    if (K == 0 || Cout == 0 || (stride != 1 && stride != 2)) return fail(FE_EINVAL, "bad conv shape");
    fe_layout L = *in_lay;
    FE_TRY(layout_fill(c->N, &L));
    if (K > L.H || K > L.W) return fail(FE_EINVAL, "kernel larger than the map");
    if (stride == 2 && L.S % 2) return fail(FE_EINVAL, "stride 2 needs an even fragment size");
    if (depthwise && Cout != L.C) return fail(FE_EINVAL, "depthwise conv keeps the channel count");
    if (in_period && (L.cpc % in_period || L.C > in_period || L.groups != 1))
        return fail(FE_EINVAL, "replicated input needs c_valid | cpc and one group");
    std::unique_ptr<fe_plan> p(new fe_plan());
    p->c = c;
    p->kind = 0;
    p->level = level;
    p->lin = L;
    p->Cin = L.C;
    p->Cout = Cout;
    p->K = K;
    p->stride = stride;
    p->depthwise = depthwise;
    p->in_period = in_period;
    fe_layout O{};
    O.H = (L.H - K) / stride + 1;
    O.W = (L.W - K) / stride + 1;
    O.C = Cout;
    O.BS = L.BS;
    O.S = L.S / stride;
    O.m = L.m;
    FE_TRY(layout_fill(c->N, &O));
    p->lout = O;
    p->n_in = L.n_ct;
    p->n_out = O.n_ct;
    const int S = L.S, m = L.m, BS = L.BS, cpc = L.cpc, blk = m * m * BS;
    const int G_in = in_period ? 1 : L.groups, G_out = O.groups;
    // channel diagonals of every output group
    std::vector<std::vector<int>> diag_of(G_out);
    for (int h = 0; h < G_out; h++) {
        if (depthwise) {
            diag_of[h] = {0};
        } else if (in_period) {
            for (uint32_t d = 0; d < in_period; d++) diag_of[h].push_back(d);
        } else {
            std::set<int> ds;
            for (uint32_t cc = 0; cc < L.C; cc++)
                for (int ol = 0; ol < cpc; ol++)
                    if (h * cpc + ol < (int)Cout) ds.insert((((int)(cc % cpc) - ol) % cpc + cpc) % cpc);
            diag_of[h].assign(ds.begin(), ds.end());
        }
    }
    // baby-step / giant-step split of the diagonals (0: linear outer rotations)
    const int n1 = (bsgs_n1 && !depthwise && !in_period && cpc > 1) ? std::min<int>((int)bsgs_n1, cpc) : 0;
    const int n2 = n1 ? (cpc + n1 - 1) / n1 : 0;
    p->bsgs_n1 = n1;
    std::set<int> babies{0};
    if (n1)
        for (auto& ds : diag_of)
            for (int d : ds) babies.insert(d % n1);
    auto offs = inner_offsets(S, K, stride);
    // rotated copies of the inputs: block offset (a, b) of a tap plus baby step i,
    // all from one hoisted ModUp per input ciphertext
    std::map<std::tuple<int, int, int, int>, int> rslot;  // (ci, a, b, i) -> R slot
    for (int g = 0; g < G_in; g++)
        for (int u = 0; u < S; u++)
            for (int v = 0; v < S; v++) {
                int ci = (g * S + u) * S + v;
                for (int a : offs[u])
                    for (int bb : offs[v])
                        for (int i : babies)
                            if (a || bb || i) {
                                rslot[std::make_tuple(ci, a, bb, i)] = (int)p->inner.size();
                                p->inner.push_back({ci, (a * m + bb) * BS + i * blk});
                            }
            }
    auto spatial_ok = [&](int up, int extent) {
        for (int bi = 0; bi < m; bi++) {
            int hp = bi * S + up;
            if (hp > extent - (int)K) break;
            if (hp % stride == 0) return true;
        }
        return false;
    };
    // structurally nonzero: some channel pair of diagonal d in input group g
    auto channels_meet = [&](int h, int d, int g) {
        for (int cl = 0; cl < cpc; cl++) {
            int cc = in_period ? cl % (int)in_period : g * cpc + cl;
            if (!in_period && cc >= (int)L.C) continue;
            int o = h * cpc + ((cl - d) % cpc + cpc) % cpc;
            if (o >= (int)Cout) continue;
            if (depthwise && o != cc) continue;
            return true;
        }
        return false;
    };
    auto add_terms = [&](fe_plan::Group& grp, int h, int up, int vp, int d, int i_baby) {
        for (int g = 0; g < G_in; g++) {
            if (!channels_meet(h, d, g)) continue;
            for (uint32_t ti = 0; ti < K; ti++)
                for (uint32_t tj = 0; tj < K; tj++) {
                    int u = (up + ti) % S, a = (up + ti) / S;
                    int v = (vp + tj) % S, bb = (vp + tj) / S;
                    int ci = (g * S + u) * S + v;
                    int src = (a || bb || i_baby) ? rslot.at(std::make_tuple(ci, a, bb, i_baby)) : -(ci + 1);
                    p->terms.push_back({src, p->n_pt});
                    p->cpts.push_back({h, up, vp, d, g, (int)ti, (int)tj, i_baby * blk});
                    p->n_pt++;
                    grp.nt++;
                }
        }
    };
    p->outs.resize(p->n_out);
    for (int h = 0; h < G_out; h++) {
        const std::set<int> dset(diag_of[h].begin(), diag_of[h].end());
        for (int up = 0; up < S; up += stride)
            for (int vp = 0; vp < S; vp += stride) {
                int oi = (h * O.S + up / stride) * O.S + vp / stride;
                fe_plan::Out& ou = p->outs[oi];
                if (!(spatial_ok(up, L.H) && spatial_ok(vp, L.W))) continue;
                if (!n1) {
                    for (int d : diag_of[h]) {
                        fe_plan::Group grp{d ? d * blk : 0, (int)p->terms.size(), 0};
                        add_terms(grp, h, up, vp, d, 0);
                        if (grp.nt) ou.groups.push_back(grp);
                    }
                } else {
                    // giant step j collects diagonals j n1 + i with plaintexts rotated by i blk
                    for (int j = 0; j < n2; j++) {
                        fe_plan::Group grp{j ? j * n1 * blk : 0, (int)p->terms.size(), 0};
                        for (int i = 0; i < n1; i++) {
                            const int d = j * n1 + i;
                            if (d < cpc && dset.count(d)) add_terms(grp, h, up, vp, d, i);
                        }
                        if (grp.nt) ou.groups.push_back(grp);
                    }
                }
            }
    }
    finish_plan(p.get());
    if (out_lay) *out_lay = O;
    *out = p.release();
    return FE_OK;
}

namespace fe {
namespace {
// FC planner core: diagonal method with baby-step / giant-step over P positions.
// `sparse` (optional) decides which (t, c, gam, beta) diagonals are nonzero; by
// default every diagonal with a valid (neuron, feature) pair is planned (dense W).
// n1 = 0 takes the default split 2^ceil(log2(P) / 2).
int plan_fc_core(fe_ctx* c, uint32_t n_in_ct, uint32_t P, uint32_t BS, const int32_t* feat, uint32_t F_in,
                 uint32_t F_out, uint32_t level, const std::function<bool(int, int, int, int)>* sparse,
                 int n1_req, std::unique_ptr<fe_plan>& p, const std::vector<int>* rowmap = nullptr);
}  // namespace
}  // namespace fe

extern "C" int fe_plan_fc(fe_ctx* c, uint32_t n_in_ct, uint32_t P, uint32_t BS, const int32_t* feat,
                          uint32_t F_in, uint32_t F_out, uint32_t level, fe_plan** out) {
    if (!c || !feat || !out) return fail(FE_EINVAL, "null argument");
    std::unique_ptr<fe_plan> p;
    FE_TRY(plan_fc_core(c, n_in_ct, P, BS, feat, F_in, F_out, level, nullptr, 0, p));
    *out = p.release();
    return FE_OK;
}

namespace fe {
namespace {
int plan_fc_core(fe_ctx* c, uint32_t n_in_ct, uint32_t P, uint32_t BS, const int32_t* feat, uint32_t F_in,
                 uint32_t F_out, uint32_t level, const std::function<bool(int, int, int, int)>* sparse,
                 int n1_req, std::unique_ptr<fe_plan>& p, const std::vector<int>* rowmap) {
    if (level == 0 || (int)level > c->L) return fail(FE_ELEVEL, "fc needs a level to rescale");
    if ((uint64_t)P * BS != (uint64_t)c->N / 2 || (P & (P - 1)) || !n_in_ct || !F_out)
        return fail(FE_EINVAL, "fc needs P BS = N/2 with P a power of two");
    p.reset(new fe_plan());
    p->c = c;
    p->kind = 1;
    p->level = level;
    p->P = P;
    p->BS = BS;
    p->F_in = F_in;
    p->F_out = F_out;
    for (size_t i = 0; i < (size_t)n_in_ct * P; i++)
        if (feat[i] >= (int)F_in) return fail(FE_EINVAL, "feature index out of range");
    p->feat.assign(feat, feat + (size_t)n_in_ct * P);
    int kbits = 0;
    while ((1u << kbits) < P) kbits++;
    p->n1 = n1_req > 0 ? n1_req : 1 << ((kbits + 1) / 2);
    if (p->n1 > (int)P || (p->n1 & (p->n1 - 1))) return fail(FE_EINVAL, "n1 must be a power of two <= P");
    p->n2 = P / p->n1;
    p->n_in = n_in_ct;
    const int T = (F_out + P - 1) / P;
    p->n_out = T;
    auto present = [&](int t, int cc, int gam, int beta) {
        if (sparse) return (*sparse)(t, cc, gam, beta);
        for (uint32_t q = 0; q < P; q++) {
            int p0 = (((int)q - p->n1 * gam) % (int)P + (int)P) % (int)P;
            int n = t * P + p0;
            int f = p->feat[(size_t)cc * P + (q + beta) % P];
            if (n < (int)F_out && f >= 0 && (!rowmap || (*rowmap)[n] >= 0)) return true;
        }
        return false;
    };
    std::map<std::pair<int, int>, int> rslot;
    for (int cc = 0; cc < (int)n_in_ct; cc++) {
        std::set<int> need;
        for (int t = 0; t < T; t++)
            for (int gam = 0; gam < p->n2; gam++)
                for (int beta = 0; beta < p->n1; beta++)
                    if (present(t, cc, gam, beta)) need.insert(beta);
        for (int beta : need)
            if (beta) {
                rslot[{cc, beta}] = (int)p->inner.size();
                p->inner.push_back({cc, beta * (int32_t)BS});
            }
    }
    p->outs.resize(T);
    for (int t = 0; t < T; t++) {
        for (int gam = 0; gam < p->n2; gam++) {
            fe_plan::Group grp{gam ? p->n1 * gam * (int32_t)BS : 0, (int)p->terms.size(), 0};
            for (int cc = 0; cc < (int)n_in_ct; cc++)
                for (int beta = 0; beta < p->n1; beta++)
                    if (present(t, cc, gam, beta)) {
                        int src = beta ? rslot.at({cc, beta}) : -(cc + 1);
                        p->terms.push_back({src, p->n_pt});
                        p->fpts.push_back({t, cc, gam, beta});
                        p->n_pt++;
                        grp.nt++;
                    }
            if (grp.nt) p->outs[t].groups.push_back(grp);
        }
    }
    finish_plan(p.get());
    return FE_OK;
}

// feature table of a fragment layout: position p of ciphertext ci holds element
// (ch, h, w) = (c H + h) W + w, or -1 (padding)
std::vector<int32_t> layout_features(const fe_layout& L) {
    const uint32_t P = L.cpc * L.m * L.m;
    std::vector<int32_t> feat((size_t)L.n_ct * P, -1);
    for (uint32_t ci = 0; ci < L.n_ct; ci++) {
        const uint32_t g = ci / (L.S * L.S), u = (ci / L.S) % L.S, v = ci % L.S;
        for (uint32_t p = 0; p < P; p++) {
            const uint32_t c_loc = p / (L.m * L.m), k = p % (L.m * L.m);
            const uint32_t ch = g * L.cpc + c_loc, h = (k / L.m) * L.S + u, w = (k % L.m) * L.S + v;
            if (ch < L.C && h < L.H && w < L.W) feat[(size_t)ci * P + p] = (int32_t)((ch * L.H + h) * L.W + w);
        }
    }
    return feat;
}

// (ciphertext, position) of element (ch, h, w) under a fragment layout (Algorithm 1)
inline void layout_position(const fe_layout& L, uint32_t ch, uint32_t h, uint32_t w, uint32_t* ct, uint32_t* pos) {
    const uint32_t g = ch / L.cpc, c_loc = ch % L.cpc;
    *ct = (g * L.S + h % L.S) * L.S + w % L.S;
    *pos = (c_loc * L.m + h / L.S) * L.m + w / L.S;
}
}  // namespace
}  // namespace fe

extern "C" int fe_plan_repack(fe_ctx* c, const fe_layout* from, const fe_layout* to, uint32_t level,
                              fe_plan** out) {
    if (!c || !from || !to || !out) return fail(FE_EINVAL, "null argument");
    if (level == 0 || (int)level > c->L) return fail(FE_ELEVEL, "the repack needs a level to rescale");
    fe_layout A = *from, B = *to;
    FE_TRY(layout_fill(c->N, &A));
    FE_TRY(layout_fill(c->N, &B));
    if (A.C != B.C || A.H != B.H || A.W != B.W || A.BS != B.BS)
        return fail(FE_EINVAL, "both layouts must describe the same (BS, C, H, W) map");
    const uint32_t P = A.cpc * A.m * A.m;
    // every element's source and target (ciphertext, position), and the shift d = source - target
    struct Move {
        uint32_t cs, ct, d;
    };
    std::vector<Move> moves;
    moves.reserve((size_t)A.C * A.H * A.W);
    for (uint32_t ch = 0; ch < A.C; ch++)
        for (uint32_t h = 0; h < A.H; h++)
            for (uint32_t w = 0; w < A.W; w++) {
                uint32_t cs, ps, ct, pt;
                layout_position(A, ch, h, w, &cs, &ps);
                layout_position(B, ch, h, w, &ct, &pt);
                moves.push_back({cs, ct, (ps + P - pt) % P});
            }
    // baby steps n1: the power of two that minimises distinct nonzero baby steps per
    // source plus distinct nonzero giant steps per target (ties to the smaller n1)
    int best_n1 = 1;
    size_t best = SIZE_MAX;
    for (uint32_t n1 = 1; n1 <= P; n1 *= 2) {
        std::set<std::pair<uint32_t, uint32_t>> baby, giant;
        for (const Move& mv : moves) {
            if (mv.d % n1) baby.insert({mv.cs, mv.d % n1});
            if (mv.d / n1) giant.insert({mv.ct, mv.d / n1});
        }
        if (baby.size() + giant.size() < best) {
            best = baby.size() + giant.size();
            best_n1 = (int)n1;
        }
    }
    std::set<std::tuple<int, int, int, int>> nz;
    for (const Move& mv : moves)
        nz.insert({(int)mv.ct, (int)mv.cs, (int)(mv.d / best_n1), (int)(mv.d % best_n1)});
    std::function<bool(int, int, int, int)> sparse = [&](int t, int cc, int gam, int beta) {
        return nz.count({t, cc, gam, beta}) != 0;
    };
    const std::vector<int32_t> feat = layout_features(A);
    std::unique_ptr<fe_plan> p;
    FE_TRY(plan_fc_core(c, A.n_ct, P, A.BS, feat.data(), A.C * A.H * A.W, B.n_ct * P, level, &sparse, best_n1, p));
    p->repack = 1;
    p->lin = A;
    p->lout = B;
    *out = p.release();
    return FE_OK;
}

namespace fe {
namespace {
int token_layout_fill(int N, fe_token_layout* t) {
    if (!t->n_tok || !t->E || !t->S) return fail(FE_EINVAL, "token layout: zero extent");
    if ((N / 2) % t->n_tok) return fail(FE_EINVAL, "token layout: n_tok must divide N / 2");
    t->P = (uint32_t)(N / 2) / t->n_tok;
    t->F = (t->E + t->S - 1) / t->S;
    if (t->F > t->P) return fail(FE_EINVAL, "token layout: E / S positions do not fit a ciphertext");
    t->n_ct = t->S;
    return FE_OK;
}

// slots[s][f n_tok + t] = x[t][f S + s], zero outside the embedding
__global__ void k_token_pack(const double* x, double* slots, fe_token_layout T, int half) {
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= half) return;
    const int s = blockIdx.y;
    const int f = l / (int)T.n_tok, t = l % (int)T.n_tok;
    const int e = f * (int)T.S + s;
    slots[(size_t)s * half + l] = f < (int)T.F && e < (int)T.E ? x[(size_t)t * T.E + e] : 0.0;
}

// the reverse: x[t][f S + s] = slots[s][f n_tok + t]
__global__ void k_token_unpack(const double* slots, double* x, fe_token_layout T, int half) {
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= half) return;
    const int s = blockIdx.y;
    const int f = l / (int)T.n_tok, t = l % (int)T.n_tok;
    const int e = f * (int)T.S + s;
    if (f < (int)T.F && e < (int)T.E) x[(size_t)t * T.E + e] = slots[(size_t)s * half + l];
}
}  // namespace
}  // namespace fe

extern "C" int fe_token_layout_make(const fe_ctx* c, fe_token_layout* t) {
    if (!c || !t) return fail(FE_EINVAL, "null argument");
    return token_layout_fill(c->N, t);
}

extern "C" int fe_token_pack(const fe_ctx* c, const fe_token_layout* lay, const double* x_dev, double* slots_dev,
                             void* stream) {
    if (!c || !lay || !x_dev || !slots_dev) return fail(FE_EINVAL, "null argument");
    FE_ALIGNED(x_dev);
    FE_ALIGNED(slots_dev);
    fe_token_layout T = *lay;
    FE_TRY(token_layout_fill(c->N, &T));
    const int half = c->N / 2;
    k_token_pack<<<dim3((half + kB - 1) / kB, T.n_ct), kB, 0, (cudaStream_t)stream>>>(x_dev, slots_dev, T, half);
    FE_CUDA_TRY(cudaGetLastError());
    return FE_OK;
}

extern "C" int fe_token_unpack(const fe_ctx* c, const fe_token_layout* lay, const double* slots_dev, double* x_dev,
                               void* stream) {
    if (!c || !lay || !x_dev || !slots_dev) return fail(FE_EINVAL, "null argument");
    FE_ALIGNED(x_dev);
    FE_ALIGNED(slots_dev);
    fe_token_layout T = *lay;
    FE_TRY(token_layout_fill(c->N, &T));
    const int half = c->N / 2;
    k_token_unpack<<<dim3((half + kB - 1) / kB, T.n_ct), kB, 0, (cudaStream_t)stream>>>(slots_dev, x_dev, T, half);
    FE_CUDA_TRY(cudaGetLastError());
    return FE_OK;
}

extern "C" int fe_plan_token_linear(fe_ctx* c, const fe_token_layout* in_lay, uint32_t E_out, uint32_t level,
                                    fe_token_layout* out_lay, fe_plan** out) {
    if (!c || !in_lay || !out || !E_out) return fail(FE_EINVAL, "null argument or E_out = 0");
    fe_token_layout A = *in_lay;
    FE_TRY(token_layout_fill(c->N, &A));
    fe_token_layout B{A.n_tok, E_out, A.S, 0, 0, 0};
    FE_TRY(token_layout_fill(c->N, &B));
    const uint32_t P = A.P;
    // input feature of position p of ciphertext s: element p S + s; output neuron
    // s' P + f' carries output element f' S + s' (row f' S + s' of the caller's W)
    std::vector<int32_t> feat((size_t)A.n_ct * P, -1);
    for (uint32_t s2 = 0; s2 < A.n_ct; s2++)
        for (uint32_t p = 0; p < A.F; p++)
            if (p * A.S + s2 < A.E) feat[(size_t)s2 * P + p] = (int32_t)(p * A.S + s2);
    std::vector<int> rowmap((size_t)B.n_ct * P, -1);
    for (uint32_t k = 0; k < E_out; k++) rowmap[(size_t)(k % B.S) * P + k / B.S] = (int)k;
    std::unique_ptr<fe_plan> p;
    FE_TRY(plan_fc_core(c, A.n_ct, P, A.n_tok, feat.data(), A.E, B.n_ct * P, level, nullptr, 0, p, &rowmap));
    p->rowmap = std::move(rowmap);
    p->w_rows = (int)E_out;
    if (out_lay) *out_lay = B;
    *out = p.release();
    return FE_OK;
}

extern "C" int fe_plan_fc_layout(fe_ctx* c, const fe_layout* in_lay, uint32_t F_out, uint32_t level,
                                 fe_plan** out) {
    if (!c || !in_lay || !out) return fail(FE_EINVAL, "null argument");
    fe_layout L = *in_lay;
    FE_TRY(layout_fill(c->N, &L));
    // feature (c, h, w) -> (c H + h) W + w, the row-major flattening of a (C, H, W) map
    const std::vector<int32_t> feat = layout_features(L);
    return fe_plan_fc(c, L.n_ct, L.cpc * L.m * L.m, L.BS, feat.data(), L.C * L.H * L.W, F_out, level, out);
}

extern "C" int fe_plan_fc_next(fe_ctx* c, const fe_plan* prev, uint32_t F_out, uint32_t level, fe_plan** out) {
    if (!c || !prev || !out) return fail(FE_EINVAL, "null argument");
    if (prev->kind != 1) return fail(FE_EINVAL, "fe_plan_fc_next continues a fully connected plan");
    const uint32_t P = (uint32_t)prev->P, n_in = (uint32_t)prev->n_out, F_in = (uint32_t)prev->F_out;
    std::vector<int32_t> feat((size_t)n_in * P);
    for (size_t i = 0; i < feat.size(); i++) feat[i] = i < F_in ? (int32_t)i : -1;
    return fe_plan_fc(c, n_in, P, (uint32_t)prev->BS, feat.data(), F_in, F_out, level, out);
}

namespace fe {
namespace {
// logits y[b][n] = slot (n mod P) BS + b of ciphertext n / P
__global__ void k_fc_unpack(const double* slots, double* y, int P, int BS, int F, int half) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;  // i = b F + n
    if (i >= BS * F) return;
    const int b = i / F, n = i % F;
    y[i] = slots[(size_t)(n / P) * half + (size_t)(n % P) * BS + b];
}
}  // namespace
}  // namespace fe

extern "C" int fe_fc_unpack(const fe_ctx* c, const fe_plan* p, const double* slots_dev, double* y_dev,
                            void* stream) {
    if (!c || !p || !slots_dev || !y_dev) return fail(FE_EINVAL, "null argument");
    FE_ALIGNED(slots_dev);
    FE_ALIGNED(y_dev);
    if (p->kind != 1) return fail(FE_EINVAL, "not a fully connected plan");
    const int total = p->BS * p->F_out;
    k_fc_unpack<<<(total + kB - 1) / kB, kB, 0, (cudaStream_t)stream>>>(slots_dev, y_dev, p->P, p->BS, p->F_out,
                                                                        c->N / 2);
    FE_CUDA_TRY(cudaGetLastError());
    return FE_OK;
}

extern "C" int fe_plan_out_scale(const fe_plan* p, double in_scale, double* out_scale) {
    if (!p || !out_scale) return fail(FE_EINVAL, "null argument");
    if (p->w_scale == 0) return fail(FE_EINVAL, "the plan's weights are not loaded");
    if (!(in_scale > 0)) return fail(FE_EINVAL, "scale must be positive");
    *out_scale = (in_scale * p->w_scale) / (double)p->c->mod[p->level];
    return FE_OK;
}

extern "C" void fe_plan_destroy(fe_plan* p) { delete p; }

// workspace for n_req requests: the whole outer stage in one chunk, unless the
// chunk's scratch would exceed 8 GiB
static size_t default_workspace(const fe_plan* p, size_t n_req) {
    size_t chunk = std::max<size_t>(1, n_req * p->n_outer);
    while (chunk > 1 && plan_workspace(p, chunk, n_req) - plan_workspace(p, 1, n_req) > (8ull << 30))
        chunk = (chunk + 1) / 2;
    return plan_workspace(p, chunk, n_req);
}

extern "C" size_t fe_plan_workspace_bytes(const fe_plan* p, uint32_t n_req, int minimum) {
    if (!p || n_req == 0) return 0;
    return minimum ? plan_workspace(p, 1, n_req) : default_workspace(p, n_req);
}

extern "C" int fe_plan_query(const fe_plan* p, fe_plan_info* info) {
    if (!p || !info) return fail(FE_EINVAL, "null argument");
    const fe_ctx* c = p->c;
    info->pt_bytes = (size_t)p->n_pt * (p->level + 1 + (p->dhoist ? c->k : 0)) * pt_limb_bytes(c);
    info->in_bytes = (size_t)p->n_in * ct_words(c, p->level) * 8;
    info->out_bytes = (size_t)p->n_out * ct_words(c, p->level - 1) * 8;
    // default: the whole outer stage in one chunk, unless its scratch exceeds 8 GiB
    info->workspace_bytes = default_workspace(p, 1);
    info->workspace_min_bytes = plan_workspace(p, 1);
    info->n_in_ct = p->n_in;
    info->n_out_ct = p->n_out;
    info->n_pt = p->n_pt;
    info->n_inner_rot = (uint32_t)p->inner.size();
    info->n_outer_rot = p->n_outer;
    info->bsgs_n1 = (uint32_t)p->bsgs_n1;
    info->double_hoist = (uint32_t)p->dhoist;
    return FE_OK;
}

extern "C" int fe_plan_rotation_steps(const fe_plan* p, int32_t* steps, uint32_t max, uint32_t* n) {
    if (!p || !n) return fail(FE_EINVAL, "null argument");
    *n = (uint32_t)p->steps.size();
    if (steps)
        for (uint32_t i = 0; i < std::min<uint32_t>(max, *n); i++) steps[i] = p->steps[i];
    return FE_OK;
}

extern "C" int fe_plan_load_weights(fe_ctx* c, fe_plan* p, const double* W_host, double wmul, double w_scale,
                                    void* pt_dev, void* stream) {
    FE_ALIGNED(pt_dev);
    if (!c || !p || (!W_host && !p->repack) || !pt_dev) return fail(FE_EINVAL, "null argument");
    if (p->n_pt == 0) {
        p->w_scale = w_scale;
        return FE_OK;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int N = c->N, half = N / 2, nl = p->level + 1 + (p->dhoist ? c->k : 0);
    size_t wcount = p->repack ? 1
                    : p->kind == 0 ? (p->depthwise ? (size_t)p->Cin * p->K * p->K
                                                   : (size_t)p->Cout * p->Cin * p->K * p->K)
                    : !p->rowmap.empty() ? (size_t)p->w_rows * p->F_in
                                         : (size_t)p->F_out * p->F_in;
    double* dW;
    FE_CUDA_TRY(cudaMallocAsync(&dW, wcount * 8, st));
    if (!p->repack) FE_CUDA_TRY(cudaMemcpyAsync(dW, W_host, wcount * 8, cudaMemcpyHostToDevice, st));
    // chunks of plaintexts: slot vectors (<= 64 MiB) and 64-bit limbs (<= 1 GiB)
    // before they are compacted into pt_dev
    const int chunk = std::max(1, std::min({p->n_pt, (int)((64ull << 20) / ((size_t)half * 8)),
                                            (int)((1ull << 30) / ((size_t)nl * N * 8))}));
    double* z;
    u64* limbs;
    void* descs;
    int* dfeat = nullptr;
    int* drow = nullptr;
    FE_CUDA_TRY(cudaMallocAsync(&z, (size_t)chunk * half * 8, st));
    FE_CUDA_TRY(cudaMallocAsync(&limbs, (size_t)chunk * nl * N * 8, st));
    size_t dbytes = p->kind == 0 ? p->cpts.size() * sizeof(fe_plan::ConvPt) : p->fpts.size() * sizeof(fe_plan::FcPt);
    FE_CUDA_TRY(cudaMallocAsync(&descs, std::max<size_t>(dbytes, 16), st));
    if (p->kind == 0) {
        FE_CUDA_TRY(cudaMemcpyAsync(descs, p->cpts.data(), dbytes, cudaMemcpyHostToDevice, st));
    } else {
        FE_CUDA_TRY(cudaMemcpyAsync(descs, p->fpts.data(), dbytes, cudaMemcpyHostToDevice, st));
        FE_CUDA_TRY(cudaMallocAsync(&dfeat, p->feat.size() * sizeof(int), st));
        FE_CUDA_TRY(cudaMemcpyAsync(dfeat, p->feat.data(), p->feat.size() * sizeof(int), cudaMemcpyHostToDevice, st));
        if (!p->rowmap.empty()) {
            FE_CUDA_TRY(cudaMallocAsync(&drow, p->rowmap.size() * sizeof(int), st));
            FE_CUDA_TRY(cudaMemcpyAsync(drow, p->rowmap.data(), p->rowmap.size() * sizeof(int), cudaMemcpyHostToDevice,
                                        st));
        }
    }
    int rc = FE_OK;
    for (int s0 = 0; s0 < p->n_pt && rc == FE_OK; s0 += chunk) {
        int cn = std::min(chunk, p->n_pt - s0);
        if (p->kind == 0) {
            ConvPtArgs a{(const fe_plan::ConvPt*)descs + s0, dW, wmul, (int)p->lin.S, (int)p->lin.m, (int)p->lin.BS,
                         (int)p->lin.cpc, (int)p->lin.H, (int)p->lin.W, p->K, p->stride, p->Cin, p->Cout,
                         p->depthwise, p->in_period};
            k_conv_pt_slots<<<dim3((half + kB - 1) / kB, cn), kB, 0, st>>>(a, z, half);
        } else if (p->repack) {
            RepackPtArgs a{(const fe_plan::FcPt*)descs + s0, dfeat, p->lout, p->P, p->BS, p->n1};
            k_repack_pt_slots<<<dim3((half + kB - 1) / kB, cn), kB, 0, st>>>(a, z, half);
        } else {
            FcPtArgs a{(const fe_plan::FcPt*)descs + s0, dW, dfeat, drow, wmul, p->P, p->BS, p->n1, p->F_in, p->F_out};
            k_fc_pt_slots<<<dim3((half + kB - 1) / kB, cn), kB, 0, st>>>(a, z, half);
        }
        rc = encode_batch(c, z, cn, p->level, w_scale, limbs, st, p->dhoist != 0);
        if (rc == FE_OK)
            launch_pt_compact(c, limbs, (uint8_t*)pt_dev + (size_t)s0 * nl * pt_limb_bytes(c), cn * nl, st);
    }
    cudaFreeAsync(dW, st);
    cudaFreeAsync(z, st);
    cudaFreeAsync(limbs, st);
    cudaFreeAsync(descs, st);
    if (dfeat) cudaFreeAsync(dfeat, st);
    if (drow) cudaFreeAsync(drow, st);
    FE_CUDA_TRY(cudaStreamSynchronize(st));
    if (rc == FE_OK) p->w_scale = w_scale;
    return rc;
}

extern "C" int fe_he_conv(fe_ctx* c, const fe_evk* evk, const fe_plan* p, const void* pt_dev, const void* in_dev,
                          void* out_dev, void* ws, size_t ws_bytes, int mode, void* stream) {
    FE_ALIGNED(pt_dev); FE_ALIGNED(in_dev); FE_ALIGNED(out_dev); FE_ALIGNED(ws);
    if (!c || !evk || !p || !pt_dev || !in_dev || !out_dev || !ws) return fail(FE_EINVAL, "null argument");
    if (p->kind != 0) return fail(FE_EINVAL, "not a conv plan");
    return run_plan(c, evk, p, (const u64*)in_dev, (const u64*)pt_dev, (u64*)out_dev, ws, ws_bytes, mode,
                    (cudaStream_t)stream, 3);
}

extern "C" int fe_he_fc(fe_ctx* c, const fe_evk* evk, const fe_plan* p, const void* pt_dev, const void* in_dev,
                        void* out_dev, void* ws, size_t ws_bytes, int mode, void* stream) {
    FE_ALIGNED(pt_dev); FE_ALIGNED(in_dev); FE_ALIGNED(out_dev); FE_ALIGNED(ws);
    if (!c || !evk || !p || !pt_dev || !in_dev || !out_dev || !ws) return fail(FE_EINVAL, "null argument");
    if (p->kind != 1) return fail(FE_EINVAL, "not an fc plan");
    return run_plan(c, evk, p, (const u64*)in_dev, (const u64*)pt_dev, (u64*)out_dev, ws, ws_bytes, mode,
                    (cudaStream_t)stream, 3);
}

extern "C" int fe_he_repack(fe_ctx* c, const fe_evk* evk, const fe_plan* p, const void* pt_dev, const void* in_dev,
                            void* out_dev, void* ws, size_t ws_bytes, int mode, void* stream) {
    if (p && !p->repack) return fail(FE_EINVAL, "not a repack plan");
    return fe_he_fc(c, evk, p, pt_dev, in_dev, out_dev, ws, ws_bytes, mode, stream);
}

extern "C" int fe_he_layer_batch(fe_ctx* c, const fe_evk* evk, const fe_plan* p, const void* pt_dev, const void* in_dev,
                                 void* out_dev, uint32_t n_req, void* ws, size_t ws_bytes, int mode, void* stream) {
    FE_ALIGNED(pt_dev); FE_ALIGNED(in_dev); FE_ALIGNED(out_dev); FE_ALIGNED(ws);
    if (!c || !evk || !p || !pt_dev || !in_dev || !out_dev || !ws) return fail(FE_EINVAL, "null argument");
    if (n_req == 0) return FE_OK;
    return run_plan(c, evk, p, (const u64*)in_dev, (const u64*)pt_dev, (u64*)out_dev, ws, ws_bytes, mode,
                    (cudaStream_t)stream, 3, (int)n_req);
}

extern "C" int fe_he_layer_timing(fe_ctx* c, const fe_evk* evk, const fe_plan* p, const void* pt_pool_dev,
                                  uint32_t n_pool, const void* in_dev, void* out_dev, void* ws, size_t ws_bytes,
                                  void* stream) {
    FE_ALIGNED(pt_pool_dev); FE_ALIGNED(in_dev); FE_ALIGNED(out_dev); FE_ALIGNED(ws);
    if (!c || !evk || !p || !pt_pool_dev || !in_dev || !out_dev || !ws) return fail(FE_EINVAL, "null argument");
    if (n_pool == 0) return fail(FE_EINVAL, "empty plaintext pool");
    return run_plan(c, evk, p, (const u64*)in_dev, (const u64*)pt_pool_dev, (u64*)out_dev, ws, ws_bytes, 1,
                    (cudaStream_t)stream, 3, 1, (int)n_pool);
}

extern "C" int fe_plan_truncate(fe_plan* p, uint32_t max_out_ct) {
    if (!p) return fail(FE_EINVAL, "null argument");
    if (max_out_ct == 0) return fail(FE_EINVAL, "max_out_ct must be positive");
    if ((int)max_out_ct >= p->n_out) return FE_OK;
    // terms (and plaintexts, one per term) are laid out in output order: the kept
    // outputs' terms are a prefix
    int t_keep = 0;
    for (uint32_t o = 0; o < max_out_ct; o++)
        for (const auto& g : p->outs[o].groups) t_keep = std::max(t_keep, g.t0 + g.nt);
    p->terms.resize(t_keep);
    if (p->kind == 0) p->cpts.resize(t_keep);
    else p->fpts.resize(t_keep);
    p->n_pt = t_keep;
    p->outs.resize(max_out_ct);
    p->n_out = (int)max_out_ct;
    // drop the inner rotations that no kept term reads, renumbering the rest
    std::vector<int> remap(p->inner.size(), -1);
    std::vector<fe_plan::Inner> inner;
    for (auto& t : p->terms)
        if (t.src >= 0) {
            if (remap[t.src] < 0) {
                remap[t.src] = (int)inner.size();
                inner.push_back(p->inner[t.src]);
            }
            t.src = remap[t.src];
        }
    p->inner = inner;
    finish_plan(p);
    return FE_OK;
}

extern "C" int fe_plan_set_mac_ways(fe_plan* p, uint32_t ways) {
    if (!p) return fail(FE_EINVAL, "null argument");
    if (ways != 1 && ways != 2 && ways != 4) return fail(FE_EINVAL, "mac ways must be 1, 2 or 4");
    p->mac_ways = (int)ways;
    return FE_OK;
}

extern "C" int fe_plan_set_lift_fusion(fe_plan* p, int enable) {
    if (!p) return fail(FE_EINVAL, "null argument");
    if (enable != 0 && enable != 1) return fail(FE_EINVAL, "enable must be 0 or 1");
    p->lift_mac = enable;
    return FE_OK;
}

extern "C" int fe_plan_set_hoisting(fe_plan* p, int double_hoist) {
    if (!p) return fail(FE_EINVAL, "null argument");
    if (double_hoist < 0 || double_hoist > 2) return fail(FE_EINVAL, "hoisting must be 0, 1 or 2");
    p->dhoist = double_hoist;
    return FE_OK;
}
