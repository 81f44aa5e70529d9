// Layers around the convolution: x^2 activation (CMult + relinearisation +
// rescale), 2x2 average pooling by fragment sums, Arch-aware Ciphertext
// Compression (rotate-and-add replication), and CUDA-graph capture of a
// sequence of planned layers.
#include <algorithm>
#include <memory>

#include "plan.h"

struct fe_graph {
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    // the captured sequence's external inputs (layer inputs no earlier layer writes)
    // and final outputs (layer outputs no later layer reads), in layer order
    struct Io {
        void* dev;
        size_t bytes;
    };
    std::vector<Io> in, out;
};

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
    const int N = c->N, nl = level + 1;
    Carver cv(ws, ws_bytes);
    KsScratch s;
    carve_ks(cv, c, n, level, &s);
    CombineItem* dcb = cv.take<CombineItem>(n);
    u64* d012 = cv.take<u64>((size_t)n * 3 * nl * N);
    u64* tmp = cv.take<u64>((size_t)n * 2 * nl * N);
    u64* rs = cv.take<u64>(rescale_tmp_words(c, n, level));
    if (!cv.ok) return fail(FE_ENOMEM, "workspace too small");
    std::vector<KsItem> ks(n);
    std::vector<CombineItem> cb(n);
    for (uint32_t i = 0; i < n; i++) {
        ks[i] = KsItem{s.ext + i * ext_words(c, level), evk->relin, s.acc + i * acc_words(c, level)};
        const u64* d = d012 + (size_t)i * 3 * nl * N;
        cb[i] = CombineItem{s.acc + i * acc_words(c, level), s.conv + i * ct_words(c, level), d, d + (size_t)nl * N,
                            tmp + i * ct_words(c, level), 1, 0};
    }
    std::vector<KsGroup> kg{KsGroup{evk->relin, 0, (int)n}};
    FE_TRY(upload(ks, s.ks, st));
    FE_TRY(upload(kg, s.kg, st));
    FE_TRY(upload(cb, dcb, st));
    launch_tensor(c, (const u64*)in_dev, (const u64*)in_dev, d012, n, level, st);
    modup(c, d012 + 2 * (size_t)nl * N, 3 * (size_t)nl * N, n, level, s.coef, s.ext, st);
    launch_keyip_grouped(c, s.kg, s.ks, 1, (int)n, level, st);
    moddown_prepare(c, s.acc, n, level, s.conv, st);
    launch_combine(c, dcb, n, level, st);
    rescale_batch(c, tmp, n, level, (u64*)out_dev, rs, rs + 2 * (size_t)n * N, st);
    c->cnt.cmult += n;
    c->cnt.keyswitch += n;
    FE_CUDA_TRY(cudaGetLastError());
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

extern "C" int fe_compress(fe_ctx* c, const fe_evk* evk, const fe_layout* lay, uint32_t c_valid, const void* in_dev,
                           uint32_t n, uint32_t level, void* out_dev, void* ws, size_t ws_bytes, void* stream) {
    FE_ALIGNED(in_dev); FE_ALIGNED(out_dev); FE_ALIGNED(ws);
    if (!c || !evk || !lay || !in_dev || !out_dev || !ws) return fail(FE_EINVAL, "null argument");
    if ((int)level > c->L) return fail(FE_ELEVEL, "level above L");
    fe_layout L = *lay;
    FE_TRY(layout_fill(c->N, &L));
    if (c_valid == 0 || L.cpc % c_valid) return fail(FE_EINVAL, "c_valid must divide cpc");
    if (ws_bytes < fe_compress_workspace_bytes(c, n, level)) return fail(FE_ENOMEM, "workspace too small");
    cudaStream_t st = (cudaStream_t)stream;
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
        if (!read_later)
            g->out.push_back({outs[j], (size_t)n_req * plans[j]->n_out * 2 * plans[j]->level * c->limb_bytes()});
    }
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

extern "C" int fe_graph_io(const fe_graph* g, uint32_t* n_in, size_t* in_bytes, uint32_t* n_out,
                           size_t* out_bytes) {
    if (!g || !n_in || !n_out) return fail(FE_EINVAL, "null argument");
    if (in_bytes)
        for (size_t i = 0; i < g->in.size(); i++) in_bytes[i] = g->in[i].bytes;
    if (out_bytes)
        for (size_t i = 0; i < g->out.size(); i++) out_bytes[i] = g->out[i].bytes;
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
    for (size_t i = 0; i < g->out.size(); i++)
        FE_CUDA_TRY(cudaMemcpyAsync(out_host[i], g->out[i].dev, g->out[i].bytes, cudaMemcpyDeviceToHost, st));
    return FE_OK;
}

extern "C" void fe_graph_destroy(fe_graph* g) {
    if (!g) return;
    cudaGraphExecDestroy(g->exec);
    cudaGraphDestroy(g->graph);
    delete g;
}
