// Request loop for encrypted inference: continuous batching of requests of
// several models (each bound to its own ring and keys), admission by device
// memory, keys and plaintexts resident, latency percentiles.
//
// A model is a chain of operations (planned conv / FC layers, x^2, 2x2 pooling)
// registered once; its keys and plaintexts stay on the device.  Requests carry
// host input and output buffers.  One scheduler thread:
//   1. retires launch groups whose completion event has fired (results are in
//      the callers' host buffers), releasing their device memory and stream;
//   2. while a stream is free, forms a launch group from the oldest pending
//      request's model: up to max_batch pending requests of that model, shrunk
//      until its device memory (two ping-pong ciphertext buffers and the largest
//      per-layer workspace, all sized for the group) fits the budget next to the
//      groups in flight; a request that does not fit even alone into the whole
//      budget is rejected with FE_ENOMEM;
//   3. enqueues the group on its stream: host-to-device copies, every layer once
//      for the whole group (keys and plaintexts streamed once per layer for all
//      of its requests), device-to-host copies, an event.
// Requests that arrive while groups are running are admitted as soon as a
// stream and memory free up, and their work overlaps with the running groups on
// the device.  Each request's arithmetic does not depend on the group it ran
// in, so its result is the same alone and in any mix.
//
// Waits are bounded: fe_server_wait returns FE_ETIMEOUT after its limit; the
// scheduler never blocks on the device (it polls events).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>

#include "plan.h"

using namespace fe;

namespace {

using Clock = std::chrono::steady_clock;

struct Op {
    fe_op d;
    uint32_t in_ct, out_ct, in_level, out_level;
};

struct Model {
    fe_ctx* c;
    const fe_evk* evk;
    std::vector<Op> ops;
    uint32_t in_ct, in_level, out_ct, out_level;
    size_t in_bytes, out_bytes, max_ct_bytes;  // per request
};

struct Request {
    uint64_t id;
    uint32_t model;
    const void* in_host;
    void* out_host;
    Clock::time_point t_submit, t_done;
    int status = 1;  // 1 pending/running, FE_OK or an error when finished
};

struct Group {
    uint32_t model;
    std::vector<uint64_t> reqs;
    std::vector<const void*> in_host;  // copied from the requests: launch runs without the lock
    std::vector<void*> out_host;
    cudaStream_t stream;
    cudaEvent_t start = nullptr, done = nullptr;  // timing events: the group's interval on the device
    void* mem;
    size_t bytes;
};

}  // namespace

struct fe_server {
    fe_server_config cfg;
    size_t budget = 0;
    std::deque<Model> models;  // stable references: launches read models without the lock
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<uint64_t> pending;
    std::map<uint64_t, Request> reqs;
    std::vector<Group> inflight;
    std::vector<cudaStream_t> free_streams;
    std::vector<cudaStream_t> all_streams;
    uint64_t next_id = 1;
    size_t in_use = 0, peak_use = 0;
    uint64_t submitted = 0, completed = 0, rejected = 0, groups = 0, max_group = 0, max_inflight_seen = 0;
    std::vector<double> lat_ms;
    // device intervals (ms after `epoch`) of finished groups: from the moment the
    // group's stream starts its work (input copies) to its completion
    std::vector<std::pair<float, float>> intervals;
    cudaEvent_t epoch = nullptr;
    Clock::time_point t0;
    bool stop = false;
    bool paused = false;
    int device = 0;
    std::thread worker;

    size_t group_bytes(const Model& m, uint32_t R) const;
    int launch(Group& g, const Model& m);
    void loop();
};

namespace {

size_t round256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

size_t fe_server::group_bytes(const Model& m, uint32_t R) const {
    size_t ws = 0;
    for (const Op& op : m.ops) {
        size_t w = 0;
        if (op.d.kind == FE_OP_LAYER) w = fe_plan_workspace_bytes(op.d.plan, R, 0);
        else if (op.d.kind == FE_OP_SQUARE) w = fe_square_workspace_bytes(m.c, R * op.in_ct, op.in_level);
        else if (op.d.kind == FE_OP_POLY_ACT) w = fe_poly_act_workspace_bytes(m.c, R * op.in_ct, op.in_level);
        else if (op.d.kind == FE_OP_REFRESH)  // level-0 inputs of the refresh, then its scratch
            w = round256((size_t)R * op.in_ct * ct_words(m.c, 0) * 8) +
                std::max(fe_boot_prepare_workspace_bytes(m.c, R * op.in_ct),
                         fe_boot_workspace_bytes(op.d.boot, R * op.in_ct));
        ws = std::max(ws, w);
    }
    return 2 * round256(R * m.max_ct_bytes) + round256(ws);
}

int fe_server::launch(Group& g, const Model& m) {
    const uint32_t R = (uint32_t)g.reqs.size();
    char* base = (char*)g.mem;
    const size_t buf = round256(R * m.max_ct_bytes);
    char* bufs[2] = {base, base + buf};
    char* ws = base + 2 * buf;
    const size_t ws_bytes = g.bytes - 2 * buf;
    cudaStream_t st = g.stream;
    FE_CUDA_TRY(cudaEventRecord(g.start, st));
    for (uint32_t r = 0; r < R; r++)
        FE_CUDA_TRY(cudaMemcpyAsync(bufs[0] + r * m.in_bytes, g.in_host[r], m.in_bytes, cudaMemcpyHostToDevice, st));
    int cur = 0;
    for (const Op& op : m.ops) {
        void* in = bufs[cur];
        void* out = bufs[1 - cur];
        if (op.d.kind == FE_OP_LAYER) {
            FE_TRY(fe_he_layer_batch(m.c, m.evk, op.d.plan, op.d.pt_dev, in, out, R, ws, ws_bytes, 1, st));
        } else if (op.d.kind == FE_OP_SQUARE) {
            FE_TRY(fe_he_square(m.c, m.evk, in, R * op.in_ct, op.in_level, out, ws, ws_bytes, st));
        } else if (op.d.kind == FE_OP_POLY_ACT) {
            double out_scale;
            FE_TRY(fe_he_poly_act(m.c, m.evk, op.d.a, op.d.b, op.d.c, in, R * op.in_ct, op.in_level, op.d.in_scale,
                                  out, &out_scale, ws, ws_bytes, st));
        } else if (op.d.kind == FE_OP_REFRESH) {
            const uint32_t n = R * op.in_ct;
            const size_t lv0_bytes = round256((size_t)n * ct_words(m.c, 0) * 8);
            FE_TRY(fe_boot_prepare(m.c, op.d.boot, in, n, op.in_level, op.d.in_scale, ws, ws + lv0_bytes,
                                   ws_bytes - lv0_bytes, st));
            FE_TRY(fe_he_bootstrap(m.c, m.evk, op.d.boot, ws, n, out, ws + lv0_bytes, ws_bytes - lv0_bytes, st));
        } else {
            // pooling sums the fragments of one request: one launch per request
            const size_t in_b = (size_t)op.in_ct * ct_words(m.c, op.in_level) * 8;
            const size_t out_b = (size_t)op.out_ct * ct_words(m.c, op.out_level) * 8;
            for (uint32_t r = 0; r < R; r++)
                FE_TRY(fe_he_avgpool(m.c, &op.d.layout, (char*)in + r * in_b, op.in_level, (char*)out + r * out_b,
                                     nullptr, st));
        }
        cur = 1 - cur;
    }
    for (uint32_t r = 0; r < R; r++)
        FE_CUDA_TRY(cudaMemcpyAsync(g.out_host[r], bufs[cur] + r * m.out_bytes, m.out_bytes, cudaMemcpyDeviceToHost, st));
    FE_CUDA_TRY(cudaEventRecord(g.done, st));
    return FE_OK;
}

void fe_server::loop() {
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lk(mu);
    while (!stop) {
        // 1. retire finished groups
        for (size_t i = 0; i < inflight.size();) {
            Group& g = inflight[i];
            cudaError_t e = cudaEventQuery(g.done);
            if (e == cudaErrorNotReady) {
                i++;
                continue;
            }
            const auto now = Clock::now();
            for (uint64_t id : g.reqs) {
                Request& q = reqs.at(id);
                q.status = e == cudaSuccess ? FE_OK : FE_ECUDA;
                q.t_done = now;
                if (q.status == FE_OK) {
                    completed++;
                    lat_ms.push_back(std::chrono::duration<double, std::milli>(now - q.t_submit).count());
                }
            }
            float t_s = 0, t_e = 0;
            if (e == cudaSuccess && cudaEventElapsedTime(&t_s, epoch, g.start) == cudaSuccess &&
                cudaEventElapsedTime(&t_e, epoch, g.done) == cudaSuccess) {
                intervals.push_back({t_s, t_e});
                // peak concurrency: the most intervals that hold one instant.  A
                // largest set of pairwise-overlapping intervals all hold the latest
                // start among them, so the starts that fall inside this interval
                // (its own included) are the only instants to count; the set is
                // found when its last member retires.
                auto held = [&](float p) {
                    uint64_t k = 0;
                    for (const auto& iv : intervals) k += iv.first <= p && p < iv.second;
                    return k;
                };
                uint64_t over = std::max<uint64_t>(1, held(t_s));
                for (const auto& iv : intervals)
                    if (iv.first > t_s && iv.first < t_e) over = std::max(over, held(iv.first));
                max_inflight_seen = std::max(max_inflight_seen, over);
                if (intervals.size() > 4096) intervals.erase(intervals.begin(), intervals.begin() + 2048);
            }
            cudaFreeAsync(g.mem, g.stream);
            cudaEventDestroy(g.start);
            cudaEventDestroy(g.done);
            in_use -= g.bytes;
            free_streams.push_back(g.stream);
            inflight.erase(inflight.begin() + i);
            cv_done.notify_all();
        }
        // 2. admit new groups while a stream is free
        while (!paused && !pending.empty() && !free_streams.empty()) {
            const uint32_t mid = reqs.at(pending.front()).model;
            const Model& m = models[mid];
            std::vector<uint64_t> pick;
            for (uint64_t id : pending)
                if (reqs.at(id).model == mid && pick.size() < cfg.max_batch) pick.push_back(id);
            uint32_t R = (uint32_t)pick.size();
            while (R > 0 && in_use + group_bytes(m, R) > budget) R--;
            if (R == 0) {
                if (group_bytes(m, 1) > budget) {  // can never fit: reject
                    Request& q = reqs.at(pick[0]);
                    q.status = FE_ENOMEM;
                    q.t_done = Clock::now();
                    rejected++;
                    pending.erase(std::find(pending.begin(), pending.end(), pick[0]));
                    cv_done.notify_all();
                    continue;
                }
                break;  // wait for memory
            }
            pick.resize(R);
            Group g;
            g.model = mid;
            g.reqs = pick;
            for (uint64_t id : pick) {
                g.in_host.push_back(reqs.at(id).in_host);
                g.out_host.push_back(reqs.at(id).out_host);
                pending.erase(std::find(pending.begin(), pending.end(), id));
            }
            g.stream = free_streams.back();
            free_streams.pop_back();
            g.bytes = group_bytes(m, R);
            in_use += g.bytes;  // reserved before the lock is released
            g.mem = nullptr;
            // enqueueing a group takes host time (item tables of every layer):
            // submissions proceed meanwhile
            lk.unlock();
            int rc = FE_OK;
            if (cudaMallocAsync(&g.mem, g.bytes, g.stream) != cudaSuccess) rc = FE_ENOMEM;
            if (rc == FE_OK && (cudaEventCreate(&g.start) != cudaSuccess || cudaEventCreate(&g.done) != cudaSuccess))
                rc = FE_ECUDA;
            if (rc == FE_OK) rc = launch(g, models[mid]);
            lk.lock();
            if (rc != FE_OK) {
                in_use -= g.bytes;
                free_streams.push_back(g.stream);
                for (uint64_t id : pick) {
                    reqs.at(id).status = rc;
                    reqs.at(id).t_done = Clock::now();
                    rejected++;
                }
                if (g.mem) cudaFreeAsync(g.mem, g.stream);
                if (g.start) cudaEventDestroy(g.start);
                if (g.done) cudaEventDestroy(g.done);
                cv_done.notify_all();
                continue;
            }
            peak_use = std::max(peak_use, in_use);
            groups++;
            max_group = std::max<uint64_t>(max_group, R);
            inflight.push_back(g);
        }
        cv_work.wait_for(lk, std::chrono::microseconds(inflight.empty() ? 2000 : 100));
    }
}

extern "C" int fe_server_create(const fe_server_config* cfg, fe_server** out) {
    if (!cfg || !out) return fail(FE_EINVAL, "null argument");
    if (cfg->max_batch == 0 || cfg->max_inflight == 0 || cfg->max_inflight > 64)
        return fail(FE_EINVAL, "max_batch must be positive and max_inflight in [1, 64]");
    std::unique_ptr<fe_server> s(new fe_server());
    s->cfg = *cfg;
    FE_CUDA_TRY(cudaGetDevice(&s->device));
    if (cfg->hbm_budget_bytes) {
        s->budget = cfg->hbm_budget_bytes;
    } else {
        size_t fr = 0, tot = 0;
        FE_CUDA_TRY(cudaMemGetInfo(&fr, &tot));
        s->budget = fr > cfg->hbm_reserve_bytes ? fr - cfg->hbm_reserve_bytes : 0;
    }
    for (uint32_t i = 0; i < cfg->max_inflight; i++) {
        cudaStream_t st;
        FE_CUDA_TRY(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
        s->all_streams.push_back(st);
        s->free_streams.push_back(st);
    }
    FE_CUDA_TRY(cudaEventCreate(&s->epoch));
    FE_CUDA_TRY(cudaEventRecord(s->epoch, s->all_streams[0]));
    FE_CUDA_TRY(cudaEventSynchronize(s->epoch));
    s->t0 = Clock::now();
    fe_server* raw = s.get();
    s->worker = std::thread([raw] { raw->loop(); });
    *out = s.release();
    return FE_OK;
}

extern "C" int fe_server_add_model(fe_server* s, fe_ctx* c, const fe_evk* evk, const fe_op* ops, uint32_t n_ops,
                                   uint32_t in_ct, uint32_t in_level, uint32_t* model_id) {
    if (!s || !c || !evk || !ops || !n_ops || !in_ct || !model_id) return fail(FE_EINVAL, "null argument");
    Model m;
    m.c = c;
    m.evk = evk;
    m.in_ct = in_ct;
    m.in_level = in_level;
    uint32_t n = in_ct, lv = in_level;
    m.max_ct_bytes = (size_t)n * ct_words(c, lv) * 8;
    for (uint32_t i = 0; i < n_ops; i++) {
        Op op;
        op.d = ops[i];
        op.in_ct = n;
        op.in_level = lv;
        if (op.d.kind == FE_OP_LAYER) {
            fe_plan_info info;
            if (!op.d.plan || !op.d.pt_dev) return fail(FE_EINVAL, "layer op without plan or plaintexts");
            FE_TRY(fe_plan_query(op.d.plan, &info));
            if ((uint32_t)op.d.plan->level != lv || info.n_in_ct != n)
                return fail(FE_EINVAL, "op " + std::to_string(i) + ": plan level / input count do not chain");
            n = info.n_out_ct;
            lv -= 1;
        } else if (op.d.kind == FE_OP_SQUARE) {
            if (lv == 0) return fail(FE_ELEVEL, "x^2 at level 0");
            if (!evk->relin) return fail(FE_EKEY, "x^2 needs a relinearisation key");
            lv -= 1;
        } else if (op.d.kind == FE_OP_POOL) {
            fe_layout L = op.d.layout;
            FE_TRY(layout_fill(c->N, &L));
            if (L.n_ct != n || L.S % 2) return fail(FE_EINVAL, "pool layout does not chain or has odd S");
            n = L.n_ct / 4;
        } else if (op.d.kind == FE_OP_POLY_ACT) {
            if (lv == 0) return fail(FE_ELEVEL, "activation at level 0");
            if (op.d.a != 0 && !evk->relin) return fail(FE_EKEY, "the activation needs a relinearisation key");
            if (!(op.d.in_scale > 0)) return fail(FE_EINVAL, "activation op without a positive in_scale");
            lv -= 1;
        } else if (op.d.kind == FE_OP_REFRESH) {
            if (!op.d.boot) return fail(FE_EINVAL, "refresh op without a refresh");
            if (lv == 0) return fail(FE_ELEVEL, "a refresh input needs level >= 1 (fe_boot_prepare)");
            if (!evk->relin) return fail(FE_EKEY, "the refresh needs a relinearisation key");
            if (!(op.d.in_scale > 0)) return fail(FE_EINVAL, "refresh op without a positive in_scale");
            uint32_t out_level = 0;
            FE_TRY(fe_boot_output(op.d.boot, &out_level, nullptr));
            lv = out_level;
        } else {
            return fail(FE_EINVAL, "unknown op kind");
        }
        op.out_ct = n;
        op.out_level = lv;
        m.max_ct_bytes = std::max(m.max_ct_bytes, (size_t)n * ct_words(c, lv) * 8);
        m.ops.push_back(op);
    }
    m.out_ct = n;
    m.out_level = lv;
    m.in_bytes = (size_t)in_ct * ct_words(c, in_level) * 8;
    m.out_bytes = (size_t)n * ct_words(c, lv) * 8;
    std::lock_guard<std::mutex> lk(s->mu);
    *model_id = (uint32_t)s->models.size();
    s->models.push_back(m);
    return FE_OK;
}

extern "C" int fe_server_model_io(fe_server* s, uint32_t model, uint32_t* out_ct, uint32_t* out_level,
                                  size_t* in_bytes, size_t* out_bytes) {
    if (!s) return fail(FE_EINVAL, "null argument");
    std::lock_guard<std::mutex> lk(s->mu);
    if (model >= s->models.size()) return fail(FE_EINVAL, "unknown model");
    const Model& m = s->models[model];
    if (out_ct) *out_ct = m.out_ct;
    if (out_level) *out_level = m.out_level;
    if (in_bytes) *in_bytes = m.in_bytes;
    if (out_bytes) *out_bytes = m.out_bytes;
    return FE_OK;
}

extern "C" int fe_server_pause(fe_server* s, int paused) {
    if (!s) return fail(FE_EINVAL, "null argument");
    std::lock_guard<std::mutex> lk(s->mu);
    s->paused = paused != 0;
    s->cv_work.notify_one();
    return FE_OK;
}

extern "C" int fe_server_submit(fe_server* s, uint32_t model, const void* in_host, void* out_host, uint64_t* req_id) {
    if (!s || !in_host || !out_host || !req_id) return fail(FE_EINVAL, "null argument");
    std::lock_guard<std::mutex> lk(s->mu);
    if (model >= s->models.size()) return fail(FE_EINVAL, "unknown model");
    Request q;
    q.id = s->next_id++;
    q.model = model;
    q.in_host = in_host;
    q.out_host = out_host;
    q.t_submit = Clock::now();
    s->reqs[q.id] = q;
    s->pending.push_back(q.id);
    s->submitted++;
    *req_id = q.id;
    s->cv_work.notify_one();
    return FE_OK;
}

extern "C" int fe_server_wait(fe_server* s, uint64_t req_id, uint32_t timeout_ms, int* status, double* latency_ms) {
    if (!s) return fail(FE_EINVAL, "null argument");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(req_id);
    if (it == s->reqs.end()) return fail(FE_EINVAL, "unknown request");
    const bool ok = s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms),
                                        [&] { return s->reqs.at(req_id).status != 1; });
    if (!ok) return fail(FE_ETIMEOUT, "request " + std::to_string(req_id) + " not finished within the limit");
    const Request& q = s->reqs.at(req_id);
    if (status) *status = q.status;
    if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(q.t_done - q.t_submit).count();
    return FE_OK;
}

extern "C" int fe_server_stats(fe_server* s, fe_server_stats_t* out) {
    if (!s || !out) return fail(FE_EINVAL, "null argument");
    std::lock_guard<std::mutex> lk(s->mu);
    out->submitted = s->submitted;
    out->completed = s->completed;
    out->rejected = s->rejected;
    out->groups = s->groups;
    out->max_group = s->max_group;
    out->max_inflight = s->max_inflight_seen;
    out->peak_bytes = s->peak_use;
    out->budget_bytes = s->budget;
    out->wall_s = std::chrono::duration<double>(Clock::now() - s->t0).count();
    std::vector<double> v = s->lat_ms;
    std::sort(v.begin(), v.end());
    auto pct = [&](double p) -> double {
        if (v.empty()) return 0.0;
        size_t i = (size_t)std::ceil(p * v.size()) - 1;  // nearest-rank percentile
        return v[std::min(i, v.size() - 1)];
    };
    out->p50_ms = pct(0.50);
    out->p99_ms = pct(0.99);
    double sum = 0;
    for (double x : v) sum += x;
    out->mean_ms = v.empty() ? 0.0 : sum / v.size();
    return FE_OK;
}

extern "C" void fe_server_destroy(fe_server* s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        s->cv_work.notify_all();
    }
    if (s->worker.joinable()) s->worker.join();
    for (auto& g : s->inflight) {
        cudaEventSynchronize(g.done);
        cudaFreeAsync(g.mem, g.stream);
        cudaEventDestroy(g.start);
        cudaEventDestroy(g.done);
    }
    if (s->epoch) cudaEventDestroy(s->epoch);
    for (cudaStream_t st : s->all_streams) {
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
    }
    delete s;
}
