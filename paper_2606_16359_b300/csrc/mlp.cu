// Small fully connected latency model (fp32): in_dim -> hidden x n_hidden
// (ReLU) -> 1, trained with full-batch Adam on mean squared error, used to
// predict per-layer latency from layer features.  Features and targets are
// standardised with the training set's column means and standard deviations
// (kept for prediction).  One training step (forward, loss gradient, backward,
// Adam) is captured once as a CUDA graph and replayed; Adam's step counter
// lives on the device so that replays advance it.
//
// Every reduction runs in a fixed order (one thread per output element looping
// over its inputs), so training is deterministic for a given initialisation.
#include <cmath>
#include <memory>

#include "common.h"

struct fe_mlp {
    std::vector<int> dims;  // [in, h, ..., h, 1]
    std::vector<size_t> w_off, b_off;
    size_t n_params = 0;
    float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
    float *x_mean = nullptr, *x_std = nullptr, *y_stat = nullptr;  // y_stat: mean, std
    int* t = nullptr;
    bool trained = false;
};

namespace {

constexpr int kT = 256;

__global__ void k_col_stats(const float* X, int n, int d, float* mean, float* stdv) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= d) return;
    double s = 0, s2 = 0;
    for (int i = 0; i < n; i++) {
        const double x = X[(size_t)i * d + j];
        s += x;
        s2 += x * x;
    }
    const double mu = s / n;
    const double var = fmax(s2 / n - mu * mu, 0.0);
    mean[j] = (float)mu;
    stdv[j] = var > 1e-12 ? (float)sqrt(var) : 1.0f;
}

__global__ void k_standardise(const float* X, int n, int d, const float* mean, const float* stdv, float* out) {
    const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= (size_t)n * d) return;
    const int j = k % d;
    out[k] = (X[k] - mean[j]) / stdv[j];
}

// Y[i][o] = b[o] + sum_j X[i][j] W[o][j], ReLU unless `linear`
__global__ void k_dense_fwd(const float* X, const float* W, const float* b, float* Y, int n, int din, int dout,
                            int linear) {
    const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= (size_t)n * dout) return;
    const int i = k / dout, o = k % dout;
    float acc = b[o];
    const float* x = X + (size_t)i * din;
    const float* w = W + (size_t)o * din;
    for (int j = 0; j < din; j++) acc = fmaf(x[j], w[j], acc);
    Y[k] = linear ? acc : fmaxf(acc, 0.0f);
}

// dP[i] = 2 (P[i] - y[i]) / n
__global__ void k_mse_grad(const float* P, const float* y, float* dP, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    dP[i] = 2.0f * (P[i] - y[i]) / n;
}

__global__ void k_mse(const float* P, const float* y, int n, float* loss) {
    if (blockIdx.x || threadIdx.x) return;
    double s = 0;
    for (int i = 0; i < n; i++) {
        const double e = (double)P[i] - y[i];
        s += e * e;
    }
    *loss = (float)(s / n);
}

// dX[i][j] = (A[i][j] > 0) * sum_o dY[i][o] W[o][j]   (A: the ReLU output that fed the layer)
__global__ void k_dense_bwd_data(const float* dY, const float* W, const float* A, float* dX, int n, int din,
                                 int dout) {
    const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= (size_t)n * din) return;
    const int i = k / din, j = k % din;
    float acc = 0.0f;
    for (int o = 0; o < dout; o++) acc = fmaf(dY[(size_t)i * dout + o], W[(size_t)o * din + j], acc);
    dX[k] = A[k] > 0.0f ? acc : 0.0f;
}

// dW[o][j] = sum_i dY[i][o] X[i][j]; db[o] = sum_i dY[i][o]  (thread per (o, j), j = din for the bias)
__global__ void k_dense_bwd_w(const float* X, const float* dY, float* dW, float* db, int n, int din, int dout) {
    const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= (size_t)dout * (din + 1)) return;
    const int o = k / (din + 1), j = k % (din + 1);
    float acc = 0.0f;
    if (j < din)
        for (int i = 0; i < n; i++) acc = fmaf(dY[(size_t)i * dout + o], X[(size_t)i * din + j], acc);
    else
        for (int i = 0; i < n; i++) acc += dY[(size_t)i * dout + o];
    if (j < din) dW[(size_t)o * din + j] = acc;
    else db[o] = acc;
}

// Adam (Kingma & Ba) with decoupled weight decay; the step counter is read and
// advanced on the device (thread 0 of block 0 after everyone read it: the
// counter is advanced by a separate single-thread kernel)
__global__ void k_adam(float* p, const float* g, float* m, float* v, size_t count, const int* t, float lr, float b1,
                       float b2, float eps, float wd) {
    const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= count) return;
    const int step = *t + 1;
    const float gk = g[k];
    const float mk = b1 * m[k] + (1.0f - b1) * gk;
    const float vk = b2 * v[k] + (1.0f - b2) * gk * gk;
    m[k] = mk;
    v[k] = vk;
    const float mh = mk / (1.0f - powf(b1, (float)step));
    const float vh = vk / (1.0f - powf(b2, (float)step));
    p[k] -= lr * (mh / (sqrtf(vh) + eps) + wd * p[k]);
}

__global__ void k_step_inc(int* t) {
    if (blockIdx.x == 0 && threadIdx.x == 0) *t += 1;
}

unsigned blocks_for(size_t n) { return (unsigned)((n + kT - 1) / kT); }

uint64_t splitmix(uint64_t& s) {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

struct Acts {
    std::vector<float*> a;  // a[0] = standardised input, a[l+1] = output of layer l
    float *y = nullptr, *dp = nullptr, *loss = nullptr;
    std::vector<float*> d;  // gradients w.r.t. a[l+1]
    char* base = nullptr;
};

int carve_acts(const fe_mlp* m, int n, cudaStream_t st, Acts* A) {
    const int L = (int)m->dims.size() - 1;
    size_t words = 0;
    for (int l = 0; l <= L; l++) words += (size_t)n * m->dims[l] * 2;
    words += 3 * (size_t)n + 64;
    FE_CUDA_TRY(cudaMallocAsync(&A->base, words * sizeof(float), st));
    float* p = (float*)A->base;
    A->a.resize(L + 1);
    A->d.resize(L + 1);
    for (int l = 0; l <= L; l++) {
        A->a[l] = p;
        p += (size_t)n * m->dims[l];
        A->d[l] = p;
        p += (size_t)n * m->dims[l];
    }
    A->y = p;
    p += n;
    A->dp = p;
    p += n;
    A->loss = p;
    return FE_OK;
}

void forward(const fe_mlp* m, Acts& A, int n, cudaStream_t st) {
    const int L = (int)m->dims.size() - 1;
    for (int l = 0; l < L; l++) {
        const int din = m->dims[l], dout = m->dims[l + 1];
        k_dense_fwd<<<blocks_for((size_t)n * dout), kT, 0, st>>>(A.a[l], m->p + m->w_off[l], m->p + m->b_off[l],
                                                                   A.a[l + 1], n, din, dout, l == L - 1);
    }
}

}  // namespace

using namespace fe;

extern "C" int fe_mlp_create(uint32_t in_dim, uint32_t hidden, uint32_t n_hidden, uint64_t seed, fe_mlp** out) {
    if (!out || in_dim == 0 || in_dim > 1024 || hidden == 0 || hidden > 1024 || n_hidden == 0 || n_hidden > 16)
        return fail(FE_EINVAL, "fe_mlp_create: in_dim, hidden in [1, 1024], n_hidden in [1, 16]");
    std::unique_ptr<fe_mlp> m(new fe_mlp());
    m->dims.push_back((int)in_dim);
    for (uint32_t i = 0; i < n_hidden; i++) m->dims.push_back((int)hidden);
    m->dims.push_back(1);
    for (size_t l = 0; l + 1 < m->dims.size(); l++) {
        m->w_off.push_back(m->n_params);
        m->n_params += (size_t)m->dims[l] * m->dims[l + 1];
        m->b_off.push_back(m->n_params);
        m->n_params += m->dims[l + 1];
    }
    // He-uniform weights from SplitMix64(seed), zero biases
    std::vector<float> h(m->n_params, 0.0f);
    uint64_t s = seed;
    for (size_t l = 0; l + 1 < m->dims.size(); l++) {
        const float lim = std::sqrt(6.0f / m->dims[l]);
        for (size_t k = 0; k < (size_t)m->dims[l] * m->dims[l + 1]; k++) {
            const double u = (splitmix(s) >> 11) * (1.0 / 9007199254740992.0);
            h[m->w_off[l] + k] = (float)((2.0 * u - 1.0) * lim);
        }
    }
    const size_t P = m->n_params;
    FE_CUDA_TRY(cudaMalloc(&m->p, 4 * P * sizeof(float) + (2 * (size_t)in_dim + 2) * sizeof(float) + 256));
    m->g = m->p + P;
    m->m = m->g + P;
    m->v = m->m + P;
    m->x_mean = m->v + P;
    m->x_std = m->x_mean + in_dim;
    m->y_stat = m->x_std + in_dim;
    FE_CUDA_TRY(cudaMalloc(&m->t, sizeof(int)));
    FE_CUDA_TRY(cudaMemset(m->p, 0, 4 * P * sizeof(float) + (2 * (size_t)in_dim + 2) * sizeof(float)));
    FE_CUDA_TRY(cudaMemset(m->t, 0, sizeof(int)));
    FE_CUDA_TRY(cudaMemcpy(m->p, h.data(), P * sizeof(float), cudaMemcpyHostToDevice));
    *out = m.release();
    return FE_OK;
}

extern "C" void fe_mlp_destroy(fe_mlp* m) {
    if (!m) return;
    cudaFree(m->p);
    cudaFree(m->t);
    delete m;
}

extern "C" size_t fe_mlp_param_count(const fe_mlp* m) { return m ? m->n_params : 0; }

extern "C" int fe_mlp_get_params(const fe_mlp* m, float* host) {
    if (!m || !host) return fail(FE_EINVAL, "null argument");
    FE_CUDA_TRY(cudaMemcpy(host, m->p, m->n_params * sizeof(float), cudaMemcpyDeviceToHost));
    return FE_OK;
}

extern "C" int fe_mlp_set_params(fe_mlp* m, const float* host) {
    if (!m || !host) return fail(FE_EINVAL, "null argument");
    FE_CUDA_TRY(cudaMemcpy(m->p, host, m->n_params * sizeof(float), cudaMemcpyHostToDevice));
    return FE_OK;
}

extern "C" int fe_mlp_get_scaling(const fe_mlp* m, float* x_mean, float* x_std, float* y_mean_std) {
    if (!m || !x_mean || !x_std || !y_mean_std) return fail(FE_EINVAL, "null argument");
    const int d = m->dims[0];
    FE_CUDA_TRY(cudaMemcpy(x_mean, m->x_mean, d * sizeof(float), cudaMemcpyDeviceToHost));
    FE_CUDA_TRY(cudaMemcpy(x_std, m->x_std, d * sizeof(float), cudaMemcpyDeviceToHost));
    FE_CUDA_TRY(cudaMemcpy(y_mean_std, m->y_stat, 2 * sizeof(float), cudaMemcpyDeviceToHost));
    return FE_OK;
}

extern "C" int fe_mlp_train(fe_mlp* m, const float* X_dev, const float* y_dev, uint32_t n, uint32_t steps, float lr,
                            float weight_decay, float* final_loss, void* stream) {
    FE_ALIGNED(X_dev); FE_ALIGNED(y_dev);
    if (!m || !X_dev || !y_dev) return fail(FE_EINVAL, "null argument");
    if (n < 2) return fail(FE_EINVAL, "fe_mlp_train needs at least 2 samples");
    cudaStream_t st = (cudaStream_t)stream;
    if (!st) return fail(FE_EINVAL, "fe_mlp_train needs a non-default stream (the step is graph-captured)");
    const int L = (int)m->dims.size() - 1, D = m->dims[0];
    Acts A;
    FE_TRY(carve_acts(m, (int)n, st, &A));
    // standardisation from the training set
    k_col_stats<<<blocks_for(D), kT, 0, st>>>(X_dev, (int)n, D, m->x_mean, m->x_std);
    k_col_stats<<<1, kT, 0, st>>>(y_dev, (int)n, 1, m->y_stat, m->y_stat + 1);
    k_standardise<<<blocks_for((size_t)n * D), kT, 0, st>>>(X_dev, (int)n, D, m->x_mean, m->x_std, A.a[0]);
    k_standardise<<<blocks_for(n), kT, 0, st>>>(y_dev, (int)n, 1, m->y_stat, m->y_stat + 1, A.y);
    FE_CUDA_TRY(cudaGetLastError());
    FE_CUDA_TRY(cudaStreamSynchronize(st));
    // one training step as a graph
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    FE_CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    forward(m, A, (int)n, st);
    k_mse_grad<<<blocks_for(n), kT, 0, st>>>(A.a[L], A.y, A.d[L], (int)n);
    for (int l = L - 1; l >= 0; l--) {
        const int din = m->dims[l], dout = m->dims[l + 1];
        k_dense_bwd_w<<<blocks_for((size_t)dout * (din + 1)), kT, 0, st>>>(A.a[l], A.d[l + 1], m->g + m->w_off[l],
                                                                         m->g + m->b_off[l], (int)n, din, dout);
        if (l > 0)
            k_dense_bwd_data<<<blocks_for((size_t)n * din), kT, 0, st>>>(A.d[l + 1], m->p + m->w_off[l], A.a[l],
                                                                       A.d[l], (int)n, din, dout);
    }
    k_adam<<<blocks_for(m->n_params), kT, 0, st>>>(m->p, m->g, m->m, m->v, m->n_params, m->t, lr, 0.9f, 0.999f,
                                                  1e-8f, weight_decay);
    k_step_inc<<<1, 32, 0, st>>>(m->t);
    cudaError_t e = cudaStreamEndCapture(st, &graph);
    if (e != cudaSuccess) return fail(FE_ECUDA, std::string("mlp capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(&exec, graph, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(graph);
        return fail(FE_ECUDA, std::string("mlp instantiate: ") + cudaGetErrorString(e));
    }
    for (uint32_t s = 0; s < steps && e == cudaSuccess; s++) e = cudaGraphLaunch(exec, st);
    if (e == cudaSuccess) {
        forward(m, A, (int)n, st);
        k_mse<<<1, 32, 0, st>>>(A.a[L], A.y, (int)n, A.loss);
        if (final_loss) e = cudaMemcpyAsync(final_loss, A.loss, sizeof(float), cudaMemcpyDeviceToHost, st);
    }
    cudaFreeAsync(A.base, st);
    cudaStreamSynchronize(st);
    cudaGraphExecDestroy(exec);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return fail(FE_ECUDA, std::string("mlp train: ") + cudaGetErrorString(e));
    m->trained = true;
    return FE_OK;
}

__global__ void k_unstandardise(float* y, int n, const float* stat) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = y[i] * stat[1] + stat[0];
}

extern "C" int fe_mlp_predict(fe_mlp* m, const float* X_dev, uint32_t n, float* y_dev, void* stream) {
    FE_ALIGNED(X_dev); FE_ALIGNED(y_dev);
    if (!m || !X_dev || !y_dev) return fail(FE_EINVAL, "null argument");
    if (!m->trained) return fail(FE_EINVAL, "fe_mlp_predict before fe_mlp_train (no feature scaling yet)");
    if (n == 0) return FE_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const int L = (int)m->dims.size() - 1, D = m->dims[0];
    Acts A;
    FE_TRY(carve_acts(m, (int)n, st, &A));
    k_standardise<<<blocks_for((size_t)n * D), kT, 0, st>>>(X_dev, (int)n, D, m->x_mean, m->x_std, A.a[0]);
    forward(m, A, (int)n, st);
    k_unstandardise<<<blocks_for(n), kT, 0, st>>>(A.a[L], (int)n, m->y_stat);
    FE_CUDA_TRY(cudaMemcpyAsync(y_dev, A.a[L], n * sizeof(float), cudaMemcpyDeviceToDevice, st));
    cudaFreeAsync(A.base, st);
    FE_CUDA_TRY(cudaGetLastError());
    return FE_OK;
}
