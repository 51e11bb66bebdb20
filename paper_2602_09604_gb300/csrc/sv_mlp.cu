// Learned fusion cost model: a 16 -> 64 -> 64 -> 64 -> 1 fp32 MLP (ReLU) that predicts the device
// time of one fused gate from its size, target positions, kernel path and the qubit count.  The
// paper picks its fusion size f per machine with a synthetic benchmark (section VI-C); here the
// simulator times its own kernels and learns the cost instead.
//
// Target: y = ln(microseconds) - n ln 2, the log time per amplitude (a pass streams 2^n
// amplitudes, so this removes the exponential dependence on n), standardised with the training
// mean and deviation.  Loss: mean squared error.  Optimiser: Adam.  Forward, backward and the
// Adam update are hand-written kernels; the host only shuffles indices and loops over batches.
//
// Flat parameter order: W1 (64x16, row-major), b1, W2 (64x64), b2, W3 (64x64), b3, W4 (1x64), b4.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "sv_internal.h"

using namespace svg;

namespace {

constexpr int kIn = 16, kH = 64;
constexpr int kSizes[5] = {kIn, kH, kH, kH, 1};
constexpr int kLayers = 4;
constexpr int kParams = kH * kIn + kH + kH * kH + kH + kH * kH + kH + kH + 1;   // 9473
constexpr int kMaxBatch = 1024;

int w_off(int l)
{
    int o = 0;
    for (int i = 0; i < l; ++i) o += kSizes[i + 1] * kSizes[i] + kSizes[i + 1];
    return o;
}
int b_off(int l) { return w_off(l) + kSizes[l + 1] * kSizes[l]; }

// ------------------------------------------------------------------------------------- kernels
// out_pre[b][o] = bias[o] + sum_i in[b][i] W[o][i]; out_act = relu(out_pre) (or copy when linear)
__global__ void dense_forward(const float *__restrict__ in, const float *__restrict__ W, const float *__restrict__ bias,
                              float *__restrict__ pre, float *__restrict__ act, int B, int fin, int fout, int relu)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= B * fout) return;
    const int b = idx / fout, o = idx % fout;
    float acc = bias[o];
    for (int i = 0; i < fin; ++i) acc = fmaf(in[b * fin + i], W[o * fin + i], acc);
    pre[idx] = acc;
    act[idx] = relu ? fmaxf(acc, 0.f) : acc;
}

// delta[b] = 2 (y[b] - t[b]) / B; loss = mean (y - t)^2 (one block of 1024 threads, fixed order)
__global__ void __launch_bounds__(1024) mse_grad(const float *__restrict__ y, const float *__restrict__ t,
                                                 float *__restrict__ delta, float *__restrict__ loss, int B)
{
    __shared__ float part[1024];
    float s = 0.f;
    for (int b = threadIdx.x; b < B; b += blockDim.x) {
        const float r = y[b] - t[b];
        delta[b] = 2.f * r / (float)B;
        s = fmaf(r, r, s);
    }
    part[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *loss = part[0] / (float)B;
}

// gW[o][i] = sum_b delta[b][o] in[b][i]  (i == fin: gb[o] = sum_b delta[b][o])
__global__ void dense_backward_w(const float *__restrict__ delta, const float *__restrict__ in, float *__restrict__ gW,
                                 float *__restrict__ gb, int B, int fin, int fout)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= fout * (fin + 1)) return;
    const int o = idx / (fin + 1), i = idx % (fin + 1);
    float acc = 0.f;
    if (i < fin) {
        for (int b = 0; b < B; ++b) acc = fmaf(delta[b * fout + o], in[b * fin + i], acc);
        gW[o * fin + i] = acc;
    } else {
        for (int b = 0; b < B; ++b) acc += delta[b * fout + o];
        gb[o] = acc;
    }
}

// dprev[b][i] = (sum_o delta[b][o] W[o][i]) * (pre_prev[b][i] > 0)
__global__ void dense_backward_x(const float *__restrict__ delta, const float *__restrict__ W, const float *__restrict__ pre_prev,
                                 float *__restrict__ dprev, int B, int fin, int fout)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= B * fin) return;
    const int b = idx / fin, i = idx % fin;
    float acc = 0.f;
    for (int o = 0; o < fout; ++o) acc = fmaf(delta[b * fout + o], W[o * fin + i], acc);
    dprev[idx] = pre_prev[idx] > 0.f ? acc : 0.f;
}

__global__ void adam_update(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m, float *__restrict__ v,
                            int P, float lr, float b1, float b2, float eps, float c1, float c2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// rows of X / t picked by idx into the batch buffers
__global__ void gather_rows(const float *__restrict__ X, const float *__restrict__ T, const int *__restrict__ idx,
                            float *__restrict__ xb, float *__restrict__ tb, int B)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < B * kIn) xb[e] = X[(size_t)idx[e / kIn] * kIn + e % kIn];
    if (e < B) tb[e] = T[idx[e]];
}

int blocks(int n, int t) { return (n + t - 1) / t; }

uint64_t splitmix(uint64_t &s)
{
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
double uniform01(uint64_t &s) { return (double)(splitmix(s) >> 11) * (1.0 / 9007199254740992.0); }

}  // namespace

struct sv_mlp {
    int device = 0;
    cudaStream_t stream = nullptr;
    float *d_p = nullptr, *d_g = nullptr, *d_m = nullptr, *d_v = nullptr;
    // activations: x (B x 16), pre/act per layer, deltas per layer
    float *d_x = nullptr, *d_t = nullptr, *d_pre[kLayers] = {}, *d_act[kLayers] = {}, *d_del[kLayers] = {};
    float *d_loss = nullptr;
    float *d_X = nullptr, *d_T = nullptr;   // uploaded training set
    int *d_idx = nullptr;
    long long n_data = 0;
    long long step = 0;
    float y_mean = 0.f, y_std = 1.f;
    float val_mape = 1e30f;
    int trained = 0;
    int fallback_k = 4;
};

namespace {

int mlp_alloc_scratch(sv_mlp *m)
{
    SV_CUDA_TRY(cudaMalloc(&m->d_x, sizeof(float) * kMaxBatch * kIn));
    SV_CUDA_TRY(cudaMalloc(&m->d_t, sizeof(float) * kMaxBatch));
    for (int l = 0; l < kLayers; ++l) {
        SV_CUDA_TRY(cudaMalloc(&m->d_pre[l], sizeof(float) * kMaxBatch * kSizes[l + 1]));
        SV_CUDA_TRY(cudaMalloc(&m->d_act[l], sizeof(float) * kMaxBatch * kSizes[l + 1]));
        SV_CUDA_TRY(cudaMalloc(&m->d_del[l], sizeof(float) * kMaxBatch * kSizes[l + 1]));
    }
    SV_CUDA_TRY(cudaMalloc(&m->d_loss, sizeof(float)));
    SV_CUDA_TRY(cudaMalloc(&m->d_idx, sizeof(int) * kMaxBatch));
    return SV_OK;
}

// forward over the batch already in d_x; prediction (standardised) ends in d_act[3]
int mlp_forward(sv_mlp *m, int B)
{
    const float *in = m->d_x;
    for (int l = 0; l < kLayers; ++l) {
        const int fin = kSizes[l], fout = kSizes[l + 1];
        dense_forward<<<blocks(B * fout, 256), 256, 0, m->stream>>>(in, m->d_p + w_off(l), m->d_p + b_off(l), m->d_pre[l],
                                                                    m->d_act[l], B, fin, fout, l < kLayers - 1);
        in = m->d_act[l];
    }
    SV_CUDA_TRY(cudaGetLastError());
    return SV_OK;
}

// loss + full gradient into d_g for the batch in d_x / d_t
int mlp_backward(sv_mlp *m, int B)
{
    mse_grad<<<1, 1024, 0, m->stream>>>(m->d_act[kLayers - 1], m->d_t, m->d_del[kLayers - 1], m->d_loss, B);
    for (int l = kLayers - 1; l >= 0; --l) {
        const int fin = kSizes[l], fout = kSizes[l + 1];
        const float *in = l == 0 ? m->d_x : m->d_act[l - 1];
        dense_backward_w<<<blocks(fout * (fin + 1), 256), 256, 0, m->stream>>>(m->d_del[l], in, m->d_g + w_off(l),
                                                                              m->d_g + b_off(l), B, fin, fout);
        if (l > 0)
            dense_backward_x<<<blocks(B * fin, 256), 256, 0, m->stream>>>(m->d_del[l], m->d_p + w_off(l), m->d_pre[l - 1],
                                                                         m->d_del[l - 1], B, fin, fout);
    }
    SV_CUDA_TRY(cudaGetLastError());
    return SV_OK;
}

int mlp_adam(sv_mlp *m, float lr)
{
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    m->step += 1;
    const float c1 = 1.f - (float)std::pow(b1, (double)m->step);
    const float c2 = 1.f - (float)std::pow(b2, (double)m->step);
    adam_update<<<blocks(kParams, 256), 256, 0, m->stream>>>(m->d_p, m->d_g, m->d_m, m->d_v, kParams, lr, b1, b2, eps, c1, c2);
    SV_CUDA_TRY(cudaGetLastError());
    return SV_OK;
}

}  // namespace

namespace svg {

// Feature vector of one fused gate (see include/sv_gb300.h, sv_mlp_features).
void mlp_features(int k, const int *targets_sorted, int path, int n, int post, float *f)
{
    for (int i = 0; i < kIn; ++i) f[i] = 0.f;
    f[0] = (float)k / 6.f;
    for (int i = 0; i < 6; ++i) f[1 + i] = i < k ? (float)targets_sorted[i] / (float)n : -1.f;
    if (path >= SV_PATH_LOW && path <= SV_PATH_TC_BF16X3) f[7 + (path - SV_PATH_LOW)] = 1.f;
    f[12] = (float)n / 34.f;
    int low = 0, mx = 0;
    for (int i = 0; i < k; ++i) {
        low += targets_sorted[i] < 5;
        mx = std::max(mx, targets_sorted[i]);
    }
    f[13] = (float)low / 5.f;
    f[14] = (float)mx / (float)n;
    f[15] = post ? 1.f : 0.f;
}

// Predicted microseconds of each feature row (rows on the host); model must be trained.
int mlp_predict_us(sv_mlp *m, const float *X, int rows, double *out_us)
{
    SV_CUDA_TRY(cudaSetDevice(m->device));
    std::vector<float> y(kMaxBatch);
    for (int r0 = 0; r0 < rows; r0 += kMaxBatch) {
        const int B = std::min(kMaxBatch, rows - r0);
        SV_CUDA_TRY(cudaMemcpyAsync(m->d_x, X + (size_t)r0 * kIn, sizeof(float) * B * kIn, cudaMemcpyHostToDevice, m->stream));
        SV_TRY(mlp_forward(m, B));
        SV_CUDA_TRY(cudaMemcpyAsync(y.data(), m->d_act[kLayers - 1], sizeof(float) * B, cudaMemcpyDeviceToHost, m->stream));
        SV_CUDA_TRY(cudaStreamSynchronize(m->stream));
        for (int b = 0; b < B; ++b) {
            const double n = std::round((double)X[(size_t)(r0 + b) * kIn + 12] * 34.0);
            out_us[r0 + b] = std::exp((double)y[b] * m->y_std + m->y_mean + n * std::log(2.0));
        }
    }
    return SV_OK;
}

bool mlp_usable(const sv_mlp *m, double max_mape) { return m && m->trained && m->val_mape <= max_mape; }
int mlp_fallback_k(const sv_mlp *m) { return m ? m->fallback_k : 4; }

}  // namespace svg

// ================================================================================== C ABI
extern "C" int sv_mlp_num_params(void) { return kParams; }

extern "C" int sv_mlp_create(uint64_t seed, void *cuda_stream, sv_mlp **out)
{
    clear_error();
    if (!out) { set_error("sv_mlp_create: out is NULL"); return SV_EINVAL; }
    *out = nullptr;
    sv_mlp *m = new (std::nothrow) sv_mlp();
    if (!m) { set_error("sv_mlp_create: out of host memory"); return SV_ENOMEM; }
    cudaGetDevice(&m->device);
    m->stream = static_cast<cudaStream_t>(cuda_stream);
    int rc = SV_OK;
    cudaError_t e = cudaMalloc(&m->d_p, sizeof(float) * kParams);
    if (e == cudaSuccess) e = cudaMalloc(&m->d_g, sizeof(float) * kParams);
    if (e == cudaSuccess) e = cudaMalloc(&m->d_m, sizeof(float) * kParams);
    if (e == cudaSuccess) e = cudaMalloc(&m->d_v, sizeof(float) * kParams);
    if (e != cudaSuccess) { set_error("sv_mlp_create: %s", cudaGetErrorString(e)); rc = SV_ENOMEM; }
    if (rc == SV_OK) rc = mlp_alloc_scratch(m);
    if (rc == SV_OK) {
        // He-normal weights (Box-Muller over splitmix64), zero biases
        std::vector<float> p(kParams, 0.f);
        uint64_t s = seed;
        for (int l = 0; l < kLayers; ++l) {
            const double sd = std::sqrt(2.0 / kSizes[l]);
            for (int i = 0; i < kSizes[l + 1] * kSizes[l]; ++i) {
                const double u1 = std::max(uniform01(s), 1e-300), u2 = uniform01(s);
                p[size_t(w_off(l) + i)] = (float)(sd * std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2));
            }
        }
        e = cudaMemcpy(m->d_p, p.data(), sizeof(float) * kParams, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemset(m->d_m, 0, sizeof(float) * kParams);
        if (e == cudaSuccess) e = cudaMemset(m->d_v, 0, sizeof(float) * kParams);
        if (e != cudaSuccess) { set_error("sv_mlp_create: %s", cudaGetErrorString(e)); rc = SV_ECUDA; }
    }
    if (rc != SV_OK) {
        sv_mlp_free(m);
        return rc;
    }
    *out = m;
    return SV_OK;
}

extern "C" void sv_mlp_free(sv_mlp *m)
{
    if (!m) return;
    cudaStreamSynchronize(m->stream);
    cudaFree(m->d_p); cudaFree(m->d_g); cudaFree(m->d_m); cudaFree(m->d_v);
    cudaFree(m->d_x); cudaFree(m->d_t); cudaFree(m->d_loss); cudaFree(m->d_idx);
    cudaFree(m->d_X); cudaFree(m->d_T);
    for (int l = 0; l < kLayers; ++l) { cudaFree(m->d_pre[l]); cudaFree(m->d_act[l]); cudaFree(m->d_del[l]); }
    delete m;
}

extern "C" int sv_mlp_get_params(const sv_mlp *m, float *out)
{
    clear_error();
    if (!m || !out) { set_error("sv_mlp_get_params: NULL argument"); return SV_EINVAL; }
    SV_CUDA_TRY(cudaMemcpy(out, m->d_p, sizeof(float) * kParams, cudaMemcpyDeviceToHost));
    return SV_OK;
}

extern "C" int sv_mlp_set_params(sv_mlp *m, const float *in)
{
    clear_error();
    if (!m || !in) { set_error("sv_mlp_set_params: NULL argument"); return SV_EINVAL; }
    SV_CUDA_TRY(cudaMemcpy(m->d_p, in, sizeof(float) * kParams, cudaMemcpyHostToDevice));
    return SV_OK;
}

extern "C" int sv_mlp_features(int k, const int *targets, int path, int n_qubits, int post_phases, float *out)
{
    clear_error();
    if (!targets || !out || k < 1 || k > SV_MAX_K || n_qubits < 1 || n_qubits > SV_MAX_QUBITS || post_phases < 0 ||
        post_phases > 1) {
        set_error("sv_mlp_features: bad argument");
        return SV_EINVAL;
    }
    int t[SV_MAX_K];
    for (int i = 0; i < k; ++i) t[i] = targets[i];
    std::sort(t, t + k);
    mlp_features(k, t, path, n_qubits, post_phases, out);
    return SV_OK;
}

extern "C" int sv_mlp_gradients(sv_mlp *m, const float *X, const float *t, int B, float *loss, float *grads)
{
    clear_error();
    if (!m || !X || !t || !loss || !grads || B < 1 || B > kMaxBatch) { set_error("sv_mlp_gradients: bad argument (1 <= B <= %d)", kMaxBatch); return SV_EINVAL; }
    SV_CUDA_TRY(cudaMemcpyAsync(m->d_x, X, sizeof(float) * B * kIn, cudaMemcpyHostToDevice, m->stream));
    SV_CUDA_TRY(cudaMemcpyAsync(m->d_t, t, sizeof(float) * B, cudaMemcpyHostToDevice, m->stream));
    SV_TRY(mlp_forward(m, B));
    SV_TRY(mlp_backward(m, B));
    SV_CUDA_TRY(cudaMemcpyAsync(loss, m->d_loss, sizeof(float), cudaMemcpyDeviceToHost, m->stream));
    SV_CUDA_TRY(cudaMemcpyAsync(grads, m->d_g, sizeof(float) * kParams, cudaMemcpyDeviceToHost, m->stream));
    SV_CUDA_TRY(cudaStreamSynchronize(m->stream));
    return SV_OK;
}

extern "C" int sv_mlp_adam_step(sv_mlp *m, float lr)
{
    clear_error();
    if (!m) { set_error("sv_mlp_adam_step: NULL model"); return SV_EINVAL; }
    SV_TRY(mlp_adam(m, lr));
    SV_CUDA_TRY(cudaStreamSynchronize(m->stream));
    return SV_OK;
}

extern "C" int sv_mlp_train(sv_mlp *m, const float *X, const float *us, long long N, const sv_mlp_train_opts *o_in,
                            sv_mlp_stats *stats)
{
    clear_error();
    if (!m || !X || !us || N < 8) { set_error("sv_mlp_train: bad argument (need >= 8 samples)"); return SV_EINVAL; }
    sv_mlp_train_opts o{};
    o.epochs = 200; o.batch = 256; o.lr = 1e-3f; o.seed = 1; o.val_frac = 0.1f; o.fallback_k = 4;
    if (o_in) o = *o_in;
    if (o.batch < 1 || o.batch > kMaxBatch || o.epochs < 1 || !(o.lr > 0.f) || !(o.val_frac >= 0.f && o.val_frac < 0.9f)) {
        set_error("sv_mlp_train: bad options");
        return SV_EINVAL;
    }
    // targets: standardised log time per amplitude
    std::vector<float> T((size_t)N);
    double mean = 0.0, sq = 0.0;
    for (long long i = 0; i < N; ++i) {
        if (!(us[i] > 0.f)) { set_error("sv_mlp_train: time %lld is not positive", i); return SV_EINVAL; }
        const double n = std::round((double)X[i * kIn + 12] * 34.0);
        const double y = std::log((double)us[i]) - n * std::log(2.0);
        T[(size_t)i] = (float)y;
        mean += y;
        sq += y * y;
    }
    mean /= (double)N;
    const double sd = std::max(std::sqrt(std::max(sq / (double)N - mean * mean, 0.0)), 1e-6);
    for (auto &v : T) v = (float)((v - mean) / sd);
    m->y_mean = (float)mean;
    m->y_std = (float)sd;
    // seeded split into training and validation rows
    std::vector<int> perm((size_t)N);
    for (long long i = 0; i < N; ++i) perm[(size_t)i] = (int)i;
    uint64_t s = o.seed;
    for (long long i = N - 1; i > 0; --i) std::swap(perm[(size_t)i], perm[(size_t)(splitmix(s) % (uint64_t)(i + 1))]);
    const long long n_val = (long long)(o.val_frac * (double)N);
    const long long n_tr = N - n_val;
    cudaFree(m->d_X);
    cudaFree(m->d_T);
    m->d_X = m->d_T = nullptr;
    SV_CUDA_TRY(cudaMalloc(&m->d_X, sizeof(float) * (size_t)N * kIn));
    SV_CUDA_TRY(cudaMalloc(&m->d_T, sizeof(float) * (size_t)N));
    SV_CUDA_TRY(cudaMemcpy(m->d_X, X, sizeof(float) * (size_t)N * kIn, cudaMemcpyHostToDevice));
    SV_CUDA_TRY(cudaMemcpy(m->d_T, T.data(), sizeof(float) * (size_t)N, cudaMemcpyHostToDevice));
    m->n_data = N;
    std::vector<int> tr(perm.begin(), perm.begin() + n_tr);
    float last = 0.f;
    std::vector<float> batch_loss;
    for (int ep = 0; ep < o.epochs; ++ep) {
        for (long long i = n_tr - 1; i > 0; --i) std::swap(tr[(size_t)i], tr[(size_t)(splitmix(s) % (uint64_t)(i + 1))]);
        double ep_loss = 0.0;
        int nb = 0;
        for (long long b0 = 0; b0 < n_tr; b0 += o.batch) {
            const int B = (int)std::min<long long>(o.batch, n_tr - b0);
            SV_CUDA_TRY(cudaMemcpyAsync(m->d_idx, tr.data() + b0, sizeof(int) * B, cudaMemcpyHostToDevice, m->stream));
            gather_rows<<<blocks(B * kIn, 256), 256, 0, m->stream>>>(m->d_X, m->d_T, m->d_idx, m->d_x, m->d_t, B);
            SV_TRY(mlp_forward(m, B));
            SV_TRY(mlp_backward(m, B));
            SV_TRY(mlp_adam(m, o.lr));
            if (ep == o.epochs - 1) {
                float l = 0.f;
                SV_CUDA_TRY(cudaMemcpyAsync(&l, m->d_loss, sizeof(float), cudaMemcpyDeviceToHost, m->stream));
                SV_CUDA_TRY(cudaStreamSynchronize(m->stream));
                ep_loss += l;
                ++nb;
            }
        }
        if (ep == o.epochs - 1) last = (float)(ep_loss / std::max(nb, 1));
    }
    SV_CUDA_TRY(cudaStreamSynchronize(m->stream));
    m->trained = 1;
    m->fallback_k = o.fallback_k;
    // validation: mean absolute percentage error of predicted times
    double mape = 0.0;
    if (n_val > 0) {
        std::vector<float> xv((size_t)n_val * kIn);
        for (long long i = 0; i < n_val; ++i)
            std::memcpy(&xv[(size_t)i * kIn], X + (size_t)perm[(size_t)(n_tr + i)] * kIn, sizeof(float) * kIn);
        std::vector<double> pred((size_t)n_val);
        SV_TRY(mlp_predict_us(m, xv.data(), (int)n_val, pred.data()));
        for (long long i = 0; i < n_val; ++i) {
            const double meas = us[perm[(size_t)(n_tr + i)]];
            mape += std::fabs(pred[(size_t)i] - meas) / meas;
        }
        mape /= (double)n_val;
    }
    m->val_mape = n_val > 0 ? (float)mape : 1e30f;
    if (stats) {
        stats->train_loss = last;
        stats->val_mape = m->val_mape;
        stats->n_train = n_tr;
        stats->n_val = n_val;
        stats->steps = m->step;
        stats->trained = m->trained;
        stats->y_mean = m->y_mean;
        stats->y_std = m->y_std;
        stats->fallback_k = m->fallback_k;
    }
    return SV_OK;
}

extern "C" int sv_mlp_predict(sv_mlp *m, const float *X, int rows, double *out_us)
{
    clear_error();
    if (!m || !X || !out_us || rows < 0) { set_error("sv_mlp_predict: bad argument"); return SV_EINVAL; }
    if (!m->trained) { set_error("sv_mlp_predict: model is not trained"); return SV_ESTATE; }
    return mlp_predict_us(m, X, rows, out_us);
}

extern "C" int sv_mlp_get_stats(const sv_mlp *m, sv_mlp_stats *stats)
{
    clear_error();
    if (!m || !stats) { set_error("sv_mlp_get_stats: NULL argument"); return SV_EINVAL; }
    std::memset(stats, 0, sizeof(*stats));
    stats->val_mape = m->val_mape;
    stats->steps = m->step;
    stats->trained = m->trained;
    stats->y_mean = m->y_mean;
    stats->y_std = m->y_std;
    stats->fallback_k = m->fallback_k;
    return SV_OK;
}

namespace {
const char kMagic[8] = {'S', 'V', 'M', 'L', 'P', '1', 0, 0};
}

extern "C" int sv_mlp_save(const sv_mlp *m, const char *path)
{
    clear_error();
    if (!m || !path) { set_error("sv_mlp_save: NULL argument"); return SV_EINVAL; }
    std::vector<float> p(kParams);
    SV_CUDA_TRY(cudaMemcpy(p.data(), m->d_p, sizeof(float) * kParams, cudaMemcpyDeviceToHost));
    FILE *fh = std::fopen(path, "wb");
    if (!fh) { set_error("sv_mlp_save: cannot open %s", path); return SV_EINVAL; }
    const int32_t hdr[3] = {kParams, m->trained, m->fallback_k};
    const float fl[3] = {m->y_mean, m->y_std, m->val_mape};
    bool ok = std::fwrite(kMagic, 1, 8, fh) == 8 && std::fwrite(hdr, 4, 3, fh) == 3 && std::fwrite(fl, 4, 3, fh) == 3 &&
              std::fwrite(p.data(), 4, kParams, fh) == (size_t)kParams;
    ok = (std::fclose(fh) == 0) && ok;
    if (!ok) { set_error("sv_mlp_save: write to %s failed", path); return SV_EINVAL; }
    return SV_OK;
}

extern "C" int sv_mlp_load(const char *path, void *cuda_stream, sv_mlp **out)
{
    clear_error();
    if (!path || !out) { set_error("sv_mlp_load: NULL argument"); return SV_EINVAL; }
    *out = nullptr;
    FILE *fh = std::fopen(path, "rb");
    if (!fh) { set_error("sv_mlp_load: cannot open %s", path); return SV_EINVAL; }
    char magic[8];
    int32_t hdr[3];
    float fl[3];
    std::vector<float> p(kParams);
    bool ok = std::fread(magic, 1, 8, fh) == 8 && std::memcmp(magic, kMagic, 8) == 0 && std::fread(hdr, 4, 3, fh) == 3 &&
              hdr[0] == kParams && std::fread(fl, 4, 3, fh) == 3 && std::fread(p.data(), 4, kParams, fh) == (size_t)kParams;
    std::fclose(fh);
    if (!ok) { set_error("sv_mlp_load: %s is not a cost-model file of this version", path); return SV_EINVAL; }
    for (float v : p)
        if (!std::isfinite(v)) { set_error("sv_mlp_load: %s holds non-finite parameters", path); return SV_EINVAL; }
    sv_mlp *m = nullptr;
    SV_TRY(sv_mlp_create(0, cuda_stream, &m));
    if (sv_mlp_set_params(m, p.data()) != SV_OK) { sv_mlp_free(m); return SV_ECUDA; }
    m->trained = hdr[1];
    m->fallback_k = hdr[2];
    m->y_mean = fl[0];
    m->y_std = fl[1];
    m->val_mape = fl[2];
    *out = m;
    return SV_OK;
}
