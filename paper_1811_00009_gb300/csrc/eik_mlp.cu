// Training and batched inference of the restart-schedule network (eik_mlp.cuh).
//
// Gradients are deterministic: per-sample quantities are written to a caller
// workspace, each parameter's gradient is summed over fixed chunks of 256
// samples and then over the chunks, always in the same order (no atomics), so
// repeated training runs give the same weights bit for bit.
#include "eik.h"
#include "eik_mlp.cuh"

#include <string>

namespace {

using namespace eikg;

thread_local std::string g_mlp_err;

eik_status mlp_fail(eik_status s, const std::string& m) {
    g_mlp_err = m;
    return s;
}

// workspace layout per sample: h1 (kHid), h2 (kHid), d1 (kHid), d2 (kHid), e (1)
constexpr int kWork = 4 * kHid + 1;

__global__ void k_mlp_forward(const float* __restrict__ w, const float* __restrict__ X, int B, float* __restrict__ Y) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= B) return;
    float x[kIn], y[kAct];
    for (int j = 0; j < kIn; ++j) x[j] = X[s * kIn + j];
    mlp_forward_one(w, x, y, nullptr, nullptr);
    for (int a = 0; a < kAct; ++a) Y[s * kAct + a] = y[a];
}

// per sample: forward, error of the taken action, and the backpropagated deltas
__global__ void k_mlp_deltas(const float* __restrict__ w, const float* __restrict__ X, const int* __restrict__ act,
                             const float* __restrict__ tgt, int B, float* __restrict__ work) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= B) return;
    float x[kIn], y[kAct], h1[kHid], h2[kHid];
    for (int j = 0; j < kIn; ++j) x[j] = X[s * kIn + j];
    mlp_forward_one(w, x, y, h1, h2);
    const int a = act[s];
    const float e = y[a] - tgt[s];
    const float dy = 2.0f * e / static_cast<float>(B);     // d loss / d y_a, loss = mean e^2
    float d2[kHid], d1[kHid];
    for (int j = 0; j < kHid; ++j) d2[j] = dy * w[kOffW3 + a * kHid + j] * (1.0f - h2[j] * h2[j]);
    for (int j = 0; j < kHid; ++j) {
        float t = 0.0f;
        for (int i = 0; i < kHid; ++i) t += d2[i] * w[kOffW2 + i * kHid + j];
        d1[j] = t * (1.0f - h1[j] * h1[j]);
    }
    float* o = work + static_cast<size_t>(s) * kWork;
    for (int j = 0; j < kHid; ++j) {
        o[j] = h1[j];
        o[kHid + j] = h2[j];
        o[2 * kHid + j] = d1[j];
        o[3 * kHid + j] = d2[j];
    }
    o[4 * kHid] = e;
}

// per-sample contribution to parameter p (and, for p == kParams, the squared error)
__device__ inline float param_term(int p, int s, int B, const float* __restrict__ X, const int* __restrict__ act,
                                   const float* __restrict__ work) {
    const float* o = work + static_cast<size_t>(s) * kWork;
    if (p == kParams) return o[4 * kHid] * o[4 * kHid];
    const float* x = X + static_cast<size_t>(s) * kIn;
    if (p < kOffB1) {                       // W1[i][j] : d1_i x_j
        const int i = (p - kOffW1) / kIn, j = (p - kOffW1) % kIn;
        return o[2 * kHid + i] * x[j];
    }
    if (p < kOffW2) return o[2 * kHid + (p - kOffB1)];                 // b1[i]
    if (p < kOffB2) {                       // W2[i][j] : d2_i h1_j
        const int i = (p - kOffW2) / kHid, j = (p - kOffW2) % kHid;
        return o[3 * kHid + i] * o[j];
    }
    if (p < kOffW3) return o[3 * kHid + (p - kOffB2)];                 // b2[i]
    const float dy = 2.0f * o[4 * kHid] / static_cast<float>(B);      // d loss / d y of the taken action
    if (p < kOffB3) {                       // W3[a][j] : dy_a h2_j, taken action only
        const int a = (p - kOffW3) / kHid, j = (p - kOffW3) % kHid;
        return (act[s] == a) ? dy * o[kHid + j] : 0.0f;
    }
    return (act[s] == p - kOffB3) ? dy : 0.0f;                         // b3[a]
}

constexpr int kChunk = 256;   // samples per partial sum

// level 1: partial[c][p] = sum over the samples of chunk c, in order
__global__ void k_mlp_partial(const float* __restrict__ X, const int* __restrict__ act, int B,
                              const float* __restrict__ work, float* __restrict__ partial) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    const int c = blockIdx.y;
    if (p > kParams) return;
    const int s0 = c * kChunk, s1 = min(B, s0 + kChunk);
    float acc = 0.0f;
    for (int s = s0; s < s1; ++s) acc += param_term(p, s, B, X, act, work);
    partial[static_cast<size_t>(c) * (kParams + 1) + p] = acc;
}

// level 2: the chunks' partial sums added in order
__global__ void k_mlp_total(int nchunks, const float* __restrict__ partial, int B, float* __restrict__ grad,
                            float* __restrict__ loss) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p > kParams) return;
    float acc = 0.0f;
    for (int c = 0; c < nchunks; ++c) acc += partial[static_cast<size_t>(c) * (kParams + 1) + p];
    if (p == kParams) {
        if (loss) *loss = acc / static_cast<float>(B);
    } else {
        grad[p] = acc;
    }
}

// Adam (Kingma and Ba, 2015), element-wise
__global__ void k_mlp_adam(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                           float* __restrict__ v, int n, float lr, float b1, float b2, float eps, float c1, float c2) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const float gp = g[p];
    const float mp = b1 * m[p] + (1.0f - b1) * gp;
    const float vp = b2 * v[p] + (1.0f - b2) * gp * gp;
    m[p] = mp;
    v[p] = vp;
    w[p] -= lr * (mp / c1) / (sqrtf(vp / c2) + eps);
}

}  // namespace

extern "C" {

const char* eik_mlp_last_error(void) { return g_mlp_err.c_str(); }

int32_t eik_mlp_work_floats(int32_t B) {
    return B > 0 ? B * kWork + ((B + kChunk - 1) / kChunk) * (kParams + 1) : 0;
}

eik_status eik_mlp_forward(const float* w, const float* X, int32_t B, float* Y, void* stream) {
    if (!w || !X || !Y || B < 1) return mlp_fail(EIK_EINVAL, "eik_mlp_forward: bad argument");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    k_mlp_forward<<<(B + 127) / 128, 128, 0, s>>>(w, X, B, Y);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return mlp_fail(EIK_ECUDA, cudaGetErrorString(e));
    return EIK_OK;
}

eik_status eik_mlp_grad(const float* w, const float* X, const int32_t* act, const float* tgt, int32_t B, float* grad,
                        float* loss, float* work, void* stream) {
    if (!w || !X || !act || !tgt || !grad || !work || B < 1) return mlp_fail(EIK_EINVAL, "eik_mlp_grad: bad argument");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int nchunks = (B + kChunk - 1) / kChunk;
    float* partial = work + static_cast<size_t>(B) * kWork;
    k_mlp_deltas<<<(B + 127) / 128, 128, 0, s>>>(w, X, act, tgt, B, work);
    k_mlp_partial<<<dim3((kParams + 1 + 127) / 128, nchunks), 128, 0, s>>>(X, act, B, work, partial);
    k_mlp_total<<<(kParams + 1 + 127) / 128, 128, 0, s>>>(nchunks, partial, B, grad, loss);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return mlp_fail(EIK_ECUDA, cudaGetErrorString(e));
    return EIK_OK;
}

eik_status eik_mlp_adam(float* w, const float* grad, float* m, float* v, int32_t n, float lr, float b1, float b2,
                        float eps, int32_t t, void* stream) {
    if (!w || !grad || !m || !v || n < 1 || t < 1) return mlp_fail(EIK_EINVAL, "eik_mlp_adam: bad argument");
    const float c1 = 1.0f - powf(b1, static_cast<float>(t));
    const float c2 = 1.0f - powf(b2, static_cast<float>(t));
    k_mlp_adam<<<(n + 255) / 256, 256, 0, static_cast<cudaStream_t>(stream)>>>(w, grad, m, v, n, lr, b1, b2, eps, c1,
                                                                                c2);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return mlp_fail(EIK_ECUDA, cudaGetErrorString(e));
    return EIK_OK;
}

eik_status eik_sched_actions(double* stride_h, int32_t* block_dim, int32_t cap, int32_t* n) {
    if (!n) return mlp_fail(EIK_EINVAL, "eik_sched_actions: n is NULL");
    *n = kAct;
    for (int a = 0; a < kAct && a < cap; ++a) {
        if (stride_h) stride_h[a] = action_stride_h(a);
        if (block_dim) block_dim[a] = action_block(a);
    }
    return EIK_OK;
}

}  // extern "C"
