// The restart-schedule network (no counterpart in the paper): a small MLP that
// maps statistics of the front after restart k to a predicted log cost rate
// (device milliseconds per unit of bound advance) for each action, where an
// action is a (stride, block edge) pair for restart k+1.  The schedule only
// decides which restart does which work; the solution does not depend on it.
//
// x (kIn) -> tanh(W1 x + b1) (kHid) -> tanh(W2 h1 + b2) (kHid) -> W3 h2 + b3 (kAct)
// Parameters: one flat float vector W1 (kHid x kIn, row-major), b1, W2, b2, W3, b3.
#pragma once

namespace eikg {

constexpr int kIn = 10;
constexpr int kHid = 32;
constexpr int kAct = 12;
constexpr int kParams = kHid * kIn + kHid + kHid * kHid + kHid + kAct * kHid + kAct;
constexpr int kOffW1 = 0;
constexpr int kOffB1 = kOffW1 + kHid * kIn;
constexpr int kOffW2 = kOffB1 + kHid;
constexpr int kOffB2 = kOffW2 + kHid * kHid;
constexpr int kOffW3 = kOffB2 + kHid;
constexpr int kOffB3 = kOffW3 + kAct * kHid;

// Actions: (stride in units of h, block edge).  Eight strides with 8^3 blocks
// and four with 16^3 blocks.
__host__ __device__ inline double action_stride_h(int a) {
    const double s[kAct] = {1.0, 1.5, 2.0, 2.5, 3.0, 3.5, 4.0, 5.0, 2.0, 3.0, 4.0, 6.0};
    return s[a];
}
__host__ __device__ inline int action_block(int a) { return a < 8 ? 8 : 16; }

// One sample, one thread: outputs y and (optionally) the hidden activations.
__device__ inline void mlp_forward_one(const float* __restrict__ w, const float* x, float* y, float* h1o, float* h2o) {
    float h1[kHid], h2[kHid];
#pragma unroll 4
    for (int i = 0; i < kHid; ++i) {
        float s = w[kOffB1 + i];
        for (int j = 0; j < kIn; ++j) s += w[kOffW1 + i * kIn + j] * x[j];
        h1[i] = tanhf(s);
    }
#pragma unroll 4
    for (int i = 0; i < kHid; ++i) {
        float s = w[kOffB2 + i];
        for (int j = 0; j < kHid; ++j) s += w[kOffW2 + i * kHid + j] * h1[j];
        h2[i] = tanhf(s);
    }
    for (int a = 0; a < kAct; ++a) {
        float s = w[kOffB3 + a];
        for (int j = 0; j < kHid; ++j) s += w[kOffW3 + a * kHid + j] * h2[j];
        y[a] = s;
    }
    if (h1o)
        for (int i = 0; i < kHid; ++i) h1o[i] = h1[i];
    if (h2o)
        for (int i = 0; i < kHid; ++i) h2o[i] = h2[i];
}

}  // namespace eikg
