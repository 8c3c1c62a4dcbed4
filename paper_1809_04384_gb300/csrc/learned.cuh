// Learned interpolation order and truncation rank (no counterpart in the paper, which uses
// one order m for the whole matrix, Section 5, and finds ranks by SVD truncation, Section
// 3.2): per-pair features from the geometry, the interpolation-error probe that labels the
// training data, and a small MLP (8 -> 128 -> 128 -> 2, ReLU, BF16 weights, FP32
// accumulation) with its forward, backward and Adam kernels.
#pragma once

#include <cuda_bf16.h>

#include "common.cuh"
#include "numeric.cuh"
#include "structure.cuh"

namespace dh2 {
namespace learned {

constexpr int kIn = 8, kHid = 128, kOut = 2;
// packed parameters: W1 [128][8], b1 [128], W2 [128][128], b2 [128], W3 [2][128], b3 [2]
constexpr int kOffW1 = 0;
constexpr int kOffB1 = kOffW1 + kHid * kIn;
constexpr int kOffW2 = kOffB1 + kHid;
constexpr int kOffB2 = kOffW2 + kHid * kHid;
constexpr int kOffW3 = kOffB2 + kHid;
constexpr int kOffB3 = kOffW3 + kOut * kHid;
constexpr int kParams = kOffB3 + kOut;     // 17922
constexpr int kOrders = 6;                 // probe orders m = 3..8
constexpr double kMScale = 8.0, kRankScale = 64.0;   // output 0 = m / 8, output 1 = rank / 64
constexpr double kOrderQuantile = 0.99;              // the matrix order: this quantile of the pairs' orders

struct Model {
    DBuf<float> master, mom1, mom2, grad, part, loss;   // FP32 master weights, Adam moments
    DBuf<__nv_bfloat16> wb;                             // BF16 copies used by the forward pass
    int64_t step = 0;
    int dev = 0;
};

void model_init(Model& md, const float* host_params, cudaStream_t s);
// Y[n][2] = MLP(X[n][8]); device pointers
void model_forward(Model& md, const float* X, int64_t n, float* Y, cudaStream_t s);
// loss and gradient of L = sum (y - t)^2 / (2n) into md.loss / md.grad; with adam = true
// also one Adam step of learning rate lr on the master weights
void model_grad(Model& md, const float* X, const float* T, int64_t n, bool adam, float lr, cudaStream_t s);

// features F[ntc][8] (device) of every pair (t, c) of the structure
void features(const Tree& tr, const Structure& st, float* F, cudaStream_t s);
// err[ntc][6] (device, FP64): x-side interpolation error of each pair at m = 3..8 (0 for
// pairs without admissible blocks)
void probe(const Tree& tr, const Structure& st, const HostStructure& hs, double* err, cudaStream_t s);

// The learned choice for one matrix: the order m (the 99th percentile of the orders predicted
// for the active pairs, rounded down and clamped to [3, 8]) and a cap on the truncation rank
// of every active pair (1.25 x the predicted rank + 4).
void choose(const Tree& tr, const Structure& st, const HostStructure& hs, Model& md, cudaStream_t s,
            int32_t* m_out, std::vector<int32_t>& caps);

}  // namespace learned
}  // namespace dh2
