// Learned per-element Davidson preconditioner: a 5 -> 64 -> 64 -> 1 tanh MLP
// g(x) that scales the diagonal (Jacobi) correction, t_i = -g_i r_i / (H_ii - theta).
// Inputs per element i: ((H_ii - theta)/s, theta/s, r_i/|r|_inf, N_L/N, 2Sz_L/N)
// with s = max_i |H_ii - theta|.  Trained on the GPU (FP32 weights, Adam) on
// targets g_i = -t_i (H_ii - theta) / r_i taken from Jacobi-Davidson correction
// equations solved to convergence by the plain method; inference runs with
// bf16 weights.  g = 1 everywhere is the Jacobi preconditioner (the fallback).
#pragma once

#include <cuda_bf16.h>

#include <cstdint>
#include <vector>

#include "common.h"

namespace dmrg {

constexpr int kMlpIn = 5, kMlpHid = 64;
// flattened parameters: W1 [64 x 5], b1 [64], W2 [64 x 64], b2 [64], W3 [64], b3 [1]
constexpr int kMlpOffW1 = 0, kMlpOffB1 = kMlpOffW1 + kMlpHid * kMlpIn, kMlpOffW2 = kMlpOffB1 + kMlpHid,
              kMlpOffB2 = kMlpOffW2 + kMlpHid * kMlpHid, kMlpOffW3 = kMlpOffB2 + kMlpHid,
              kMlpOffB3 = kMlpOffW3 + kMlpHid, kMlpParams = kMlpOffB3 + 1;

struct Mlp {
    float* d_w = nullptr;            // FP32 parameters
    __nv_bfloat16* d_wb = nullptr;   // bf16 copy used by inference
    float* d_adam = nullptr;         // Adam moments (2 x params)
    float* d_grad = nullptr;         // gradient (params) + loss accumulator
    int64_t adam_t = 0;
    bool trained = false;
    // training set: features (n x 5) and targets (n), FP32, on the device
    float* d_x = nullptr;
    float* d_y = nullptr;
    float* d_wt = nullptr;  // pair weights (r_i / (H_ii - theta))^2, mean 1 per solve
    int64_t n_set = 0, cap_set = 0;
    // training workspace (per batch): activations and their gradients
    float* d_work = nullptr;
    int64_t cap_work = 0;
    // per-sector quantum-number features of the current bond
    int64_t* d_sec_off = nullptr;
    float* d_sec_q = nullptr;
    int n_sec = 0;
    void release();
};

// parameters <- seeded initialisation with g(x) = 1 (the Jacobi preconditioner)
void mlp_init(Mlp& m, uint32_t seed, cudaStream_t st);
// per-element features of residual r (n) at Ritz value theta (device arrays)
void mlp_features(const Mlp& m, const double* hd, const double* r, double theta, double s, double rmax, int64_t n,
                  float* x, cudaStream_t st);
// g = MLP(x) for n feature rows; bf16 = 1 uses the bf16 weights
void mlp_forward(const Mlp& m, const float* x, int64_t n, float* g, bool bf16, cudaStream_t st);
// gradient of the weighted mean squared error (1/n) sum w_i (g(x_i) - y_i)^2
// (w = 1 when w is null) with respect to the parameters into grad (kMlpParams)
// and the loss into *loss (device)
void mlp_gradient(Mlp& m, const float* x, const float* y, const float* w, int64_t n, float* grad, float* loss,
                  cudaStream_t st);
// one Adam step on the parameters with the gradient in m.d_grad
void mlp_adam(Mlp& m, float lr, cudaStream_t st);
// bf16 copy of the parameters for inference
void mlp_publish(Mlp& m, cudaStream_t st);
// t = -clip(g) r / (hd - theta) (|hd - theta| clamped to 1e-8, keeping its sign), n elements
void mlp_apply(const double* r, const double* hd, double theta, const float* g, double* t, int64_t n,
               cudaStream_t st);
// append up to max_take samples (strided) of (features, target) where target
// g_i = -t_i (hd_i - theta) / r_i is well defined, clipped to [-10, 10]
int64_t mlp_collect(Mlp& m, const double* hd, const double* r, const double* t, double theta, double s, double rmax,
                    int64_t n, int64_t max_take, cudaStream_t st);

// max_i |x_i - shift| (host result; work holds >= 512 doubles)
double dev_absmax(const double* x, double shift, int64_t n, double* work, cudaStream_t st);

// steps Adam steps on batches of B pairs drawn (counter-based, seeded) from the
// first nine tenths of the training set (weighted loss); loss of the first and
// last batch, and of the held-out last tenth before and after, to the host;
// publishes the bf16 weights and marks the network trained
void mlp_train(Mlp& m, int steps, int64_t B, float lr, uint64_t seed, float* loss_first, float* loss_last,
               float* held_first, float* held_last, cudaStream_t st);

}  // namespace dmrg
