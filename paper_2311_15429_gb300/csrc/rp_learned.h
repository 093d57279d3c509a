// Learned far field: the network, its training step, and the kernels that
// turn source moments into network rows and network outputs into the far
// path's target coefficients (rp_learned.cu, rp_learned_data.cu).
#pragma once

#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "rp_internal.h"

namespace rp {

constexpr int kLWin = 16;                 // delay samples per window
constexpr int kLMom = 10;                 // moments per field (l <= 2)
constexpr int kLIn = 2 * kLWin * kLMom;   // network inputs: the window and the window * L0/R
constexpr int kLHid = 256;                // hidden width (three hidden layers)
constexpr int kLNodes = 4;                // canonical nodes per axis
constexpr int kLOut = kLNodes * kLNodes * kLNodes;   // outputs: values at the 64 canonical nodes
constexpr float kLLeak = 0.2f;            // leaky slope of the hidden activations
constexpr double kLL0 = 1000.0;           // length scale of the 1/R feature copy (bohr)
constexpr float kLGradScale = 256.0f;     // scale of the fp16 output gradients (undone in Adam)

// Network and training buffers.  Layer l maps d[l] -> d[l+1] with
// d = {kLIn, kLHid, kLHid, kLHid, kLOut}; weights are [out][in] row-major.
struct Mlp {
    int cap = 0;                         // rows per batch (multiple of 128)
    float *W[4] = {}, *G[4] = {}, *m[4] = {}, *v[4] = {};
    __half *W16[4] = {}, *Wt16[4] = {};  // fp16 weights [out][in] and transposed [in][out]
    __half *X16 = nullptr, *Xt16 = nullptr;   // batch inputs [cap][kLIn], [kLIn][cap]
    float *Z[4] = {};                    // pre-activations [cap][d[l+1]]
    __half *A16[3] = {}, *At16[3] = {};  // hidden activations [cap][256], [256][cap]
    __half *dZ16[4] = {}, *dZt16[4] = {};    // output gradients; dZt16[3] is [128][cap], rows >= 64 zero
    float *dA = nullptr;                 // [cap][256]
    float *Y = nullptr;                  // targets [cap][kLOut]
    float *Wlin = nullptr;               // linear skip, transposed: [kLIn][kLOut] fp32 (y = Wlin x + out_scale * network(x))
    float out_scale = 1.0f;              // the network's output scale (RMS of what the skip leaves)
    float *loss_part = nullptr;          // per-block loss partials
    float *work = nullptr;               // split-K partials
    int work_floats = 0;
    int *d_err = nullptr;
    int step = 0;                        // Adam steps taken
    CUtensorMap mX, mXt, mA[3], mAt[3], mW[4], mWt[4], mdZ[4], mdZt[4];
    bool maps = false;
};

// Allocates (cudaMalloc) the buffers for `cap` rows, initialises the weights
// (seeded, scaled uniform) and encodes the tensor maps.
cudaError_t mlp_create(Mlp &n, int cap, uint64_t seed, void *encode_fn);
void mlp_destroy(Mlp &n);
// Host FP32 weights in/out ([out][in] per layer, concatenated).
cudaError_t mlp_set_weights(Mlp &n, const float *h_w, cudaStream_t s);
cudaError_t mlp_get_weights(const Mlp &n, float *h_w, cudaStream_t s);
long long mlp_weight_count();

// Forward pass over rows [0, rows) of X16 (rows a multiple of 128); the
// output is Z[3] ([rows][kLOut] fp32).  `train` also writes the transposed
// activations the weight gradients need.
cudaError_t mlp_forward(Mlp &n, int rows, bool train, int smem_optin, int sms, cudaStream_t s);
// Loss and gradients for targets Y (after mlp_forward(train)); G[l] holds
// dLoss/dW scaled by kLGradScale * rows.  Loss partials in loss_part.
cudaError_t mlp_backward(Mlp &n, int rows, int smem_optin, int sms, cudaStream_t s);
// One Adam step from G (t = ++step).
cudaError_t mlp_adam(Mlp &n, int rows, float lr, cudaStream_t s);
// Sum of the loss partials of the last backward pass, in a fixed order.
cudaError_t mlp_loss(const Mlp &n, int rows, float *h_loss, cudaStream_t s);
// fp32 rows [rows][kLIn] (device) -> X16 and Xt16.
cudaError_t mlp_load_rows(Mlp &n, const float *X, const float *Y, int rows, cudaStream_t s);
// fp16 rows gathered by index from a data set: X16/Xt16/Y of the batch.
cudaError_t mlp_gather(Mlp &n, const __half *Xall, const float *Yall, const int *idx, int rows, cudaStream_t s);

// The linear skip: out[r][o] = scale * (sign * sum_i WlinT[i][o] X[r][i] + add[r][o]),
// fp32 rows X [rows][kLIn] (add optional); the map is stored transposed.
cudaError_t linear_apply(const float *Wlin, const float *X, int rows, const float *add, float sign, float *out,
                         cudaStream_t s, float scale = 1.0f);
// Zero the last layer (the network then starts as the zero function).
cudaError_t mlp_zero_last(Mlp &n, cudaStream_t s);
// Normal equations of the linear skip in FP64: G = X^T X [kLIn][kLIn], B = X^T Y [kLIn][kLOut].
cudaError_t linear_normal(const float *X, const float *Y, int rows, double *G, double *B, cudaStream_t s);

}  // namespace rp
