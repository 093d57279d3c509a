// The learned far field's network: a bias-free MLP
//
//   x (kLIn) -> W1 -> leaky -> W2 -> leaky -> W3 -> leaky -> W4 -> y (kLOut)
//
// with fp16 weights and activations as tensor-core operands and fp32
// accumulation (tcgen05 GEMMs of rp_gemm_tc.cu, kind::f16 with fp16 A and
// B), trained by its own backward pass and Adam kernels.  The loss is
// (1 / 2B) sum over the B rows of |y - target|^2.
//
// Layouts: weights [out][in]; activations [rows][width] for the forward
// GEMMs (A operand) and transposed [width][rows] for the weight gradients
// dW = dZ^T A (both operands K-major with K = rows).  The output gradients
// are carried in fp16 scaled by kLGradScale (with the loss's 1/B left out);
// Adam divides both back out in fp32.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "rp_learned.h"

namespace rp {

namespace {

constexpr int kDims[5] = {kLIn, kLHid, kLHid, kLHid, kLOut};

// ---------------------------------------------------------------- elementwise kernels

// A = leaky(Z) in fp16, and (if At) its transpose; a block is a 32 x 32 tile.
__global__ void k_act_fwd(const float *__restrict__ Z, __half *__restrict__ A, __half *__restrict__ At, int n, int ldt)
{
    __shared__ __half t[32][33];
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const size_t o = (size_t)(r0 + i) * n + c0 + threadIdx.x;
        const float z = Z[o];
        const __half h = __float2half_rn(z >= 0.0f ? z : kLLeak * z);
        A[o] = h;
        t[i][threadIdx.x] = h;
    }
    if (!At) return;
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y)
        At[(size_t)(c0 + i) * ldt + r0 + threadIdx.x] = t[threadIdx.x][i];
}

// dZ = dA * leaky'(Z) in fp16, and its transpose.
__global__ void k_act_bwd(const float *__restrict__ dA, const float *__restrict__ Z, __half *__restrict__ dZ,
                          __half *__restrict__ dZt, int n, int ldt)
{
    __shared__ __half t[32][33];
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const size_t o = (size_t)(r0 + i) * n + c0 + threadIdx.x;
        const float g = dA[o] * (Z[o] >= 0.0f ? 1.0f : kLLeak);
        const __half h = __float2half_rn(g);
        dZ[o] = h;
        t[i][threadIdx.x] = h;
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y)
        dZt[(size_t)(c0 + i) * ldt + r0 + threadIdx.x] = t[threadIdx.x][i];
}

// Output layer: r = y - target; dZ = kLGradScale * r (fp16, and transposed);
// one loss partial (sum of r^2, fixed-order tree) per block.
__global__ void k_out_loss(const float *__restrict__ Z, const float *__restrict__ Y, __half *__restrict__ dZ,
                           __half *__restrict__ dZt, int ldt, float *__restrict__ part)
{
    __shared__ __half t[32][33];
    __shared__ float red[256];
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    float acc = 0.0f;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const size_t o = (size_t)(r0 + i) * kLOut + c0 + threadIdx.x;
        const float r = Z[o] - Y[o];
        acc = fmaf(r, r, acc);
        const __half h = __float2half_rn(kLGradScale * r);
        dZ[o] = h;
        t[i][threadIdx.x] = h;
    }
    const int tid = threadIdx.y * 32 + threadIdx.x;
    red[tid] = acc;
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y)
        dZt[(size_t)(c0 + i) * ldt + r0 + threadIdx.x] = t[threadIdx.x][i];
    for (int w = 128; w > 0; w >>= 1) {
        if (tid < w) red[tid] += red[tid + w];
        __syncthreads();
    }
    if (tid == 0) part[blockIdx.y * gridDim.x + blockIdx.x] = red[0];
}

__global__ void k_loss_sum(const float *__restrict__ part, int n, float *out)
{
    if (threadIdx.x || blockIdx.x) return;
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += part[i];
    out[0] = (float)s;
}

// Adam (Kingma and Ba): g = G * inv_scale; m, v moments; bias-corrected step.
__global__ void k_adam(float *__restrict__ W, const float *__restrict__ G, float *__restrict__ m,
                       float *__restrict__ v, __half *__restrict__ W16, __half *__restrict__ Wt16, int n_out, int n_in,
                       float lr, float b1, float b2, float eps, float bc1, float bc2, float inv_scale)
{
    const int total = n_out * n_in;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        const float g = G[i] * inv_scale;
        const float mi = b1 * m[i] + (1.0f - b1) * g;
        const float vi = b2 * v[i] + (1.0f - b2) * g * g;
        m[i] = mi;
        v[i] = vi;
        const float w = W[i] - lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
        W[i] = w;
        const __half h = __float2half_rn(w);
        W16[i] = h;
        if (Wt16) Wt16[(size_t)(i % n_in) * n_out + i / n_in] = h;
    }
}

__global__ void k_weights_to_half(const float *__restrict__ W, __half *__restrict__ W16, __half *__restrict__ Wt16,
                                  int n_out, int n_in)
{
    const int total = n_out * n_in;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        const __half h = __float2half_rn(W[i]);
        W16[i] = h;
        if (Wt16) Wt16[(size_t)(i % n_in) * n_out + i / n_in] = h;
    }
}

// fp32 rows -> X16 and transposed Xt16 (32 x 32 tiles); Y copied.
__global__ void k_rows_to_half(const float *__restrict__ X, __half *__restrict__ X16, __half *__restrict__ Xt16,
                               int ldt)
{
    __shared__ __half t[32][33];
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const size_t o = (size_t)(r0 + i) * kLIn + c0 + threadIdx.x;
        const __half h = __float2half_rn(X[o]);
        X16[o] = h;
        t[i][threadIdx.x] = h;
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y)
        Xt16[(size_t)(c0 + i) * ldt + r0 + threadIdx.x] = t[threadIdx.x][i];
}

// Batch rows gathered from a data set: X16 / Xt16 (tiles) and Y.
__global__ void k_gather(const __half *__restrict__ Xall, const float *__restrict__ Yall, const int *__restrict__ idx,
                         __half *__restrict__ X16, __half *__restrict__ Xt16, float *__restrict__ Y, int ldt)
{
    __shared__ __half t[32][33];
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int src = idx[r0 + i];
        const __half h = Xall[(size_t)src * kLIn + c0 + threadIdx.x];
        X16[(size_t)(r0 + i) * kLIn + c0 + threadIdx.x] = h;
        t[i][threadIdx.x] = h;
        if (c0 < kLOut) Y[(size_t)(r0 + i) * kLOut + c0 + threadIdx.x] = Yall[(size_t)src * kLOut + c0 + threadIdx.x];
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y)
        Xt16[(size_t)(c0 + i) * ldt + r0 + threadIdx.x] = t[threadIdx.x][i];
}

// out[r][o] = scale (sign * sum_i WT[i][o] X[r][i] + add): a block takes 8
// rows into shared memory; thread (q, o) sums the i of k-slice q for all 8
// rows (WT[i][o] read once, coalesced across o), and the 4 slices are added
// in a fixed order.
constexpr int kLinRows = 8, kLinSlices = 4;
__global__ void __launch_bounds__(kLinSlices * kLOut) k_linear(const float *__restrict__ WT,
                                                               const float *__restrict__ X, int rows,
                                                               const float *__restrict__ add, float sign,
                                                               float *__restrict__ out, float scale)
{
    __shared__ float xs[kLinRows][kLIn];
    __shared__ float part[kLinSlices][kLinRows][kLOut];
    const int r0 = blockIdx.x * kLinRows;
    for (int i = threadIdx.x; i < kLinRows * kLIn; i += blockDim.x) {
        const int rr = r0 + i / kLIn;
        xs[i / kLIn][i % kLIn] = rr < rows ? X[(size_t)rr * kLIn + i % kLIn] : 0.0f;
    }
    __syncthreads();
    const int q = threadIdx.x / kLOut, o = threadIdx.x % kLOut;
    constexpr int per = kLIn / kLinSlices;
    float acc[kLinRows] = {};
#pragma unroll 4
    for (int i = q * per; i < (q + 1) * per; ++i) {
        const float w = __ldg(WT + (size_t)i * kLOut + o);
#pragma unroll
        for (int rr = 0; rr < kLinRows; ++rr) acc[rr] = fmaf(w, xs[rr][i], acc[rr]);
    }
#pragma unroll
    for (int rr = 0; rr < kLinRows; ++rr) part[q][rr][o] = acc[rr];
    __syncthreads();
    for (int t = threadIdx.x; t < kLinRows * kLOut; t += blockDim.x) {
        const int rr = t / kLOut, oo = t % kLOut;
        if (r0 + rr >= rows) continue;
        float a = 0.0f;
        for (int k = 0; k < kLinSlices; ++k) a += part[k][rr][oo];
        const size_t oi = (size_t)(r0 + rr) * kLOut + oo;
        out[oi] = scale * (sign * a + (add ? add[oi] : 0.0f));
    }
}

// G[i][j] = sum_r X[r][i] X[r][j] and B[i][o] = sum_r X[r][i] Y[r][o] in FP64;
// a block owns a 32 x 32 tile of [G | B] and sums the rows in a fixed order.
__global__ void __launch_bounds__(256) k_normal(const float *__restrict__ X, const float *__restrict__ Y, int rows,
                                                double *__restrict__ G, double *__restrict__ B)
{
    __shared__ float xa[32][33], xb[32][33];
    const int i0 = blockIdx.y * 32, j0 = blockIdx.x * 32;       // columns of [X | Y]
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;      // 32 x 8
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    auto col = [&](int r, int j) -> float {
        return j < kLIn ? X[(size_t)r * kLIn + j] : Y[(size_t)r * kLOut + (j - kLIn)];
    };
    for (int r0 = 0; r0 < rows; r0 += 32) {
        for (int k = ty; k < 32; k += 8) {
            const int r = r0 + k;
            xa[k][tx] = r < rows ? X[(size_t)r * kLIn + i0 + tx] : 0.0f;
            xb[k][tx] = r < rows ? col(r, j0 + tx) : 0.0f;
        }
        __syncthreads();
        for (int q = 0; q < 4; ++q) {
            const int ii = ty + 8 * q;
            double s = 0.0;
            for (int k = 0; k < 32; ++k) s += (double)xa[k][ii] * (double)xb[k][tx];
            acc[q] += s;
        }
        __syncthreads();
    }
    for (int q = 0; q < 4; ++q) {
        const int i = i0 + ty + 8 * q, j = j0 + tx;
        if (j < kLIn) G[(size_t)i * kLIn + j] = acc[q];
        else B[(size_t)i * kLOut + (j - kLIn)] = acc[q];
    }
}

// splitmix64: the seeded weight initialisation
uint64_t splitmix(uint64_t &x)
{
    uint64_t z = (x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

template <class T>
cudaError_t alloc(T **p, size_t n)
{
    return cudaMalloc(reinterpret_cast<void **>(p), std::max<size_t>(n, 1) * sizeof(T));
}

cudaError_t gemm(const CUtensorMap &a, const CUtensorMap &b, float *D, int M, int N, int K, Mlp &n, int optin, int sms,
                 cudaStream_t s, bool split)
{
    int splits = 1;
    if (split) {
        splits = std::max(1, gemm_splits(M, K, 0, sms, 2) / std::max(1, N / gemm_tile_n(N)));
        while (splits > 1 && (long long)splits * M * N > n.work_floats) --splits;
    }
    return launch_gemm_bf16_tn(a, b, D, M, N, K, N, optin, n.d_err, s, splits, n.work, 0, 1);
}

}  // namespace

long long mlp_weight_count()
{
    long long c = 0;
    for (int l = 0; l < 4; ++l) c += (long long)kDims[l] * kDims[l + 1];
    return c;
}

cudaError_t mlp_create(Mlp &n, int cap, uint64_t seed, void *enc)
{
    if (cap <= 0 || cap % 128) return cudaErrorInvalidValue;
    n.cap = cap;
    cudaError_t e;
#define RP_TRY(x) \
    if ((e = (x))) return e;
    for (int l = 0; l < 4; ++l) {
        const size_t w = (size_t)kDims[l] * kDims[l + 1];
        RP_TRY(alloc(&n.W[l], w));
        RP_TRY(alloc(&n.G[l], l == 3 ? (size_t)128 * kDims[3] : w));
        RP_TRY(alloc(&n.m[l], w));
        RP_TRY(alloc(&n.v[l], w));
        RP_TRY(alloc(&n.W16[l], w));
        if (l > 0) RP_TRY(alloc(&n.Wt16[l], w));
        RP_TRY(alloc(&n.Z[l], (size_t)cap * kDims[l + 1]));
        RP_TRY(alloc(&n.dZ16[l], (size_t)cap * kDims[l + 1]));
        RP_TRY(alloc(&n.dZt16[l], (size_t)(l == 3 ? 128 : kDims[l + 1]) * cap));
        RP_TRY(cudaMemset(n.m[l], 0, w * sizeof(float)));
        RP_TRY(cudaMemset(n.v[l], 0, w * sizeof(float)));
    }
    RP_TRY(cudaMemset(n.dZt16[3], 0, (size_t)128 * cap * sizeof(__half)));
    for (int l = 0; l < 3; ++l) {
        RP_TRY(alloc(&n.A16[l], (size_t)cap * kLHid));
        RP_TRY(alloc(&n.At16[l], (size_t)cap * kLHid));
    }
    RP_TRY(alloc(&n.X16, (size_t)cap * kLIn));
    RP_TRY(alloc(&n.Xt16, (size_t)cap * kLIn));
    RP_TRY(alloc(&n.dA, (size_t)cap * kLHid));
    RP_TRY(alloc(&n.Y, (size_t)cap * kLOut));
    RP_TRY(alloc(&n.Wlin, (size_t)kLOut * kLIn));
    RP_TRY(cudaMemset(n.Wlin, 0, (size_t)kLOut * kLIn * sizeof(float)));
    RP_TRY(alloc(&n.loss_part, (size_t)cap / 32 * (kLOut / 32)));
    n.work_floats = 76 * 256 * 320;
    RP_TRY(alloc(&n.work, (size_t)n.work_floats));
    RP_TRY(alloc(&n.d_err, 1));
    RP_TRY(cudaMemset(n.d_err, 0, sizeof(int)));
    // seeded uniform weights, bound sqrt(6 / ((1 + a^2) fan_in)) (He et al. for the leaky slope a)
    std::vector<float> h(mlp_weight_count());
    uint64_t st = seed;
    size_t o = 0;
    for (int l = 0; l < 4; ++l) {
        const double bound = std::sqrt(6.0 / ((1.0 + (double)kLLeak * kLLeak) * kDims[l]));
        for (int i = 0; i < kDims[l] * kDims[l + 1]; ++i) {
            const double u = (double)(splitmix(st) >> 11) * (1.0 / 9007199254740992.0);
            h[o++] = (float)((2.0 * u - 1.0) * bound);
        }
    }
    RP_TRY(mlp_set_weights(n, h.data(), nullptr));
    RP_TRY(cudaDeviceSynchronize());
    // tensor maps (fp16 data; the copy engine moves 16-bit elements either way)
    bool ok = encode_bf16_rows(enc, &n.mX, n.X16, cap, kLIn, 128) &&
              encode_bf16_rows(enc, &n.mXt, n.Xt16, kLIn, cap, (uint32_t)gemm_tile_n(kLIn));
    for (int l = 0; l < 3; ++l)
        ok = ok && encode_bf16_rows(enc, &n.mA[l], n.A16[l], cap, kLHid, 128) &&
             encode_bf16_rows(enc, &n.mAt[l], n.At16[l], kLHid, cap, (uint32_t)gemm_tile_n(kLHid));
    for (int l = 0; l < 4; ++l) {
        ok = ok && encode_bf16_rows(enc, &n.mW[l], n.W16[l], kDims[l + 1], kDims[l],
                                    (uint32_t)gemm_tile_n(kDims[l + 1]));
        if (l > 0)
            ok = ok && encode_bf16_rows(enc, &n.mWt[l], n.Wt16[l], kDims[l], kDims[l + 1],
                                        (uint32_t)gemm_tile_n(kDims[l]));
        ok = ok && encode_bf16_rows(enc, &n.mdZ[l], n.dZ16[l], cap, kDims[l + 1], 128) &&
             encode_bf16_rows(enc, &n.mdZt[l], n.dZt16[l], l == 3 ? 128 : kDims[l + 1], cap, 128);
    }
#undef RP_TRY
    if (!ok) return cudaErrorInvalidValue;
    n.maps = true;
    n.step = 0;
    return cudaSuccess;
}

void mlp_destroy(Mlp &n)
{
    for (int l = 0; l < 4; ++l) {
        cudaFree(n.W[l]); cudaFree(n.G[l]); cudaFree(n.m[l]); cudaFree(n.v[l]);
        cudaFree(n.W16[l]); cudaFree(n.Wt16[l]); cudaFree(n.Z[l]); cudaFree(n.dZ16[l]); cudaFree(n.dZt16[l]);
    }
    for (int l = 0; l < 3; ++l) { cudaFree(n.A16[l]); cudaFree(n.At16[l]); }
    cudaFree(n.X16); cudaFree(n.Xt16); cudaFree(n.dA); cudaFree(n.Y); cudaFree(n.loss_part); cudaFree(n.Wlin);
    cudaFree(n.work); cudaFree(n.d_err);
    n = Mlp{};
}

cudaError_t mlp_set_weights(Mlp &n, const float *h_w, cudaStream_t s)
{
    size_t o = 0;
    for (int l = 0; l < 4; ++l) {
        const size_t w = (size_t)kDims[l] * kDims[l + 1];
        cudaError_t e = cudaMemcpyAsync(n.W[l], h_w + o, w * sizeof(float), cudaMemcpyHostToDevice, s);
        if (e) return e;
        k_weights_to_half<<<(int)((w + 255) / 256), 256, 0, s>>>(n.W[l], n.W16[l], n.Wt16[l], kDims[l + 1], kDims[l]);
        o += w;
    }
    return cudaGetLastError();
}

cudaError_t mlp_get_weights(const Mlp &n, float *h_w, cudaStream_t s)
{
    size_t o = 0;
    for (int l = 0; l < 4; ++l) {
        const size_t w = (size_t)kDims[l] * kDims[l + 1];
        cudaError_t e = cudaMemcpyAsync(h_w + o, n.W[l], w * sizeof(float), cudaMemcpyDeviceToHost, s);
        if (e) return e;
        o += w;
    }
    return cudaStreamSynchronize(s);
}

cudaError_t mlp_load_rows(Mlp &n, const float *X, const float *Y, int rows, cudaStream_t s)
{
    if (rows <= 0 || rows % 128 || rows > n.cap) return cudaErrorInvalidValue;
    k_rows_to_half<<<dim3(kLIn / 32, rows / 32), dim3(32, 8), 0, s>>>(X, n.X16, n.Xt16, n.cap);
    if (Y) {
        cudaError_t e = cudaMemcpyAsync(n.Y, Y, (size_t)rows * kLOut * sizeof(float), cudaMemcpyDeviceToDevice, s);
        if (e) return e;
    }
    return cudaGetLastError();
}

cudaError_t mlp_gather(Mlp &n, const __half *Xall, const float *Yall, const int *idx, int rows, cudaStream_t s)
{
    if (rows <= 0 || rows % 128 || rows > n.cap) return cudaErrorInvalidValue;
    k_gather<<<dim3(kLIn / 32, rows / 32), dim3(32, 8), 0, s>>>(Xall, Yall, idx, n.X16, n.Xt16, n.Y, n.cap);
    return cudaGetLastError();
}

cudaError_t linear_apply(const float *Wlin, const float *X, int rows, const float *add, float sign, float *out,
                         cudaStream_t s, float scale)
{
    if (rows <= 0) return cudaSuccess;
    k_linear<<<(rows + kLinRows - 1) / kLinRows, kLinSlices * kLOut, 0, s>>>(Wlin, X, rows, add, sign, out, scale);
    return cudaGetLastError();
}

cudaError_t mlp_zero_last(Mlp &n, cudaStream_t s)
{
    const size_t w = (size_t)kDims[3] * kDims[4];
    cudaError_t e = cudaMemsetAsync(n.W[3], 0, w * sizeof(float), s);
    if (!e) e = cudaMemsetAsync(n.W16[3], 0, w * sizeof(__half), s);
    if (!e) e = cudaMemsetAsync(n.Wt16[3], 0, w * sizeof(__half), s);
    return e;
}

cudaError_t linear_normal(const float *X, const float *Y, int rows, double *G, double *B, cudaStream_t s)
{
    k_normal<<<dim3((kLIn + kLOut) / 32, kLIn / 32), 256, 0, s>>>(X, Y, rows, G, B);
    return cudaGetLastError();
}

cudaError_t mlp_forward(Mlp &n, int rows, bool train, int optin, int sms, cudaStream_t s)
{
    if (rows <= 0 || rows % 128 || rows > n.cap) return cudaErrorInvalidValue;
    cudaError_t e;
    const CUtensorMap *in = &n.mX;
    for (int l = 0; l < 4; ++l) {
        if ((e = gemm(*in, n.mW[l], n.Z[l], rows, kDims[l + 1], kDims[l], n, optin, sms, s, false))) return e;
        if (l < 3) {
            k_act_fwd<<<dim3(kLHid / 32, rows / 32), dim3(32, 8), 0, s>>>(n.Z[l], n.A16[l], train ? n.At16[l] : nullptr,
                                                                           kLHid, n.cap);
            in = &n.mA[l];
        }
    }
    return cudaGetLastError();
}

cudaError_t mlp_backward(Mlp &n, int rows, int optin, int sms, cudaStream_t s)
{
    if (rows <= 0 || rows % 128 || rows > n.cap) return cudaErrorInvalidValue;
    cudaError_t e;
    k_out_loss<<<dim3(kLOut / 32, rows / 32), dim3(32, 8), 0, s>>>(n.Z[3], n.Y, n.dZ16[3], n.dZt16[3], n.cap,
                                                                    n.loss_part);
    for (int l = 3; l >= 0; --l) {
        // dW_l = dZ_l^T A_{l-1}  (M = out rows, padded to 128 for the last layer)
        const CUtensorMap &B = l == 0 ? n.mXt : n.mAt[l - 1];
        const int M = l == 3 ? 128 : kDims[l + 1];
        if ((e = gemm(n.mdZt[l], B, n.G[l], M, kDims[l], rows, n, optin, sms, s, true))) return e;
        if (l == 0) break;
        // dA_{l-1} = dZ_l W_l, then through the activation
        if ((e = gemm(n.mdZ[l], n.mWt[l], n.dA, rows, kDims[l], kDims[l + 1], n, optin, sms, s, false))) return e;
        k_act_bwd<<<dim3(kLHid / 32, rows / 32), dim3(32, 8), 0, s>>>(n.dA, n.Z[l - 1], n.dZ16[l - 1], n.dZt16[l - 1],
                                                                       kLHid, n.cap);
    }
    return cudaGetLastError();
}

cudaError_t mlp_adam(Mlp &n, int rows, float lr, cudaStream_t s)
{
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    ++n.step;
    const float bc1 = 1.0f - std::pow(b1, (float)n.step), bc2 = 1.0f - std::pow(b2, (float)n.step);
    const float inv = 1.0f / (kLGradScale * (float)rows);
    for (int l = 0; l < 4; ++l) {
        const int w = kDims[l] * kDims[l + 1];
        k_adam<<<std::min((w + 255) / 256, 1024), 256, 0, s>>>(n.W[l], n.G[l], n.m[l], n.v[l], n.W16[l], n.Wt16[l],
                                                                kDims[l + 1], kDims[l], lr, b1, b2, eps, bc1, bc2, inv);
    }
    return cudaGetLastError();
}

cudaError_t mlp_loss(const Mlp &n, int rows, float *h_loss, cudaStream_t s)
{
    float *d = n.work;   // scratch word (the split-K partials are dead between steps)
    k_loss_sum<<<1, 32, 0, s>>>(n.loss_part, rows / 32 * (kLOut / 32), d);
    cudaError_t e = cudaMemcpyAsync(h_loss, d, sizeof(float), cudaMemcpyDeviceToHost, s);
    if (e) return e;
    e = cudaStreamSynchronize(s);
    if (!e) *h_loss = *h_loss * 0.5f / (float)rows;
    return e;
}

}  // namespace rp
