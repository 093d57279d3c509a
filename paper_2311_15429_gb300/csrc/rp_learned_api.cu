// C-ABI entry points that run the learned far field's network on its own:
// its layer sizes, one forward pass, and one loss + gradient evaluation.
// They exist so that the network's kernels can be checked against a plain
// CPU implementation of the same network.
#include <cstring>
#include <vector>

#include "rp.h"
#include "rp_learned.h"
#include "rp_learned_train.h"

namespace rp {
namespace {

void *tensor_map_encoder()
{
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return fn;
}

// A network for `rows` rows on `device` with the given host weights.
rp_status open_net(Mlp &n, const float *h_w, int rows, int device, int *optin, int *sms)
{
    if (cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        return RP_ERR_CUDA;
    }
    void *enc = tensor_map_encoder();
    if (!enc) return RP_ERR_CUDA;
    if (cudaDeviceGetAttribute(optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) != cudaSuccess ||
        cudaDeviceGetAttribute(sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
        mlp_create(n, rows, 1, enc) != cudaSuccess || mlp_set_weights(n, h_w, nullptr) != cudaSuccess) {
        cudaGetLastError();
        mlp_destroy(n);
        return RP_ERR_CUDA;
    }
    return RP_OK;
}

rp_status finish(Mlp &n, cudaError_t e)
{
    if (!e) e = cudaDeviceSynchronize();
    int flag = 0;
    if (!e) e = cudaMemcpy(&flag, n.d_err, sizeof(int), cudaMemcpyDeviceToHost);
    mlp_destroy(n);
    if (e) {
        cudaGetLastError();
        return RP_ERR_CUDA;
    }
    return flag ? RP_ERR_TIMEOUT : RP_OK;
}

}  // namespace
}  // namespace rp

using namespace rp;

extern "C" {

int rp_mlp_layout(int *dims)
{
    if (dims) {
        const int d[5] = {kLIn, kLHid, kLHid, kLHid, kLOut};
        std::memcpy(dims, d, sizeof(d));
    }
    return (int)mlp_weight_count();
}

rp_status rp_mlp_forward(const float *h_w, const float *h_x, int rows, float *h_y, int device)
{
    if (!h_w || !h_x || !h_y || rows <= 0 || rows % 128) return RP_ERR_ARG;
    Mlp n;
    int optin = 0, sms = 0;
    rp_status st = open_net(n, h_w, rows, device, &optin, &sms);
    if (st) return st;
    float *dx = nullptr;
    cudaError_t e = cudaMalloc(&dx, (size_t)rows * kLIn * sizeof(float));
    if (!e) e = cudaMemcpy(dx, h_x, (size_t)rows * kLIn * sizeof(float), cudaMemcpyHostToDevice);
    if (!e) e = mlp_load_rows(n, dx, nullptr, rows, nullptr);
    if (!e) e = mlp_forward(n, rows, false, optin, sms, nullptr);
    if (!e) e = cudaMemcpy(h_y, n.Z[3], (size_t)rows * kLOut * sizeof(float), cudaMemcpyDeviceToHost);
    cudaFree(dx);
    return finish(n, e);
}

rp_status rp_mlp_grad(const float *h_w, const float *h_x, const float *h_t, int rows, float *h_g, float *h_loss,
                      int device)
{
    if (!h_w || !h_x || !h_t || !h_g || !h_loss || rows <= 0 || rows % 128) return RP_ERR_ARG;
    Mlp n;
    int optin = 0, sms = 0;
    rp_status st = open_net(n, h_w, rows, device, &optin, &sms);
    if (st) return st;
    float *dx = nullptr, *dt = nullptr;
    cudaError_t e = cudaMalloc(&dx, (size_t)rows * kLIn * sizeof(float));
    if (!e) e = cudaMalloc(&dt, (size_t)rows * kLOut * sizeof(float));
    if (!e) e = cudaMemcpy(dx, h_x, (size_t)rows * kLIn * sizeof(float), cudaMemcpyHostToDevice);
    if (!e) e = cudaMemcpy(dt, h_t, (size_t)rows * kLOut * sizeof(float), cudaMemcpyHostToDevice);
    if (!e) e = mlp_load_rows(n, dx, dt, rows, nullptr);
    if (!e) e = mlp_forward(n, rows, true, optin, sms, nullptr);
    if (!e) e = mlp_backward(n, rows, optin, sms, nullptr);
    if (!e) e = mlp_loss(n, rows, h_loss, nullptr);
    if (!e) {
        const int d[5] = {kLIn, kLHid, kLHid, kLHid, kLOut};
        const float scale = 1.0f / (kLGradScale * (float)rows);
        size_t o = 0;
        for (int l = 0; l < 4 && !e; ++l) {
            const size_t w = (size_t)d[l] * d[l + 1];
            e = cudaMemcpy(h_g + o, n.G[l], w * sizeof(float), cudaMemcpyDeviceToHost);
            for (size_t i = 0; i < w; ++i) h_g[o + i] *= scale;
            o += w;
        }
    }
    cudaFree(dx);
    cudaFree(dt);
    return finish(n, e);
}

int rp_learned_desc_size() { return kLDesc; }

rp_status rp_learned_dataset(const int n_s[3], double h_s, const double Lt[3], const double dir[3], double Rc,
                             unsigned long long seed, int histories, int samples, double c, double dt, float *h_x,
                             float *h_y, double *h_desc, int device)
{
    if (!n_s || !Lt || !dir || !h_x || !h_y || !h_desc || histories <= 0 || samples <= 0 || !(h_s > 0.0) ||
        !(c > 0.0) || !(dt > 0.0) || !(Rc > 0.0))
        return RP_ERR_ARG;
    for (int k = 0; k < 3; ++k)
        if (n_s[k] < 2 || !(Lt[k] >= 0.0)) return RP_ERR_ARG;
    LGeom g{};
    for (int k = 0; k < 3; ++k) {
        g.n_s[k] = n_s[k];
        g.Lt[k] = Lt[k];
        g.dir[k] = dir[k];
    }
    g.h_s = h_s;
    g.Rc = Rc;
    g.random = false;
    if (samples > max_samples(g, c * dt)) return RP_ERR_ARG;
    if (cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        return RP_ERR_CUDA;
    }
    const size_t rows = (size_t)histories * samples * 4;
    __half *X = nullptr;
    float *Y = nullptr;
    std::vector<__half> hx(rows * kLIn);
    cudaError_t e = cudaMalloc(&X, rows * kLIn * sizeof(__half));
    if (!e) e = cudaMalloc(&Y, rows * kLOut * sizeof(float));
    if (!e) e = learned_dataset(g, seed, histories, samples, c, dt, X, nullptr, Y, nullptr, h_desc);
    if (!e) e = cudaMemcpy(hx.data(), X, rows * kLIn * sizeof(__half), cudaMemcpyDeviceToHost);
    if (!e) e = cudaMemcpy(h_y, Y, rows * kLOut * sizeof(float), cudaMemcpyDeviceToHost);
    if (!e)
        for (size_t i = 0; i < hx.size(); ++i) h_x[i] = __half2float(hx[i]);
    cudaFree(X);
    cudaFree(Y);
    if (e) {
        cudaGetLastError();
        return RP_ERR_CUDA;
    }
    return RP_OK;
}

}  // extern "C"
