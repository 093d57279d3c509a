// The fields of App. B from the potentials on one domain's grid:
//
//   E = -grad phi - (1/c) dA/dt,    B = curl A        (atomic units)
//
// Space derivatives: second-order central differences, second-order
// one-sided ones on the grid faces.  Time derivative: the second-order
// backward difference (3 A_l - 4 A_{l-1} + A_{l-2}) / (2 dt), or the
// first-order one (A_l - A_{l-1}) / dt without A_{l-2}.  One thread per node;
// neighbours come through L1.
#include <cuda_runtime.h>

#include "rp_internal.h"

namespace rp {

namespace {

constexpr int kFieldThreads = 256;

// d f / d(axis) at index i of n along a stride s, times 1/(2h) by the caller.
__device__ __forceinline__ float diff2(const float *__restrict__ f, long long at, int i, int n, long long s)
{
    if (i == 0) return -3.0f * __ldg(f + at) + 4.0f * __ldg(f + at + s) - __ldg(f + at + 2 * s);
    if (i == n - 1) return 3.0f * __ldg(f + at) - 4.0f * __ldg(f + at - s) + __ldg(f + at - 2 * s);
    return __ldg(f + at + s) - __ldg(f + at - s);
}

__global__ void __launch_bounds__(kFieldThreads)
    k_fields(int nx, int ny, int nz, float inv_2h, float inv_c, float inv_dt, const float *__restrict__ phi,
             const float *__restrict__ A, const float *__restrict__ A1, const float *__restrict__ A2,
             float *__restrict__ E, float *__restrict__ B)
{
    const long long N = (long long)nx * ny * nz;
    const long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (k >= N) return;
    const int x = (int)(k % nx), y = (int)((k / nx) % ny), z = (int)(k / ((long long)nx * ny));
    const long long sx = 1, sy = nx, sz = (long long)nx * ny;
    // grad phi
    const float gx = diff2(phi, k, x, nx, sx) * inv_2h;
    const float gy = diff2(phi, k, y, ny, sy) * inv_2h;
    const float gz = diff2(phi, k, z, nz, sz) * inv_2h;
    // dA/dt per component
    float dt3[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float a0 = __ldg(A + a * N + k), a1 = __ldg(A1 + a * N + k);
        dt3[a] = A2 ? (3.0f * a0 - 4.0f * a1 + __ldg(A2 + a * N + k)) * (0.5f * inv_dt) : (a0 - a1) * inv_dt;
    }
    E[k] = -gx - inv_c * dt3[0];
    E[N + k] = -gy - inv_c * dt3[1];
    E[2 * N + k] = -gz - inv_c * dt3[2];
    if (B) {
        const float *Ax = A, *Ay = A + N, *Az = A + 2 * N;
        const float dyAz = diff2(Az, k, y, ny, sy), dzAy = diff2(Ay, k, z, nz, sz);
        const float dzAx = diff2(Ax, k, z, nz, sz), dxAz = diff2(Az, k, x, nx, sx);
        const float dxAy = diff2(Ay, k, x, nx, sx), dyAx = diff2(Ax, k, y, ny, sy);
        B[k] = (dyAz - dzAy) * inv_2h;
        B[N + k] = (dzAx - dxAz) * inv_2h;
        B[2 * N + k] = (dxAy - dyAx) * inv_2h;
    }
}

}  // namespace

cudaError_t launch_fields(int nx, int ny, int nz, double h, double c, double dt, const float *phi, const float *A,
                          const float *A1, const float *A2, float *E, float *B, cudaStream_t s)
{
    const long long N = (long long)nx * ny * nz;
    if (N <= 0) return cudaSuccess;
    const int blocks = (int)((N + kFieldThreads - 1) / kFieldThreads);
    k_fields<<<blocks, kFieldThreads, 0, s>>>(nx, ny, nz, (float)(0.5 / h), (float)(1.0 / c), (float)(1.0 / dt),
                                              phi, A, A1, A2, E, B);
    return cudaGetLastError();
}

}  // namespace rp
