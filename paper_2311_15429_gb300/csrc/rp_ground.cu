// Small elementwise kernels of the step bookkeeping.
//
//   k_ground_delta: the ground-state split of Eqs. 9-12 -- with the first
//                   sample S(0) taken as the ground state, the histories hold
//                   Delta S = S - S(0): Delta S of one domain's pushed slice
//                   (rho and J at their own pointers) into the library's
//                   [4][N] scratch;
//   k_step_advance: graph replay -- the device step counter, +1 per replay.
#include <cuda_runtime.h>

#include <algorithm>

#include "rp_internal.h"

namespace rp {

namespace {

constexpr int kGroundThreads = 256;

__global__ void __launch_bounds__(kGroundThreads)
    k_ground_delta(const float *__restrict__ rho, const float *__restrict__ J, const float *__restrict__ ground,
                   float *__restrict__ delta, long long N)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < 4 * N;
         i += (long long)gridDim.x * blockDim.x) {
        const float s = i < N ? __ldg(rho + i) : __ldg(J + (i - N));
        delta[i] = s - __ldg(ground + i);
    }
}

int grid_for(long long n, int sms)
{
    return (int)std::max<long long>(1, std::min<long long>((n + kGroundThreads - 1) / kGroundThreads,
                                                           8LL * std::max(sms, 1)));
}

// Graph replay: the step the replayed kernels read.
__global__ void k_step_advance(long long *d_step) { *d_step += 1; }

}  // namespace

cudaError_t launch_step_advance(long long *d_step, cudaStream_t s)
{
    k_step_advance<<<1, 1, 0, s>>>(d_step);
    return cudaGetLastError();
}

cudaError_t launch_ground_delta(const float *rho, const float *J, const float *ground, float *delta, long long N,
                                int sms, cudaStream_t s)
{
    if (N <= 0) return cudaSuccess;
    k_ground_delta<<<grid_for(4 * N, sms), kGroundThreads, 0, s>>>(rho, J, ground, delta, N);
    return cudaGetLastError();
}

}  // namespace rp
