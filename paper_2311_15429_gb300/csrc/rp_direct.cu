// Direct retarded sum (the plain path of every pair in RP_MODE_DIRECT, and
// of pairs of unequal spacing in RP_MODE_FFT):
//
//   P(r_k, l) += sum_{k' in source} h_s^3 S(k', l - tau) / R,   tau = R/(c dt),
//   S(l - tau) = (1 - w) S_{l-m} + w S_{l-m-1},  m = floor(tau), w = tau - m
//
// (Eq. 8 with the hat interpolation of Eq. 7; at R = 0 of the self pair the
// cell-averaged weight C h^2 at lag 0).  One thread per target node; a block
// stages kDirTile source nodes with their samples for the pair's lag window
// in shared memory; each of the four sums is Kahan-compensated in FP32.
#include <cuda_runtime.h>

#include "rp_internal.h"

namespace rp {

namespace {

constexpr int kDirThreads = 128;
constexpr int kDirTile = 64;

__device__ __forceinline__ void kahan_add(float &sum, float &comp, float x)
{
    const float y = x - comp;
    const float t = sum + y;
    comp = (t - sum) - y;
    sum = t;
}

__global__ void __launch_bounds__(kDirThreads) k_direct(const DirectTarget *__restrict__ tgts, int ntgt,
                                                          const DirectPair *__restrict__ pairs, OutPtrs out,
                                                          long long step, int clamp, float inv_cdt, float inv_c)
{
    extern __shared__ float4 smem_f4[];
    float *sm = reinterpret_cast<float *>(smem_f4);
    const int b = blockIdx.x;
    int lo = 0, hi = ntgt;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (tgts[mid].block0 <= b) lo = mid; else hi = mid;
    }
    const DirectTarget T = tgts[lo];
    if (step < 0) step = *T.d_step;   // graph replay: the step from the device counter
    const long long k = (long long)(b - T.block0) * kDirThreads + threadIdx.x;
    const bool valid = k < T.n;
    const int ix = (int)(k % T.nx), iy = (int)((k / T.nx) % T.ny), iz = (int)(k / ((long long)T.nx * T.ny));

    float sum[4] = {0.f, 0.f, 0.f, 0.f}, comp[4] = {0.f, 0.f, 0.f, 0.f};

    float *sx = sm, *sy = sx + kDirTile, *sz = sy + kDirTile;
    float *S = sz + kDirTile;   // [nlag][4][kDirTile]

    for (int p = T.p0; p < T.p1; ++p) {
        const DirectPair P = pairs[p];
        // target node relative to the source origin, once in FP64
        const float rx = (float)(P.dx + T.ht * ix), ry = (float)(P.dy + T.ht * iy),
                    rz = (float)(P.dz + T.ht * iz);
        for (long long j0 = 0; j0 < P.n_s; j0 += kDirTile) {
            const int cnt = (int)min((long long)kDirTile, P.n_s - j0);
            __syncthreads();
            for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
                const long long q = j0 + i;
                sx[i] = P.hs * (float)(q % P.nx_s);
                sy[i] = P.hs * (float)((q / P.nx_s) % P.ny_s);
                sz[i] = P.hs * (float)(q / ((long long)P.nx_s * P.ny_s));
            }
            for (int i = threadIdx.x; i < P.nlag * 4 * kDirTile; i += blockDim.x) {
                const int jj = i % kDirTile, fl = i / kDirTile;
                const int f = fl & 3, li = fl >> 2;
                float v = 0.0f;
                if (jj < cnt) {
                    long long j = step - (P.lag_lo + li);
                    if (clamp && j < 0) j = 0;
                    v = P.raw[((j % P.depth) * 4 + f) * P.n_s + j0 + jj];
                }
                S[i] = v;
            }
            __syncthreads();
            if (!valid) continue;
            for (int jj = 0; jj < cnt; ++jj) {
                const float dx = rx - sx[jj], dy = ry - sy[jj], dz = rz - sz[jj];
                const float R2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                if (P.is_self && j0 + jj == k) {
#pragma unroll
                    for (int f = 0; f < 4; ++f) kahan_add(sum[f], comp[f], P.self_w * S[f * kDirTile + jj]);
                    continue;
                }
                const float inv = rsqrtf(R2);
                const float tau = R2 * inv * inv_cdt;
                const float m = floorf(tau);
                const float w = tau - m;
                int li = (int)m - P.lag_lo;
                li = max(0, min(li, P.nlag - 2));
                const float a = P.vol * inv;
                const float *s0 = S + (li * 4) * kDirTile + jj;
                const float *s1 = s0 + 4 * kDirTile;
#pragma unroll
                for (int f = 0; f < 4; ++f) {
                    const float x0 = s0[f * kDirTile], x1 = s1[f * kDirTile];
                    kahan_add(sum[f], comp[f], a * fmaf(w, x1 - x0, x0));
                }
            }
        }
    }
    if (!valid) return;
    const long long N = T.n;
#pragma unroll
    for (int f = 0; f < 4; ++f) {
        float *o = f == 0 ? out.phi[T.dom] + k : out.A[T.dom] + (long long)(f - 1) * N + k;
        float v = sum[f] - comp[f];
        if (f > 0) v *= inv_c;
        if (T.accumulate) v += *o;
        *o = v;
    }
}

}  // namespace

size_t smem_direct(int max_nlag) { return sizeof(float) * (size_t)kDirTile * (3 + 4 * (size_t)max_nlag); }

int direct_blocks(long long n) { return (int)((n + kDirThreads - 1) / kDirThreads); }

cudaError_t open_direct_smem_limit(int max_optin)
{
    return cudaFuncSetAttribute(k_direct, cudaFuncAttributeMaxDynamicSharedMemorySize, max_optin);
}

cudaError_t launch_direct(const DirectTarget *d_tgts, int ntgt, const DirectPair *d_pairs, const OutPtrs &out,
                          int nblocks, size_t smem, long long step, int clamp, float inv_cdt, float inv_c,
                          cudaStream_t s)
{
    if (nblocks <= 0) return cudaSuccess;
    k_direct<<<nblocks, kDirThreads, smem, s>>>(d_tgts, ntgt, d_pairs, out, step, clamp, inv_cdt, inv_c);
    return cudaGetLastError();
}

}  // namespace rp
