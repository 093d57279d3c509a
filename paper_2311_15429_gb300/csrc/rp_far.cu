// Far pairs: a low-rank (interpolative) factorisation of the lag-stacked
// operator [G_lo ... G_hi] of Eq. 11, applied with the tensor-core GEMM.
//
// For a far pair (target t, source n) the retarded potential is smooth over
// the target box, so it is represented by its values at p^3 Chebyshev nodes
// x_a of the box and interpolated (tensor-product Lagrange) to the grid:
//
//   P_t(r_k, l) ~= sum_a L_a(r_k) c_t[a](l),
//   c_t[a](l)   = sum_n sum_{m = lo..hi} sum_{k'} W_{tn,m}[a][k'] S_n(k', l - m),
//   W_{tn,m}[a][k'] = h^3 T(m dt - R(x_a, r_k')/c) / R(x_a, r_k')   (Eq. 11 at the nodes).
//
// The source-side contraction runs time-batched: every `batch` pushes, the
// GEMM  Z_n = W_n X_n^T  (W_n: rows (t, m, a) x source nodes; X_n: the
// batch's slices, one row per (slice, field); both as bf16 hi/lo pairs, with
// the three products hi*hi + hi*lo + lo*hi accumulated in fp32) gives
// every node value for every (lag, slice) pair; k_far_scatter then adds
// Z[(t, m, a)][(k, f)] into the coefficient ring of target t at step
// j0 + k + m.  A far pair needs lag_lo >= batch - 1 so that step l's
// coefficients are complete when step l is evaluated.
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include "rp_internal.h"

namespace rp {

namespace {

constexpr int kFarThreads = 256;

// W rows of one source: row r has the node position (relative to the source
// origin) and the lag of the row (lag < 0: padding row).  The factor is
// computed in FP64 and stored as two bf16 planes, W = W_hi + W_lo with
// W_hi = bf16(W) and W_lo = bf16(W - W_hi) (row layout [W_hi | W_lo], each
// half `ks` wide), which carries about 16 significant bits.
__global__ void __launch_bounds__(kFarThreads) k_far_build_w(const FarRow *__restrict__ rows, int nrows, int nx,
                                                              int ny, int nz, double h, double inv_cdt, double vol,
                                                              int ks, __nv_bfloat16 *W)
{
    const long long ns = (long long)nx * ny * nz;
    const long long total = (long long)nrows * ks;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(i / ks);
        const long long q = i % ks;
        double w = 0.0;
        const FarRow fr = rows[r];
        if (fr.lag >= 0 && q < ns) {
            const int ix = (int)(q % nx), iy = (int)((q / nx) % ny), iz = (int)(q / ((long long)nx * ny));
            const double dx = fr.x - h * ix, dy = fr.y - h * iy, dz = fr.z - h * iz;
            const double R = sqrt(dx * dx + dy * dy + dz * dz);
            const double T = 1.0 - fabs((double)fr.lag - R * inv_cdt);
            if (T > 0.0) w = vol * T / R;
        }
        const __nv_bfloat16 hi = __float2bfloat16((float)w);
        const __nv_bfloat16 lo = __float2bfloat16((float)(w - (double)__bfloat162float(hi)));
        W[(long long)r * 2 * ks + q] = hi;
        W[(long long)r * 2 * ks + ks + q] = lo;
    }
}

// One slice of each far source into row block (slot) of its batch matrix X,
// split like W into [X_hi | X_lo] (the low part is exact in fp32: v - hi).
__global__ void __launch_bounds__(kFarThreads) k_far_convert(const FarSource *__restrict__ srcs, int nsrc, IoPtrs in,
                                                              int slot)
{
    const int si = blockIdx.y;
    if (si >= nsrc) return;
    const FarSource S = srcs[si];
    const float *rho = in.rho[S.dom], *J = in.J[S.dom];
    if (!rho) return;
    const long long n = S.n;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < 4 * n;
         i += (long long)gridDim.x * blockDim.x) {
        const int f = (int)(i / n);
        const long long q = i % n;
        const float v = f == 0 ? rho[q] : J[(long long)(f - 1) * n + q];
        const __nv_bfloat16 hi = __float2bfloat16(v);
        __nv_bfloat16 *row = S.X + ((long long)slot * 4 + f) * 2 * S.ks;
        row[q] = hi;
        row[S.ks + q] = __float2bfloat16(v - __bfloat162float(hi));
    }
}

// Zero the coefficient-ring slots of steps (j1 - batch + hi_t, j1 + hi_t] of
// every far target: the steps the batch ending at slice j1 reaches first.
__global__ void __launch_bounds__(kFarThreads) k_far_zero(const FarTarget *__restrict__ tgts, int ntgt,
                                                           long long j1, int batch)
{
    const int ti = blockIdx.y;
    if (ti >= ntgt) return;
    const FarTarget T = tgts[ti];
    // a target with no low-rank pairs (only learned ones) has its slot set
    // whole at evaluation and is not zeroed here
    if (T.lag_hi_max < 0) return;
    const int per = T.r * 4;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < batch * per; i += gridDim.x * blockDim.x) {
        const long long s = j1 - batch + T.lag_hi_max + 1 + i / per;
        if (s < 0) continue;   // steps before the first push receive nothing
        T.cring[(s % T.depth) * per + i % per] = 0.0f;
    }
}

// Add the GEMM result of one source into its targets' coefficient rings:
// thread (link, a, f, d) sums Z[(t, m, a)][k*4 + f] over k + m = d.
__global__ void __launch_bounds__(kFarThreads) k_far_scatter(const FarLink *__restrict__ links, int nlinks,
                                                              const float *__restrict__ Z, int ldz, long long j0,
                                                              int batch)
{
    int rem = blockIdx.x * blockDim.x + threadIdx.x;
    int li = 0;
    for (; li < nlinks; ++li) {
        const FarLink &L = links[li];
        const int cnt = L.r * 4 * (L.nlag + batch - 1);
        if (rem < cnt) break;
        rem -= cnt;
    }
    if (li >= nlinks) return;
    const FarLink L = links[li];
    const int d = rem / (L.r * 4), af = rem % (L.r * 4);
    const int a = af / 4, f = af % 4;
    float acc = 0.0f;
    for (int k = 0; k < batch; ++k) {
        const int mi = d - k;                       // lag index within the window
        if (mi < 0 || mi >= L.nlag) continue;
        acc += Z[(long long)(L.row0 + mi * L.r + a) * ldz + k * 4 + f];
    }
    const long long s = j0 + L.lag_lo + d;          // step that receives it
    float *c = L.cring + (s % L.depth) * (L.r * 4) + af;
    *c += acc;
}

// The far coefficients of step `step` interpolated onto the grid of a far
// target that has no FFT pass of its own (its inverse plane pass adds them
// otherwise): written, or added when direct pairs wrote the output first.
// One block per z-plane.
__global__ void __launch_bounds__(kFarThreads) k_far_interp(const FarTarget *__restrict__ tgts, int ntgt, OutPtrs out,
                                                             long long step, const long long *d_step, float inv_c)
{
    if (step < 0) step = *d_step;   // graph replay: the step from the device counter
    __shared__ float cz[kMaxFarPts * kMaxFarPts * 4];   // coefficients contracted over z
    int b = blockIdx.x, ti = 0;
    for (; ti < ntgt; ++ti) {
        if (b < tgts[ti].nz) break;
        b -= tgts[ti].nz;
    }
    if (ti >= ntgt) return;
    const FarTarget T = tgts[ti];
    const int z = b;
    const float *c = T.cring + (step % T.depth) * (T.r * 4);
    for (int i = threadIdx.x; i < T.px * T.py * 4; i += blockDim.x) {
        const int f = i % 4, ab = i / 4;
        float s = 0.0f;
        for (int cc = 0; cc < T.pz; ++cc) s = fmaf(T.Lz[z * T.pz + cc], c[((cc * T.py) * T.px + ab) * 4 + f], s);
        cz[i] = s;   // index (b * px + a) * 4 + f with node a fastest
    }
    __syncthreads();
    const long long N = (long long)T.nx * T.ny * T.nz;
    for (int i = threadIdx.x; i < T.nx * T.ny; i += blockDim.x) {
        const int x = i % T.nx, y = i / T.nx;
        float v[4] = {0.f, 0.f, 0.f, 0.f};
        for (int bb = 0; bb < T.py; ++bb) {
            const float wy = T.Ly[y * T.py + bb];
            for (int aa = 0; aa < T.px; ++aa) {
                const float w = wy * T.Lx[x * T.px + aa];
                const float *q = cz + (bb * T.px + aa) * 4;
                v[0] = fmaf(w, q[0], v[0]);
                v[1] = fmaf(w, q[1], v[1]);
                v[2] = fmaf(w, q[2], v[2]);
                v[3] = fmaf(w, q[3], v[3]);
            }
        }
        const long long k = (long long)z * T.nx * T.ny + i;
        float *o[4] = {out.phi[T.dom] + k, out.A[T.dom] + k, out.A[T.dom] + N + k, out.A[T.dom] + 2 * N + k};
#pragma unroll
        for (int f = 0; f < 4; ++f) {
            const float val = f == 0 ? v[f] : inv_c * v[f];
            *o[f] = T.interp_add ? *o[f] + val : val;
        }
    }
}

}  // namespace

cudaError_t launch_far_interp(const FarTarget *d_tgts, int ntgt, int nplanes, const OutPtrs &out, long long step,
                              const long long *d_step, float inv_c, cudaStream_t s)
{
    if (ntgt <= 0 || nplanes <= 0) return cudaSuccess;
    k_far_interp<<<nplanes, kFarThreads, 0, s>>>(d_tgts, ntgt, out, step, d_step, inv_c);
    return cudaGetLastError();
}

cudaError_t launch_far_build_w(const FarRow *d_rows, int nrows, const int n[3], double h, double inv_cdt, int ks,
                               __nv_bfloat16 *W, cudaStream_t s)
{
    const long long total = (long long)nrows * ks;
    const int blocks = (int)std::min<long long>((total + kFarThreads - 1) / kFarThreads, 65535LL * 16);
    k_far_build_w<<<blocks, kFarThreads, 0, s>>>(d_rows, nrows, n[0], n[1], n[2], h, inv_cdt, h * h * h, ks, W);
    return cudaGetLastError();
}

cudaError_t launch_far_convert(const FarSource *d_srcs, int nsrc, const IoPtrs &in, int slot, long long max_n,
                               cudaStream_t s)
{
    if (nsrc <= 0) return cudaSuccess;
    const int bx = (int)std::min<long long>((4 * max_n + kFarThreads - 1) / kFarThreads, 1024);
    k_far_convert<<<dim3(bx, nsrc), kFarThreads, 0, s>>>(d_srcs, nsrc, in, slot);
    return cudaGetLastError();
}

cudaError_t launch_far_zero(const FarTarget *d_tgts, int ntgt, long long j1, int batch, int max_r, cudaStream_t s)
{
    if (ntgt <= 0) return cudaSuccess;
    const int bx = (batch * max_r * 4 + kFarThreads - 1) / kFarThreads;
    k_far_zero<<<dim3(bx, ntgt), kFarThreads, 0, s>>>(d_tgts, ntgt, j1, batch);
    return cudaGetLastError();
}

cudaError_t launch_far_scatter(const FarLink *d_links, int nlinks, int nthreads, const float *Z, int ldz, long long j0,
                               int batch, cudaStream_t s)
{
    if (nlinks <= 0 || nthreads <= 0) return cudaSuccess;
    k_far_scatter<<<(nthreads + kFarThreads - 1) / kFarThreads, kFarThreads, 0, s>>>(d_links, nlinks, Z, ldz, j0,
                                                                                      batch);
    return cudaGetLastError();
}

}  // namespace rp
