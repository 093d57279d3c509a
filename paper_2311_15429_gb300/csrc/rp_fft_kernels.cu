// FFT-path kernels: the zero-padded (Hockney) convolution of each target with
// the lag kernels G_m of Eq. 11 of every FFT-path source, itself included,
// summed in the spectral domain over (source, lag) as in Eq. 12.
//
//   push   : k_ring_push   raw (rho, J) slice -> raw history ring (direct pairs only)
//            k_fwd_plane   R2C along x + FFT along y of one z-plane of a source
//            k_fwd_column  FFT along z of a (kx, ky-tile) column block -> spectral ring
//   eval   : k_mac_inv_col sum over (source, lag) of G_m * S(l - m) for a column
//                          block, then inverse FFT along z (kept z < nz of the target)
//            k_inv_plane   inverse FFT along y then C2R along x of one z-plane,
//                          crop to the target grid, scale (1/c for A), write phi / A
//
// Layouts: a spectrum is [field][kx][kz][ky] with ky fastest and kx <= mx/2;
// the scratch after a plane pass is [field][kx][z][ky]; every field array of
// a domain is [z][y][x].
#include <cuda_runtime.h>

#include "rp_fft.cuh"
#include "rp_internal.h"

namespace rp {

namespace {

// index r in [lo, hi) of the last record whose first block (field) is <= b
template <class T>
__device__ __forceinline__ int owner_of(const T *arr, int lo, int hi, int b, int T::*field)
{
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (arr[mid].*field <= b) lo = mid; else hi = mid;
    }
    return lo;
}

// ---------------------------------------------------------------- raw ring push

struct PushPrefix {
    int block0[kMaxDomains + 1];
};

__global__ void __launch_bounds__(kThreads) k_ring_push(const RawRing *__restrict__ rings, IoPtrs in,
                                                          PushPrefix pre, int d0, int d1, long long step)
{
    int b = blockIdx.x;
    int lo = d0, hi = d1;
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (pre.block0[mid] <= b) lo = mid; else hi = mid;
    }
    const int d = lo;
    const RawRing rr = rings[d];
    if (rr.ring == nullptr) return;
    const long long n = rr.n;
    float *dst = rr.ring + (long long)(step % rr.depth) * 4 * n;
    const long long chunk = (long long)kThreads * 8;
    const long long base = (long long)(b - pre.block0[d]) * chunk;
    for (long long i = base + threadIdx.x; i < base + chunk && i < 4 * n; i += kThreads) {
        const float *src = i < n ? in.rho[d] + i : in.J[d] + (i - n);
        dst[i] = *src;
    }
}

// ---------------------------------------------------------------- forward plane pass

struct FwdPlaneX {
    const FwdRing &R;
    const float *plane;
    float2 *Q;      // [ny][qs]
    int qs;
    float2 *W;      // per-group scratch, M each
    const float2 *tw;
    int lane, warp, nwarps;

    template <int RX>
    __device__ void run()
    {
        const Axis &a = R.ax;
        const int G = 32 >> a.logL;
        const int grp = lane >> a.logL, g = lane & (a.L - 1);
        const int pairs = (R.ny + 1) >> 1;
        const int per_iter = nwarps * G;
        float2 *Wg = W + (warp * G + grp) * a.M;
        for (int base = 0; base < pairs; base += per_iter) {
            const int p = base + warp * G + grp;
            const bool valid = p < pairs;
            const int ya = 2 * p, yb = 2 * p + 1;
            const bool vb = valid && yb < R.ny;
            float2 v[RX];
#pragma unroll
            for (int n = 0; n < RX; ++n) {
                const int xi = n * a.L + g;
                const bool in_x = xi < R.nx;
                v[n].x = (valid && in_x) ? plane[ya * R.nx + xi] : 0.0f;
                v[n].y = (vb && in_x) ? plane[yb * R.nx + xi] : 0.0f;
            }
            line_fft<RX, false>(v, g, a, tw);
            const int kb = bitrev_lanes(g, a.logL) * RX;
#pragma unroll
            for (int k1 = 0; k1 < RX; ++k1) Wg[k1 + kb] = v[k1];
            __syncwarp();
            // two real rows from one complex transform:
            //   A[k] = (Z[k] + conj Z[M-k]) / 2,  B[k] = (Z[k] - conj Z[M-k]) / (2i)
            for (int k = g; k < R.kx; k += a.L) {
                const float2 zk = Wg[k];
                const float2 zc = cconj(Wg[(a.M - k) % a.M]);
                const float2 A = cscale(cadd(zk, zc), 0.5f);
                const float2 D = csub(zk, zc);
                const float2 B = make_float2(0.5f * D.y, -0.5f * D.x);
                if (valid) Q[ya * qs + k] = A;
                if (vb) Q[yb * qs + k] = B;
            }
            __syncwarp();
        }
    }
};

struct FwdPlaneY {
    const FwdRing &R;
    const float2 *Q;
    int qs;
    float2 *out;    // t1 + ((f*kx + 0)*nz + z)*my ; row kx at out + kx*nz*my
    const float2 *tw;
    int lane, warp, nwarps;

    template <int RY>
    __device__ void run()
    {
        const Axis &a = R.ay;
        const int G = 32 >> a.logL;
        const int grp = lane >> a.logL, g = lane & (a.L - 1);
        const int per_iter = nwarps * G;
        const long long row_stride = (long long)R.nz * a.M;
        for (int base = 0; base < R.kx; base += per_iter) {
            const int kxi = base + warp * G + grp;
            const bool valid = kxi < R.kx;
            float2 v[RY];
#pragma unroll
            for (int n = 0; n < RY; ++n) {
                const int yi = n * a.L + g;
                v[n] = (valid && yi < R.ny) ? Q[yi * qs + kxi] : make_float2(0.0f, 0.0f);
            }
            line_fft<RY, false>(v, g, a, tw);
            const int kb = bitrev_lanes(g, a.logL) * RY;
            if (valid) {
                float2 *row = out + kxi * row_stride;
#pragma unroll
                for (int k1 = 0; k1 < RY; ++k1) row[k1 + kb] = v[k1];
            }
        }
    }
};

__global__ void __launch_bounds__(kThreads) k_fwd_plane(const FwdRing *__restrict__ rings, IoPtrs in,
                                                          int r0, int r1, int block_lo)
{
    extern __shared__ float4 smem_f4[];
    float2 *sm = reinterpret_cast<float2 *>(smem_f4);
    const int b = blockIdx.x + block_lo;
    const int r = owner_of(rings, r0, r1, b, &FwdRing::plane0);
    const FwdRing &R = rings[r];
    const int local = b - R.plane0;
    const int f = local / R.nz, z = local % R.nz;
    const long long N = (long long)R.nx * R.ny * R.nz;

    float2 *twx = sm;
    float2 *twy = twx + R.ax.M;
    const int qs = R.kx | 1;
    float2 *Q = twy + R.ay.M;
    float2 *W = Q + R.ny * qs;
    load_twiddles(twx, R.tw_x, R.ax.M);
    load_twiddles(twy, R.tw_y, R.ay.M);
    __syncthreads();

    const float *src = f == 0 ? in.rho[R.src] : in.J[R.src] + (long long)(f - 1) * N;
    const float *plane = src + (long long)z * R.nx * R.ny;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;

    FwdPlaneX px{R, plane, Q, qs, W, twx, lane, warp, nwarps};
    dispatch_radix(R.ax.R, px);
    __syncthreads();
    float2 *out = R.t1 + ((long long)f * R.kx * R.nz + z) * R.ay.M;
    FwdPlaneY py{R, Q, qs, out, twy, lane, warp, nwarps};
    dispatch_radix(R.ay.R, py);
}

// ---------------------------------------------------------------- forward column pass

struct ColumnFFT {
    const Axis &a;
    float2 *V;        // [M][kTileYPad] (per field block: base passed in)
    long long field_stride;  // float2 between fields in V (0 if one field)
    int ncols;        // columns per field
    int nfields;
    int keep;         // outputs kept: index < keep
    const float2 *tw;
    bool inverse;
    int lane, warp, nwarps;

    template <int RR>
    __device__ void run()
    {
        const int G = 32 >> a.logL;
        const int grp = lane >> a.logL, g = lane & (a.L - 1);
        const int lines = ncols * nfields;
        const int per_iter = nwarps * G;
        for (int base = 0; base < lines; base += per_iter) {
            const int line = base + warp * G + grp;
            const bool valid = line < lines;
            const int fld = valid ? line / ncols : 0, c = valid ? line % ncols : 0;
            float2 *col = V + fld * field_stride + c;
            float2 v[RR];
#pragma unroll
            for (int n = 0; n < RR; ++n) v[n] = col[(n * a.L + g) * kTileYPad];
            if (inverse) line_fft<RR, true>(v, g, a, tw); else line_fft<RR, false>(v, g, a, tw);
            __syncwarp();
            const int kb = bitrev_lanes(g, a.logL) * RR;
            if (valid) {
#pragma unroll
                for (int k1 = 0; k1 < RR; ++k1)
                    if (k1 + kb < keep) col[(k1 + kb) * kTileYPad] = v[k1];
            }
            __syncwarp();
        }
    }
};

__global__ void __launch_bounds__(kThreads) k_fwd_column(const FwdRing *__restrict__ rings, int r0, int r1,
                                                           int block_lo, long long step)
{
    extern __shared__ float4 smem_f4[];
    float2 *sm = reinterpret_cast<float2 *>(smem_f4);
    const int b = blockIdx.x + block_lo;
    const int r = owner_of(rings, r0, r1, b, &FwdRing::tile0);
    const FwdRing &R = rings[r];
    const int my = R.ay.M, mz = R.az.M;
    const int ntile = (my + kTileY - 1) / kTileY;
    const int local = b - R.tile0;
    const int per_field = R.kx * ntile;
    const int f = local / per_field, rem = local % per_field;
    const int kxi = rem / ntile, ky0 = (rem % ntile) * kTileY;

    float2 *tw = sm;
    float2 *V = tw + mz;
    load_twiddles(tw, R.tw_z, mz);
    const float2 *src = R.t1 + ((long long)f * R.kx + kxi) * R.nz * my;
    for (int i = threadIdx.x; i < mz * kTileY; i += blockDim.x) {
        const int zi = i / kTileY, c = i % kTileY;
        float2 v = make_float2(0.0f, 0.0f);
        if (zi < R.nz && ky0 + c < my) v = src[(long long)zi * my + ky0 + c];
        V[zi * kTileYPad + c] = v;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int ncols = min(kTileY, my - ky0);
    ColumnFFT cf{R.az, V, 0, ncols, 1, mz, tw, false, lane, warp, nwarps};
    dispatch_radix(R.az.R, cf);
    __syncthreads();
    float2 *dst = R.ring + (long long)(step % R.depth) * R.slot_elems +
                  ((long long)f * R.kx + kxi) * mz * my;
    for (int i = threadIdx.x; i < mz * kTileY; i += blockDim.x) {
        const int kz = i / kTileY, c = i % kTileY;
        if (c < ncols) dst[(long long)kz * my + ky0 + c] = V[kz * kTileYPad + c];
    }
}

// ---------------------------------------------------------------- MAC + inverse column pass

__global__ void __launch_bounds__(kThreads) k_mac_inv_column(const InvTarget *__restrict__ tgts, int ntgt,
                                                               const MacEntry *__restrict__ entries,
                                                               long long step, int clamp)
{
    extern __shared__ float4 smem_f4[];
    float2 *sm = reinterpret_cast<float2 *>(smem_f4);
    const int b = blockIdx.x;
    const int t = owner_of(tgts, 0, ntgt, b, &InvTarget::tile0);
    const InvTarget &T = tgts[t];
    const int my = T.ay.M, mz = T.az.M;
    const int ntile = (my + kTileY - 1) / kTileY;
    const int local = b - T.tile0;
    const int kxi = local / ntile, ky0 = (local % ntile) * kTileY;
    const int ncols = min(kTileY, my - ky0);
    const long long fstride = (long long)T.kx * mz * my;
    const long long col0 = (long long)kxi * mz * my + ky0;

    float2 *tw = sm;
    float2 *acc = tw + mz;                 // [4][mz][kTileYPad]
    const int fs = mz * kTileYPad;
    load_twiddles(tw, T.tw_z, mz);
    for (int i = threadIdx.x; i < 4 * fs; i += blockDim.x) acc[i] = make_float2(0.0f, 0.0f);
    __syncthreads();

    // Each thread owns the (kz, c) cells i = threadIdx.x + k*blockDim.x; the
    // same cells for every entry, so no barrier is needed between entries.
    for (int e = T.e0; e < T.e1; ++e) {
        const MacEntry E = entries[e];
        long long j = step - E.lag;
        if (clamp && j < 0) j = 0;
        const float2 *S = E.ring + (j % E.depth) * E.slot_elems + col0;
        const float *Gr = static_cast<const float *>(E.g) + col0;
        const float2 *Gc = static_cast<const float2 *>(E.g) + col0;
#pragma unroll 2
        for (int i = threadIdx.x; i < mz * kTileY; i += blockDim.x) {
            const int kz = i / kTileY, c = i % kTileY;
            if (c >= ncols) continue;
            const long long off = (long long)kz * my + c;
            const float2 g = E.is_real ? make_float2(__ldg(Gr + off), 0.0f) : __ldg(Gc + off);
            const float2 s0 = __ldg(S + off);
            const float2 s1 = __ldg(S + fstride + off);
            const float2 s2 = __ldg(S + 2 * fstride + off);
            const float2 s3 = __ldg(S + 3 * fstride + off);
            const int a = kz * kTileYPad + c;
            acc[a] = cadd(acc[a], cmul(g, s0));
            acc[fs + a] = cadd(acc[fs + a], cmul(g, s1));
            acc[2 * fs + a] = cadd(acc[2 * fs + a], cmul(g, s2));
            acc[3 * fs + a] = cadd(acc[3 * fs + a], cmul(g, s3));
        }
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    ColumnFFT cf{T.az, acc, fs, ncols, 4, T.nz, tw, true, lane, warp, nwarps};
    dispatch_radix(T.az.R, cf);
    __syncthreads();
    for (int i = threadIdx.x; i < 4 * T.nz * kTileY; i += blockDim.x) {
        const int f = i / (T.nz * kTileY), rem = i % (T.nz * kTileY);
        const int zi = rem / kTileY, c = rem % kTileY;
        if (c < ncols)
            T.t2[(((long long)f * T.kx + kxi) * T.nz + zi) * my + ky0 + c] = acc[f * fs + zi * kTileYPad + c];
    }
}

// ---------------------------------------------------------------- inverse plane pass

struct InvPlaneY {
    const InvTarget &T;
    float2 *P;
    int ps;
    const float2 *tw;
    int lane, warp, nwarps;

    template <int RY>
    __device__ void run()
    {
        const Axis &a = T.ay;
        const int G = 32 >> a.logL;
        const int grp = lane >> a.logL, g = lane & (a.L - 1);
        const int per_iter = nwarps * G;
        for (int base = 0; base < T.kx; base += per_iter) {
            const int kxi = base + warp * G + grp;
            const bool valid = kxi < T.kx;
            float2 *row = P + (valid ? kxi : 0) * ps;
            float2 v[RY];
#pragma unroll
            for (int n = 0; n < RY; ++n) v[n] = row[n * a.L + g];
            line_fft<RY, true>(v, g, a, tw);
            __syncwarp();
            const int kb = bitrev_lanes(g, a.logL) * RY;
            if (valid) {
#pragma unroll
                for (int k1 = 0; k1 < RY; ++k1)
                    if (k1 + kb < T.ny) row[k1 + kb] = v[k1];
            }
            __syncwarp();
        }
    }
};

struct InvPlaneX {
    const InvTarget &T;
    const float2 *P;
    int ps;
    float *O;       // [ny][nx]
    float scale;
    const float2 *tw;
    int lane, warp, nwarps;

    template <int RX>
    __device__ void run()
    {
        const Axis &a = T.ax;
        const int G = 32 >> a.logL;
        const int grp = lane >> a.logL, g = lane & (a.L - 1);
        const int pairs = (T.ny + 1) >> 1;
        const int half = a.M >> 1;
        const int per_iter = nwarps * G;
        for (int base = 0; base < pairs; base += per_iter) {
            const int p = base + warp * G + grp;
            const bool valid = p < pairs;
            const int ya = valid ? 2 * p : 0, yb = ya + 1;
            const bool vb = valid && yb < T.ny;
            float2 v[RX];
#pragma unroll
            for (int n = 0; n < RX; ++n) {
                const int k = n * a.L + g;
                const bool lower = k <= half;
                const int kk = lower ? k : a.M - k;
                float2 A = P[kk * ps + ya];
                float2 B = vb ? P[kk * ps + yb] : make_float2(0.0f, 0.0f);
                if (!lower) { A = cconj(A); B = cconj(B); }
                if (k == 0 || k == half) { A.y = 0.0f; B.y = 0.0f; }
                v[n] = make_float2(A.x - B.y, A.y + B.x);   // A + iB
            }
            line_fft<RX, true>(v, g, a, tw);
            const int kb = bitrev_lanes(g, a.logL) * RX;
            if (valid) {
#pragma unroll
                for (int k1 = 0; k1 < RX; ++k1) {
                    const int x = k1 + kb;
                    if (x < T.nx) {
                        O[ya * T.nx + x] = scale * v[k1].x;
                        if (vb) O[yb * T.nx + x] = scale * v[k1].y;
                    }
                }
            }
        }
    }
};

__global__ void __launch_bounds__(kThreads) k_inv_plane(const InvTarget *__restrict__ tgts, int ntgt, OutPtrs out,
                                                          float inv_c)
{
    extern __shared__ float4 smem_f4[];
    float2 *sm = reinterpret_cast<float2 *>(smem_f4);
    const int b = blockIdx.x;
    const int t = owner_of(tgts, 0, ntgt, b, &InvTarget::plane0);
    const InvTarget &T = tgts[t];
    const int local = b - T.plane0;
    const int f = local / T.nz, z = local % T.nz;
    const int my = T.ay.M;
    const int ps = my | 1;

    float2 *twx = sm;
    float2 *twy = twx + T.ax.M;
    float2 *P = twy + my;                                   // [kx][ps]
    float *O = reinterpret_cast<float *>(P + T.kx * ps);    // [ny][nx]
    load_twiddles(twx, T.tw_x, T.ax.M);
    load_twiddles(twy, T.tw_y, my);
    const float2 *src = T.t2 + ((long long)f * T.kx * T.nz + z) * my;
    const long long row_stride = (long long)T.nz * my;
    for (int i = threadIdx.x; i < T.kx * my; i += blockDim.x) {
        const int kxi = i / my, ky = i % my;
        P[kxi * ps + ky] = src[kxi * row_stride + ky];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    InvPlaneY py{T, P, ps, twy, lane, warp, nwarps};
    dispatch_radix(T.ay.R, py);
    __syncthreads();
    InvPlaneX px{T, P, ps, O, f == 0 ? 1.0f : inv_c, twx, lane, warp, nwarps};
    dispatch_radix(T.ax.R, px);
    __syncthreads();
    const long long N = (long long)T.nx * T.ny * T.nz;
    float *dst = (f == 0 ? out.phi[T.dom] : out.A[T.dom] + (long long)(f - 1) * N) +
                 (long long)z * T.nx * T.ny;
    for (int i = threadIdx.x; i < T.nx * T.ny; i += blockDim.x) dst[i] = O[i];
}

}  // namespace

// ---------------------------------------------------------------- launchers

size_t smem_fwd_plane(int ny, const Axis &ax)
{
    const int kx = ax.M / 2 + 1;
    const int qs = kx | 1;
    // twiddles (x and y, bounded by kMaxFFT each) + Q + per-group scratch
    return sizeof(float2) * (2 * kMaxFFT + (size_t)ny * qs + (size_t)(kThreads / 32) * 32 * ax.R);
}

size_t smem_fwd_column(const Axis &az) { return sizeof(float2) * ((size_t)az.M + (size_t)az.M * kTileYPad); }

size_t smem_mac_inv_column(const Axis &az)
{
    return sizeof(float2) * ((size_t)az.M + 4 * (size_t)az.M * kTileYPad);
}

size_t smem_inv_plane(int nx, int ny, const Axis &ax, const Axis &ay)
{
    const int kx = ax.M / 2 + 1;
    const int ps = ay.M | 1;
    return sizeof(float2) * ((size_t)ax.M + ay.M + (size_t)kx * ps) + sizeof(float) * (size_t)nx * ny;
}

// The dynamic shared-memory limit is an attribute of the kernel function,
// shared by every context in the process, so each kernel is opened up to the
// device's opt-in maximum once (contexts never lower it for one another).
cudaError_t open_kernel_smem_limits(int max_optin)
{
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_fwd_plane, cudaFuncAttributeMaxDynamicSharedMemorySize, max_optin))) return e;
    if ((e = cudaFuncSetAttribute(k_fwd_column, cudaFuncAttributeMaxDynamicSharedMemorySize, max_optin))) return e;
    if ((e = cudaFuncSetAttribute(k_mac_inv_column, cudaFuncAttributeMaxDynamicSharedMemorySize, max_optin))) return e;
    if ((e = cudaFuncSetAttribute(k_inv_plane, cudaFuncAttributeMaxDynamicSharedMemorySize, max_optin))) return e;
    return cudaSuccess;
}

cudaError_t launch_ring_push(const RawRing *d_rings, const IoPtrs &in, int d0, int d1,
                             const int *h_block0, int nblocks, long long step, cudaStream_t s)
{
    if (nblocks <= 0) return cudaSuccess;
    PushPrefix pre;
    for (int d = 0; d <= kMaxDomains; ++d) pre.block0[d] = 0;
    for (int d = d0; d <= d1; ++d) pre.block0[d] = h_block0[d];
    k_ring_push<<<nblocks, kThreads, 0, s>>>(d_rings, in, pre, d0, d1, step);
    return cudaGetLastError();
}

cudaError_t launch_fwd_plane(const FwdRing *d_rings, const IoPtrs &in, int r0, int r1, int block_lo,
                             int nblocks, size_t smem, cudaStream_t s)
{
    if (nblocks <= 0) return cudaSuccess;
    k_fwd_plane<<<nblocks, kThreads, smem, s>>>(d_rings, in, r0, r1, block_lo);
    return cudaGetLastError();
}

cudaError_t launch_fwd_column(const FwdRing *d_rings, int r0, int r1, int block_lo, int nblocks,
                              size_t smem, long long step, cudaStream_t s)
{
    if (nblocks <= 0) return cudaSuccess;
    k_fwd_column<<<nblocks, kThreads, smem, s>>>(d_rings, r0, r1, block_lo, step);
    return cudaGetLastError();
}

cudaError_t launch_mac_inv_column(const InvTarget *d_tgts, int ntgt, const MacEntry *d_entries, int nblocks,
                                  size_t smem, long long step, int clamp, cudaStream_t s)
{
    if (nblocks <= 0) return cudaSuccess;
    k_mac_inv_column<<<nblocks, kThreads, smem, s>>>(d_tgts, ntgt, d_entries, step, clamp);
    return cudaGetLastError();
}

cudaError_t launch_inv_plane(const InvTarget *d_tgts, int ntgt, const OutPtrs &out, int nblocks, size_t smem,
                             float inv_c, cudaStream_t s)
{
    if (nblocks <= 0) return cudaSuccess;
    k_inv_plane<<<nblocks, kThreads, smem, s>>>(d_tgts, ntgt, out, inv_c);
    return cudaGetLastError();
}

}  // namespace rp
