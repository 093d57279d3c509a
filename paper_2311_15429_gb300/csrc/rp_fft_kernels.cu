// FFT-path kernels: the zero-padded (Hockney) convolution of each target with
// the lag kernels G_m of Eq. 11 of every FFT-path source, itself included,
// summed in the spectral domain over (source, lag) as in Eq. 12.
//
//   push   : k_ring_push   raw (rho, J) slice -> raw history ring (direct pairs only)
//            k_fwd_plane   R2C along x + FFT along y of one z-plane of a source
//            k_fwd_column  FFT along z of a (kx, 16 ky) column block, 4 fields -> spectral ring
//   eval   : k_mac_inv_col sum over (source, lag) of G_m * S(l - m) for a column
//                          block, then inverse FFT along z (kept z < nz of the target)
//            k_inv_plane   inverse FFT along y then C2R along x of one z-plane,
//                          crop to the target grid, scale (1/c for A), write phi / A
//
// Layouts: a spectrum is [field][kx][kz][ky] with ky fastest and kx <= mx/2;
// the scratch after a plane pass is [field][kx][z][ky]; every field array of
// a domain is [z][y][x].
//
// The passes come in two forms.  k_fwd_plane16, k_fwd_column16 and
// k_inv_plane16 run the two-stage shared-memory tile transform of rp_fft.cuh
// (M = 16 B: the plane passes for M = 64, 96, 128, the column pass also for
// 192).  k_fwd_plane, k_fwd_column and k_inv_plane run the lane-shuffle line
// transform for the other cubic sizes (32, 48, and 192 for the plane passes)
// and for M = 0 (any supported shape, read at run time).  The MAC with its
// inverse column transform is instantiated for every class.
#include <cuda_runtime.h>

#include "rp_fft.cuh"
#include "rp_internal.h"

namespace rp {

namespace {

__host__ __device__ constexpr int radix_R(int M) { return lane_radix(M); }
__host__ __device__ constexpr int radix_L(int M) { return M / radix_R(M); }
__host__ __device__ constexpr int ilog2c(int x) { return x <= 1 ? 0 : 1 + ilog2c(x / 2); }

template <int M>
__device__ __forceinline__ Axis axis_of(const Axis &rt)
{
    if constexpr (M == 0) return rt;
    else return Axis{M, radix_R(M), radix_L(M), ilog2c(radix_L(M))};
}

template <int M, class F>
__device__ __forceinline__ void run_radix(int R_rt, F &f)
{
    if constexpr (M == 0) dispatch_radix(R_rt, f);
    else f.template run<radix_R(M)>();
}

__host__ __device__ constexpr int lane_class(int M) { return M > 0 ? M : 32; }

// One line FFT: the compiled-size transform with precomputed lane twiddles
// for M > 0, else the table-driven runtime transform.
template <int M, bool INV, int RR>
__device__ __forceinline__ void do_line(float2 (&v)[RR], int g, const Axis &a, const float2 *tw,
                                        const LaneTw<lane_class(M), INV> *lt)
{
    if constexpr (M > 0) line_fft_c<M, INV>(v, *lt);
    else line_fft<RR, INV>(v, g, a, tw);
}

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

__device__ __forceinline__ float4 ldg4(const float2 *p) { return __ldg(reinterpret_cast<const float4 *>(p)); }

// 16-byte asynchronous global -> shared copy (both addresses 16-byte aligned)
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((unsigned)__cvta_generic_to_shared(smem)),
                 "l"(gmem)
                 : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

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
    if (step < 0) step = *rr.d_step;   // graph replay: the step from the device counter
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

template <int M>
struct FwdPlaneX {
    const LaneTw<lane_class(M), false> *lt;
    Axis a;
    int nx, ny, kx;
    const float *plane;
    float2 *Q;      // [ny][qs]
    int qs;
    float2 *W;      // per-group scratch, M each
    const float2 *tw;
    int lane, warp, nwarps;

    template <int RX>
    __device__ __forceinline__ void run()
    {
        const int G = 32 >> a.logL;
        const int grp = lane >> a.logL, g = lane & (a.L - 1);
        const int pairs = (ny + 1) >> 1;
        const int per_iter = nwarps * G;
        float2 *Wg = W + (warp * G + grp) * a.M;
        for (int base = 0; base < pairs; base += per_iter) {
            const int p = base + warp * G + grp;
            const bool valid = p < pairs;
            const int ya = 2 * p, yb = 2 * p + 1;
            const bool vb = valid && yb < ny;
            float2 v[RX];
#pragma unroll
            for (int n = 0; n < RX; ++n) {
                const int xi = n * a.L + g;
                const bool in_x = xi < nx;
                v[n].x = (valid && in_x) ? plane[ya * nx + xi] : 0.0f;
                v[n].y = (vb && in_x) ? plane[yb * nx + xi] : 0.0f;
            }
            do_line<M, false>(v, g, a, tw, lt);
            const int kb = bitrev_lanes(g, a.logL) * RX;
#pragma unroll
            for (int k1 = 0; k1 < RX; ++k1) Wg[k1 + kb] = v[k1];
            __syncwarp();
            // two real rows from one complex transform:
            //   A[k] = (Z[k] + conj Z[M-k]) / 2,  B[k] = (Z[k] - conj Z[M-k]) / (2i)
            for (int k = g; k < kx; k += a.L) {
                const float2 zk = Wg[k];
                const float2 zc = cconj(Wg[k == 0 ? 0 : a.M - k]);
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

template <int M>
struct FwdPlaneY {
    const LaneTw<lane_class(M), false> *lt;
    Axis a;
    int ny, kx, nz;
    const float2 *Q;
    int qs;
    float2 *out;    // row kx at out + kx*nz*my
    const float2 *tw;
    int lane, warp, nwarps;

    template <int RY>
    __device__ __forceinline__ void run()
    {
        const int G = 32 >> a.logL;
        const int grp = lane >> a.logL, g = lane & (a.L - 1);
        const int per_iter = nwarps * G;
        const long long row_stride = (long long)nz * a.M;
        for (int base = 0; base < kx; base += per_iter) {
            const int kxi = base + warp * G + grp;
            const bool valid = kxi < kx;
            float2 v[RY];
#pragma unroll
            for (int n = 0; n < RY; ++n) {
                const int yi = n * a.L + g;
                v[n] = (valid && yi < ny) ? Q[yi * qs + kxi] : make_float2(0.0f, 0.0f);
            }
            do_line<M, false>(v, g, a, tw, lt);
            const int kb = bitrev_lanes(g, a.logL) * RY;
            if (valid) {
                float2 *row = out + kxi * row_stride;
#pragma unroll
                for (int k1 = 0; k1 < RY; ++k1) row[k1 + kb] = v[k1];
            }
        }
    }
};

template <int M>
__global__ void __launch_bounds__(kPlaneThreads) k_fwd_plane(const FwdRing *__restrict__ rings, IoPtrs in,
                                                          int r0, int r1, int block_lo, int far_slot)
{
    extern __shared__ float4 smem_f4[];
    float2 *sm = reinterpret_cast<float2 *>(smem_f4);
    const int b = blockIdx.x + block_lo;
    const int r = owner_of(rings, r0, r1, b, &FwdRing::plane0);
    const FwdRing &R = rings[r];
    const Axis ax = axis_of<M>(R.ax), ay = axis_of<M>(R.ay);
    const int nx = R.nx, ny = R.ny, nz = R.nz;
    const int kx = ax.M / 2 + 1;
    const int local = b - R.plane0;
    const int f = local / nz, z = local % nz;
    const long long N = (long long)nx * ny * nz;

    float2 *twx = sm;
    float2 *twy = twx + ax.M;
    const int qs = kx | 1;
    float2 *Q = twy + ay.M;
    float2 *W = Q + ny * qs;
    load_twiddles(twx, R.tw_x, ax.M);
    load_twiddles(twy, R.tw_y, ay.M);
    pdl_trigger();
    pdl_wait();   // the input slice may come from the previous kernel; t1 was read by it
    __syncthreads();

    const float *src = f == 0 ? in.rho[R.src] : in.J[R.src] + (long long)(f - 1) * N;
    const float *plane = src + (long long)z * nx * ny;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;

    LaneTw<lane_class(M), false> lt;
    if constexpr (M > 0) lt.init(twx, lane & (ax.L - 1));
    FwdPlaneX<M> px{&lt, ax, nx, ny, kx, plane, Q, qs, W, twx, lane, warp, nwarps};
    run_radix<M>(ax.R, px);
    __syncthreads();
    float2 *out = R.t1 + ((long long)f * kx * nz + z) * ay.M;
    FwdPlaneY<M> py{&lt, ay, ny, kx, nz, Q, qs, out, twy, lane, warp, nwarps};
    run_radix<M>(ay.R, py);
    if (R.far_x) {
        // far path: this plane as bf16 hi/lo into row (slot, field) of the batch matrix
        __nv_bfloat16 *row = R.far_x + ((long long)far_slot * 4 + f) * 2 * R.far_ks + (long long)z * nx * ny;
        for (int i = threadIdx.x; i < nx * ny; i += blockDim.x) {
            const float v = __ldg(plane + i);
            const __nv_bfloat16 hi = __float2bfloat16(v);
            row[i] = hi;
            row[R.far_ks + i] = __float2bfloat16(v - __bfloat162float(hi));
        }
    }
}

// ---------------------------------------------------------------- column passes

// Line FFTs down the columns of a shared-memory tile [field][M][kTileYPad].
template <int M, bool INV>
struct ColumnFFT {
    const LaneTw<lane_class(M), INV> *lt;
    Axis a;
    float2 *V;
    int field_stride;  // float2 between fields in V
    int ncols;         // columns per field
    int nfields;
    int keep;          // outputs kept: index < keep
    const float2 *tw;
    int lane, warp, nwarps;

    template <int RR>
    __device__ __forceinline__ void run()
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
            do_line<M, INV>(v, g, a, tw, lt);
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

// Forward FFT along z of the four fields of one (kx, 16-ky) column block.
template <int M>
__global__ void __launch_bounds__(kColumnThreads) k_fwd_column(const FwdRing *__restrict__ rings, int r0, int r1,
                                                           int block_lo, long long step)
{
    extern __shared__ float4 smem_f4[];
    float2 *sm = reinterpret_cast<float2 *>(smem_f4);
    const int b = blockIdx.x + block_lo;
    const int r = owner_of(rings, r0, r1, b, &FwdRing::tile0);
    const FwdRing &R = rings[r];
    const Axis az = axis_of<M>(R.az);
    const int my = M ? M : R.ay.M, mz = az.M, nz = R.nz;
    const int kx = M ? M / 2 + 1 : R.kx;
    const int ntile = (my + kTileY - 1) / kTileY;
    const int local = b - R.tile0;
    const int kxi = local / ntile, ky0 = (local % ntile) * kTileY;
    const int ncols = min(kTileY, my - ky0);
    const int fs = mz * kTileYPad;

    float2 *tw = sm;
    float2 *V = tw + mz;
    load_twiddles(tw, R.tw_z, mz);
    pdl_trigger();
    pdl_wait();   // t1 is written by the plane pass
    if (step < 0) step = *R.d_step;   // graph replay: the step from the device counter
    const long long t1_field = (long long)kx * nz * my;
    const float2 *src = R.t1 + (long long)kxi * nz * my + ky0;
    if constexpr (M > 0) {
        // 16-byte loads of column pairs; rows z >= nz are the zero padding
        for (int i = threadIdx.x; i < 4 * mz * (kTileY / 2); i += blockDim.x) {
            const int f = i / (mz * (kTileY / 2)), rem = i % (mz * (kTileY / 2));
            const int zi = rem / (kTileY / 2), p = rem % (kTileY / 2);
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (zi < nz) v = ldg4(src + f * t1_field + (long long)zi * my + 2 * p);
            float2 *d = V + f * fs + zi * kTileYPad + 2 * p;
            d[0] = make_float2(v.x, v.y);
            d[1] = make_float2(v.z, v.w);
        }
    } else {
        for (int i = threadIdx.x; i < 4 * mz * kTileY; i += blockDim.x) {
            const int f = i / (mz * kTileY), rem = i % (mz * kTileY);
            const int zi = rem / kTileY, c = rem % kTileY;
            float2 v = make_float2(0.0f, 0.0f);
            if (zi < nz && c < ncols) v = src[f * t1_field + (long long)zi * my + c];
            V[f * fs + zi * kTileYPad + c] = v;
        }
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    LaneTw<lane_class(M), false> lt;
    if constexpr (M > 0) lt.init(tw, lane & (az.L - 1));
    ColumnFFT<M, false> cf{&lt, az, V, fs, ncols, 4, mz, tw, lane, warp, nwarps};
    run_radix<M>(az.R, cf);
    __syncthreads();
    // the tile's four field tiles sit next to each other in the slot
    const long long ring_field = (long long)mz * kTileY;
    float2 *dst = R.ring + (long long)((step - R.lag_off) % R.depth) * R.slot_elems +
                  (long long)(kxi * ntile + ky0 / kTileY) * 4 * ring_field;
    if constexpr (M > 0) {
        for (int i = threadIdx.x; i < 4 * mz * (kTileY / 2); i += blockDim.x) {
            const int f = i / (mz * (kTileY / 2)), rem = i % (mz * (kTileY / 2));
            const int kz = rem / (kTileY / 2), p = rem % (kTileY / 2);
            const float2 *s = V + f * fs + kz * kTileYPad + 2 * p;
            *reinterpret_cast<float4 *>(dst + f * ring_field + kz * kTileY + 2 * p) =
                make_float4(s[0].x, s[0].y, s[1].x, s[1].y);
        }
    } else {
        for (int i = threadIdx.x; i < 4 * mz * kTileY; i += blockDim.x) {
            const int f = i / (mz * kTileY), rem = i % (mz * kTileY);
            const int kz = rem / kTileY, c = rem % kTileY;
            dst[f * ring_field + kz * kTileY + c] = c < ncols ? V[f * fs + kz * kTileYPad + c] : make_float2(0.f, 0.f);
        }
    }
}

// The forward column pass for M = 16 B, B even (M = 64, 96, 128, 192): the
// tile [field][z][16] dense in shared memory, one warp per field with the
// two-stage tile transform (rows z >= nz are the zero padding: neither loaded
// nor read; when nz <= M/2 the first layer skips the zero half), then each
// spectral row copied from its tile row to the ring slot.
constexpr int kColumn16Threads = 256;   // two warps per field

__host__ __device__ constexpr bool tile16_class(int M) { return M == 64 || M == 96 || M == 128 || M == 192; }

template <int M>
__global__ void __launch_bounds__(kColumn16Threads) k_fwd_column16(const FwdRing *__restrict__ rings, int r0, int r1,
                                                                    int block_lo, long long step)
{
    constexpr int B = M / 16, kx = M / 2 + 1, ntile = M / kTileY;
    static_assert(tile16_class(M), "k_fwd_column16: M = 16 B, B even");
    extern __shared__ float4 smem_f4[];
    float2 *sm = reinterpret_cast<float2 *>(smem_f4);
    const int b = blockIdx.x + block_lo;
    const int r = owner_of(rings, r0, r1, b, &FwdRing::tile0);
    const FwdRing &R = rings[r];
    const int nz = R.nz;
    const int local = b - R.tile0;
    const int kxi = local / ntile, kyt = local % ntile;
    float2 *tw = sm;
    float2 *V = tw + M;   // [field][M rows][16]
    load_twiddles(tw, R.tw_z, M);
    pdl_trigger();
    pdl_wait();   // t1 is written by the plane pass
    if (step < 0) step = *R.d_step;   // graph replay: the step from the device counter
    __syncthreads();   // the twiddles
    // the warp pair 2f, 2f + 1 owns field f from copy-in to store (named
    // barrier 1 + f): no block barrier, so the fields' copies, transforms and
    // stores interleave
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, f = warp >> 1, half = warp & 1;
    const int t64 = threadIdx.x & 63, p = t64 & 7, zr = t64 >> 3;   // column pair p, rows zr + 8 j
    float2 *Vf = V + f * M * kTileY;
    {
        const long long t1_field = (long long)kx * nz * M;
        const float2 *src = R.t1 + f * t1_field + (long long)kxi * nz * M + kyt * kTileY + 2 * p;
        for (int z = zr; z < nz; z += 8) cp_async16(Vf + z * kTileY + 2 * p, src + (long long)z * M);
        cp_async_wait_all();
    }
    asm volatile("bar.sync %0, 64;" ::"r"(1 + f) : "memory");
    // a source as large as the target's padded half (the usual case) skips the
    // zero half in the first layer; a larger source of a cross pair does not
    if (nz <= M / 2) tile_fft16_pair<B, false, true>(Vf, tw, nz, lane, half, 1 + f);
    else tile_fft16_pair<B, false, false>(Vf, tw, nz, lane, half, 1 + f);
    float2 *dst = R.ring + (long long)((step - R.lag_off) % R.depth) * R.slot_elems +
                  (long long)(kxi * ntile + kyt) * 4 * M * kTileY + f * M * kTileY;
#pragma unroll 4
    for (int kz = zr; kz < M; kz += 8)
        *reinterpret_cast<float4 *>(dst + kz * kTileY + 2 * p) =
            *reinterpret_cast<const float4 *>(Vf + tile_row<B>(kz) * kTileY + 2 * p);
}

// Kahan-compensated addition (the total is s - c; see k_mac_tma).
__device__ __forceinline__ void kahan_add(float &s, float &c, float x)
{
    const float y = x - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
}

// Spectral multiply-accumulate over the target's (source, lag) entries for
// one (kx, 16-ky) column block and all four fields, then the inverse FFT
// along z of the 64 columns; rows z < nz of the target go to T2.  COMP: the
// sum over entries is Kahan-compensated per spectral coefficient.
template <int M, bool COMP>
__global__ void __launch_bounds__(kThreads) k_mac_inv_column(const InvTarget *__restrict__ tgts, int t0, int t1,
                                                               int block_lo, const MacEntry *__restrict__ entries,
                                                               long long step, int clamp)
{
    extern __shared__ float4 smem_f4[];
    float2 *sm = reinterpret_cast<float2 *>(smem_f4);
    const int b = blockIdx.x + block_lo;
    const int t = owner_of(tgts, t0, t1, b, &InvTarget::tile0);
    const InvTarget &T = tgts[t];
    const Axis az = axis_of<M>(T.az);
    const int my = M ? M : T.ay.M, mz = az.M;
    const int kx = M ? M / 2 + 1 : T.kx;
    const int ntile = (my + kTileY - 1) / kTileY;
    const int local = b - T.tile0;
    const int kxi = local / ntile, ky0 = (local % ntile) * kTileY;
    const int ncols = min(kTileY, my - ky0);
    const long long col0 = (long long)(kxi * ntile + ky0 / kTileY) * mz * kTileY;   // tile in a kernel spectrum
    const long long fstride = (long long)mz * kTileY;                             // field tile in a ring slot
    const long long sbase = 3 * col0;   // + col0: the tile's first field tile in a ring slot (4 per tile)
    const int fs = mz * kTileYPad;

    float2 *tw = sm;
    float2 *acc = tw + mz;                 // [4][mz][kTileYPad]
    load_twiddles(tw, T.tw_z, mz);
    pdl_trigger();
    pdl_wait();   // the newest ring slot is written by the column pass
    if (step < 0) step = *T.d_step;   // graph replay: the step from the device counter

    if constexpr (M > 0) {
        // Thread (p, r0) owns ky columns 2p, 2p+1 and kz rows r0 + 32 i.  All
        // operands of an entry (kernel + four fields, CH rows) are loaded
        // before the multiply-adds, so 5*CH 16-byte loads are in flight.
        constexpr int ROWS = (M + 31) / 32;
        constexpr int CH = ROWS < 3 ? ROWS : 3;
        constexpr int NCH = (ROWS + CH - 1) / CH;
        const int p = threadIdx.x & 7, r0 = threadIdx.x >> 3;
#pragma unroll 1
        for (int ch = 0; ch < NCH; ++ch) {
            float4 a[4][CH], cmp[4][COMP ? CH : 1];
#pragma unroll
            for (int f = 0; f < 4; ++f)
#pragma unroll
                for (int j = 0; j < CH; ++j) a[f][j] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int f = 0; f < 4; ++f)
#pragma unroll
                for (int j = 0; j < (COMP ? CH : 1); ++j) cmp[f][j] = make_float4(0.f, 0.f, 0.f, 0.f);
            long long off[CH];
            bool ok[CH];
#pragma unroll
            for (int j = 0; j < CH; ++j) {
                const int row = r0 + 32 * (ch * CH + j);
                ok[j] = row < M;
                off[j] = col0 + (ok[j] ? row : 0) * kTileY + 2 * p;
            }
#pragma unroll 2
            for (int e = T.e0; e < T.er; ++e) {   // self pair: real kernel
                const MacEntry E = entries[e];
                long long j = step - E.lag;
                if (clamp && j < 0) j = 0;
                const float2 *S = E.ring + (j % E.depth) * E.slot_elems + sbase;
                const float *G = static_cast<const float *>(E.g);
                float2 g[CH];
                float4 s[4][CH];
#pragma unroll
                for (int jj = 0; jj < CH; ++jj) {
                    g[jj] = __ldg(reinterpret_cast<const float2 *>(G + off[jj]));
#pragma unroll
                    for (int f = 0; f < 4; ++f) s[f][jj] = ldg4(S + f * fstride + off[jj]);
                }
#pragma unroll
                for (int jj = 0; jj < CH; ++jj)
#pragma unroll
                    for (int f = 0; f < 4; ++f) {
                        if constexpr (COMP) {
                            float4 &c = cmp[f][COMP ? jj : 0];
                            kahan_add(a[f][jj].x, c.x, g[jj].x * s[f][jj].x);
                            kahan_add(a[f][jj].y, c.y, g[jj].x * s[f][jj].y);
                            kahan_add(a[f][jj].z, c.z, g[jj].y * s[f][jj].z);
                            kahan_add(a[f][jj].w, c.w, g[jj].y * s[f][jj].w);
                        } else {
                            a[f][jj].x = fmaf(g[jj].x, s[f][jj].x, a[f][jj].x);
                            a[f][jj].y = fmaf(g[jj].x, s[f][jj].y, a[f][jj].y);
                            a[f][jj].z = fmaf(g[jj].y, s[f][jj].z, a[f][jj].z);
                            a[f][jj].w = fmaf(g[jj].y, s[f][jj].w, a[f][jj].w);
                        }
                    }
            }
#pragma unroll 2
            for (int e = T.er; e < T.e1; ++e) {   // other sources: complex kernel
                const MacEntry E = entries[e];
                long long j = step - E.lag;
                if (clamp && j < 0) j = 0;
                const float2 *S = E.ring + (j % E.depth) * E.slot_elems + sbase;
                const float2 *G = static_cast<const float2 *>(E.g);
                float4 g[CH];
                float4 s[4][CH];
#pragma unroll
                for (int jj = 0; jj < CH; ++jj) {
                    g[jj] = ldg4(G + off[jj]);
#pragma unroll
                    for (int f = 0; f < 4; ++f) s[f][jj] = ldg4(S + f * fstride + off[jj]);
                }
#pragma unroll
                for (int jj = 0; jj < CH; ++jj)
#pragma unroll
                    for (int f = 0; f < 4; ++f) {
                        float4 &x = a[f][jj];
                        const float4 gg = g[jj], ss = s[f][jj];
                        if constexpr (COMP) {
                            float4 &c = cmp[f][COMP ? jj : 0];
                            kahan_add(x.x, c.x, fmaf(gg.x, ss.x, -gg.y * ss.y));
                            kahan_add(x.y, c.y, fmaf(gg.x, ss.y, gg.y * ss.x));
                            kahan_add(x.z, c.z, fmaf(gg.z, ss.z, -gg.w * ss.w));
                            kahan_add(x.w, c.w, fmaf(gg.z, ss.w, gg.w * ss.z));
                        } else {
                            x.x = fmaf(gg.x, ss.x, fmaf(-gg.y, ss.y, x.x));
                            x.y = fmaf(gg.x, ss.y, fmaf(gg.y, ss.x, x.y));
                            x.z = fmaf(gg.z, ss.z, fmaf(-gg.w, ss.w, x.z));
                            x.w = fmaf(gg.z, ss.w, fmaf(gg.w, ss.z, x.w));
                        }
                    }
            }
#pragma unroll
            for (int jj = 0; jj < CH; ++jj) {
                if (!ok[jj]) continue;
                const int row = r0 + 32 * (ch * CH + jj);
#pragma unroll
                for (int f = 0; f < 4; ++f) {
                    if constexpr (COMP) {
                        const float4 &c = cmp[f][COMP ? jj : 0];
                        a[f][jj] = make_float4(a[f][jj].x - c.x, a[f][jj].y - c.y, a[f][jj].z - c.z, a[f][jj].w - c.w);
                    }
                    float2 *d = acc + f * fs + row * kTileYPad + 2 * p;
                    d[0] = make_float2(a[f][jj].x, a[f][jj].y);
                    d[1] = make_float2(a[f][jj].z, a[f][jj].w);
                }
            }
        }
    } else {
        for (int i = threadIdx.x; i < 4 * fs; i += blockDim.x) acc[i] = make_float2(0.0f, 0.0f);
        __syncthreads();
        // Each thread owns the (kz, c) cells i = threadIdx.x + k*blockDim.x and
        // sums every entry of one cell in registers (entries in order, the
        // warp's lanes reading consecutive cells of an entry), then stores it.
        for (int i = threadIdx.x; i < mz * kTileY; i += blockDim.x) {
            const int kz = i / kTileY, c = i % kTileY;
            if (c >= ncols) continue;
            const long long off = kz * kTileY + c;
            float2 v[4], cv[4];
#pragma unroll
            for (int f = 0; f < 4; ++f) v[f] = cv[f] = make_float2(0.0f, 0.0f);
            for (int e = T.e0; e < T.e1; ++e) {
                const MacEntry E = entries[e];
                long long j = step - E.lag;
                if (clamp && j < 0) j = 0;
                const float2 *S = E.ring + (j % E.depth) * E.slot_elems + 4 * col0;
                const float2 g = E.is_real ? make_float2(__ldg(static_cast<const float *>(E.g) + col0 + off), 0.0f)
                                           : __ldg(static_cast<const float2 *>(E.g) + col0 + off);
#pragma unroll
                for (int f = 0; f < 4; ++f) {
                    const float2 t = cmul(g, __ldg(S + f * fstride + off));
                    if constexpr (COMP) {
                        kahan_add(v[f].x, cv[f].x, t.x);
                        kahan_add(v[f].y, cv[f].y, t.y);
                    } else {
                        v[f] = cadd(v[f], t);
                    }
                }
            }
            const int a_ = kz * kTileYPad + c;
#pragma unroll
            for (int f = 0; f < 4; ++f) acc[f * fs + a_] = COMP ? make_float2(v[f].x - cv[f].x, v[f].y - cv[f].y) : v[f];
        }
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    LaneTw<lane_class(M), true> lt;
    if constexpr (M > 0) lt.init(tw, lane & (az.L - 1));
    ColumnFFT<M, true> cf{&lt, az, acc, fs, ncols, 4, T.nz, tw, lane, warp, nwarps};
    run_radix<M>(az.R, cf);
    __syncthreads();
    const int nz = T.nz;
    const long long t2_field = (long long)kx * nz * my;
    float2 *dst = T.t2 + (long long)kxi * nz * my + ky0;
    if constexpr (M > 0) {
        for (int i = threadIdx.x; i < 4 * nz * (kTileY / 2); i += blockDim.x) {
            const int f = i / (nz * (kTileY / 2)), rem = i % (nz * (kTileY / 2));
            const int zi = rem / (kTileY / 2), p = rem % (kTileY / 2);
            const float2 *s = acc + f * fs + zi * kTileYPad + 2 * p;
            *reinterpret_cast<float4 *>(dst + f * t2_field + (long long)zi * my + 2 * p) =
                make_float4(s[0].x, s[0].y, s[1].x, s[1].y);
        }
    } else {
        for (int i = threadIdx.x; i < 4 * nz * kTileY; i += blockDim.x) {
            const int f = i / (nz * kTileY), rem = i % (nz * kTileY);
            const int zi = rem / kTileY, c = rem % kTileY;
            if (c < ncols) dst[f * t2_field + (long long)zi * my + c] = acc[f * fs + zi * kTileYPad + c];
        }
    }
}

// ---------------------------------------------------------------- inverse plane pass

template <int M>
struct InvPlaneY {
    const LaneTw<lane_class(M), true> *lt;
    Axis a;
    int kx, ny;
    float2 *P;
    int ps;
    const float2 *tw;
    int lane, warp, nwarps;

    template <int RY>
    __device__ __forceinline__ void run()
    {
        const int G = 32 >> a.logL;
        const int grp = lane >> a.logL, g = lane & (a.L - 1);
        const int per_iter = nwarps * G;
        for (int base = 0; base < kx; base += per_iter) {
            const int kxi = base + warp * G + grp;
            const bool valid = kxi < kx;
            float2 *row = P + (valid ? kxi : 0) * ps;
            float2 v[RY];
#pragma unroll
            for (int n = 0; n < RY; ++n) v[n] = row[n * a.L + g];
            do_line<M, true>(v, g, a, tw, lt);
            __syncwarp();
            const int kb = bitrev_lanes(g, a.logL) * RY;
            if (valid) {
#pragma unroll
                for (int k1 = 0; k1 < RY; ++k1)
                    if (k1 + kb < ny) row[k1 + kb] = v[k1];
            }
            __syncwarp();
        }
    }
};

template <int M>
struct InvPlaneX {
    const LaneTw<lane_class(M), true> *lt;
    Axis a;
    int nx, ny;
    const float2 *P;
    int ps;
    float *O;       // [ny][nx]
    float scale;
    const float2 *tw;
    int lane, warp, nwarps;

    template <int RX>
    __device__ __forceinline__ void run()
    {
        const int G = 32 >> a.logL;
        const int grp = lane >> a.logL, g = lane & (a.L - 1);
        const int pairs = (ny + 1) >> 1;
        const int half = a.M >> 1;
        const int per_iter = nwarps * G;
        for (int base = 0; base < pairs; base += per_iter) {
            const int p = base + warp * G + grp;
            const bool valid = p < pairs;
            const int ya = valid ? 2 * p : 0, yb = ya + 1;
            const bool vb = valid && yb < ny;
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
            do_line<M, true>(v, g, a, tw, lt);
            const int kb = bitrev_lanes(g, a.logL) * RX;
            if (valid) {
#pragma unroll
                for (int k1 = 0; k1 < RX; ++k1) {
                    const int x = k1 + kb;
                    if (x < nx) {
                        O[ya * nx + x] = scale * v[k1].x;
                        if (vb) O[yb * nx + x] = scale * v[k1].y;
                    }
                }
            }
        }
    }
};

template <int M>
__global__ void __launch_bounds__(kPlaneThreads) k_inv_plane(const InvTarget *__restrict__ tgts, int t0, int t1,
                                                          int block_lo, OutPtrs out, float inv_c, long long step)
{
    extern __shared__ float4 smem_f4[];
    float2 *sm = reinterpret_cast<float2 *>(smem_f4);
    const int b = blockIdx.x + block_lo;
    const int t = owner_of(tgts, t0, t1, b, &InvTarget::plane0);
    const InvTarget &T = tgts[t];
    const Axis ax = axis_of<M>(T.ax), ay = axis_of<M>(T.ay);
    const int nx = T.nx, ny = T.ny, nz = T.nz;
    const int kx = ax.M / 2 + 1, my = ay.M;
    const int local = b - T.plane0;
    const int f = local / nz, z = local % nz;
    const int ps = my | 1;

    float2 *twx = sm;
    float2 *twy = twx + ax.M;
    float2 *P = twy + my;                                   // [kx][ps]
    float *O = reinterpret_cast<float *>(P + kx * ps);      // [ny][nx]
    load_twiddles(twx, T.tw_x, ax.M);
    load_twiddles(twy, T.tw_y, my);
    // far pairs: the target's Lagrange weights (constant) into shared memory
    // now, so that the interpolation at the end reads no global table
    const FarTarget *Fp = T.far;
    int fpx = 0, fpy = 0, fpz = 0, fr = 0, fdepth = 1;
    const float *fcring = nullptr;
    float *cz = O + nx * ny;                                // [py][px]
    float *ux = cz + kMaxFarPts * kMaxFarPts;               // [py][nx]
    float *sLx = ux + kMaxFarPts * nx;                      // [nx][px]
    float *sLy = sLx + kMaxFarPts * nx;                     // [ny][py]
    float *sLz = sLy + kMaxFarPts * ny;                     // [pz], row z
    float *sc = sLz + kMaxFarPts;                           // [r]: this step's coefficients of field f
    if (Fp) {
        fpx = Fp->px; fpy = Fp->py; fpz = Fp->pz; fr = Fp->r; fdepth = Fp->depth; fcring = Fp->cring;
        for (int i = threadIdx.x; i < nx * fpx; i += blockDim.x) sLx[i] = __ldg(Fp->Lx + i);
        for (int i = threadIdx.x; i < ny * fpy; i += blockDim.x) sLy[i] = __ldg(Fp->Ly + i);
        for (int i = threadIdx.x; i < fpz; i += blockDim.x) sLz[i] = __ldg(Fp->Lz + z * fpz + i);
    }
    pdl_trigger();
    pdl_wait();   // T2 is written by the MAC, the coefficient ring by the far scatter or the learned field
    if (step < 0) step = *T.d_step;   // graph replay: the step from the device counter
    const float2 *src = T.t2 + ((long long)f * kx * nz + z) * my;
    const long long row_stride = (long long)nz * my;
    if constexpr (M > 0) {
        for (int i = threadIdx.x; i < kx * (M / 2); i += blockDim.x) {
            const int kxi = i / (M / 2), q = i % (M / 2);
            const float4 v = ldg4(src + kxi * row_stride + 2 * q);
            P[kxi * ps + 2 * q] = make_float2(v.x, v.y);
            P[kxi * ps + 2 * q + 1] = make_float2(v.z, v.w);
        }
    } else {
        for (int i = threadIdx.x; i < kx * my; i += blockDim.x) {
            const int kxi = i / my, ky = i % my;
            P[kxi * ps + ky] = src[kxi * row_stride + ky];
        }
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    LaneTw<lane_class(M), true> lt;
    if constexpr (M > 0) lt.init(twx, lane & (ax.L - 1));
    InvPlaneY<M> py{&lt, ay, kx, ny, P, ps, twy, lane, warp, nwarps};
    run_radix<M>(ay.R, py);
    __syncthreads();
    InvPlaneX<M> px{&lt, ax, nx, ny, P, ps, O, f == 0 ? 1.0f : inv_c, twx, lane, warp, nwarps};
    run_radix<M>(ax.R, px);
    __syncthreads();
    const long long N = (long long)nx * ny * nz;
    float *dst = (f == 0 ? out.phi[T.dom] : out.A[T.dom] + (long long)(f - 1) * N) + (long long)z * nx * ny;
    if (!Fp) {
        for (int i = threadIdx.x; i < nx * ny; i += blockDim.x) dst[i] = O[i];
        return;
    }
    // far pairs: tensor-product Lagrange interpolation of this step's node
    // coefficients (field f), contracted over z first
    const float *c = fcring + (step % fdepth) * (fr * 4);
    for (int i = threadIdx.x; i < fr; i += blockDim.x) sc[i] = c[i * 4 + f];
    __syncthreads();
    const int pxy = fpx * fpy;
    for (int i = threadIdx.x; i < pxy; i += blockDim.x) {
        float s = 0.0f;
        for (int cc = 0; cc < fpz; ++cc) s = fmaf(sLz[cc], sc[cc * pxy + i], s);
        cz[i] = s;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < fpy * nx; i += blockDim.x) {
        const int bb = i / nx, x = i % nx;
        float u = 0.0f;
        for (int aa = 0; aa < fpx; ++aa) u = fmaf(sLx[x * fpx + aa], cz[bb * fpx + aa], u);
        ux[i] = u;
    }
    __syncthreads();
    const float scale = f == 0 ? 1.0f : inv_c;
    for (int i = threadIdx.x; i < nx * ny; i += blockDim.x) {
        const int x = i % nx, y = i / nx;
        float v = 0.0f;
        for (int bb = 0; bb < fpy; ++bb) v = fmaf(sLy[y * fpy + bb], ux[bb * nx + x], v);
        dst[i] = fmaf(scale, v, O[i]);
    }
}

// ---------------------------------------------------------------- plane passes on tiles (M = 64, 96, 128)
//
// The plane passes on the two-stage tile transform.  Forward: the plane's
// rows in pairs (row 2c the real part of line c, row 2c + 1 the imaginary
// part) transformed along x as row lines, split into the two rows' spectra
// (Z[k] +- conj Z[M-k]), then along y as column lines over kx.  The columns
// kx = 0 and kx = M/2 of a real plane are real, so they travel as one
// complex column (kx = 0 in the real part, M/2 in the imaginary part) and are
// split after the y transform: the y pass is M/32 whole tiles.  Inverse: the
// same steps in reverse order, the rows kx = 0 and M/2 packed as S_0 + i S_M/2
// (their transforms along y are real up to rounding), and the C2R transform
// along x as one complex transform per pair of output rows.  A class runs
// these while its planes fit in about one wave (plane_tile_form: 3 blocks of
// 256 threads per SM); over many waves the lane-shuffle passes, with twice
// the blocks per SM, finish first.
constexpr int kPlane16Threads = 256;

__host__ __device__ constexpr bool plane16_class(int M) { return M == 64 || M == 96 || M == 128; }
__host__ __device__ constexpr int plane16_xtiles(int ny) { return ((ny + 1) / 2 + 15) / 16; }

// 4-byte asynchronous global -> shared copy
__device__ __forceinline__ void cp_async4(void *smem, const void *gmem)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((unsigned)__cvta_generic_to_shared(smem)), "l"(gmem)
                 : "memory");
}
// 8-byte asynchronous global -> shared copy
__device__ __forceinline__ void cp_async8(void *smem, const void *gmem)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((unsigned)__cvta_generic_to_shared(smem)), "l"(gmem)
                 : "memory");
}

template <int M>
__global__ void __launch_bounds__(kPlane16Threads, 3) k_fwd_plane16(const FwdRing *__restrict__ rings, IoPtrs in, int r0,
                                                                 int r1, int block_lo, int far_slot)
{
    constexpr int B = M / 16, H = M / 2, SX = M + 1, SQ = H + 1;
    static_assert(plane16_class(M), "k_fwd_plane16: M = 64, 96 or 128");
    extern __shared__ float4 smem_f4[];
    float2 *sm = reinterpret_cast<float2 *>(smem_f4);
    const int b = blockIdx.x + block_lo;
    const int r = owner_of(rings, r0, r1, b, &FwdRing::plane0);
    const FwdRing &R = rings[r];
    const int nx = R.nx, ny = R.ny, nz = R.nz;
    const int local = b - R.plane0;
    const int f = local / nz, z = local % nz;
    const long long N = (long long)nx * ny * nz;
    const int pairs = (ny + 1) >> 1, xt = (pairs + 15) >> 4;
    float2 *twx = sm, *twy = sm + M;
    float2 *X = twy + M;            // x pass: line c (rows 2c, 2c + 1) at X + c * SX
    float2 *Q = X + xt * 16 * SX;   // y pass: [M rows y][SQ]; column 0 = kx 0 and H, column k = kx k
    load_twiddles(twx, R.tw_x, M);
    load_twiddles(twy, R.tw_y, M);
    pdl_trigger();
    pdl_wait();   // the input slice may come from the previous kernel; t1 was read by it
    const float *src = f == 0 ? in.rho[R.src] : in.J[R.src] + (long long)(f - 1) * N;
    const float *plane = src + (long long)z * nx * ny;
    float *Xf = reinterpret_cast<float *>(X);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (int y = warp; y < ny; y += nwarps)
        for (int x = lane; x < nx; x += 32) cp_async4(Xf + 2 * ((y >> 1) * SX + x) + (y & 1), plane + y * nx + x);
    if (ny & 1)
        for (int x = threadIdx.x; x < nx; x += blockDim.x) Xf[2 * ((ny >> 1) * SX + x) + 1] = 0.0f;
    cp_async_wait_all();
    __syncthreads();
    if (nx <= H) tiles_fft_block<B, false, true, 1, SX>(X, 16 * SX, xt, twx, nx);
    else tiles_fft_block<B, false, false, 1, SX>(X, 16 * SX, xt, twx, nx);
    // two real rows from one complex transform:
    //   A[k] = (Z[k] + conj Z[M-k]) / 2,  B[k] = (Z[k] - conj Z[M-k]) / (2i)
    for (int i = threadIdx.x; i < pairs * H; i += blockDim.x) {
        const int c = i / H, k = i - c * H;
        const float2 *L = X + c * SX;
        const int ya = 2 * c, yb = ya + 1;
        if (k == 0) {
            const float2 z0 = L[tile_row<B>(0)], zh = L[tile_row<B>(H)];
            Q[ya * SQ] = make_float2(z0.x, zh.x);
            if (yb < ny) Q[yb * SQ] = make_float2(z0.y, zh.y);
        } else {
            const float2 zk = L[tile_row<B>(k)], zc = cconj(L[tile_row<B>(M - k)]);
            const float2 D = csub(zk, zc);
            Q[ya * SQ + k] = cscale(cadd(zk, zc), 0.5f);
            if (yb < ny) Q[yb * SQ + k] = make_float2(0.5f * D.y, -0.5f * D.x);
        }
    }
    __syncthreads();
    if (ny <= H) tiles_fft_block<B, false, true, SQ, 1>(Q, 16, H / 16, twy, ny);
    else tiles_fft_block<B, false, false, SQ, 1>(Q, 16, H / 16, twy, ny);
    // rows kx of T1 (ky natural), kx = 0 and H split from the packed column
    float2 *out = R.t1 + ((long long)f * (H + 1) * nz + z) * M;
    const long long rs = (long long)nz * M;
    for (int kxi = warp; kxi <= H; kxi += nwarps) {
        float2 *row = out + kxi * rs;
        if (kxi > 0 && kxi < H) {
            for (int ky = 2 * lane; ky < M; ky += 64) {
                const float2 a = Q[tile_row<B>(ky) * SQ + kxi], c = Q[tile_row<B>(ky + 1) * SQ + kxi];
                *reinterpret_cast<float4 *>(row + ky) = make_float4(a.x, a.y, c.x, c.y);
            }
        } else {
            for (int ky = lane; ky < M; ky += 32) {
                const float2 zk = Q[tile_row<B>(ky) * SQ], zc = cconj(Q[tile_row<B>(ky == 0 ? 0 : M - ky) * SQ]);
                const float2 D = csub(zk, zc);
                row[ky] = kxi == 0 ? cscale(cadd(zk, zc), 0.5f) : make_float2(0.5f * D.y, -0.5f * D.x);
            }
        }
    }
    if (R.far_x) {
        // far path: this plane as bf16 hi/lo into row (slot, field) of the batch matrix
        __nv_bfloat16 *row = R.far_x + ((long long)far_slot * 4 + f) * 2 * R.far_ks + (long long)z * nx * ny;
        for (int i = threadIdx.x; i < nx * ny; i += blockDim.x) {
            const float v = __ldg(plane + i);
            const __nv_bfloat16 hi = __float2bfloat16(v);
            row[i] = hi;
            row[R.far_ks + i] = __float2bfloat16(v - __bfloat162float(hi));
        }
    }
}

template <int M>
__global__ void __launch_bounds__(kPlane16Threads, 3) k_inv_plane16(const InvTarget *__restrict__ tgts, int t0, int t1,
                                                                 int block_lo, OutPtrs out, float inv_c, long long step)
{
    constexpr int B = M / 16, H = M / 2, SP = M + 1, SX = 17;
    static_assert(plane16_class(M), "k_inv_plane16: M = 64, 96 or 128");
    extern __shared__ float4 smem_f4[];
    float2 *sm = reinterpret_cast<float2 *>(smem_f4);
    const int b = blockIdx.x + block_lo;
    const int t = owner_of(tgts, t0, t1, b, &InvTarget::plane0);
    const InvTarget &T = tgts[t];
    const int nx = T.nx, ny = T.ny, nz = T.nz;
    const int local = b - T.plane0;
    const int f = local / nz, z = local % nz;
    const int pairs = (ny + 1) >> 1, xt = (pairs + 15) >> 4;
    float2 *twx = sm, *twy = sm + M;
    float2 *P = twy + M;            // y pass: line kx (row lines, ky along), line 0 = kx 0 and H packed
    float2 *X = P + H * SP;         // x pass: [xt][M rows k][SX], 16 lines (pairs of output rows) per tile
    float *O = reinterpret_cast<float *>(P);                  // [ny][nx] output plane (P is dead by then)
    float *fw = reinterpret_cast<float *>(X + xt * M * SX);   // far weights and scratch
    load_twiddles(twx, T.tw_x, M);
    load_twiddles(twy, T.tw_y, M);
    const FarTarget *Fp = T.far;
    int fpx = 0, fpy = 0, fpz = 0, fr = 0, fdepth = 1;
    const float *fcring = nullptr;
    float *cz = fw;                                         // [py][px]
    float *ux = cz + kMaxFarPts * kMaxFarPts;               // [py][nx]
    float *sLx = ux + kMaxFarPts * nx;                      // [nx][px]
    float *sLy = sLx + kMaxFarPts * nx;                     // [ny][py]
    float *sLz = sLy + kMaxFarPts * ny;                     // [pz], row z
    float *sc = sLz + kMaxFarPts;                           // [r]: this step's coefficients of field f
    if (Fp) {
        fpx = Fp->px; fpy = Fp->py; fpz = Fp->pz; fr = Fp->r; fdepth = Fp->depth; fcring = Fp->cring;
        for (int i = threadIdx.x; i < nx * fpx; i += blockDim.x) sLx[i] = __ldg(Fp->Lx + i);
        for (int i = threadIdx.x; i < ny * fpy; i += blockDim.x) sLy[i] = __ldg(Fp->Ly + i);
        for (int i = threadIdx.x; i < fpz; i += blockDim.x) sLz[i] = __ldg(Fp->Lz + z * fpz + i);
    }
    pdl_trigger();
    pdl_wait();   // T2 is written by the MAC, the coefficient ring by the far scatter or the learned field
    if (step < 0) step = *T.d_step;   // graph replay: the step from the device counter
    const float2 *src = T.t2 + ((long long)f * (H + 1) * nz + z) * M;
    const long long rs = (long long)nz * M;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (int kxi = 1 + warp; kxi < H; kxi += nwarps)
        for (int ky = lane; ky < M; ky += 32) cp_async8(P + kxi * SP + ky, src + kxi * rs + ky);
    for (int ky = threadIdx.x; ky < M; ky += blockDim.x) {
        const float2 a = src[ky], h = src[H * rs + ky];
        P[ky] = make_float2(a.x - h.y, a.y + h.x);   // S_0 + i S_H
    }
    cp_async_wait_all();
    __syncthreads();
    tiles_fft_block<B, true, false, 1, SP>(P, 16 * SP, H / 16, twy, M);
    // x-pass input of the pair (ya, yb): A + iB over k < M, from the rows'
    // half spectra (kx = 0 and H real: the real and imaginary parts of line 0)
    for (int c = warp; c < pairs; c += nwarps)
        for (int k = lane; k < M; k += 32) {
        const int ya = 2 * c, yb = ya + 1;
        const bool vb = yb < ny;
        const int kk = k <= H ? k : M - k;
        float2 A, Bv;
        if (kk == 0 || kk == H) {
            const float2 pa = P[tile_row<B>(ya)], pb = vb ? P[tile_row<B>(yb)] : make_float2(0.0f, 0.0f);
            A = make_float2(kk == 0 ? pa.x : pa.y, 0.0f);
            Bv = make_float2(kk == 0 ? pb.x : pb.y, 0.0f);
        } else {
            const float2 *L = P + kk * SP;
            A = L[tile_row<B>(ya)];
            Bv = vb ? L[tile_row<B>(yb)] : make_float2(0.0f, 0.0f);
            if (k > H) { A = cconj(A); Bv = cconj(Bv); }
        }
        X[(c >> 4) * M * SX + k * SX + (c & 15)] = make_float2(A.x - Bv.y, A.y + Bv.x);
        }
    __syncthreads();
    tiles_fft_block<B, true, false, SX, 1>(X, M * SX, xt, twx, M);
    const long long Nt = (long long)nx * ny * nz;
    float *dst = (f == 0 ? out.phi[T.dom] : out.A[T.dom] + (long long)(f - 1) * Nt) + (long long)z * nx * ny;
    const float scale = f == 0 ? 1.0f : inv_c;
    float *O_or_dst = Fp ? O : dst;
    for (int y = warp; y < ny; y += nwarps) {
        const int c = y >> 1;
        const float2 *L = X + (c >> 4) * M * SX + (c & 15);
        for (int x = lane; x < nx; x += 32) {
            const float2 v = L[tile_row<B>(x) * SX];
            O_or_dst[y * nx + x] = scale * ((y & 1) ? v.y : v.x);
        }
    }
    if (!Fp) return;
    // far pairs: tensor-product Lagrange interpolation of this step's node
    // coefficients (field f), contracted over z first
    const float *c = fcring + (step % fdepth) * (fr * 4);
    for (int i = threadIdx.x; i < fr; i += blockDim.x) sc[i] = c[i * 4 + f];
    __syncthreads();
    const int pxy = fpx * fpy;
    for (int i = threadIdx.x; i < pxy; i += blockDim.x) {
        float s = 0.0f;
        for (int cc = 0; cc < fpz; ++cc) s = fmaf(sLz[cc], sc[cc * pxy + i], s);
        cz[i] = s;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < fpy * nx; i += blockDim.x) {
        const int bb = i / nx, x = i % nx;
        float u = 0.0f;
        for (int aa = 0; aa < fpx; ++aa) u = fmaf(sLx[x * fpx + aa], cz[bb * fpx + aa], u);
        ux[i] = u;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nx * ny; i += blockDim.x) {
        const int x = i % nx, y = i / nx;
        float v = 0.0f;
        for (int bb = 0; bb < fpy; ++bb) v = fmaf(sLy[y * fpy + bb], ux[bb * nx + x], v);
        dst[i] = fmaf(scale, v, O[i]);
    }
}

// ---------------------------------------------------------------- inverse plane pass for M = 192, in chunks
//
// At M = 192 a plane of spectra (97 lines of 192) takes 150 KB of shared
// memory, so the lane-shuffle pass runs one block per SM.  This one runs the
// tile transform through a single work tile in chunks of 16 lines: along y,
// 16 kx lines at a time (kx = 0 and M/2 packed as one line, as in
// k_inv_plane16), keeping only the rows y < ny of each in a compact buffer Y
// (odd line stride: no bank conflicts); then along x, 16 pairs of output rows
// at a time, each row written out with the far coefficients' interpolation
// added (no output plane in shared memory).  About 109 KB per block: two
// blocks per SM.
constexpr int kPlaneBigThreads = 256;

__host__ __device__ constexpr int plane_big_ystride(int ny) { return ny | 1; }

template <int M>
__global__ void __launch_bounds__(kPlaneBigThreads, 2) k_inv_plane_big(const InvTarget *__restrict__ tgts, int t0,
                                                                       int t1, int block_lo, OutPtrs out, float inv_c,
                                                                       long long step)
{
    constexpr int B = M / 16, H = M / 2, SW = M + 1, SX = 17;
    static_assert(M == 192, "k_inv_plane_big: M = 192");
    extern __shared__ float4 smem_f4[];
    float2 *sm = reinterpret_cast<float2 *>(smem_f4);
    const int b = blockIdx.x + block_lo;
    const int t = owner_of(tgts, t0, t1, b, &InvTarget::plane0);
    const InvTarget &T = tgts[t];
    const int nx = T.nx, ny = T.ny, nz = T.nz;
    const int local = b - T.plane0;
    const int f = local / nz, z = local % nz;
    const int pairs = (ny + 1) >> 1, SY = plane_big_ystride(ny);
    float2 *twx = sm, *twy = sm + M;
    float2 *Y = twy + M;                                  // [H lines][SY]: rows y < ny of the y transform
    float2 *W = Y + H * SY;                               // work tile: 16 row lines of SW, or M rows of SX
    float *ux = reinterpret_cast<float *>(W + M * SX);    // far: [py][nx]
    float *sc = ux + kMaxFarPts * nx;                     // far: [r], this step's coefficients of field f
    float *cz = sc + kMaxFarPts * kMaxFarPts * kMaxFarPts;   // far: [py][px]
    load_twiddles(twx, T.tw_x, M);
    load_twiddles(twy, T.tw_y, M);
    pdl_trigger();
    pdl_wait();   // T2 is written by the MAC, the coefficient ring by the far path
    if (step < 0) step = *T.d_step;   // graph replay: the step from the device counter
    const float2 *src = T.t2 + ((long long)f * (H + 1) * nz + z) * M;
    const long long rs = (long long)nz * M;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    __syncthreads();
    // along y, 16 kx lines per chunk; only the rows y < ny are kept
    for (int ch = 0; ch < H / 16; ++ch) {
        for (int l = warp; l < 16; l += nwarps) {
            const int kxi = 16 * ch + l;
            float2 *L = W + l * SW;
            if (kxi == 0) {
                for (int ky = lane; ky < M; ky += 32) {
                    const float2 a = src[ky], h = src[H * rs + ky];
                    L[ky] = make_float2(a.x - h.y, a.y + h.x);   // S_0 + i S_H
                }
            } else {
                for (int ky = lane; ky < M; ky += 32) cp_async8(L + ky, src + kxi * rs + ky);
            }
        }
        cp_async_wait_all();
        __syncthreads();
        tiles_fft_block<B, true, false, 1, SW>(W, 16 * SW, 1, twy, M);   // ends synchronised
        for (int i = threadIdx.x; i < 16 * ny; i += blockDim.x) {
            const int l = i & 15, y = i >> 4;
            Y[(16 * ch + l) * SY + y] = W[l * SW + tile_row<B>(y)];
        }
        __syncthreads();
    }
    // far pairs: this step's node coefficients of field f contracted over z,
    // then over x (the weights read from global memory)
    const FarTarget *Fp = T.far;
    if (Fp) {
        const int px = Fp->px, py = Fp->py, pz = Fp->pz, r = Fp->r, pxy = px * py;
        const float *c = Fp->cring + (step % Fp->depth) * (r * 4);
        for (int i = threadIdx.x; i < r; i += blockDim.x) sc[i] = c[i * 4 + f];
        __syncthreads();
        for (int i = threadIdx.x; i < pxy; i += blockDim.x) {
            float s = 0.0f;
            for (int cc = 0; cc < pz; ++cc) s = fmaf(__ldg(Fp->Lz + z * pz + cc), sc[cc * pxy + i], s);
            cz[i] = s;
        }
        __syncthreads();
        for (int i = threadIdx.x; i < py * nx; i += blockDim.x) {
            const int bb = i / nx, x = i % nx;
            float u = 0.0f;
            for (int aa = 0; aa < px; ++aa) u = fmaf(__ldg(Fp->Lx + x * px + aa), cz[bb * px + aa], u);
            ux[i] = u;
        }
    }
    // along x (C2R), 16 pairs of output rows per chunk
    const long long Nt = (long long)nx * ny * nz;
    float *dst = (f == 0 ? out.phi[T.dom] : out.A[T.dom] + (long long)(f - 1) * Nt) + (long long)z * nx * ny;
    const float scale = f == 0 ? 1.0f : inv_c;
    for (int c0 = 0; c0 < pairs; c0 += 16) {
        for (int i = threadIdx.x; i < 16 * M; i += blockDim.x) {
            const int k = i % M, cc = i / M, c = c0 + cc;
            float2 v = make_float2(0.0f, 0.0f);
            if (c < pairs) {
                const int ya = 2 * c, yb = ya + 1;
                const bool vb = yb < ny;
                const int kk = k <= H ? k : M - k;
                float2 A, Bv;
                if (kk == 0 || kk == H) {   // the real rows kx = 0 and H: parts of line 0
                    const float2 pa = Y[ya], pb = vb ? Y[yb] : make_float2(0.0f, 0.0f);
                    A = make_float2(kk == 0 ? pa.x : pa.y, 0.0f);
                    Bv = make_float2(kk == 0 ? pb.x : pb.y, 0.0f);
                } else {
                    A = Y[kk * SY + ya];
                    Bv = vb ? Y[kk * SY + yb] : make_float2(0.0f, 0.0f);
                    if (k > H) { A = cconj(A); Bv = cconj(Bv); }
                }
                v = make_float2(A.x - Bv.y, A.y + Bv.x);   // A + iB
            }
            W[k * SX + cc] = v;
        }
        __syncthreads();
        tiles_fft_block<B, true, false, SX, 1>(W, M * SX, 1, twx, M);   // ends synchronised
        const int rows = min(32, ny - 2 * c0);
        for (int i = threadIdx.x; i < rows * nx; i += blockDim.x) {
            const int yy = i / nx, x = i - yy * nx, y = 2 * c0 + yy;
            const float2 v = W[tile_row<B>(x) * SX + (yy >> 1)];
            float o = scale * ((yy & 1) ? v.y : v.x);
            if (Fp) {
                float s = 0.0f;
                for (int bb = 0; bb < Fp->py; ++bb) s = fmaf(__ldg(Fp->Ly + y * Fp->py + bb), ux[bb * nx + x], s);
                o = fmaf(scale, s, o);
            }
            dst[y * nx + x] = o;
        }
        __syncthreads();
    }
}
#define RP_FOR_EACH_CLASS(X) X(0) X(32) X(48) X(64) X(96) X(128) X(192)

}  // namespace

// ---------------------------------------------------------------- host side

int size_class(const Axis &ax, const Axis &ay, const Axis &az)
{
    if (ax.M != ay.M || ax.M != az.M) return 0;
    switch (ax.M) {
    case 32: case 48: case 64: case 96: case 128: case 192: return ax.M;
    default: return 0;
    }
}

bool plane_tile_class(int size_class) { return plane16_class(size_class); }

size_t smem_fwd_plane(int cls, bool tile, int ny, const Axis &ax)
{
    if (tile && plane16_class(cls)) {
        const size_t M = cls;
        return sizeof(float2) * (2 * M + (size_t)plane16_xtiles(ny) * 16 * (M + 1) + M * (M / 2 + 1));
    }
    const int kx = ax.M / 2 + 1;
    const int qs = kx | 1;
    // twiddles (x and y, bounded by kMaxFFT each) + Q + per-group scratch
    return sizeof(float2) * (2 * kMaxFFT + (size_t)ny * qs + (size_t)(kPlaneThreads / 32) * 32 * ax.R);
}

size_t smem_fwd_column(const Axis &az) { return sizeof(float2) * ((size_t)az.M + 4 * (size_t)az.M * kTileYPad); }

static size_t smem_fwd_column16(int M) { return sizeof(float2) * ((size_t)M + 4 * (size_t)M * kTileY); }

size_t smem_mac_inv_column(const Axis &az)
{
    return sizeof(float2) * ((size_t)az.M + 4 * (size_t)az.M * kTileYPad);
}

size_t smem_inv_plane(int cls, bool tile, int nx, int ny, const Axis &ax, const Axis &ay)
{
    if (cls == 192) {   // k_inv_plane_big, whatever the form flag
        const size_t M = 192;
        return sizeof(float2) * (2 * M + (M / 2) * (size_t)plane_big_ystride(ny) + M * 17) +
               sizeof(float) * ((size_t)kMaxFarPts * nx + kMaxFarPts * kMaxFarPts * kMaxFarPts + kMaxFarPts * kMaxFarPts);
    }
    if (tile && plane16_class(cls)) {
        const size_t M = cls;
        return sizeof(float2) * (2 * M + (M / 2) * (M + 1) + (size_t)plane16_xtiles(ny) * M * 17) +
               sizeof(float) * kMaxFarPts * (kMaxFarPts + 2 * (size_t)nx + ny + 1 + kMaxFarPts * kMaxFarPts);
    }
    const int kx = ax.M / 2 + 1;
    const int ps = ay.M | 1;
    // + the far path: coefficients contracted over z, then over x; the
    // Lagrange weights per axis; this step's node coefficients
    return sizeof(float2) * ((size_t)ax.M + ay.M + (size_t)kx * ps) + sizeof(float) * (size_t)nx * ny +
           sizeof(float) * kMaxFarPts * (kMaxFarPts + 2 * (size_t)nx + ny + 1 + kMaxFarPts * kMaxFarPts);
}

// The dynamic shared-memory limit is an attribute of the kernel function,
// shared by every context in the process, so each kernel is opened up to the
// device's opt-in maximum once (contexts never lower it for one another).
// Each size class opens the kernels it runs: the tile-transform passes where
// the class has them, the lane-shuffle passes elsewhere.
template <int M>
static cudaError_t open_class_smem(int max_optin)
{
    cudaError_t e;
    const auto open = [&](auto kern) { return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                                    max_optin); };
    if constexpr (plane16_class(M))
        if ((e = open(k_fwd_plane16<M>)) || (e = open(k_inv_plane16<M>))) return e;
    if ((e = open(k_fwd_plane<M>))) return e;
    if constexpr (M == 192) {
        if ((e = open(k_inv_plane_big<M>))) return e;
    } else {
        if ((e = open(k_inv_plane<M>))) return e;
    }
    if constexpr (tile16_class(M)) {
        if ((e = open(k_fwd_column16<M>))) return e;
    } else {
        if ((e = open(k_fwd_column<M>))) return e;
    }
    if ((e = open(k_mac_inv_column<M, false>)) || (e = open(k_mac_inv_column<M, true>))) return e;
    return cudaSuccess;
}

cudaError_t open_kernel_smem_limits(int max_optin)
{
    cudaError_t e;
#define RP_OPEN(M) \
    if ((e = open_class_smem<M>(max_optin))) return e;
    RP_FOR_EACH_CLASS(RP_OPEN)
#undef RP_OPEN
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

#define RP_CASE(M, KERNEL, THREADS, ...) \
    case M: if (cudaError_t e_ = launch_pdl(KERNEL<M>, dim3(nblocks), dim3(THREADS), smem, s, __VA_ARGS__)) return e_; break;

template <int M>
static cudaError_t launch_fwd_plane_cls(bool tile, const FwdRing *d_rings, const IoPtrs &in, int r0, int r1,
                                        int block_lo, int nblocks, size_t smem, int far_slot, cudaStream_t s)
{
    if constexpr (plane16_class(M))
        if (tile)
            return launch_pdl(k_fwd_plane16<M>, dim3(nblocks), dim3(kPlane16Threads), smem, s, d_rings, in, r0, r1,
                              block_lo, far_slot);
    return launch_pdl(k_fwd_plane<M>, dim3(nblocks), dim3(kPlaneThreads), smem, s, d_rings, in, r0, r1, block_lo,
                      far_slot);
}

template <int M>
static cudaError_t launch_inv_plane_cls(bool tile, const InvTarget *d_tgts, int t0, int t1, int block_lo,
                                        const OutPtrs &out, int nblocks, size_t smem, float inv_c, long long step,
                                        cudaStream_t s)
{
    if constexpr (plane16_class(M))
        if (tile)
            return launch_pdl(k_inv_plane16<M>, dim3(nblocks), dim3(kPlane16Threads), smem, s, d_tgts, t0, t1,
                              block_lo, out, inv_c, step);
    if constexpr (M == 192)
        return launch_pdl(k_inv_plane_big<M>, dim3(nblocks), dim3(kPlaneBigThreads), smem, s, d_tgts, t0, t1,
                          block_lo, out, inv_c, step);
    else
        return launch_pdl(k_inv_plane<M>, dim3(nblocks), dim3(kPlaneThreads), smem, s, d_tgts, t0, t1, block_lo, out,
                          inv_c, step);
}

cudaError_t launch_fwd_plane(int cls, bool tile, const FwdRing *d_rings, const IoPtrs &in, int r0, int r1,
                             int block_lo, int nblocks, size_t smem, int far_slot, cudaStream_t s)
{
    if (nblocks <= 0) return cudaSuccess;
    switch (cls) {
#define X(M)                                                                                                    \
    case M:                                                                                                     \
        if (cudaError_t e_ = launch_fwd_plane_cls<M>(tile, d_rings, in, r0, r1, block_lo, nblocks, smem, far_slot, s)) \
            return e_;                                                                                          \
        break;
        RP_FOR_EACH_CLASS(X)
#undef X
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <int M>
static cudaError_t launch_fwd_column_cls(const FwdRing *d_rings, int r0, int r1, int block_lo, int nblocks,
                                         size_t smem, long long step, cudaStream_t s)
{
    if constexpr (tile16_class(M))
        return launch_pdl(k_fwd_column16<M>, dim3(nblocks), dim3(kColumn16Threads), smem_fwd_column16(M), s, d_rings,
                          r0, r1, block_lo, step);
    else
        return launch_pdl(k_fwd_column<M>, dim3(nblocks), dim3(kColumnThreads), smem, s, d_rings, r0, r1, block_lo,
                          step);
}

cudaError_t launch_fwd_column(int cls, const FwdRing *d_rings, int r0, int r1, int block_lo, int nblocks,
                              size_t smem, long long step, cudaStream_t s)
{
    if (nblocks <= 0) return cudaSuccess;
    switch (cls) {
#define X(M)                                                                                        \
    case M:                                                                                         \
        if (cudaError_t e_ = launch_fwd_column_cls<M>(d_rings, r0, r1, block_lo, nblocks, smem, step, s)) \
            return e_;                                                                              \
        break;
        RP_FOR_EACH_CLASS(X)
#undef X
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_mac_inv_column(int cls, bool comp, const InvTarget *d_tgts, int t0, int t1, int block_lo,
                                  const MacEntry *d_entries, int nblocks, size_t smem, long long step, int clamp,
                                  cudaStream_t s)
{
    if (nblocks <= 0) return cudaSuccess;
    switch (cls) {
#define X(M)                                                                                                   \
    case M:                                                                                                    \
        if (cudaError_t e_ = launch_pdl(comp ? k_mac_inv_column<M, true> : k_mac_inv_column<M, false>,        \
                                        dim3(nblocks), dim3(kThreads), smem, s, d_tgts, t0, t1, block_lo,      \
                                        d_entries, step, clamp))                                               \
            return e_;                                                                                         \
        break;
        RP_FOR_EACH_CLASS(X)
#undef X
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_inv_plane(int cls, bool tile, const InvTarget *d_tgts, int t0, int t1, int block_lo,
                             const OutPtrs &out, int nblocks, size_t smem, float inv_c, long long step, cudaStream_t s)
{
    if (nblocks <= 0) return cudaSuccess;
    switch (cls) {
#define X(M)                                                                                                      \
    case M:                                                                                                       \
        if (cudaError_t e_ = launch_inv_plane_cls<M>(tile, d_tgts, t0, t1, block_lo, out, nblocks, smem, inv_c, step, s)) \
            return e_;                                                                                            \
        break;
        RP_FOR_EACH_CLASS(X)
#undef X
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace rp
