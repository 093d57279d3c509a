// Device building blocks of the FFT path: complex helpers, the lane-shuffle
// line FFT and the two-stage shared-memory tile transform (further below).
//
// A line of length M = R * L is transformed by L lanes of one warp (several
// lines share a warp when L < 32).  Lane g holds x[n*L + g] for n < R in
// registers.  With n = n1*L + n2 and k = k1 + R*k2,
//
//   X[k1 + R k2] = sum_{n2} W_L^{n2 k2} [ W_M^{n2 k1} sum_{n1} x[n1 L + n2] W_R^{n1 k1} ],
//
// so each lane first does an R-point DFT over its registers, multiplies by
// W_M^{g k1}, and the lanes then do an L-point decimation-in-frequency FFT
// across the lane group with __shfl_xor_sync butterflies.  Lane g ends up
// holding X[k1 + R * bitrev_L(g)] in register k1.
#pragma once

#include <cuda_runtime.h>

#include "rp_internal.h"

namespace rp {

// Programmatic dependent launch: the per-step kernels are launched so that
// they may start while the previous kernel of the stream finishes.  Each
// calls pdl_wait() -- which returns once that kernel has completed and its
// writes are visible -- before it touches memory the previous kernels write
// or read; what comes before (shared-memory setup, constant tables) overlaps
// with their tail.  pdl_trigger() lets the next kernel be scheduled as soon as
// every block of this one has started.  Both are no-ops for a kernel launched
// without the attribute.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Host side: launch `kernel` with programmatic stream serialization.
template <class... KArgs, class... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

__host__ __device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__host__ __device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__host__ __device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }

// W_M^j (forward) or its conjugate (inverse) from a table of exp(-2 pi i j/M).
template <bool INV>
__host__ __device__ __forceinline__ float2 twid(const float2 *tw, int j)
{
    float2 w = tw[j];
    if (INV) w.y = -w.y;
    return w;
}

__device__ __forceinline__ int bitrev_lanes(int g, int logL)
{
    return logL == 0 ? 0 : (int)(__brev((unsigned)g) >> (32 - logL));
}

// In-register R-point DFT (twiddles W_R^j = W_M^{j L} from the M table).
template <int R, bool INV>
__device__ __forceinline__ void small_dft(float2 (&v)[R], const float2 *tw, int L)
{
    if constexpr (R == 2) {
        float2 a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    } else if constexpr (R == 4) {
        // radix 4: W_4 = -i (forward) / +i (inverse)
        float2 a0 = cadd(v[0], v[2]), a1 = csub(v[0], v[2]);
        float2 b0 = cadd(v[1], v[3]), b1 = csub(v[1], v[3]);
        float2 jb1 = INV ? make_float2(-b1.y, b1.x) : make_float2(b1.y, -b1.x);  // W_4 * b1
        v[0] = cadd(a0, b0);
        v[2] = csub(a0, b0);
        v[1] = cadd(a1, jb1);
        v[3] = csub(a1, jb1);
    } else if constexpr (R > 2) {
        float2 o[R];
#pragma unroll
        for (int k = 0; k < R; ++k) {
            float2 acc = v[0];
#pragma unroll
            for (int n = 1; n < R; ++n) acc = cadd(acc, cmul(v[n], twid<INV>(tw, ((n * k) % R) * L)));
            o[k] = acc;
        }
#pragma unroll
        for (int k = 0; k < R; ++k) v[k] = o[k];
    }
}

// The line FFT described above.  All 32 lanes of the warp must call it
// together (the shuffles use the full mask); g is the lane index within its
// group of L lanes.
template <int R, bool INV>
__device__ __forceinline__ void line_fft(float2 (&v)[R], int g, const Axis &a, const float2 *tw)
{
    small_dft<R, INV>(v, tw, a.L);
#pragma unroll
    for (int k = 1; k < R; ++k) v[k] = cmul(v[k], twid<INV>(tw, g * k));
    for (int h = a.L >> 1; h >= 1; h >>= 1) {
        const bool upper = (g & h) != 0;
        const float2 w = twid<INV>(tw, (g & (h - 1)) * (a.M / (2 * h)));
#pragma unroll
        for (int k = 0; k < R; ++k) {
            float2 p;
            p.x = __shfl_xor_sync(0xffffffffu, v[k].x, h);
            p.y = __shfl_xor_sync(0xffffffffu, v[k].y, h);
            v[k] = upper ? cmul(csub(p, v[k]), w) : cadd(v[k], p);
        }
    }
}

// ---------------------------------------------------------------- compiled-size line FFT
//
// The same transform for a length M known at compile time.  The twiddles a
// lane needs (W_M^{g k} for its R registers, and one multiplier per lane
// butterfly stage) are read once per kernel into a LaneTw, and the R-point
// DFTs are written out as butterflies.

__host__ __device__ constexpr int lane_radix(int M)
{
    return M % 3 == 0 ? (M / 3 <= 32 ? 3 : 6) : (M <= 32 ? 1 : M / 32);
}
__host__ __device__ constexpr int lane_count(int M) { return M / lane_radix(M); }
__host__ __device__ constexpr int lane_log2(int x) { return x <= 1 ? 0 : 1 + lane_log2(x / 2); }

constexpr float kSin60 = 0.866025403784438647f;   // sqrt(3)/2

template <int M, bool INV>
struct LaneTw {
    static constexpr int R = lane_radix(M), L = lane_count(M), LOGL = lane_log2(L);
    float2 b[R > 1 ? R - 1 : 1];        // W_M^{g k}, k = 1..R-1
    float2 s[LOGL > 0 ? LOGL : 1];      // stage h = L/2 >> i: w for upper lanes, 1 for lower
    float sg[LOGL > 0 ? LOGL : 1];      // -1 for upper lanes, +1 for lower

    __device__ __forceinline__ void init(const float2 *tw, int g)
    {
#pragma unroll
        for (int k = 1; k < R; ++k) b[k - 1] = twid<INV>(tw, g * k);
#pragma unroll
        for (int i = 0; i < LOGL; ++i) {
            const int h = (L >> 1) >> i;
            const bool upper = (g & h) != 0;
            s[i] = upper ? twid<INV>(tw, (g & (h - 1)) * (M / (2 * h))) : make_float2(1.0f, 0.0f);
            sg[i] = upper ? -1.0f : 1.0f;
        }
    }
};

// radix 3: W = exp(-+2 pi i/3) = -1/2 -+ i sqrt3/2
template <bool INV>
__host__ __device__ __forceinline__ void dft3(float2 &a, float2 &b, float2 &c)
{
    const float2 s = cadd(b, c), d = csub(b, c);
    const float2 m = make_float2(fmaf(-0.5f, s.x, a.x), fmaf(-0.5f, s.y, a.y));
    a = cadd(a, s);
    // forward: X1 = m - i sqrt3/2 d, X2 = m + i sqrt3/2 d (inverse: swapped)
    const float2 t = make_float2(kSin60 * d.y, -kSin60 * d.x);   // -i sqrt3/2 d
    if (INV) { b = csub(m, t); c = cadd(m, t); }
    else { b = cadd(m, t); c = csub(m, t); }
}

template <int R, bool INV>
__host__ __device__ __forceinline__ void small_dft_c(float2 (&v)[R])
{
    if constexpr (R == 2) {
        const float2 a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    } else if constexpr (R == 3) {
        dft3<INV>(v[0], v[1], v[2]);
    } else if constexpr (R == 4) {
        float2 a0 = cadd(v[0], v[2]), a1 = csub(v[0], v[2]);
        float2 b0 = cadd(v[1], v[3]), b1 = csub(v[1], v[3]);
        float2 jb1 = INV ? make_float2(-b1.y, b1.x) : make_float2(b1.y, -b1.x);
        v[0] = cadd(a0, b0);
        v[2] = csub(a0, b0);
        v[1] = cadd(a1, jb1);
        v[3] = csub(a1, jb1);
    } else if constexpr (R == 6) {
        // n = 3a + b, k = c + 2d: radix 2 over a, twiddle W_6^{bc}, radix 3 over b
        float2 y0[3], y1[3];
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            y0[b] = cadd(v[b], v[b + 3]);
            y1[b] = csub(v[b], v[b + 3]);
        }
        // W_6^1 = 1/2 -+ i sqrt3/2, W_6^2 = -1/2 -+ i sqrt3/2
        const float sgn = INV ? 1.0f : -1.0f;
        y1[1] = cmul(y1[1], make_float2(0.5f, sgn * kSin60));
        y1[2] = cmul(y1[2], make_float2(-0.5f, sgn * kSin60));
        dft3<INV>(y0[0], y0[1], y0[2]);
        dft3<INV>(y1[0], y1[1], y1[2]);
        v[0] = y0[0]; v[2] = y0[1]; v[4] = y0[2];
        v[1] = y1[0]; v[3] = y1[1]; v[5] = y1[2];
    }
}

// Lane g holds x[n L + g] in v[n]; afterwards X[k + R bitrev_L(g)] in v[k].
template <int M, bool INV>
__device__ __forceinline__ void line_fft_c(float2 (&v)[LaneTw<M, INV>::R], const LaneTw<M, INV> &t)
{
    constexpr int R = LaneTw<M, INV>::R, L = LaneTw<M, INV>::L, LOGL = LaneTw<M, INV>::LOGL;
    small_dft_c<R, INV>(v);
#pragma unroll
    for (int k = 1; k < R; ++k) v[k] = cmul(v[k], t.b[k - 1]);
#pragma unroll
    for (int i = 0; i < LOGL; ++i) {
        const int h = (L >> 1) >> i;
#pragma unroll
        for (int k = 0; k < R; ++k) {
            float2 p;
            p.x = __shfl_xor_sync(0xffffffffu, v[k].x, h);
            p.y = __shfl_xor_sync(0xffffffffu, v[k].y, h);
            const float2 u = make_float2(fmaf(t.sg[i], v[k].x, p.x), fmaf(t.sg[i], v[k].y, p.y));
            v[k] = (i == LOGL - 1) ? u : cmul(u, t.s[i]);   // last stage: w = 1
        }
    }
}

// ---------------------------------------------------------------- tile transform, M = 16 B
//
// The 16 columns of a shared-memory tile T[p * 16 + c] (row p < M, column
// c < 16, one float2 each: rows of 128 bytes) transformed in place by one
// warp.  With n = B n1 + n2 and k = k1 + 16 k2 (n1, k1 < 16; n2, k2 < B),
//
//   X[k1 + 16 k2] = sum_{n2} W_B^{n2 k2} [ W_M^{n2 k1} sum_{n1} x[B n1 + n2] W_16^{n1 k1} ].
//
// Stage 1, task (c, n2): the 16-point DFT of rows B n1 + n2 of column c, times
// W_M^{n2 k1}, written back to the rows it read (row B k1 + n2 for k1).
// Stage 2, task (c, k1): the B-point DFT of rows B k1 .. B k1 + B - 1, written
// back to the same rows.  Afterwards row tile_row<B>(k) = B (k mod 16) + k / 16
// holds X[k].  The tasks of a stage touch disjoint rows, and every warp
// access covers whole 128-byte rows, so the tile needs neither padding nor
// synchronisation inside a stage.  HALF: rows n >= M/2 are zero (a
// zero-padded input), and the first radix-4 layer skips them.

template <int B>
__host__ __device__ constexpr int tile_row(int k) { return B * (k & 15) + (k >> 4); }

constexpr float kCos8 = 0.923879532511286756f;   // cos(pi/8)
constexpr float kSin8 = 0.382683432365089772f;   // sin(pi/8)
constexpr float kRt2 = 0.707106781186547524f;    // 1/sqrt(2)

// times -i (forward) or +i (inverse)
template <bool INV>
__host__ __device__ __forceinline__ float2 mul_mi(float2 a)
{
    return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// W_16^m (forward: exp(-2 pi i m/16); inverse: its conjugate), m in {1, 2, 3, 6, 9}
template <int m, bool INV>
__host__ __device__ __forceinline__ float2 w16()
{
    const float s = INV ? -1.0f : 1.0f;
    if constexpr (m == 1) return make_float2(kCos8, -s * kSin8);
    else if constexpr (m == 2) return make_float2(kRt2, -s * kRt2);
    else if constexpr (m == 3) return make_float2(kSin8, -s * kCos8);
    else if constexpr (m == 6) return make_float2(-kRt2, -s * kRt2);
    else return make_float2(-kCos8, s * kSin8);   // m == 9
}

// radix 4 in natural order; HALF: v2 = v3 = 0
template <bool INV, bool HALF = false>
__host__ __device__ __forceinline__ void r4(float2 &v0, float2 &v1, float2 &v2, float2 &v3)
{
    if constexpr (HALF) {
        const float2 a = v0, jb = mul_mi<INV>(v1);
        v2 = csub(a, v1);
        v0 = cadd(a, v1);
        v1 = cadd(a, jb);
        v3 = csub(a, jb);
    } else {
        const float2 a0 = cadd(v0, v2), a1 = csub(v0, v2);
        const float2 b0 = cadd(v1, v3), jb1 = mul_mi<INV>(csub(v1, v3));
        v0 = cadd(a0, b0);
        v2 = csub(a0, b0);
        v1 = cadd(a1, jb1);
        v3 = csub(a1, jb1);
    }
}

// 16-point DFT in natural order (n = 4a + b, k = c + 4d: radix 4 over a,
// twiddle W_16^{bc}, radix 4 over b); HALF: x[8..15] = 0.
template <bool INV, bool HALF>
__host__ __device__ __forceinline__ void dft16(float2 (&x)[16])
{
#pragma unroll
    for (int b = 0; b < 4; ++b) r4<INV, HALF>(x[b], x[4 + b], x[8 + b], x[12 + b]);
    // x[4c + b] = U_b[c]
    x[5] = cmul(x[5], w16<1, INV>());
    x[6] = cmul(x[6], w16<2, INV>());
    x[7] = cmul(x[7], w16<3, INV>());
    x[9] = cmul(x[9], w16<2, INV>());
    x[10] = mul_mi<INV>(x[10]);
    x[11] = cmul(x[11], w16<6, INV>());
    x[13] = cmul(x[13], w16<3, INV>());
    x[14] = cmul(x[14], w16<6, INV>());
    x[15] = cmul(x[15], w16<9, INV>());
#pragma unroll
    for (int c = 0; c < 4; ++c) r4<INV>(x[4 * c], x[4 * c + 1], x[4 * c + 2], x[4 * c + 3]);
    // x[4c + d] = Y[c + 4d]
    float2 y[16];
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int d = 0; d < 4; ++d) y[c + 4 * d] = x[4 * c + d];
#pragma unroll
    for (int k = 0; k < 16; ++k) x[k] = y[k];
}

// 8-point DFT in natural order (n = 2p + q, k = k1 + 4 k2)
template <bool INV>
__host__ __device__ __forceinline__ void dft8(float2 (&x)[8])
{
    r4<INV>(x[0], x[2], x[4], x[6]);
    r4<INV>(x[1], x[3], x[5], x[7]);
    // x[2 k1 + q] = U_q[k1]; times W_8^{q k1}
    const float s = INV ? -1.0f : 1.0f;
    x[3] = cmul(x[3], make_float2(kRt2, -s * kRt2));
    x[5] = mul_mi<INV>(x[5]);
    x[7] = cmul(x[7], make_float2(-kRt2, -s * kRt2));
    float2 y[8];
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
        y[k1] = cadd(x[2 * k1], x[2 * k1 + 1]);
        y[k1 + 4] = csub(x[2 * k1], x[2 * k1 + 1]);
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = y[k];
}

// 12-point DFT in natural order (n = 3p + q, k = k1 + 4 k2)
template <bool INV>
__host__ __device__ __forceinline__ void dft12(float2 (&x)[12])
{
#pragma unroll
    for (int q = 0; q < 3; ++q) r4<INV>(x[q], x[3 + q], x[6 + q], x[9 + q]);
    // x[3 k1 + q] = U_q[k1]; times W_12^{q k1}
    const float s = INV ? -1.0f : 1.0f;
    x[4] = cmul(x[4], make_float2(kSin60, -s * 0.5f));    // W^1
    x[5] = cmul(x[5], make_float2(0.5f, -s * kSin60));    // W^2
    x[7] = cmul(x[7], make_float2(0.5f, -s * kSin60));    // W^2
    x[8] = cmul(x[8], make_float2(-0.5f, -s * kSin60));   // W^4
    x[10] = mul_mi<INV>(x[10]);                           // W^3
    x[11] = make_float2(-x[11].x, -x[11].y);              // W^6
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) dft3<INV>(x[3 * k1], x[3 * k1 + 1], x[3 * k1 + 2]);
    float2 y[12];
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1)
#pragma unroll
        for (int k2 = 0; k2 < 3; ++k2) y[k1 + 4 * k2] = x[3 * k1 + k2];
#pragma unroll
    for (int k = 0; k < 12; ++k) x[k] = y[k];
}

template <int B, bool INV>
__host__ __device__ __forceinline__ void dft_b(float2 (&v)[B])
{
    if constexpr (B == 4) r4<INV>(v[0], v[1], v[2], v[3]);
    else if constexpr (B == 8) dft8<INV>(v);
    else if constexpr (B == 12) dft12<INV>(v);
    else small_dft_c<B, INV>(v);
}

// Element (row p, line c) of a tile sits at T[p * SP + c * SC]: SP = 16 (or
// more), SC = 1 for lines down the columns (rows of 16 consecutive lines), or
// SP = 1 and SC odd for lines along the rows.  A half warp always serves the
// 16 lines of one row, so both forms are free of bank conflicts.
//
// Stage 1, task (c, n2): rows >= nin (and, with HALF, >= M/2) read as zero.
template <int B, bool INV, bool HALF, int SP = 16, int SC = 1>
__host__ __device__ __forceinline__ void tile_stage1(float2 *T, const float2 *tw, int nin, int c, int n2)
{
    float2 *L = T + c * SC;
    float2 x[16];
    constexpr int NR = HALF ? 8 : 16;   // rows that may be nonzero: n1 < NR
    if (nin >= NR * B) {                // all of them present: no per-row test
#pragma unroll
        for (int n1 = 0; n1 < 16; ++n1) x[n1] = n1 < NR ? L[(B * n1 + n2) * SP] : make_float2(0.0f, 0.0f);
    } else {
#pragma unroll
        for (int n1 = 0; n1 < 16; ++n1) {
            const int p = B * n1 + n2;
            x[n1] = (n1 < NR && p < nin) ? L[p * SP] : make_float2(0.0f, 0.0f);
        }
    }
    dft16<INV, HALF>(x);
    L[n2 * SP] = x[0];
#pragma unroll
    for (int k1 = 1; k1 < 16; ++k1) L[(B * k1 + n2) * SP] = cmul(x[k1], twid<INV>(tw, n2 * k1));
}

// Stage 2, task (c, k1).
template <int B, bool INV, int SP = 16, int SC = 1>
__host__ __device__ __forceinline__ void tile_stage2(float2 *T, int c, int k1)
{
    float2 *L = T + c * SC + B * k1 * SP;
    float2 v[B];
#pragma unroll
    for (int n2 = 0; n2 < B; ++n2) v[n2] = L[n2 * SP];
    dft_b<B, INV>(v);
#pragma unroll
    for (int k2 = 0; k2 < B; ++k2) L[k2 * SP] = v[k2];
}

// The whole tile by a pair of warps (the 64 threads that call it with
// half = 0 and 1; named barrier bar_id with 64 threads between the stages and
// at the end): stage 1 in B/2 rounds of 32 tasks, stage 2 in 8, the rounds of
// each stage alternating between the two warps.  tw: exp(-2 pi i j/M), j < M.
template <int B, bool INV, bool HALF>
__device__ __forceinline__ void tile_fft16_pair(float2 *T, const float2 *tw, int nin, int lane, int half, int bar_id)
{
    static_assert(B % 2 == 0, "tile transform: B even");
    const int c = lane & 15, hi = lane >> 4;
#pragma unroll 1
    for (int r = half; r < B / 2; r += 2) tile_stage1<B, INV, HALF>(T, tw, nin, c, 2 * r + hi);
    asm volatile("bar.sync %0, 64;" ::"r"(bar_id) : "memory");
#pragma unroll 1
    for (int r = half; r < 8; r += 2) tile_stage2<B, INV>(T, c, 2 * r + hi);
    asm volatile("bar.sync %0, 64;" ::"r"(bar_id) : "memory");
}

// ntiles tiles (tile i at T + i * tile_stride) by the whole block, the tasks
// of each stage spread over its threads (16 consecutive threads take the 16
// lines of one row); ends with the block synchronised.
template <int B, bool INV, bool HALF, int SP, int SC>
__device__ __forceinline__ void tiles_fft_block(float2 *T, int tile_stride, int ntiles, const float2 *tw, int nin)
{
    const int n1 = ntiles * 16 * B;
#pragma unroll 1
    for (int i = threadIdx.x; i < n1; i += blockDim.x) {
        const int c = i & 15, rest = i >> 4;
        const int tile = rest / B, n2 = rest - tile * B;
        tile_stage1<B, INV, HALF, SP, SC>(T + tile * tile_stride, tw, nin, c, n2);
    }
    __syncthreads();
    const int n2t = ntiles * 256;
#pragma unroll 1
    for (int i = threadIdx.x; i < n2t; i += blockDim.x)
        tile_stage2<B, INV, SP, SC>(T + (i >> 8) * tile_stride, i & 15, (i >> 4) & 15);
    __syncthreads();
}

// Runtime dispatch on R for a functor templated on R:  f.template run<R>().
template <class F>
__device__ __forceinline__ void dispatch_radix(int R, F &f)
{
    switch (R) {
    case 1: f.template run<1>(); break;
    case 2: f.template run<2>(); break;
    case 3: f.template run<3>(); break;
    case 4: f.template run<4>(); break;
    case 6: f.template run<6>(); break;
    default: break;
    }
}

// Copy a twiddle table into shared memory.
__device__ __forceinline__ void load_twiddles(float2 *dst, const float2 *src, int M)
{
    for (int i = threadIdx.x; i < M; i += blockDim.x) dst[i] = src[i];
}

}  // namespace rp
