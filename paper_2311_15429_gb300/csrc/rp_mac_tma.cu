// Spectral multiply-accumulate + inverse column FFT, fed by the tensor memory
// accelerator.
//
// Same arithmetic as k_mac_inv_column (the sum over a target's (source, lag)
// entries of G_m * S(l - m), Eq. 12 in the spectral domain, then the inverse
// FFT along z kept to the target's z < nz), restructured so that the
// operands stream through shared memory asynchronously:
//
//   * persistent blocks, one per SM, each walking (kx, 16-ky) column tiles;
//   * the last warp is the producer: one lane issues cp.async.bulk.tensor copies of
//     each entry's kernel tile and its four field tiles (M rows x 128 B) into
//     a ring of shared-memory stages, each stage guarded by a "full" mbarrier
//     (transaction bytes) and an "empty" mbarrier (one arrival per consumer
//     warp);
//   * the other CW warps (8, 12 or 16, picked per size class by timing the
//     variants on the context's own plan) are consumers: they multiply-accumulate in registers,
//     then write the tile to a separate shared-memory region for the column
//     FFT (two columns per warp at a time), so the producer keeps prefetching
//     the next tile's operands meanwhile.
//
// Every wait is bounded (clock64 limit).  On a timeout the kernel sets the
// context's error flag, stops waiting, and the producer waits (bounded) for
// the copies it has in flight before the block exits.
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "rp_fft.cuh"
#include "rp_internal.h"

namespace rp {

namespace {

constexpr long long kWaitLimit = 4000000000LL;   // SM clock cycles (about 2 s)
constexpr int kMaxStages = 24;

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, int count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for the phase of `parity` to complete; false after kWaitLimit cycles.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity)
{
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > kWaitLimit) return false;
    return true;
}

// Contiguous copy of `bytes` (multiple of 16, both addresses 16-byte aligned)
// by the bulk-copy engine, completing on `bar`.
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

template <class T>
__device__ __forceinline__ int owner(const T *arr, int lo, int hi, int b, int T::*field)
{
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (arr[mid].*field <= b) lo = mid; else hi = mid;
    }
    return lo;
}

template <int CW>
__device__ __forceinline__ void consumer_sync() { asm volatile("bar.sync 1, %0;" ::"n"(CW * 32) : "memory"); }

// M: padded FFT size of the class; CW: consumer warps (the block has CW + 1).
template <int M, int CW>
__global__ void __launch_bounds__((CW + 1) * 32, 1)
    k_mac_tma(const InvTarget *__restrict__ tgts, int t0, int t1, int tile_lo, int ntiles,
              const MacEntry *__restrict__ entries, const CUtensorMap *__restrict__ maps, int nmaps, long long step,
              int clamp, int nstages, int *err)
{
    constexpr int STAGE = M * 128;                  // one M x 16 complex tile
    constexpr int kConsumerWarps = CW;
    constexpr int RSTEP = kConsumerWarps * 32 / 8;   // rows covered by one pass of the consumers
    constexpr int ROWS = (M + RSTEP - 1) / RSTEP;
    constexpr int NTY = M / kTileY;
    constexpr int FS = M * kTileYPad;                // float2 per field of the FFT tile
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char *stages = smem;
    float2 *acc = reinterpret_cast<float2 *>(smem + (size_t)nstages * STAGE);
    float2 *tw = acc + 4 * FS;
    uint64_t *full = reinterpret_cast<uint64_t *>(tw + M);
    uint64_t *empty = full + nstages;
    volatile int *abort_flag = reinterpret_cast<volatile int *>(empty + nstages);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < nstages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], kConsumerWarps);
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    load_twiddles(tw, tgts[t0].tw_z, M);
    __syncthreads();

    if (warp == kConsumerWarps) {
        // ------------------------------------------------------------ producer
        if (lane != 0) return;
        // the descriptors were written through the generic proxy (host copy)
        for (int m = 0; m < nmaps; ++m)
            asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(
                             reinterpret_cast<uint64_t>(maps + m))
                         : "memory");
        uint32_t q = 0;
        bool ok = true;
        for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
            const int b = tile + tile_lo;
            const InvTarget &T = tgts[owner(tgts, t0, t1, b, &InvTarget::tile0)];
            const long long tile_off = (long long)(b - T.tile0) * M * kTileY;
            const int nr = T.er - T.e0, nc = T.e1 - T.er;   // real (self) entries come first
            for (int k = 0; k < nr + nc && ok; ++k) {
                const MacEntry &E = entries[T.e0 + k];
                long long j = step - E.lag;
                if (clamp && j < 0) j = 0;
                const int slot = (int)(j % E.depth);
                for (int o = 0; o < 5; ++o, ++q) {
                    const int s = q % nstages;
                    if (*abort_flag || !mbar_wait(&empty[s], ((q / nstages) & 1) ^ 1)) {
                        ok = false;
                        *abort_flag = 1;
                        atomicExch(err, 1);
                        break;
                    }
                    void *dst = stages + (size_t)s * STAGE;
                    if (o == 0) {
                        const uint32_t bytes = E.is_real ? M * 64 : M * 128;
                        mbar_expect_tx(&full[s], bytes);
                        const void *src = E.is_real ? (const void *)(static_cast<const float *>(E.g) + tile_off)
                                                    : (const void *)(static_cast<const float2 *>(E.g) + tile_off);
                        bulk_load(dst, src, bytes, &full[s]);
                    } else {
                        mbar_expect_tx(&full[s], M * 128);
                        const float2 *src = E.ring + (long long)slot * E.slot_elems +
                                            (long long)(o - 1) * (E.slot_elems / 4) + tile_off;
                        bulk_load(dst, src, M * 128, &full[s]);
                    }
                }
            }
        }
        // no copy may still be landing when the block exits
        const uint32_t first = q > (uint32_t)nstages ? q - nstages : 0;
        for (uint32_t r = first; r < q; ++r)
            if (!mbar_wait(&full[r % nstages], (r / nstages) & 1)) atomicExch(err, 1);
        return;
    }

    // ---------------------------------------------------------------- consumers
    const int p = threadIdx.x & 7, r0 = threadIdx.x >> 3;   // ky pair p, rows r0 + RSTEP i
    LaneTw<M, true> lt;
    lt.init(tw, lane & (LaneTw<M, true>::L - 1));
    uint32_t q = 0;

    // wait for stage q; returns its address (or nullptr after an abort/timeout)
    auto take = [&](uint32_t qq) -> const unsigned char * {
        const int s = qq % nstages;
        if (*abort_flag) return nullptr;
        if (!mbar_wait(&full[s], (qq / nstages) & 1)) {
            *abort_flag = 1;
            atomicExch(err, 1);
            return nullptr;
        }
        return stages + (size_t)s * STAGE;
    };
    auto give = [&](uint32_t qq) {
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[qq % nstages]);
    };

    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int b = tile + tile_lo;
        const InvTarget &T = tgts[owner(tgts, t0, t1, b, &InvTarget::tile0)];
        const int local = b - T.tile0, kxi = local / NTY, ky0 = (local % NTY) * kTileY;

        float4 a[ROWS][4];
#pragma unroll
        for (int i = 0; i < ROWS; ++i)
#pragma unroll
            for (int f = 0; f < 4; ++f) a[i][f] = make_float4(0.f, 0.f, 0.f, 0.f);

        for (int e = T.e0; e < T.er; ++e) {   // real kernels (self pair)
            float2 g[ROWS];
            const unsigned char *st = take(q);
            const float *Gt = reinterpret_cast<const float *>(st);   // [M][16]
#pragma unroll
            for (int i = 0; i < ROWS; ++i) {
                const int r = r0 + RSTEP * i;
                g[i] = (st && r < M) ? *reinterpret_cast<const float2 *>(Gt + r * 16 + 2 * p) : make_float2(0.f, 0.f);
            }
            give(q++);
#pragma unroll
            for (int f = 0; f < 4; ++f) {
                const unsigned char *sf = take(q);
                const float4 *S4 = reinterpret_cast<const float4 *>(sf);   // [M][8]
#pragma unroll
                for (int i = 0; i < ROWS; ++i) {
                    const int r = r0 + RSTEP * i;
                    if (sf && r < M) {
                        const float4 s = S4[r * 8 + p];
                        a[i][f].x = fmaf(g[i].x, s.x, a[i][f].x);
                        a[i][f].y = fmaf(g[i].x, s.y, a[i][f].y);
                        a[i][f].z = fmaf(g[i].y, s.z, a[i][f].z);
                        a[i][f].w = fmaf(g[i].y, s.w, a[i][f].w);
                    }
                }
                give(q++);
            }
        }
        for (int e = T.er; e < T.e1; ++e) {   // complex kernels (other sources)
            float4 g[ROWS];
            const unsigned char *st = take(q);
            const float4 *G4 = reinterpret_cast<const float4 *>(st);
#pragma unroll
            for (int i = 0; i < ROWS; ++i) {
                const int r = r0 + RSTEP * i;
                g[i] = (st && r < M) ? G4[r * 8 + p] : make_float4(0.f, 0.f, 0.f, 0.f);
            }
            give(q++);
#pragma unroll
            for (int f = 0; f < 4; ++f) {
                const unsigned char *sf = take(q);
                const float4 *S4 = reinterpret_cast<const float4 *>(sf);
#pragma unroll
                for (int i = 0; i < ROWS; ++i) {
                    const int r = r0 + RSTEP * i;
                    if (sf && r < M) {
                        const float4 s = S4[r * 8 + p];
                        float4 &x = a[i][f];
                        x.x = fmaf(g[i].x, s.x, fmaf(-g[i].y, s.y, x.x));
                        x.y = fmaf(g[i].x, s.y, fmaf(g[i].y, s.x, x.y));
                        x.z = fmaf(g[i].z, s.z, fmaf(-g[i].w, s.w, x.z));
                        x.w = fmaf(g[i].z, s.w, fmaf(g[i].w, s.z, x.w));
                    }
                }
                give(q++);
            }
        }

        // inverse FFT along z of the 64 columns, then rows z < nz to T2
#pragma unroll
        for (int i = 0; i < ROWS; ++i) {
            const int r = r0 + RSTEP * i;
            if (r >= M) continue;
#pragma unroll
            for (int f = 0; f < 4; ++f) {
                float2 *d = acc + f * FS + r * kTileYPad + 2 * p;
                d[0] = make_float2(a[i][f].x, a[i][f].y);
                d[1] = make_float2(a[i][f].z, a[i][f].w);
            }
        }
        consumer_sync<CW>();
        {
            // 64 columns; each warp transforms two at a time (independent
            // instruction streams for the scheduler to interleave)
            constexpr int R = LaneTw<M, true>::R, L = LaneTw<M, true>::L, LOGL = LaneTw<M, true>::LOGL;
            constexpr int G = 32 / L;
            constexpr int PER = 2 * kConsumerWarps * G;   // columns per pass
            const int grp = lane / L, g = lane % L;
            const int kb = bitrev_lanes(g, LOGL) * R;
            for (int base = 0; base < 4 * kTileY; base += PER) {
                const int l0 = base + (warp * G + grp) * 2;
                float2 *c0 = acc + (l0 / kTileY) * FS + l0 % kTileY;
                float2 *c1 = acc + ((l0 + 1) / kTileY) * FS + (l0 + 1) % kTileY;
                const bool ok = l0 < 4 * kTileY;
                float2 v0[R], v1[R];
#pragma unroll
                for (int n = 0; n < R; ++n) {
                    v0[n] = ok ? c0[(n * L + g) * kTileYPad] : make_float2(0.f, 0.f);
                    v1[n] = ok ? c1[(n * L + g) * kTileYPad] : make_float2(0.f, 0.f);
                }
                line_fft_c<M, true>(v0, lt);
                line_fft_c<M, true>(v1, lt);
                __syncwarp();
                if (ok) {
#pragma unroll
                    for (int k1 = 0; k1 < R; ++k1)
                        if (k1 + kb < T.nz) {
                            c0[(k1 + kb) * kTileYPad] = v0[k1];
                            c1[(k1 + kb) * kTileYPad] = v1[k1];
                        }
                }
                __syncwarp();
            }
        }
        consumer_sync<CW>();
        const int nz = T.nz;
        const long long t2_field = (long long)(M / 2 + 1) * nz * M;
        float2 *dst = T.t2 + (long long)kxi * nz * M + ky0;
        for (int i = threadIdx.x; i < 4 * nz * (kTileY / 2); i += kConsumerWarps * 32) {
            const int f = i / (nz * (kTileY / 2)), rem = i % (nz * (kTileY / 2));
            const int zi = rem / (kTileY / 2), pp = rem % (kTileY / 2);
            const float2 *s = acc + f * FS + zi * kTileYPad + 2 * pp;
            *reinterpret_cast<float4 *>(dst + f * t2_field + (long long)zi * M + 2 * pp) =
                make_float4(s[0].x, s[0].y, s[1].x, s[1].y);
        }
        consumer_sync<CW>();   // the FFT tile is rewritten by the next tile
    }
}

#define RP_TMA_CLASSES(X) X(32) X(48) X(64) X(96) X(128) X(192)

}  // namespace

int mac_tma_stages(int M, int smem_optin)
{
    const long long stage = (long long)M * 128;
    const long long fixed = sizeof(float2) * (4LL * M * kTileYPad + M) + 16;   // FFT tile, twiddles, abort flag
    long long n = (smem_optin - fixed) / (stage + 16);                          // + two mbarriers per stage
    if (n > kMaxStages) n = kMaxStages;
    return (int)n;
}

size_t mac_tma_smem(int M, int nstages)
{
    return (size_t)nstages * M * 128 + sizeof(float2) * (4 * (size_t)M * kTileYPad + M) + 16 * (size_t)nstages + 16;
}

cudaError_t open_mac_tma_smem_limit(int max_optin)
{
    cudaError_t e;
#define X(M)                                                                                            \
    if ((e = cudaFuncSetAttribute(k_mac_tma<M, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_optin)) || \
        (e = cudaFuncSetAttribute(k_mac_tma<M, 12>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_optin)) || \
        (e = cudaFuncSetAttribute(k_mac_tma<M, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_optin))) \
        return e;
    RP_TMA_CLASSES(X)
#undef X
    return cudaSuccess;
}

cudaError_t launch_mac_tma(int cls, int cw, const InvTarget *d_tgts, int t0, int t1, int tile_lo, int ntiles,
                           const MacEntry *d_entries, const CUtensorMap *d_maps, int nmaps, long long step, int clamp,
                           int nstages, int grid, int *d_err, cudaStream_t s)
{
    if (ntiles <= 0) return cudaSuccess;
    if (cw != 8 && cw != 12 && cw != 16) return cudaErrorInvalidValue;
    const size_t smem = mac_tma_smem(cls, nstages);
    const int threads = (cw + 1) * 32;
#define RP_GO(M, CW)                                                                                      \
    k_mac_tma<M, CW><<<grid, threads, smem, s>>>(d_tgts, t0, t1, tile_lo, ntiles, d_entries, d_maps, nmaps, step, \
                                                 clamp, nstages, d_err)
    switch (cls) {
#define X(M)                                                                                            \
    case M:                                                                                             \
        if (cw == 8) RP_GO(M, 8);                                                                       \
        else if (cw == 12) RP_GO(M, 12);                                                                \
        else RP_GO(M, 16);                                                                              \
        break;
        RP_TMA_CLASSES(X)
#undef X
    default: return cudaErrorInvalidValue;
    }
#undef RP_GO
    return cudaGetLastError();
}

}  // namespace rp
