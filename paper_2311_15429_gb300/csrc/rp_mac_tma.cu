// Spectral multiply-accumulate + inverse column FFT, fed by the tensor memory
// accelerator.
//
// Same arithmetic as k_mac_inv_column (the sum over a target's (source, lag)
// entries of G_m * S(l - m), Eq. 12 in the spectral domain, then the inverse
// FFT along z kept to the target's z < nz), restructured so that the
// operands stream through shared memory asynchronously:
//
//   * persistent blocks, one per SM, each walking (kx, 16-ky) column tiles;
//   * the last warp is the producer: one lane issues bulk copies
//     (cp.async.bulk) into two rings of shared-memory stages, one for the
//     entries' kernel tiles (M rows x 128 B, or 64 B for a real kernel) and
//     one for their source field tiles.  The ring stores a tile's four field
//     tiles next to each other, so one copy brings FPC of them (4 up to
//     M = 96, 2 at 128, 1 at 192): the copy engine spends a roughly fixed time
//     per copy, and copies under about 16 KB leave HBM bandwidth unused.  Each
//     stage is guarded by a "full" mbarrier (transaction bytes) and an "empty"
//     mbarrier (one arrival per consumer warp);
//   * the other CW warps (8, 12 or 16, picked per size class by timing the
//     variants on the context's own plan) are consumers: they multiply-accumulate in registers,
//     then write the tile to a separate shared-memory region, where the FFT
//     warps run the inverse column transform (the two-stage tile transform of
//     rp_fft.cuh) and store T2, so the producer keeps prefetching the next
//     tile's operands meanwhile.
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
constexpr int kKernelStages = 2;   // depth of the kernel-tile ring
constexpr int kFftWarps = 7;       // warps of the inverse column FFT and the T2 store: with the
                                   // producer, 8 + 8/12/16 MAC warps, a whole number of warps per
                                   // scheduler for the register split; 7 keep up with tiles of few
                                   // entries (the self lags alone), where 3 left the MAC warps waiting

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
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, long long limit = kWaitLimit)
{
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > limit) return false;
    return true;
}

// Self-test of the bounded wait: one mbarrier that nothing arrives on, waited
// through mbar_wait with a short limit; it runs out, raises the error flag
// and the block exits.
__global__ void k_wait_selftest(long long limit, int *err)
{
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0 && !mbar_wait(&bar, 0, limit)) atomicExch(err, 1);
}

// Contiguous copy of `bytes` (multiple of 16, both addresses 16-byte aligned)
// by the bulk-copy engine, completing on `bar`, with an L2 eviction-priority
// policy for the source lines.
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar, uint64_t policy)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
            smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(smem_u32(bar)), "l"(policy)
        : "memory");
}

__device__ __forceinline__ uint64_t policy_evict_first()
{
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}

__device__ __forceinline__ uint64_t policy_evict_last()
{
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
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

// Kahan-compensated addition: s + c carries the sum of the added terms with
// the rounding of each addition kept in c (the error stays near one rounding
// of the sum of magnitudes, whatever the number of terms); the total is s - c.
__device__ __forceinline__ void kahan_add(float &s, float &c, float x)
{
    const float y = x - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
}

// barrier `id` among the first (or last) `threads` threads of the block
__device__ __forceinline__ void named_sync(int id, int threads)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(threads) : "memory");
}

// Inverse FFT along z of the NF field tiles of `acc` ([field][M][16], dense;
// fields f0 .. f0 + NF - 1) by the two-stage tile transform (rp_fft.cuh), its
// tasks shared by warps w = 0 .. nw-1 (this one is w; barrier `bar` of nw
// warps between the stages), then rows z < nz (row z of the transform sits at
// tile_row(z)) to T2.
template <int M, int NF>
__device__ __forceinline__ void column_tile_store(float2 *acc, const float2 *tw, const InvTarget &T, int kxi, int ky0,
                                                  int f0, int w, int nw, int lane, int bar)
{
    constexpr int B = M / 16, FS = M * kTileY;
    const int tid = w * 32 + lane, nt = nw * 32;
    for (int i = tid; i < NF * 16 * B; i += nt) {
        const int c = i & 15, rest = i >> 4, f = rest / B, n2 = rest - f * B;
        tile_stage1<B, true, false>(acc + f * FS, tw, M, c, n2);
    }
    named_sync(bar, nt);
    for (int i = tid; i < NF * 256; i += nt) tile_stage2<B, true>(acc + (i >> 8) * FS, i & 15, (i >> 4) & 15);
    named_sync(bar, nt);
    const int nz = T.nz;
    const long long t2_field = (long long)(M / 2 + 1) * nz * M;
    float2 *dst = T.t2 + (long long)f0 * t2_field + (long long)kxi * nz * M + ky0;
    for (int i = tid; i < NF * nz * (kTileY / 2); i += nt) {
        const int f = i / (nz * (kTileY / 2)), rem = i - f * nz * (kTileY / 2);
        const int zi = rem >> 3, pp = rem & 7;
        *reinterpret_cast<float4 *>(dst + f * t2_field + (long long)zi * M + 2 * pp) =
            *reinterpret_cast<const float4 *>(acc + f * FS + tile_row<B>(zi) * kTileY + 2 * pp);
    }
}

// Warps of the inverse column FFT: fewer in the compensated variant, whose
// MAC warps hold twice the accumulators and need the registers.
template <bool COMP>
__host__ __device__ constexpr int fft_warps() { return COMP ? 3 : kFftWarps; }

// Field groups per tile: the compensated MAC at M = 192 would hold 128
// accumulator and compensation floats per MAC thread for all four fields (and
// spill them), so it sums the tile in two passes of two fields each, every
// pass over all the tile's entries (the kernel tile read again, mostly from
// L2), and hands each pass's two fields to the FFT warps on its own.
__host__ __device__ constexpr int field_groups(int M, bool comp) { return comp && M == 192 ? 2 : 1; }

// M: padded FFT size of the class; CW: multiply-accumulate warps (the block
// has CW + fft_warps + 1); FPC: field tiles per ring copy (1, 2 or 4; they
// are contiguous in the ring); COMP: the sum over (source, lag) entries is
// Kahan-compensated per spectral coefficient (the default; RP_FLAG_PLAIN_SUM
// selects the plain chain).
template <int M, int CW, int FPC, bool COMP>
__global__ void __launch_bounds__((CW + fft_warps<COMP>() + 1) * 32, 1)
    k_mac_tma(const InvTarget *__restrict__ tgts, int t0, int t1, int tile_lo, int ntiles,
              const MacEntry *__restrict__ entries, long long step, int clamp, int ns, int *err)
{
    constexpr int STAGE = M * 128;                  // one M x 16 complex tile
    constexpr int SSTAGE = FPC * STAGE;             // FPC field tiles of one entry
    constexpr int NG = kKernelStages;
    constexpr int kConsumerWarps = CW;
    constexpr int FW = fft_warps<COMP>();
    constexpr int RSTEP = kConsumerWarps * 32 / 8;   // rows covered by one pass of the consumers
    constexpr int ROWS = (M + RSTEP - 1) / RSTEP;
    constexpr int NTY = M / kTileY;
    constexpr int FS = M * kTileY;                   // float2 per field of the FFT tile (dense rows)
    constexpr int NFG = field_groups(M, COMP);      // passes per tile
    constexpr int FH = 4 / NFG;                      // fields per pass
    static_assert(FH % FPC == 0, "k_mac_tma: whole field copies per pass");
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char *sstages = smem;                                   // [ns][SSTAGE]
    unsigned char *gstages = smem + (size_t)ns * SSTAGE;             // [NG][STAGE]
    float2 *acc = reinterpret_cast<float2 *>(gstages + (size_t)NG * STAGE);
    float2 *tw = acc + FH * FS;                                      // acc: [FH][M][16]
    uint64_t *sfull = reinterpret_cast<uint64_t *>(tw + M);
    uint64_t *sempty = sfull + ns;
    uint64_t *gfull = sempty + ns;
    uint64_t *gempty = gfull + NG;
    uint64_t *accfull = gempty + NG;    // the FFT tile holds a tile's sums (one arrival per MAC warp)
    uint64_t *accempty = accfull + 1;   // the FFT warps are done with it (one arrival per FFT warp)
    volatile int *abort_flag = reinterpret_cast<volatile int *>(accempty + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < ns; ++s) {
            mbar_init(&sfull[s], 1);
            mbar_init(&sempty[s], kConsumerWarps);
        }
        for (int s = 0; s < NG; ++s) {
            mbar_init(&gfull[s], 1);
            mbar_init(&gempty[s], kConsumerWarps);
        }
        mbar_init(accfull, kConsumerWarps);
        mbar_init(accempty, FW);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    load_twiddles(tw, tgts[t0].tw_z, M);
    pdl_trigger();
    pdl_wait();   // the newest ring slot is written by the column pass; T2 was read by the last plane pass
    if (step < 0) step = *tgts[t0].d_step;   // graph replay: the step from the device counter
    __syncthreads();

    // wait for a phase; false (and the error raised) on abort/timeout
    auto wait_or_abort = [&](uint64_t *bar, uint32_t parity) {
        if (*abort_flag) return false;
        if (!mbar_wait(bar, parity)) {
            *abort_flag = 1;
            atomicExch(err, 1);
            return false;
        }
        return true;
    };

    if (warp == kConsumerWarps + FW) {
        // ------------------------------------------------------------ producer
        if (lane != 0) return;
        uint32_t qg = 0, qs = 0;
        bool ok = true;
        // The kernel tiles (tens of MB, read every step) stay in L2; the ring
        // tiles (read once per step per entry) pass through without evicting them.
        const uint64_t keep = policy_evict_last(), stream = policy_evict_first();
        // wait until stage q of a ring is free; false (and the error raised) on abort/timeout
        auto acquire = [&](uint64_t *empty, int n, uint32_t q) {
            if (*abort_flag || !mbar_wait(&empty[q % n], ((q / n) & 1) ^ 1)) {
                *abort_flag = 1;
                atomicExch(err, 1);
                return false;
            }
            return true;
        };
        for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
            const int b = tile + tile_lo;
            const InvTarget &T = tgts[owner(tgts, t0, t1, b, &InvTarget::tile0)];
            const long long tile_off = (long long)(b - T.tile0) * M * kTileY;
            const int nr = T.er - T.e0, nc = T.e1 - T.er;   // real (self) entries come first
            for (int k = 0; k < NFG * (nr + nc) && ok; ++k) {   // pass h = k / (nr + nc) of the tile
                const int h = k / (nr + nc);
                const MacEntry &E = entries[T.e0 + k - h * (nr + nc)];
                long long j = step - E.lag;
                if (clamp && j < 0) j = 0;
                const int slot = (int)(j % E.depth);
                // the kernel tile
                if (!(ok = acquire(gempty, NG, qg))) break;
                {
                    const int s = qg % NG;
                    const uint32_t bytes = E.is_real ? M * 64 : M * 128;
                    const void *src = E.is_real ? (const void *)(static_cast<const float *>(E.g) + tile_off)
                                                : (const void *)(static_cast<const float2 *>(E.g) + tile_off);
                    mbar_expect_tx(&gfull[s], bytes);
                    bulk_load(gstages + (size_t)s * STAGE, src, bytes, &gfull[s], keep);
                    ++qg;
                }
                // the pass's field tiles of the source spectrum (fields h FH ..), FPC per copy
                const float2 *fields = E.ring + (long long)slot * E.slot_elems + 4 * tile_off;
                for (int o = 0; o < FH / FPC; ++o) {
                    if (!(ok = acquire(sempty, ns, qs))) break;
                    const int s = qs % ns;
                    mbar_expect_tx(&sfull[s], SSTAGE);
                    bulk_load(sstages + (size_t)s * SSTAGE, fields + (long long)(h * FH + o * FPC) * M * kTileY,
                              SSTAGE, &sfull[s], stream);
                    ++qs;
                }
            }
        }
        // no copy may still be landing when the block exits
        for (uint32_t r = qg > (uint32_t)NG ? qg - NG : 0; r < qg; ++r)
            if (!mbar_wait(&gfull[r % NG], (r / NG) & 1)) atomicExch(err, 1);
        for (uint32_t r = qs > (uint32_t)ns ? qs - ns : 0; r < qs; ++r)
            if (!mbar_wait(&sfull[r % ns], (r / ns) & 1)) atomicExch(err, 1);
        return;
    }

    // Hand-over, per pass of a tile (one pass of all four fields, or two of
    // two): the MAC warps accumulate the pass in registers, store it to the
    // FFT tile and signal accfull; the FFT warps transform and store it while
    // the MAC warps accumulate the next pass, then signal accempty.  A
    // block's last pass has no successor, so all its consumer warps share
    // that transform (barrier 2 in place of the two signals).
    constexpr int kBarFft = 1, kBarAll = 2;
    if (warp >= kConsumerWarps) {
        // ------------------------------------------------------------ FFT warps
        const int fw = warp - kConsumerWarps;
        uint32_t it = 0;
        for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
            const int b = tile + tile_lo;
            const InvTarget &T = tgts[owner(tgts, t0, t1, b, &InvTarget::tile0)];
            const int local = b - T.tile0, kxi = local / NTY, ky0 = (local % NTY) * kTileY;
            for (int h = 0; h < NFG; ++h, ++it) {
                if (tile + (int)gridDim.x >= ntiles && h == NFG - 1) {
                    named_sync(kBarAll, (kConsumerWarps + FW) * 32);
                    column_tile_store<M, FH>(acc, tw, T, kxi, ky0, h * FH, warp, kConsumerWarps + FW, lane, kBarAll);
                    return;
                }
                const bool have = wait_or_abort(accfull, it & 1);
                // on an abort the sums are not used: skip the transform, keep the barriers
                if (have) column_tile_store<M, FH>(acc, tw, T, kxi, ky0, h * FH, fw, FW, lane, kBarFft);
                else {
                    named_sync(kBarFft, FW * 32);
                    named_sync(kBarFft, FW * 32);
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(accempty);
            }
        }
        return;
    }

    // ---------------------------------------------------------------- MAC warps
    const int p = threadIdx.x & 7, r0 = threadIdx.x >> 3;   // ky pair p, rows r0 + RSTEP i
    uint32_t qg = 0, qs = 0, it = 0;

    // wait for stage q of a ring; its address (or nullptr after an abort/timeout)
    auto take = [&](unsigned char *base, int bytes, uint64_t *full, int n, uint32_t q) -> const unsigned char * {
        if (!wait_or_abort(&full[q % n], (q / n) & 1)) return nullptr;
        return base + (size_t)(q % n) * bytes;
    };
    auto give = [&](uint64_t *empty, int n, uint32_t q) {
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[q % n]);
    };

    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int b = tile + tile_lo;
        const InvTarget &T = tgts[owner(tgts, t0, t1, b, &InvTarget::tile0)];
        for (int h = 0; h < NFG; ++h, ++it) {   // pass h: fields h FH .. h FH + FH - 1
            float4 a[ROWS][FH];
            float4 cmp[COMP ? ROWS : 1][FH];   // Kahan compensation (COMP only)
#pragma unroll
            for (int i = 0; i < ROWS; ++i)
#pragma unroll
                for (int f = 0; f < FH; ++f) a[i][f] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int i = 0; i < (COMP ? ROWS : 1); ++i)
#pragma unroll
                for (int f = 0; f < FH; ++f) cmp[i][f] = make_float4(0.f, 0.f, 0.f, 0.f);

            for (int e = T.e0; e < T.er; ++e) {   // real kernels (self pair)
                float2 g[ROWS];
                const unsigned char *st = take(gstages, STAGE, gfull, NG, qg);
                const float *Gt = reinterpret_cast<const float *>(st);   // [M][16]
#pragma unroll
                for (int i = 0; i < ROWS; ++i) {
                    const int r = r0 + RSTEP * i;
                    g[i] = (st && r < M) ? *reinterpret_cast<const float2 *>(Gt + r * 16 + 2 * p)
                                         : make_float2(0.f, 0.f);
                }
                give(gempty, NG, qg++);
#pragma unroll
                for (int o = 0; o < FH / FPC; ++o) {
                    const unsigned char *sf = take(sstages, SSTAGE, sfull, ns, qs);
#pragma unroll
                    for (int ff = 0; ff < FPC; ++ff) {
                        const int f = o * FPC + ff;
                        const float4 *S4 = reinterpret_cast<const float4 *>(sf + ff * STAGE);   // [M][8]
#pragma unroll
                        for (int i = 0; i < ROWS; ++i) {
                            const int r = r0 + RSTEP * i;
                            if (sf && r < M) {
                                const float4 s = S4[r * 8 + p];
                                if constexpr (COMP) {
                                    float4 &c = cmp[COMP ? i : 0][f];
                                    kahan_add(a[i][f].x, c.x, g[i].x * s.x);
                                    kahan_add(a[i][f].y, c.y, g[i].x * s.y);
                                    kahan_add(a[i][f].z, c.z, g[i].y * s.z);
                                    kahan_add(a[i][f].w, c.w, g[i].y * s.w);
                                } else {
                                    a[i][f].x = fmaf(g[i].x, s.x, a[i][f].x);
                                    a[i][f].y = fmaf(g[i].x, s.y, a[i][f].y);
                                    a[i][f].z = fmaf(g[i].y, s.z, a[i][f].z);
                                    a[i][f].w = fmaf(g[i].y, s.w, a[i][f].w);
                                }
                            }
                        }
                    }
                    give(sempty, ns, qs++);
                }
            }
            for (int e = T.er; e < T.e1; ++e) {   // complex kernels (other sources)
                float4 g[ROWS];
                const unsigned char *st = take(gstages, STAGE, gfull, NG, qg);
                const float4 *G4 = reinterpret_cast<const float4 *>(st);
#pragma unroll
                for (int i = 0; i < ROWS; ++i) {
                    const int r = r0 + RSTEP * i;
                    g[i] = (st && r < M) ? G4[r * 8 + p] : make_float4(0.f, 0.f, 0.f, 0.f);
                }
                give(gempty, NG, qg++);
#pragma unroll
                for (int o = 0; o < FH / FPC; ++o) {
                    const unsigned char *sf = take(sstages, SSTAGE, sfull, ns, qs);
#pragma unroll
                    for (int ff = 0; ff < FPC; ++ff) {
                        const int f = o * FPC + ff;
                        const float4 *S4 = reinterpret_cast<const float4 *>(sf + ff * STAGE);
#pragma unroll
                        for (int i = 0; i < ROWS; ++i) {
                            const int r = r0 + RSTEP * i;
                            if (sf && r < M) {
                                const float4 s = S4[r * 8 + p];
                                float4 &x = a[i][f];
                                if constexpr (COMP) {
                                    float4 &c = cmp[COMP ? i : 0][f];
                                    kahan_add(x.x, c.x, fmaf(g[i].x, s.x, -g[i].y * s.y));
                                    kahan_add(x.y, c.y, fmaf(g[i].x, s.y, g[i].y * s.x));
                                    kahan_add(x.z, c.z, fmaf(g[i].z, s.z, -g[i].w * s.w));
                                    kahan_add(x.w, c.w, fmaf(g[i].z, s.w, g[i].w * s.z));
                                } else {
                                    x.x = fmaf(g[i].x, s.x, fmaf(-g[i].y, s.y, x.x));
                                    x.y = fmaf(g[i].x, s.y, fmaf(g[i].y, s.x, x.y));
                                    x.z = fmaf(g[i].z, s.z, fmaf(-g[i].w, s.w, x.z));
                                    x.w = fmaf(g[i].z, s.w, fmaf(g[i].w, s.z, x.w));
                                }
                            }
                        }
                    }
                    give(sempty, ns, qs++);
                }
            }

            // hand the sums to the FFT warps once they are done with the previous pass
            if (it == 0 || wait_or_abort(accempty, (it - 1) & 1)) {
#pragma unroll
                for (int i = 0; i < ROWS; ++i) {
                    const int r = r0 + RSTEP * i;
                    if (r >= M) continue;
#pragma unroll
                    for (int f = 0; f < FH; ++f) {
                        if constexpr (COMP) {   // the compensated total
                            const float4 &c = cmp[COMP ? i : 0][f];
                            a[i][f] = make_float4(a[i][f].x - c.x, a[i][f].y - c.y, a[i][f].z - c.z, a[i][f].w - c.w);
                        }
                        *reinterpret_cast<float4 *>(acc + f * FS + r * kTileY + 2 * p) = a[i][f];
                    }
                }
            }
            if (tile + (int)gridDim.x >= ntiles && h == NFG - 1) {
                named_sync(kBarAll, (kConsumerWarps + FW) * 32);
                const int local = b - T.tile0;
                column_tile_store<M, FH>(acc, tw, T, local / NTY, (local % NTY) * kTileY, h * FH, warp,
                                         kConsumerWarps + FW, lane, kBarAll);
                return;
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(accfull);
        }
    }
}

// (class, field tiles per ring copy): must match mac_tma_fields_per_copy
#define RP_TMA_CLASSES(X) X(32, 4) X(48, 4) X(64, 4) X(96, 4) X(128, 2) X(192, 1)

}  // namespace

cudaError_t launch_wait_selftest(long long limit_cycles, int *d_err, cudaStream_t s)
{
    k_wait_selftest<<<1, 32, 0, s>>>(limit_cycles, d_err);
    return cudaGetLastError();
}

int mac_tma_fields_per_copy(int M) { return M <= 96 ? 4 : (M == 128 ? 2 : 1); }

int mac_tma_stages(int M, int smem_optin, bool comp)
{
    const long long sstage = (long long)mac_tma_fields_per_copy(M) * M * 128;
    const long long fixed = (long long)mac_tma_smem(M, 0, comp);   // kernel-tile ring, FFT tile, twiddles, barriers
    long long n = (smem_optin - fixed) / (sstage + 16);      // + two mbarriers per stage
    if (n > kMaxStages) n = kMaxStages;
    return (int)n;
}

size_t mac_tma_smem(int M, int nstages, bool comp)
{
    const size_t stage = (size_t)M * 128, fields = 4 / field_groups(M, comp);   // fields of the FFT tile
    return (size_t)nstages * mac_tma_fields_per_copy(M) * stage + kKernelStages * stage +
           sizeof(float2) * (fields * (size_t)M * kTileY + M) + 16 * ((size_t)nstages + kKernelStages) + 16 + 16;
}

cudaError_t open_mac_tma_smem_limit(int max_optin)
{
    cudaError_t e;
#define X(M, F)                                                                                                   \
    if ((e = cudaFuncSetAttribute(k_mac_tma<M, 8, F, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,        \
                                  max_optin)) ||                                                                  \
        (e = cudaFuncSetAttribute(k_mac_tma<M, 12, F, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,       \
                                  max_optin)) ||                                                                  \
        (e = cudaFuncSetAttribute(k_mac_tma<M, 16, F, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,       \
                                  max_optin)) ||                                                                  \
        (e = cudaFuncSetAttribute(k_mac_tma<M, kCompWarps, F, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                  max_optin)))                                                                    \
        return e;
    RP_TMA_CLASSES(X)
#undef X
    return cudaSuccess;
}

cudaError_t launch_mac_tma(int cls, int cw, bool comp, const InvTarget *d_tgts, int t0, int t1, int tile_lo,
                           int ntiles, const MacEntry *d_entries, long long step, int clamp, int nstages, int grid,
                           int *d_err, cudaStream_t s)
{
    if (ntiles <= 0) return cudaSuccess;
    if (comp ? cw != kCompWarps : (cw != 8 && cw != 12 && cw != 16)) return cudaErrorInvalidValue;
    if (nstages < 2 || nstages > kMaxStages) return cudaErrorInvalidValue;
    const size_t smem = mac_tma_smem(cls, nstages, comp);
    const int threads = (cw + (comp ? fft_warps<true>() : fft_warps<false>()) + 1) * 32;
    cudaError_t e = cudaSuccess;
#define RP_GO(M, CW, F, C)                                                                                   \
    e = launch_pdl(k_mac_tma<M, CW, F, C>, dim3(grid), dim3(threads), smem, s, d_tgts, t0, t1, tile_lo, ntiles, \
                   d_entries, step, clamp, nstages, d_err)
    switch (cls) {
#define X(M, F)                                                                                         \
    case M:                                                                                             \
        if (comp) RP_GO(M, kCompWarps, F, true);                                                        \
        else if (cw == 8) RP_GO(M, 8, F, false);                                                        \
        else if (cw == 12) RP_GO(M, 12, F, false);                                                      \
        else RP_GO(M, 16, F, false);                                                                    \
        break;
        RP_TMA_CLASSES(X)
#undef X
    default: return cudaErrorInvalidValue;
    }
#undef RP_GO
    return e != cudaSuccess ? e : cudaGetLastError();
}

}  // namespace rp
