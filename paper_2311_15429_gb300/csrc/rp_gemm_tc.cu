// BF16 tensor-core GEMM on the 5th-generation tensor cores (tcgen05), FP32
// accumulation in tensor memory:
//
//   D[m][n] = sum_k A[m][k] * B[n][k]        A: M x K, B: N x K (bf16, K contiguous)
//                                            D: M x N fp32 (row stride ldd)
//
// This is the contraction of the far-field operator: the skeleton rows of the
// lag-stacked kernel [G_lo ... G_hi] (A) against a batch of source slices (B).
//
// One CTA computes a 128 x BN tile (BN = N <= 256) over the whole K range:
//   warp 0      TMA producer: 128 x 64 and BN x 64 bf16 boxes, 128-byte swizzle,
//               into a ring of shared-memory stages ("full" mbarriers carry the
//               transaction bytes);
//   warp 1      allocates BN columns of tensor memory; one lane issues
//               tcgen05.mma (128 x BN x 16, bf16 x bf16 -> fp32) four times per
//               stage and commits each stage back to its "empty" mbarrier;
//   warps 2-5   epilogue: wait for the final commit, tcgen05.ld the 128 x BN
//               fp32 accumulator (each warp its 32 tensor-memory lanes) and
//               store D.
// Waits are bounded (clock64); a timeout sets *err and the CTA drains and exits.
#include <algorithm>
#include <map>
#include <mutex>
#include <utility>
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "rp_internal.h"
#include "rp_tc.cuh"

namespace rp {

namespace {

constexpr int kGemmThreads = 192;
using namespace tc;

// blockIdx.y selects a K range of `kchunk` k-tiles (split-K); each split
// writes its own M x N slice of D (D + split * split_stride).  TERMS = 3:
// the operands are [A_hi | A_lo] and [B_hi | B_lo] (each half K wide); one
// stage holds the four tiles of a k-tile and the three products
// A_hi B_hi^T, A_hi B_lo^T and A_lo B_hi^T accumulate into one tensor-memory
// accumulator, so every operand byte is read once.
template <int BN, int TERMS>
__global__ void __launch_bounds__(kGemmThreads, 1)
    k_gemm_bf16_tn(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, float *D,
                   int K, int ldd, int stages, int *err, int kchunk, long long split_stride, uint32_t idesc)
{
    constexpr int A_BYTES = kBM * kBK * 2, B_BYTES = BN * kBK * 2;
    constexpr int HALVES = TERMS == 3 ? 2 : 1;
    constexpr int B_OFF = HALVES * A_BYTES;
    constexpr int STAGE = HALVES * (A_BYTES + B_BYTES);   // multiple of 1024
    constexpr int TCOLS = tmem_cols<BN>();
    extern __shared__ __align__(1024) unsigned char smem[];
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + (size_t)stages * STAGE);
    uint64_t *empty = full + stages;
    uint64_t *done = empty + stages;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(done + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * kBM;
    const int kt_all = K / kBK;
    const int kt0 = blockIdx.y * kchunk;
    const int ktiles = max(0, min(kchunk, kt_all - kt0));
    const int n0 = blockIdx.z * BN;                 // column tile
    D += (long long)blockIdx.y * split_stride + n0;
    // the swizzled operand descriptors assume 1024-byte aligned stages
    if (su32(smem) & 1023u) {
        if (threadIdx.x == 0) atomicExch(err, 2);
        return;
    }

    if (threadIdx.x == 0) {
        for (int s = 0; s < stages; ++s) {
            bar_init(&full[s], 1);
            bar_init(&empty[s], 1);
        }
        bar_init(done, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)),
                     "r"(TCOLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    if (warp == 0 && lane == 0) {
        // ---------------------------------------------------------------- producer
        int kt = 0;
        for (; kt < ktiles; ++kt) {
            const int s = kt % stages;
            if (*abort_flag || !bar_wait(&empty[s], ((kt / stages) & 1) ^ 1)) {
                *abort_flag = 1;
                atomicExch(err, 1);
                break;
            }
            unsigned char *st = smem + (size_t)s * STAGE;
            const int k = (kt0 + kt) * kBK;
            bar_expect(&full[s], STAGE);
            tma_2d(st, &mapA, k, m0, &full[s]);
            tma_2d(st + B_OFF, &mapB, k, n0, &full[s]);
            if constexpr (TERMS == 3) {
                tma_2d(st + A_BYTES, &mapA, K + k, m0, &full[s]);
                tma_2d(st + B_OFF + B_BYTES, &mapB, K + k, n0, &full[s]);
            }
        }
        // every copy issued has landed before the CTA may exit
        for (int r = kt > stages ? kt - stages : 0; r < kt; ++r)
            if (!bar_wait(&full[r % stages], (r / stages) & 1)) atomicExch(err, 1);
    } else if (warp == 1 && lane == 0) {
        // ---------------------------------------------------------------- MMA issue
        const uint32_t ID = idesc;
        for (int kt = 0; kt < ktiles; ++kt) {
            const int s = kt % stages;
            if (*abort_flag || !bar_wait(&full[s], (kt / stages) & 1)) {
                *abort_flag = 1;
                atomicExch(err, 1);
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a = su32(smem + (size_t)s * STAGE), b = a + B_OFF;
#pragma unroll
            for (int kk = 0; kk < kBK / 16; ++kk) {   // 16 bf16 = 32 bytes along K per instruction
                mma_bf16(tmem, desc_sw128(a + kk * 32), desc_sw128(b + kk * 32), ID, (kt | kk) ? 1u : 0u);
                if constexpr (TERMS == 3) {
                    mma_bf16(tmem, desc_sw128(a + kk * 32), desc_sw128(b + B_BYTES + kk * 32), ID, 1u);
                    mma_bf16(tmem, desc_sw128(a + A_BYTES + kk * 32), desc_sw128(b + kk * 32), ID, 1u);
                }
            }
            mma_commit(&empty[s]);                  // the stage is free once these complete
        }
        mma_commit(done);                           // all issued MMAs complete
    } else if (warp >= 2) {
        // ---------------------------------------------------------------- epilogue
        const bool ok = bar_wait(done, 0);
        if (!ok) atomicExch(err, 1);
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int quarter = warp & 3;               // tensor-memory lanes 32*quarter .. +31
        const int row = m0 + 32 * quarter + lane;
        if (ktiles == 0) {
            for (int c = 0; c < BN; c += 4)
                *reinterpret_cast<float4 *>(D + (size_t)row * ldd + c) = make_float4(0.f, 0.f, 0.f, 0.f);
        } else if (ok && !*abort_flag) {
#pragma unroll 1
            for (int c = 0; c < BN; c += 32) {
                uint32_t r[32];
                const uint32_t taddr = tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)c;
                tmem_ld32(taddr, r);
                float4 *out = reinterpret_cast<float4 *>(D + (size_t)row * ldd + c);
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    out[j] = make_float4(__uint_as_float(r[4 * j]), __uint_as_float(r[4 * j + 1]),
                                         __uint_as_float(r[4 * j + 2]), __uint_as_float(r[4 * j + 3]));
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 1) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TCOLS) : "memory");
    }
}

// Z[i] = sum over splits of P[split][i], in a fixed order: a block covers 32
// float4 outputs; its 8 thread groups take the splits g, g + 8, ... and the
// 8 partial sums are added in group order.
constexpr int kReduceGroups = 8;
__global__ void __launch_bounds__(256) k_split_reduce(const float4 *__restrict__ P, float4 *__restrict__ Z,
                                                      long long n4, int splits)
{
    __shared__ float4 part[kReduceGroups][32];
    const int g = threadIdx.x >> 5, j = threadIdx.x & 31;
    const long long i = blockIdx.x * 32LL + j;
    float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
    if (i < n4)
        for (int k = g; k < splits; k += kReduceGroups) {
            const float4 v = __ldg(P + (long long)k * n4 + i);
            s.x += v.x; s.y += v.y; s.z += v.z; s.w += v.w;
        }
    part[g][j] = s;
    __syncthreads();
    if (g == 0 && i < n4) {
        for (int k = 1; k < kReduceGroups; ++k) {
            s.x += part[k][j].x; s.y += part[k][j].y; s.z += part[k][j].z; s.w += part[k][j].w;
        }
        Z[i] = s;
    }
}

// Raises a kernel's dynamic shared-memory limit to `smem` on the current
// device the first time it is needed (a host call per launch would leave the
// GPU idle between the small launches of the learned field's network).
template <class K>
cudaError_t open_smem(K kern, size_t smem)
{
    static std::mutex mu;
    static std::map<std::pair<const void *, int>, int> opened;   // (kernel, device) -> bytes
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e) return e;
    std::lock_guard<std::mutex> lock(mu);
    const auto key = std::make_pair(reinterpret_cast<const void *>(kern), dev);
    auto it = opened.find(key);
    if (it != opened.end() && it->second >= (int)smem) return cudaSuccess;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (!e) opened[key] = (int)smem;
    return e;
}

template <int BN, int TERMS>
size_t gemm_smem(int stages)
{
    return (size_t)stages * (TERMS == 3 ? 2 : 1) * (kBM * kBK * 2 + BN * kBK * 2) + 8 * (2 * (size_t)stages + 1) +
           16;
}

}  // namespace

// 2-D bf16 descriptor over a row-major rows x cols matrix, box (64 cols, box_rows), 128-byte swizzle.
bool encode_bf16_rows(void *encode_fn, CUtensorMap *map, const void *base, uint64_t rows, uint64_t cols,
                      uint32_t box_rows)
{
    auto enc = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(encode_fn);
    const cuuint64_t dims[2] = {cols, rows};
    const cuuint64_t strides[1] = {cols * 2};
    const cuuint32_t box[2] = {(cuuint32_t)kBK, box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// D (M x N fp32, row stride ldd) = A (M x K) * B (N x K)^T, 16-bit operands
// (bf16, or fp16 with `f16`), with M % 128 == 0, K % 64 == 0 and N a
// multiple of 32; N above 256 runs in column tiles of the largest width
// <= 256 that divides it (the B map's box must be that many rows).
// `splits` > 1 runs split-K: partial products go to `work`
// (splits x M x N floats) and a reduction writes D (then ldd must be N).
// `split3`: A and B are [hi | lo] pairs (2K wide) and D is the
// three-product sum.
int gemm_tile_n(int N)
{
    if (N <= 0 || N % 32) return 0;
    for (int bn = std::min(N, 256); bn >= 32; bn -= 32)
        if (N % bn == 0) return bn;
    return 0;
}

cudaError_t launch_gemm_bf16_tn(const CUtensorMap &mapA, const CUtensorMap &mapB, float *D, int M, int N, int K,
                                int ldd, int smem_optin, int *d_err, cudaStream_t s, int splits, float *work,
                                int split3, int f16)
{
    const int BNv = gemm_tile_n(N);
    if (M % kBM || K % kBK || !BNv || splits < 1) return cudaErrorInvalidValue;
    if (splits > 1 && (!work || ldd != N)) return cudaErrorInvalidValue;
    const int kt_all = K / kBK;
    const int kchunk = (kt_all + splits - 1) / splits;
    const dim3 grid(M / kBM, splits, N / BNv);
    float *out = splits > 1 ? work : D;
    const long long stride = splits > 1 ? (long long)M * N : 0;
    const int halves = split3 ? 2 : 1;
    int stages = (int)((smem_optin - 64) / (halves * (kBM * kBK * 2 + BNv * kBK * 2)));
    if (stages > 8) stages = 8;
    if (stages < 2) return cudaErrorInvalidValue;
    cudaError_t e = cudaSuccess;
    auto go = [&](auto kern, size_t smem, int bn) {
        e = open_smem(kern, smem);
        if (!e)
            kern<<<grid, kGemmThreads, smem, s>>>(mapA, mapB, out, K, ldd, stages, d_err, kchunk, stride,
                                                  idesc_16bit(bn, f16));
    };
#define RP_GEMM_CASE(BN)                                                                             \
    case BN:                                                                                         \
        if (split3) go(k_gemm_bf16_tn<BN, 3>, gemm_smem<BN, 3>(stages), BN);                         \
        else go(k_gemm_bf16_tn<BN, 1>, gemm_smem<BN, 1>(stages), BN);                                \
        break;
    switch (BNv) {
        RP_GEMM_CASE(32)
        RP_GEMM_CASE(64)
        RP_GEMM_CASE(96)
        RP_GEMM_CASE(128)
        RP_GEMM_CASE(160)
        RP_GEMM_CASE(192)
        RP_GEMM_CASE(224)
        RP_GEMM_CASE(256)
    default: return cudaErrorInvalidValue;
    }
#undef RP_GEMM_CASE
    if (e) return e;
    e = cudaGetLastError();
    if (e || splits == 1) return e;
    const long long n4 = (long long)M * N / 4;   // N is a multiple of 32
    k_split_reduce<<<(unsigned)((n4 + 31) / 32), 256, 0, s>>>(reinterpret_cast<const float4 *>(work),
                                                               reinterpret_cast<float4 *>(D), n4, splits);
    return cudaGetLastError();
}

// Number of K splits: enough for one wave of CTAs (one per SM: the stage
// ring takes most of the shared memory), each split with at least
// `min_tiles` k-tiles -- and at least enough that no split accumulates more
// than kMaxSplitTiles k-tiles: the fp32 tensor-memory accumulator takes one
// rounding per MMA, so long K ranges (a 64^3 source is 4096 k-tiles) are cut
// into chains whose partial sums the reduction adds in a fixed order.
constexpr int kMaxSplitTiles = 64;

int gemm_splits(int M, int K, int split3, int sms, int min_tiles)
{
    (void)split3;
    const int mtiles = M / kBM;
    const int kt_all = K / kBK;
    int splits = std::max(1, sms / mtiles);
    splits = std::min(splits, std::max(1, kt_all / std::max(1, min_tiles)));
    return std::max(splits, (kt_all + kMaxSplitTiles - 1) / kMaxSplitTiles);
}

}  // namespace rp
