// Far pairs with two-sided factors: the lag-stacked operator [G_lo ... G_hi]
// of Eq. 11 between a far source box and a far target box, interpolated on
// both sides (rp_config.far_source_points > 0).
//
// With Chebyshev nodes x_a of the target box (tensor-product Lagrange
// weights L_a, as for the one-sided factors) and y_b of the source box
// (weights L'_b):
//
//   P_t(r_k, l) ~= sum_a L_a(r_k) c_t[a](l),
//   c_t[a](l)   = sum_n sum_{m = lo..hi} sum_b K_{tn,m}[a][b] q_n[b](l - m),
//   K_{tn,m}[a][b] = h_n^3 T(m dt - |x_a - y_b|/c) / |x_a - y_b|      (Eq. 11 between nodes),
//   q_n[b](j)   = sum_{k'} L'_b(r_k') S_n(k', j)                      (anterpolation of a slice).
//
// So a far source's slice enters through its q^3 node coefficients (taken
// at every push, k_far_anterp), and a far pair's factor is (B lags) blocks
// of r_t x r_s: its size does not depend on the grids.
//
// Every `batch` pushes (in a recorded graph: every step, the kernel reading
// the device step and doing nothing but on a batch's last push), one launch
// of k_far_gather gives every far target
// its node values for the next `batch` steps l0 .. l0 + batch - 1: per CTA,
//
//   D[(l, f)][a] = sum over its (source, lag) blocks of
//                  sum_b q_n[f][b](l0 + l - m) K_{tn,m}[a][b]
//
// is one tcgen05 GEMM (M = 128 rows = 32 steps x 4 fields, N = r_t padded,
// K = the blocks' source nodes), both operands bf16 hi/lo pairs with the
// three products accumulated in fp32 tensor memory.  The A tile of a block
// is a window of the source's mirrored coefficient ring (one TMA box), the
// B tile its factor block.  k_far_reduce adds each target's CTAs in a fixed
// order straight into its coefficient ring.  A far pair needs lag_lo >=
// batch, so that the window's newest sample is pushed before the launch.
#include <algorithm>
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <map>
#include <mutex>
#include <utility>

#include "rp_internal.h"
#include "rp_tc.cuh"

namespace rp {

namespace {

using namespace tc;

constexpr int kAnterpThreads = 256;
constexpr int kFarThreads2 = 256;
constexpr int kGatherThreads = 192;

__host__ __device__ __forceinline__ long long pos_mod(long long x, long long d) { return ((x % d) + d) % d; }

// 16- and 4-byte asynchronous global -> shared copies
__device__ __forceinline__ void an_cp16(void *smem, const void *gmem)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(su32(smem)), "l"(gmem) : "memory");
}
__device__ __forceinline__ void an_cp4(void *smem, const void *gmem)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(su32(smem)), "l"(gmem) : "memory");
}

// One block per (source plane z, far source): the plane's four fields
// copied into shared memory (all copies in flight at once), contracted over
// x (a thread per row, the rows of a warp starting at staggered columns so
// that they read different banks) and then over y with the source's
// Lagrange weights (per field: Q * Q partial sums); the last plane's block
// of a source adds the planes' sums in z order with the z weights and writes
// the node coefficients of this step, bf16 hi and lo, at both mirrored slots
// of the ring.  Q: the context's source nodes per axis; the weight tables
// are padded to Q columns, and a short axis's missing nodes (weight 0) are
// dropped when the coefficients are written.
template <int Q>
__global__ void __launch_bounds__(kAnterpThreads) k_far_anterp(const FarSrc2 *__restrict__ srcs, int nsrc, IoPtrs in,
                                                                long long step, const long long *d_step, int D,
                                                                int KS)
{
    constexpr int NQ = Q * Q, R3 = Q * Q * Q;
    extern __shared__ float4 an_smem[];
    __shared__ int last;
    if (step < 0) step = *d_step;   // graph replay: the step from the device counter
    const int si = blockIdx.y;
    if (si >= nsrc) return;
    const FarSrc2 S = srcs[si];
    const int z = blockIdx.x;
    if (z >= S.nz) return;
    const float *rho = in.rho[S.dom], *J = in.J[S.dom];
    const int nx = S.nx, ny = S.ny, nz = S.nz, nxy = nx * ny;
    const long long N = (long long)nxy * nz;
    float *sLx = reinterpret_cast<float *>(an_smem);    // [nx][Q] (zero-padded weights)
    float *sLy = sLx + nx * kMaxFarPts;                  // [ny][Q]
    float *tsum = sLy + ny * kMaxFarPts;                 // [4][ny][Q]; later the plane sums [nz][4][Q Q]
    float *slab = tsum + 4 * ny * kMaxFarPts;            // [4][ny][nx]
    for (int f = 0; f < 4; ++f) {
        const float *src = (f == 0 ? rho : J + (long long)(f - 1) * N) + (long long)z * nxy;
        float *dst = slab + f * nxy;
        if ((((uintptr_t)src | (uintptr_t)dst) & 15) == 0 && (nxy & 3) == 0) {
            for (int i = threadIdx.x; i < nxy / 4; i += blockDim.x) an_cp16(dst + 4 * i, src + 4 * i);
        } else {
            for (int i = threadIdx.x; i < nxy; i += blockDim.x) an_cp4(dst + i, src + i);
        }
    }
    for (int i = threadIdx.x; i < nx * Q; i += blockDim.x) sLx[i] = __ldg(S.Lx + i);
    for (int i = threadIdx.x; i < ny * Q; i += blockDim.x) sLy[i] = __ldg(S.Ly + i);
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();
    // rows of the plane: sum_i Lx[i][bx] S(i, j, z); the rows of a warp start
    // at different columns (banks) and wrap around
    for (int row = threadIdx.x; row < 4 * ny; row += blockDim.x) {
        const float *v = slab + row * nx;
        float acc[Q];
#pragma unroll
        for (int b = 0; b < Q; ++b) acc[b] = 0.0f;
        // every lane the same trip count (no divergence), columns wrapped
        int x = row % nx;
#pragma unroll 4
        for (int i = 0; i < nx; ++i) {
            const float sv = v[x];
            if constexpr (Q % 4 == 0) {   // whole 16-byte weight rows: no bank conflicts
#pragma unroll
                for (int b4 = 0; b4 < Q; b4 += 4) {
                    const float4 l = *reinterpret_cast<const float4 *>(sLx + x * Q + b4);
                    acc[b4] = fmaf(l.x, sv, acc[b4]);
                    acc[b4 + 1] = fmaf(l.y, sv, acc[b4 + 1]);
                    acc[b4 + 2] = fmaf(l.z, sv, acc[b4 + 2]);
                    acc[b4 + 3] = fmaf(l.w, sv, acc[b4 + 3]);
                }
            } else {
                const float *l = sLx + x * Q;
#pragma unroll
                for (int b = 0; b < Q; ++b) acc[b] = fmaf(l[b], sv, acc[b]);
            }
            x = x + 1 == nx ? 0 : x + 1;
        }
        if constexpr (Q % 4 == 0) {
#pragma unroll
            for (int b4 = 0; b4 < Q; b4 += 4)
                *reinterpret_cast<float4 *>(tsum + row * Q + b4) =
                    make_float4(acc[b4], acc[b4 + 1], acc[b4 + 2], acc[b4 + 3]);
        } else {
#pragma unroll
            for (int b = 0; b < Q; ++b) tsum[row * Q + b] = acc[b];
        }
    }
    __syncthreads();
    // columns: sum_j Ly[j][by] (row sums), four threads per output (rows
    // j = part, part + 4, ...), their sums added in a fixed order
    constexpr int n4 = 16 * NQ, n4w = (n4 + 31) / 32 * 32;   // whole warps: the shuffles take every lane
    for (int o4 = threadIdx.x; o4 < n4w; o4 += blockDim.x) {
        const bool act = o4 < n4;
        const int o = act ? o4 >> 2 : 0, part = o4 & 3;
        const int f = o / NQ, b = o % NQ, by = b / Q, bx = b % Q;
        const float *t = tsum + f * ny * Q + bx;
        float acc = 0.0f;
        if (act)
            for (int j = part; j < ny; j += 4) acc = fmaf(sLy[j * Q + by], t[j * Q], acc);
        acc += __shfl_xor_sync(0xffffffffu, acc, 1);
        acc += __shfl_xor_sync(0xffffffffu, acc, 2);
        if (act && part == 0) S.part[((long long)z * 4 + f) * NQ + b] = acc;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(S.count, 1u) == (unsigned)(nz - 1);
    __syncthreads();
    if (!last) return;
    __threadfence();
    // the source's last plane: sum_z Lz[z][bz] (plane sums), in z order,
    // from shared copies of every plane's sums and of the z weights (the
    // plane sums read from L2, bypassing L1, which may hold stale lines)
    const int np = nz * 4 * NQ;
    float *ps = tsum, *sLz = tsum + np;   // the slab and row sums are dead
    for (int i = threadIdx.x; i < np; i += blockDim.x) ps[i] = __ldcg(S.part + i);
    for (int i = threadIdx.x; i < nz * Q; i += blockDim.x) sLz[i] = __ldg(S.Lz + i);
    __syncthreads();
    const long long slot = pos_mod(step, D);
    for (int o = threadIdx.x; o < 4 * R3; o += blockDim.x) {
        const int f = o / R3, bp = o % R3, bz = bp / NQ, bxy = bp % NQ, by = bxy / Q, bx = bxy % Q;
        if (bx >= S.qx || by >= S.qy || bz >= S.qz) continue;   // a node a short axis lacks
        const int b = (bz * S.qy + by) * S.qx + bx;
        const float *pp = ps + f * NQ + bxy;
        float acc = 0.0f;
        for (int zz = 0; zz < nz; ++zz) acc = fmaf(sLz[zz * Q + bz], pp[zz * 4 * NQ], acc);
        const __nv_bfloat16 hi = __float2bfloat16(acc);
        const __nv_bfloat16 lo = __float2bfloat16(acc - __bfloat162float(hi));
#pragma unroll
        for (int mirror = 0; mirror < 2; ++mirror) {
            __nv_bfloat16 *row = S.qring + ((slot + mirror * D) * 4 + f) * 2 * KS;
            row[b] = hi;
            row[KS + b] = lo;
        }
    }
    if (threadIdx.x == 0) *S.count = 0u;
}

// The factor blocks in FP64: element (a, b) of block kb is Eq. 11 between
// target node a and source node b for the block's lag, h_s^3 T(m - R/(c dt))
// / R, stored as bf16 hi and lo (rows past r_t and columns past r_s zero).
__global__ void __launch_bounds__(kFarThreads2) k_far_build_fac(const FarBuild *__restrict__ blocks, int nblocks,
                                                                 const double *__restrict__ tnodes,
                                                                 const double *__restrict__ snodes, int BN, int KS,
                                                                 double inv_cdt, __nv_bfloat16 *fac)
{
    const long long per = (long long)BN * KS, total = per * nblocks;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int kb = (int)(i / per);
        const int a = (int)((i % per) / KS), b = (int)(i % KS);
        const FarBuild B = blocks[kb];
        double w = 0.0;
        if (a < B.rt && b < B.rs) {
            const double *x = tnodes + 3LL * (B.t0 + a), *y = snodes + 3LL * (B.s0 + b);
            const double dx = x[0] - y[0], dy = x[1] - y[1], dz = x[2] - y[2];
            const double R = sqrt(dx * dx + dy * dy + dz * dz);
            const double T = 1.0 - fabs((double)B.lag - R * inv_cdt);
            if (T > 0.0) w = B.vol * T / R;
        }
        const __nv_bfloat16 hi = __float2bfloat16((float)w);
        const __nv_bfloat16 lo = __float2bfloat16((float)(w - (double)__bfloat162float(hi)));
        __nv_bfloat16 *row = fac + (long long)(B.fac_row + a) * 2 * KS;
        row[b] = hi;
        row[KS + b] = lo;
    }
}

// The gathered GEMM (see the file comment).  Warp 0: TMA producer of the
// stages (A hi, A lo: a 128-row window of the source's coefficient ring; B
// hi, B lo: the factor block); warp 1: tensor-memory allocation and the MMA
// issue (three products per 16-wide K step); warps 2-5: epilogue into the
// CTA's slot of `work` ([128 rows (l, f)][BN]).  Bounded waits as in
// k_gemm_bf16_tn.
template <int BN>
__global__ void __launch_bounds__(kGatherThreads, 1)
    k_far_gather(const __grid_constant__ CUtensorMap mapQ, const __grid_constant__ CUtensorMap mapF,
                 const FarTask *__restrict__ tasks, const FarKBlock *__restrict__ kbs, int KS, int D, long long l0,
                 const long long *d_step, int batch, float *work, int stages, int *err)
{
    if (l0 < 0) {   // graph replay: every step's launch, working on the last push of a batch only
        const long long s = *d_step;
        if (s % batch != batch - 1) return;
        l0 = s + 1;
    }
    constexpr int A_BYTES = kBM * kBK * 2, B_BYTES = BN * kBK * 2;
    constexpr int B_OFF = 2 * A_BYTES;
    constexpr int STAGE = 2 * (A_BYTES + B_BYTES);
    constexpr int TCOLS = tmem_cols<BN>();
    extern __shared__ __align__(1024) unsigned char smem[];
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + (size_t)stages * STAGE);
    uint64_t *empty = full + stages;
    uint64_t *done = empty + stages;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(done + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const FarTask task = tasks[blockIdx.x];
    const int kchunks = KS / kBK;
    const int ktiles = (task.kb1 - task.kb0) * kchunks;
    float *out = work + (long long)blockIdx.x * kBM * BN;
    if (su32(smem) & 1023u) {   // the swizzled descriptors assume 1024-byte aligned stages
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
            const FarKBlock K = kbs[task.kb0 + kt / kchunks];
            const int kk = (kt % kchunks) * kBK;
            // rows of source K.src's ring holding steps l0 - lag .. l0 - lag + 31
            const int arow = (int)(((long long)K.src * 2 * D + pos_mod(l0 - K.lag, D)) * 4);
            unsigned char *st = smem + (size_t)s * STAGE;
            bar_expect(&full[s], STAGE);
            tma_2d(st, &mapQ, kk, arow, &full[s]);
            tma_2d(st + A_BYTES, &mapQ, KS + kk, arow, &full[s]);
            tma_2d(st + B_OFF, &mapF, kk, K.fac_row, &full[s]);
            tma_2d(st + B_OFF + B_BYTES, &mapF, KS + kk, K.fac_row, &full[s]);
        }
        for (int r = kt > stages ? kt - stages : 0; r < kt; ++r)
            if (!bar_wait(&full[r % stages], (r / stages) & 1)) atomicExch(err, 1);
    } else if (warp == 1 && lane == 0) {
        // ---------------------------------------------------------------- MMA issue
        const uint32_t ID = idesc_16bit(BN, 0);
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
            for (int kk = 0; kk < kBK / 16; ++kk) {
                mma_bf16(tmem, desc_sw128(a + kk * 32), desc_sw128(b + kk * 32), ID, (kt | kk) ? 1u : 0u);
                mma_bf16(tmem, desc_sw128(a + kk * 32), desc_sw128(b + B_BYTES + kk * 32), ID, 1u);
                mma_bf16(tmem, desc_sw128(a + A_BYTES + kk * 32), desc_sw128(b + kk * 32), ID, 1u);
            }
            mma_commit(&empty[s]);
        }
        mma_commit(done);
    } else if (warp >= 2) {
        // ---------------------------------------------------------------- epilogue
        const bool ok = bar_wait(done, 0);
        if (!ok) atomicExch(err, 1);
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int quarter = warp & 3;
        const int row = 32 * quarter + lane;
        if (ok && !*abort_flag && ktiles > 0) {
#pragma unroll 1
            for (int c = 0; c < BN; c += 32) {
                uint32_t r[32];
                tmem_ld32(tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)c, r);
                float4 *o = reinterpret_cast<float4 *>(out + (size_t)row * BN + c);
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    o[j] = make_float4(__uint_as_float(r[4 * j]), __uint_as_float(r[4 * j + 1]),
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

// Node values of steps l0 .. l0 + batch - 1 of every far target with
// low-rank pairs: its CTAs' partial sums added in task order, written (not
// added) into its coefficient ring.  Thread (l, a, f) of target blockIdx.y.
__global__ void __launch_bounds__(kFarThreads2) k_far_reduce(const FarTarget *__restrict__ tgts, int ntgt,
                                                              const float *__restrict__ work, int BN, long long l0,
                                                              const long long *d_step, int batch)
{
    if (l0 < 0) {   // graph replay, as k_far_gather
        const long long s = *d_step;
        if (s % batch != batch - 1) return;
        l0 = s + 1;
    }
    const int ti = blockIdx.y;
    if (ti >= ntgt) return;
    const FarTarget T = tgts[ti];
    if (T.lag_hi_max < 0 || T.task1 <= T.task0) return;
    const int per = T.r * 4;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < batch * per; i += gridDim.x * blockDim.x) {
        const int l = i / per, a = (i % per) / 4, f = i % 4;
        float s = 0.0f;
        for (int t = T.task0; t < T.task1; ++t) s += work[((long long)t * kBM + l * 4 + f) * BN + a];
        T.cring[pos_mod(l0 + l, T.depth) * per + a * 4 + f] = s;
    }
}

template <class K>
cudaError_t open_smem2(K kern, size_t smem)
{
    static std::mutex mu;
    static std::map<std::pair<const void *, int>, int> opened;
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

}  // namespace

int far_gather_bn(int r)
{
    for (int bn : {32, 64, 128, 256})
        if (r <= bn) return bn;
    return 0;
}

size_t smem_far_anterp(int max_plane, int max_n)
{
    // the x and y weights, the row sums (4 x ny x qx), one plane of the four
    // fields; the last block reuses the last two for every plane's sums
    // (nz x 4 x qx qy) and the z weights (nz x qz)
    const size_t main = 2 * (size_t)max_n * kMaxFarPts + 4 * (size_t)max_n * kMaxFarPts + 4 * (size_t)max_plane;
    const size_t tail = 2 * (size_t)max_n * kMaxFarPts + (size_t)max_n * (4 * kMaxFarPts * kMaxFarPts + kMaxFarPts);
    return sizeof(float) * std::max(main, tail);
}

cudaError_t launch_far_anterp(const FarSrc2 *d_srcs, int nsrc, int q, int max_nz, int max_plane, int max_n,
                              const IoPtrs &in, long long step, const long long *d_step, int D, int KS, cudaStream_t s)
{
    if (nsrc <= 0) return cudaSuccess;
    const size_t smem = smem_far_anterp(max_plane, max_n);
    cudaError_t e = cudaErrorInvalidValue;
    auto go = [&](auto kern) {
        e = open_smem2(kern, smem);
        if (!e) kern<<<dim3(max_nz, nsrc), kAnterpThreads, smem, s>>>(d_srcs, nsrc, in, step, d_step, D, KS);
    };
    switch (q) {
    case 2: go(k_far_anterp<2>); break;
    case 3: go(k_far_anterp<3>); break;
    case 4: go(k_far_anterp<4>); break;
    case 5: go(k_far_anterp<5>); break;
    case 6: go(k_far_anterp<6>); break;
    case 7: go(k_far_anterp<7>); break;
    case 8: go(k_far_anterp<8>); break;
    default: return cudaErrorInvalidValue;
    }
    return e ? e : cudaGetLastError();
}

cudaError_t launch_far_build_fac(const FarBuild *d_blocks, int nblocks, const double *d_tnodes,
                                 const double *d_snodes, int BN, int KS, double inv_cdt, __nv_bfloat16 *fac,
                                 cudaStream_t s)
{
    if (nblocks <= 0) return cudaSuccess;
    const long long total = (long long)nblocks * BN * KS;
    const int blocks = (int)std::min<long long>((total + kFarThreads2 - 1) / kFarThreads2, 65535LL * 16);
    k_far_build_fac<<<blocks, kFarThreads2, 0, s>>>(d_blocks, nblocks, d_tnodes, d_snodes, BN, KS, inv_cdt, fac);
    return cudaGetLastError();
}

cudaError_t launch_far_gather(const CUtensorMap &mapQ, const CUtensorMap &mapF, const FarTask *d_tasks, int ntasks,
                              const FarKBlock *d_kb, int BN, int KS, int D, long long l0, const long long *d_step,
                              int batch, float *work, int smem_optin, int *d_err, cudaStream_t s)
{
    if (ntasks <= 0) return cudaSuccess;
    if (KS % kBK || D < 32) return cudaErrorInvalidValue;
    const size_t stage = 2 * ((size_t)kBM * kBK * 2 + (size_t)BN * kBK * 2);
    int stages = (int)((smem_optin - 1024 - 64) / stage);
    if (stages > 6) stages = 6;
    if (stages < 2) return cudaErrorInvalidValue;
    const size_t smem = (size_t)stages * stage + 8 * (2 * (size_t)stages + 1) + 16 + 1024;
    cudaError_t e = cudaSuccess;
    auto go = [&](auto kern) {
        e = open_smem2(kern, smem);
        if (!e)
            kern<<<ntasks, kGatherThreads, smem, s>>>(mapQ, mapF, d_tasks, d_kb, KS, D, l0, d_step, batch, work, stages,
                                                     d_err);
    };
    switch (BN) {
    case 32: go(k_far_gather<32>); break;
    case 64: go(k_far_gather<64>); break;
    case 128: go(k_far_gather<128>); break;
    case 256: go(k_far_gather<256>); break;
    default: return cudaErrorInvalidValue;
    }
    return e ? e : cudaGetLastError();
}

cudaError_t launch_far_reduce(const FarTarget *d_tgts, int ntgt, const float *work, int BN, long long l0,
                              const long long *d_step, int batch, int max_r, cudaStream_t s)
{
    if (ntgt <= 0) return cudaSuccess;
    const int bx = (batch * max_r * 4 + kFarThreads2 - 1) / kFarThreads2;
    k_far_reduce<<<dim3(bx, ntgt), kFarThreads2, 0, s>>>(d_tgts, ntgt, work, BN, l0, d_step, batch);
    return cudaGetLastError();
}

}  // namespace rp
