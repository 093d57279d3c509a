// Internal structures shared by the host planner (rp_api.cu) and the kernels.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace rp {

constexpr int kMaxDomains = 256;
constexpr int kMaxFFT = 192;   // largest padded FFT length per axis
constexpr int kThreads = 256;        // threads per block: ring push, register-blocked MAC
constexpr int kPlaneThreads = 256;   // threads per block of the forward and inverse plane passes
constexpr int kColumnThreads = 256;  // threads per block of the forward column pass
constexpr int kTileY = 16;     // ky columns per block of the column passes
constexpr int kTileYPad = 17;  // shared-memory row stride of a column tile (bank spread)

// Spectra (source rings and lag kernels) are stored tile-major:
// [kx][ky tile][kz][16 ky], so that the block of one (kx, 16-ky tile) over all
// kz -- what one column pass reads or writes -- is contiguous in memory.
// Columns past my in the last tile are padding (zero).
inline __host__ __device__ long long spec_cells(int kx, int my, int mz)
{
    return (long long)kx * ((my + kTileY - 1) / kTileY) * mz * kTileY;
}

// Radix split of one FFT axis: M = R * L with L a power of two (lanes) and
// R in {1, 2, 3, 4, 6} (registers per lane).
struct Axis {
    int M, R, L, logL;
};

// One (source domain, padded size) spectral history ring and its forward
// transform.  A slot holds one step's spectra, complex64, tile by tile:
// [kx][ky tile of 16][4 fields][kz][16] (4 * spec_cells in all), kx in
// [0, mx/2], so the four field tiles of one (kx, ky) tile are contiguous.
struct FarTarget;

struct FwdRing {
    int nx, ny, nz;          // source grid
    Axis ax, ay, az;         // padded sizes
    int kx;                  // mx/2 + 1
    int src;                 // source domain id
    int depth;               // ring depth in steps
    float2 *ring;            // [depth][tiles][4 fields][mz][16]
    float2 *t1;              // scratch after the plane pass: [4][kx][nz][my]
    long long slot_elems;    // float2 per slot = 4 * spec_cells
    const float2 *tw_x, *tw_y, *tw_z;  // twiddles exp(-2 pi i j/M), j < M
    int plane0;              // first block of this ring in the plane-pass grid (4 fields x nz planes)
    int tile0;               // first block of this ring in the column-pass grid (kx x ky tiles)
    __nv_bfloat16 *far_x;    // far-path batch matrix [4 batch][2 ks] of this source (one ring per source), or null
    int far_ks;              // its half row width
    int lag_off;             // the column pass of step l writes the slice of step l - lag_off (0 but for
                             // a spilled window transformed with the push, which writes step l - lo)
    const long long *d_step; // the step, for launches made with step < 0 (graph replay)
};

// One (source, lag) term of a target's spectral sum: G_m (kernel spectrum of
// Eq. 11 for lag m, scaled by 1/(mx my mz)) times the source spectrum of
// step l - m.
struct MacEntry {
    const void *g;           // [spec_cells] float (is_real) or float2
    const float2 *ring;      // the source's spectral ring at this target's size
    long long slot_elems;
    int depth;
    int lag;
    int is_real;
};

// A target domain evaluated by the FFT path.
struct InvTarget {
    int nx, ny, nz;
    Axis ax, ay, az;
    int kx;
    int dom;                 // domain id
    int e0, e1;              // its MacEntry range
    int er;                  // entries e0..er-1 have real kernels (self pair), er..e1-1 complex
    float2 *t2;              // scratch after the column pass: [4][kx][nz][my]
    const float2 *tw_x, *tw_y, *tw_z;
    int tile0;               // first block in the MAC/column grid
    int plane0;              // first block in the plane grid
    int has_direct;          // direct pairs add onto this target afterwards
    int pad_;
    const FarTarget *far;    // far-path coefficients interpolated onto this target here, or null
    const long long *d_step; // the step, for launches made with step < 0 (graph replay)
};

// A (target, source) pair evaluated by the direct retarded sum.
struct DirectPair {
    int src;
    int nx_s, ny_s, nz_s;
    long long n_s;
    double dx, dy, dz;       // o_t - o_s
    float hs;
    float vol;               // hs^3
    float self_w;            // C hs^2 (self pair only)
    int is_self;
    int lag_lo, nlag;        // samples of lags lag_lo .. lag_lo + nlag - 1
    const float *raw;        // source raw ring [depth][4][n_s]
    int depth;
    int pad_;
};

// A target of the direct kernel: its pair list and grid.
struct DirectTarget {
    int dom;
    int nx, ny, nz;
    long long n;
    double ht;
    int p0, p1;              // DirectPair range
    int block0;              // first block in the direct grid
    int accumulate;          // add onto the output (FFT pairs wrote it) instead of writing
    const long long *d_step; // the step, for launches made with step < 0 (graph replay)
};

// A raw history ring (rho, Jx, Jy, Jz per slot).
struct RawRing {
    float *ring;             // [depth][4][n]
    long long n;
    int depth;
    int pad_;
    const long long *d_step; // the step, for launches made with step < 0 (graph replay)
};

// ---- far pairs (rp_far.cu): interpolative low-rank factors

constexpr int kMaxFarPts = 8;   // interpolation nodes per axis of a target box

// One row of a source's factor matrix W: the node of a far target, relative
// to the source's origin, and a lag (lag < 0: padding row).
struct FarRow {
    float x, y, z;
    int lag;
};

// A source with far pairs: its batch matrix X (rows slice*4 + field, ks columns).
struct FarSource {
    int dom;
    int ks;                  // columns of W and X: node count rounded up to 64
    long long n;
    __nv_bfloat16 *X;
};

// A target with far pairs: interpolation weights and its coefficient ring.
struct FarTarget {
    int dom;
    int nx, ny, nz;
    int px, py, pz, r;       // nodes per axis, r = px*py*pz
    const float *Lx, *Ly, *Lz;   // [n][p] Lagrange weights per axis
    float *cring;            // [depth][r][4]
    int depth;
    int lag_hi_max;          // largest lag of the target's far pairs
    int task0, task1;        // two-sided factors: this target's CTAs of the gathered GEMM
    int interp_add;          // k_far_interp (targets without an FFT pass): add onto the output (1) or write it (0)
    int pad_;
};

// ---- two-sided far factors (rp_far2.cu, rp_config.far_source_points > 0)
//
// A far source's slice is anterpolated onto q^3 Chebyshev nodes y_b of its
// box at every push, q_b = sum_k' L_b(r_k') S(k') (tensor-product Lagrange
// weights), into a node-coefficient history ring: bf16 hi/lo rows
// [2D][4 fields][2 KS] (hi in columns 0..KS-1, lo in KS..2KS-1) with step j
// at slots j mod D and j mod D + D (mirrored, so that any window of up to D
// consecutive steps is one contiguous block of 4 * window rows).
struct FarSrc2 {
    int dom;
    int nx, ny, nz;
    int qx, qy, qz, r;       // nodes per axis, r = qx*qy*qz <= KS
    const float *Lx, *Ly, *Lz;   // [n][Q] Lagrange weights per axis (Q = far_source_points; zero past q)
    float *part;             // [nz][4][Q*Q]: per-plane partial sums of one push
    unsigned int *count;     // planes done in this push (the last plane's block reduces over z)
    __nv_bfloat16 *qring;    // this source's rows of the shared ring array
    int qrow0;               // its first row there: source index * 2D * 4
    int pad_;
};

// One block of a target's factor: Eq. 11 between the target's r_t nodes
// (rows, padded to BN) and source src's nodes (columns) for lag `lag`,
// rows fac_row .. fac_row + BN - 1 of the factor array.
struct FarKBlock {
    int src;                 // FarSrc2 index
    int lag;
    int fac_row;
    int pad_;
};

// One CTA of the gathered GEMM: k-blocks [kb0, kb1) of target `tgt`
// (FarTarget index); its partial sums go to work slot = its index.
struct FarTask {
    int tgt;
    int kb0, kb1;
    int pad_;
};

// Node positions of a factor block's build: target nodes t0 .. t0 + rt - 1,
// source nodes s0 .. s0 + rs - 1 of the node tables (bohr), source volume.
struct FarBuild {
    int t0, rt, s0, rs;
    int lag, fac_row;
    double vol;
};

// Rows of source n's W that belong to target t: row0 + (m - lag_lo) * r + a.
struct FarLink {
    int row0;
    int r;
    int nlag;
    int lag_lo;
    float *cring;
    int depth;
    int pad_;
};

struct IoPtrs {
    const float *rho[kMaxDomains];
    const float *J[kMaxDomains];
};

struct OutPtrs {
    float *phi[kMaxDomains];
    float *A[kMaxDomains];
};

// ---- launchers (rp_fft_kernels.cu, rp_direct.cu) ----
//
// `size_class` selects the kernel instantiation: a cubic padded size M in
// {32, 48, 64, 96, 128, 192} compiled with constant shapes, or 0 for the
// general runtime-shaped kernels.  Rings [r0, r1) / targets [t0, t1) of one
// launch share the class; `block_lo` is the first block of the range.

int size_class(const Axis &ax, const Axis &ay, const Axis &az);

cudaError_t launch_ring_push(const RawRing *d_rings, const IoPtrs &in, int d0, int d1,
                             const int *h_block0, int nblocks, long long step,
                             cudaStream_t s);
// The plane passes in two forms for size classes M = 64, 96, 128: tile = true
// runs the two-stage shared-memory tile transform (fewer instructions, 3
// blocks per SM: the better form while a class's planes fit in about one wave),
// tile = false the lane-shuffle line (5-6 blocks per SM: the better form over
// many waves).  The planner picks per class from its block count
// (plane_tile_form), so a plan's bits do not depend on timing.  The inverse
// pass at M = 128 takes the tile form at any block count: there both forms
// hold about 100 KB of shared memory per block (two blocks per SM), so the
// lane-shuffle form has no occupancy to trade for its extra instructions.
constexpr int kPlaneTileMaxBlocks = 1024;
bool plane_tile_class(int size_class);
inline bool plane_tile_form(int size_class, int blocks, bool inverse)
{
    if (!plane_tile_class(size_class)) return false;
    return blocks <= kPlaneTileMaxBlocks || (inverse && size_class == 128);
}
cudaError_t launch_fwd_plane(int size_class, bool tile, const FwdRing *d_rings, const IoPtrs &in, int r0, int r1,
                             int block_lo, int nblocks, size_t smem, int far_slot, cudaStream_t s);
cudaError_t launch_fwd_column(int size_class, const FwdRing *d_rings, int r0, int r1, int block_lo,
                              int nblocks, size_t smem, long long step, cudaStream_t s);
cudaError_t launch_mac_inv_column(int size_class, bool comp, const InvTarget *d_tgts, int t0, int t1, int block_lo,
                                  const MacEntry *d_entries, int nblocks, size_t smem, long long step,
                                  int clamp, cudaStream_t s);
cudaError_t launch_inv_plane(int size_class, bool tile, const InvTarget *d_tgts, int t0, int t1, int block_lo,
                             const OutPtrs &out, int nblocks, size_t smem, float inv_c, long long step,
                             cudaStream_t s);
cudaError_t launch_direct(const DirectTarget *d_tgts, int ntgt, const DirectPair *d_pairs,
                          const OutPtrs &out, int nblocks, size_t smem, long long step, int clamp,
                          float inv_cdt, float inv_c, cudaStream_t s);

// Ground-state split and graph-replay step counter (rp_ground.cu).
cudaError_t launch_step_advance(long long *d_step, cudaStream_t s);
cudaError_t launch_ground_delta(const float *rho, const float *J, const float *ground, float *delta, long long N,
                                int sms, cudaStream_t s);

// Fields from the potentials (rp_fields.cu).
cudaError_t launch_fields(int nx, int ny, int nz, double h, double c, double dt, const float *phi, const float *A,
                          const float *A1, const float *A2, float *E, float *B, cudaStream_t s);

// TMA-fed MAC (rp_mac_tma.cu): cubic classes 32..192 only.
int mac_tma_stages(int M, int smem_optin, bool comp);
cudaError_t launch_wait_selftest(long long limit_cycles, int *d_err, cudaStream_t s);
size_t mac_tma_smem(int M, int nstages, bool comp);
cudaError_t open_mac_tma_smem_limit(int max_optin);
// comp: the Kahan-compensated variant (consumer_warps must be kCompWarps)
constexpr int kCompWarps = 12;
cudaError_t launch_mac_tma(int cls, int consumer_warps, bool comp, const InvTarget *d_tgts, int t0, int t1,
                           int tile_lo, int ntiles, const MacEntry *d_entries, long long step, int clamp, int nstages,
                           int grid, int *d_err, cudaStream_t s);

// tcgen05 bf16 GEMM (rp_gemm_tc.cu): D (M x N fp32) = A (M x K) * B (N x K)^T
bool encode_bf16_rows(void *encode_fn, struct CUtensorMap_st *map, const void *base, uint64_t rows,
                      uint64_t cols, uint32_t box_rows);
cudaError_t launch_gemm_bf16_tn(const struct CUtensorMap_st &mapA, const struct CUtensorMap_st &mapB, float *D,
                                int M, int N, int K, int ldd, int smem_optin, int *d_err, cudaStream_t s,
                                int splits = 1, float *work = nullptr, int split3 = 0, int f16 = 0);
int gemm_tile_n(int N);   // column tile width of an N-wide GEMM (the B map's box rows), 0 if unsupported
int gemm_splits(int M, int K, int split3, int sms, int min_tiles);

// far-pair kernels (rp_far.cu)
cudaError_t launch_far_build_w(const FarRow *d_rows, int nrows, const int n[3], double h, double inv_cdt, int ks,
                               __nv_bfloat16 *W, cudaStream_t s);
cudaError_t launch_far_convert(const FarSource *d_srcs, int nsrc, const IoPtrs &in, int slot, long long max_n,
                               cudaStream_t s);
cudaError_t launch_far_zero(const FarTarget *d_tgts, int ntgt, long long j1, int batch, int max_r, cudaStream_t s);
cudaError_t launch_far_interp(const FarTarget *d_tgts, int ntgt, int nplanes, const OutPtrs &out, long long step,
                              const long long *d_step, float inv_c, cudaStream_t s);
cudaError_t launch_far_scatter(const FarLink *d_links, int nlinks, int nthreads, const float *Z, int ldz, long long j0,
                               int batch, cudaStream_t s);

// two-sided far factors (rp_far2.cu)
// step / l0 < 0: read the step from d_step (graph replay; the gather and the
// reduction then run on a batch's last push only)
cudaError_t launch_far_anterp(const FarSrc2 *d_srcs, int nsrc, int q, int max_nz, int max_plane, int max_n,
                              const IoPtrs &in, long long step, const long long *d_step, int D, int KS, cudaStream_t s);
size_t smem_far_anterp(int max_plane, int max_n);   // max_plane: nx ny, max_n: nx, ny and nz, over the far sources
cudaError_t launch_far_build_fac(const FarBuild *d_blocks, int nblocks, const double *d_tnodes,
                                 const double *d_snodes, int BN, int KS, double inv_cdt, __nv_bfloat16 *fac,
                                 cudaStream_t s);
cudaError_t launch_far_gather(const CUtensorMap &mapQ, const CUtensorMap &mapF, const FarTask *d_tasks, int ntasks,
                              const FarKBlock *d_kb, int BN, int KS, int D, long long l0, const long long *d_step,
                              int batch, float *work, int smem_optin, int *d_err, cudaStream_t s);
cudaError_t launch_far_reduce(const FarTarget *d_tgts, int ntgt, const float *work, int BN, long long l0,
                              const long long *d_step, int batch, int max_r, cudaStream_t s);
int far_gather_bn(int r);   // gathered-GEMM column tile for r target nodes (0 if more than 256)

// shared-memory sizes the kernels need for the given shapes
size_t smem_fwd_plane(int size_class, bool tile, int ny, const Axis &ax);   // of the form the class runs
size_t smem_fwd_column(const Axis &az);   // four fields per block
size_t smem_mac_inv_column(const Axis &az);
size_t smem_inv_plane(int size_class, bool tile, int nx, int ny, const Axis &ax, const Axis &ay);
cudaError_t open_kernel_smem_limits(int max_optin);

// ---- host FP64 kernel spectra (rp_spectra.cpp) ----

// The kernel of Eq. 11 for one lag m of the pair (target t, source s),
// placed for a linear (non-cyclic) convolution on an mx x my x mz grid and
// transformed with an FP64 FFT; returns the half spectrum (kx <= mx/2) in the
// tile-major layout of spec_cells, scaled by 1/(mx my mz).  If real_out, only real parts are
// written to out_real (the self pair's kernel is even, so its spectrum is real).
void build_kernel_spectrum(const double o_t[3], const int n_t[3], const double o_s[3],
                           const int n_s[3], double h, bool self_pair, int lag, double c,
                           double dt, const int m[3], bool real_out, float *out_real,
                           float2 *out_cplx);

// Cell-averaged 1/R over a cube of side 1 (the self weight is this times h^2).
double cube_average_constant();

}  // namespace rp
