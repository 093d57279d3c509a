// Learned far field, data path: source moments, canonical network rows,
// training labels from the direct retarded sum, and the output stage that
// adds the network's node values to the far path's target coefficients.
//
// Moments (l <= 2) of a slice about its box centre c_s, per field (FP32 per
// thread, FP64 across warps and planes):
//   Q = sum S h^3,  p_i = sum S d_i h^3,  q_ij = sum S d_i d_j h^3
// (d = r - c_s; q as xx xy xz yy yz zz), the monopole, dipole and quadrupole
// that carry the far interaction (Sec. IV).  A pair's network rows are these
// moments rotated into the pair's canonical frame (first axis from c_s to
// c_t; the current's components rotate as a vector) and sampled by linear
// interpolation in time (Eq. 7's hat basis) at the W times t - tau_c - o_k,
// tau_c = |c_t - c_s| / (c dt), o_k = k - (W/2 - 1); each field's row is
// the window and the window times L0/|c_t - c_s|, divided by nu, the RMS of
// its first half.  The network returns y_a = R_a value'(x_a) / nu at the
// 64 canonical nodes x_a (R_a = |x_a - c_s|), from which the output stage
// re-interpolates the target's own nodes and rotates the current's
// potentials back.
#include <algorithm>
#include <cmath>

#include "rp_learned.h"
#include "rp_learned_data.h"

namespace rp {

namespace {

constexpr int kMomThreads = 256;

// ---------------------------------------------------------------- moments

// Partial moments of one z-plane of one field: each thread sums its few
// points in FP32 (coordinates relative to the box centre), the warps reduce
// by shuffles, and the warp partials are added in FP64 in a fixed order.
__global__ void __launch_bounds__(kMomThreads) k_moment_part(const MomentJob *__restrict__ jobs, IoPtrs in)
{
    __shared__ double red[kMomThreads / 32][kLMom];
    const MomentJob &J = jobs[blockIdx.z];
    const int z = blockIdx.x, f = blockIdx.y;
    if (z >= J.nz) return;
    const long long N = (long long)J.nx * J.ny * J.nz;
    const float *rho = J.rho ? J.rho : in.rho[J.dom];
    const float *cur = J.rho ? J.J : in.J[J.dom];
    const float *S = (f == 0 ? rho : cur + (long long)(f - 1) * N) + (long long)z * J.nx * J.ny;
    const float h = (float)J.h, ox = (float)J.ox, oy = (float)J.oy;
    const float dz = (float)(J.oz + J.h * z);
    float acc[kLMom] = {};
    for (int i = threadIdx.x; i < J.nx * J.ny; i += blockDim.x) {
        const float dx = fmaf(h, (float)(i % J.nx), ox), dy = fmaf(h, (float)(i / J.nx), oy);
        const float s = __ldg(S + i);
        const float sx = s * dx, sy = s * dy, sz = s * dz;
        acc[0] += s;
        acc[1] += sx; acc[2] += sy; acc[3] += sz;
        acc[4] = fmaf(sx, dx, acc[4]); acc[5] = fmaf(sx, dy, acc[5]); acc[6] = fmaf(sx, dz, acc[6]);
        acc[7] = fmaf(sy, dy, acc[7]); acc[8] = fmaf(sy, dz, acc[8]); acc[9] = fmaf(sz, dz, acc[9]);
    }
#pragma unroll
    for (int m = 0; m < kLMom; ++m)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc[m] += __shfl_xor_sync(0xffffffffu, acc[m], o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0)
        for (int m = 0; m < kLMom; ++m) red[warp][m] = acc[m];
    __syncthreads();
    if (threadIdx.x < kLMom) {
        double t = 0.0;
        for (int w = 0; w < kMomThreads / 32; ++w) t += red[w][threadIdx.x];
        J.part[((long long)f * J.nz + z) * kLMom + threadIdx.x] = t * J.h * J.h * J.h;
    }
}

__global__ void k_moment_final(const MomentJob *__restrict__ jobs, long long slot)
{
    const MomentJob J = jobs[blockIdx.x];
    const int t = threadIdx.x;
    if (t >= 4 * kLMom) return;
    const int f = t / kLMom, m = t % kLMom;
    double s = 0.0;
    for (int z = 0; z < J.nz; ++z) s += J.part[((long long)f * J.nz + z) * kLMom + m];
    J.out[(slot % J.out_depth) * 4 * kLMom + t] = (float)s;
}

// ---------------------------------------------------------------- network rows

// Rotate one [4][10] moment set into the frame with rows R.
__device__ void rotate_moments(const float *M, const float *R, float *out)
{
    float sp[4][kLMom];
    for (int f = 0; f < 4; ++f) {
        const float *m = M + f * kLMom;
        sp[f][0] = m[0];
        for (int i = 0; i < 3; ++i) sp[f][1 + i] = R[3 * i] * m[1] + R[3 * i + 1] * m[2] + R[3 * i + 2] * m[3];
        const float q[3][3] = {{m[4], m[5], m[6]}, {m[5], m[7], m[8]}, {m[6], m[8], m[9]}};
        float rq[3][3];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) rq[i][j] = R[3 * i] * q[0][j] + R[3 * i + 1] * q[1][j] + R[3 * i + 2] * q[2][j];
        float qq[3][3];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) qq[i][j] = rq[i][0] * R[3 * j] + rq[i][1] * R[3 * j + 1] + rq[i][2] * R[3 * j + 2];
        sp[f][4] = qq[0][0]; sp[f][5] = qq[0][1]; sp[f][6] = qq[0][2];
        sp[f][7] = qq[1][1]; sp[f][8] = qq[1][2]; sp[f][9] = qq[2][2];
    }
    for (int m = 0; m < kLMom; ++m) {
        out[m] = sp[0][m];
        for (int k = 0; k < 3; ++k)
            out[(1 + k) * kLMom + m] = R[3 * k] * sp[1][m] + R[3 * k + 1] * sp[2][m] + R[3 * k + 2] * sp[3][m];
    }
}

// One block per (pair, sample): the window of canonical moments, then the
// four fields' rows X16[4 * row + f] and scales nu.
__global__ void k_features(const LPair *__restrict__ pairs, const FeatRow *__restrict__ rows, int nrows,
                           long long step, __half *__restrict__ X16, float *__restrict__ Xf, float *__restrict__ nu)
{
    __shared__ float win[kLWin][4 * kLMom];
    __shared__ float scale[4];
    const int r = blockIdx.x;
    if (r >= nrows) return;
    const FeatRow fr = rows ? rows[r] : FeatRow{r, (double)step - pairs[r].tau_c};
    const LPair &P = pairs[fr.pair];
    __shared__ float raw[kLWin][4 * kLMom];
    if (threadIdx.x < 4 * kLWin) {
        // thread (k, f): field f of window sample k, linear in time between steps j and j + 1
        const int k = threadIdx.x >> 2, f = threadIdx.x & 3;
        const double s = fr.tc - (double)(k - (kLWin / 2 - 1));
        const long long j = (long long)floor(s);
        const float w = (float)(s - (double)j);
        const float *a = P.mom + (j % P.mdepth) * 4 * kLMom + f * kLMom;
        const float *b = P.mom + ((j + 1) % P.mdepth) * 4 * kLMom + f * kLMom;
        for (int i = 0; i < kLMom; ++i) raw[k][f * kLMom + i] = w == 0.0f ? a[i] : (1.0f - w) * a[i] + w * b[i];
    }
    __syncthreads();
    if (threadIdx.x < kLWin) rotate_moments(raw[threadIdx.x], P.R, win[threadIdx.x]);
    __syncthreads();
    if (threadIdx.x < 4 * 32) {
        // warp f: the RMS of field f's window
        const int f = threadIdx.x >> 5, lane = threadIdx.x & 31;
        float ss = 0.0f;
        for (int i = lane; i < kLWin * kLMom; i += 32) {
            const float x = win[i / kLMom][f * kLMom + i % kLMom];
            ss = fmaf(x, x, ss);
        }
        for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
        if (lane == 0) {
            const float v = sqrtf(ss / (kLWin * kLMom));
            scale[f] = v;
            nu[4 * r + f] = v;
        }
    }
    __syncthreads();
    const float lr = (float)(kLL0 / P.Rc);
    for (int i = threadIdx.x; i < 4 * kLIn; i += blockDim.x) {
        const int f = i / kLIn, c = i % kLIn;
        const int cc = c % (kLWin * kLMom), k = cc / kLMom, m = cc % kLMom;
        const float inv = scale[f] > 0.0f ? 1.0f / scale[f] : 0.0f;
        float x = win[k][f * kLMom + m] * inv;
        if (c >= kLWin * kLMom) x *= lr;
        X16[(size_t)(4 * r + f) * kLIn + c] = __float2half_rn(x);
        if (Xf) Xf[(size_t)(4 * r + f) * kLIn + c] = x;
    }
}

// ---------------------------------------------------------------- training sources

// Basis fields of one history's Gaussians on the source grid:
//   B[g][0] = unit Gaussian g_g(r),  B[g][1..3] = grad Phi_g(r),
//   Phi_g = erf(|r - c_g| / (sqrt2 sigma_g)) / |r - c_g| (the potential of g_g).
__global__ void k_train_basis(const TrainHist *__restrict__ hist, int nx, int ny, int nz, float h, float *__restrict__ B)
{
    const TrainHist &H = hist[blockIdx.y];
    const long long N = (long long)nx * ny * nz;
    float *out = B + (long long)blockIdx.y * kLGauss * 4 * N;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < N; q += (long long)gridDim.x * blockDim.x) {
        const float x = h * (q % nx), y = h * ((q / nx) % ny), z = h * (q / ((long long)nx * ny));
        for (int g = 0; g < kLGauss; ++g) {
            const float dx = x - H.cx[g], dy = y - H.cy[g], dz = z - H.cz[g];
            const float s = H.sigma[g];
            const float r2 = dx * dx + dy * dy + dz * dz, r = sqrtf(r2);
            const float norm = 1.0f / (powf(2.0f * 3.14159265358979f * s * s, 1.5f));
            const float gg = norm * expf(-r2 / (2.0f * s * s));
            float over_r;
            if (r < 1e-4f * s) {
                over_r = -0.797884560802865f / (3.0f * s * s * s);   // -sqrt(2/pi) / (3 sigma^3)
            } else {
                const float dphidr = (0.797884560802865f / s * expf(-r2 / (2.0f * s * s)) * r -
                                      erff(r / (1.41421356237310f * s))) / r2;
                over_r = dphidr / r;
            }
            out[((long long)g * 4 + 0) * N + q] = gg;
            out[((long long)g * 4 + 1) * N + q] = dx * over_r;
            out[((long long)g * 4 + 2) * N + q] = dy * over_r;
            out[((long long)g * 4 + 3) * N + q] = dz * over_r;
        }
    }
}

// Moments of every slice of every history from the basis moments:
// rho's are sum_g A_g(j) Mb[g][0], J_k's sum_g dA_g(j)/(4 pi) Mb[g][1+k].
__global__ void k_train_moments(const TrainHist *__restrict__ hist, const float *__restrict__ Mb, int T,
                                float *__restrict__ mom)
{
    const int hh = blockIdx.x;
    const TrainHist &H = hist[hh];
    for (int i = threadIdx.x; i < T * 4 * kLMom; i += blockDim.x) {
        const int j = i / (4 * kLMom), t = i % (4 * kLMom), f = t / kLMom;
        float s = 0.0f;
        for (int g = 0; g < kLGauss; ++g) {
            const float a = f == 0 ? H.amp[g][j] : H.damp[g][j];
            s = fmaf(a, Mb[((long long)hh * kLGauss + g) * 4 * kLMom + t], s);
        }
        mom[(long long)hh * T * 4 * kLMom + i] = s;
    }
}

// Labels: the direct retarded sum (Eqs. 2, 7, 8) at the 64 canonical nodes of
// a history's geometry, for kLSampGroup consecutive samples per block:
//   value(x_a, t) = sum_{r'} h^3 / R  S(r', t - R / (c dt))   (times in steps),
// S between samples by linear interpolation.  R = |D_a - rho|, D_a = x_a - c_s
// (FP64 on the host), rho = r' - c_s; R - |D_a| is formed from
// (|rho|^2 - 2 D_a.rho) / |D_a|^2 without cancellation.  Output: raw sums
// (phi, and J without 1/c) [hist][sample][64][4].
__global__ void __launch_bounds__(256) k_train_labels(const TrainHist *__restrict__ hist, const float *__restrict__ B,
                                                      int nx, int ny, int nz, float h, int samples,
                                                      float inv_cdt, float *__restrict__ out)
{
    __shared__ float amp[kLGauss][kLHistT], damp[kLGauss][kLHistT];
    __shared__ double red[256];
    const int hh = blockIdx.z, a = blockIdx.y, k0 = blockIdx.x * kLSampGroup;
    const TrainHist &H = hist[hh];
    for (int i = threadIdx.x; i < kLGauss * kLHistT; i += blockDim.x) {
        amp[i / kLHistT][i % kLHistT] = H.amp[i / kLHistT][i % kLHistT];
        damp[i / kLHistT][i % kLHistT] = H.damp[i / kLHistT][i % kLHistT];
    }
    __syncthreads();
    const long long N = (long long)nx * ny * nz;
    const float *Bh = B + (long long)hh * kLGauss * 4 * N;
    const float Dx = H.D[a][0], Dy = H.D[a][1], Dz = H.D[a][2];
    const float D = H.Dn[a], invD2 = 1.0f / (D * D);
    const float base = H.base[a];   // t_0 - |D_a| / (c dt): sample k's time index is base + k
    float acc[kLSampGroup][4];
    for (int k = 0; k < kLSampGroup; ++k)
        for (int f = 0; f < 4; ++f) acc[k][f] = 0.0f;
    const float vol = h * h * h;
    for (long long q = threadIdx.x; q < N; q += blockDim.x) {
        const float rx = h * (q % nx) - H.csx, ry = h * ((q / nx) % ny) - H.csy, rz = h * (q / ((long long)nx * ny)) - H.csz;
        const float num = rx * rx + ry * ry + rz * rz - 2.0f * (Dx * rx + Dy * ry + Dz * rz);
        const float u = num * invD2;
        const float dR = num / (D * (sqrtf(1.0f + u) + 1.0f));   // R - |D_a|
        const float w = vol / (D + dR);
        const float s = base - dR * inv_cdt;                     // retarded time index of sample 0
        const int j = (int)floorf(s);
        const float fr = s - (float)j;
        float b[kLGauss][4];
        for (int g = 0; g < kLGauss; ++g)
            for (int f = 0; f < 4; ++f) b[g][f] = w * Bh[((long long)g * 4 + f) * N + q];
        for (int k = 0; k < kLSampGroup; ++k) {
            const int jj = j + k0 + k;
            for (int g = 0; g < kLGauss; ++g) {
                const float A = (1.0f - fr) * amp[g][jj] + fr * amp[g][jj + 1];
                const float dA = (1.0f - fr) * damp[g][jj] + fr * damp[g][jj + 1];
                acc[k][0] = fmaf(A, b[g][0], acc[k][0]);
                acc[k][1] = fmaf(dA, b[g][1], acc[k][1]);
                acc[k][2] = fmaf(dA, b[g][2], acc[k][2]);
                acc[k][3] = fmaf(dA, b[g][3], acc[k][3]);
            }
        }
    }
    for (int k = 0; k < kLSampGroup; ++k)
        for (int f = 0; f < 4; ++f) {
            red[threadIdx.x] = acc[k][f];
            __syncthreads();
            for (int wdt = 128; wdt > 0; wdt >>= 1) {
                if ((int)threadIdx.x < wdt) red[threadIdx.x] += red[threadIdx.x + wdt];
                __syncthreads();
            }
            if (threadIdx.x == 0 && k0 + k < samples)
                out[(((long long)hh * samples + k0 + k) * kLOut + a) * 4 + f] = (float)red[0];
            __syncthreads();
        }
}

// Network targets from labels: y[4 row + f][a] = R_a value'_f(a) / nu (the
// current's sums rotated into the canonical frame).
__global__ void k_label_rows(const TrainHist *__restrict__ hist, const float *__restrict__ labels,
                             const float *__restrict__ nu, int samples, float *__restrict__ Y)
{
    const int row = blockIdx.x;   // hist * samples + sample
    const int hh = row / samples;
    const TrainHist &H = hist[hh];
    const int a = threadIdx.x;
    if (a >= kLOut) return;
    const float *v = labels + ((long long)row * kLOut + a) * 4;
    float vc[4];
    vc[0] = v[0];
    for (int k = 0; k < 3; ++k) vc[1 + k] = H.R[3 * k] * v[1] + H.R[3 * k + 1] * v[2] + H.R[3 * k + 2] * v[3];
    for (int f = 0; f < 4; ++f) {
        const float s = nu[4 * row + f];
        Y[(long long)(4 * row + f) * kLOut + a] = s > 0.0f ? H.Dn[a] * vc[f] / s : 0.0f;
    }
}

// ---------------------------------------------------------------- output stage

// Output stage, part 1: one block per learned pair.  Thread (f, b) forms the
// pair's value of canonical field f at target node b by re-interpolation,
// then, after the block has all four fields of b, writes the rotated-back
// field f of node b to the pair's contribution contrib[pair][b][f].
__global__ void __launch_bounds__(4 * kLOut) k_learned_pair(const LPair *__restrict__ pairs, int npairs,
                                                            const int *__restrict__ pair_r,
                                                            const float *__restrict__ Y,
                                                            const float *__restrict__ Ylin,
                                                            const float *__restrict__ nu, float *__restrict__ contrib)
{
    __shared__ float v[4][kLOut];
    __shared__ float u[4][kLOut];
    const int pi = blockIdx.x;
    if (pi >= npairs) return;
    const LPair &P = pairs[pi];
    const int r = pair_r[pi];
    const int f = threadIdx.x / kLOut, b = threadIdx.x % kLOut;
    {
        const long long o = (long long)(4 * pi + f) * kLOut + b;   // canonical node a = b here
        float y = Ylin[o];
        if (P.yscale != 0.0f) y = fmaf(P.yscale, Y[o], y);
        v[f][b] = nu[4 * pi + f] * y / P.Ra[b];
    }
    __syncthreads();
    if (b < r) {
        float s0 = 0.0f, s1 = 0.0f;
#pragma unroll 8
        for (int a = 0; a < kLOut; a += 2) {
            s0 = fmaf(__ldg(P.P + (long long)a * r + b), v[f][a], s0);
            s1 = fmaf(__ldg(P.P + (long long)(a + 1) * r + b), v[f][a + 1], s1);
        }
        u[f][b] = s0 + s1;
    }
    __syncthreads();
    if (b < r) {
        const float x = f == 0 ? u[0][b]
                               : P.R[f - 1] * u[1][b] + P.R[3 + f - 1] * u[2][b] + P.R[6 + f - 1] * u[3][b];
        contrib[((long long)pi * kLOut + b) * 4 + f] = x;
    }
}

// Output stage, part 2: one block per target; thread (b, f) sums its pairs'
// contributions in pair order and sets (no low-rank pairs) or adds to the
// coefficient slot of this step.
__global__ void __launch_bounds__(4 * kLOut) k_learned_out(const LTarget *__restrict__ tgts,
                                                           const float *__restrict__ contrib, long long step)
{
    const LTarget T = tgts[blockIdx.x];
    const int b = threadIdx.x / 4, f = threadIdx.x % 4;
    if (b >= T.r) return;
    float acc = 0.0f;
    for (int pi = T.p0; pi < T.p1; ++pi) acc += contrib[((long long)pi * kLOut + b) * 4 + f];
    float *c = T.cring + (step % T.depth) * (T.r * 4) + b * 4 + f;
    *c = T.overwrite ? acc : *c + acc;
}

}  // namespace

cudaError_t launch_moments(const MomentJob *d_jobs, int njobs, int max_nz, long long slot, const IoPtrs *in,
                           cudaStream_t s)
{
    if (njobs <= 0) return cudaSuccess;
    IoPtrs none{};
    k_moment_part<<<dim3(max_nz, 4, njobs), kMomThreads, 0, s>>>(d_jobs, in ? *in : none);
    k_moment_final<<<njobs, 64, 0, s>>>(d_jobs, slot);
    return cudaGetLastError();
}

cudaError_t launch_features(const LPair *d_pairs, const FeatRow *d_rows, int nrows, long long step, __half *X16,
                            float *Xf, float *nu, cudaStream_t s)
{
    if (nrows <= 0) return cudaSuccess;
    k_features<<<nrows, 128, 0, s>>>(d_pairs, d_rows, nrows, step, X16, Xf, nu);
    return cudaGetLastError();
}

cudaError_t launch_train_basis(const TrainHist *d_hist, int nhist, const int n[3], float h, float *B, cudaStream_t s)
{
    const long long N = (long long)n[0] * n[1] * n[2];
    k_train_basis<<<dim3((unsigned)std::min<long long>((N + 255) / 256, 1024), nhist), 256, 0, s>>>(d_hist, n[0], n[1],
                                                                                                 n[2], h, B);
    return cudaGetLastError();
}

cudaError_t launch_train_moments(const TrainHist *d_hist, int nhist, const float *Mb, int T, float *mom, cudaStream_t s)
{
    k_train_moments<<<nhist, 256, 0, s>>>(d_hist, Mb, T, mom);
    return cudaGetLastError();
}

cudaError_t launch_train_labels(const TrainHist *d_hist, int nhist, const float *B, const int n[3], float h,
                                int samples, double cdt, float *labels, cudaStream_t s)
{
    const dim3 grid((samples + kLSampGroup - 1) / kLSampGroup, kLOut, nhist);
    k_train_labels<<<grid, 256, 0, s>>>(d_hist, B, n[0], n[1], n[2], h, samples, (float)(1.0 / cdt), labels);
    return cudaGetLastError();
}

cudaError_t launch_label_rows(const TrainHist *d_hist, int nhist, const float *labels, const float *nu, int samples,
                              float *Y, cudaStream_t s)
{
    k_label_rows<<<nhist * samples, kLOut, 0, s>>>(d_hist, labels, nu, samples, Y);
    return cudaGetLastError();
}

cudaError_t launch_learned_out(const LTarget *d_tgts, int ntgt, const LPair *d_pairs, int npairs, const int *d_pair_r,
                               const float *Y, const float *Ylin, const float *nu, float *contrib, long long step,
                               cudaStream_t s)
{
    if (ntgt <= 0 || npairs <= 0) return cudaSuccess;
    k_learned_pair<<<npairs, 4 * kLOut, 0, s>>>(d_pairs, npairs, d_pair_r, Y, Ylin, nu, contrib);
    k_learned_out<<<ntgt, 4 * kLOut, 0, s>>>(d_tgts, contrib, step);
    return cudaGetLastError();
}

}  // namespace rp
