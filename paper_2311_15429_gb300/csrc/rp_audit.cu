// FP64 error audit on the GPU (RP_FLAG_AUDIT, rp_audit, rp_audit_values).
//
// The plain definition of the result -- the direct retarded sum of Eq. 8
// with the hat interpolation of Eq. 7 (Eqs. 11-12 give the same number),
// every source node of every domain, the cell-averaged weight C h^2 at
// R = 0 of a node with itself, at lag 0 -- evaluated in FP64 at sampled
// target nodes from the context's own history: under RP_FLAG_AUDIT every
// source keeps a raw (rho, J) ring as deep as its deepest pair reads.  One
// block per target node; its threads stride over the source nodes, each
// summing its share in FP64, and the block adds the partial sums in a fixed
// tree order.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "rp_ctx.h"

namespace rp {

namespace {

constexpr int kAuditThreads = 256;

struct AuditSrc {
    const float *raw;   // [depth][4][N]
    long long N;
    int nx, ny, depth, dom;
    double ox, oy, oz, h;
};

struct AuditTgt {
    double ox, oy, oz, h;
    int nx, ny, pad_[2];
    long long N;
    const float *phi, *A;   // outputs to gather at the sampled nodes, or null
};

struct AuditPt {
    int dom, pad_;
    long long node;
};

__global__ void __launch_bounds__(kAuditThreads) k_audit(const AuditSrc *__restrict__ srcs, int nsrc,
                                                           const AuditTgt *__restrict__ tgts,
                                                           const AuditPt *__restrict__ pts, int npts, long long step,
                                                           int clamp, double inv_cdt, double inv_c, double self_c,
                                                           double *__restrict__ vals, float *__restrict__ got)
{
    __shared__ double red[kAuditThreads / 32][4];
    for (int p = blockIdx.x; p < npts; p += gridDim.x) {
        const AuditPt P = pts[p];
        const AuditTgt T = tgts[P.dom];
        const long long k = P.node;
        const double rx = T.ox + T.h * (double)(k % T.nx);
        const double ry = T.oy + T.h * (double)((k / T.nx) % T.ny);
        const double rz = T.oz + T.h * (double)(k / ((long long)T.nx * T.ny));
        double acc[4] = {0.0, 0.0, 0.0, 0.0};
        for (int s = 0; s < nsrc; ++s) {
            const AuditSrc S = srcs[s];
            const double vol = S.h * S.h * S.h;
            const long long N = S.N;
            for (long long q = threadIdx.x; q < N; q += blockDim.x) {
                if (S.dom == P.dom && q == k) {   // the node itself: cell average, lag 0
                    const double w0 = self_c * S.h * S.h;
                    const float *x = S.raw + (step % S.depth) * 4 * N + q;
#pragma unroll
                    for (int f = 0; f < 4; ++f) acc[f] += w0 * (double)x[f * N];
                    continue;
                }
                const double dx = rx - (S.ox + S.h * (double)(q % S.nx));
                const double dy = ry - (S.oy + S.h * (double)((q / S.nx) % S.ny));
                const double dz = rz - (S.oz + S.h * (double)(q / ((long long)S.nx * S.ny)));
                const double R = sqrt(dx * dx + dy * dy + dz * dz);
                const double tau = R * inv_cdt;
                const double m = floor(tau);
                const double w = tau - m;
                long long j0 = step - (long long)m, j1 = j0 - 1;
                if (clamp && j0 < 0) j0 = 0;
                if (clamp && j1 < 0) j1 = 0;
                const float *x0 = S.raw + (j0 % S.depth) * 4 * N + q;
                const float *x1 = S.raw + (j1 % S.depth) * 4 * N + q;
                const double a = vol / R;
#pragma unroll
                for (int f = 0; f < 4; ++f) {
                    double v = (1.0 - w) * (double)x0[f * N];
                    if (w > 0.0) v += w * (double)x1[f * N];   // at an integer delay the older sample is not read
                    acc[f] += a * v;
                }
            }
        }
#pragma unroll
        for (int f = 0; f < 4; ++f)
            for (int o = 16; o > 0; o >>= 1) acc[f] += __shfl_down_sync(0xffffffffu, acc[f], o);
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        if (lane == 0)
            for (int f = 0; f < 4; ++f) red[warp][f] = acc[f];
        __syncthreads();
        if (threadIdx.x < 4) {
            const int f = threadIdx.x;
            double v = 0.0;
            for (int i = 0; i < kAuditThreads / 32; ++i) v += red[i][f];
            vals[(long long)p * 4 + f] = f == 0 ? v : v * inv_c;
            if (got) got[(long long)p * 4 + f] = f == 0 ? T.phi[k] : T.A[(long long)(f - 1) * T.N + k];
        }
        __syncthreads();
    }
}

unsigned long long splitmix64(unsigned long long x)
{
    x += 0x9E3779B97F4A7C15ULL;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ULL;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBULL;
    return x ^ (x >> 31);
}

// Device scratch of the audit for npts points (grown on demand; released at rp_destroy).
rp_status audit_scratch(rp_ctx *ctx, int npts)
{
    const int nd = (int)ctx->doms.size();
    if (npts <= ctx->audit_cap) return RP_OK;
    const size_t bytes = (size_t)nd * (sizeof(AuditSrc) + sizeof(AuditTgt)) + (size_t)npts * (sizeof(AuditPt) + 32 + 16);
    char *p = nullptr;
    rp_status st = dev_alloc(ctx, &p, bytes);
    if (st) return st;
    ctx->audit_buf = p;
    ctx->audit_cap = npts;
    return RP_OK;
}

// FP64 values at the points (and the outputs gathered there when `tgt_out`),
// on the context stream, waited for.
rp_status audit_run(rp_ctx *ctx, const std::vector<AuditPt> &pts, const float *const *d_phi, const float *const *d_A,
                    std::vector<double> &vals, std::vector<float> *got)
{
    const int nd = (int)ctx->doms.size();
    for (int d = 0; d < nd; ++d)
        if (ctx->owned[d] && !ctx->raw[d].ring)
            return fail(ctx, RP_ERR_STATE, "the FP64 audit needs RP_FLAG_AUDIT (every source's raw history)");
    if (ctx->step < 0 || ctx->npushed != nd) return fail(ctx, RP_ERR_STATE, "audit before every domain pushed the step");
    if (!ctx->clamp && ctx->step - ctx->max_lag < 0)
        return fail(ctx, RP_ERR_HISTORY, "audit of step " + std::to_string(ctx->step) + " needs samples " +
                                             std::to_string(ctx->max_lag) + " steps back");
    const int npts = (int)pts.size();
    rp_status st = audit_scratch(ctx, npts);
    if (st) return st;
    if (ctx->overlap) RP_CUDA(ctx, cudaStreamWaitEvent(ctx->stream, ctx->ev_pushed, 0));   // the rings' last push
    // the sources this context owns (all of them but under a source partition)
    std::vector<AuditSrc> hs;
    std::vector<AuditTgt> ht(nd);
    for (int d = 0; d < nd; ++d) {
        const DomainDesc &D = ctx->doms[d];
        if (ctx->owned[d])
            hs.push_back(AuditSrc{ctx->raw[d].ring, D.N, D.n[0], D.n[1], ctx->raw[d].depth, d, D.o[0], D.o[1], D.o[2],
                                  D.h});
        ht[d] = AuditTgt{D.o[0], D.o[1], D.o[2], D.h, D.n[0], D.n[1], {0, 0}, D.N, got ? d_phi[d] : nullptr,
                         got ? d_A[d] : nullptr};
    }
    char *b = ctx->audit_buf;
    AuditSrc *d_src = reinterpret_cast<AuditSrc *>(b);
    AuditTgt *d_tgt = reinterpret_cast<AuditTgt *>(d_src + nd);
    AuditPt *d_pts = reinterpret_cast<AuditPt *>(d_tgt + nd);
    double *d_vals = reinterpret_cast<double *>(d_pts + npts);
    float *d_got = reinterpret_cast<float *>(d_vals + 4 * (size_t)npts);
    RP_CUDA(ctx, cudaMemcpyAsync(d_src, hs.data(), hs.size() * sizeof(AuditSrc), cudaMemcpyHostToDevice, ctx->stream));
    RP_CUDA(ctx, cudaMemcpyAsync(d_tgt, ht.data(), nd * sizeof(AuditTgt), cudaMemcpyHostToDevice, ctx->stream));
    RP_CUDA(ctx, cudaMemcpyAsync(d_pts, pts.data(), npts * sizeof(AuditPt), cudaMemcpyHostToDevice, ctx->stream));
    const int grid = std::max(1, std::min(npts, 16 * std::max(1, ctx->sm_count)));
    k_audit<<<grid, kAuditThreads, 0, ctx->stream>>>(d_src, (int)hs.size(), d_tgt, d_pts, npts, ctx->step, ctx->clamp ? 1 : 0,
                                                     1.0 / (ctx->cfg.c * ctx->cfg.dt), 1.0 / ctx->cfg.c,
                                                     cube_average_constant(), d_vals, got ? d_got : nullptr);
    RP_CUDA(ctx, cudaGetLastError());
    vals.resize(4 * (size_t)npts);
    RP_CUDA(ctx, cudaMemcpyAsync(vals.data(), d_vals, vals.size() * sizeof(double), cudaMemcpyDeviceToHost,
                                 ctx->stream));
    if (got) {
        got->resize(4 * (size_t)npts);
        RP_CUDA(ctx, cudaMemcpyAsync(got->data(), d_got, got->size() * sizeof(float), cudaMemcpyDeviceToHost,
                                     ctx->stream));
    }
    RP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return RP_OK;
}

}  // namespace

}  // namespace rp

extern "C" {

rp_status rp_audit_values(rp_ctx *ctx, int target, const long long *h_nodes, int count, double *h_out)
{
    if (!ctx) return RP_ERR_ARG;
    if (!ctx->finalized || ctx->plan_only) return fail(ctx, RP_ERR_STATE, "context not finalized for execution");
    rp_status st = use_device(ctx);
    if (st) return st;
    const int nd = (int)ctx->doms.size();
    if (target < 0 || target >= nd || count < 0 || (count > 0 && (!h_nodes || !h_out)))
        return fail(ctx, RP_ERR_ARG, "rp_audit_values: bad target, count or pointer");
    std::vector<AuditPt> pts(count);
    for (int i = 0; i < count; ++i) {
        if (h_nodes[i] < 0 || h_nodes[i] >= ctx->doms[target].N)
            return fail(ctx, RP_ERR_ARG, "rp_audit_values: node out of range");
        pts[i] = AuditPt{target, 0, h_nodes[i]};
    }
    if (count == 0) return RP_OK;
    std::vector<double> vals;
    if ((st = audit_run(ctx, pts, nullptr, nullptr, vals, nullptr))) return st;
    std::memcpy(h_out, vals.data(), vals.size() * sizeof(double));
    return RP_OK;
}

rp_status rp_audit(rp_ctx *ctx, const float *const *d_phi, const float *const *d_A, int nodes_per_domain,
                   unsigned long long seed, double *h_rel_l2)
{
    if (!ctx) return RP_ERR_ARG;
    if (!ctx->finalized || ctx->plan_only) return fail(ctx, RP_ERR_STATE, "context not finalized for execution");
    rp_status st = use_device(ctx);
    if (st) return st;
    const int nd = (int)ctx->doms.size();
    if (!d_phi || !d_A || nodes_per_domain < 1) return fail(ctx, RP_ERR_ARG, "rp_audit: bad pointer or count");
    for (int d = 0; d < nd; ++d)
        if (!d_phi[d] || !d_A[d]) return fail(ctx, RP_ERR_ARG, "rp_audit: NULL output buffer");
    // stratified seeded sample: node i of domain d from the i-th of c equal strata
    std::vector<AuditPt> pts;
    std::vector<int> first(nd + 1, 0);
    for (int d = 0; d < nd; ++d) {
        const long long N = ctx->doms[d].N;
        const long long c = std::min<long long>(nodes_per_domain, N);
        for (long long i = 0; i < c; ++i) {
            const long long a = i * N / c, b = (i + 1) * N / c;
            const unsigned long long r = splitmix64(seed ^ ((unsigned long long)d << 40) ^ (unsigned long long)i);
            pts.push_back(AuditPt{d, 0, a + (long long)(r % (unsigned long long)(b - a))});
        }
        first[d + 1] = (int)pts.size();
    }
    std::vector<double> vals;
    std::vector<float> got;
    if ((st = audit_run(ctx, pts, d_phi, d_A, vals, &got))) return st;
    double worst = 0.0;
    for (int d = 0; d < nd; ++d)
        for (int f = 0; f < 4; ++f) {
            double num = 0.0, den = 0.0;
            for (int p = first[d]; p < first[d + 1]; ++p) {
                const double e = (double)got[4 * (size_t)p + f] - vals[4 * (size_t)p + f];
                num += e * e;
                den += vals[4 * (size_t)p + f] * vals[4 * (size_t)p + f];
            }
            const double rel = den > 0.0 ? std::sqrt(num / den) : (num > 0.0 ? INFINITY : 0.0);
            if (h_rel_l2) h_rel_l2[4 * d + f] = rel;
            worst = std::max(worst, rel);
        }
    ctx->audit_rel_l2 = worst;
    ctx->audit_step = ctx->step;
    return RP_OK;
}

}  // extern "C"
