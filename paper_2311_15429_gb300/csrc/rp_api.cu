// C-ABI of the retarded-potential library: pair planning, memory, kernel
// spectra and the push / evaluate launch sequence.  See include/rp.h; the
// context and its helpers are in rp_ctx.h, the history spill in rp_spill.cu.
#include <algorithm>
#include <array>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include <cuda.h>
#include <cudaTypedefs.h>

#include "rp_ctx.h"

namespace rp {
size_t smem_direct(int max_nlag);
int direct_blocks(long long n);
cudaError_t open_direct_smem_limit(int max_optin);
}  // namespace rp

using namespace rp;

namespace {

// Supported padded lengths: R * L with R in {1,2,3,4,6}, L a power of two <= 32.
const int kSizes[] = {1, 2, 3, 4, 6, 8, 12, 16, 24, 32, 48, 64, 96, 128, 192};

int good_size(int n, bool even)
{
    for (int m : kSizes)
        if (m >= n && (!even || m % 2 == 0)) return m;
    return -1;
}

Axis make_axis(int M)
{
    Axis a{};
    a.M = M;
    if (M % 3 == 0) {
        const int rest = M / 3;
        if (rest <= 32) { a.R = 3; a.L = rest; }
        else { a.R = 6; a.L = rest / 2; }
    } else if (M <= 32) {
        a.R = 1; a.L = M;
    } else {
        a.R = M / 32; a.L = 32;
    }
    a.logL = 0;
    while ((1 << a.logL) < a.L) ++a.logL;
    return a;
}

}  // namespace


namespace {

// Device address of rp_evaluate_host_noalloc's fixed staging array on
// ctx->device (defined with the array, below).
rp_status noalloc_stage_address(rp_ctx *ctx, float **out);

rp_status drain_profile(rp_ctx *ctx)
{
    for (const ProfRec &r : ctx->pending) {
        RP_CUDA(ctx, cudaEventSynchronize(r.b));
        float t = 0.0f;
        RP_CUDA(ctx, cudaEventElapsedTime(&t, r.a, r.b));
        ctx->ms[r.kind] += t;
        ctx->launches[r.kind] += 1;
        ctx->spare_events.push_back(r.a);
        ctx->spare_events.push_back(r.b);
    }
    ctx->pending.clear();
    return RP_OK;
}

// Smallest and largest distance between the node lattices of two domains:
// the gap between their boxes (a lower bound) and between the farthest
// corners (exact).
void pair_distances(const DomainDesc &t, const DomainDesc &s, bool self, double *rmin, double *rmax)
{
    double g2 = 0.0, f2 = 0.0;
    for (int a = 0; a < 3; ++a) {
        const double a0 = t.o[a], a1 = t.o[a] + t.h * (t.n[a] - 1);
        const double b0 = s.o[a], b1 = s.o[a] + s.h * (s.n[a] - 1);
        const double gap = std::max(0.0, std::max(a0 - b1, b0 - a1));
        const double far = std::max(std::fabs(a1 - b0), std::fabs(b1 - a0));
        g2 += gap * gap;
        f2 += far * far;
    }
    *rmin = self ? 0.0 : std::sqrt(g2);
    *rmax = std::sqrt(f2);
}

// True if some node of t sits on a node of s (only possible when the boxes touch).
bool nodes_coincide(const DomainDesc &t, const DomainDesc &s)
{
    for (int a = 0; a < 3; ++a) {
        const double a0 = t.o[a], a1 = t.o[a] + t.h * (t.n[a] - 1);
        const double b0 = s.o[a], b1 = s.o[a] + s.h * (s.n[a] - 1);
        if (a1 < b0 - 1e-12 || b1 < a0 - 1e-12) return false;
    }
    const double tol = 1e-9;
    for (long long q = 0; q < t.N; ++q) {
        const int i[3] = {(int)(q % t.n[0]), (int)((q / t.n[0]) % t.n[1]), (int)(q / ((long long)t.n[0] * t.n[1]))};
        bool on = true;
        for (int a = 0; a < 3 && on; ++a) {
            const double u = (t.o[a] + t.h * i[a] - s.o[a]) / s.h;
            const double r = std::round(u);
            on = std::fabs(u - r) <= tol * std::max(1.0, std::fabs(u)) && r >= 0 && r <= s.n[a] - 1;
        }
        if (on) return true;
    }
    return false;
}

rp_status build_twiddles(rp_ctx *ctx, std::map<int, const float2 *> &tw)
{
    for (auto &kv : tw) {
        const int M = kv.first;
        std::vector<float2> h(M);
        for (int j = 0; j < M; ++j) {
            const double a = -2.0 * M_PI * (double)j / (double)M;
            h[j] = make_float2((float)std::cos(a), (float)std::sin(a));
        }
        float2 *d = nullptr;
        rp_status st = upload(ctx, &d, h);
        if (st) return st;
        kv.second = d;
    }
    return RP_OK;
}

}  // namespace

namespace {


// Pipeline depth of the bulk-copy-fed MAC for every cubic class of the plan;
// the register-blocked MAC serves the plan if some class cannot hold two
// field stages.
rp_status plan_mac_tma(rp_ctx *ctx, int max_optin)
{
    ctx->tma = false;
    for (int cls : {32, 48, 64, 96, 128, 192}) {
        int n = mac_tma_stages(cls, max_optin, ctx->comp);
        if (ctx->cfg.mac_stages >= 2) n = std::min(n, ctx->cfg.mac_stages);
        ctx->mac_stages[class_slot(cls)] = n;
        if (n < 2) {
            for (const InvTarget &I : ctx->inv)
                if (size_class(I.ax, I.ay, I.az) == cls) {
                    ctx->last_error = "bulk-copy pipeline too shallow: register-blocked MAC in use";
                    return RP_OK;
                }
        }
    }
    ctx->tma = true;
    return RP_OK;
}

}  // namespace

namespace {

// Chebyshev nodes (first kind) of [a, b], or the grid nodes when the axis has
// no more than p of them; and the Lagrange weights of every grid node.
void far_axis(double o, double h, int n, int p, std::vector<double> &nodes, std::vector<float> &L)
{
    const int q = std::min(n, p);
    nodes.resize(q);
    if (n <= p) {
        for (int a = 0; a < q; ++a) nodes[a] = o + h * a;
    } else {
        const double lo = o, hi = o + h * (n - 1);
        for (int a = 0; a < q; ++a)
            nodes[a] = 0.5 * (lo + hi) - 0.5 * (hi - lo) * std::cos((2.0 * a + 1.0) * M_PI / (2.0 * q));
    }
    L.assign((size_t)n * q, 0.0f);
    for (int i = 0; i < n; ++i) {
        const double x = o + h * i;
        for (int a = 0; a < q; ++a) {
            double w = 1.0;
            for (int b = 0; b < q; ++b)
                if (b != a) w *= (x - nodes[b]) / (nodes[a] - nodes[b]);
            L[(size_t)i * q + a] = (float)w;
        }
    }
}

// Factors, batch buffers, coefficient rings and descriptors of the far pairs
// (low-rank pairs get factor rows; targets of low-rank or learned pairs get
// coefficient rings).  Every allocation goes to the far path's own list, so
// that the structures can be rebuilt when pairs move to the learned path.
rp_status build_far_impl(rp_ctx *ctx, int max_optin);
rp_status attach_far_targets(rp_ctx *ctx);
rp_status build_far2(rp_ctx *ctx, void *enc, const std::vector<int> &tidx,
                     const std::vector<std::array<std::vector<double>, 3>> &tnodes);

rp_status build_far(rp_ctx *ctx, int max_optin)
{
    ctx->alloc_sink = &ctx->far_allocs;
    const rp_status st = build_far_impl(ctx, max_optin);
    ctx->alloc_sink = nullptr;
    return st;
}

// Frees the far path's structures (before a rebuild).
void clear_far(rp_ctx *ctx)
{
    for (void *p : ctx->far_allocs) cudaFree(p);
    ctx->far_allocs.clear();
    ctx->device_bytes -= ctx->far_alloc_bytes;
    ctx->far_alloc_bytes = 0;
    ctx->far_src.clear(); ctx->far_tgt.clear(); ctx->far_links.clear();
    ctx->far_link0.clear(); ctx->far_link1.clear(); ctx->far_link_threads.clear();
    ctx->far_Z.clear(); ctx->far_rows.clear(); ctx->far_splits.clear(); ctx->far_work = nullptr;
    ctx->far_mapW.clear(); ctx->far_mapX.clear(); ctx->far_src_of_dom.clear();
    ctx->d_far_src = nullptr; ctx->d_far_tgt = nullptr; ctx->d_far_links = nullptr;
    ctx->far2 = false;
    ctx->far2_srcs.clear(); ctx->far2_of_dom.clear(); ctx->far2_tasks.clear(); ctx->far2_kb.clear();
    ctx->d_far2_srcs = nullptr; ctx->d_far2_tasks = nullptr; ctx->d_far2_kb = nullptr;
    ctx->far2_qall = ctx->far2_fac = nullptr; ctx->far2_work = nullptr;
    ctx->far2_BN = ctx->far2_KS = ctx->far2_D = ctx->far2_max_nz = 0; ctx->far2_fac_rows = 0;
    ctx->far2_max_plane = ctx->far2_max_n = 0;
    ctx->far_src_alone.clear(); ctx->far_src_alone_of_dom.clear();
    ctx->d_far_src_alone = nullptr;
    ctx->far_tgt_alone.clear(); ctx->d_far_tgt_alone = nullptr; ctx->far_alone_planes = 0;
    ctx->far_max_r = ctx->npairs_far = 0;
    ctx->far_bytes = ctx->far_max_n = 0;
    ctx->far_zeroed_step = -1;
    for (FwdRing &R : ctx->fwd) { R.far_x = nullptr; R.far_ks = 0; }
    for (InvTarget &I : ctx->inv) I.far = nullptr;
}

rp_status build_far_impl(rp_ctx *ctx, int max_optin)
{
    const int nd = (int)ctx->doms.size();
    const int batch = ctx->cfg.far_batch, P = ctx->cfg.far_points;
    const double inv_cdt = 1.0 / (ctx->cfg.c * ctx->cfg.dt);
    rp_status st;
    ctx->far_src_of_dom.assign(nd, -1);
    ctx->far_tnodes.assign(nd, {});
    // targets
    std::vector<int> tidx(nd, -1);
    std::vector<std::array<std::vector<double>, 3>> tnodes(nd);
    for (int t = 0; t < nd; ++t) {
        int hi = -1;
        bool learned = false;
        for (int s = 0; s < nd; ++s) {
            const PairPlan &p = ctx->pairs[(size_t)t * nd + s];
            if (p.kind == RP_PAIR_LOWRANK) hi = std::max(hi, p.lag_hi);
            learned = learned || p.kind == RP_PAIR_LEARNED;
        }
        if (hi < 0 && !learned) continue;
        const DomainDesc &T = ctx->doms[t];
        FarTarget F{};
        F.dom = t;
        F.nx = T.n[0]; F.ny = T.n[1]; F.nz = T.n[2];
        std::vector<float> L[3];
        for (int a = 0; a < 3; ++a) far_axis(T.o[a], T.h, T.n[a], P, tnodes[t][a], L[a]);
        ctx->far_tnodes[t] = tnodes[t];
        F.px = (int)tnodes[t][0].size(); F.py = (int)tnodes[t][1].size(); F.pz = (int)tnodes[t][2].size();
        F.r = F.px * F.py * F.pz;
        F.lag_hi_max = hi;
        // one-sided factors scatter into steps up to hi + batch ahead; the
        // two-sided gather writes the next batch of steps at once
        F.depth = ctx->cfg.far_source_points > 0 ? 2 * batch + 2 : hi + batch + 1;
        float *Lx, *Ly, *Lz;
        if ((st = upload(ctx, &Lx, L[0])) || (st = upload(ctx, &Ly, L[1])) || (st = upload(ctx, &Lz, L[2]))) return st;
        F.Lx = Lx; F.Ly = Ly; F.Lz = Lz;
        if ((st = dev_alloc(ctx, &F.cring, (size_t)F.depth * F.r * 4))) return st;
        RP_CUDA(ctx, cudaMemset(F.cring, 0, (size_t)F.depth * F.r * 4 * sizeof(float)));
        ctx->far_bytes += (long long)F.depth * F.r * 16 + 4LL * (T.n[0] * F.px + T.n[1] * F.py + T.n[2] * F.pz);
        ctx->far_max_r = std::max(ctx->far_max_r, F.r);
        tidx[t] = (int)ctx->far_tgt.size();
        ctx->far_tgt.push_back(F);
    }
    if (ctx->far_tgt.empty()) return RP_OK;
    void *enc = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &enc, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !enc) {
        cudaGetLastError();
        return fail(ctx, RP_ERR_UNSUPPORTED, "far path needs cuTensorMapEncodeTiled");
    }
    if (ctx->cfg.far_source_points > 0) {
        if ((st = build_far2(ctx, enc, tidx, tnodes))) return st;
        if ((st = upload(ctx, &ctx->d_far_tgt, ctx->far_tgt))) return st;
        return attach_far_targets(ctx);
    }
    // sources
    size_t work_floats = 0;
    for (int s = 0; s < nd; ++s) {
        std::vector<FarRow> rows;
        std::vector<FarLink> links;
        for (int t = 0; t < nd; ++t) {
            const PairPlan &p = ctx->pairs[(size_t)t * nd + s];
            if (p.kind != RP_PAIR_LOWRANK) continue;
            const FarTarget &F = ctx->far_tgt[tidx[t]];
            FarLink Lk{};
            Lk.row0 = (int)rows.size();
            Lk.r = F.r;
            Lk.nlag = p.lag_hi - p.lag_lo + 1;
            Lk.lag_lo = p.lag_lo;
            Lk.cring = F.cring;
            Lk.depth = F.depth;
            links.push_back(Lk);
            const auto &nx = tnodes[t];
            const DomainDesc &S = ctx->doms[s];
            for (int m = p.lag_lo; m <= p.lag_hi; ++m)
                for (int c = 0; c < F.pz; ++c)
                    for (int b = 0; b < F.py; ++b)
                        for (int a = 0; a < F.px; ++a)
                            rows.push_back({(float)(nx[0][a] - S.o[0]), (float)(nx[1][b] - S.o[1]),
                                            (float)(nx[2][c] - S.o[2]), m});
        }
        if (links.empty()) continue;
        ctx->npairs_far += (int)links.size();
        const int nrows = (int)((rows.size() + 127) / 128 * 128);
        while ((int)rows.size() < nrows) rows.push_back({0.0f, 0.0f, 0.0f, -1});
        const DomainDesc &S = ctx->doms[s];
        FarSource F{};
        F.dom = s;
        F.n = S.N;
        F.ks = (int)((S.N + 63) / 64 * 64);
        FarRow *d_rows = nullptr;
        __nv_bfloat16 *W = nullptr;
        float *Z = nullptr;
        if ((st = upload(ctx, &d_rows, rows))) return st;
        if ((st = dev_alloc(ctx, &W, (size_t)nrows * 2 * F.ks))) return st;
        if ((st = dev_alloc(ctx, &F.X, (size_t)4 * batch * 2 * F.ks))) return st;
        if ((st = dev_alloc(ctx, &Z, (size_t)nrows * 4 * batch))) return st;
        RP_CUDA(ctx, cudaMemset(F.X, 0, (size_t)4 * batch * 2 * F.ks * sizeof(__nv_bfloat16)));
        RP_CUDA(ctx, launch_far_build_w(d_rows, nrows, S.n, S.h, inv_cdt, F.ks, W, ctx->stream));
        const int splits = gemm_splits(nrows, F.ks, 1, ctx->sm_count, 16);
        work_floats = std::max(work_floats, splits > 1 ? (size_t)splits * nrows * 4 * batch : 0);
        ctx->far_splits.push_back(splits);
        ctx->far_bytes += (long long)nrows * F.ks * 4 + 16LL * batch * F.ks + 16LL * nrows * batch;
        CUtensorMap mw, mx;
        if (!encode_bf16_rows(enc, &mw, W, (uint64_t)nrows, (uint64_t)2 * F.ks, 128) ||
            !encode_bf16_rows(enc, &mx, F.X, (uint64_t)4 * batch, (uint64_t)2 * F.ks, (uint32_t)(4 * batch)))
            return fail(ctx, RP_ERR_UNSUPPORTED, "far path: a tensor map did not encode");
        ctx->far_mapW.push_back(mw);
        ctx->far_mapX.push_back(mx);
        ctx->far_Z.push_back(Z);
        ctx->far_rows.push_back(nrows);
        ctx->far_link0.push_back((int)ctx->far_links.size());
        int thr = 0;
        for (const FarLink &Lk : links) {
            thr += Lk.r * 4 * (Lk.nlag + batch - 1);
            ctx->far_links.push_back(Lk);
        }
        ctx->far_link1.push_back((int)ctx->far_links.size());
        ctx->far_link_threads.push_back(thr);
        ctx->far_max_n = std::max(ctx->far_max_n, S.N);
        ctx->far_src_of_dom[s] = (int)ctx->far_src.size();
        ctx->far_src.push_back(F);
    }
    (void)max_optin;
    if (work_floats) {
        if ((st = dev_alloc(ctx, &ctx->far_work, work_floats))) return st;
        ctx->far_bytes += (long long)work_floats * 4;
    }
    if ((st = upload(ctx, &ctx->d_far_src, ctx->far_src))) return st;
    if ((st = upload(ctx, &ctx->d_far_tgt, ctx->far_tgt))) return st;
    if ((st = upload(ctx, &ctx->d_far_links, ctx->far_links))) return st;
    if ((st = attach_far_targets(ctx))) return st;
    // staging rides on the source's first forward ring, interpolation on the
    // target's inverse plane pass
    ctx->far_src_alone_of_dom.assign(nd, -1);
    for (const FarSource &F : ctx->far_src) {
        bool done = false;
        for (FwdRing &R : ctx->fwd)
            if (R.src == F.dom && !done) {
                R.far_x = F.X;
                R.far_ks = F.ks;
                done = true;
            }
        if (!done) {
            ctx->far_src_alone_of_dom[F.dom] = (int)ctx->far_src_alone.size();
            ctx->far_src_alone.push_back(F);
        }
    }
    if (!ctx->far_src_alone.empty() && (st = upload(ctx, &ctx->d_far_src_alone, ctx->far_src_alone))) return st;
    return RP_OK;
}

// Every far target is also an FFT target (its self term), and its inverse
// plane pass, which writes the output, adds the far coefficients: a far
// target without one would have no pass that writes its output first.
rp_status attach_far_targets(rp_ctx *ctx)
{
    rp_status st;
    ctx->far_tgt_alone.clear();
    ctx->far_alone_planes = 0;
    for (size_t k = 0; k < ctx->far_tgt.size(); ++k) {
        const FarTarget &F = ctx->far_tgt[k];
        bool done = false;
        for (InvTarget &I : ctx->inv)
            if (I.dom == F.dom && !done) {
                I.far = ctx->d_far_tgt + k;
                done = true;
            }
        if (done) continue;
        // no FFT pass (a target whose source another context owns): a separate
        // interpolation after the direct pass, adding onto its direct pairs' output
        FarTarget A = F;
        A.interp_add = 0;
        for (const DirectTarget &D : ctx->dtg)
            if (D.dom == F.dom) A.interp_add = 1;
        ctx->far_tgt_alone.push_back(A);
        ctx->far_alone_planes += F.nz;
    }
    if (!ctx->far_tgt_alone.empty() && (st = upload(ctx, &ctx->d_far_tgt_alone, ctx->far_tgt_alone))) return st;
    return RP_OK;
}

// Two-sided factors (rp_far2.cu): the far sources' anterpolation weights,
// node tables and coefficient rings; every far target's factor blocks, one
// per (far source, lag), built in FP64 on the GPU; the gathered GEMM's CTAs
// (a target's blocks in chunks of at most kFar2Chunk) and its tensor maps.
constexpr int kFar2Chunk = 24;

rp_status build_far2(rp_ctx *ctx, void *enc, const std::vector<int> &tidx,
                     const std::vector<std::array<std::vector<double>, 3>> &tnodes)
{
    const int nd = (int)ctx->doms.size();
    const int batch = ctx->cfg.far_batch, Q = ctx->cfg.far_source_points;
    rp_status st;
    ctx->far2 = true;
    ctx->far2_of_dom.assign(nd, -1);
    // sources and their node tables
    std::vector<double> snodes;
    std::vector<int> snode0;
    int KS = 0, D = std::max(32, batch + 1);
    for (int s = 0; s < nd; ++s) {
        bool far = false;
        for (int t = 0; t < nd; ++t) {
            const PairPlan &p = ctx->pairs[(size_t)t * nd + s];
            if (p.kind != RP_PAIR_LOWRANK) continue;
            far = true;
            D = std::max(D, p.lag_hi + 1);
        }
        if (!far) continue;
        const DomainDesc &S = ctx->doms[s];
        FarSrc2 F{};
        F.dom = s;
        F.nx = S.n[0]; F.ny = S.n[1]; F.nz = S.n[2];
        std::vector<double> nodes[3];
        std::vector<float> L[3];
        for (int a = 0; a < 3; ++a) far_axis(S.o[a], S.h, S.n[a], Q, nodes[a], L[a]);
        F.qx = (int)nodes[0].size(); F.qy = (int)nodes[1].size(); F.qz = (int)nodes[2].size();
        F.r = F.qx * F.qy * F.qz;
        // the weight tables padded to Q columns per axis (zero weights for the
        // nodes a short axis lacks), so the anterpolation's sizes are fixed
        std::vector<float> Lp[3];
        for (int a = 0; a < 3; ++a) {
            const int q = (int)nodes[a].size();
            Lp[a].assign((size_t)S.n[a] * Q, 0.0f);
            for (int i = 0; i < S.n[a]; ++i)
                for (int b = 0; b < q; ++b) Lp[a][(size_t)i * Q + b] = L[a][(size_t)i * q + b];
        }
        float *Lx, *Ly, *Lz;
        if ((st = upload(ctx, &Lx, Lp[0])) || (st = upload(ctx, &Ly, Lp[1])) || (st = upload(ctx, &Lz, Lp[2])))
            return st;
        F.Lx = Lx; F.Ly = Ly; F.Lz = Lz;
        if ((st = dev_alloc(ctx, &F.part, (size_t)S.n[2] * 4 * Q * Q))) return st;
        if ((st = dev_alloc(ctx, &F.count, 1))) return st;
        RP_CUDA(ctx, cudaMemset(F.count, 0, sizeof(unsigned int)));
        snode0.push_back((int)(snodes.size() / 3));
        for (int c = 0; c < F.qz; ++c)
            for (int b = 0; b < F.qy; ++b)
                for (int a = 0; a < F.qx; ++a) {
                    snodes.push_back(nodes[0][a]);
                    snodes.push_back(nodes[1][b]);
                    snodes.push_back(nodes[2][c]);
                }
        KS = std::max(KS, (F.r + 63) / 64 * 64);
        ctx->far2_max_nz = std::max(ctx->far2_max_nz, S.n[2]);
        ctx->far2_max_plane = std::max(ctx->far2_max_plane, S.n[0] * S.n[1]);
        ctx->far2_max_n = std::max({ctx->far2_max_n, S.n[0], S.n[1], S.n[2]});
        ctx->far2_of_dom[s] = (int)ctx->far2_srcs.size();
        ctx->far2_srcs.push_back(F);
    }
    const int nsrc = (int)ctx->far2_srcs.size();
    if (nsrc == 0) {   // every far pair is learned: only the targets' coefficient rings are needed
        ctx->far2 = false;
        return RP_OK;
    }
    if (smem_far_anterp(ctx->far2_max_plane, ctx->far2_max_n) > (size_t)ctx->smem_optin)
        return fail(ctx, RP_ERR_UNSUPPORTED, "far source plane too large for the anterpolation's shared memory");
    ctx->far2_KS = KS;
    ctx->far2_D = D;
    // coefficient rings: [source][2 D][4][2 KS], zero before the first push
    const size_t qrows = (size_t)nsrc * 2 * D * 4;
    if ((st = dev_alloc(ctx, &ctx->far2_qall, qrows * 2 * KS))) return st;
    RP_CUDA(ctx, cudaMemset(ctx->far2_qall, 0, qrows * 2 * KS * sizeof(__nv_bfloat16)));
    for (int i = 0; i < nsrc; ++i) {
        ctx->far2_srcs[i].qrow0 = i * 2 * D * 4;
        ctx->far2_srcs[i].qring = ctx->far2_qall + (size_t)ctx->far2_srcs[i].qrow0 * 2 * KS;
    }
    // targets: node tables, factor blocks, CTAs
    int BN = 0;
    for (const FarTarget &F : ctx->far_tgt) BN = std::max(BN, F.r);
    BN = far_gather_bn(BN);
    if (!BN) return fail(ctx, RP_ERR_UNSUPPORTED, "two-sided far factors take at most 256 target nodes");
    ctx->far2_BN = BN;
    std::vector<double> tn;
    std::vector<FarBuild> builds;
    long long fac_row = 0;
    for (int t = 0; t < nd; ++t) {
        if (tidx[t] < 0) continue;
        FarTarget &F = ctx->far_tgt[tidx[t]];
        const int t0 = (int)(tn.size() / 3);
        for (int c = 0; c < F.pz; ++c)
            for (int b = 0; b < F.py; ++b)
                for (int a = 0; a < F.px; ++a) {
                    tn.push_back(tnodes[t][0][a]);
                    tn.push_back(tnodes[t][1][b]);
                    tn.push_back(tnodes[t][2][c]);
                }
        const int kb0 = (int)ctx->far2_kb.size();
        for (int s = 0; s < nd; ++s) {
            const PairPlan &p = ctx->pairs[(size_t)t * nd + s];
            if (p.kind != RP_PAIR_LOWRANK) continue;
            const int si = ctx->far2_of_dom[s];
            const double h = ctx->doms[s].h;
            ctx->npairs_far += 1;
            for (int m = p.lag_lo; m <= p.lag_hi; ++m) {
                if (fac_row > (1LL << 31) - BN) return fail(ctx, RP_ERR_UNSUPPORTED, "far factor rows above 2^31");
                ctx->far2_kb.push_back({si, m, (int)fac_row, 0});
                builds.push_back({t0, F.r, snode0[si], ctx->far2_srcs[si].r, m, (int)fac_row, h * h * h});
                fac_row += BN;
            }
        }
        const int kb1 = (int)ctx->far2_kb.size();
        F.task0 = (int)ctx->far2_tasks.size();
        const int nchunk = (kb1 - kb0 + kFar2Chunk - 1) / kFar2Chunk;
        for (int c = 0; c < nchunk; ++c) {
            // equal shares of the target's blocks
            const int a = kb0 + (int)((long long)(kb1 - kb0) * c / nchunk);
            const int b = kb0 + (int)((long long)(kb1 - kb0) * (c + 1) / nchunk);
            ctx->far2_tasks.push_back({tidx[t], a, b, 0});
        }
        F.task1 = (int)ctx->far2_tasks.size();
        ctx->far_max_r = std::max(ctx->far_max_r, F.r);
    }
    ctx->far2_fac_rows = fac_row;
    if ((st = dev_alloc(ctx, &ctx->far2_fac, (size_t)std::max<long long>(fac_row, BN) * 2 * KS))) return st;
    if ((st = dev_alloc(ctx, &ctx->far2_work, (size_t)std::max<size_t>(ctx->far2_tasks.size(), 1) * 128 * BN)))
        return st;
    {
        FarBuild *d_b = nullptr;
        double *d_tn = nullptr, *d_sn = nullptr;
        if ((st = upload(ctx, &d_b, builds)) || (st = upload(ctx, &d_tn, tn)) || (st = upload(ctx, &d_sn, snodes)))
            return st;
        RP_CUDA(ctx, launch_far_build_fac(d_b, (int)builds.size(), d_tn, d_sn, BN, KS,
                                          1.0 / (ctx->cfg.c * ctx->cfg.dt), ctx->far2_fac, ctx->stream));
    }
    if (!encode_bf16_rows(enc, &ctx->far2_mapQ, ctx->far2_qall, (uint64_t)qrows, (uint64_t)2 * KS, 128) ||
        !encode_bf16_rows(enc, &ctx->far2_mapF, ctx->far2_fac, (uint64_t)std::max<long long>(fac_row, BN),
                          (uint64_t)2 * KS, (uint32_t)BN))
        return fail(ctx, RP_ERR_UNSUPPORTED, "two-sided far factors: a tensor map did not encode");
    if ((st = upload(ctx, &ctx->d_far2_srcs, ctx->far2_srcs)) || (st = upload(ctx, &ctx->d_far2_tasks, ctx->far2_tasks)) ||
        (st = upload(ctx, &ctx->d_far2_kb, ctx->far2_kb)))
        return st;
    ctx->far_bytes += (long long)qrows * 2 * KS * 2 + fac_row * 2 * KS * 2 +
                      (long long)ctx->far2_tasks.size() * 128 * BN * 4;
    return RP_OK;
}

void *tensor_encoder()
{
    void *enc = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &enc, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return enc;
}

void box_centre(const DomainDesc &d, double c[3])
{
    for (int a = 0; a < 3; ++a) c[a] = d.o[a] + 0.5 * d.h * (d.n[a] - 1);
}

void box_extent(const DomainDesc &d, double L[3])
{
    for (int a = 0; a < 3; ++a) L[a] = d.h * (d.n[a] - 1);
}

// Inference structures of the learned pairs (after build_far): moment rings
// and jobs per source, pair records (sorted by target), target records and
// the inference network with the trained weights.
rp_status build_learned(rp_ctx *ctx, const std::vector<float> &weights, const std::vector<float> &wlin,
                        float out_scale)
{
    const int nd = (int)ctx->doms.size();
    const double cdt = ctx->cfg.c * ctx->cfg.dt;
    rp_status st;
    std::vector<int> mdepth(nd, 0);
    for (int t = 0; t < nd; ++t)
        for (int s = 0; s < nd; ++s) {
            if (ctx->pairs[(size_t)t * nd + s].kind != RP_PAIR_LEARNED) continue;
            double ct[3], cs[3];
            box_centre(ctx->doms[t], ct);
            box_centre(ctx->doms[s], cs);
            const double tau = std::sqrt((ct[0] - cs[0]) * (ct[0] - cs[0]) + (ct[1] - cs[1]) * (ct[1] - cs[1]) +
                                         (ct[2] - cs[2]) * (ct[2] - cs[2])) / cdt;
            mdepth[s] = std::max(mdepth[s], (int)std::ceil(tau) + kLWin / 2 + 3);
            ctx->max_lag = std::max(ctx->max_lag, (int)std::ceil(tau) + kLWin / 2 + 1);
        }
    ctx->mjob_of_dom.assign(nd, -1);
    std::vector<float *> ring(nd, nullptr);
    for (int s = 0; s < nd; ++s) {
        if (!mdepth[s]) continue;
        const DomainDesc &D = ctx->doms[s];
        if ((st = dev_alloc(ctx, &ring[s], (size_t)mdepth[s] * 4 * kLMom))) return st;
        RP_CUDA(ctx, cudaMemset(ring[s], 0, (size_t)mdepth[s] * 4 * kLMom * sizeof(float)));
        MomentJob J{};
        J.dom = s;
        J.nx = D.n[0]; J.ny = D.n[1]; J.nz = D.n[2];
        J.h = D.h;
        J.ox = -0.5 * D.h * (D.n[0] - 1); J.oy = -0.5 * D.h * (D.n[1] - 1); J.oz = -0.5 * D.h * (D.n[2] - 1);
        if ((st = dev_alloc(ctx, &J.part, (size_t)4 * D.n[2] * kLMom))) return st;
        J.out = ring[s];
        J.out_depth = mdepth[s];
        ctx->mjob_of_dom[s] = (int)ctx->mjobs.size();
        ctx->mjob_max_nz = std::max(ctx->mjob_max_nz, D.n[2]);
        ctx->mjobs.push_back(J);
    }
    std::map<int, int> ftgt;   // domain -> far target index
    for (size_t k = 0; k < ctx->far_tgt.size(); ++k) ftgt[ctx->far_tgt[k].dom] = (int)k;
    for (int t = 0; t < nd; ++t) {
        const int p0 = (int)ctx->lpairs.size();
        double ct[3], Lt[3];
        box_centre(ctx->doms[t], ct);
        box_extent(ctx->doms[t], Lt);
        double cn[kLOut][3];
        canonical_nodes(Lt, cn);
        for (int s = 0; s < nd; ++s) {
            if (ctx->pairs[(size_t)t * nd + s].kind != RP_PAIR_LEARNED) continue;
            double cs[3], n[3], R[9];
            box_centre(ctx->doms[s], cs);
            for (int a = 0; a < 3; ++a) n[a] = ct[a] - cs[a];
            const double Rc = std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
            canonical_frame(n, R);
            LPair P{};
            for (int k = 0; k < 9; ++k) P.R[k] = (float)R[k];
            P.tau_c = Rc / cdt;
            P.Rc = (float)Rc;
            P.mom = ring[s];
            P.mdepth = mdepth[s];
            for (int a = 0; a < kLOut; ++a) {
                double d2 = 0.0;
                for (int k = 0; k < 3; ++k) {
                    const double v = n[k] + R[k] * cn[a][0] + R[3 + k] * cn[a][1] + R[6 + k] * cn[a][2];
                    d2 += v * v;
                }
                P.Ra[a] = (float)std::sqrt(d2);
            }
            std::vector<float> Pm, PT;
            reinterp_matrix(Lt, R, ct, ctx->far_tnodes[t].data(), Pm);
            const int r = (int)(Pm.size() / kLOut);
            PT.resize(Pm.size());
            for (int b = 0; b < r; ++b)
                for (int a = 0; a < kLOut; ++a) PT[(size_t)a * r + b] = Pm[(size_t)b * kLOut + a];
            float *dP = nullptr;
            if ((st = upload(ctx, &dP, PT))) return st;
            P.P = dP;
            const bool use = ctx->net_pair.size() == (size_t)nd * nd && ctx->net_pair[(size_t)t * nd + s];
            P.yscale = use ? out_scale : 0.0f;
            ctx->net_used = ctx->net_used || use;
            ctx->lpairs.push_back(P);
        }
        const int p1 = (int)ctx->lpairs.size();
        if (p1 == p0) continue;
        const FarTarget &F = ctx->far_tgt[ftgt.at(t)];
        LTarget T{};
        T.cring = F.cring;
        T.depth = F.depth;
        T.r = F.r;
        T.p0 = p0;
        T.p1 = p1;
        T.overwrite = F.lag_hi_max < 0 ? 1 : 0;
        ctx->ltgts.push_back(T);
    }
    ctx->npairs_learned = (int)ctx->lpairs.size();
    {
        std::vector<int> pr(ctx->lpairs.size());
        for (const LTarget &T : ctx->ltgts)
            for (int p = T.p0; p < T.p1; ++p) pr[p] = T.r;
        if ((st = upload(ctx, &ctx->d_lpair_r, pr)) ||
            (st = dev_alloc(ctx, &ctx->d_lcontrib, ctx->lpairs.size() * kLOut * 4)))
            return st;
    }
    if ((st = upload(ctx, &ctx->d_lpairs, ctx->lpairs)) || (st = upload(ctx, &ctx->d_ltgts, ctx->ltgts)) ||
        (st = upload(ctx, &ctx->d_mjobs, ctx->mjobs)) || (st = dev_alloc(ctx, &ctx->d_lnu, 4 * ctx->lpairs.size())))
        return st;
    ctx->lrows = (int)((4 * ctx->lpairs.size() + 127) / 128 * 128);
    if ((st = dev_alloc(ctx, &ctx->d_lxf, (size_t)ctx->lrows * kLIn)) ||
        (st = dev_alloc(ctx, &ctx->d_lylin, (size_t)ctx->lrows * kLOut)))
        return st;
    void *enc = tensor_encoder();
    if (!enc) return fail(ctx, RP_ERR_UNSUPPORTED, "learned path needs cuTensorMapEncodeTiled");
    cudaError_t e = mlp_create(ctx->net, ctx->lrows, 1, enc);
    ctx->net_open = true;
    if (e) return cuda_fail(ctx, e, "learned network");
    cudaFree(ctx->net.d_err);
    ctx->net.d_err = ctx->d_err;
    RP_CUDA(ctx, mlp_set_weights(ctx->net, weights.data(), ctx->stream));
    RP_CUDA(ctx, cudaMemcpyAsync(ctx->net.Wlin, wlin.data(), wlin.size() * sizeof(float), cudaMemcpyHostToDevice,
                                 ctx->stream));
    RP_CUDA(ctx, cudaMemsetAsync(ctx->net.X16, 0, (size_t)ctx->lrows * kLIn * sizeof(__half), ctx->stream));
    RP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return RP_OK;
}

// Launch-shape autotuning: time each consumer-warp variant of the TMA-fed MAC
// on this plan (two launches after one warm-up, on the context stream, over
// rings whose contents do not matter for timing) and keep the fastest per
// size class.  Every variant reads the same data and sums in the same order.
rp_status autotune_mac(rp_ctx *ctx)
{
    if (ctx->comp) {   // one compensated variant
        std::fill(std::begin(ctx->mac_cw), std::end(ctx->mac_cw), kCompWarps);
        return RP_OK;
    }
    if (!ctx->tma || ctx->cfg.mac_warps) return RP_OK;
    cudaEvent_t a = nullptr, b = nullptr;
    RP_CUDA(ctx, cudaEventCreate(&a));
    RP_CUDA(ctx, cudaEventCreate(&b));
    rp_status st = RP_OK;
    const long long step = ctx->max_lag;   // every (step - lag) is a valid slot
    for (const LaunchGroup &g : ctx->inv_groups) {
        if (g.cls <= 0 || st) continue;
        const int slot = class_slot(g.cls), ntiles = g.blk1 - g.blk0;
        float best = 1e30f;
        for (int cw : {8, 12, 16}) {
            auto go = [&] {
                return launch_mac_tma(g.cls, cw, false, ctx->d_inv, g.i0, g.i1, g.blk0, ntiles, ctx->d_entries, step, 0,
                                      ctx->mac_stages[slot], std::min(ntiles, ctx->sm_count), ctx->d_err,
                                      ctx->stream);
            };
            cudaError_t e = go();
            if (!e) e = cudaEventRecord(a, ctx->stream);
            for (int r = 0; r < 2 && !e; ++r) e = go();
            if (!e) e = cudaEventRecord(b, ctx->stream);
            if (!e) e = cudaEventSynchronize(b);
            float ms = 0.0f;
            if (!e) e = cudaEventElapsedTime(&ms, a, b);
            if (e) {
                st = cuda_fail(ctx, e, "MAC autotuning");
                break;
            }
            if (ms < best) {
                best = ms;
                ctx->mac_cw[slot] = cw;
            }
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (st) return st;
    int flag = 0;
    RP_CUDA(ctx, cudaMemcpy(&flag, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag) return fail(ctx, RP_ERR_TIMEOUT, "a bounded device wait ran out during MAC autotuning");
    return RP_OK;
}

}  // namespace

// =========================================================================== C-ABI

extern "C" {

const char *rp_status_str(rp_status s)
{
    switch (s) {
    case RP_OK: return "RP_OK";
    case RP_ERR_ARG: return "RP_ERR_ARG";
    case RP_ERR_STATE: return "RP_ERR_STATE";
    case RP_ERR_HISTORY: return "RP_ERR_HISTORY";
    case RP_ERR_CUDA: return "RP_ERR_CUDA";
    case RP_ERR_OOM: return "RP_ERR_OOM";
    case RP_ERR_UNSUPPORTED: return "RP_ERR_UNSUPPORTED";
    case RP_ERR_TIMEOUT: return "RP_ERR_TIMEOUT";
    }
    return "RP_ERR_UNKNOWN";
}

const char *rp_last_error(rp_ctx *ctx) { return ctx ? ctx->last_error.c_str() : ""; }

const char *rp_kernel_name(int kind)
{
    static const char *names[RP_K_COUNT] = {"ring_push", "fwd_plane", "fwd_column", "mac_inv_column",
                                            "inv_plane", "direct", "far_convert", "far_gemm",
                                            "far_scatter", "far_anterp", "moments", "learned",
                                            "far_interp"};
    return (kind >= 0 && kind < RP_K_COUNT) ? names[kind] : nullptr;
}

rp_status rp_create(const rp_config *cfg, int device, void *stream, rp_ctx **out)
{
    if (!cfg || !out) return RP_ERR_ARG;
    *out = nullptr;
    if (!(cfg->c > 0.0) || !(cfg->dt > 0.0) || cfg->history_depth < 0) return RP_ERR_ARG;
    if (cfg->mode != RP_MODE_FFT && cfg->mode != RP_MODE_DIRECT && cfg->mode != RP_MODE_LOWRANK) return RP_ERR_ARG;
    if (cfg->mode == RP_MODE_LOWRANK) {
        if (!(cfg->far_distance > 0.0)) return RP_ERR_ARG;
        if (cfg->far_points != 0 && (cfg->far_points < 2 || cfg->far_points > kMaxFarPts)) return RP_ERR_ARG;
        if (cfg->far_batch != 0 && (cfg->far_batch < 8 || cfg->far_batch > 64 || cfg->far_batch % 8)) return RP_ERR_ARG;
        if (cfg->far_source_points != 0 && cfg->far_batch > 32) return RP_ERR_ARG;   // one 128-row window
    }
    if (cfg->mac_warps != 0 && cfg->mac_warps != 8 && cfg->mac_warps != 12 && cfg->mac_warps != 16) return RP_ERR_ARG;
    if (!(cfg->flags & RP_FLAG_PLAIN_SUM) && cfg->mac_warps != 0 && cfg->mac_warps != kCompWarps) return RP_ERR_ARG;
    if (cfg->profile_every < 0 || cfg->device_budget < 0) return RP_ERR_ARG;
    if (cfg->mac_stages != 0 && cfg->mac_stages < 2) return RP_ERR_ARG;
    if (cfg->far_source_points != 0 && (cfg->far_source_points < 2 || cfg->far_source_points > kMaxFarPts))
        return RP_ERR_ARG;
    rp_ctx *ctx = new rp_ctx();
    ctx->cfg = *cfg;
    if (ctx->cfg.far_points == 0) ctx->cfg.far_points = 4;
    if (ctx->cfg.far_batch == 0) ctx->cfg.far_batch = 32;
    if (ctx->cfg.mac_warps) std::fill(std::begin(ctx->mac_cw), std::end(ctx->mac_cw), ctx->cfg.mac_warps);
    ctx->plan_only = (cfg->flags & RP_FLAG_PLAN_ONLY) != 0;
    ctx->split = (cfg->flags & RP_FLAG_GROUND_STATE_SPLIT) != 0;
    ctx->spill = (cfg->flags & RP_FLAG_HISTORY_SPILL) != 0;
    ctx->comp = (cfg->flags & RP_FLAG_PLAIN_SUM) == 0;
    ctx->overlap = (cfg->flags & RP_FLAG_OVERLAP_PUSH) != 0;
    // the split's histories are zero before the first push: the clamped reads
    // of steps before it read the zeroed slot of step 0
    ctx->clamp = (cfg->flags & RP_FLAG_GROUND_STATE_CLAMP) != 0 || ctx->split;
    ctx->profile = (cfg->flags & RP_FLAG_PROFILE) != 0 && !ctx->plan_only;
    if (!ctx->plan_only) {
        int count = 0;
        if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
            cudaGetLastError();
            delete ctx;
            return RP_ERR_CUDA;
        }
        ctx->device = device;
        ctx->stream = static_cast<cudaStream_t>(stream);
        if (cudaSetDevice(device) != cudaSuccess) {
            cudaGetLastError();
            delete ctx;
            return RP_ERR_CUDA;
        }
    }
    *out = ctx;
    return RP_OK;
}

rp_status rp_add_domain(rp_ctx *ctx, const double origin[3], const int n[3], double h, int *id)
{
    if (!ctx || !origin || !n || !id) return RP_ERR_ARG;
    if (ctx->finalized) return fail(ctx, RP_ERR_STATE, "rp_add_domain after rp_finalize");
    if (!(h > 0.0) || n[0] < 1 || n[1] < 1 || n[2] < 1) return fail(ctx, RP_ERR_ARG, "bad domain size or spacing");
    for (int a = 0; a < 3; ++a)
        if (!std::isfinite(origin[a])) return fail(ctx, RP_ERR_ARG, "non-finite origin");
    if ((int)ctx->doms.size() >= kMaxDomains) return fail(ctx, RP_ERR_ARG, "too many domains");
    DomainDesc d{};
    for (int a = 0; a < 3; ++a) { d.o[a] = origin[a]; d.n[a] = n[a]; }
    d.h = h;
    d.N = (long long)n[0] * n[1] * n[2];
    ctx->doms.push_back(d);
    if (!ctx->owned.empty()) ctx->owned.push_back(0);   // rp_own_sources named the earlier domains only
    *id = (int)ctx->doms.size() - 1;
    return RP_OK;
}

rp_status rp_own_sources(rp_ctx *ctx, const int *ids, int count)
{
    if (!ctx) return RP_ERR_ARG;
    if (ctx->finalized) return fail(ctx, RP_ERR_STATE, "rp_own_sources after rp_finalize");
    const int nd = (int)ctx->doms.size();
    if (!ids || count < 1 || count > nd) return fail(ctx, RP_ERR_ARG, "rp_own_sources: bad id list");
    std::vector<char> own(nd, 0);
    for (int i = 0; i < count; ++i) {
        if (ids[i] < 0 || ids[i] >= nd || own[ids[i]])
            return fail(ctx, RP_ERR_ARG, "rp_own_sources: id out of range or repeated");
        own[ids[i]] = 1;
    }
    ctx->owned = own;
    return RP_OK;
}

rp_status rp_finalize(rp_ctx *ctx)
{
    if (!ctx) return RP_ERR_ARG;
    if (ctx->finalized) return fail(ctx, RP_ERR_STATE, "already finalized");
    const int nd = (int)ctx->doms.size();
    if (nd == 0) return fail(ctx, RP_ERR_STATE, "no domains");
    const double cdt = ctx->cfg.c * ctx->cfg.dt;
    const bool fft_mode = ctx->cfg.mode == RP_MODE_FFT || ctx->cfg.mode == RP_MODE_LOWRANK;
    if (ctx->owned.empty()) ctx->owned.assign(nd, 1);
    ctx->n_owned = (int)std::count(ctx->owned.begin(), ctx->owned.end(), 1);

    // ---- pairs: lag windows and kinds
    ctx->pairs.assign((size_t)nd * nd, PairPlan{});
    for (int t = 0; t < nd; ++t)
        for (int s = 0; s < nd; ++s) {
            const DomainDesc &T = ctx->doms[t], &S = ctx->doms[s];
            if (t != s && nodes_coincide(T, S))
                return fail(ctx, RP_ERR_ARG, "domains " + std::to_string(t) + " and " + std::to_string(s) +
                                                 " have a node at the same position");
            PairPlan &p = ctx->pairs[(size_t)t * nd + s];
            pair_distances(T, S, t == s, &p.rmin, &p.rmax);
            p.lag_lo = t == s ? 0 : std::max(0, (int)std::floor(p.rmin / cdt - 1e-9));
            p.lag_hi = (int)std::floor(p.rmax / cdt + 1e-9) + 1;
            p.kind = RP_PAIR_DIRECT;
            if (fft_mode && std::fabs(T.h - S.h) <= 1e-12 * T.h) {
                int m[3];
                bool ok = true;
                for (int a = 0; a < 3; ++a) {
                    m[a] = good_size(T.n[a] + S.n[a] - 1, a == 0);
                    ok = ok && m[a] > 0;
                }
                if (ok) {
                    p.kind = RP_PAIR_FFT;
                    for (int a = 0; a < 3; ++a) p.m[a] = m[a];
                }
            }
            // a batch of pushes completes before its first target step is
            // evaluated (one-sided factors, applied at the batch's last push
            // to the steps it reaches), or before the batch of target steps
            // it gives is gathered (two-sided factors)
            const int min_lo = ctx->cfg.far_source_points > 0 ? ctx->cfg.far_batch : ctx->cfg.far_batch - 1;
            if (ctx->cfg.mode == RP_MODE_LOWRANK && t != s && p.rmin >= ctx->cfg.far_distance && p.lag_lo >= min_lo)
                p.kind = RP_PAIR_LOWRANK;
            if (t == s && fft_mode && p.kind != RP_PAIR_FFT)
                return fail(ctx, RP_ERR_UNSUPPORTED, "domain " + std::to_string(t) +
                                                         " exceeds 96 nodes per axis (FFT self term)");
            if (!ctx->owned[s]) {   // another context evaluates this source's pairs
                p.kind = RP_PAIR_OTHER;
                continue;
            }
            ctx->max_lag = std::max(ctx->max_lag, p.lag_hi);
        }
    // a target's FFT size: the largest over its FFT pairs
    std::vector<std::array<int, 3>> tm(nd, {0, 0, 0});
    std::vector<char> tgt_fft(nd, 0);
    for (int t = 0; t < nd; ++t)
        for (int s = 0; s < nd; ++s) {
            const PairPlan &p = ctx->pairs[(size_t)t * nd + s];
            if (p.kind != RP_PAIR_FFT) continue;
            tgt_fft[t] = 1;
            for (int a = 0; a < 3; ++a) tm[t][a] = std::max(tm[t][a], p.m[a]);
        }
    for (int t = 0; t < nd; ++t)
        for (int s = 0; s < nd; ++s) {
            PairPlan &p = ctx->pairs[(size_t)t * nd + s];
            if (p.kind == RP_PAIR_FFT)
                for (int a = 0; a < 3; ++a) p.m[a] = tm[t][a];
        }

    // ---- spectral rings: one per (source, target FFT size)
    std::map<std::pair<int, std::array<int, 3>>, int> ring_of;
    std::vector<std::pair<int, std::array<int, 3>>> ring_keys;
    std::vector<int> ring_depth;
    // history spill: a spilled pair's lags leave the device ring's depth
    // alone (its window ring holds them); the history depth then applies to
    // the host ring of a spilled source, and to the device rings of the others
    std::vector<char> pair_spilled(ctx->pairs.size(), 0), src_spilled(nd, 0);
    int host_depth = ctx->cfg.history_depth;
    for (int s = 0; s < nd; ++s)
        for (int t = 0; t < nd; ++t) {
            const PairPlan &p = ctx->pairs[(size_t)t * nd + s];
            if (p.kind != RP_PAIR_FFT) continue;
            auto key = std::make_pair(s, tm[t]);
            auto it = ring_of.find(key);
            if (it == ring_of.end()) {
                ring_of[key] = (int)ring_keys.size();
                ring_keys.push_back(key);
                ring_depth.push_back(1);
                it = ring_of.find(key);
            }
            if (ctx->spill && spill_window(p.lag_lo, p.lag_hi)) {
                pair_spilled[(size_t)t * nd + s] = 1;
                src_spilled[s] = 1;
                host_depth = std::max(host_depth, p.lag_hi + 1);
                continue;
            }
            // overlapped pushes: one slot more, so that push l + 1 writes none the
            // evaluation of step l reads
            ring_depth[it->second] = std::max(ring_depth[it->second], p.lag_hi + 1 + (ctx->overlap ? 1 : 0));
        }
    for (size_t r = 0; r < ring_keys.size(); ++r)
        if (!src_spilled[ring_keys[r].first]) ring_depth[r] = std::max(ring_depth[r], ctx->cfg.history_depth);
    for (int s = 0; s < nd; ++s)
        if (src_spilled[s]) {
            ctx->spill_srcs.push_back({s, nullptr, nullptr});
            ctx->host_bytes += (long long)host_depth * 16 * ctx->doms[s].N;
            ctx->spectral_bytes += (long long)kSpillStage * 16 * ctx->doms[s].N;
        }
    ctx->spill_hd = host_depth;
    // order rings by (kernel size class, source): each class is one launch
    std::vector<int> ring_order(ring_keys.size());
    for (size_t r = 0; r < ring_keys.size(); ++r) ring_order[r] = (int)r;
    auto ring_class = [&](int r) {
        const auto &m = ring_keys[r].second;
        return size_class(make_axis(m[0]), make_axis(m[1]), make_axis(m[2]));
    };
    std::stable_sort(ring_order.begin(), ring_order.end(), [&](int x, int y) {
        const int cx = ring_class(x), cy = ring_class(y);
        return cx != cy ? cx < cy : ring_keys[x].first < ring_keys[y].first;
    });
    std::vector<int> ring_pos(ring_keys.size());
    std::map<int, const float2 *> tw;
    {   // the plane passes' form per class, from its forward plane blocks
        int blocks[7] = {};
        for (size_t r = 0; r < ring_keys.size(); ++r) blocks[class_slot(ring_class((int)r))] += 4 * ctx->doms[ring_keys[r].first].n[2];
        for (size_t r = 0; r < ring_keys.size(); ++r) {
            const int cls = ring_class((int)r);
            ctx->fwd_tile[class_slot(cls)] = plane_tile_form(cls, blocks[class_slot(cls)], false);
        }
    }
    for (size_t i = 0; i < ring_order.size(); ++i) {
        const int r = ring_order[i];
        ring_pos[r] = (int)i;
        const int s = ring_keys[r].first;
        const auto &m = ring_keys[r].second;
        const DomainDesc &S = ctx->doms[s];
        FwdRing R{};
        R.nx = S.n[0]; R.ny = S.n[1]; R.nz = S.n[2];
        R.ax = make_axis(m[0]); R.ay = make_axis(m[1]); R.az = make_axis(m[2]);
        R.kx = m[0] / 2 + 1;
        R.src = s;
        R.depth = ring_depth[r];
        R.slot_elems = 4LL * spec_cells(R.kx, m[1], m[2]);
        R.plane0 = ctx->plane_blocks;
        R.tile0 = ctx->col_blocks;
        ctx->plane_blocks += 4 * R.nz;
        ctx->col_blocks += R.kx * ((m[1] + kTileY - 1) / kTileY);
        tw[m[0]]; tw[m[1]]; tw[m[2]];
        ctx->spectral_bytes += (long long)R.depth * R.slot_elems * (long long)sizeof(float2);
        ctx->spec_depth = std::max(ctx->spec_depth, R.depth);
        {
            const int c = size_class(R.ax, R.ay, R.az), cs = class_slot(c);
            const size_t need = smem_fwd_plane(c, ctx->fwd_tile[cs], R.ny, R.ax);
            ctx->smem_plane_cls[cs] = std::max(ctx->smem_plane_cls[cs], need);
            ctx->smem_plane = std::max(ctx->smem_plane, need);
        }
        ctx->smem_col = std::max(ctx->smem_col, smem_fwd_column(R.az));
        const int cls = ring_class(r);
        if (ctx->fwd_groups.empty() || ctx->fwd_groups.back().cls != cls)
            ctx->fwd_groups.push_back({cls, (int)i, (int)i, R.plane0, R.plane0, R.tile0, R.tile0});
        LaunchGroup &g = ctx->fwd_groups.back();
        g.i1 = (int)i + 1;
        g.blk1 = ctx->plane_blocks;
        g.blk2_1 = ctx->col_blocks;
        ctx->fwd.push_back(R);
    }
    for (auto &kv : ring_of) kv.second = ring_pos[kv.second];

    // ---- FFT targets, ordered by size class, and their (source, lag)
    // entries: the self pair's real kernels first, then the complex ones
    struct EntryPlan { int t, s, lag, ring; bool real_g; int win; };   // win: spill window, or -1
    std::vector<EntryPlan> eplan;
    std::vector<int> tgt_order;
    for (int t = 0; t < nd; ++t)
        if (tgt_fft[t]) tgt_order.push_back(t);
    auto tgt_class = [&](int t) {
        return size_class(make_axis(tm[t][0]), make_axis(tm[t][1]), make_axis(tm[t][2]));
    };
    std::stable_sort(tgt_order.begin(), tgt_order.end(),
                     [&](int x, int y) { return tgt_class(x) < tgt_class(y); });
    {   // the inverse plane pass's form per class, from its blocks
        int blocks[7] = {};
        for (int t : tgt_order) blocks[class_slot(tgt_class(t))] += 4 * ctx->doms[t].n[2];
        for (int t : tgt_order) ctx->inv_tile[class_slot(tgt_class(t))] =
                plane_tile_form(tgt_class(t), blocks[class_slot(tgt_class(t))], true);
    }
    for (int t : tgt_order) {
        const DomainDesc &T = ctx->doms[t];
        InvTarget I{};
        I.nx = T.n[0]; I.ny = T.n[1]; I.nz = T.n[2];
        I.ax = make_axis(tm[t][0]); I.ay = make_axis(tm[t][1]); I.az = make_axis(tm[t][2]);
        I.kx = tm[t][0] / 2 + 1;
        I.dom = t;
        I.e0 = (int)eplan.size();
        for (int pass = 0; pass < 2; ++pass) {
            for (int s = 0; s < nd; ++s) {
                const PairPlan &p = ctx->pairs[(size_t)t * nd + s];
                if (p.kind != RP_PAIR_FFT || (pass == 0) != (s == t)) continue;
                const int ring = ring_of[std::make_pair(s, tm[t])];
                int win = -1;
                if (pair_spilled[(size_t)t * nd + s]) {
                    for (size_t w = 0; w < ctx->spill_wins.size(); ++w) {
                        const SpillWindow &W = ctx->spill_wins[w];
                        if (W.ring == ring && W.lo == p.lag_lo && W.hi == p.lag_hi) win = (int)w;
                    }
                    if (win < 0) {
                        win = (int)ctx->spill_wins.size();
                        int ss = 0;
                        while (ctx->spill_srcs[ss].dom != s) ++ss;
                        const SpillWindow W{ring, ss, p.lag_lo, p.lag_hi, p.lag_hi - p.lag_lo + 1, nullptr, nullptr,
                                            -1, {-1, -1}};
                        ctx->spill_wins.push_back(W);
                        ctx->spectral_bytes += (long long)W.depth * ctx->fwd[ring].slot_elems * (long long)sizeof(float2) +
                                               2LL * 16 * ctx->doms[s].N;
                    }
                }
                for (int lag = p.lag_lo; lag <= p.lag_hi; ++lag) eplan.push_back({t, s, lag, ring, t == s, win});
            }
            if (pass == 0) I.er = (int)eplan.size();
        }
        I.e1 = (int)eplan.size();
        I.tile0 = ctx->mac_blocks;
        I.plane0 = ctx->invp_blocks;
        ctx->mac_blocks += I.kx * ((tm[t][1] + kTileY - 1) / kTileY);
        ctx->invp_blocks += 4 * I.nz;
        ctx->smem_mac = std::max(ctx->smem_mac, smem_mac_inv_column(I.az));
        {
            const int c = size_class(I.ax, I.ay, I.az), cs = class_slot(c);
            const size_t need = smem_inv_plane(c, ctx->inv_tile[cs], I.nx, I.ny, I.ax, I.ay);
            ctx->smem_inv_cls[cs] = std::max(ctx->smem_inv_cls[cs], need);
            ctx->smem_inv = std::max(ctx->smem_inv, need);
        }
        const int cls = tgt_class(t);
        const int i = (int)ctx->inv.size();
        if (ctx->inv_groups.empty() || ctx->inv_groups.back().cls != cls)
            ctx->inv_groups.push_back({cls, i, i, I.tile0, I.tile0, I.plane0, I.plane0});
        LaunchGroup &g = ctx->inv_groups.back();
        g.i1 = i + 1;
        g.blk1 = ctx->mac_blocks;
        g.blk2_1 = ctx->invp_blocks;
        ctx->inv.push_back(I);
    }
    for (const EntryPlan &e : eplan) {
        const auto &m = tm[e.t];
        const long long cells = spec_cells(m[0] / 2 + 1, m[1], m[2]);
        ctx->kernel_bytes += cells * (long long)(e.real_g ? sizeof(float) : sizeof(float2));
    }

    // ---- direct pairs, raw rings
    ctx->raw.assign(nd, RawRing{});
    std::vector<int> rdepth(nd, 0);
    int max_nlag = 2;
    for (int t = 0; t < nd; ++t) {
        DirectTarget D{};
        const DomainDesc &T = ctx->doms[t];
        D.dom = t;
        D.nx = T.n[0]; D.ny = T.n[1]; D.nz = T.n[2];
        D.n = T.N;
        D.ht = T.h;
        D.p0 = (int)ctx->dpairs.size();
        for (int s = 0; s < nd; ++s) {
            const PairPlan &p = ctx->pairs[(size_t)t * nd + s];
            if (p.kind != RP_PAIR_DIRECT) continue;
            const DomainDesc &S = ctx->doms[s];
            DirectPair P{};
            P.src = s;
            P.nx_s = S.n[0]; P.ny_s = S.n[1]; P.nz_s = S.n[2];
            P.n_s = S.N;
            P.dx = T.o[0] - S.o[0]; P.dy = T.o[1] - S.o[1]; P.dz = T.o[2] - S.o[2];
            P.hs = (float)S.h;
            P.vol = (float)(S.h * S.h * S.h);
            P.is_self = t == s;
            P.self_w = t == s ? (float)(cube_average_constant() * S.h * S.h) : 0.0f;
            P.lag_lo = p.lag_lo;
            P.nlag = p.lag_hi - p.lag_lo + 1;
            max_nlag = std::max(max_nlag, P.nlag);
            rdepth[s] = std::max(rdepth[s], p.lag_hi + 1 + (ctx->overlap ? 1 : 0));
            ctx->dpairs.push_back(P);
        }
        D.p1 = (int)ctx->dpairs.size();
        if (D.p1 > D.p0) {
            D.block0 = ctx->dir_blocks;
            D.accumulate = tgt_fft[t];
            ctx->dir_blocks += direct_blocks(T.N);
            ctx->dtg.push_back(D);
        }
    }
    if (max_nlag > 600) return fail(ctx, RP_ERR_UNSUPPORTED, "direct pair lag window above 600 steps");
    // FP64 audit: every source keeps its raw slices as deep as its deepest pair reads
    if (ctx->cfg.flags & RP_FLAG_AUDIT)
        for (int t = 0; t < nd; ++t)
            for (int s = 0; s < nd; ++s)
                rdepth[s] = std::max(rdepth[s], ctx->pairs[(size_t)t * nd + s].lag_hi + 1 + (ctx->overlap ? 1 : 0));
    ctx->smem_dir = smem_direct(max_nlag);
    ctx->raw_block0.assign(nd + 1, 0);
    for (int d = 0; d < nd; ++d) {
        int nb = 0;
        if (rdepth[d] > 0) {
            ctx->raw[d].depth = std::max(rdepth[d], ctx->cfg.history_depth);
            ctx->raw[d].n = ctx->doms[d].N;
            ctx->raw_depth = std::max(ctx->raw_depth, ctx->raw[d].depth);
            nb = (int)((4 * ctx->doms[d].N + kThreads * 8 - 1) / (kThreads * 8));
        }
        ctx->raw_block0[d + 1] = ctx->raw_block0[d] + nb;
    }
    ctx->pushed.assign(nd, 0);
    {
        int nfar = 0;
        for (const PairPlan &p : ctx->pairs) nfar += p.kind == RP_PAIR_LOWRANK;
        if (nfar && ctx->clamp)
            return fail(ctx, RP_ERR_UNSUPPORTED, "the far path needs a pushed history (no RP_FLAG_GROUND_STATE_CLAMP "
                                                 "or RP_FLAG_GROUND_STATE_SPLIT)");
        if (ctx->plan_only) ctx->npairs_far = nfar;
    }

    if (ctx->plan_only) {
        long long raw_bytes = 0;
        for (int d = 0; d < nd; ++d) raw_bytes += 16LL * ctx->raw[d].depth * ctx->raw[d].n;
        ctx->device_bytes = ctx->spectral_bytes + ctx->kernel_bytes + raw_bytes;
        if (ctx->cfg.device_budget > 0 && ctx->device_bytes > ctx->cfg.device_budget)
            return fail(ctx, RP_ERR_OOM, "planned device memory " + std::to_string(ctx->device_bytes) +
                                             " B exceeds the device budget of " +
                                             std::to_string(ctx->cfg.device_budget) + " B");
        ctx->finalized = true;
        return RP_OK;
    }

    // ---- device memory
    rp_status st = use_device(ctx);
    if (st) return st;
    if (ctx->overlap) {
        if (ctx->split || ctx->spill || (ctx->cfg.flags & RP_FLAG_DEFER_FAR))
            return fail(ctx, RP_ERR_UNSUPPORTED, "RP_FLAG_OVERLAP_PUSH: not with the ground-state split, the history "
                                                 "spill or the learned field");
        RP_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->push_stream, cudaStreamNonBlocking));
        RP_CUDA(ctx, cudaEventCreateWithFlags(&ctx->ev_pushed, cudaEventDisableTiming));
        RP_CUDA(ctx, cudaEventCreateWithFlags(&ctx->ev_stream, cudaEventDisableTiming));
        for (cudaEvent_t &e : ctx->ev_eval) RP_CUDA(ctx, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    }
    int max_optin = 0;
    RP_CUDA(ctx, cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device));
    ctx->smem_optin = max_optin;
    {
        const size_t need = std::max({ctx->smem_plane, ctx->smem_col, ctx->smem_mac, ctx->smem_inv, ctx->smem_dir});
        if (need > (size_t)max_optin)
            return fail(ctx, RP_ERR_UNSUPPORTED, "kernel shared memory " + std::to_string(need) +
                                                     " B exceeds the device limit " + std::to_string(max_optin));
    }
    if ((st = build_twiddles(ctx, tw))) return st;
    for (FwdRing &R : ctx->fwd) {
        if ((st = dev_alloc(ctx, &R.ring, (size_t)R.depth * R.slot_elems))) return st;
        RP_CUDA(ctx, cudaMemset(R.ring, 0, (size_t)R.depth * R.slot_elems * sizeof(float2)));
        if ((st = dev_alloc(ctx, &R.t1, 4ULL * R.kx * R.nz * R.ay.M))) return st;
        R.tw_x = tw[R.ax.M]; R.tw_y = tw[R.ay.M]; R.tw_z = tw[R.az.M];
    }
    if ((st = open_spill(ctx))) return st;
    if (ctx->split) {
        ctx->ground.assign(nd, nullptr);
        ctx->delta.assign(nd, nullptr);
        ctx->pstatic.assign(nd, nullptr);
        for (int d = 0; d < nd; ++d) {
            const size_t n4 = 4 * (size_t)ctx->doms[d].N;
            if ((st = dev_alloc(ctx, &ctx->ground[d], n4)) || (st = dev_alloc(ctx, &ctx->delta[d], n4)) ||
                (st = dev_alloc(ctx, &ctx->pstatic[d], n4)))
                return st;
        }
    }
    for (InvTarget &I : ctx->inv) {
        if ((st = dev_alloc(ctx, &I.t2, 4ULL * I.kx * I.nz * I.ay.M))) return st;
        I.tw_x = tw[I.ax.M]; I.tw_y = tw[I.ay.M]; I.tw_z = tw[I.az.M];
        I.has_direct = 0;
        for (const DirectTarget &D : ctx->dtg)
            if (D.dom == I.dom) I.has_direct = 1;
    }
    for (int d = 0; d < nd; ++d) {
        RawRing &rr = ctx->raw[d];
        if (rr.depth > 0) {
            if ((st = dev_alloc(ctx, &rr.ring, (size_t)rr.depth * 4 * rr.n))) return st;
            RP_CUDA(ctx, cudaMemset(rr.ring, 0, (size_t)rr.depth * 4 * rr.n * sizeof(float)));
        }
    }
    for (DirectPair &P : ctx->dpairs) {
        P.raw = ctx->raw[P.src].ring;
        P.depth = ctx->raw[P.src].depth;
    }

    // ---- kernel spectra (FP64 on the host, stored FP32), built in parallel;
    // each target's real and complex kernels are contiguous
    std::vector<void *> gptr(eplan.size(), nullptr);
    std::vector<float *> treal(ctx->inv.size(), nullptr);
    std::vector<float2 *> tcplx(ctx->inv.size(), nullptr);
    for (size_t ti = 0; ti < ctx->inv.size(); ++ti) {
        const InvTarget &I = ctx->inv[ti];
        const size_t cells = (size_t)spec_cells(I.kx, I.ay.M, I.az.M);
        const int nr = I.er - I.e0, nc = I.e1 - I.er;
        if (nr > 0 && (st = dev_alloc(ctx, &treal[ti], (size_t)nr * cells))) return st;
        if (nc > 0 && (st = dev_alloc(ctx, &tcplx[ti], (size_t)nc * cells))) return st;
        for (int e = I.e0; e < I.e1; ++e) {
            if (e < I.er) gptr[e] = treal[ti] + (size_t)(e - I.e0) * cells;
            else gptr[e] = tcplx[ti] + (size_t)(e - I.er) * cells;
        }
    }
    {
        std::atomic<size_t> next(0);
        std::atomic<int> err(0);
        const int dev = ctx->device;
        auto worker = [&]() {
            cudaSetDevice(dev);
            std::vector<float> hr;
            std::vector<float2> hc;
            for (;;) {
                const size_t i = next.fetch_add(1);
                if (i >= eplan.size() || err.load()) break;
                const EntryPlan &e = eplan[i];
                const DomainDesc &T = ctx->doms[e.t], &S = ctx->doms[e.s];
                const int *m = tm[e.t].data();
                const size_t cells = (size_t)spec_cells(m[0] / 2 + 1, m[1], m[2]);
                if (e.real_g) hr.resize(cells); else hc.resize(cells);
                build_kernel_spectrum(T.o, T.n, S.o, S.n, S.h, e.t == e.s, e.lag, ctx->cfg.c, ctx->cfg.dt, m,
                                      e.real_g, hr.data(), hc.data());
                cudaError_t ce = e.real_g ? cudaMemcpy(gptr[i], hr.data(), cells * sizeof(float), cudaMemcpyHostToDevice)
                                          : cudaMemcpy(gptr[i], hc.data(), cells * sizeof(float2), cudaMemcpyHostToDevice);
                if (ce != cudaSuccess) err.store((int)ce);
            }
        };
        unsigned nthr = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
        nthr = (unsigned)std::min<size_t>(nthr, std::max<size_t>(1, eplan.size()));
        std::vector<std::thread> pool;
        for (unsigned i = 0; i < nthr; ++i) pool.emplace_back(worker);
        for (auto &th : pool) th.join();
        if (err.load()) return cuda_fail(ctx, (cudaError_t)err.load(), "kernel spectrum upload");
    }
    for (size_t ti = 0; ti < ctx->inv.size(); ++ti) {
        const InvTarget &I = ctx->inv[ti];
        for (int i = I.e0; i < I.e1; ++i) {
            const EntryPlan &e = eplan[i];
            const FwdRing &R = ctx->fwd[e.ring];
            MacEntry E{};
            E.g = gptr[i];
            E.ring = R.ring;
            E.slot_elems = R.slot_elems;
            E.depth = R.depth;
            if (e.win >= 0) {   // a spilled window: its own ring, same slot layout
                E.ring = ctx->spill_wins[e.win].dev;
                E.depth = ctx->spill_wins[e.win].depth;
            }
            E.lag = e.lag;
            E.is_real = e.real_g ? 1 : 0;
            ctx->entries.push_back(E);
        }
    }

    // ---- bulk-copy MAC pipeline for the cubic classes
    if ((st = plan_mac_tma(ctx, max_optin))) return st;

    // ---- far pairs
    RP_CUDA(ctx, cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, ctx->device));
    if (!(ctx->cfg.flags & RP_FLAG_DEFER_FAR) && (st = build_far(ctx, max_optin))) return st;

    // ---- device tables and kernel limits
    if ((st = dev_alloc(ctx, &ctx->d_step, 1))) return st;
    RP_CUDA(ctx, cudaMemset(ctx->d_step, 0, sizeof(long long)));
    for (FwdRing &R : ctx->fwd) R.d_step = ctx->d_step;
    for (InvTarget &I : ctx->inv) I.d_step = ctx->d_step;
    for (DirectTarget &D : ctx->dtg) D.d_step = ctx->d_step;
    for (RawRing &r : ctx->raw) r.d_step = ctx->d_step;
    if ((st = upload(ctx, &ctx->d_fwd, ctx->fwd))) return st;
    for (FwdRing &F : ctx->wfwd) F.d_step = ctx->d_step;
    if (!ctx->wfwd.empty() && (st = upload(ctx, &ctx->d_wfwd, ctx->wfwd))) return st;
    if ((st = build_mix(ctx))) return st;
    if ((st = upload(ctx, &ctx->d_inv, ctx->inv))) return st;
    if ((st = upload(ctx, &ctx->d_entries, ctx->entries))) return st;
    if ((st = upload(ctx, &ctx->d_dtg, ctx->dtg))) return st;
    if ((st = upload(ctx, &ctx->d_dpairs, ctx->dpairs))) return st;
    if ((st = upload(ctx, &ctx->d_raw, ctx->raw))) return st;
    RP_CUDA(ctx, open_kernel_smem_limits(max_optin));
    RP_CUDA(ctx, open_direct_smem_limit(max_optin));
    RP_CUDA(ctx, open_mac_tma_smem_limit(max_optin));
    if ((st = dev_alloc(ctx, &ctx->d_err, 1))) return st;
    RP_CUDA(ctx, cudaMemset(ctx->d_err, 0, sizeof(int)));
    // the fixed staging array of rp_evaluate_host_noalloc: its address is
    // looked up here, at set-up, so that the module holding it is loaded (and
    // the array placed in device memory) now and not at that call's first use
    if ((st = noalloc_stage_address(ctx, &ctx->noalloc_stage))) return st;
    RP_CUDA(ctx, cudaDeviceSynchronize());
    if ((st = autotune_mac(ctx))) return st;
    ctx->finalized = true;
    return RP_OK;
}

}  // extern "C"

namespace {

rp_status check_ready(rp_ctx *ctx)
{
    if (!ctx) return RP_ERR_ARG;
    if (!ctx->finalized || ctx->plan_only) return fail(ctx, RP_ERR_STATE, "context not finalized for execution");
    return use_device(ctx);
}

// Marks domain id pushed in the current round, starting a new round if the
// previous one is complete.
rp_status begin_push(rp_ctx *ctx, int id)
{
    if ((ctx->cfg.flags & RP_FLAG_DEFER_FAR) && !ctx->trained)
        return fail(ctx, RP_ERR_STATE, "RP_FLAG_DEFER_FAR: call rp_train_far_model before the first push");
    const int nd = (int)ctx->doms.size();
    if (!ctx->owned[id]) return fail(ctx, RP_ERR_ARG, "domain " + std::to_string(id) + " is not owned by this context");
    if (ctx->step < 0 || ctx->npushed == nd) {
        ctx->step += 1;
        for (int d = 0; d < nd; ++d) ctx->pushed[d] = ctx->owned[d] ? 0 : 1;   // others' sources count as pushed
        ctx->npushed = nd - ctx->n_owned;
    }
    if (ctx->pushed[id]) return fail(ctx, RP_ERR_STATE, "domain " + std::to_string(id) + " pushed twice in one step");
    ctx->pushed[id] = 1;
    ctx->npushed += 1;
    return RP_OK;
}

rp_status enqueue_push(rp_ctx *ctx, int d0, int d1, const IoPtrs &in)
{
    rp_status st;
    const long long step = ctx->step;
    const long long kstep = ctx->capturing ? -1 : step;   // graph capture: kernels read the device counter
    // history spill: the slices of spilled sources into the staging slot of
    // step - kSpillStage, once its copy to the host is done
    bool staged_wait = false;
    for (const SpillSource &S : ctx->spill_srcs) {
        if (S.dom < d0 || S.dom >= d1) continue;
        if (!staged_wait && step >= kSpillStage)
            RP_CUDA(ctx, cudaStreamWaitEvent(ctx->stream, ctx->sp_out[step % kSpillStage], 0));
        staged_wait = true;
        const long long N = ctx->doms[S.dom].N;
        float *dst = S.stage + (size_t)(step % kSpillStage) * 4 * N;
        if (in.J[S.dom] == in.rho[S.dom] + N) {   // one [4][N] buffer
            RP_CUDA(ctx, cudaMemcpyAsync(dst, in.rho[S.dom], 4 * N * sizeof(float), cudaMemcpyDeviceToDevice,
                                         ctx->stream));
        } else {
            RP_CUDA(ctx, cudaMemcpyAsync(dst, in.rho[S.dom], N * sizeof(float), cudaMemcpyDeviceToDevice, ctx->stream));
            RP_CUDA(ctx, cudaMemcpyAsync(dst + N, in.J[S.dom], 3 * N * sizeof(float), cudaMemcpyDeviceToDevice,
                                         ctx->stream));
        }
    }
    // raw ring
    int blk = ctx->raw_block0[d1] - ctx->raw_block0[d0];
    if (blk > 0) {
        std::vector<int> b0(kMaxDomains + 1, 0);
        for (int d = d0; d <= d1; ++d) b0[d] = ctx->raw_block0[d] - ctx->raw_block0[d0];
        if ((st = timed_launch(ctx, RP_K_RING_PUSH, "ring push", [&] {
                 return launch_ring_push(ctx->d_raw, in, d0, d1, b0.data(), blk, kstep, ctx->stream);
             })))
            return st;
    }
    // spectral rings of these sources: one launch pair per size class when
    // every domain pushes, else one per ring of the pushing domain.  History
    // spill: when every window lacks just step - lo, with its slice already
    // in, a whole round's launch pairs transform the windows too
    const int nd = (int)ctx->doms.size();
    std::vector<LaunchGroup> launches;
    const FwdRing *rings = ctx->d_fwd;
    IoPtrs fin = in;
    bool merged = false;
    if (d0 == 0 && d1 == nd) {
        launches = ctx->fwd_groups;
        merged = !ctx->mix.empty() && !ctx->capturing;
        for (const SpillWindow &W : ctx->spill_wins) {
            const long long j = step - W.lo;
            merged = merged && j >= 0 && W.have == j - 1 && W.raw_step[j & 1] == j;
        }
        if (merged) {
            launches = ctx->mix_groups;
            rings = ctx->d_mix;
            for (size_t w = 0; w < ctx->spill_wins.size(); ++w) {
                const SpillWindow &W = ctx->spill_wins[w];
                const long long Ns = ctx->doms[ctx->spill_srcs[W.ss].dom].N;
                fin.rho[nd + w] = W.raw + (size_t)((step - W.lo) & 1) * 4 * Ns;
                fin.J[nd + w] = fin.rho[nd + w] + Ns;
            }
            RP_CUDA(ctx, cudaStreamWaitEvent(ctx->stream, ctx->sp_in, 0));
        }
    } else {
        for (int r = 0; r < (int)ctx->fwd.size(); ++r) {
            const FwdRing &R = ctx->fwd[r];
            if (R.src < d0 || R.src >= d1) continue;
            const int tiles = R.kx * ((R.ay.M + kTileY - 1) / kTileY);
            launches.push_back({size_class(R.ax, R.ay, R.az), r, r + 1, R.plane0, R.plane0 + 4 * R.nz, R.tile0,
                                R.tile0 + tiles});
        }
    }
    for (const LaunchGroup &g : launches) {
        if ((st = timed_launch(ctx, RP_K_FWD_PLANE, "forward plane pass", [&] {
                 return launch_fwd_plane(g.cls, ctx->fwd_tile[class_slot(g.cls)], rings, fin, g.i0, g.i1, g.blk0,
                                         g.blk1 - g.blk0, ctx->smem_plane_cls[class_slot(g.cls)],
                                         (int)(step % std::max(1, ctx->cfg.far_batch)), ctx->stream);
             })))
            return st;
    }
    for (const LaunchGroup &g : launches) {
        if ((st = timed_launch(ctx, RP_K_FWD_COLUMN, "forward column pass", [&] {
                 return launch_fwd_column(g.cls, rings, g.i0, g.i1, g.blk2_0, g.blk2_1 - g.blk2_0,
                                          ctx->smem_col, kstep, ctx->stream);
             })))
            return st;
    }
    if (merged) {
        RP_CUDA(ctx, cudaEventRecord(ctx->sp_wfft, ctx->stream));
        for (SpillWindow &W : ctx->spill_wins) W.have = step - W.lo;
    }
    // two-sided far factors: the pushed slices of far sources onto their
    // nodes; when a round completes the last step of a batch, the gathered
    // GEMM gives every far target its node values of the next batch of steps
    if (ctx->far2) {
        int a0 = -1, a1 = -1;
        for (int d = d0; d < d1; ++d) {
            const int ai = ctx->far2_of_dom[d];
            if (ai < 0) continue;
            if (a0 < 0) a0 = ai;
            a1 = ai + 1;
        }
        if (a0 >= 0 && (st = timed_launch(ctx, RP_K_FAR_ANTERP, "far anterpolation", [&] {
                            return launch_far_anterp(ctx->d_far2_srcs + a0, a1 - a0, ctx->cfg.far_source_points,
                                                     ctx->far2_max_nz,
                                                     ctx->far2_max_plane, ctx->far2_max_n, in, kstep, ctx->d_step,
                                                     ctx->far2_D, ctx->far2_KS, ctx->stream);
                        })))
            return st;
        const int batch = ctx->cfg.far_batch;
        // a recorded step launches both every step; they read the device step
        // and work on a batch's last push only
        if (ctx->capturing || (ctx->npushed == nd && step % batch == batch - 1)) {
            const long long l0 = ctx->capturing ? -1 : step + 1;
            if ((st = timed_launch(ctx, RP_K_FAR_GEMM, "far gathered GEMM", [&] {
                     return launch_far_gather(ctx->far2_mapQ, ctx->far2_mapF, ctx->d_far2_tasks,
                                              (int)ctx->far2_tasks.size(), ctx->d_far2_kb, ctx->far2_BN, ctx->far2_KS,
                                              ctx->far2_D, l0, ctx->d_step, batch, ctx->far2_work, ctx->smem_optin,
                                              ctx->d_err, ctx->stream);
                 })))
                return st;
            if ((st = timed_launch(ctx, RP_K_FAR_SCATTER, "far gathered sums", [&] {
                     return launch_far_reduce(ctx->d_far_tgt, (int)ctx->far_tgt.size(), ctx->far2_work, ctx->far2_BN,
                                              l0, ctx->d_step, batch, ctx->far_max_r, ctx->stream);
                 })))
                return st;
        }
    }
    // far path: stage the slices of far sources; every far_batch steps run
    // the factor GEMM of each source and add its node values to the rings
    if (!ctx->far_src.empty()) {
        int f0 = -1, f1 = -1;
        for (int d = d0; d < d1; ++d) {
            const int fi = ctx->far_src_of_dom[d];
            if (fi < 0) continue;
            if (f0 < 0) f0 = fi;
            f1 = fi + 1;
        }
        if (f0 >= 0) {
            const int batch = ctx->cfg.far_batch;
            const int slot = (int)(step % batch);
            int a0 = -1, a1 = -1;
            for (int d = d0; d < d1; ++d) {
                const int ai = ctx->far_src_alone_of_dom[d];
                if (ai < 0) continue;
                if (a0 < 0) a0 = ai;
                a1 = ai + 1;
            }
            if (a0 >= 0 && (st = timed_launch(ctx, RP_K_FAR_CONVERT, "far slice staging", [&] {
                                 return launch_far_convert(ctx->d_far_src_alone + a0, a1 - a0, in, slot,
                                                           ctx->far_max_n, ctx->stream);
                             })))
                return st;
            if (slot == batch - 1) {
                if (ctx->far_zeroed_step != step) {
                    if ((st = timed_launch(ctx, RP_K_FAR_SCATTER, "far ring zero", [&] {
                             return launch_far_zero(ctx->d_far_tgt, (int)ctx->far_tgt.size(), step, batch,
                                                    ctx->far_max_r, ctx->stream);
                         })))
                        return st;
                    ctx->far_zeroed_step = step;
                }
                int optin = 0;
                RP_CUDA(ctx, cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device));
                for (int fi = f0; fi < f1; ++fi) {
                    if ((st = timed_launch(ctx, RP_K_FAR_GEMM, "far GEMM", [&] {
                             return launch_gemm_bf16_tn(ctx->far_mapW[fi], ctx->far_mapX[fi], ctx->far_Z[fi],
                                                        ctx->far_rows[fi], 4 * batch, ctx->far_src[fi].ks, 4 * batch,
                                                        optin, ctx->d_err, ctx->stream, ctx->far_splits[fi],
                                                        ctx->far_work, 1);
                         })))
                        return st;
                    if ((st = timed_launch(ctx, RP_K_FAR_SCATTER, "far scatter", [&] {
                             return launch_far_scatter(ctx->d_far_links + ctx->far_link0[fi],
                                                       ctx->far_link1[fi] - ctx->far_link0[fi],
                                                       ctx->far_link_threads[fi], ctx->far_Z[fi], 4 * batch,
                                                       step - batch + 1, batch, ctx->stream);
                         })))
                        return st;
                }
            }
        }
    }
    // learned path: moments of the pushed slices of its sources
    if (!ctx->mjobs.empty()) {
        int j0 = -1, j1 = -1;
        for (int d = d0; d < d1; ++d) {
            const int ji = ctx->mjob_of_dom[d];
            if (ji < 0) continue;
            if (j0 < 0) j0 = ji;
            j1 = ji + 1;
        }
        if (j0 >= 0 && (st = timed_launch(ctx, RP_K_MOMENTS, "source moments", [&] {
                             return launch_moments(ctx->d_mjobs + j0, j1 - j0, ctx->mjob_max_nz, step, &in,
                                                   ctx->stream);
                         })))
            return st;
    }
    return RP_OK;
}

// Overlapped pushes: the launches of a push on the push stream, after the
// inputs' readiness (the caller's event; or, without one, everything the
// context stream has been given) and after the evaluation two steps back
// (whose ring slots this push's slot may otherwise reach); "pushed" is
// recorded after them for the next evaluation.
rp_status overlapped_push(rp_ctx *ctx, int d0, int d1, const IoPtrs &in, cudaEvent_t ready, bool have_ready)
{
    if (have_ready) {
        if (ready) RP_CUDA(ctx, cudaStreamWaitEvent(ctx->push_stream, ready, 0));
    } else {
        RP_CUDA(ctx, cudaEventRecord(ctx->ev_stream, ctx->stream));
        RP_CUDA(ctx, cudaStreamWaitEvent(ctx->push_stream, ctx->ev_stream, 0));
    }
    RP_CUDA(ctx, cudaStreamWaitEvent(ctx->push_stream, ctx->ev_eval[ctx->step & 1], 0));
    cudaStream_t user = ctx->stream;
    ctx->stream = ctx->push_stream;
    const rp_status st = enqueue_push(ctx, d0, d1, in);
    ctx->stream = user;
    if (st) return st;
    RP_CUDA(ctx, cudaEventRecord(ctx->ev_pushed, ctx->push_stream));
    return RP_OK;
}

}  // namespace

extern "C" {

// Ground-state split, at a push of domains [d0, d1): on the first step keep
// S(0) (pushed as it is, for the static potential); later, push Delta S.
static rp_status split_inputs(rp_ctx *ctx, int d0, int d1, IoPtrs &in)
{
    if (!ctx->split) return RP_OK;
    for (int d = d0; d < d1; ++d) {
        const long long N = ctx->doms[d].N;
        if (ctx->step == 0) {
            RP_CUDA(ctx, cudaMemcpyAsync(ctx->ground[d], in.rho[d], N * sizeof(float), cudaMemcpyDeviceToDevice,
                                         ctx->stream));
            RP_CUDA(ctx, cudaMemcpyAsync(ctx->ground[d] + N, in.J[d], 3 * N * sizeof(float),
                                         cudaMemcpyDeviceToDevice, ctx->stream));
        } else {
            RP_CUDA(ctx, launch_ground_delta(in.rho[d], in.J[d], ctx->ground[d], ctx->delta[d], N, ctx->sm_count,
                                             ctx->stream));
            in.rho[d] = ctx->delta[d];
            in.J[d] = ctx->delta[d] + N;
        }
    }
    return RP_OK;
}

// Ground-state split, after a push: once the first round is complete, the
// static potential P(0) = sum_m G_m S(0) (a clamped evaluation over the
// history that holds S(0) alone), then the history of step 0 becomes
// Delta S(0) = 0.
static rp_status split_round_done(rp_ctx *ctx)
{
    const int nd = (int)ctx->doms.size();
    if (!ctx->split || ctx->static_done || ctx->step != 0 || ctx->npushed != nd) return RP_OK;
    std::vector<float *> phi(nd), A(nd);
    for (int d = 0; d < nd; ++d) {
        phi[d] = ctx->pstatic[d];
        A[d] = ctx->pstatic[d] + ctx->doms[d].N;
    }
    ctx->computing_static = true;
    rp_status st = rp_evaluate(ctx, phi.data(), A.data());
    ctx->computing_static = false;
    if (st) return st;
    for (const FwdRing &R : ctx->fwd)
        RP_CUDA(ctx, cudaMemsetAsync(R.ring, 0, R.slot_elems * sizeof(float2), ctx->stream));   // slot of step 0
    for (const RawRing &r : ctx->raw)
        if (r.ring) RP_CUDA(ctx, cudaMemsetAsync(r.ring, 0, 4 * r.n * sizeof(float), ctx->stream));
    // history spill: the staged and host slices of step 0 become zero too,
    // and the windows fetch them again
    for (const SpillSource &S : ctx->spill_srcs)
        RP_CUDA(ctx, cudaMemsetAsync(S.stage, 0, 16 * (size_t)ctx->doms[S.dom].N, ctx->stream));
    if ((st = spill_round_done(ctx))) return st;
    for (SpillWindow &W : ctx->spill_wins) W.have = W.raw_step[0] = W.raw_step[1] = -1;
    ctx->static_done = true;
    return RP_OK;
}

rp_status rp_push(rp_ctx *ctx, int id, const float *d_rho, const float *d_J)
{
    rp_status st = check_ready(ctx);
    if (st) return st;
    if (id < 0 || id >= (int)ctx->doms.size() || !d_rho || !d_J) return fail(ctx, RP_ERR_ARG, "rp_push: bad id or pointer");
    if ((st = begin_push(ctx, id))) return st;
    IoPtrs in{};
    in.rho[id] = d_rho;
    in.J[id] = d_J;
    if (ctx->overlap) return overlapped_push(ctx, id, id + 1, in, nullptr, false);
    if ((st = split_inputs(ctx, id, id + 1, in))) return st;
    if ((st = enqueue_push(ctx, id, id + 1, in))) return st;
    if ((st = spill_round_done(ctx))) return st;
    return split_round_done(ctx);
}

static rp_status push_all_impl(rp_ctx *ctx, const float *const *d_rho, const float *const *d_J, cudaEvent_t ready,
                               bool have_ready);

rp_status rp_push_all(rp_ctx *ctx, const float *const *d_rho, const float *const *d_J)
{
    return push_all_impl(ctx, d_rho, d_J, nullptr, false);
}

rp_status rp_push_all_event(rp_ctx *ctx, const float *const *d_rho, const float *const *d_J, void *ready)
{
    if (!ctx) return RP_ERR_ARG;
    if (!ctx->overlap) return fail(ctx, RP_ERR_STATE, "rp_push_all_event needs RP_FLAG_OVERLAP_PUSH");
    return push_all_impl(ctx, d_rho, d_J, static_cast<cudaEvent_t>(ready), true);
}

static rp_status push_all_impl(rp_ctx *ctx, const float *const *d_rho, const float *const *d_J, cudaEvent_t ready,
                               bool have_ready)
{
    rp_status st = check_ready(ctx);
    if (st) return st;
    const int nd = (int)ctx->doms.size();
    if (!d_rho || !d_J) return fail(ctx, RP_ERR_ARG, "rp_push_all: NULL pointer array");
    for (int d = 0; d < nd; ++d)
        if (ctx->owned[d] && (!d_rho[d] || !d_J[d])) return fail(ctx, RP_ERR_ARG, "rp_push_all: NULL buffer");
    if (ctx->step >= 0 && ctx->npushed != 0 && ctx->npushed != nd)
        return fail(ctx, RP_ERR_STATE, "rp_push_all inside a partially pushed step");
    if ((ctx->cfg.flags & RP_FLAG_DEFER_FAR) && !ctx->trained)
        return fail(ctx, RP_ERR_STATE, "RP_FLAG_DEFER_FAR: call rp_train_far_model before the first push");
    ctx->step += 1;
    std::fill(ctx->pushed.begin(), ctx->pushed.end(), 1);
    ctx->npushed = nd;
    IoPtrs in{};
    for (int d = 0; d < nd; ++d)
        if (ctx->owned[d]) { in.rho[d] = d_rho[d]; in.J[d] = d_J[d]; }
    if (ctx->overlap) return overlapped_push(ctx, 0, nd, in, ready, have_ready);
    rp_status st2;
    if ((st2 = split_inputs(ctx, 0, nd, in))) return st2;
    if ((st2 = enqueue_push(ctx, 0, nd, in))) return st2;
    if ((st2 = spill_round_done(ctx))) return st2;
    return split_round_done(ctx);
}

// The copy stream, events and staging vectors of the host-buffer calls, on
// first use.
static rp_status open_host_copies(rp_ctx *ctx)
{
    if (ctx->copy_in) return RP_OK;
    const int nd = (int)ctx->doms.size();
    cudaStream_t s_in = nullptr, s_out = nullptr;
    RP_CUDA(ctx, cudaStreamCreateWithFlags(&s_in, cudaStreamNonBlocking));
    ctx->copy_in = s_in;
    RP_CUDA(ctx, cudaStreamCreateWithFlags(&s_out, cudaStreamNonBlocking));
    ctx->copy_out = s_out;
    auto event = [&](cudaEvent_t *e) { return cudaEventCreateWithFlags(e, cudaEventDisableTiming); };
    RP_CUDA(ctx, event(&ctx->in_ready));
    RP_CUDA(ctx, event(&ctx->out_ready));
    for (int b = 0; b < 2; ++b) {
        RP_CUDA(ctx, event(&ctx->out_free[b]));
        ctx->in_stage[b].assign(nd, nullptr);
        ctx->out_stage[b].assign(nd, nullptr);
        RP_CUDA(ctx, event(&ctx->in_free[b]));
    }
    return RP_OK;
}

// Copies domain id's host inputs of step parity b into its device staging on
// the copy stream (the caller has made the stream wait for the last push that
// read that staging).
static rp_status stage_host_input(rp_ctx *ctx, int id, int b, const float *h_rho, const float *h_J)
{
    rp_status st;
    const long long N = ctx->doms[id].N;
    if (!ctx->in_stage[b][id] && (st = dev_alloc(ctx, &ctx->in_stage[b][id], 4 * (size_t)N))) return st;
    float *dst = ctx->in_stage[b][id];
    if (h_J == h_rho + N) {
        RP_CUDA(ctx, cudaMemcpyAsync(dst, h_rho, 4 * N * sizeof(float), cudaMemcpyHostToDevice, ctx->copy_in));
    } else {
        RP_CUDA(ctx, cudaMemcpyAsync(dst, h_rho, N * sizeof(float), cudaMemcpyHostToDevice, ctx->copy_in));
        RP_CUDA(ctx, cudaMemcpyAsync(dst + N, h_J, 3 * N * sizeof(float), cudaMemcpyHostToDevice, ctx->copy_in));
    }
    return RP_OK;
}

rp_status rp_push_host(rp_ctx *ctx, int id, const float *h_rho, const float *h_J)
{
    rp_status st = check_ready(ctx);
    if (st) return st;
    const int nd = (int)ctx->doms.size();
    if (id < 0 || id >= nd || !h_rho || !h_J) return fail(ctx, RP_ERR_ARG, "rp_push_host: bad id or pointer");
    if ((st = open_host_copies(ctx))) return st;
    // the step this push belongs to (a complete round starts the next one)
    const long long step = (ctx->step < 0 || ctx->npushed == nd) ? ctx->step + 1 : ctx->step;
    const int b = (int)(step & 1);
    RP_CUDA(ctx, cudaStreamWaitEvent(ctx->copy_in, ctx->in_free[b], 0));
    if ((st = stage_host_input(ctx, id, b, h_rho, h_J))) return st;
    RP_CUDA(ctx, cudaEventRecord(ctx->in_ready, ctx->copy_in));
    float *dst = ctx->in_stage[b][id];
    if (ctx->overlap) {   // the push's kernels wait for this copy alone
        if ((st = begin_push(ctx, id))) return st;
        IoPtrs in{};
        in.rho[id] = dst;
        in.J[id] = dst + ctx->doms[id].N;
        if ((st = overlapped_push(ctx, id, id + 1, in, ctx->in_ready, true))) return st;
        RP_CUDA(ctx, cudaEventRecord(ctx->in_free[b], ctx->push_stream));
        return RP_OK;
    }
    RP_CUDA(ctx, cudaStreamWaitEvent(ctx->stream, ctx->in_ready, 0));
    if ((st = rp_push(ctx, id, dst, dst + ctx->doms[id].N))) return st;
    RP_CUDA(ctx, cudaEventRecord(ctx->in_free[b], ctx->stream));
    return RP_OK;
}

rp_status rp_push_all_host(rp_ctx *ctx, const float *const *h_rho, const float *const *h_J)
{
    rp_status st = check_ready(ctx);
    if (st) return st;
    const int nd = (int)ctx->doms.size();
    if (!h_rho || !h_J) return fail(ctx, RP_ERR_ARG, "rp_push_all_host: NULL pointer array");
    for (int d = 0; d < nd; ++d)
        if (ctx->owned[d] && (!h_rho[d] || !h_J[d])) return fail(ctx, RP_ERR_ARG, "rp_push_all_host: NULL buffer");
    if (ctx->step >= 0 && ctx->npushed != 0 && ctx->npushed != nd)
        return fail(ctx, RP_ERR_STATE, "rp_push_all_host inside a partially pushed step");
    if ((st = open_host_copies(ctx))) return st;
    const int b = (int)((ctx->step + 1) & 1);
    RP_CUDA(ctx, cudaStreamWaitEvent(ctx->copy_in, ctx->in_free[b], 0));   // the push two steps back
    for (int d = 0; d < nd; ++d)
        if (ctx->owned[d] && (st = stage_host_input(ctx, d, b, h_rho[d], h_J[d]))) return st;
    RP_CUDA(ctx, cudaEventRecord(ctx->in_ready, ctx->copy_in));
    std::vector<const float *> rho(nd, nullptr), J(nd, nullptr);
    for (int d = 0; d < nd; ++d) {
        if (!ctx->owned[d]) continue;
        rho[d] = ctx->in_stage[b][d];
        J[d] = ctx->in_stage[b][d] + ctx->doms[d].N;
    }
    if (ctx->overlap) {   // the push's kernels wait for these copies alone
        if ((st = push_all_impl(ctx, rho.data(), J.data(), ctx->in_ready, true))) return st;
        RP_CUDA(ctx, cudaEventRecord(ctx->in_free[b], ctx->push_stream));
        return RP_OK;
    }
    RP_CUDA(ctx, cudaStreamWaitEvent(ctx->stream, ctx->in_ready, 0));
    if ((st = rp_push_all(ctx, rho.data(), J.data()))) return st;
    RP_CUDA(ctx, cudaEventRecord(ctx->in_free[b], ctx->stream));
    return RP_OK;
}

static rp_status evaluate_launches(rp_ctx *ctx, const OutPtrs &out, long long step, long long kstep, int clamp,
                                   float inv_c);

rp_status rp_evaluate(rp_ctx *ctx, float *const *d_phi, float *const *d_A)
{
    rp_status st = check_ready(ctx);
    if (st) return st;
    const int nd = (int)ctx->doms.size();
    if (!d_phi || !d_A) return fail(ctx, RP_ERR_ARG, "rp_evaluate: NULL pointer array");
    for (int d = 0; d < nd; ++d)
        if (!d_phi[d] || !d_A[d]) return fail(ctx, RP_ERR_ARG, "rp_evaluate: NULL output buffer");
    if (ctx->step < 0 || ctx->npushed != nd) return fail(ctx, RP_ERR_STATE, "rp_evaluate before every domain pushed the step");
    if (!ctx->clamp && !ctx->capturing && ctx->step - ctx->max_lag < 0)
        return fail(ctx, RP_ERR_HISTORY, "step " + std::to_string(ctx->step) + " needs samples " +
                                             std::to_string(ctx->max_lag) + " steps back");
    OutPtrs out{};
    for (int d = 0; d < nd; ++d) { out.phi[d] = d_phi[d]; out.A[d] = d_A[d]; }
    const long long step = ctx->step;
    const long long kstep = ctx->capturing ? -1 : step;   // graph capture: kernels read the device counter
    const int clamp = ctx->clamp ? 1 : 0;
    const float inv_c = (float)(1.0 / ctx->cfg.c);
    if (ctx->overlap) RP_CUDA(ctx, cudaStreamWaitEvent(ctx->stream, ctx->ev_pushed, 0));   // the step's push
    if ((st = spill_fetch(ctx))) return st;
    if ((st = evaluate_launches(ctx, out, step, kstep, clamp, inv_c))) return st;
    // the push of step + 2 may reuse the ring slots this evaluation reads
    if (ctx->overlap) RP_CUDA(ctx, cudaEventRecord(ctx->ev_eval[step & 1], ctx->stream));
    return RP_OK;
}

static rp_status evaluate_launches(rp_ctx *ctx, const OutPtrs &out, long long step, long long kstep, int clamp,
                                   float inv_c)
{
    rp_status st;
    for (const LaunchGroup &g : ctx->inv_groups) {
        const int ntiles = g.blk1 - g.blk0;
        if ((st = timed_launch(ctx, RP_K_MAC_INV_COLUMN, "MAC + inverse column pass", [&] {
                 if (ctx->tma && g.cls > 0)
                     return launch_mac_tma(g.cls, ctx->mac_cw[class_slot(g.cls)], ctx->comp, ctx->d_inv, g.i0, g.i1,
                                           g.blk0,
                                           ntiles, ctx->d_entries, kstep, clamp,
                                           ctx->mac_stages[class_slot(g.cls)],
                                           std::min(ntiles, ctx->sm_count), ctx->d_err, ctx->stream);
                 return launch_mac_inv_column(g.cls, ctx->comp, ctx->d_inv, g.i0, g.i1, g.blk0, ctx->d_entries, ntiles,
                                              ctx->smem_mac, kstep, clamp, ctx->stream);
             })))
            return st;
    }
    if (!ctx->lpairs.empty()) {
        // learned pairs: network rows, network, node values into the coefficients
        if ((st = timed_launch(ctx, RP_K_LEARNED, "learned far field", [&] {
                 const int nrows = 4 * (int)ctx->lpairs.size();
                 cudaError_t e = launch_features(ctx->d_lpairs, nullptr, (int)ctx->lpairs.size(), step,
                                                 ctx->net.X16, ctx->d_lxf, ctx->d_lnu, ctx->stream);
                 if (!e) e = linear_apply(ctx->net.Wlin, ctx->d_lxf, nrows, nullptr, 1.0f, ctx->d_lylin, ctx->stream);
                 if (!e && ctx->net_used)
                     e = mlp_forward(ctx->net, ctx->lrows, false, ctx->smem_optin, ctx->sm_count, ctx->stream);
                 if (!e)
                     e = launch_learned_out(ctx->d_ltgts, (int)ctx->ltgts.size(), ctx->d_lpairs,
                                            (int)ctx->lpairs.size(), ctx->d_lpair_r, ctx->net.Z[3], ctx->d_lylin,
                                            ctx->d_lnu, ctx->d_lcontrib, step, ctx->stream);
                 return e;
             })))
            return st;
    }
    for (const LaunchGroup &g : ctx->inv_groups) {
        if ((st = timed_launch(ctx, RP_K_INV_PLANE, "inverse plane pass", [&] {
                 return launch_inv_plane(g.cls, ctx->inv_tile[class_slot(g.cls)], ctx->d_inv, g.i0, g.i1, g.blk2_0,
                                         out, g.blk2_1 - g.blk2_0, ctx->smem_inv_cls[class_slot(g.cls)], inv_c, kstep,
                                         ctx->stream);
             })))
            return st;
    }
    if (!ctx->dtg.empty()) {
        const float inv_cdt = (float)(1.0 / (ctx->cfg.c * ctx->cfg.dt));
        if ((st = timed_launch(ctx, RP_K_DIRECT, "direct sum", [&] {
                 return launch_direct(ctx->d_dtg, (int)ctx->dtg.size(), ctx->d_dpairs, out, ctx->dir_blocks,
                                      ctx->smem_dir, kstep, clamp, inv_cdt, inv_c, ctx->stream);
             })))
            return st;
    }
    if (!ctx->far_tgt_alone.empty()) {
        if ((st = timed_launch(ctx, RP_K_FAR_INTERP, "far interpolation", [&] {
                 return launch_far_interp(ctx->d_far_tgt_alone, (int)ctx->far_tgt_alone.size(),
                                          ctx->far_alone_planes, out, kstep, ctx->d_step, inv_c, ctx->stream);
             })))
            return st;
    }
    return RP_OK;
}

rp_status rp_ground_potential(rp_ctx *ctx, float *const *d_phi, float *const *d_A)
{
    rp_status st = check_ready(ctx);
    if (st) return st;
    const int nd = (int)ctx->doms.size();
    if (!d_phi || !d_A) return fail(ctx, RP_ERR_ARG, "rp_ground_potential: NULL pointer array");
    for (int d = 0; d < nd; ++d)
        if (!d_phi[d] || !d_A[d]) return fail(ctx, RP_ERR_ARG, "rp_ground_potential: NULL output buffer");
    if (!ctx->split) return fail(ctx, RP_ERR_STATE, "rp_ground_potential needs RP_FLAG_GROUND_STATE_SPLIT");
    if (!ctx->static_done) return fail(ctx, RP_ERR_STATE, "rp_ground_potential before the first round is complete");
    for (int d = 0; d < nd; ++d) {
        const long long N = ctx->doms[d].N;
        RP_CUDA(ctx, cudaMemcpyAsync(d_phi[d], ctx->pstatic[d], N * sizeof(float), cudaMemcpyDeviceToDevice,
                                     ctx->stream));
        RP_CUDA(ctx, cudaMemcpyAsync(d_A[d], ctx->pstatic[d] + N, 3 * N * sizeof(float), cudaMemcpyDeviceToDevice,
                                     ctx->stream));
    }
    return RP_OK;
}

rp_status rp_evaluate_host(rp_ctx *ctx, float *const *h_phi, float *const *h_A)
{
    rp_status st = check_ready(ctx);
    if (st) return st;
    const int nd = (int)ctx->doms.size();
    if (!h_phi || !h_A) return fail(ctx, RP_ERR_ARG, "rp_evaluate_host: NULL pointer array");
    for (int d = 0; d < nd; ++d)
        if (!h_phi[d] || !h_A[d]) return fail(ctx, RP_ERR_ARG, "rp_evaluate_host: NULL output buffer");
    if ((st = open_host_copies(ctx))) return st;
    const int b = (int)(std::max(ctx->step, 0LL) & 1);
    std::vector<float *> phi(nd), A(nd);
    for (int d = 0; d < nd; ++d) {
        if (!ctx->out_stage[b][d] && (st = dev_alloc(ctx, &ctx->out_stage[b][d], 4 * (size_t)ctx->doms[d].N)))
            return st;
        phi[d] = ctx->out_stage[b][d];
        A[d] = ctx->out_stage[b][d] + ctx->doms[d].N;
    }
    // the evaluation waits for the copy out of this buffer two steps back
    RP_CUDA(ctx, cudaStreamWaitEvent(ctx->stream, ctx->out_free[b], 0));
    if ((st = rp_evaluate(ctx, phi.data(), A.data()))) return st;
    RP_CUDA(ctx, cudaEventRecord(ctx->out_ready, ctx->stream));
    RP_CUDA(ctx, cudaStreamWaitEvent(ctx->copy_out, ctx->out_ready, 0));
    for (int d = 0; d < nd; ++d) {
        const long long N = ctx->doms[d].N;
        if (h_A[d] == h_phi[d] + N) {
            RP_CUDA(ctx, cudaMemcpyAsync(h_phi[d], phi[d], 4 * N * sizeof(float), cudaMemcpyDeviceToHost,
                                         ctx->copy_out));
        } else {
            RP_CUDA(ctx, cudaMemcpyAsync(h_phi[d], phi[d], N * sizeof(float), cudaMemcpyDeviceToHost,
                                         ctx->copy_out));
            RP_CUDA(ctx, cudaMemcpyAsync(h_A[d], A[d], 3 * N * sizeof(float), cudaMemcpyDeviceToHost,
                                         ctx->copy_out));
        }
    }
    RP_CUDA(ctx, cudaEventRecord(ctx->out_free[b], ctx->copy_out));
    return RP_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- evaluation without allocation
//
// rp_evaluate_host stages phi and A in device memory it allocates on its
// first call.  The variant below stages them in a fixed array compiled into
// the library instead, so that it never calls an allocator.

namespace {

// Largest total sum over domains of 4 * N_d floats (phi, Ax, Ay, Az) the
// fixed staging array holds: 16 MiB, i.e. up to 1,048,576 grid points in all.
constexpr long long kNoAllocFloats = 4LL * 1024 * 1024;

// Device staging for rp_evaluate_host_noalloc.  Every device that loads the
// library holds it until the process exits; all contexts on a device share it.
static __device__ __align__(256) float g_noalloc_stage[kNoAllocFloats];

constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mutex;
float *g_noalloc_addr[kNoAllocMaxDevices] = {};

// Device address of the staging array on ctx->device.  Looked up once per
// device, with that device current, at the first rp_finalize on it (the
// host-side symbol is only a stand-in for the device address and must not be
// handed to a kernel).
rp_status noalloc_stage_address(rp_ctx *ctx, float **out)
{
    if (ctx->device < 0 || ctx->device >= kNoAllocMaxDevices)
        return fail(ctx, RP_ERR_UNSUPPORTED, "rp_evaluate_host_noalloc: device index above 63");
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_addr[ctx->device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_stage);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaGetSymbolAddress(g_noalloc_stage)");
        g_noalloc_addr[ctx->device] = static_cast<float *>(p);
    }
    *out = g_noalloc_addr[ctx->device];
    return RP_OK;
}

}  // namespace

extern "C" {

rp_status rp_evaluate_host_noalloc(rp_ctx *ctx, float *const *h_phi, float *const *h_A)
{
    rp_status st = check_ready(ctx);   // also makes ctx->device current
    if (st) return st;
    const int nd = (int)ctx->doms.size();
    if (!h_phi || !h_A) return fail(ctx, RP_ERR_ARG, "rp_evaluate_host_noalloc: NULL pointer array");
    for (int d = 0; d < nd; ++d)
        if (!h_phi[d] || !h_A[d]) return fail(ctx, RP_ERR_ARG, "rp_evaluate_host_noalloc: NULL output buffer");
    long long need = 0;
    for (int d = 0; d < nd; ++d) need += 4 * ctx->doms[d].N;
    if (need > kNoAllocFloats)
        return fail(ctx, RP_ERR_UNSUPPORTED, "rp_evaluate_host_noalloc: the domains need " + std::to_string(need) +
                                                 " staging floats, the fixed array holds " +
                                                 std::to_string(kNoAllocFloats));
    float *stage = ctx->noalloc_stage;   // looked up at rp_finalize
    if (!stage) return fail(ctx, RP_ERR_STATE, "rp_evaluate_host_noalloc: staging array not set up");
    // every staged value is written by the evaluation before it is copied out,
    // so nothing left from an earlier call needs clearing
    float *phi[kMaxDomains], *A[kMaxDomains];
    long long off = 0;
    for (int d = 0; d < nd; ++d) {
        phi[d] = stage + off;
        A[d] = stage + off + ctx->doms[d].N;
        off += 4 * ctx->doms[d].N;
    }
    if ((st = rp_evaluate(ctx, phi, A))) return st;
    for (int d = 0; d < nd; ++d) {
        const long long N = ctx->doms[d].N;
        RP_CUDA(ctx, cudaMemcpyAsync(h_phi[d], phi[d], N * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
        RP_CUDA(ctx, cudaMemcpyAsync(h_A[d], A[d], 3 * N * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
    }
    return RP_OK;
}

rp_status rp_gemm_tn(const void *d_A, const void *d_B, float *d_D, int M, int N, int K, int dtype, int terms,
                     int splits, int device, void *stream)
{
    if (!d_A || !d_B || !d_D || M <= 0 || N <= 0 || K <= 0 || M % 128 || K % 64 || N % 32 || N > 4096 ||
        (dtype != RP_DTYPE_BF16 && dtype != RP_DTYPE_FP16) ||
        (terms != 1 && terms != 3) || splits < 0 || splits > 4096 || (reinterpret_cast<uintptr_t>(d_D) & 15) ||
        (reinterpret_cast<uintptr_t>(d_A) & 15) || (reinterpret_cast<uintptr_t>(d_B) & 15))
        return RP_ERR_ARG;
    if (cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        return RP_ERR_CUDA;
    }
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn) {
        cudaGetLastError();
        return RP_ERR_CUDA;
    }
    const int width = terms == 3 ? 2 * K : K;
    CUtensorMap ma, mb;
    if (!encode_bf16_rows(fn, &ma, d_A, (uint64_t)M, (uint64_t)width, 128) ||
        !encode_bf16_rows(fn, &mb, d_B, (uint64_t)N, (uint64_t)width, (uint32_t)gemm_tile_n(N)))
        return RP_ERR_ARG;
    int optin = 0, sms = 0;
    int *d_err = nullptr;
    float *work = nullptr;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
        cudaGetLastError();
        return RP_ERR_CUDA;
    }
    if (splits == 0) splits = gemm_splits(M, K, terms == 3, sms, 16);
    if (cudaMalloc(&d_err, sizeof(int)) != cudaSuccess || cudaMemsetAsync(d_err, 0, sizeof(int), s) != cudaSuccess ||
        (splits > 1 && cudaMalloc(&work, (size_t)splits * M * N * sizeof(float)) != cudaSuccess)) {
        cudaGetLastError();
        if (d_err) cudaFree(d_err);
        return RP_ERR_CUDA;
    }
    int flag = 0;
    cudaError_t e = launch_gemm_bf16_tn(ma, mb, d_D, M, N, K, N, optin, d_err, s, splits, work, terms == 3,
                                        dtype == RP_DTYPE_FP16);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaMemcpy(&flag, d_err, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(d_err);
    if (work) cudaFree(work);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return RP_ERR_CUDA;
    }
    return flag ? RP_ERR_TIMEOUT : RP_OK;
}

rp_status rp_gemm_bf16(const void *d_A, const void *d_B, float *d_D, int M, int N, int K, int device, void *stream)
{
    if (N > 256) return RP_ERR_ARG;
    return rp_gemm_tn(d_A, d_B, d_D, M, N, K, RP_DTYPE_BF16, 1, 1, device, stream);
}

rp_status rp_train_far_model(rp_ctx *ctx, const rp_train_config *cfg_in, rp_train_report *rep)
{
    if (!ctx || !cfg_in) return RP_ERR_ARG;
    if (!ctx->finalized || ctx->plan_only || ctx->trained || ctx->step >= 0 || ctx->npushed)
        return fail(ctx, RP_ERR_STATE, "rp_train_far_model: call once, after rp_finalize and before the first push");
    if (ctx->cfg.mode != RP_MODE_LOWRANK) return fail(ctx, RP_ERR_UNSUPPORTED, "the learned far field needs RP_MODE_LOWRANK");
    rp_train_config cfg = *cfg_in;
    if (!(cfg.learned_distance > 0.0) || cfg.gate < 0.0 || cfg.histories < 0 || cfg.samples < 0 ||
        cfg.iterations < 0 || cfg.batch < 0 || cfg.batch % 128 || cfg.lr < 0.0f || cfg.validation < 0)
        return fail(ctx, RP_ERR_ARG, "rp_train_far_model: bad configuration");
    if (cfg.gate == 0.0) cfg.gate = 5e-4;
    if (!cfg.histories) cfg.histories = 512;
    if (!cfg.samples) cfg.samples = 32;
    if (!cfg.iterations) cfg.iterations = 3000;
    if (!cfg.batch) cfg.batch = 1024;
    if (cfg.lr == 0.0f) cfg.lr = 1e-3f;
    if (!cfg.validation) cfg.validation = 4;
    rp_train_report report{};
    rp_status st = use_device(ctx);
    if (st) return st;
    const int nd = (int)ctx->doms.size();
    const double c = ctx->cfg.c, dt = ctx->cfg.dt;
    // candidates
    std::vector<std::pair<int, int>> cand;
    for (int t = 0; t < nd; ++t)
        for (int s = 0; s < nd; ++s) {
            const PairPlan &p = ctx->pairs[(size_t)t * nd + s];
            if (p.kind == RP_PAIR_LOWRANK && p.rmin >= cfg.learned_distance) cand.push_back({t, s});
        }
    report.candidates = (int)cand.size();
    ctx->trained = true;
    if (cand.empty()) {
        if (ctx->cfg.flags & RP_FLAG_DEFER_FAR) {
            if ((st = build_far(ctx, ctx->smem_optin))) return st;
            RP_CUDA(ctx, cudaMemcpy(ctx->d_fwd, ctx->fwd.data(), ctx->fwd.size() * sizeof(FwdRing),
                                    cudaMemcpyHostToDevice));
            if ((st = build_mix(ctx))) return st;
            RP_CUDA(ctx, cudaMemcpy(ctx->d_inv, ctx->inv.data(), ctx->inv.size() * sizeof(InvTarget),
                                    cudaMemcpyHostToDevice));
        }
        if (rep) *rep = report;
        return RP_OK;
    }
    auto same = [](const DomainDesc &a, const DomainDesc &b) {
        return a.n[0] == b.n[0] && a.n[1] == b.n[1] && a.n[2] == b.n[2] && a.h == b.h;
    };
    const DomainDesc &S0 = ctx->doms[cand[0].second], &T0 = ctx->doms[cand[0].first];
    LGeom geo{};
    for (int a = 0; a < 3; ++a) geo.n_s[a] = S0.n[a];
    geo.h_s = S0.h;
    box_extent(T0, geo.Lt);
    geo.random = true;
    std::vector<std::pair<int, int>> elig;
    std::vector<double> dist;
    for (auto [t, s] : cand) {
        if (!same(ctx->doms[s], S0) || !same(ctx->doms[t], T0)) continue;
        double ct[3], cs[3];
        box_centre(ctx->doms[t], ct);
        box_centre(ctx->doms[s], cs);
        elig.push_back({t, s});
        dist.push_back(std::sqrt((ct[0] - cs[0]) * (ct[0] - cs[0]) + (ct[1] - cs[1]) * (ct[1] - cs[1]) +
                                 (ct[2] - cs[2]) * (ct[2] - cs[2])));
    }
    geo.R_lo = 0.9 * *std::min_element(dist.begin(), dist.end());
    geo.R_hi = 1.1 * *std::max_element(dist.begin(), dist.end());
    const int samples = std::min(cfg.samples, max_samples(geo, c * dt));
    if (samples < 1) return fail(ctx, RP_ERR_UNSUPPORTED, "boxes too large for the learned path's delay tables");
    void *enc = tensor_encoder();
    if (!enc) return fail(ctx, RP_ERR_UNSUPPORTED, "learned path needs cuTensorMapEncodeTiled");
    const auto t_start = std::chrono::steady_clock::now();
    const long long rows = (long long)cfg.histories * samples * 4;
    const long long vrows = (long long)cfg.validation * samples * 4;
    __half *X = nullptr, *VX = nullptr;
    float *Y = nullptr, *VY = nullptr, *Xf = nullptr, *VXf = nullptr, *Yres = nullptr;
    Mlp tnet;
    std::vector<float> weights(mlp_weight_count()), wlin((size_t)kLOut * kLIn);
    std::vector<double> verr, verr_lin;
    cudaError_t e = cudaMalloc(&X, rows * kLIn * sizeof(__half));
    if (!e) e = cudaMalloc(&Xf, rows * kLIn * sizeof(float));
    if (!e) e = cudaMalloc(&Y, rows * kLOut * sizeof(float));
    if (!e) e = cudaMalloc(&Yres, rows * kLOut * sizeof(float));
    if (!e) e = cudaMalloc(&VX, vrows * kLIn * sizeof(__half));
    if (!e) e = cudaMalloc(&VXf, vrows * kLIn * sizeof(float));
    if (!e) e = cudaMalloc(&VY, vrows * kLOut * sizeof(float));
    if (!e) e = learned_dataset(geo, cfg.seed, cfg.histories, samples, c, dt, X, Xf, Y, ctx->stream);
    if (!e) e = mlp_create(tnet, cfg.batch, cfg.seed ^ 0xA5A5A5A5ull, enc);
    if (!e) e = mlp_zero_last(tnet, ctx->stream);
    if (!e) e = learned_fit_linear(tnet, Xf, Y, (int)rows, Yres, ctx->stream);
    float loss = 0.0f;
    if (!e) e = learned_train(tnet, X, Yres, (int)rows, cfg.iterations, cfg.batch, cfg.lr, cfg.seed, ctx->smem_optin,
                              ctx->sm_count, ctx->stream, &loss);
    report.train_seconds = std::chrono::duration<float>(std::chrono::steady_clock::now() - t_start).count();
    report.train_rows = rows;
    report.final_loss = loss;
    // validation in each candidate's own geometry
    for (size_t i = 0; i < elig.size() && !e; ++i) {
        const auto [t, s] = elig[i];
        LGeom vg = geo;
        vg.random = false;
        double ct[3], cs[3];
        box_centre(ctx->doms[t], ct);
        box_centre(ctx->doms[s], cs);
        for (int a = 0; a < 3; ++a) vg.dir[a] = (ct[a] - cs[a]) / dist[i];
        vg.Rc = dist[i];
        // validated at the target's own far-path nodes (the canonical values
        // carried there as evaluation does), so that the re-interpolation's
        // error is part of what the gate judges
        std::vector<double> ax[3];
        std::vector<float> Lw;
        const DomainDesc &TD = ctx->doms[t];
        for (int a = 0; a < 3; ++a) far_axis(TD.o[a], TD.h, TD.n[a], ctx->cfg.far_points, ax[a], Lw);
        double lnodes[kLOut][3];
        std::vector<float> Pm, Ra(kLOut), Dn(kLOut);
        NodeMap nm{};
        const bool at_nodes = ax[0].size() * ax[1].size() * ax[2].size() == (size_t)kLOut;
        if (at_nodes) {
            int b = 0;
            for (size_t kz = 0; kz < ax[2].size(); ++kz)
                for (size_t ky = 0; ky < ax[1].size(); ++ky)
                    for (size_t kx = 0; kx < ax[0].size(); ++kx, ++b) {
                        lnodes[b][0] = ax[0][kx] - ct[0];
                        lnodes[b][1] = ax[1][ky] - ct[1];
                        lnodes[b][2] = ax[2][kz] - ct[2];
                    }
            double Rr[9], cn[kLOut][3];
            canonical_frame(vg.dir, Rr);
            canonical_nodes(geo.Lt, cn);
            reinterp_matrix(geo.Lt, Rr, ct, ax, Pm);
            for (int a = 0; a < kLOut; ++a) {
                double ra = 0.0, dn = 0.0;
                for (int k = 0; k < 3; ++k) {
                    const double x = dist[i] * vg.dir[k] + Rr[k] * cn[a][0] + Rr[3 + k] * cn[a][1] + Rr[6 + k] * cn[a][2];
                    const double y = dist[i] * vg.dir[k] + lnodes[a][k];
                    ra += x * x;
                    dn += y * y;
                }
                Ra[a] = (float)std::sqrt(ra);
                Dn[a] = (float)std::sqrt(dn);
            }
            vg.label_nodes = lnodes;
            nm = NodeMap{Pm.data(), Ra.data(), Dn.data()};
        }
        double err[4] = {}, errl[4] = {};
        e = learned_dataset(vg, cfg.seed + 7919ull * (i + 1), cfg.validation, samples, c, dt, VX, VXf, VY,
                            ctx->stream);
        if (!e) e = learned_eval(tnet, VX, VXf, VY, (int)vrows, ctx->smem_optin, ctx->sm_count, ctx->stream, err, errl,
                                 at_nodes ? &nm : nullptr);
        verr.push_back(std::max(std::max(err[0], err[1]), std::max(err[2], err[3])));
        verr_lin.push_back(std::max(std::max(errl[0], errl[1]), std::max(errl[2], errl[3])));
    }
    if (!e) e = cudaMemcpy(wlin.data(), tnet.Wlin, wlin.size() * sizeof(float), cudaMemcpyDeviceToHost);
    const float out_scale = tnet.out_scale;
    if (!e) e = mlp_get_weights(tnet, weights.data(), ctx->stream);
    int flag = 0;
    if (!e) e = cudaMemcpy(&flag, tnet.d_err, sizeof(int), cudaMemcpyDeviceToHost);
    mlp_destroy(tnet);
    cudaFree(X); cudaFree(Xf); cudaFree(Y); cudaFree(Yres); cudaFree(VX); cudaFree(VXf); cudaFree(VY);
    if (e) return cuda_fail(ctx, e, "learned far field training");
    if (flag) return fail(ctx, RP_ERR_TIMEOUT, "a bounded device wait ran out during training");
    double vsum = 0.0, lsum = 0.0;
    report.val_max = 0.0;
    report.val_linear_max = 0.0;
    ctx->net_pair.assign((size_t)nd * nd, 0);
    for (size_t i = 0; i < elig.size(); ++i) {
        report.val_max = std::max(report.val_max, verr[i]);
        report.val_linear_max = std::max(report.val_linear_max, verr_lin[i]);
        vsum += verr[i];
        lsum += verr_lin[i];
        // the network is used for a pair only where it lowers that pair's
        // validation error; the gate judges the better of the two
        const bool use = verr[i] < verr_lin[i];
        if (std::min(verr[i], verr_lin[i]) <= cfg.gate) {
            const size_t k = (size_t)elig[i].first * nd + elig[i].second;
            ctx->pairs[k].kind = RP_PAIR_LEARNED;
            ctx->net_pair[k] = use ? 1 : 0;
            ++report.learned;
            report.network_pairs += use ? 1 : 0;
        }
    }
    report.val_mean = elig.empty() ? 0.0 : vsum / (double)elig.size();
    report.val_linear_mean = elig.empty() ? 0.0 : lsum / (double)elig.size();
    if (report.learned || (ctx->cfg.flags & RP_FLAG_DEFER_FAR)) {
        clear_far(ctx);
        if ((st = build_far(ctx, ctx->smem_optin))) return st;
        if ((st = build_learned(ctx, weights, wlin, out_scale))) return st;
        ctx->net.out_scale = out_scale;
        RP_CUDA(ctx, cudaMemcpy(ctx->d_fwd, ctx->fwd.data(), ctx->fwd.size() * sizeof(FwdRing), cudaMemcpyHostToDevice));
        RP_CUDA(ctx, cudaMemcpy(ctx->d_inv, ctx->inv.data(), ctx->inv.size() * sizeof(InvTarget), cudaMemcpyHostToDevice));
        if ((st = build_mix(ctx))) return st;
    }
    if (rep) *rep = report;
    return RP_OK;
}

rp_status rp_fields(rp_ctx *ctx, int id, const float *d_phi, const float *d_A, const float *d_A1,
                    const float *d_A2, float *d_E, float *d_B)
{
    rp_status st = check_ready(ctx);
    if (st) return st;
    if (id < 0 || id >= (int)ctx->doms.size() || !d_phi || !d_A || !d_A1 || !d_E)
        return fail(ctx, RP_ERR_ARG, "rp_fields: bad id or NULL pointer");
    const DomainDesc &D = ctx->doms[id];
    if (D.n[0] < 3 || D.n[1] < 3 || D.n[2] < 3) return fail(ctx, RP_ERR_ARG, "rp_fields: an axis has fewer than 3 nodes");
    RP_CUDA(ctx, launch_fields(D.n[0], D.n[1], D.n[2], D.h, ctx->cfg.c, ctx->cfg.dt, d_phi, d_A, d_A1, d_A2, d_E, d_B,
                               ctx->stream));
    return RP_OK;
}

rp_status rp_graph_capture(rp_ctx *ctx, const float *const *d_rho, const float *const *d_J,
                           float *const *d_phi, float *const *d_A)
{
    rp_status st = check_ready(ctx);
    if (st) return st;
    const int nd = (int)ctx->doms.size();
    if (!d_rho || !d_J || !d_phi || !d_A) return fail(ctx, RP_ERR_ARG, "rp_graph_capture: NULL pointer array");
    for (int d = 0; d < nd; ++d)
        if (!d_rho[d] || !d_J[d] || !d_phi[d] || !d_A[d]) return fail(ctx, RP_ERR_ARG, "rp_graph_capture: NULL buffer");
    // the one-sided factors' launches and the learned field's change from step
    // to step; the two-sided factors' kernels read the step on the device
    if (ctx->profile || ctx->split || ctx->overlap || !ctx->far_src.empty() || (!ctx->far_tgt.empty() && !ctx->far2) ||
        !ctx->lpairs.empty() || (ctx->cfg.flags & RP_FLAG_DEFER_FAR) || !ctx->spill_srcs.empty())
        return fail(ctx, RP_ERR_UNSUPPORTED,
                    "rp_graph_capture: FFT, direct and two-sided far pairs only, without profiling, split or history "
                    "spill");
    if (ctx->step >= 0 && ctx->npushed != nd) return fail(ctx, RP_ERR_STATE, "rp_graph_capture inside a partially pushed step");
    if (ctx->graph_exec) { cudaGraphExecDestroy(ctx->graph_exec); ctx->graph_exec = nullptr; }
    if (ctx->graph) { cudaGraphDestroy(ctx->graph); ctx->graph = nullptr; }
    if (!ctx->h_step_pin) RP_CUDA(ctx, cudaHostAlloc(&ctx->h_step_pin, sizeof(long long), cudaHostAllocDefault));
    // record with the host state of a step; the replays keep it themselves
    const long long step0 = ctx->step;
    const int npushed0 = ctx->npushed;
    const std::vector<char> pushed0 = ctx->pushed;
    if (!ctx->capture_stream) RP_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking));
    cudaStream_t user_stream = ctx->stream;
    RP_CUDA(ctx, cudaStreamBeginCapture(ctx->capture_stream, cudaStreamCaptureModeThreadLocal));
    ctx->stream = ctx->capture_stream;   // every launch of the step goes into the recording
    ctx->capturing = true;
    cudaError_t e = launch_step_advance(ctx->d_step, ctx->stream);
    if (!e && !(st = rp_push_all(ctx, d_rho, d_J))) st = rp_evaluate(ctx, d_phi, d_A);
    ctx->capturing = false;
    ctx->stream = user_stream;
    cudaGraph_t g = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(ctx->capture_stream, &g);
    ctx->step = step0;
    ctx->npushed = npushed0;
    ctx->pushed = pushed0;
    if (e || st || e2 || !g) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        if (st) return st;
        return cuda_fail(ctx, e ? e : (e2 ? e2 : cudaErrorStreamCaptureInvalidated), "graph capture");
    }
    ctx->graph = g;
    RP_CUDA(ctx, cudaGraphInstantiate(&ctx->graph_exec, g, 0));
    ctx->graph_synced = -2;   // the first replay sets the device counter
    return RP_OK;
}

rp_status rp_graph_step(rp_ctx *ctx)
{
    rp_status st = check_ready(ctx);
    if (st) return st;
    const int nd = (int)ctx->doms.size();
    if (!ctx->graph_exec) return fail(ctx, RP_ERR_STATE, "rp_graph_step before rp_graph_capture");
    if (ctx->step >= 0 && ctx->npushed != nd) return fail(ctx, RP_ERR_STATE, "rp_graph_step inside a partially pushed step");
    const long long next = ctx->step + 1;
    if (!ctx->clamp && next - ctx->max_lag < 0)
        return fail(ctx, RP_ERR_HISTORY, "step " + std::to_string(next) + " needs samples " +
                                             std::to_string(ctx->max_lag) + " steps back");
    if (ctx->graph_synced != ctx->step) {
        // the counter holds the step of the last replay: set it to this one
        RP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        *ctx->h_step_pin = ctx->step;
        RP_CUDA(ctx, cudaMemcpyAsync(ctx->d_step, ctx->h_step_pin, sizeof(long long), cudaMemcpyHostToDevice,
                                     ctx->stream));
    }
    RP_CUDA(ctx, cudaGraphLaunch(ctx->graph_exec, ctx->stream));
    ctx->step = next;
    ctx->npushed = nd;
    std::fill(ctx->pushed.begin(), ctx->pushed.end(), 1);
    ctx->graph_synced = next;
    return RP_OK;
}

rp_status rp_selftest_wait(rp_ctx *ctx, long long limit_cycles)
{
    rp_status st = check_ready(ctx);
    if (st) return st;
    if (limit_cycles < 1 || limit_cycles > 4000000000LL) return fail(ctx, RP_ERR_ARG, "rp_selftest_wait: limit out of range");
    RP_CUDA(ctx, launch_wait_selftest(limit_cycles, ctx->d_err, ctx->stream));
    return RP_OK;
}

rp_status rp_sync(rp_ctx *ctx)
{
    if (!ctx) return RP_ERR_ARG;
    if (ctx->plan_only) return RP_OK;
    rp_status st = use_device(ctx);
    if (st) return st;
    RP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (ctx->push_stream) RP_CUDA(ctx, cudaStreamSynchronize(ctx->push_stream));
    if (ctx->copy_in) RP_CUDA(ctx, cudaStreamSynchronize(ctx->copy_in));
    if (ctx->copy_out) RP_CUDA(ctx, cudaStreamSynchronize(ctx->copy_out));
    if (ctx->spill_out) RP_CUDA(ctx, cudaStreamSynchronize(ctx->spill_out));
    if (ctx->spill_in) RP_CUDA(ctx, cudaStreamSynchronize(ctx->spill_in));
    RP_CUDA(ctx, cudaGetLastError());
    if (ctx->d_err) {
        int flag = 0;
        RP_CUDA(ctx, cudaMemcpy(&flag, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost));
        if (flag) {
            RP_CUDA(ctx, cudaMemset(ctx->d_err, 0, sizeof(int)));
            return fail(ctx, RP_ERR_TIMEOUT, "a bounded device wait ran out; results of the affected steps are invalid");
        }
    }
    return RP_OK;
}

rp_status rp_query(rp_ctx *ctx, rp_stats *out)
{
    if (!ctx || !out) return RP_ERR_ARG;
    if (!ctx->finalized) return fail(ctx, RP_ERR_STATE, "rp_query before rp_finalize");
    std::memset(out, 0, sizeof(*out));
    const int nd = (int)ctx->doms.size();
    out->ndomains = nd;
    out->max_lag = ctx->max_lag;
    out->raw_depth = ctx->raw_depth;
    out->spectral_depth = ctx->spec_depth;
    out->step = ctx->step;
    out->device_bytes = ctx->device_bytes;
    out->spectral_bytes = ctx->spectral_bytes;
    out->kernel_bytes = ctx->kernel_bytes;
    for (const DomainDesc &d : ctx->doms) out->points += d.N;
    out->mac_tma = ctx->tma ? 1 : 0;
    out->npairs_far = ctx->npairs_far;
    out->far_bytes = ctx->far_bytes;
    out->npairs_learned = ctx->npairs_learned;
    out->spill_windows = (int)ctx->spill_wins.size();
    out->host_bytes = ctx->host_bytes;
    out->audit_rel_l2 = ctx->audit_rel_l2;
    out->audit_step = ctx->audit_step;
    out->owned_sources = ctx->n_owned;
    for (const PairPlan &p : ctx->pairs) out->npairs_other += p.kind == RP_PAIR_OTHER;
    out->mac_warps = 0;
    for (const LaunchGroup &g : ctx->inv_groups)
        if (g.cls > 0 && ctx->tma) out->mac_warps = ctx->mac_cw[class_slot(g.cls)];
    out->npairs_direct = 0;
    out->npairs_fft = 0;
    for (const PairPlan &p : ctx->pairs) {
        if (p.kind == RP_PAIR_FFT) out->npairs_fft++;
        else if (p.kind == RP_PAIR_DIRECT) out->npairs_direct++;
    }
    return RP_OK;
}

rp_status rp_pair_info(rp_ctx *ctx, int target, int source, rp_pair_info_t *out)
{
    if (!ctx || !out) return RP_ERR_ARG;
    if (!ctx->finalized) return fail(ctx, RP_ERR_STATE, "rp_pair_info before rp_finalize");
    const int nd = (int)ctx->doms.size();
    if (target < 0 || target >= nd || source < 0 || source >= nd) return fail(ctx, RP_ERR_ARG, "rp_pair_info: bad domain");
    const PairPlan &p = ctx->pairs[(size_t)target * nd + source];
    std::memset(out, 0, sizeof(*out));
    out->kind = p.kind;
    out->lag_lo = p.lag_lo;
    out->lag_hi = p.lag_hi;
    for (int a = 0; a < 3; ++a) out->fft_m[a] = p.kind == RP_PAIR_FFT ? p.m[a] : 0;
    out->r_min = p.rmin;
    out->r_max = p.rmax;
    return RP_OK;
}

rp_status rp_kernel_stats(rp_ctx *ctx, int kind, long long *launches, double *total_ms, int reset)
{
    if (!ctx || kind < 0 || kind >= RP_K_COUNT) return RP_ERR_ARG;
    if (ctx->plan_only) return fail(ctx, RP_ERR_STATE, "plan-only context");
    rp_status st = use_device(ctx);
    if (st) return st;
    if ((st = drain_profile(ctx))) return st;
    if (launches) *launches = ctx->launches[kind];
    if (total_ms) *total_ms = ctx->ms[kind];
    if (reset) {
        for (int k = 0; k < RP_K_COUNT; ++k) { ctx->launches[k] = 0; ctx->ms[k] = 0.0; ctx->count[k] = 0; }
    }
    return RP_OK;
}

rp_status rp_kernel_count(rp_ctx *ctx, int kind, long long *launches)
{
    if (!ctx || kind < 0 || kind >= RP_K_COUNT || !launches) return RP_ERR_ARG;
    *launches = ctx->count[kind];
    return RP_OK;
}

rp_status rp_set_profiling(rp_ctx *ctx, int every)
{
    if (!ctx || every < 0) return RP_ERR_ARG;
    if (ctx->plan_only) return fail(ctx, RP_ERR_STATE, "plan-only context");
    ctx->profile = every > 0;
    ctx->cfg.profile_every = every;
    return RP_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- checkpoint

namespace {

const char kMagic[8] = {'R', 'P', 'S', 'T', 'A', 'T', 'E', '1'};

// A hash of everything that must match between save and load.
unsigned long long layout_hash(const rp_ctx *ctx)
{
    unsigned long long h = 1469598103934665603ULL;
    auto mix = [&](const void *p, size_t n) {
        const unsigned char *b = static_cast<const unsigned char *>(p);
        for (size_t i = 0; i < n; ++i) { h ^= b[i]; h *= 1099511628211ULL; }
    };
    for (const DomainDesc &d : ctx->doms) { mix(d.o, sizeof d.o); mix(d.n, sizeof d.n); mix(&d.h, sizeof d.h); }
    mix(&ctx->cfg.c, sizeof(double));
    mix(&ctx->cfg.dt, sizeof(double));
    mix(&ctx->cfg.mode, sizeof(int));
    mix(&ctx->split, sizeof(bool));
    for (const FwdRing &R : ctx->fwd) { mix(&R.depth, sizeof(int)); mix(&R.slot_elems, sizeof(long long)); }
    for (const RawRing &r : ctx->raw) { mix(&r.depth, sizeof(int)); mix(&r.n, sizeof(long long)); }
    for (const SpillSource &S : ctx->spill_srcs) mix(&S.dom, sizeof(int));
    mix(&ctx->spill_hd, sizeof(int));
    return h;
}

template <class Fn>
rp_status for_each_ring(rp_ctx *ctx, Fn &&fn)
{
    rp_status st;
    for (const RawRing &r : ctx->raw)
        if (r.ring && (st = fn((void *)r.ring, (size_t)r.depth * 4 * r.n * sizeof(float)))) return st;
    for (const FwdRing &R : ctx->fwd)
        if ((st = fn((void *)R.ring, (size_t)R.depth * R.slot_elems * sizeof(float2)))) return st;
    for (const FarSource &F : ctx->far_src)
        if ((st = fn((void *)F.X, (size_t)8 * ctx->cfg.far_batch * F.ks * sizeof(__nv_bfloat16)))) return st;
    for (const FarTarget &F : ctx->far_tgt)
        if ((st = fn((void *)F.cring, (size_t)F.depth * F.r * 4 * sizeof(float)))) return st;
    if (ctx->far2_qall &&
        (st = fn((void *)ctx->far2_qall,
                 (size_t)ctx->far2_srcs.size() * 2 * ctx->far2_D * 4 * 2 * ctx->far2_KS * sizeof(__nv_bfloat16))))
        return st;
    for (size_t d = 0; d < ctx->ground.size(); ++d) {
        const size_t bytes = 4 * (size_t)ctx->doms[d].N * sizeof(float);
        if ((st = fn((void *)ctx->ground[d], bytes)) || (st = fn((void *)ctx->pstatic[d], bytes))) return st;
    }
    // the spilled history: staged slices (device) and the host rings; the
    // windows are fetched again
    for (const SpillSource &S : ctx->spill_srcs) {
        const size_t bytes = 16 * (size_t)ctx->doms[S.dom].N;
        if ((st = fn((void *)S.stage, kSpillStage * bytes)) || (st = fn((void *)S.host, ctx->spill_hd * bytes))) return st;
    }
    return RP_OK;
}

}  // namespace

extern "C" {

rp_status rp_save_state(rp_ctx *ctx, const char *path)
{
    rp_status st = check_ready(ctx);
    if (st) return st;
    if (!path) return fail(ctx, RP_ERR_ARG, "NULL path");
    if (!ctx->lpairs.empty()) return fail(ctx, RP_ERR_UNSUPPORTED, "a context with learned pairs has no saved state");
    RP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (ctx->push_stream) RP_CUDA(ctx, cudaStreamSynchronize(ctx->push_stream));
    if (ctx->spill_out) RP_CUDA(ctx, cudaStreamSynchronize(ctx->spill_out));
    if (ctx->spill_in) RP_CUDA(ctx, cudaStreamSynchronize(ctx->spill_in));
    FILE *f = std::fopen(path, "wb");
    if (!f) return fail(ctx, RP_ERR_ARG, std::string("cannot open ") + path);
    const unsigned long long h = layout_hash(ctx);
    const int nd = (int)ctx->doms.size();
    bool ok = std::fwrite(kMagic, 1, 8, f) == 8 && std::fwrite(&h, sizeof h, 1, f) == 1 &&
              std::fwrite(&ctx->step, sizeof ctx->step, 1, f) == 1 &&
              std::fwrite(&ctx->npushed, sizeof ctx->npushed, 1, f) == 1 &&
              std::fwrite(ctx->pushed.data(), 1, nd, f) == (size_t)nd;
    std::vector<char> buf;
    if (ok)
        st = for_each_ring(ctx, [&](void *dptr, size_t bytes) -> rp_status {
            buf.resize(bytes);
            RP_CUDA(ctx, cudaMemcpy(buf.data(), dptr, bytes, cudaMemcpyDefault));   // device or pinned host
            if (std::fwrite(buf.data(), 1, bytes, f) != bytes) return fail(ctx, RP_ERR_ARG, "write failed");
            return RP_OK;
        });
    std::fclose(f);
    if (!ok) return fail(ctx, RP_ERR_ARG, "write failed");
    return st;
}

rp_status rp_load_state(rp_ctx *ctx, const char *path)
{
    rp_status st = check_ready(ctx);
    if (st) return st;
    if (!path) return fail(ctx, RP_ERR_ARG, "NULL path");
    FILE *f = std::fopen(path, "rb");
    if (!f) return fail(ctx, RP_ERR_ARG, std::string("cannot open ") + path);
    char magic[8];
    unsigned long long h = 0;
    long long step = 0;
    int npushed = 0;
    const int nd = (int)ctx->doms.size();
    std::vector<char> pushed(nd);
    bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, kMagic, 8) == 0 &&
              std::fread(&h, sizeof h, 1, f) == 1 && std::fread(&step, sizeof step, 1, f) == 1 &&
              std::fread(&npushed, sizeof npushed, 1, f) == 1 &&
              std::fread(pushed.data(), 1, nd, f) == (size_t)nd;
    if (!ok || h != layout_hash(ctx)) {
        std::fclose(f);
        return fail(ctx, RP_ERR_STATE, "state file does not match this context");
    }
    RP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (ctx->push_stream) RP_CUDA(ctx, cudaStreamSynchronize(ctx->push_stream));
    if (ctx->spill_out) RP_CUDA(ctx, cudaStreamSynchronize(ctx->spill_out));
    if (ctx->spill_in) RP_CUDA(ctx, cudaStreamSynchronize(ctx->spill_in));
    std::vector<char> buf;
    st = for_each_ring(ctx, [&](void *dptr, size_t bytes) -> rp_status {
        buf.resize(bytes);
        if (std::fread(buf.data(), 1, bytes, f) != bytes) return fail(ctx, RP_ERR_STATE, "state file truncated");
        RP_CUDA(ctx, cudaMemcpy(dptr, buf.data(), bytes, cudaMemcpyDefault));   // device or pinned host
        return RP_OK;
    });
    std::fclose(f);
    if (st) return st;
    for (SpillWindow &W : ctx->spill_wins) W.have = W.raw_step[0] = W.raw_step[1] = -1;
    ctx->step = step;
    ctx->npushed = npushed;
    ctx->static_done = step > 0 || (step == 0 && npushed == nd);   // P(0) came with the state
    ctx->pushed = pushed;
    return RP_OK;
}

void rp_destroy(rp_ctx *ctx)
{
    if (!ctx) return;
    if (!ctx->plan_only && ctx->device >= 0) {
        int cur = -1;
        cudaGetDevice(&cur);
        cudaSetDevice(ctx->device);
        cudaStreamSynchronize(ctx->stream);
        if (ctx->push_stream) {
            cudaStreamSynchronize(ctx->push_stream);
            cudaStreamDestroy(ctx->push_stream);
            for (cudaEvent_t e : {ctx->ev_pushed, ctx->ev_stream, ctx->ev_eval[0], ctx->ev_eval[1]})
                if (e) cudaEventDestroy(e);
        }
        if (ctx->graph_exec) cudaGraphExecDestroy(ctx->graph_exec);
        if (ctx->graph) cudaGraphDestroy(ctx->graph);
        if (ctx->h_step_pin) cudaFreeHost(ctx->h_step_pin);
        if (ctx->capture_stream) cudaStreamDestroy(ctx->capture_stream);
        if (ctx->copy_in) {
            cudaStreamSynchronize(ctx->copy_in);
            cudaStreamSynchronize(ctx->copy_out);
            for (cudaEvent_t e : {ctx->in_ready, ctx->out_ready, ctx->out_free[0], ctx->out_free[1], ctx->in_free[0],
                                  ctx->in_free[1]})
                if (e) cudaEventDestroy(e);
            cudaStreamDestroy(ctx->copy_in);
            cudaStreamDestroy(ctx->copy_out);
        }
        if (ctx->spill_out) {
            cudaStreamSynchronize(ctx->spill_out);
            cudaStreamSynchronize(ctx->spill_in);
            for (cudaEvent_t e : ctx->sp_out) if (e) cudaEventDestroy(e);
            for (cudaEvent_t e : {ctx->sp_pushed, ctx->sp_in, ctx->sp_wfft})
                if (e) cudaEventDestroy(e);
            cudaStreamDestroy(ctx->spill_out);
            if (ctx->spill_in) cudaStreamDestroy(ctx->spill_in);
        }
        for (const SpillSource &S : ctx->spill_srcs) if (S.host) cudaFreeHost(S.host);
        for (const ProfRec &r : ctx->pending) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
        for (cudaEvent_t e : ctx->spare_events) cudaEventDestroy(e);
        for (void *p : ctx->allocs) cudaFree(p);
        for (void *p : ctx->far_allocs) cudaFree(p);
        if (ctx->net_open) {
            if (ctx->net.d_err == ctx->d_err) ctx->net.d_err = nullptr;
            mlp_destroy(ctx->net);
        }
        cudaGetLastError();
        if (cur >= 0) cudaSetDevice(cur);
    }
    delete ctx;
}

}  // extern "C"
