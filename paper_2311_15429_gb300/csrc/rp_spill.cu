// History spill to host memory (RP_FLAG_HISTORY_SPILL).  Sec. IV keeps every
// sample of the window [l - N_R,max, l] for the steps to come, while a step
// reads only each pair's Delta N_R of them.  A pair whose lag window starts
// far back reads its source spectra from a small device window ring; the
// source's (rho, J) slices go to a pinned host ring and come back one a
// step, through the same forward passes as a push (in the push's own
// launches in the steady state).  Two copy streams carry the copies, ordered
// against the kernels by events.
#include <algorithm>
#include <cstring>
#include <vector>

#include "rp_ctx.h"

namespace rp {

// History spill: the staging and window rings (device, zeroed), the pinned
// host rings, the window descriptors (after the forward rings' buffers), the
// two copy streams and their events.
rp_status open_spill(rp_ctx *ctx)
{
    if (ctx->spill_srcs.empty()) return RP_OK;
    rp_status st;
    for (SpillSource &S : ctx->spill_srcs) {
        const size_t n4 = 4 * (size_t)ctx->doms[S.dom].N;
        if ((st = dev_alloc(ctx, &S.stage, kSpillStage * n4))) return st;
        RP_CUDA(ctx, cudaMemset(S.stage, 0, kSpillStage * n4 * sizeof(float)));
        void *p = nullptr;
        RP_CUDA(ctx, cudaHostAlloc(&p, (size_t)ctx->spill_hd * n4 * sizeof(float), cudaHostAllocDefault));
        S.host = static_cast<float *>(p);
        std::memset(p, 0, (size_t)ctx->spill_hd * n4 * sizeof(float));
    }
    int plane0 = 0, tile0 = 0;
    for (SpillWindow &W : ctx->spill_wins) {
        const FwdRing &R = ctx->fwd[W.ring];
        const size_t elems = (size_t)W.depth * R.slot_elems;
        const size_t n4 = 4 * (size_t)ctx->doms[R.src].N;
        if ((st = dev_alloc(ctx, &W.dev, elems)) || (st = dev_alloc(ctx, &W.raw, 2 * n4))) return st;
        RP_CUDA(ctx, cudaMemset(W.dev, 0, elems * sizeof(float2)));
        FwdRing F = R;            // same sizes and twiddles
        F.src = (int)ctx->wfwd.size() % kMaxDomains;   // its input's slot in a launch's pointer table
        F.depth = W.depth;
        F.ring = W.dev;
        // its own scratch between the two passes: a push's launch may transform
        // the window beside the ring it copies
        if ((st = dev_alloc(ctx, &F.t1, 4ULL * F.kx * F.nz * F.ay.M))) return st;
        F.far_x = nullptr;
        F.far_ks = 0;
        F.plane0 = plane0;
        F.tile0 = tile0;
        plane0 += 4 * F.nz;
        tile0 += F.kx * ((F.ay.M + kTileY - 1) / kTileY);
        ctx->wfwd.push_back(F);
    }
    RP_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->spill_out, cudaStreamNonBlocking));
    RP_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->spill_in, cudaStreamNonBlocking));
    auto event = [](cudaEvent_t *e) { return cudaEventCreateWithFlags(e, cudaEventDisableTiming); };
    RP_CUDA(ctx, event(&ctx->sp_pushed));
    RP_CUDA(ctx, event(&ctx->sp_in));
    RP_CUDA(ctx, event(&ctx->sp_wfft));
    ctx->sp_out.assign(kSpillStage, nullptr);
    for (cudaEvent_t &e : ctx->sp_out) RP_CUDA(ctx, event(&e));
    return RP_OK;
}

// History spill: the merged descriptor table (rp_ctx::mix) from the current
// forward rings and windows, uploaded.  Called once the forward rings'
// descriptors are final, and again whenever they change (far factors built
// or rebuilt later).
rp_status build_mix(rp_ctx *ctx)
{
    const int nd = (int)ctx->doms.size(), nw = (int)ctx->spill_wins.size();
    ctx->mix.clear();
    ctx->mix_groups.clear();
    if (nw == 0 || nd + nw > kMaxDomains) return RP_OK;
    int p0 = 0, t0 = 0;
    for (const LaunchGroup &g : ctx->fwd_groups) {
        LaunchGroup m{g.cls, (int)ctx->mix.size(), 0, p0, 0, t0, 0};
        auto add = [&](FwdRing F) {
            F.plane0 = p0;
            F.tile0 = t0;
            F.d_step = ctx->d_step;
            p0 += 4 * F.nz;
            t0 += F.kx * ((F.ay.M + kTileY - 1) / kTileY);
            ctx->mix.push_back(F);
        };
        for (int r = g.i0; r < g.i1; ++r) add(ctx->fwd[r]);
        for (int w = 0; w < nw; ++w) {
            FwdRing F = ctx->wfwd[w];
            if (size_class(F.ax, F.ay, F.az) != g.cls) continue;
            F.src = nd + w;
            F.lag_off = ctx->spill_wins[w].lo;
            add(F);
        }
        m.i1 = (int)ctx->mix.size();
        m.blk1 = p0;
        m.blk2_1 = t0;
        ctx->mix_groups.push_back(m);
    }
    rp_status st;
    if (!ctx->d_mix && (st = dev_alloc(ctx, &ctx->d_mix, ctx->mix.size()))) return st;
    RP_CUDA(ctx, cudaMemcpy(ctx->d_mix, ctx->mix.data(), ctx->mix.size() * sizeof(FwdRing), cudaMemcpyHostToDevice));
    return RP_OK;
}

// History spill, once a round's pushes are queued: the round's staged slices
// of the spilled sources into their host rings (spill_out waits for the
// staging copies, and for the copies back from the host ring queued so far,
// the last readers of the host slot it overwrites).
rp_status spill_round_done(rp_ctx *ctx)
{
    if (ctx->spill_srcs.empty() || ctx->npushed != (int)ctx->doms.size()) return RP_OK;
    const long long l = ctx->step;
    RP_CUDA(ctx, cudaEventRecord(ctx->sp_pushed, ctx->stream));
    RP_CUDA(ctx, cudaStreamWaitEvent(ctx->spill_out, ctx->sp_pushed, 0));
    RP_CUDA(ctx, cudaStreamWaitEvent(ctx->spill_out, ctx->sp_in, 0));
    for (const SpillSource &S : ctx->spill_srcs) {
        const size_t n4 = 4 * (size_t)ctx->doms[S.dom].N;
        RP_CUDA(ctx, cudaMemcpyAsync(S.host + (size_t)(l % ctx->spill_hd) * n4, S.stage + (size_t)(l % kSpillStage) * n4,
                                     n4 * sizeof(float), cudaMemcpyDeviceToHost, ctx->spill_out));
    }
    RP_CUDA(ctx, cudaEventRecord(ctx->sp_out[l % kSpillStage], ctx->spill_out));
    return RP_OK;
}

// History spill: the host slice of step j into input buffer j % 2 of window
// W on spill_in (the caller has made spill_in wait for the copy out of j and
// for the buffer's last reader, and records sp_in after).
static rp_status spill_raw_in(rp_ctx *ctx, SpillWindow &W, long long j)
{
    const SpillSource &S = ctx->spill_srcs[W.ss];
    const size_t n4 = 4 * (size_t)ctx->doms[S.dom].N;
    RP_CUDA(ctx, cudaMemcpyAsync(W.raw + (size_t)(j & 1) * n4, S.host + (size_t)(j % ctx->spill_hd) * n4,
                                 n4 * sizeof(float), cudaMemcpyHostToDevice, ctx->spill_in));
    W.raw_step[j & 1] = j;
    return RP_OK;
}

// History spill: the forward passes of windows [w0, w1) (one size class,
// fewer than kMaxDomains of them), each on the slice of step j in its input
// buffer j % 2, into slot j % B of its ring.
static rp_status spill_transform(rp_ctx *ctx, int w0, int w1, long long j)
{
    rp_status st;
    IoPtrs in{};
    for (int w = w0; w < w1; ++w) {
        const SpillWindow &W = ctx->spill_wins[w];
        const long long Ns = ctx->doms[ctx->spill_srcs[W.ss].dom].N;
        const FwdRing &F = ctx->wfwd[w];
        in.rho[F.src] = W.raw + (size_t)(j & 1) * 4 * Ns;
        in.J[F.src] = in.rho[F.src] + Ns;
    }
    const FwdRing &F0 = ctx->wfwd[w0], &F1 = ctx->wfwd[w1 - 1];
    const int cls = size_class(F0.ax, F0.ay, F0.az);
    const int planes = F1.plane0 + 4 * F1.nz - F0.plane0;
    const int tiles = F1.tile0 + F1.kx * ((F1.ay.M + kTileY - 1) / kTileY) - F0.tile0;
    if ((st = timed_launch(ctx, RP_K_FWD_PLANE, "window forward plane pass", [&] {
             return launch_fwd_plane(cls, ctx->fwd_tile[class_slot(cls)], ctx->d_wfwd, in, w0, w1, F0.plane0, planes,
                                     ctx->smem_plane_cls[class_slot(cls)], 0, ctx->stream);
         })))
        return st;
    return timed_launch(ctx, RP_K_FWD_COLUMN, "window forward column pass", [&] {
        return launch_fwd_column(cls, ctx->d_wfwd, w0, w1, F0.tile0, tiles, ctx->smem_col, j, ctx->stream);
    });
}

// History spill, before the MAC of step l: every window must hold the
// spectra of source steps l - hi .. l - lo (clamped at 0 under
// RP_FLAG_GROUND_STATE_CLAMP).  Normally each window lacks only step l - lo,
// whose slice was fetched during the previous step: then one pair of forward
// passes per run of windows of one size class and one such step transforms
// them into the windows' rings, on the context stream where the MAC reads
// them (slot j % B held step j - B < l - hi, which this and later MACs do not
// read).  Otherwise (the first steps, skipped evaluations, a loaded state)
// the missing steps go one at a time: slice in, transform.  Then each
// window's slice for step l + 1 (j = l + 1 - lo <= l - 3, as a spilled window
// has lo >= 4) is fetched, after the copy out of step l - 1 and the last
// transform (the reader of its buffer), to arrive under this step's
// remaining kernels.
rp_status spill_fetch(rp_ctx *ctx)
{
    if (ctx->spill_srcs.empty()) return RP_OK;
    const long long l = ctx->step;
    const int nw = (int)ctx->spill_wins.size();
    rp_status st;
    std::vector<long long> next(nw, -1);   // the one step a window lacks, or -1
    bool steady = true;
    for (int w = 0; w < nw; ++w) {
        const SpillWindow &W = ctx->spill_wins[w];
        long long a = l - W.hi, b = l - W.lo;
        if (ctx->clamp) { a = std::max(a, 0LL); b = std::max(b, 0LL); }
        if (a < 0) return fail(ctx, RP_ERR_HISTORY, "spilled window before the first push");
        const long long from = std::max(a, W.have + 1);
        if (from > b) continue;
        if (from == b && W.raw_step[b & 1] == b) next[w] = b;
        else steady = false;
    }
    if (steady) {
        bool any = false;
        for (int w = 0; w < nw;) {
            if (next[w] < 0) { ++w; continue; }
            if (!any) RP_CUDA(ctx, cudaStreamWaitEvent(ctx->stream, ctx->sp_in, 0));
            any = true;
            const FwdRing &F = ctx->wfwd[w];
            const int cls = size_class(F.ax, F.ay, F.az);
            int w1 = w + 1;
            while (w1 < nw && w1 - w < kMaxDomains && next[w1] == next[w] &&
                   size_class(ctx->wfwd[w1].ax, ctx->wfwd[w1].ay, ctx->wfwd[w1].az) == cls)
                ++w1;
            if ((st = spill_transform(ctx, w, w1, next[w]))) return st;
            for (int v = w; v < w1; ++v) ctx->spill_wins[v].have = next[w];
            w = w1;
        }
        if (any) RP_CUDA(ctx, cudaEventRecord(ctx->sp_wfft, ctx->stream));
    } else {
        for (int w = 0; w < nw; ++w) {
            SpillWindow &W = ctx->spill_wins[w];
            long long a = l - W.hi, b = l - W.lo;
            if (ctx->clamp) { a = std::max(a, 0LL); b = std::max(b, 0LL); }
            for (long long j = std::max(a, W.have + 1); j <= b; ++j) {
                if (W.raw_step[j & 1] != j) {
                    RP_CUDA(ctx, cudaStreamWaitEvent(ctx->spill_in, ctx->sp_out[l % kSpillStage], 0));
                    RP_CUDA(ctx, cudaStreamWaitEvent(ctx->spill_in, ctx->sp_wfft, 0));
                    if ((st = spill_raw_in(ctx, W, j))) return st;
                    RP_CUDA(ctx, cudaEventRecord(ctx->sp_in, ctx->spill_in));
                }
                RP_CUDA(ctx, cudaStreamWaitEvent(ctx->stream, ctx->sp_in, 0));
                if ((st = spill_transform(ctx, w, w + 1, j))) return st;
                RP_CUDA(ctx, cudaEventRecord(ctx->sp_wfft, ctx->stream));
                W.have = j;
            }
        }
    }
    if (l < 1) return RP_OK;
    bool any = false;
    for (SpillWindow &W : ctx->spill_wins) {
        const long long j = l + 1 - W.lo;
        if (j < 0 || j != W.have + 1 || W.raw_step[j & 1] == j) continue;
        if (!any) {
            RP_CUDA(ctx, cudaStreamWaitEvent(ctx->spill_in, ctx->sp_out[(l - 1) % kSpillStage], 0));
            RP_CUDA(ctx, cudaStreamWaitEvent(ctx->spill_in, ctx->sp_wfft, 0));
        }
        any = true;
        if ((st = spill_raw_in(ctx, W, j))) return st;
    }
    if (any) RP_CUDA(ctx, cudaEventRecord(ctx->sp_in, ctx->spill_in));
    return RP_OK;
}

}  // namespace rp
