// The library's context (the opaque rp_ctx of the C-ABI), the plan types it
// holds, and the helpers every part of the library uses on it: error
// recording, device selection, allocation and timed launches; plus the entry
// points of the history spill (rp_spill.cu).
#pragma once

#include <algorithm>
#include <array>
#include <map>
#include <string>
#include <vector>

#include <cuda.h>
#include <cudaTypedefs.h>

#include "../../include/rp.h"
#include "rp_internal.h"
#include "rp_learned.h"
#include "rp_learned_data.h"
#include "rp_learned_train.h"

namespace rp {

struct DomainDesc {
    double o[3];
    int n[3];
    double h;
    long long N;
};

struct PairPlan {
    int kind;       // rp_pair_kind
    int lag_lo, lag_hi;
    double rmin, rmax;
    int m[3];       // FFT size of the target (FFT pairs)
};

struct ProfRec {
    int kind;
    cudaEvent_t a, b;
};

// One launch of a kernel pair over a contiguous range [i0, i1) of rings (or
// targets) of one size class: first kernel's blocks [blk0, blk1), second
// kernel's blocks [blk2_0, blk2_1).
// Index of a kernel size class (0: the run-time shape) in the per-class tables.
inline int class_slot(int cls)
{
    switch (cls) {
    case 32: return 1; case 48: return 2; case 64: return 3; case 96: return 4; case 128: return 5; case 192: return 6;
    default: return 0;
    }
}

struct LaunchGroup {
    int cls;
    int i0, i1;
    int blk0, blk1;
    int blk2_0, blk2_1;
};

// History spill (RP_FLAG_HISTORY_SPILL).  A source domain with a spilled
// pair: device staging of its last kSpillStage pushed slices and the pinned
// host ring of its history, [depth][4][N] float each.
struct SpillSource {
    int dom;
    float *stage;
    float *host;
};

// A spilled lag window [lo, hi] of one spectral ring: a device spectral ring
// of depth B = hi - lo + 1 holding the source spectra of steps j at slot
// j % B.  The forward passes make them (window descriptor w of the window
// ring table: the ring's sizes, this ring as output) from raw slices copied
// in from the host ring into one of two input buffers, by parity of j.
// `have`: the newest step transformed in (-1: none); raw_step: the step each
// input buffer holds.
struct SpillWindow {
    int ring, ss;            // forward ring, SpillSource
    int lo, hi, depth;
    float2 *dev;
    float *raw;              // [2][4][N of the source]
    long long have;
    long long raw_step[2];
};

constexpr int kSpillStage = 3;   // staging slots: a round's copy to the host has two more rounds to finish

// A pair's lag window is spilled when its window ring is at most half the
// ring depth it would otherwise need.
inline bool spill_window(int lo, int hi) { return lo >= 2 * (hi - lo + 2); }

}  // namespace rp

using namespace rp;   // the library's translation units work in namespace rp

struct rp_ctx {
    rp_config cfg{};
    int device = -1;
    cudaStream_t stream = nullptr;
    bool plan_only = false, clamp = false, profile = false;
    bool comp = true;    // Kahan-compensated spectral sums (off under RP_FLAG_PLAIN_SUM)
    // overlapped pushes (RP_FLAG_OVERLAP_PUSH): the push stream, "the last
    // push round is done" on it, and "the evaluation of step s is done" on the
    // context stream by parity of s (the push of step s + 2 waits for it)
    bool overlap = false;
    cudaStream_t push_stream = nullptr;
    cudaEvent_t ev_pushed = nullptr, ev_stream = nullptr;
    cudaEvent_t ev_eval[2] = {nullptr, nullptr};
    // ground-state split (RP_FLAG_GROUND_STATE_SPLIT): S(0), Delta S scratch
    // and the static potential P(0), [4][N] per domain
    bool split = false, static_done = false, computing_static = false;
    // graph replay of a step (rp_graph_capture / rp_graph_step): the step as
    // the step-dependent kernels read it on replay, and the captured graph
    long long *d_step = nullptr;
    long long *h_step_pin = nullptr;          // pinned source of the counter's re-sync
    cudaStream_t capture_stream = nullptr;    // the recording's own stream (the context stream may be
                                              // the legacy default stream, which cannot be captured)
    bool capturing = false;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    long long graph_synced = -2;              // host step the device counter holds (-2: unknown)
    std::vector<float *> ground, delta, pstatic;
    // history spill to host memory (RP_FLAG_HISTORY_SPILL): the spilled
    // sources (host ring depth spill_hd), the windows with their descriptors
    // for the forward passes, and the copy streams with their events:
    //   sp_pushed   on the context stream once a round's slices are staged;
    //   sp_out[k]   on spill_out after the copy to the host of step s, k = s % kSpillStage
    //               (the push of step s + kSpillStage waits for it before reusing the staging slot);
    //   sp_in       on spill_in after the last copy into a window's input buffer;
    //   sp_wfft     on the context stream after the last window transform (the
    //               input buffers' last reader).
    bool spill = false;
    int spill_hd = 0;
    std::vector<SpillSource> spill_srcs;
    std::vector<SpillWindow> spill_wins;
    std::vector<FwdRing> wfwd;
    FwdRing *d_wfwd = nullptr;
    // the forward rings and, after those of each size class, that class's
    // windows (lag_off = lo, inputs in pointer slots nd + w): one launch pair
    // per class pushes a round and transforms the windows' steady-state
    // slices (empty when the slots do not fit)
    std::vector<FwdRing> mix;
    FwdRing *d_mix = nullptr;
    std::vector<LaunchGroup> mix_groups;
    long long host_bytes = 0;
    cudaStream_t spill_out = nullptr, spill_in = nullptr;
    cudaEvent_t sp_pushed = nullptr, sp_in = nullptr, sp_wfft = nullptr;
    std::vector<cudaEvent_t> sp_out;
    bool finalized = false;
    std::vector<DomainDesc> doms;
    std::vector<PairPlan> pairs;   // [t * ndom + s]

    // plan
    std::vector<FwdRing> fwd;
    std::vector<LaunchGroup> fwd_groups;             // (plane pass, column pass) per size class
    std::vector<LaunchGroup> inv_groups;             // (MAC + column pass, plane pass) per size class
    std::vector<InvTarget> inv;
    std::vector<MacEntry> entries;
    std::vector<DirectTarget> dtg;
    std::vector<DirectPair> dpairs;
    std::vector<RawRing> raw;
    std::vector<int> raw_block0;                     // [ndom + 1], blocks of k_ring_push
    int plane_blocks = 0, col_blocks = 0, mac_blocks = 0, invp_blocks = 0, dir_blocks = 0;
    size_t smem_plane = 0, smem_col = 0, smem_mac = 0, smem_inv = 0, smem_dir = 0;
    bool fwd_tile[7] = {}, inv_tile[7] = {};            // plane-pass form per class (index by class_slot)
    size_t smem_plane_cls[7] = {}, smem_inv_cls[7] = {}; // their shared memory per launch
    int max_lag = 0, raw_depth = 0, spec_depth = 0;
    long long spectral_bytes = 0, kernel_bytes = 0, device_bytes = 0;

    // device
    FwdRing *d_fwd = nullptr;
    InvTarget *d_inv = nullptr;
    MacEntry *d_entries = nullptr;
    DirectTarget *d_dtg = nullptr;
    DirectPair *d_dpairs = nullptr;
    RawRing *d_raw = nullptr;
    bool tma = false;                // TMA-fed MAC available for the cubic classes
    int mac_stages[7] = {};          // pipeline depth per class (index by class_slot)
    int mac_cw[7] = {16, 16, 16, 16, 16, 16, 16};   // consumer warps of the MAC per class
    int sm_count = 0;
    int *d_err = nullptr;            // set by a kernel whose bounded wait ran out
    // far pairs (low-rank path)
    std::vector<FarSource> far_src;
    std::vector<FarTarget> far_tgt;
    std::vector<FarLink> far_links;
    std::vector<int> far_link0, far_link1, far_link_threads;   // per far source
    std::vector<float *> far_Z;
    std::vector<int> far_rows;                                  // padded W rows per far source
    std::vector<int> far_splits;                                // split-K count per far source
    float *far_work = nullptr;                                  // split-K partial products
    std::vector<CUtensorMap> far_mapW, far_mapX;
    std::vector<int> far_src_of_dom;                            // far source index of a domain, -1
    FarSource *d_far_src = nullptr;
    FarTarget *d_far_tgt = nullptr;
    // two-sided far factors (far_source_points > 0; rp_far2.cu): the far
    // sources with their anterpolation weights and coefficient rings (one
    // array, far2_qall: [source][2 D][4][2 KS] bf16), the factor blocks of
    // every target, the gathered GEMM's CTAs and its partial sums
    bool far2 = false;
    std::vector<FarSrc2> far2_srcs;
    std::vector<int> far2_of_dom;                               // FarSrc2 index of a domain, -1
    std::vector<FarTask> far2_tasks;
    std::vector<FarKBlock> far2_kb;
    FarSrc2 *d_far2_srcs = nullptr;
    FarTask *d_far2_tasks = nullptr;
    FarKBlock *d_far2_kb = nullptr;
    __nv_bfloat16 *far2_qall = nullptr, *far2_fac = nullptr;
    float *far2_work = nullptr;
    CUtensorMap far2_mapQ{}, far2_mapF{};
    int far2_BN = 0, far2_KS = 0, far2_D = 0, far2_max_nz = 0, far2_max_plane = 0, far2_max_n = 0;
    long long far2_fac_rows = 0;
    // far sources with no forward ring of their own: staged by a separate
    // kernel; far targets with no FFT pass: interpolated by a separate kernel
    // after the direct pass (only under a source partition)
    std::vector<FarSource> far_src_alone;
    std::vector<FarTarget> far_tgt_alone;
    FarTarget *d_far_tgt_alone = nullptr;
    int far_alone_planes = 0;
    std::vector<int> far_src_alone_of_dom;
    FarSource *d_far_src_alone = nullptr;
    FarLink *d_far_links = nullptr;
    int far_max_r = 0, npairs_far = 0;
    long long far_bytes = 0, far_max_n = 0, far_zeroed_step = -1;
    std::vector<void *> allocs;
    std::vector<void *> *alloc_sink = nullptr;   // where dev_alloc records (the far path's own list while built)
    std::vector<void *> far_allocs;
    long long far_alloc_bytes = 0;
    std::vector<std::array<std::vector<double>, 3>> far_tnodes;   // far targets' per-axis nodes, by domain
    // learned far field
    bool trained = false;
    Mlp net;                          // inference network
    bool net_open = false;
    std::vector<LPair> lpairs;        // sorted by target
    std::vector<LTarget> ltgts;
    std::vector<MomentJob> mjobs;     // sorted by source domain
    std::vector<int> mjob_of_dom;
    LPair *d_lpairs = nullptr;
    LTarget *d_ltgts = nullptr;
    MomentJob *d_mjobs = nullptr;
    float *d_lnu = nullptr;
    float *d_lxf = nullptr, *d_lylin = nullptr;   // fp32 network rows and linear-skip outputs
    float *d_lcontrib = nullptr;      // per-pair contributions [pairs][64][4]
    int *d_lpair_r = nullptr;         // per-pair target node count
    int lrows = 0, npairs_learned = 0, mjob_max_nz = 0;
    bool net_used = false;            // some learned pair adds the network's output
    std::vector<char> net_pair;       // [t * ndom + s]: the pair uses the network (else the linear skip alone)
    int smem_optin = 0;
    float *noalloc_stage = nullptr;   // device address of rp_evaluate_host_noalloc's fixed array (set at finalize)
    // FP64 audit (RP_FLAG_AUDIT): its device scratch and the last result
    char *audit_buf = nullptr;
    int audit_cap = 0;                // points the scratch holds
    double audit_rel_l2 = -1.0;       // largest rel-L2 of the last rp_audit, -1 before the first
    long long audit_step = -1;
    // Host-buffer calls: device staging per domain ([4][N]), two sets
    // alternating by step parity, and a copy stream, so that a step's copies
    // run while the kernels of the steps around it do; events order the two
    // streams.
    std::vector<float *> in_stage[2];
    std::vector<float *> out_stage[2];
    cudaStream_t copy_in = nullptr;            // host-to-device copies
    cudaStream_t copy_out = nullptr;           // device-to-host copies (apart, so that a step's
                                               // inputs never queue behind the last step's results)
    cudaEvent_t in_ready = nullptr;            // the last host push's copy is done
    cudaEvent_t in_free[2] = {nullptr, nullptr};    // the last push that read in_stage[b] has run
                                                    // (pushes run in order on the context stream)
    cudaEvent_t out_ready = nullptr;           // the last host evaluation's results are staged
    cudaEvent_t out_free[2] = {nullptr, nullptr};   // the copy out of out_stage[b] is done

    // step state.  Under a source partition (rp_own_sources) the domains
    // another context owns count as pushed from the start of every round.
    long long step = -1;
    std::vector<char> pushed;
    int npushed = 0;
    std::vector<char> owned;          // [ndom]: this context owns the domain's source
    int n_owned = 0;

    // profiling
    std::vector<ProfRec> pending;
    std::vector<cudaEvent_t> spare_events;
    long long launches[RP_K_COUNT] = {};   // timed launches
    double ms[RP_K_COUNT] = {};
    long long count[RP_K_COUNT] = {};      // every launch

    std::string last_error;
};

namespace rp {

inline rp_status fail(rp_ctx *ctx, rp_status st, const std::string &msg)
{
    if (ctx) ctx->last_error = msg;
    return st;
}

inline rp_status cuda_fail(rp_ctx *ctx, cudaError_t e, const char *what)
{
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    return fail(ctx, e == cudaErrorMemoryAllocation ? RP_ERR_OOM : RP_ERR_CUDA, m);
}

#define RP_CUDA(ctx, expr)                                           \
    do {                                                             \
        cudaError_t e_ = (expr);                                     \
        if (e_ != cudaSuccess) return cuda_fail((ctx), e_, #expr);   \
    } while (0)

inline rp_status use_device(rp_ctx *ctx)
{
    int cur = -1;
    RP_CUDA(ctx, cudaGetDevice(&cur));
    if (cur != ctx->device) RP_CUDA(ctx, cudaSetDevice(ctx->device));
    return RP_OK;
}

template <class T>
rp_status dev_alloc(rp_ctx *ctx, T **p, size_t count)
{
    void *q = nullptr;
    const size_t bytes = std::max<size_t>(count * sizeof(T), 16);
    if (ctx->cfg.device_budget > 0 && ctx->device_bytes + (long long)bytes > ctx->cfg.device_budget)
        return fail(ctx, RP_ERR_OOM, "device budget of " + std::to_string(ctx->cfg.device_budget) +
                                         " B exceeded: " + std::to_string(ctx->device_bytes) + " B held, " +
                                         std::to_string(bytes) + " B asked");
    cudaError_t e = cudaMalloc(&q, bytes);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMalloc");
    (ctx->alloc_sink ? *ctx->alloc_sink : ctx->allocs).push_back(q);
    if (ctx->alloc_sink) ctx->far_alloc_bytes += (long long)bytes;
    ctx->device_bytes += (long long)bytes;
    *p = static_cast<T *>(q);
    return RP_OK;
}

template <class T>
rp_status upload(rp_ctx *ctx, T **dst, const std::vector<T> &v)
{
    rp_status st = dev_alloc(ctx, dst, v.size());
    if (st) return st;
    if (!v.empty()) RP_CUDA(ctx, cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
    return RP_OK;
}

inline cudaEvent_t take_event(rp_ctx *ctx)
{
    if (!ctx->spare_events.empty()) {
        cudaEvent_t e = ctx->spare_events.back();
        ctx->spare_events.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Runs `launch` (returns cudaError_t), bracketed by events when profiling
// and the current step is sampled.
template <class F>
rp_status timed_launch(rp_ctx *ctx, int kind, const char *what, F &&launch)
{
    cudaEvent_t a = nullptr, b = nullptr;
    const int every = ctx->cfg.profile_every;
    const bool timed = ctx->profile && (every <= 1 || ctx->step < 0 || ctx->step % every == 0);
    ctx->count[kind] += 1;
    if (timed) {
        a = take_event(ctx);
        b = take_event(ctx);
        RP_CUDA(ctx, cudaEventRecord(a, ctx->stream));
    }
    cudaError_t e = launch();
    if (e != cudaSuccess) return cuda_fail(ctx, e, what);
    if (timed) {
        RP_CUDA(ctx, cudaEventRecord(b, ctx->stream));
        ctx->pending.push_back({kind, a, b});
    }
    return RP_OK;
}

// History spill (rp_spill.cu).
rp_status open_spill(rp_ctx *ctx);         // at finalize: rings, host rings, window descriptors, streams
rp_status build_mix(rp_ctx *ctx);          // the merged descriptor table, whenever the forward rings change
rp_status spill_round_done(rp_ctx *ctx);   // after a round's pushes: its slices to the host
rp_status spill_fetch(rp_ctx *ctx);        // before the MAC: windows complete, next slices fetched

}  // namespace rp
