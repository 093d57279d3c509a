/*
 * rp.h -- C-ABI of the GB300 retarded-potential library (librp.so).
 *
 * The library evaluates, at every time step, the retarded scalar and vector
 * potentials of a set of sub-domains on every sub-domain grid:
 *
 *   phi(r_k, l) = sum_n sum_{k' in d_n} h_n^3 rho_n(k', l dt - R/c) / R
 *   A(r_k, l)   = (1/c) sum_n sum_{k'} h_n^3 J_n(k', l dt - R/c) / R,   R = |r_k - r_k'|
 *
 * i.e. the Lorenz-gauge integral of Eq. 2 summed over sub-domains (Eqs. 3-4),
 * sampled on each domain's grid (Eq. 8), with the sources between time samples
 * given by the hat-function interpolation of Eq. 7 -- equivalently the
 * space-time sampled Green's function G_m = h^3 T(m dt - R/c)/R of Eq. 11
 * applied as in Eq. 12.  At R = 0 (a node and itself) the 1/R singularity is
 * replaced by its average over the node's cell, C h^2 with
 * C = 3 ln(2 + sqrt 3) - pi/2, at lag 0 (the paper's "smoothed Green's
 * function" for the self domain, Sec. III after Eq. 6).  The electron charge
 * q_e of the paper's four-vector source (Sec. II, before Eq. 2) is NOT
 * applied; multiply by q_e = -1 if wanted.  Atomic units throughout.
 *
 * Grids: a domain has origin o (position of node (0,0,0)), n = (nx, ny, nz)
 * nodes and spacing h; node (i,j,k) is at o + h(i,j,k) and has id
 * i + nx*(j + ny*k).  Every per-domain field array is float32, x fastest.
 *
 * Ownership: the caller owns every input and output buffer it passes; the
 * library owns its history rings, kernel spectra, plan and workspace.  Device
 * pointers must be device memory of the context's device.  All work is
 * enqueued on the context's stream and is asynchronous unless stated: a
 * buffer passed to a call may be reused once the stream has passed that call
 * (e.g. after rp_sync or a stream-ordered event).
 *
 * Errors: bad arguments and calls out of order are detected synchronously and
 * returned as a status; nothing aborts.  A CUDA failure from earlier
 * asynchronous work is returned by the next call that checks the stream, or
 * by rp_sync.  rp_last_error() gives a one-line description of the last
 * failure of a context.
 */
#ifndef RP_H
#define RP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    RP_OK = 0,
    RP_ERR_ARG = 1,         /* invalid argument (NULL, non-positive size, ...) */
    RP_ERR_STATE = 2,       /* call out of order (see rp_push / rp_evaluate) */
    RP_ERR_HISTORY = 3,     /* a needed past sample is older than the first push */
    RP_ERR_CUDA = 4,        /* CUDA runtime error, or no usable device */
    RP_ERR_OOM = 5,         /* device allocation failed */
    RP_ERR_UNSUPPORTED = 6, /* sizes beyond what the kernels handle */
    RP_ERR_TIMEOUT = 7      /* a bounded device-side wait ran out */
} rp_status;

/* How pairs of domains are evaluated. */
typedef enum {
    /* Self term by zero-padded (Hockney) FFT convolution with the cell-averaged
     * kernel; cross pairs of equal spacing by FFT convolution split by lag
     * ("delay bin") with a spectral history ring; other pairs by direct sum. */
    RP_MODE_FFT = 0,
    /* Every pair by the direct retarded sum in FP32 with compensated
     * accumulation (the plain path). */
    RP_MODE_DIRECT = 1,
    /* As RP_MODE_FFT, but pairs at least far_distance apart go through an
     * interpolative low-rank factorisation of their lag-stacked operator
     * [G_lo ... G_hi] (Eq. 11): the target's potential is represented by its
     * values at far_points^3 Chebyshev nodes of the target box and
     * interpolated (tensor-product Lagrange) to the grid; the node values are
     * contracted with the source history as time-batched bf16 tensor-core
     * GEMMs with fp32 accumulation.  Its accuracy rests on the far potential
     * being smooth across the target box (sources slow on the light-crossing
     * time of a box); it is not an extension in the paper (its Summary only
     * mentions a multipole approximation as a further speed-up). */
    RP_MODE_LOWRANK = 2
} rp_mode;

/* Samples before the first push equal the first push: S(t <= 0) = S(0), the
 * reading of Eqs. 7 and 9.  Without it, evaluating a step that needs such a
 * sample returns RP_ERR_HISTORY. */
#define RP_FLAG_GROUND_STATE_CLAMP 0x1u
/* Plan only: no CUDA call is made and nothing is allocated; rp_finalize
 * computes the pair plan (see rp_pair_info / rp_query) and push/evaluate
 * return RP_ERR_STATE.  Usable on a host without a GPU. */
#define RP_FLAG_PLAN_ONLY 0x2u
/* Time kernel launches with CUDA events on the context stream (all of them,
 * or those of one step in every rp_config.profile_every); read the totals
 * with rp_kernel_stats and the launch counts with rp_kernel_count. */
#define RP_FLAG_PROFILE 0x4u
/* RP_MODE_LOWRANK: build the far pairs' factors in rp_train_far_model (for
 * the pairs the learned field does not take) instead of in rp_finalize, so
 * that factors of pairs that move to the network are never made.  Until
 * rp_train_far_model has run, rp_push returns RP_ERR_STATE. */
#define RP_FLAG_DEFER_FAR 0x8u
/* The ground-state split of Eqs. 9-12.  The first push of every domain is
 * its ground state S(0).  When that first round is complete the library
 * computes the static potential P(0) = sum_m G_m S(0) of every target (the
 * c -> infinity sum h^3 S(0)/R, since the hat weights of a pair's lags sum to
 * one; read it with rp_ground_potential) and from then on keeps
 * Delta S = S - S(0) in its histories, zero before the first push.
 * rp_evaluate then returns the induced part sum_m G_m Delta S(l-m), so that
 * P(l) = P(0) + rp_evaluate's output equals the plain sum under
 * RP_FLAG_GROUND_STATE_CLAMP (implied) up to rounding.  The FP32 rounding of
 * the history, the per-step sums and the output then scales with |Delta S|
 * rather than |S|: the induced part keeps its digits when a large static
 * density carries a small response.  FFT and direct pairs only: rp_finalize
 * returns RP_ERR_UNSUPPORTED with far pairs.  Costs one elementwise pass per
 * push. */
#define RP_FLAG_GROUND_STATE_SPLIT 0x10u
/* History spill to host memory (Sec. IV: every sample of the window
 * [l - N_R,max, l] is kept for the steps to come, while a step reads only a
 * pair's Delta N_R of them, and the store need not be the fast memory).
 * A pair whose lag window [lag_lo, lag_hi] starts far back
 * (lag_lo >= 2 (lag_hi - lag_lo + 2)) reads its source's spectra from a
 * device window ring of B = lag_hi - lag_lo + 1 slots instead of the
 * full-depth spectral ring.  The (rho, J) slices of such a source, 16 B per
 * point (an eighth of its doubled-size spectrum), are copied once each round
 * into a pinned host ring of depth max(history_depth, largest spilled
 * lag_hi + 1); each step, every window gets back the one slice it newly
 * needs, a step ahead, and transforms it into its ring with the same forward
 * passes as a push.  The device spectral rings keep only the unspilled lags.
 * Same kernels, same summation order: results are bit-identical to the
 * unspilled context.  The copies ride on two streams of the context's own,
 * ordered against the kernels by events.  FFT pairs only (direct and far
 * pairs are unaffected); not with rp_graph_capture (RP_ERR_UNSUPPORTED).
 * rp_stats.host_bytes and spill_windows report the host ring and the number
 * of windows; spectral_bytes then includes the window rings, their input
 * slices and a three-slot staging ring per spilled source. */
#define RP_FLAG_HISTORY_SPILL 0x20u
/* FP64 error audit on the GPU (rp_audit, rp_audit_values): every source
 * keeps a raw (rho, J) ring as deep as its deepest pair reads (16 B per point
 * and step, in rp_stats.device_bytes), written at every push. */
#define RP_FLAG_AUDIT 0x40u
/* By default the spectral sum over a target's (source, lag) entries (Eq. 12
 * per spectral coefficient, before the one inverse FFT per target and field)
 * is Kahan-compensated in FP32: its rounding stays near one rounding of the
 * sum of magnitudes however many entries a target has (the MAC then runs one
 * variant, 12 multiply-add warps and 3 inverse-FFT warps; rp_config.mac_warps
 * must be 0 or 12).  This flag makes it a plain FP32 multiply-add chain,
 * whose error grows like the square root of the entry count, with the
 * autotuned 8/12/16-warp variants. */
#define RP_FLAG_PLAIN_SUM 0x80u
/* Overlapped pushes: a push's kernels (ring writes, forward passes, far
 * anterpolation and batch GEMMs) run on a stream of the library's own, so
 * that step l+1's push overlaps step l's evaluation on the context stream
 * (the push is latency-bound, the evaluation's spectral MAC bound by HBM).
 * The rings get one slot more than the deepest lag, so that a push never
 * overwrites a slot the previous step's evaluation still reads, and a push
 * waits for the evaluation two steps back.  rp_evaluate waits for the push.
 * The inputs of a push must be complete when its kernels start: rp_push_all_event
 * names the event after which they are; rp_push_all_host uses its own copy;
 * rp_push and rp_push_all wait for the context stream (and so overlap
 * nothing).  Same kernels and sums: results are bit-identical to a context
 * without the flag.  Not with RP_FLAG_GROUND_STATE_SPLIT,
 * RP_FLAG_HISTORY_SPILL, the learned field (RP_FLAG_DEFER_FAR) or
 * rp_graph_capture (RP_ERR_UNSUPPORTED). */
#define RP_FLAG_OVERLAP_PUSH 0x100u

typedef struct {
    double c;            /* speed of light, > 0 (137.036 in atomic units) */
    double dt;           /* time step, > 0 */
    int history_depth;   /* minimum history ring depth in steps (0: what the geometry needs); under
                          * RP_FLAG_HISTORY_SPILL, of the host ring */
    int mode;            /* rp_mode */
    unsigned int flags;  /* RP_FLAG_* */
    int far_points;      /* RP_MODE_LOWRANK: interpolation nodes per axis, 2..8 (0: 4) */
    double far_distance; /* RP_MODE_LOWRANK: smallest box distance of a far pair (bohr, > 0) */
    int far_batch;       /* RP_MODE_LOWRANK: source slices per GEMM, multiple of 8 in 8..64 (0: 32);
                          * a far pair also needs lag_lo >= far_batch - 1 */
    int mac_warps;       /* consumer warps of the TMA-fed spectral MAC: 8, 12 or 16, or 0 to let
                          * rp_finalize time the three variants on this plan (two launches each
                          * per FFT size class) and keep the fastest.  The variants sum the same
                          * terms in the same order: the choice changes timing, never results.
                          * Only with RP_FLAG_PLAIN_SUM; the compensated sum has one variant (12). */
    int profile_every;   /* RP_FLAG_PROFILE: time the launches of step s only when s % profile_every == 0
                          * (launches outside the step cycle always), >= 0; 0 or 1: every step.  The
                          * events sit between kernels and hold back the next launch, so sampling
                          * keeps them off most steps.  rp_set_profiling changes it later. */
    int far_source_points; /* RP_MODE_LOWRANK: 0 keeps every source node exact in the far factors; 2..8
                          * interpolates the source side too (two-sided): each far source's slice is
                          * anterpolated onto far_source_points^3 Chebyshev nodes of its box at push
                          * (q_b = sum_k' L_b(r_k') h^3 S(k')), and the factors hold Eq. 11 between
                          * target and source nodes, so that their size no longer grows with the
                          * source grid */
    long long device_budget; /* largest device memory the context may hold, in bytes (rp_stats.device_bytes);
                          * an allocation that would pass it returns RP_ERR_OOM without calling the
                          * allocator (with RP_FLAG_PLAN_ONLY, rp_finalize compares the planned bytes).
                          * 0: no limit.  Not in the paper: a resource guard of the library. */
    int mac_stages;      /* field-tile stages of the TMA-fed MAC's copy pipeline, 2 .. (as many as the
                          * shared memory holds), or 0 for the most that fit; fewer stages leave
                          * shared memory on each SM for other kernels' blocks (the overlapped push's
                          * forward passes).  Timing only: results do not depend on it. */
    int reserved[3];     /* set to zero */
} rp_config;

typedef struct rp_ctx rp_ctx;

/* Pair kinds reported by rp_pair_info. */
typedef enum {
    RP_PAIR_FFT = 0, RP_PAIR_DIRECT = 1, RP_PAIR_LOWRANK = 2, RP_PAIR_LEARNED = 3,
    RP_PAIR_OTHER = 4   /* not evaluated here: its source is owned by another context (rp_own_sources) */
} rp_pair_kind;

typedef struct {
    int kind;          /* rp_pair_kind */
    int lag_lo;        /* smallest lag m with a nonzero hat weight T(m dt - R/c) */
    int lag_hi;        /* largest such lag; the pair reads steps l-lag_hi .. l-lag_lo */
    int fft_m[3];      /* padded FFT size per axis (0 for direct pairs) */
    double r_min;      /* smallest node distance between the two grids (0 for self) */
    double r_max;      /* largest node distance */
} rp_pair_info_t;

typedef struct {
    int ndomains;
    int npairs_fft;
    int npairs_direct;
    int max_lag;              /* largest lag_hi over all pairs */
    int raw_depth;            /* raw (rho, J) ring depth in steps, 0 if no pair reads it */
    int spectral_depth;       /* largest spectral ring depth in steps */
    long long step;           /* index of the last completed push round, -1 before the first */
    long long device_bytes;   /* device memory held by the context */
    long long spectral_bytes; /* of which: spectral history rings (under RP_FLAG_HISTORY_SPILL also the
                               * window rings, their input slices and the staging rings) */
    long long kernel_bytes;   /* of which: kernel spectra */
    long long points;         /* sum of grid points over all domains */
    int mac_tma;              /* 1: the spectral MAC of cubic targets is fed by TMA copies */
    int npairs_far;           /* pairs on the low-rank far path */
    long long far_bytes;      /* device memory of the far path (factors, batches, rings) */
    int mac_warps;            /* consumer warps of the MAC variant in use (last size class), 0 if none */
    int npairs_learned;       /* pairs on the learned far path (after rp_train_far_model) */
    int spill_windows;        /* RP_FLAG_HISTORY_SPILL: lag windows read from host-refilled window rings */
    int reserved;
    long long host_bytes;     /* pinned host memory of the spilled history ((rho, J) slices) */
    double audit_rel_l2;      /* largest per-(domain, field) rel-L2 of the last rp_audit, -1 before the first */
    long long audit_step;     /* the step it audited, -1 before the first */
    int owned_sources;        /* source domains this context owns (rp_own_sources; all by default) */
    int npairs_other;         /* pairs whose source another context owns (RP_PAIR_OTHER) */
} rp_stats;

/* Kernel classes timed under RP_FLAG_PROFILE. */
typedef enum {
    RP_K_RING_PUSH = 0,     /* raw slice into the history ring */
    RP_K_FWD_PLANE = 1,     /* forward FFT, x and y axes, one z-plane per block */
    RP_K_FWD_COLUMN = 2,    /* forward FFT along z, into the spectral ring */
    RP_K_MAC_INV_COLUMN = 3,/* spectral multiply-accumulate over (source, lag) + inverse FFT along z */
    RP_K_INV_PLANE = 4,     /* inverse FFT along y and x, crop, scale, write phi/A */
    RP_K_DIRECT = 5,        /* direct retarded sum */
    RP_K_FAR_CONVERT = 6,   /* far path: slice to bf16 batch matrix */
    RP_K_FAR_GEMM = 7,      /* far path: tcgen05 GEMM of factors and batch (two-sided: the gathered GEMM) */
    RP_K_FAR_SCATTER = 8,   /* far path: node values into coefficient rings (two-sided: the CTAs' sums) */
    RP_K_FAR_ANTERP = 9,    /* far path (two-sided factors): a pushed slice anterpolated onto its source's nodes */
    RP_K_MOMENTS = 10,      /* learned path: moments of the pushed slices */
    RP_K_LEARNED = 11,      /* learned path: network rows, network, output into the coefficients */
    RP_K_FAR_INTERP = 12,   /* far path: coefficients onto the grid of a target with no FFT pass (source partition) */
    RP_K_COUNT = 13
} rp_kernel_kind;

/*
 * rp_create -- make a context on CUDA device `device` using `stream`
 * (a cudaStream_t; NULL = the legacy default stream).  With
 * RP_FLAG_PLAN_ONLY, device and stream are ignored and no CUDA call is made.
 * cfg is copied.  Returns RP_ERR_ARG for c <= 0, dt <= 0, an unknown mode or
 * NULL pointers; RP_ERR_CUDA if the device cannot be used.
 */
rp_status rp_create(const rp_config *cfg, int device, void *stream, rp_ctx **out);

/*
 * rp_add_domain -- declare sub-domain d_n (Eqs. 3-4): origin[3] is the
 * position of node (0,0,0), n[3] the node counts (>= 1), h > 0 the spacing.
 * Writes the new domain's id (0, 1, ...) to *id.  Only before rp_finalize.
 * Two domains may not have a node at the same position (RP_ERR_ARG at
 * finalize).  At most 256 domains.
 */
rp_status rp_add_domain(rp_ctx *ctx, const double origin[3], const int n[3], double h, int *id);

/*
 * rp_own_sources -- source partition (Sec. IV: one process per domain, each
 * computing its domain's contributions to every domain): this context owns
 * the source domains ids[0 .. count-1] and no other.  It keeps only their
 * histories and evaluates only the pairs (target, owned source), for every
 * target: the pairs of other sources are RP_PAIR_OTHER.  rp_push / rp_push_host
 * accept only owned domains (RP_ERR_ARG otherwise); a round is complete when
 * every owned domain has pushed; rp_push_all reads only the owned domains'
 * pointers (the others may be NULL).  rp_evaluate then writes, for every
 * domain, the sum of the owned sources' contributions (every pair of an
 * owned source is evaluated, so each target gets some): adding the outputs
 * of contexts that own complementary
 * sets of sources (one per GPU, summed by a reduce-scatter at each target's
 * owner) gives the whole sum.  Before rp_finalize only; at least one id;
 * RP_ERR_ARG for ids out of range or repeated.  Default: every domain owned.
 */
rp_status rp_own_sources(rp_ctx *ctx, const int *ids, int count);

/*
 * rp_finalize -- plan every ordered pair (target, source), self pairs
 * included (Eq. 3): its lag window [lag_lo, lag_hi] from the smallest and
 * largest node distance (Sec. IV: only Delta N_R = Delta D/(c dt) past steps
 * contribute), its kind, the FFT sizes; build the kernel spectra of Eq. 11 in
 * FP64 on the host and store them in FP32; allocate the history rings
 * (Sec. IV: samples for [l - N_Rmax, l] are kept).  Synchronous.
 * RP_ERR_UNSUPPORTED if a domain exceeds 96 nodes per axis in FFT mode.
 */
rp_status rp_finalize(rp_ctx *ctx);

/*
 * rp_push -- hand over the sample of step l of domain `id`: d_rho[N] and
 * d_J[3][N] (Jx, Jy, Jz), device float32.  The library copies what it needs
 * into its rings (and in FFT mode transforms it into the spectral ring)
 * on the stream before returning control of the buffers.  The first push
 * after a complete round (every domain pushed) starts step l + 1.  Pushing a
 * domain twice in one round returns RP_ERR_STATE.
 */
rp_status rp_push(rp_ctx *ctx, int id, const float *d_rho, const float *d_J);

/*
 * rp_push_all -- rp_push for every domain in id order with batched launches:
 * d_rho[n] and d_J[n] are the device buffers of domain n.  Only at the start
 * of a round (no domain pushed yet in it).
 */
rp_status rp_push_all(rp_ctx *ctx, const float *const *d_rho, const float *const *d_J);

/*
 * rp_push_all_event -- rp_push_all for a context with RP_FLAG_OVERLAP_PUSH
 * whose inputs are complete once `ready` (a cudaEvent_t the caller recorded
 * after writing them; NULL: already complete when the call is made) has
 * completed: the push's kernels wait for that event alone, not for the
 * context stream, so they overlap the evaluation before them.  The buffers
 * must stay unchanged until the next rp_evaluate has been enqueued and its
 * stream has passed it (or rp_sync).  RP_ERR_STATE without the flag.
 */
rp_status rp_push_all_event(rp_ctx *ctx, const float *const *d_rho, const float *const *d_J, void *ready);

/*
 * rp_push_host -- rp_push from HOST buffers h_rho[N], h_J[3][N] (pinned
 * memory recommended; one copy when h_J == h_rho + N).  The library copies
 * them to device staging of its own on a host-to-device copy stream of the
 * context, ordered before the push's kernels by an event, so that the copy
 * overlaps kernels of earlier steps still running.  The host buffers must
 * stay valid and unchanged until rp_sync.
 */
rp_status rp_push_host(rp_ctx *ctx, int id, const float *h_rho, const float *h_J);

/*
 * rp_push_all_host -- rp_push_all from HOST buffers: h_rho[n] (N_n floats)
 * and h_J[n] (3*N_n floats) of every domain n, copied as in rp_push_host,
 * then one batched push.  Only at the start of a round.  The host buffers
 * must stay valid and unchanged until rp_sync.
 */
rp_status rp_push_all_host(rp_ctx *ctx, const float *const *h_rho, const float *const *h_J);

/*
 * rp_evaluate -- the retarded phi and A of the last complete step l on every
 * domain (Eq. 12: each target sums the contributions of every source, itself
 * included; lag 0 is included since the step's own samples are visible,
 * App. A uses j at the current time for A at the next step).  d_phi[n] has
 * N_n floats, d_A[n] has 3*N_n floats (Ax, Ay, Az), device memory, written
 * (not accumulated).  Returns RP_ERR_STATE if the last round is incomplete or
 * no step was pushed, RP_ERR_HISTORY if a needed sample predates the first
 * push and RP_FLAG_GROUND_STATE_CLAMP is not set.
 */
rp_status rp_evaluate(rp_ctx *ctx, float *const *d_phi, float *const *d_A);

/*
 * rp_graph_capture -- record one whole step (rp_push_all of d_rho / d_J, then
 * rp_evaluate into d_phi / d_A; arrays of device pointers, one per domain, as
 * for those calls) as a CUDA graph, without running it (the recording uses a
 * stream of its own; the replays run on the context stream).
 * The buffers are fixed: each rp_graph_step replays the step on their current
 * contents.  Call at a step boundary.  FFT, direct and two-sided far pairs
 * (rp_config.far_source_points > 0: their kernels read the step on the
 * device, and the batch GEMM's launch, recorded in every step, works on a
 * batch's last push only), without RP_FLAG_PROFILE or
 * RP_FLAG_GROUND_STATE_SPLIT (RP_ERR_UNSUPPORTED otherwise, and for
 * one-sided far pairs and the learned field, whose launches change from
 * step to step).  A new
 * capture replaces the previous graph.  Not with RP_FLAG_HISTORY_SPILL (its
 * copies address the slots of the current step).  (No counterpart in the paper: a
 * property of the library.)
 */
rp_status rp_graph_capture(rp_ctx *ctx, const float *const *d_rho, const float *const *d_J,
                           float *const *d_phi, float *const *d_A);

/*
 * rp_graph_step -- the next step by one replay of the captured graph: the
 * same result as rp_push_all + rp_evaluate on the captured buffers, with one
 * launch from the host.  Steps made by the other calls in between are allowed
 * (the device step counter is re-synchronised, which waits for the stream).
 * RP_ERR_STATE without a graph or inside a partially pushed step,
 * RP_ERR_HISTORY as for rp_evaluate.
 */
rp_status rp_graph_step(rp_ctx *ctx);

/*
 * rp_ground_potential -- under RP_FLAG_GROUND_STATE_SPLIT: the static
 * potential P(0) of the ground state (the first pushed round), Eq. 12's
 * P~_n(0) summed over sources, into d_phi[n] (N_n floats) and d_A[n]
 * (3*N_n floats), device memory, written; on the context stream.
 * RP_ERR_STATE without the flag or before the first round is complete.
 */
rp_status rp_ground_potential(rp_ctx *ctx, float *const *d_phi, float *const *d_A);

/*
 * rp_evaluate_host -- rp_evaluate into HOST buffers h_phi[n] (N_n floats) and
 * h_A[n] (3*N_n floats; one copy when h_A[n] == h_phi[n] + N_n): the results
 * are staged in device memory of the library (two sets, alternating by step)
 * and copied device-to-host on a device-to-host copy stream of the context
 * (apart from the host-to-device one), overlapping the next step's kernels.
 * They are valid after rp_sync (which waits for every stream of the
 * context), not after a synchronisation of the context stream alone.
 */
rp_status rp_evaluate_host(rp_ctx *ctx, float *const *h_phi, float *const *h_A);

/*
 * rp_evaluate_host_noalloc -- rp_evaluate_host without any device allocation.
 * (No counterpart in the paper: this is a property of the library, not of the
 * method.)
 *
 * rp_evaluate_host stages phi and A in device memory that it allocates with
 * cudaMalloc on its first call.  Some callers cannot allow that: a process
 * whose device memory is handed out by another allocator or fixed budget once
 * the run has started, where the library may not call cudaMalloc after
 * set-up.  This variant stages the results instead in a fixed array compiled
 * into the library (16 MiB: at most 1,048,576 grid points summed over all
 * domains; more returns RP_ERR_UNSUPPORTED before any work) and calls no
 * allocating routine.  Every GPU that loads the library holds that array
 * until the process exits.
 *
 * Arguments, layout and results are those of rp_evaluate_host: h_phi[n] gets
 * N_n floats and h_A[n] 3*N_n floats, valid after rp_sync.  The array's
 * device address is looked up (cudaGetSymbolAddress) by the first
 * rp_finalize on each device, which is when the 16 MiB are placed in device
 * memory; this call only reads the address, so device memory in use is the
 * same before and after it.  All calls in the process on a device share the
 * one array and each call overwrites it, so calls whose work overlaps on the
 * GPU (two contexts on different streams, say) race and may return each
 * other's values: order them on one stream, or synchronise between them.
 */
rp_status rp_evaluate_host_noalloc(rp_ctx *ctx, float *const *h_phi, float *const *h_A);

/*
 * rp_fields -- the fields of App. B (Eqs. B1a, B1b) on domain `id`'s grid from
 * its potentials as rp_evaluate writes them (atomic units):
 *     E = -grad phi - (1/c) dA/dt,    B = curl A.
 * Space derivatives are second-order central differences, second-order
 * one-sided on the grid faces (each axis needs >= 3 nodes).  The time
 * derivative is (3 A_l - 4 A_{l-1} + A_{l-2}) / (2 dt), or (A_l - A_{l-1})/dt
 * when d_A2 is NULL.  Device pointers of domain `id`: d_phi [N] (step l),
 * d_A, d_A1, d_A2 [3][N] (steps l, l-1, l-2), d_E [3][N], d_B [3][N] or NULL
 * (not computed); node id = x + nx (y + ny z).  The caller owns every buffer;
 * nothing is allocated.  On the context stream; after rp_finalize.
 * RP_ERR_ARG for a bad id, a NULL required pointer or an axis under 3 nodes.
 */
rp_status rp_fields(rp_ctx *ctx, int id, const float *d_phi, const float *d_A, const float *d_A1,
                    const float *d_A2, float *d_E, float *d_B);

/*
 * rp_gemm_bf16 -- D = A B^T on the tensor cores (tcgen05.mma, bf16 operands,
 * fp32 accumulation in tensor memory).  A is M x K and B is N x K, bf16,
 * row-major with K contiguous; D is M x N fp32 row-major.  All three are
 * device pointers on `device`; `stream` is a cudaStream_t (NULL = legacy).
 * Shapes: M a multiple of 128, K a multiple of 64, N a multiple of 32 up to
 * 256.  This is the contraction the low-rank far field applies (skeleton rows
 * of the lag-stacked kernel of Eq. 11 against a batch of source slices); it
 * is exposed so that the tensor-core path can be checked on its own.
 * Synchronous.  RP_ERR_ARG for other shapes or NULL pointers, RP_ERR_CUDA if
 * the device or the tensor-map encoder is unusable, RP_ERR_TIMEOUT if a
 * bounded device wait ran out.
 */
rp_status rp_gemm_bf16(const void *d_A, const void *d_B, float *d_D, int M, int N, int K, int device,
                       void *stream);

/* Operand types of rp_gemm_tn. */
#define RP_DTYPE_BF16 0
#define RP_DTYPE_FP16 1

/*
 * rp_gemm_tn -- the tensor-core contraction in the forms the far field and
 * the learned far field use (Eq. 11 applied through skeleton rows, as for
 * rp_gemm_bf16; and the layers of the learned stand-in's network).
 *   dtype: RP_DTYPE_BF16 or RP_DTYPE_FP16 -- both operands of that type
 *          (tcgen05.mma kind::f16, fp32 accumulation in tensor memory).
 *   terms = 1: A is M x K, B is N x K; D = A B^T.
 *   terms = 3: A is M x 2K holding [A_hi | A_lo] per row and B is N x 2K
 *              holding [B_hi | B_lo]; D = A_hi B_hi^T + A_hi B_lo^T +
 *              A_lo B_hi^T, i.e. the product of A_hi + A_lo and B_hi + B_lo
 *              less the lo*lo term (about 16 significant bits per operand).
 * For terms = 3 each pipeline stage holds the four tiles of a K step and the
 * three products accumulate in one fp32 accumulator, so every operand byte
 * is read once.  N may exceed 256: it runs in column tiles of the widest
 * multiple of 32 up to 256 that divides N.  `splits` cuts the K range into
 * that many chunks run by separate CTAs whose fp32 partial products are then
 * summed in a fixed order (deterministic); 0 picks the count the far path
 * uses (one wave of CTAs, one per SM).  The partial products need
 * splits x M x N floats of device memory, which this call allocates and
 * frees.  Shapes: M a multiple of 128, K of 64, N of 32 (N <= 4096); D is
 * M x N fp32 row-major, all device pointers on `device`.  Synchronous.
 * RP_ERR_ARG for other shapes, an unknown dtype, terms other than 1 or 3,
 * splits outside [0, 4096] or pointers that are not 16-byte aligned;
 * RP_ERR_CUDA if the device or the tensor-map encoder is unusable;
 * RP_ERR_TIMEOUT if a bounded device wait ran out.
 */
rp_status rp_gemm_tn(const void *d_A, const void *d_B, float *d_D, int M, int N, int K, int dtype, int terms,
                     int splits, int device, void *stream);

/*
 * Learned far field: the network on its own.
 *
 * The learned stand-in for far pairs (north of the low-rank path; see
 * rp_train_far_model) is a bias-free multilayer perceptron
 *     x -> W1 -> leaky -> W2 -> leaky -> W3 -> leaky -> W4 -> y
 * with leaky(z) = z for z >= 0 and 0.2 z otherwise, fp16 weights and
 * activations as tensor-core operands (tcgen05.mma kind::f16) and fp32
 * accumulation.  Its inputs are a source's monopole, dipole and quadrupole
 * moments over a delay window and its outputs the potentials at 64 nodes of
 * the target (the multipole description of the far interaction, Sec. IV).
 * These three calls exist so that the network's kernels can be checked on
 * their own; all are synchronous and allocate and free their own device
 * memory on `device`.
 *
 * rp_mlp_layout -- writes the five layer widths (input, three hidden,
 * output) to dims[5] if dims is not NULL; returns the number of weights.
 * Weights are passed as one float array: W1 [d1][d0], W2 [d2][d1],
 * W3 [d3][d2], W4 [d4][d3], each row-major (output index major).
 *
 * rp_mlp_forward -- y[rows][d4] = network(x[rows][d0]) for host arrays, with
 * rows a multiple of 128.  Weights and inputs are rounded to fp16 on the way
 * in.  RP_ERR_ARG for NULL pointers or rows, RP_ERR_CUDA on a device error,
 * RP_ERR_TIMEOUT if a bounded device wait ran out.
 *
 * rp_mlp_grad -- the loss L = (1 / 2 rows) sum |y - t|^2 over the rows
 * (t: host targets [rows][d4]) and dL/dW for every weight (host g, the
 * weight layout), from the network's own backward pass.  Errors as for
 * rp_mlp_forward.
 */
int rp_mlp_layout(int *dims);
rp_status rp_mlp_forward(const float *h_w, const float *h_x, int rows, float *h_y, int device);
rp_status rp_mlp_grad(const float *h_w, const float *h_x, const float *h_t, int rows, float *h_g, float *h_loss,
                      int device);

/*
 * rp_learned_dataset -- the learned field's training data for one fixed
 * geometry, exposed so that its data path can be checked against a plain
 * implementation.  A source box of n_s[3] nodes at spacing h_s holds, per
 * history, three Gaussians with amplitudes a (1 + e sin(w t + phi)) and the
 * continuity-consistent current (dA/dt / 4 pi) grad Phi of each Gaussian
 * (seeded); the target box has extents Lt[3] and its centre lies Rc bohr
 * from the source centre in direction dir.  For each history and each of
 * `samples` consecutive steps the call writes four network rows (phi and
 * the current's three components in the pair's canonical frame):
 *   h_x [histories * samples * 4][d0]  inputs: the canonical moment window
 *                                      (moments l <= 2, Sec. IV), as fp16
 *                                      values widened to float;
 *   h_y [same][d4]                     targets: R_a times the direct
 *                                      retarded sum (Eqs. 2, 7, 8) at the 64
 *                                      canonical nodes, divided by the row's
 *                                      input scale;
 *   h_desc [histories][rp_learned_desc_size()] each history's description:
 *     for g in 0..2: centre (x, y, z) relative to the source origin, sigma;
 *     amplitude A_g(t_j) for g in 0..2, j in 0..63 (t_j a step index);
 *     dA_g/dt(t_j) / (4 pi) for g in 0..2, j in 0..63;
 *     t0 (window centre time of sample 0, in steps of the tables),
 *     dir (unit, 3 values), Rc.
 * Synchronous; allocates and frees its own device memory.  RP_ERR_ARG for
 * NULL pointers, non-positive sizes, n_s < 2, or more samples than the
 * 64-step tables allow for this geometry; RP_ERR_CUDA on a device error.
 */
int rp_learned_desc_size(void);
rp_status rp_learned_dataset(const int n_s[3], double h_s, const double Lt[3], const double dir[3], double Rc,
                             unsigned long long seed, int histories, int samples, double c, double dt, float *h_x,
                             float *h_y, double *h_desc, int device);

/*
 * rp_train_far_model -- train the learned far field and move the far pairs
 * it reproduces onto it.
 *
 * Candidates are the context's low-rank far pairs (RP_MODE_LOWRANK) whose
 * boxes are at least learned_distance apart and whose source and target
 * grids have the sizes of the first candidate.  The network (see
 * rp_mlp_layout) maps the source's monopole, dipole and quadrupole moments
 * (the multipole description of the far interaction, Sec. IV) over a
 * 16-step delay window, in the pair's canonical frame, to the potentials at
 * 64 canonical nodes around the target.  Its output is added to a linear
 * skip: an fp32 linear map of the same inputs fitted first by least squares
 * (FP64 normal equations); the network is then trained on what the skip
 * leaves, on the GPU with its own forward, backward and Adam kernels, on
 * synthetic histories (Gaussian
 * charges with oscillating amplitudes and their continuity-consistent
 * currents, random directions and distances spanning the candidates'),
 * whose targets are the direct retarded sums (Eqs. 2, 7, 8) at those nodes.
 * Each candidate is then validated on fresh histories in its own geometry,
 * with and without the network's output; the pair keeps the network only if
 * it lowers the error, and if the better rel-L2 error (worst of the four
 * fields) is at most `gate`, the pair becomes RP_PAIR_LEARNED: its low-rank factors are
 * dropped, its source's moments are taken at every push, and each
 * rp_evaluate runs the learned stand-in for it.  Otherwise it stays on the low-rank
 * path, which remains the fallback and the reference the network's error is
 * measured against.
 *
 * Call after rp_finalize and before the first push, on a context that has
 * not been trained.  Synchronous on the context's stream.  Zero fields of
 * the configuration take the defaults given.  RP_ERR_STATE if called at
 * another time or on a plan-only context, RP_ERR_UNSUPPORTED outside
 * RP_MODE_LOWRANK, RP_ERR_ARG for bad fields, RP_ERR_CUDA / RP_ERR_OOM /
 * RP_ERR_TIMEOUT on device errors.  A context with learned pairs does not
 * support rp_save_state.
 */
typedef struct {
    double learned_distance; /* smallest box distance of a candidate (bohr, > 0) */
    double gate;             /* largest validation rel-L2 of a learned pair (0: 5e-4, half the 1e-3
                              * bar of the far field: the validation sees a few histories and not
                              * the final interpolation onto the grid) */
    int histories;           /* training histories (0: 512) */
    int samples;             /* samples per history (0: 32, capped by the delay tables) */
    int iterations;          /* Adam steps (0: 3000) */
    int batch;               /* rows per step, a multiple of 128 (0: 1024) */
    float lr;                /* peak learning rate, cosine decay (0: 1e-3) */
    int validation;          /* validation histories per candidate (0: 4) */
    unsigned long long seed; /* seed of the histories and the initial weights */
    int reserved[8];         /* set to zero */
} rp_train_config;

typedef struct {
    int candidates;          /* pairs considered */
    int learned;             /* pairs moved onto the network */
    long long train_rows;    /* network rows in the training set */
    float final_loss;        /* training loss of the last minibatch */
    float train_seconds;     /* wall time of data generation and training */
    double val_max;          /* largest validation rel-L2 over the candidates */
    double val_mean;         /* mean validation rel-L2 */
    double val_linear_max;   /* the same with the linear skip alone (no network) */
    double val_linear_mean;
    int network_pairs;       /* learned pairs that add the network's output (the others use the
                              * linear skip alone, where the network did not lower their
                              * validation error) */
    int reserved[3];
} rp_train_report;

rp_status rp_train_far_model(rp_ctx *ctx, const rp_train_config *cfg, rp_train_report *report);

/*
 * rp_audit_values -- under RP_FLAG_AUDIT: the potentials of the last
 * complete step at `count` nodes h_nodes[] (host, node ids of domain
 * `target`) in FP64, into host h_out[count][4] (phi, Ax, Ay, Az): the plain
 * direct retarded sum of Eq. 8 with the hat interpolation of Eq. 7 over
 * every source node of every domain (the cell average C h^2 at R = 0, lag
 * 0), from the context's own history, on the GPU in FP64 (one block per
 * node, per-thread sums added in a fixed tree order).  It reads the same
 * FP32 samples as the evaluation, so it scores the path alone.  Under
 * RP_FLAG_GROUND_STATE_SPLIT it gives the induced part, as rp_evaluate does.
 * Synchronous on the context stream; allocates its scratch on first use.
 * RP_ERR_STATE without the flag or inside a partly pushed step,
 * RP_ERR_HISTORY as for rp_evaluate, RP_ERR_ARG for bad nodes.
 */
rp_status rp_audit_values(rp_ctx *ctx, int target, const long long *h_nodes, int count, double *h_out);

/*
 * rp_audit -- under RP_FLAG_AUDIT: the FP64 error audit of an evaluation.
 * d_phi / d_A are the device outputs rp_evaluate wrote for the last complete
 * step (as for rp_evaluate).  In every domain, min(nodes_per_domain, N)
 * nodes are drawn (one from each of that many equal strata of the node ids,
 * seeded); the FP64 sums of rp_audit_values there are compared with the
 * outputs, and h_rel_l2[4 * n + f] (host, may be NULL) gets
 * ||out - ref||_2 / ||ref||_2 over the sampled nodes of domain n for field
 * f (phi, Ax, Ay, Az).  The largest is kept for rp_stats.audit_rel_l2.
 * Synchronous.  Errors as for rp_audit_values; RP_ERR_ARG for
 * nodes_per_domain < 1 or NULL buffers.  (The final error audit in FP64 on
 * the GPU is a property of the library; the paper states no error measure.)
 */
rp_status rp_audit(rp_ctx *ctx, const float *const *d_phi, const float *const *d_A, int nodes_per_domain,
                   unsigned long long seed, double *h_rel_l2);

/* rp_sync -- wait for the context's stream; reports asynchronous failures. */
rp_status rp_sync(rp_ctx *ctx);

/* rp_query -- plan and memory summary (see rp_stats).  After rp_finalize. */
rp_status rp_query(rp_ctx *ctx, rp_stats *out);

/* rp_pair_info -- plan of the ordered pair (target, source).  After rp_finalize. */
rp_status rp_pair_info(rp_ctx *ctx, int target, int source, rp_pair_info_t *out);

/*
 * rp_kernel_stats -- timed launches (RP_FLAG_PROFILE or rp_set_profiling) and
 * their summed device time (ms, CUDA events on the context stream) of kernel
 * class `kind` since the last reset; waits for the stream.  reset != 0 clears
 * all counters (these and rp_kernel_count's) after reading.
 */
rp_status rp_kernel_stats(rp_ctx *ctx, int kind, long long *launches, double *total_ms,
                          int reset);

/*
 * rp_kernel_count -- every launch of kernel class `kind` since the last
 * reset (rp_kernel_stats with reset != 0), timed or not: a host-side count
 * kept on every context, with or without RP_FLAG_PROFILE; no wait.
 */
rp_status rp_kernel_count(rp_ctx *ctx, int kind, long long *launches);

/*
 * rp_set_profiling -- switch the per-launch CUDA events of RP_FLAG_PROFILE on
 * (every >= 1: the launches of steps s % every == 0) or off (every = 0) for
 * the launches that follow, on any context that is not plan-only.  Lets a
 * caller time a run without events between its kernels and then measure the
 * kernels in a separate pass on the same context.  RP_ERR_ARG for every < 0.
 * (No counterpart in the paper: a property of the library.)
 */
rp_status rp_set_profiling(rp_ctx *ctx, int every);

/*
 * rp_selftest_wait -- a library self-test, no counterpart in the paper.  One
 * block waits, through the same bounded mbarrier wait as the spectral MAC's
 * pipeline, on a barrier that nothing arrives on, for at most limit_cycles
 * SM clock cycles (1 .. 4e9; about 1 ms is 2e6 at 2 GHz).  The wait runs out,
 * sets the context's device error flag and the block exits: nothing faults
 * or hangs, and the next rp_sync returns RP_ERR_TIMEOUT and clears the flag,
 * leaving the context usable.  RP_ERR_ARG for a limit out of range.
 */
rp_status rp_selftest_wait(rp_ctx *ctx, long long limit_cycles);

/* rp_kernel_name -- short name of a kernel class (NULL if out of range). */
const char *rp_kernel_name(int kind);

/*
 * rp_save_state / rp_load_state -- write / read the history rings and the
 * step counter to / from a file, so that a run resumes with bit-identical
 * outputs.  Synchronous.  load requires a finalized context with the same
 * domains and configuration (RP_ERR_STATE otherwise).
 */
rp_status rp_save_state(rp_ctx *ctx, const char *path);
rp_status rp_load_state(rp_ctx *ctx, const char *path);

/* rp_destroy -- free everything (waits for the stream).  NULL is a no-op. */
void rp_destroy(rp_ctx *ctx);

/* rp_status_str -- static name of a status code. */
const char *rp_status_str(rp_status s);

/* rp_last_error -- one-line description of the context's last failure ("" if none). */
const char *rp_last_error(rp_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* RP_H */
