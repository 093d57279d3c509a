"""rp_evaluate_host_noalloc: the host-output evaluation that never allocates.

It stages phi and A in a fixed device array compiled into the library
instead of device memory allocated on first use, for callers whose device
memory belongs to another allocator or budget once a run has started.  These
checks call it through the C-ABI, twice in a row on consecutive steps, and
compare each call with rp_evaluate_host (the existing entry point) at the
same step: both run the same kernels in the same order on the same stream,
so the outputs must be identical bit for bit.  One step is also checked
against the FP64 oracle, and a fresh context whose first output call is this
one must leave the free device memory and the context's own byte count
unchanged.  This file is collected last so that a run stopping at its first
failure has already run every other test; it also passes on its own in a
fresh process.
"""
import numpy as np
import pytest

import oracle
from paper_2311_15429_gb300 import rp, synth

pytestmark = pytest.mark.gpu
TOL = 1e-6


def _host_outputs(domains):
    bufs = [np.zeros(4 * d.N, np.float32) for d in domains]
    return bufs, [b[: d.N] for b, d in zip(bufs, domains)], [b[d.N:] for b, d in zip(bufs, domains)]


def _rel(a, b):
    return float(np.linalg.norm(a.astype(np.float64) - b) / max(np.linalg.norm(b.astype(np.float64)), 1e-300))


def _geometry(name):
    if name == "cfg1":
        w = synth.workload("cfg1")
        return w.domains, w.sources, w.c, w.dt
    # an FFT-path target with a direct-path pair added onto it
    doms = [synth.cubic((0.0, 0.0, 0.0), 12, 0.3), synth.cubic((9.0, 2.0, -1.0), 10, 0.25)]
    return doms, synth.seeded_sources(doms), synth.C_AU, 0.05


@pytest.mark.parametrize("geometry", ["cfg1", "mixed_spacing"])
def test_noalloc_matches_evaluate_host_on_two_calls(geometry):
    doms, srcs, c, dt = _geometry(geometry)
    T = 12
    hists = [s.history(0, T, dt) for s in srcs]
    ctx = rp.rp_create(c, dt)
    try:
        for d in doms:
            rp.rp_add_domain(ctx, d.origin, d.n, d.h)
        rp.rp_finalize(ctx)
        checked = 0
        for i in range(T):
            for dd in range(len(doms)):
                rp.rp_push_host(ctx, dd, np.ascontiguousarray(hists[dd][i, 0]),
                                np.ascontiguousarray(hists[dd][i, 1:]).reshape(-1))
                rp.rp_sync(ctx)
            if i < T - 2:
                continue
            ref, ref_phi, ref_A = _host_outputs(doms)
            rp.rp_evaluate_host(ctx, ref_phi, ref_A)
            rp.rp_sync(ctx)
            got, got_phi, got_A = _host_outputs(doms)
            rp.rp_evaluate_host_noalloc(ctx, got_phi, got_A)
            rp.rp_sync(ctx)
            for t, (a, b, d) in enumerate(zip(got, ref, doms)):
                assert np.all(np.isfinite(a))
                diag = max(_rel(a[f * d.N:(f + 1) * d.N], b[f * d.N:(f + 1) * d.N].astype(np.float64))
                           for f in range(4))
                assert np.array_equal(a, b), f"step {i} domain {t}: not bit-identical (rel-L2 {diag:.2e})"
                if i == T - 1:   # and the right numbers: the FP64 oracle at every node
                    want = oracle.eval_points([x.origin for x in doms], [x.n for x in doms], [x.h for x in doms],
                                              hists, 0, c, dt, t, i, np.arange(d.N))
                    for f in range(4):
                        assert _rel(a[f * d.N:(f + 1) * d.N], want[:, f]) <= TOL, (t, f)
            checked += 1
        assert checked == 2
    finally:
        rp.rp_destroy(ctx)


def test_noalloc_first_output_call_allocates_nothing():
    """A fresh context whose first output call is rp_evaluate_host_noalloc:
    the free device memory (cudaMemGetInfo) and the context's own device
    bytes are the same before and after it.  The kernels' code is loaded
    first by a throw-away context, so that lazy module loading does not
    count; the inputs and the check's outputs are allocated before the
    measurement."""
    import torch
    doms, srcs, c, dt = _geometry("cfg1")
    T = 6
    hists = [s.history(0, T, dt) for s in srcs]
    dev = torch.device("cuda", 0)
    rho = [[torch.from_numpy(np.ascontiguousarray(h[i, 0])).to(dev) for h in hists] for i in range(T)]
    J = [[torch.from_numpy(np.ascontiguousarray(h[i, 1:]).reshape(-1)).to(dev) for h in hists] for i in range(T)]
    phi = [torch.empty(d.N, device=dev) for d in doms]
    A = [torch.empty(3 * d.N, device=dev) for d in doms]
    for fresh in (False, True):
        ctx = rp.rp_create(c, dt, flags=rp.RP_FLAG_GROUND_STATE_CLAMP)
        try:
            for d in doms:
                rp.rp_add_domain(ctx, d.origin, d.n, d.h)
            rp.rp_finalize(ctx)
            for i in range(T):
                rp.rp_push_all(ctx, rho[i], J[i])
            if not fresh:   # loads every kernel of an evaluation once in this process
                rp.rp_evaluate(ctx, phi, A)
                got, got_phi, got_A = _host_outputs(doms)
                rp.rp_evaluate_host_noalloc(ctx, got_phi, got_A)
                rp.rp_sync(ctx)
                continue
            rp.rp_sync(ctx)
            torch.cuda.synchronize()
            free0, _ = torch.cuda.mem_get_info(dev)
            held0 = rp.rp_query(ctx)["device_bytes"]
            got, got_phi, got_A = _host_outputs(doms)
            rp.rp_evaluate_host_noalloc(ctx, got_phi, got_A)
            rp.rp_sync(ctx)
            free1, _ = torch.cuda.mem_get_info(dev)
            held1 = rp.rp_query(ctx)["device_bytes"]
            assert free1 == free0, f"free device memory moved by {free0 - free1} B"
            assert held1 == held0
            rp.rp_evaluate(ctx, phi, A)
            rp.rp_sync(ctx)
            for t, d in enumerate(doms):
                ref = torch.cat([phi[t], A[t]]).cpu().numpy()
                assert np.array_equal(got[t], ref), f"domain {t}: not bit-identical to rp_evaluate"
        finally:
            rp.rp_destroy(ctx)


def test_noalloc_rejects_domains_beyond_its_fixed_array():
    """96^3 + 64^3 = 1,146,880 points exceed the 1,048,576 the array holds."""
    doms = [synth.cubic((0.0, 0.0, 0.0), 96, 0.3), synth.cubic((60.0, 0.0, 0.0), 64, 0.3)]
    ctx = rp.rp_create(synth.C_AU, 0.05, flags=rp.RP_FLAG_GROUND_STATE_CLAMP)
    try:
        for d in doms:
            rp.rp_add_domain(ctx, d.origin, d.n, d.h)
        rp.rp_finalize(ctx)
        bufs, phis, As = _host_outputs(doms)
        z = [np.zeros(d.N, np.float32) for d in doms]
        zJ = [np.zeros(3 * d.N, np.float32) for d in doms]
        for dd in range(2):
            rp.rp_push_host(ctx, dd, z[dd], zJ[dd])
        rp.rp_sync(ctx)
        with pytest.raises(rp.RPError) as e:
            rp.rp_evaluate_host_noalloc(ctx, phis, As)
        assert e.value.status == rp.RP_ERR_UNSUPPORTED
        rp.rp_sync(ctx)
    finally:
        rp.rp_destroy(ctx)
