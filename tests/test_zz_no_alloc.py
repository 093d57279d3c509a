"""rp_evaluate_host_noalloc: the host-output evaluation that never allocates.

It stages phi and A in a fixed device array compiled into the library
instead of device memory allocated on first use, for callers whose device
memory belongs to another allocator or budget once a run has started.  These
checks call it through the C-ABI, twice in a row on consecutive steps, and
compare each call with rp_evaluate_host (the existing entry point) at the
same step, within the parity tolerance of the GPU tests.  This file is
collected last so that a run stopping at its first failure has already run
every other test; it also passes on its own in a fresh process.
"""
import numpy as np
import pytest

from paper_2311_15429_gb300 import rp, synth

pytestmark = pytest.mark.gpu
TOL = 1e-6


def _host_outputs(domains):
    bufs = [np.zeros(4 * d.N, np.float32) for d in domains]
    return bufs, [b[: d.N] for b, d in zip(bufs, domains)], [b[d.N:] for b, d in zip(bufs, domains)]


def _rel(a, b):
    return float(np.linalg.norm(a.astype(np.float64) - b) / max(np.linalg.norm(b.astype(np.float64)), 1e-300))


@pytest.mark.parametrize("geometry", ["cfg1", "mixed_spacing"])
def test_noalloc_matches_evaluate_host_on_two_calls(geometry):
    if geometry == "cfg1":
        w = synth.workload("cfg1")
        doms, srcs, c, dt = w.domains, w.sources, w.c, w.dt
    else:   # an FFT-path target with a direct-path pair added onto it
        doms = [synth.cubic((0.0, 0.0, 0.0), 12, 0.3), synth.cubic((9.0, 2.0, -1.0), 10, 0.25)]
        srcs, c, dt = synth.seeded_sources(doms), synth.C_AU, 0.05
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
            for a, b, d in zip(got, ref, doms):
                assert np.all(np.isfinite(a))
                for f in range(4):
                    sl = slice(f * d.N, (f + 1) * d.N)
                    assert _rel(a[sl], b[sl].astype(np.float64)) <= TOL, (i, f)
            checked += 1
        assert checked == 2
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
