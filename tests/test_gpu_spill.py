"""GPU: the history spill to host memory (RP_FLAG_HISTORY_SPILL).

Sec. IV keeps every sample of [l - N_R,max, l] while a step reads only each
pair's Delta N_R of them.  With the flag, a pair whose lag window starts far
back reads its source spectra from a small device window ring; the source's
(rho, J) slices go to a pinned host ring and come back, one a step, through
the same forward passes as a push.  The kernels and their summation order do
not change, so the spilled context must reproduce the unspilled one bit for
bit, whatever the call pattern (per-domain pushes, skipped evaluations, the
ground-state split, a saved and reloaded state).
"""
import os
import tempfile

import numpy as np
import pytest

from paper_2311_15429_gb300 import rp, synth

from _harness import histories, oracle_values, rel_l2, run_library

pytestmark = pytest.mark.gpu
SPILL = rp.RP_FLAG_HISTORY_SPILL
CLAMP = rp.RP_FLAG_GROUND_STATE_CLAMP
SPLIT = rp.RP_FLAG_GROUND_STATE_SPLIT


def two_far():
    """2 x 16^3 at 205 bohr: cross lags 29..31 (window ring of 3 slots)."""
    return synth.two_domain(16, 0.25, 205.0)


def three_mixed():
    """A near pair (8 bohr, lags from 0, stays on the device) and a third
    domain 205 bohr away whose two cross windows per target spill."""
    doms = [synth.cubic((-100.0, 0.0, 0.0), 16, 0.25), synth.cubic((-92.0, 0.5, 0.0), 16, 0.25),
            synth.cubic((105.0, 0.0, -0.5), 16, 0.25)]
    return synth.Workload("three", doms, synth.C_AU, 0.05, 0, 8, "3 x 16^3, near pair + far domain",
                          synth.seeded_sources(doms))


def query(w, flags):
    ctx = rp.rp_create(w.c, w.dt, 0, rp.RP_MODE_FFT, rp.RP_FLAG_PLAN_ONLY | flags)
    try:
        for d in w.domains:
            rp.rp_add_domain(ctx, d.origin, d.n, d.h)
        rp.rp_finalize(ctx)
        return rp.rp_query(ctx)
    finally:
        rp.rp_destroy(ctx)


def assert_same(a, b):
    assert a.keys() == b.keys()
    for j in a:
        for x, y in zip(a[j], b[j]):
            np.testing.assert_array_equal(x, y, err_msg=f"step {j}")


@pytest.mark.parametrize("geom", ["two", "three"])
@pytest.mark.parametrize("push", ["all", "each"])
def test_spill_is_bit_identical_from_step_zero(geom, push):
    """Clamped histories, every step evaluated from step 0 through twice the
    deepest lag: the spilled context equals the unspilled one exactly."""
    w = two_far() if geom == "two" else three_mixed()
    q = query(w, SPILL)
    assert q["spill_windows"] == (2 if geom == "two" else 4)
    assert q["spectral_bytes"] < query(w, 0)["spectral_bytes"]
    T = 2 * q["max_lag"] + 6
    hists = histories(w.sources, 0, T, w.dt)
    steps = range(T)
    ref = run_library(w.domains, w.c, w.dt, hists, 0, steps, flags=CLAMP, push=push)
    got = run_library(w.domains, w.c, w.dt, hists, 0, steps, flags=CLAMP | SPILL, push=push)
    assert_same(got, ref)


def test_spill_with_skipped_evaluations_and_oracle():
    """Without the clamp (first evaluation at the deepest lag) and with
    evaluations skipped in runs longer than a window ring, so that windows are
    refilled from the host instead of one slot a step; then the FP64 oracle
    on the spilled context's output."""
    w = two_far()
    q = query(w, SPILL)
    L = q["max_lag"]
    T = 3 * L
    hists = histories(w.sources, 0, T, w.dt)
    steps = [L, L + 1, L + 2, L + 9, L + 10, L + 17, 2 * L + 3, 2 * L + 4, 3 * L - 1]
    ref = run_library(w.domains, w.c, w.dt, hists, 0, steps)
    got = run_library(w.domains, w.c, w.dt, hists, 0, steps, flags=SPILL)
    assert_same(got, ref)
    step = 3 * L - 1
    nodes = np.random.default_rng(7).choice(w.domains[0].N, 64, replace=False)
    for t in range(2):
        want = oracle_values(w.domains, hists, 0, w.c, w.dt, t, step, nodes)
        assert max(rel_l2(got[step][t][:, nodes].astype(np.float64), want)) <= 1e-6


def test_spill_with_ground_state_split():
    """The split zeroes the history of step 0 after the static potential:
    with the spill the host copy and the windows follow, so induced parts and
    P(0) equal those of the unspilled split context exactly."""
    import torch
    dev = torch.device("cuda", 0)
    w = two_far()
    T = 2 * query(w, SPILL)["max_lag"] + 4
    hists = histories(w.sources, 0, T, w.dt)

    def run(flags):
        out = []
        with rp.RetardedPotentials(w.domains, w.c, w.dt, flags=flags) as lib:
            ph = [torch.empty(d.N, device=dev) for d in w.domains]
            Ag = [torch.empty(3 * d.N, device=dev) for d in w.domains]
            for i in range(T):
                lib.push_all([torch.from_numpy(np.ascontiguousarray(h[i, 0])).to(dev) for h in hists],
                              [torch.from_numpy(np.ascontiguousarray(h[i, 1:]).reshape(-1)).to(dev) for h in hists])
                phi, A = lib.evaluate()
                torch.cuda.synchronize()
                out.append([np.concatenate([phi[d].cpu().numpy(), A[d].cpu().numpy()]) for d in range(2)])
            rp.rp_ground_potential(lib.ctx, ph, Ag)
            torch.cuda.synchronize()
            out.append([np.concatenate([ph[d].cpu().numpy(), Ag[d].cpu().numpy()]) for d in range(2)])
        return out

    ref, got = run(SPLIT), run(SPLIT | SPILL)
    for i, (x, y) in enumerate(zip(got, ref)):
        for d in range(2):
            np.testing.assert_array_equal(x[d], y[d], err_msg=f"entry {i}")
    assert np.all(got[0][0] == 0)   # the induced part of step 0


def test_spill_state_round_trip_and_graph_refusal():
    """A saved spilled context (device rings and the host history) resumes
    bit-identically, mid-window; the state does not load into an unspilled
    context; rp_graph_capture is refused."""
    import torch
    dev = torch.device("cuda", 0)
    w = two_far()
    L = query(w, SPILL)["max_lag"]
    T = 2 * L + 5
    k = L + 3
    hists = histories(w.sources, 0, T, w.dt)
    sl = lambda i: ([torch.from_numpy(np.ascontiguousarray(h[i, 0])).to(dev) for h in hists],
                    [torch.from_numpy(np.ascontiguousarray(h[i, 1:]).reshape(-1)).to(dev) for h in hists])
    path = os.path.join(tempfile.mkdtemp(), "spill.state")
    want = []
    with rp.RetardedPotentials(w.domains, w.c, w.dt, flags=SPILL) as a:
        for i in range(k):
            a.push_all(*sl(i))
            if i >= L:
                a.evaluate()
        a.sync()
        rp.rp_save_state(a.ctx, path)
        for i in range(k, T):
            a.push_all(*sl(i))
            phi, A = a.evaluate()
            want.append([(phi[d].cpu().numpy().copy(), A[d].cpu().numpy().copy()) for d in range(2)])
        bufs = ([torch.empty(d.N, device=dev) for d in w.domains], [torch.empty(3 * d.N, device=dev) for d in w.domains])
        with pytest.raises(rp.RPError) as e:
            rp.rp_graph_capture(a.ctx, *sl(0), *bufs)
        assert e.value.status == rp.RP_ERR_UNSUPPORTED
    with rp.RetardedPotentials(w.domains, w.c, w.dt) as plain:
        with pytest.raises(rp.RPError) as e:
            rp.rp_load_state(plain.ctx, path)
        assert e.value.status == rp.RP_ERR_STATE
    with rp.RetardedPotentials(w.domains, w.c, w.dt, flags=SPILL) as b:
        rp.rp_load_state(b.ctx, path)
        for n, i in enumerate(range(k, T)):
            b.push_all(*sl(i))
            phi, A = b.evaluate()
            for d in range(2):
                np.testing.assert_array_equal(phi[d].cpu().numpy(), want[n][d][0])
                np.testing.assert_array_equal(A[d].cpu().numpy(), want[n][d][1])


def test_spill_double_evaluation_and_profiling():
    """Evaluating a step twice fetches nothing the second time and gives the
    same result; under RP_FLAG_PROFILE the window transforms are timed and
    counted with the forward passes (the first evaluation fills each window by
    its own launches, later steps ride on the push's launches), and the
    results do not change."""
    import torch
    dev = torch.device("cuda", 0)
    w = two_far()
    L = query(w, SPILL)["max_lag"]
    T = L + 8
    hists = histories(w.sources, 0, T, w.dt)
    ref = run_library(w.domains, w.c, w.dt, hists, 0, range(L, T))
    got = {}
    with rp.RetardedPotentials(w.domains, w.c, w.dt, flags=SPILL | rp.RP_FLAG_PROFILE) as lib:
        for i in range(T):
            lib.push_all([torch.from_numpy(np.ascontiguousarray(h[i, 0])).to(dev) for h in hists],
                         [torch.from_numpy(np.ascontiguousarray(h[i, 1:]).reshape(-1)).to(dev) for h in hists])
            if i < L:
                continue
            outs = []
            for _ in range(2):
                phi, A = lib.evaluate()
                torch.cuda.synchronize()
                outs.append([np.concatenate([phi[d].cpu().numpy()[None], A[d].cpu().numpy().reshape(3, -1)])
                             for d in range(2)])
            for d in range(2):
                np.testing.assert_array_equal(outs[0][d], outs[1][d])
            got[i] = outs[1]
        lib.sync()
        n_push, _ = rp.rp_kernel_stats(lib.ctx, rp.RP_K_FWD_COLUMN)[:2]
    assert_same(got, ref)
    # one column pass per push (one size class), plus the first evaluation's
    # fill of B steps for each of the two windows; every later window step
    # rides on its push
    ctx = rp.rp_create(w.c, w.dt, 0, rp.RP_MODE_FFT, rp.RP_FLAG_PLAN_ONLY | SPILL)
    try:
        for d in w.domains:
            rp.rp_add_domain(ctx, d.origin, d.n, d.h)
        rp.rp_finalize(ctx)
        p = rp.rp_pair_info(ctx, 0, 1)
    finally:
        rp.rp_destroy(ctx)
    assert n_push == T + 2 * (p["lag_hi"] - p["lag_lo"] + 1)


def test_spill_with_lowrank_far_pairs():
    """RP_MODE_LOWRANK with the spill: two domains 150 bohr apart (their cross
    windows at lags 21-23 spill) and a third about 900 bohr away (four far
    pairs on the factors, whose bf16 source rows are staged by the same
    forward plane pass that now also transforms the windows).  Equal to the
    unspilled context bit for bit, steps from the deepest lag on."""
    import torch
    dev = torch.device("cuda", 0)
    doms = [synth.cubic((0.0, 0.0, 0.0), 12, 0.25), synth.cubic((150.0, 0.5, -0.3), 12, 0.25),
            synth.cubic((900.0, 50.0, -30.0), 12, 0.25)]
    srcs = synth.seeded_sources(doms)
    T = 160
    hists = [s.history(0, T, 0.05) for s in srcs]

    def run(flags):
        out = {}
        with rp.RetardedPotentials(doms, synth.C_AU, 0.05, mode=rp.RP_MODE_LOWRANK, flags=flags,
                                   far_distance=400.0, far_batch=16) as lib:
            q = lib.query()
            for i in range(T):
                lib.push_all([torch.from_numpy(h[i, 0].copy()).to(dev) for h in hists],
                             [torch.from_numpy(h[i, 1:].copy().reshape(-1)).to(dev) for h in hists])
                if i >= q["max_lag"]:
                    phi, A = lib.evaluate()
                    torch.cuda.synchronize()
                    out[i] = [np.concatenate([phi[d].cpu().numpy()[None], A[d].cpu().numpy().reshape(3, -1)])
                              for d in range(3)]
            lib.sync()
        return out, q

    ref, q0 = run(0)
    got, q1 = run(SPILL)
    assert q0["npairs_far"] == q1["npairs_far"] == 4
    assert q1["spill_windows"] == 2 and q0["spill_windows"] == 0
    assert_same(got, ref)
