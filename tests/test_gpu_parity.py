"""GPU parity: the CUDA path through the C-ABI against the FP64 oracle.

The bar is the FP32 path's: rel-L2 <= 1e-6 per (field, target domain),
pooled over the checked steps, with inputs rounded to FP32 for both sides.
"""
import numpy as np
import pytest

from paper_2311_15429_gb300 import rp, synth

from _harness import histories, oracle_values, rel_l2, run_library

pytestmark = pytest.mark.gpu
TOL = 1e-6


def _score(domains, hists, j0, c, dt, results, nodes=None, clamp=False):
    worst = 0.0
    for step, outs in results.items():
        for t, d in enumerate(domains):
            sel = np.arange(d.N) if nodes is None else nodes[t]
            want = oracle_values(domains, hists, j0, c, dt, t, step, sel, clamp=clamp)
            errs = rel_l2(outs[t][:, sel], want)
            worst = max(worst, max(errs))
            assert max(errs) <= TOL, (step, t, errs)
    return worst


@pytest.mark.parametrize("mode", [rp.RP_MODE_FFT, rp.RP_MODE_DIRECT])
def test_cfg1_full_grids(mode):
    """2 x 16^3, h = 0.3, 20 bohr apart, 64-step history, last 8 steps, every node."""
    w = synth.workload("cfg1")
    hists = histories(w.sources, 0, 64, w.dt)
    res = run_library(w.domains, w.c, w.dt, hists, 0, range(56, 64), mode=mode)
    _score(w.domains, hists, 0, w.c, w.dt, res)


def test_tma_mac_path_is_active():
    """Cubic targets (padded 32..192) use the TMA-fed spectral MAC."""
    w = synth.workload("cfg1")
    with rp.RetardedPotentials(w.domains, w.c, w.dt) as lib:
        q = lib.query()
        assert q["mac_tma"] == 1, rp.rp_last_error(lib.ctx)


def test_ragged_grids_fft():
    """Non-cubic, unequal grids (FFT sizes 12/16/... with ragged tails)."""
    doms = [synth.Domain((0.0, 0.0, 0.0), (7, 5, 6), 0.3), synth.Domain((3.1, -0.7, 0.4), (4, 9, 3), 0.3),
            synth.Domain((-2.0, 4.0, 1.5), (11, 3, 13), 0.3)]
    srcs = synth.seeded_sources(doms)
    hists = histories(srcs, 0, 12, 0.05)
    res = run_library(doms, synth.C_AU, 0.05, hists, 0, [10, 11])
    _score(doms, hists, 0, synth.C_AU, 0.05, res)


def test_mixed_spacing_direct_fallback():
    """A pair of unequal spacing goes through the direct kernel and adds onto
    the FFT result of the target's other pairs."""
    doms = [synth.cubic((0.0, 0.0, 0.0), 12, 0.3), synth.cubic((9.0, 2.0, -1.0), 10, 0.25),
            synth.cubic((-8.0, 0.0, 3.0), 9, 0.3)]
    srcs = synth.seeded_sources(doms)
    hists = histories(srcs, 0, 16, 0.05)
    res = run_library(doms, synth.C_AU, 0.05, hists, 0, [15], push="each")
    _score(doms, hists, 0, synth.C_AU, 0.05, res)


def test_slow_light_many_lags():
    """c = 5 a.u.: every pair spans tens of delay bins."""
    doms = [synth.cubic((0.0, 0.0, 0.0), 10, 0.3), synth.cubic((6.0, 1.0, 0.0), 10, 0.3)]
    srcs = synth.seeded_sources(doms)
    c, dt = 5.0, 0.05
    hists = histories(srcs, 0, 60, dt)
    res = run_library(doms, c, dt, hists, 0, [58, 59])
    _score(doms, hists, 0, c, dt, res)


def test_cfg2_full_size_sampled():
    """2 x 48^3, 2000 bohr apart, 320-step ring (cross delays 290..294 steps):
    the bench's workload in its launch configuration, checked on sampled nodes
    (corners, centre and 60 seeded random nodes per domain)."""
    w = synth.workload("cfg2")
    pre = 295
    j0, j1 = -pre, 3
    hists = histories(w.sources, j0, j1, w.dt)
    res = run_library(w.domains, w.c, w.dt, hists, j0, [1, 2], depth=w.history)
    rng = np.random.default_rng(4)
    nodes = []
    for d in w.domains:
        n = d.n[0]
        corners = [i + n * (j + n * k) for i in (0, n - 1) for j in (0, n - 1) for k in (0, n - 1)]
        centre = [n // 2 + n * (n // 2 + n * (n // 2))]
        nodes.append(np.array(corners + centre + list(rng.integers(0, d.N, 60))))
    _score(w.domains, hists, j0, w.c, w.dt, res, nodes=nodes)


@pytest.mark.parametrize("n", [24, 32, 64, 96])
def test_cubic_size_classes(n):
    """Two n^3 domains 30 bohr apart: padded sizes 48, 64, 128 and 192 (the
    compiled-shape kernels), checked at corners, centre and seeded nodes."""
    w = synth.two_domain(n, 0.25, 30.0, f"cube{n}", offset=(3.0, -2.0))
    T = 16
    hists = histories(w.sources, 0, T, w.dt)
    res = run_library(w.domains, w.c, w.dt, hists, 0, [T - 2, T - 1])
    rng = np.random.default_rng(n)
    nodes = []
    for d in w.domains:
        corners = [i + n * (j + n * k) for i in (0, n - 1) for j in (0, n - 1) for k in (0, n - 1)]
        nodes.append(np.array(corners + [n // 2 + n * (n // 2 + n * (n // 2))] + list(rng.integers(0, d.N, 40))))
    _score(w.domains, hists, 0, w.c, w.dt, res, nodes=nodes)


def test_many_planes_lane_shuffle_form():
    """Nine 32^3 domains (padded 64^3, 1152 plane blocks per pass: above the
    1024 up to which the planner keeps the tile-transform plane passes), so
    the forward and inverse plane passes run the lane-shuffle form; checked
    against the oracle on every target at its corners and seeded nodes."""
    n, h = 32, 0.25
    doms = [synth.cubic((12.0 * i, 12.0 * j, 0.5 * i), n, h) for i in range(3) for j in range(3)]
    srcs = synth.seeded_sources(doms)
    T = 12
    hists = [s.history(0, T, 0.05) for s in srcs]
    res = run_library(doms, synth.C_AU, 0.05, hists, 0, [T - 1])
    rng = np.random.default_rng(9)
    corners = [i + n * (j + n * k) for i in (0, n - 1) for j in (0, n - 1) for k in (0, n - 1)]
    nodes = [np.array(corners + list(rng.integers(0, d.N, 24))) for d in doms]
    _score(doms, hists, 0, synth.C_AU, 0.05, res, nodes=nodes)


def test_ground_state_clamp():
    """Under RP_FLAG_GROUND_STATE_CLAMP, samples before the first push equal it."""
    w = synth.workload("cfg1")
    hists = histories(w.sources, 0, 4, w.dt)
    res = run_library(w.domains, w.c, w.dt, hists, 0, [0, 1, 3], flags=rp.RP_FLAG_GROUND_STATE_CLAMP)
    _score(w.domains, hists, 0, w.c, w.dt, res, clamp=True)


def test_single_node_domain_and_zero_source():
    """A 1x1x1 domain (its self term is just C h^2 rho) beside a normal one; an
    all-zero source gives exactly zero from that source."""
    doms = [synth.Domain((5.0, 0.0, 0.0), (1, 1, 1), 0.4), synth.cubic((0.0, 0.0, 0.0), 6, 0.4)]
    rng = np.random.default_rng(2)
    T = 8
    hists = [rng.standard_normal((T, 4, 1)).astype(np.float32), np.zeros((T, 4, 216), np.float32)]
    res = run_library(doms, synth.C_AU, 0.05, hists, 0, [T - 1])
    _score(doms, hists, 0, synth.C_AU, 0.05, res)
    C = 3 * np.log(2 + np.sqrt(3)) - np.pi / 2
    out0 = res[T - 1][0][:, 0]
    want = C * 0.4 ** 2 * hists[0][T - 1, :, 0].astype(np.float64)
    want[1:] /= synth.C_AU
    np.testing.assert_allclose(out0, want, rtol=1e-6)


def test_push_paths_agree_bitwise():
    """rp_push per domain, rp_push_all and rp_push_host / rp_evaluate_host give
    identical bits."""
    import torch
    w = synth.workload("cfg1")
    hists = histories(w.sources, 0, 10, w.dt)
    a = run_library(w.domains, w.c, w.dt, hists, 0, [9], push="all")[9]
    b = run_library(w.domains, w.c, w.dt, hists, 0, [9], push="each")[9]
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)
    ctx = rp.rp_create(w.c, w.dt)
    try:
        for d in w.domains:
            rp.rp_add_domain(ctx, d.origin, d.n, d.h)
        rp.rp_finalize(ctx)
        outs = [np.zeros(4 * d.N, np.float32) for d in w.domains]
        for i in range(10):
            for dd in range(2):
                rho = np.ascontiguousarray(hists[dd][i, 0])
                J = np.ascontiguousarray(hists[dd][i, 1:]).reshape(-1)
                rp.rp_push_host(ctx, dd, rho, J)
                rp.rp_sync(ctx)
        phis = [o[: d.N] for o, d in zip(outs, w.domains)]
        As = [o[d.N:] for o, d in zip(outs, w.domains)]
        rp.rp_evaluate_host(ctx, phis, As)
        rp.rp_sync(ctx)
    finally:
        rp.rp_destroy(ctx)
    for x, o in zip(a, outs):
        np.testing.assert_array_equal(x.reshape(-1), o)


def test_state_errors_and_history():
    import torch
    w = synth.workload("cfg1")
    dev = torch.device("cuda", 0)
    with rp.RetardedPotentials(w.domains, w.c, w.dt) as lib:
        x = [torch.zeros(d.N, device=dev) for d in w.domains]
        J = [torch.zeros(3 * d.N, device=dev) for d in w.domains]
        with pytest.raises(rp.RPError) as e:
            lib.evaluate()                                   # nothing pushed
        assert e.value.status == rp.RP_ERR_STATE
        lib.push(0, x[0], J[0])
        with pytest.raises(rp.RPError) as e:
            lib.push(0, x[0], J[0])                          # twice in one step
        assert e.value.status == rp.RP_ERR_STATE
        with pytest.raises(rp.RPError) as e:
            lib.evaluate()                                   # domain 1 missing
        assert e.value.status == rp.RP_ERR_STATE
        lib.push(1, x[1], J[1])
        with pytest.raises(rp.RPError) as e:
            lib.evaluate()                                   # needs 4 steps of history
        assert e.value.status == rp.RP_ERR_HISTORY
        lib.sync()


def test_checkpoint_resume_bitwise(tmp_path):
    import torch
    w = synth.workload("cfg1")
    hists = histories(w.sources, 0, 14, w.dt)
    dev = torch.device("cuda", 0)

    def push(lib, i):
        lib.push_all([torch.from_numpy(h[i, 0].copy()).to(dev) for h in hists],
                     [torch.from_numpy(h[i, 1:].copy().reshape(-1)).to(dev) for h in hists])

    path = str(tmp_path / "state.bin")
    with rp.RetardedPotentials(w.domains, w.c, w.dt) as lib:
        for i in range(10):
            push(lib, i)
        rp.rp_save_state(lib.ctx, path)
        for i in range(10, 14):
            push(lib, i)
        ref = [t.cpu().numpy().copy() for t in lib.evaluate()[0]]
    with rp.RetardedPotentials(w.domains, w.c, w.dt) as lib:
        rp.rp_load_state(lib.ctx, path)
        assert lib.query()["step"] == 9
        for i in range(10, 14):
            push(lib, i)
        got = [t.cpu().numpy() for t in lib.evaluate()[0]]
    for a, b in zip(ref, got):
        np.testing.assert_array_equal(a, b)


def test_contexts_coexist():
    """A direct-mode context finalized after an FFT-mode one does not affect
    it (kernel attributes are process-wide), and both stay correct."""
    w = synth.workload("cfg1")
    hists = histories(w.sources, 0, 8, w.dt)
    import torch
    dev = torch.device("cuda", 0)
    a = rp.RetardedPotentials(w.domains, w.c, w.dt, mode=rp.RP_MODE_FFT)
    b = rp.RetardedPotentials(w.domains, w.c, w.dt, mode=rp.RP_MODE_DIRECT)
    try:
        for i in range(8):
            r = [torch.from_numpy(h[i, 0].copy()).to(dev) for h in hists]
            J = [torch.from_numpy(h[i, 1:].copy().reshape(-1)).to(dev) for h in hists]
            a.push(0, r[0], J[0]); a.push(1, r[1], J[1])
            b.push_all(r, J)
        for lib in (a, b):
            phi, A = lib.evaluate()
            torch.cuda.synchronize()
            for t, d in enumerate(w.domains):
                got = np.concatenate([phi[t].cpu().numpy()[None], A[t].cpu().numpy().reshape(3, -1)])
                want = oracle_values(w.domains, hists, 0, w.c, w.dt, t, 7, np.arange(d.N))
                assert max(rel_l2(got, want)) <= TOL
    finally:
        a.close()
        b.close()


@pytest.mark.parametrize("n", [16, 24, 48])
def test_mac_variants_agree_bitwise(n):
    """The consumer-warp variants of the TMA-fed MAC (8, 12, 16) sum the same
    terms in the same order: bitwise equal outputs, and the autotuned choice
    is one of them.  Padded sizes 32, 48 and 96."""
    w = synth.two_domain(n, 0.25, 3.0 * n * 0.25, f"variants{n}", offset=(1.0, 0.5))
    T = 10
    hists = histories(w.sources, 0, T, w.dt)
    outs = {cw: run_library(w.domains, w.c, w.dt, hists, 0, [T - 1], mac_warps=cw) for cw in (8, 12, 16)}
    for cw in (8, 12):
        for t in range(2):
            assert np.array_equal(outs[cw][T - 1][t], outs[16][T - 1][t]), (cw, t)
    with rp.RetardedPotentials(w.domains, w.c, w.dt) as lib:
        q = lib.query()
        assert q["mac_tma"] == 1 and q["mac_warps"] in (8, 12, 16), q
    _score(w.domains, hists, 0, w.c, w.dt, outs[12], nodes=[np.arange(0, d.N, 97) for d in w.domains])


def test_sampled_kernel_timing():
    """profile_every = 4: every launch is counted, only those of steps
    s % 4 == 0 are timed; results are unchanged by the sampling."""
    import torch
    w = synth.workload("cfg1")
    hists = histories(w.sources, 0, 24, w.dt)
    dev = torch.device("cuda", 0)
    outs = {}
    for every in (0, 4):
        flags = rp.RP_FLAG_PROFILE | rp.RP_FLAG_GROUND_STATE_CLAMP
        with rp.RetardedPotentials(w.domains, w.c, w.dt, history_depth=64, flags=flags,
                                   profile_every=every) as lib:
            for i in range(24):
                lib.push_all([torch.from_numpy(h[i, 0].copy()).to(dev) for h in hists],
                             [torch.from_numpy(h[i, 1:].copy().reshape(-1)).to(dev) for h in hists])
                if i == 0:
                    rp.rp_kernel_stats(lib.ctx, 0, reset=True)   # after finalize-time launches
                    continue
                lib.evaluate()
            torch.cuda.synchronize()
            outs[every] = [lib.phi[t].cpu().numpy().copy() for t in range(len(w.domains))]
            for kind in (rp.RP_K_MAC_INV_COLUMN, rp.RP_K_INV_PLANE):
                n_timed, ms = rp.rp_kernel_stats(lib.ctx, kind)
                n_all = rp.rp_kernel_count(lib.ctx, kind)
                assert n_all == 23, (kind, n_all)               # steps 1 .. 23 evaluated
                assert n_timed == (23 if every == 0 else 5), (kind, n_timed)   # 4, 8, .., 20
                assert ms > 0.0
    for a, b in zip(outs[0], outs[4]):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("adjacent,push_all", [(True, False), (False, False), (True, True)])
def test_host_path_pipelined_steps(adjacent, push_all):
    """rp_push_host / rp_evaluate_host on consecutive steps with no rp_sync in
    between (the copies run on the context's copy stream, staging alternates
    by step): every step's host results equal the device path's bits.
    adjacent: rho/J and phi/A in one pinned buffer each (one copy), else in
    separate pinned buffers (two copies).  push_all: rp_push_all_host with
    pointer arrays made once per step, else rp_push_host per domain."""
    import torch
    w = synth.workload("cfg1")
    T, first = 14, 6
    hists = histories(w.sources, 0, T, w.dt)
    want = run_library(w.domains, w.c, w.dt, hists, 0, range(first, T), push="all")
    nd = len(w.domains)
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    if adjacent:
        hin = [[pin(hists[d][i]) for d in range(nd)] for i in range(T)]     # [4][N] per (step, domain)
        rhos = [[hin[i][d][0] for d in range(nd)] for i in range(T)]
        Js = [[hin[i][d][1:].reshape(-1) for d in range(nd)] for i in range(T)]
        hout = {i: [torch.zeros(4 * dd.N).pin_memory() for dd in w.domains] for i in range(first, T)}
        phis = {i: [hout[i][d][: w.domains[d].N] for d in range(nd)] for i in hout}
        As = {i: [hout[i][d][w.domains[d].N:] for d in range(nd)] for i in hout}
    else:
        rhos = [[pin(hists[d][i, 0]) for d in range(nd)] for i in range(T)]
        Js = [[pin(hists[d][i, 1:].reshape(-1)) for d in range(nd)] for i in range(T)]
        phis = {i: [torch.zeros(dd.N).pin_memory() for dd in w.domains] for i in range(first, T)}
        As = {i: [torch.zeros(3 * dd.N).pin_memory() for dd in w.domains] for i in range(first, T)}
    ctx = rp.rp_create(w.c, w.dt)
    try:
        for d in w.domains:
            rp.rp_add_domain(ctx, d.origin, d.n, d.h)
        rp.rp_finalize(ctx)
        for i in range(T):
            if push_all:
                rp.rp_push_all_host(ctx, rp.pointer_array(rhos[i]), rp.pointer_array(Js[i]))
            else:
                for d in range(nd):
                    rp.rp_push_host(ctx, d, rhos[i][d], Js[i][d])
            if i >= first:
                rp.rp_evaluate_host(ctx, phis[i], As[i])
        rp.rp_sync(ctx)
    finally:
        rp.rp_destroy(ctx)
    for i in range(first, T):
        for d in range(nd):
            got = np.concatenate([phis[i][d].numpy(), As[i][d].numpy()])
            np.testing.assert_array_equal(got, want[i][d].reshape(-1), err_msg=f"step {i} domain {d}")


def test_inputs_and_outputs_next_to_other_kernels():
    """The per-step kernels start early (programmatic dependent launch) and
    wait for the previous kernel before touching its data: inputs written by
    a kernel on the same stream just before each push, and outputs read by a
    kernel just after each evaluation, give the bits of the plain run."""
    import torch
    w = synth.workload("cfg1")
    T = 12
    hists = histories(w.sources, 0, T, w.dt)
    want = run_library(w.domains, w.c, w.dt, hists, 0, range(6, T), push="all")
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    got = {}
    with rp.RetardedPotentials(w.domains, w.c, w.dt, stream=stream) as lib:
        host = [torch.from_numpy(np.ascontiguousarray(h)).to(dev) for h in hists]   # [T][4][N]
        rho = [torch.empty(d.N, device=dev) for d in w.domains]
        J = [torch.empty(3 * d.N, device=dev) for d in w.domains]
        for i in range(T):
            for d in range(len(w.domains)):
                # a long elementwise kernel writes this step's inputs
                torch.mul(host[d][i, 0], 1.0, out=rho[d])
                torch.mul(host[d][i, 1:].reshape(-1), 1.0, out=J[d])
            lib.push_all(rho, J)
            if i >= 6:
                phi, A = lib.evaluate()
                # kernels read the outputs right away, before any host sync
                got[i] = [torch.cat([phi[d][None] * 1.0, (A[d] * 1.0).reshape(3, -1)]) for d in range(len(w.domains))]
        torch.cuda.synchronize()
        for i in got:
            for d in range(len(w.domains)):
                np.testing.assert_array_equal(got[i][d].cpu().numpy(), want[i][d], err_msg=f"step {i} domain {d}")


def test_bounded_wait_runs_out_and_the_context_stays_usable():
    """A device wait that nothing satisfies (rp_selftest_wait, through the
    MAC pipeline's bounded mbarrier wait, ~1 ms limit) ends by itself: rp_sync
    reports RP_ERR_TIMEOUT once, clears it, and the next steps still match the
    plain run bit for bit."""
    import torch
    dev = torch.device("cuda", 0)
    w = synth.workload("cfg1")
    T = 10
    hists = histories(w.sources, 0, T, w.dt)
    want = run_library(w.domains, w.c, w.dt, hists, 0, [T - 1])
    with rp.RetardedPotentials(w.domains, w.c, w.dt) as lib:
        with pytest.raises(rp.RPError) as e:
            rp.rp_selftest_wait(lib.ctx, 0)
        assert e.value.status == rp.RP_ERR_ARG
        rp.rp_selftest_wait(lib.ctx, 2_000_000)
        with pytest.raises(rp.RPError) as e:
            lib.sync()
        assert e.value.status == rp.RP_ERR_TIMEOUT
        lib.sync()                                   # the flag was cleared
        for i in range(T):
            lib.push_all([torch.from_numpy(np.ascontiguousarray(h[i, 0])).to(dev) for h in hists],
                         [torch.from_numpy(np.ascontiguousarray(h[i, 1:]).reshape(-1)).to(dev) for h in hists])
        phi, A = lib.evaluate()
        lib.sync()
        for d in range(2):
            got = np.concatenate([phi[d].cpu().numpy()[None], A[d].cpu().numpy().reshape(3, -1)])
            np.testing.assert_array_equal(got, want[T - 1][d])


@pytest.mark.parametrize("mode", [rp.RP_MODE_FFT, rp.RP_MODE_DIRECT])
def test_graph_replay_matches_the_calls(mode):
    """rp_graph_capture records push_all + evaluate on fixed buffers; each
    rp_graph_step replays it (one launch) and gives the bits of the plain
    calls, also after a step made by the plain calls in between (the device
    step counter is re-synchronised)."""
    import torch
    dev = torch.device("cuda", 0)
    w = synth.workload("cfg1")
    T, pre = 16, 6
    hists = histories(w.sources, 0, T, w.dt)
    want = run_library(w.domains, w.c, w.dt, hists, 0, range(pre, T), mode=mode)
    slices = [[torch.from_numpy(np.ascontiguousarray(h[i])).to(dev) for h in hists] for i in range(T)]
    with rp.RetardedPotentials(w.domains, w.c, w.dt, mode=mode) as lib:
        with pytest.raises(rp.RPError) as e:
            rp.rp_graph_step(lib.ctx)
        assert e.value.status == rp.RP_ERR_STATE
        rho = [torch.empty(d.N, device=dev) for d in w.domains]
        J = [torch.empty(3 * d.N, device=dev) for d in w.domains]
        phi = [torch.empty(d.N, device=dev) for d in w.domains]
        A = [torch.empty(3 * d.N, device=dev) for d in w.domains]
        for i in range(pre):
            lib.push_all([s[0] for s in slices[i]], [s[1:].reshape(-1) for s in slices[i]])
        rp.rp_graph_capture(lib.ctx, rho, J, phi, A)
        got = {}
        for i in range(pre, T):
            if i == pre + 4:                       # one step by the plain calls
                lib.push_all([s[0] for s in slices[i]], [s[1:].reshape(-1) for s in slices[i]])
                p_, a_ = lib.evaluate()
                got[i] = [torch.cat([p_[d][None], a_[d].reshape(3, -1)]).clone() for d in range(2)]
                continue
            for d in range(2):
                rho[d].copy_(slices[i][d][0])
                J[d].copy_(slices[i][d][1:].reshape(-1))
            rp.rp_graph_step(lib.ctx)
            got[i] = [torch.cat([phi[d][None], A[d].reshape(3, -1)]).clone() for d in range(2)]
        lib.sync()
        for i in range(pre, T):
            for d in range(2):
                np.testing.assert_array_equal(got[i][d].cpu().numpy(), want[i][d], err_msg=f"step {i} domain {d}")


def test_graph_capture_refuses_profiling():
    import torch
    dev = torch.device("cuda", 0)
    w = synth.workload("cfg1")
    with rp.RetardedPotentials(w.domains, w.c, w.dt, flags=rp.RP_FLAG_PROFILE) as lib:
        bufs = [[torch.empty(k * d.N, device=dev) for d in w.domains] for k in (1, 3, 1, 3)]
        with pytest.raises(rp.RPError) as e:
            rp.rp_graph_capture(lib.ctx, *bufs)
        assert e.value.status == rp.RP_ERR_UNSUPPORTED
