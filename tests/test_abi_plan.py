"""CPU checks of the C-ABI library: it builds for sm_103a, loads, exports
every entry point of include/rp.h, and its host-side planner (lag windows,
FFT sizes, pair kinds, ring depths, argument and state errors) is right.
No compute call is made: contexts here are RP_FLAG_PLAN_ONLY."""
import math
import os
import re

import numpy as np
import pytest

from paper_2311_15429_gb300 import rp, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SIZES = {1, 2, 3, 4, 6, 8, 12, 16, 24, 32, 48, 64, 96, 128, 192}


def header_entry_points():
    src = open(os.path.join(ROOT, "include", "rp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rp_[a-z_]+)\s*\(", src)))


def test_library_builds_and_exports_every_declared_symbol():
    lib = rp.load()
    names = header_entry_points()
    assert len(names) >= 18
    for name in names:
        assert hasattr(lib, name), name
        assert name in rp.SIGNATURES, f"binding lacks {name}"
    out = os.popen(f"nm -D --defined-only {rp.library_path()}").read()
    for name in names:
        assert re.search(rf"\bT {name}\b", out), f"{name} not exported"


def test_status_strings_and_kernel_names():
    assert rp.rp_status_str(rp.RP_OK) == "RP_OK"
    assert rp.rp_status_str(rp.RP_ERR_HISTORY) == "RP_ERR_HISTORY"
    assert rp.rp_kernel_name(rp.RP_K_MAC_INV_COLUMN) == "mac_inv_column"
    assert rp.rp_kernel_name(rp.RP_K_COUNT) is None


def test_create_rejects_bad_config():
    for c, dt, mode in ((0.0, 0.05, 0), (137.0, -1.0, 0), (137.0, 0.05, 7)):
        with pytest.raises(rp.RPError) as e:
            rp.rp_create(c, dt, mode=mode, flags=rp.RP_FLAG_PLAN_ONLY)
        assert e.value.status == rp.RP_ERR_ARG


def _plan(domains, c=synth.C_AU, dt=0.05, mode=rp.RP_MODE_FFT, depth=0):
    ctx = rp.rp_create(c, dt, depth, mode, rp.RP_FLAG_PLAN_ONLY)
    for d in domains:
        rp.rp_add_domain(ctx, d.origin, d.n, d.h)
    rp.rp_finalize(ctx)
    return ctx


def _node_distances(a, b):
    xa, ya, za = a.coords()
    xb, yb, zb = b.coords()
    d = np.sqrt((xa[:, None] - xb[None]) ** 2 + (ya[:, None] - yb[None]) ** 2 + (za[:, None] - zb[None]) ** 2)
    return d


@pytest.mark.parametrize("geom", ["cfg1", "ragged", "offset"])
def test_lag_windows_cover_every_node_pair(geom):
    """Every lag m with a nonzero hat weight T(m - R/(c dt)) for some node pair
    lies in [lag_lo, lag_hi] (Eq. 11), and lag_hi is the tightest such bound."""
    if geom == "cfg1":
        doms = synth.workload("cfg1").domains
    elif geom == "ragged":
        doms = [synth.Domain((0.0, 0.0, 0.0), (7, 5, 6), 0.3), synth.Domain((3.1, -0.7, 0.4), (4, 9, 3), 0.3)]
    else:
        doms = [synth.Domain((0.0, 0.0, 0.0), (6, 6, 6), 0.25), synth.Domain((40.3, 17.1, -9.2), (5, 7, 4), 0.25)]
    c, dt = synth.C_AU, 0.05
    ctx = _plan(doms, c, dt)
    try:
        for t in range(len(doms)):
            for s in range(len(doms)):
                info = rp.rp_pair_info(ctx, t, s)
                R = _node_distances(doms[t], doms[s])
                tau = R / (c * dt)
                lo_need = 0 if t == s else int(np.floor(tau.min()))
                hi_need = int(np.floor(tau.max())) + 1
                assert info["lag_lo"] <= lo_need
                assert info["lag_hi"] == hi_need
                assert info["r_max"] == pytest.approx(R.max(), rel=1e-12)
                assert info["r_min"] <= R[R > 0].min() + 1e-12 or t == s
    finally:
        rp.rp_destroy(ctx)


def test_cfg2_plan():
    w = synth.workload("cfg2")
    ctx = _plan(w.domains, w.c, w.dt, depth=w.history)
    try:
        cross = rp.rp_pair_info(ctx, 0, 1)
        assert (cross["lag_lo"], cross["lag_hi"]) == (290, 294)   # B = 5 delay bins
        assert cross["kind"] == rp.RP_PAIR_FFT and cross["fft_m"] == (96, 96, 96)
        self_ = rp.rp_pair_info(ctx, 0, 0)
        assert (self_["lag_lo"], self_["lag_hi"]) == (0, 3)
        q = rp.rp_query(ctx)
        assert q["npairs_fft"] == 4 and q["npairs_direct"] == 0
        assert q["spectral_depth"] == 320 and q["raw_depth"] == 0
        # two sources x 320 slots x 4 fields x (49 x 96 x 96) complex64
        assert q["spectral_bytes"] == 2 * 320 * 4 * 49 * 96 * 96 * 8
    finally:
        rp.rp_destroy(ctx)


def test_fft_sizes_are_supported_and_large_enough():
    doms = [synth.Domain((0.0, 0.0, 0.0), (7, 5, 6), 0.3), synth.Domain((3.1, -0.7, 0.4), (4, 9, 3), 0.3),
            synth.Domain((-9.0, 2.0, 1.0), (1, 1, 1), 0.3)]
    ctx = _plan(doms)
    try:
        for t in range(3):
            m_t = None
            for s in range(3):
                info = rp.rp_pair_info(ctx, t, s)
                assert info["kind"] == rp.RP_PAIR_FFT
                m = info["fft_m"]
                assert all(v in SIZES for v in m) and m[0] % 2 == 0
                assert all(m[a] >= doms[t].n[a] + doms[s].n[a] - 1 for a in range(3))
                m_t = m_t or m
                assert m == m_t          # one spectral size per target
    finally:
        rp.rp_destroy(ctx)


def test_unequal_spacing_goes_direct_and_direct_mode():
    doms = [synth.Domain((0.0, 0.0, 0.0), (4, 4, 4), 0.3), synth.Domain((5.0, 0.0, 0.0), (4, 4, 4), 0.25)]
    ctx = _plan(doms)
    try:
        assert rp.rp_pair_info(ctx, 0, 1)["kind"] == rp.RP_PAIR_DIRECT
        assert rp.rp_pair_info(ctx, 0, 0)["kind"] == rp.RP_PAIR_FFT
        q = rp.rp_query(ctx)
        assert q["raw_depth"] >= rp.rp_pair_info(ctx, 1, 0)["lag_hi"] + 1
    finally:
        rp.rp_destroy(ctx)
    ctx = _plan(doms, mode=rp.RP_MODE_DIRECT)
    try:
        q = rp.rp_query(ctx)
        assert q["npairs_direct"] == 4 and q["npairs_fft"] == 0
    finally:
        rp.rp_destroy(ctx)


def test_plan_errors():
    # a self term beyond 96 nodes per axis is not supported by the FFT path
    with pytest.raises(rp.RPError) as e:
        _plan([synth.Domain((0.0, 0.0, 0.0), (97, 4, 4), 0.3)])
    assert e.value.status == rp.RP_ERR_UNSUPPORTED
    # coincident nodes of two domains
    with pytest.raises(rp.RPError) as e:
        _plan([synth.Domain((0.0, 0.0, 0.0), (3, 3, 3), 0.5), synth.Domain((0.5, 0.5, 0.5), (3, 3, 3), 0.5)])
    assert e.value.status == rp.RP_ERR_ARG
    ctx = rp.rp_create(137.0, 0.05, flags=rp.RP_FLAG_PLAN_ONLY)
    try:
        with pytest.raises(rp.RPError) as e:
            rp.rp_add_domain(ctx, (0, 0, 0), (0, 4, 4), 0.3)
        assert e.value.status == rp.RP_ERR_ARG
        with pytest.raises(rp.RPError) as e:
            rp.rp_finalize(ctx)                 # no domains
        assert e.value.status == rp.RP_ERR_STATE
        rp.rp_add_domain(ctx, (0, 0, 0), (4, 4, 4), 0.3)
        rp.rp_finalize(ctx)
        with pytest.raises(rp.RPError) as e:
            rp.rp_add_domain(ctx, (9, 0, 0), (4, 4, 4), 0.3)
        assert e.value.status == rp.RP_ERR_STATE
        # a plan-only context runs nothing
        import numpy as np
        x = np.zeros(64, np.float32)
        with pytest.raises(rp.RPError) as e:
            rp.rp_push(ctx, 0, x, x)
        assert e.value.status == rp.RP_ERR_STATE
    finally:
        rp.rp_destroy(ctx)


def test_no_gpu_create_fails_cleanly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(rp.RPError) as e:
        rp.rp_create(137.0, 0.05, stream=0)
    assert e.value.status == rp.RP_ERR_CUDA


def test_config_validation():
    """Out-of-range configuration fields are refused at rp_create."""
    bad = [dict(mac_warps=10), dict(mac_warps=-8), dict(mode=rp.RP_MODE_LOWRANK, far_distance=0.0),
           dict(mode=rp.RP_MODE_LOWRANK, far_distance=100.0, far_batch=12),
           dict(mode=rp.RP_MODE_LOWRANK, far_distance=100.0, far_points=9), dict(profile_every=-1),
           dict(far_source_points=1), dict(far_source_points=9), dict(device_budget=-1),
           dict(mac_stages=1), dict(mac_stages=-2)]
    for kw in bad:
        with pytest.raises(rp.RPError) as e:
            rp.rp_create(137.0, 0.05, flags=rp.RP_FLAG_PLAN_ONLY, **kw)
        assert e.value.status == rp.RP_ERR_ARG, kw
    for cw in (0, 8, 12, 16):
        rp.rp_destroy(rp.rp_create(137.0, 0.05, flags=rp.RP_FLAG_PLAN_ONLY | rp.RP_FLAG_PLAIN_SUM, mac_warps=cw))
    for cw in (0, 12):   # the compensated sum (default) has the 12-warp variant only
        rp.rp_destroy(rp.rp_create(137.0, 0.05, flags=rp.RP_FLAG_PLAN_ONLY, mac_warps=cw))
    for cw in (8, 16):
        with pytest.raises(rp.RPError):
            rp.rp_create(137.0, 0.05, flags=rp.RP_FLAG_PLAN_ONLY, mac_warps=cw)
    for n in (0, 2, 3, 6):
        rp.rp_destroy(rp.rp_create(137.0, 0.05, flags=rp.RP_FLAG_PLAN_ONLY, mac_stages=n))


def test_ground_split_refuses_far_pairs():
    """RP_FLAG_GROUND_STATE_SPLIT works on FFT and direct pairs; a plan with
    far pairs is refused at rp_finalize."""
    w = synth.workload("cfg2")
    ctx = rp.rp_create(w.c, w.dt, mode=rp.RP_MODE_LOWRANK, far_distance=1000.0,
                       flags=rp.RP_FLAG_PLAN_ONLY | rp.RP_FLAG_GROUND_STATE_SPLIT)
    try:
        for d in w.domains:
            rp.rp_add_domain(ctx, d.origin, d.n, d.h)
        with pytest.raises(rp.RPError) as e:
            rp.rp_finalize(ctx)
        assert e.value.status == rp.RP_ERR_UNSUPPORTED
    finally:
        rp.rp_destroy(ctx)
    ctx = rp.rp_create(w.c, w.dt, flags=rp.RP_FLAG_PLAN_ONLY | rp.RP_FLAG_GROUND_STATE_SPLIT)
    try:
        for d in w.domains:
            rp.rp_add_domain(ctx, d.origin, d.n, d.h)
        rp.rp_finalize(ctx)
    finally:
        rp.rp_destroy(ctx)



def test_history_spill_plan():
    """RP_FLAG_HISTORY_SPILL on the 2 x 48^3 workload (cross lags 290..294):
    each cross pair reads a 5-slot window ring (B), the spectral rings keep
    only the self lags 0..3, and the 320-step history moves to a pinned host
    ring of (rho, J) slices.  A neighbouring pair (lags from 0) stays on the
    device."""
    w = synth.workload("cfg2")
    slot = 4 * 49 * 96 * 96 * 8
    sl = 16 * 48 ** 3                      # one (rho, J) slice
    ctx = rp.rp_create(w.c, w.dt, w.history, flags=rp.RP_FLAG_PLAN_ONLY | rp.RP_FLAG_HISTORY_SPILL)
    try:
        for d in w.domains:
            rp.rp_add_domain(ctx, d.origin, d.n, d.h)
        rp.rp_finalize(ctx)
        q = rp.rp_query(ctx)
        assert q["spill_windows"] == 2
        assert q["spectral_depth"] == 4
        # per source: ring 4 + window 5 spectra, 2 window input and 3 staging slices
        assert q["spectral_bytes"] == 2 * ((4 + 5) * slot + (2 + 3) * sl)
        assert q["host_bytes"] == 2 * w.history * sl
        assert rp.rp_pair_info(ctx, 0, 1)["lag_lo"] == 290   # the pair plan itself is unchanged
    finally:
        rp.rp_destroy(ctx)
    # neighbours 1 bohr apart: every window starts near lag 0, nothing spills
    doms = [synth.Domain((0.0, 0.0, 0.0), (8, 8, 8), 0.25), synth.Domain((3.0, 0.0, 0.0), (8, 8, 8), 0.25)]
    ctx = rp.rp_create(synth.C_AU, 0.05, flags=rp.RP_FLAG_PLAN_ONLY | rp.RP_FLAG_HISTORY_SPILL)
    try:
        for d in doms:
            rp.rp_add_domain(ctx, d.origin, d.n, d.h)
        rp.rp_finalize(ctx)
        q = rp.rp_query(ctx)
        assert q["spill_windows"] == 0 and q["host_bytes"] == 0
    finally:
        rp.rp_destroy(ctx)


@pytest.mark.parametrize("distance", [6.0, 40.0, 60.0, 90.0, 205.0, 2000.0])
def test_history_spill_follows_each_pairs_lag_window(distance):
    """The spilled windows are exactly the FFT pairs with
    lag_lo >= 2 (lag_hi - lag_lo + 2), one per (source ring, window); the
    spectral bytes drop by the unspilled depth the rings no longer need; the
    host ring holds max(history_depth, largest spilled lag_hi + 1) slices of
    each spilled source."""
    w = synth.two_domain(16, 0.25, distance)
    flags = rp.RP_FLAG_PLAN_ONLY | rp.RP_FLAG_HISTORY_SPILL
    ctx = rp.rp_create(w.c, w.dt, 0, rp.RP_MODE_FFT, flags)
    try:
        for d in w.domains:
            rp.rp_add_domain(ctx, d.origin, d.n, d.h)
        rp.rp_finalize(ctx)
        q = rp.rp_query(ctx)
        spilled = []
        for t in range(2):
            for s in range(2):
                p = rp.rp_pair_info(ctx, t, s)
                if p["lag_lo"] >= 2 * (p["lag_hi"] - p["lag_lo"] + 2):
                    spilled.append((t, s, p["lag_lo"], p["lag_hi"]))
        assert q["spill_windows"] == len(spilled)
        assert all(t != s for t, s, _, _ in spilled)
        N = w.domains[0].N
        if spilled:
            hd = max(hi for _, _, _, hi in spilled) + 1
            assert q["host_bytes"] == len({s for _, s, _, _ in spilled}) * hd * 16 * N
            self_hi = rp.rp_pair_info(ctx, 0, 0)["lag_hi"]
            assert q["spectral_depth"] == self_hi + 1
        else:
            assert q["host_bytes"] == 0
    finally:
        rp.rp_destroy(ctx)


def test_device_budget_refuses_a_plan_beyond_it():
    """An allocation budget below the planned device memory makes rp_finalize
    return RP_ERR_OOM (the injected allocation failure: no allocator is
    called); the same plan passes with a budget at its planned size."""
    w = synth.workload("cfg2")
    ctx = rp.rp_create(w.c, w.dt, history_depth=w.history, flags=rp.RP_FLAG_PLAN_ONLY)
    try:
        for d in w.domains:
            rp.rp_add_domain(ctx, d.origin, d.n, d.h)
        rp.rp_finalize(ctx)
        need = rp.rp_query(ctx)["device_bytes"]
    finally:
        rp.rp_destroy(ctx)
    assert need > 2 ** 30
    for budget, ok in ((need - 1, False), (need, True)):
        ctx = rp.rp_create(w.c, w.dt, history_depth=w.history, flags=rp.RP_FLAG_PLAN_ONLY, device_budget=budget)
        try:
            for d in w.domains:
                rp.rp_add_domain(ctx, d.origin, d.n, d.h)
            if ok:
                rp.rp_finalize(ctx)
            else:
                with pytest.raises(rp.RPError) as e:
                    rp.rp_finalize(ctx)
                assert e.value.status == rp.RP_ERR_OOM
                assert "budget" in rp.rp_last_error(ctx)
        finally:
            rp.rp_destroy(ctx)


def test_cfg4_plan_two_sided_every_cross_pair_far():
    """cfg4 (64 sub-domains of 24^3-96^3 at 0.2-0.35 bohr): with two-sided
    factors and a 250 bohr far distance every one of the 4032 cross pairs is
    low-rank (each with lag_lo >= the 32-step batch the gathered GEMM needs)
    and every self pair is an FFT pair."""
    w = synth.workload("cfg4")
    ctx = rp.rp_create(w.c, w.dt, mode=rp.RP_MODE_LOWRANK, flags=rp.RP_FLAG_PLAN_ONLY, far_distance=250.0,
                       far_batch=32, far_source_points=4)
    try:
        for d in w.domains:
            rp.rp_add_domain(ctx, d.origin, d.n, d.h)
        rp.rp_finalize(ctx)
        q = rp.rp_query(ctx)
        assert q["ndomains"] == 64 and q["npairs_far"] == 4032 and q["npairs_fft"] == 64 and q["npairs_direct"] == 0
        for t in range(64):
            for s in range(64):
                p = rp.rp_pair_info(ctx, t, s)
                if t == s:
                    assert p["kind"] == rp.RP_PAIR_FFT
                else:
                    assert p["kind"] == rp.RP_PAIR_LOWRANK and p["lag_lo"] >= 32, (t, s, p)
    finally:
        rp.rp_destroy(ctx)


def test_two_sided_factors_need_a_batch_of_at_most_32():
    with pytest.raises(rp.RPError) as e:
        rp.rp_create(137.0, 0.05, mode=rp.RP_MODE_LOWRANK, flags=rp.RP_FLAG_PLAN_ONLY, far_distance=100.0,
                     far_batch=40, far_source_points=4)
    assert e.value.status == rp.RP_ERR_ARG
