"""The compensated pair sum (the default) against the plain FP32 chain (RP_FLAG_PLAIN_SUM).

A target's spectral sum runs over every (source, lag) entry of its pairs
before one inverse FFT per field (Eq. 12 per spectral coefficient).  Eight
16^3 domains two box-widths apart under slow light (c dt = 0.5 bohr) give
every target about 200 entries.  Both forms are scored against the FP64
oracle: the compensated one must stay within the FP32 bar of 1e-6, and the
plain chain's error is reported beside it (it grows like the square root of
the entry count).
"""
import numpy as np
import pytest

from paper_2311_15429_gb300 import rp, synth

from _harness import histories, oracle_values, rel_l2, run_library

pytestmark = pytest.mark.gpu


def _lattice():
    doms = [synth.cubic((8.0 * i, 8.0 * j, 8.0 * k), 16, 0.3) for k in range(2) for j in range(2) for i in range(2)]
    return doms, synth.seeded_sources(doms), 10.0, 0.05


def test_about_200_entries_per_target():
    doms, _, c, dt = _lattice()
    with rp.RetardedPotentials(doms, c, dt, flags=rp.RP_FLAG_PLAN_ONLY) as lib:
        entries = [sum(lib.pair_info(t, s)["lag_hi"] - lib.pair_info(t, s)["lag_lo"] + 1 for s in range(8))
                   for t in range(8)]
        kinds = {lib.pair_info(t, s)["kind"] for t in range(8) for s in range(8)}
    assert kinds == {rp.RP_PAIR_FFT}
    assert min(entries) >= 150 and max(entries) <= 300, entries


def test_compensated_sum_within_the_fp32_bar():
    doms, srcs, c, dt = _lattice()
    T = 60
    hists = histories(srcs, 0, T, dt)
    steps = [T - 2, T - 1]
    res = {comp: run_library(doms, c, dt, hists, 0, steps, flags=0 if comp else rp.RP_FLAG_PLAIN_SUM)
           for comp in (False, True)}
    rng = np.random.default_rng(7)
    worst = {False: 0.0, True: 0.0}
    for t, d in enumerate(doms):
        nodes = np.sort(rng.choice(d.N, 256, replace=False))
        for step in steps:
            want = oracle_values(doms, hists, 0, c, dt, t, step, nodes)
            for comp in (False, True):
                worst[comp] = max(worst[comp], max(rel_l2(res[comp][step][t][:, nodes], want)))
    print(f"\nrel-L2 vs FP64 oracle, ~200 entries per target: compensated {worst[True]:.3e}, "
          f"plain FP32 chain {worst[False]:.3e}")
    assert worst[True] <= 1e-6, worst
    assert worst[True] <= worst[False], worst


@pytest.mark.parametrize("geometry", ["cfg1", "ragged"])
def test_compensated_parity_small_and_runtime_shapes(geometry):
    """The compensated MAC on the cubic TMA path (cfg1) and on the
    runtime-shaped kernel (ragged grids)."""
    if geometry == "cfg1":
        w = synth.workload("cfg1")
        doms, srcs, c, dt = w.domains, w.sources, w.c, w.dt
    else:
        doms = [synth.Domain((0.0, 0.0, 0.0), (7, 5, 6), 0.3), synth.Domain((3.1, -0.7, 0.4), (4, 9, 3), 0.3)]
        srcs, c, dt = synth.seeded_sources(doms), synth.C_AU, 0.05
    hists = histories(srcs, 0, 12, dt)
    res = run_library(doms, c, dt, hists, 0, [11])
    for t, d in enumerate(doms):
        want = oracle_values(doms, hists, 0, c, dt, t, 11, np.arange(d.N))
        assert max(rel_l2(res[11][t], want)) <= 1e-6
