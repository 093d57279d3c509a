"""The low-rank far path (RP_MODE_LOWRANK) against the FP64 oracle.

Three 12^3 domains: two 8 bohr apart (FFT path) and one about 600 bohr away
(far pairs: interpolative factors, time-batched bf16 tcgen05 GEMMs).  The bar
for the bf16 far field is 1e-3 rel-L2, on the total and on the far field
alone (only the far source active).
"""
import numpy as np
import pytest

from paper_2311_15429_gb300 import rp, synth

from _harness import oracle_values, rel_l2

pytestmark = pytest.mark.gpu
TOL = 1e-3


def _setup():
    doms = [synth.cubic((0.0, 0.0, 0.0), 12, 0.25), synth.cubic((8.0, 0.5, -0.3), 12, 0.25),
            synth.cubic((600.0, 50.0, -30.0), 12, 0.25)]
    return doms, synth.seeded_sources(doms)


def _run(doms, hists, eval_at, batch=16, source_points=0):
    import torch
    dev = torch.device("cuda", 0)
    out = {}
    with rp.RetardedPotentials(doms, synth.C_AU, 0.05, mode=rp.RP_MODE_LOWRANK, far_distance=100.0,
                               far_batch=batch, far_source_points=source_points) as lib:
        kinds = {(t, s): lib.pair_info(t, s)["kind"] for t in range(3) for s in range(3)}
        for i in range(hists[0].shape[0]):
            lib.push_all([torch.from_numpy(h[i, 0].copy()).to(dev) for h in hists],
                         [torch.from_numpy(h[i, 1:].copy().reshape(-1)).to(dev) for h in hists])
            if i in eval_at:
                phi, A = lib.evaluate()
                torch.cuda.synchronize()
                out[i] = [np.concatenate([phi[d].cpu().numpy()[None], A[d].cpu().numpy().reshape(3, -1)])
                          for d in range(3)]
        lib.sync()
        q = lib.query()
    return out, kinds, q


def test_far_pairs_planned_lowrank():
    doms, _ = _setup()
    ctx = rp.rp_create(synth.C_AU, 0.05, mode=rp.RP_MODE_LOWRANK, flags=rp.RP_FLAG_PLAN_ONLY, far_distance=100.0,
                       far_batch=16)
    try:
        for d in doms:
            rp.rp_add_domain(ctx, d.origin, d.n, d.h)
        rp.rp_finalize(ctx)
        for t in range(3):
            for s in range(3):
                k = rp.rp_pair_info(ctx, t, s)["kind"]
                far = (t == 2) != (s == 2)
                assert k == (rp.RP_PAIR_LOWRANK if far else rp.RP_PAIR_FFT), (t, s, k)
        assert rp.rp_query(ctx)["npairs_far"] == 4
    finally:
        rp.rp_destroy(ctx)


@pytest.mark.parametrize("batch,source_points", [(16, 0), (32, 0), (16, 4), (32, 4), (24, 3)])
def test_far_path_total_and_far_field(batch, source_points):
    """source_points = 0: the source side of the factors exact; > 0: both
    sides interpolated (two-sided factors, the gathered GEMM)."""
    doms, srcs = _setup()
    T = 104
    hists = [s.history(0, T, 0.05) for s in srcs]
    steps = [T - 4, T - 1]
    out, kinds, q = _run(doms, hists, steps, batch, source_points)
    assert q["npairs_far"] == 4
    for step in steps:
        for t, d in enumerate(doms):
            want = oracle_values(doms, hists, 0, synth.C_AU, 0.05, t, step, np.arange(d.N))
            errs = rel_l2(out[step][t], want)
            assert max(errs) <= TOL, ("total", step, t, errs)
    # far field alone: only domain 2 active, seen from domains 0 and 1
    far_only = [np.zeros_like(hists[0]), np.zeros_like(hists[1]), hists[2]]
    out, _, _ = _run(doms, far_only, steps, batch, source_points)
    for step in steps:
        for t in (0, 1):
            want = oracle_values(doms, far_only, 0, synth.C_AU, 0.05, t, step, np.arange(doms[t].N))
            errs = rel_l2(out[step][t], want)
            assert max(errs) <= TOL, ("far only", step, t, errs)


@pytest.mark.parametrize("owned", [None, [2]])
def test_graph_replay_two_sided_far(owned):
    """A step with two-sided far pairs recorded as a CUDA graph: every
    replay gives the bits of the plain calls, across three batches of the
    gathered GEMM (whose launch is recorded in every step and works on a
    batch's last push only), with a plain step in between; also for a
    context that owns only the far source (its other targets written by the
    far interpolation alone)."""
    import torch
    dev = torch.device("cuda", 0)
    doms, srcs = _setup()
    T, start = 200, 100
    hists = [s.history(0, T, 0.05) for s in srcs]
    kw = dict(mode=rp.RP_MODE_LOWRANK, far_distance=100.0, far_batch=32, far_source_points=4)
    if owned is not None:
        kw["owned_sources"] = owned
    own = owned if owned is not None else [0, 1, 2]
    slices = [[torch.from_numpy(np.ascontiguousarray(h[i])).to(dev) for h in hists] for i in range(T)]

    def push(lib, i):
        lib.push_all([slices[i][d][0] if d in own else None for d in range(3)],
                     [slices[i][d][1:].reshape(-1) if d in own else None for d in range(3)])

    want = {}
    with rp.RetardedPotentials(doms, synth.C_AU, 0.05, **kw) as lib:
        for i in range(T):
            push(lib, i)
            if i >= start:
                p_, a_ = lib.evaluate()
                want[i] = [torch.cat([p_[d], a_[d]]).cpu().numpy() for d in range(3)]
    got = {}
    with rp.RetardedPotentials(doms, synth.C_AU, 0.05, **kw) as lib:
        rho = [torch.zeros(d.N, device=dev) for d in doms]
        J = [torch.zeros(3 * d.N, device=dev) for d in doms]
        phi = [torch.empty(d.N, device=dev) for d in doms]
        A = [torch.empty(3 * d.N, device=dev) for d in doms]
        for i in range(start):
            push(lib, i)
        rp.rp_graph_capture(lib.ctx, rho, J, phi, A)
        for i in range(start, T):
            if i == start + 40:                       # one step by the plain calls
                push(lib, i)
                p_, a_ = lib.evaluate()
                got[i] = [torch.cat([p_[d], a_[d]]).cpu().numpy() for d in range(3)]
                continue
            for d in own:
                rho[d].copy_(slices[i][d][0])
                J[d].copy_(slices[i][d][1:].reshape(-1))
            rp.rp_graph_step(lib.ctx)
            got[i] = [torch.cat([phi[d], A[d]]).cpu().numpy() for d in range(3)]
        lib.sync()
    for i in range(start, T):
        for d in range(3):
            np.testing.assert_array_equal(got[i][d], want[i][d], err_msg=f"step {i} domain {d}")


@pytest.mark.parametrize("cut", [150, 160])
def test_save_and_load_two_sided_far(tmp_path, cut):
    """rp_save_state in the middle of a 32-step batch of the gathered GEMM
    (cut 150) and at a batch's first push (cut 160), rp_load_state into a
    fresh context: the steps after it give the bits of the uninterrupted run
    (the source coefficient rings and the targets' node-value rings are part
    of the state)."""
    import torch
    dev = torch.device("cuda", 0)
    doms, srcs = _setup()
    T, start = 200, 100
    hists = [s.history(0, T, 0.05) for s in srcs]
    kw = dict(mode=rp.RP_MODE_LOWRANK, far_distance=100.0, far_batch=32, far_source_points=4)
    slices = [[torch.from_numpy(np.ascontiguousarray(h[i])).to(dev) for h in hists] for i in range(T)]

    def push(lib, i):
        lib.push_all([x[0] for x in slices[i]], [x[1:].reshape(-1) for x in slices[i]])

    want = {}
    with rp.RetardedPotentials(doms, synth.C_AU, 0.05, **kw) as lib:
        for i in range(T):
            push(lib, i)
            if i >= start:
                p_, a_ = lib.evaluate()
                want[i] = [torch.cat([p_[d], a_[d]]).cpu().numpy() for d in range(3)]
    path = str(tmp_path / "state.bin")
    with rp.RetardedPotentials(doms, synth.C_AU, 0.05, **kw) as lib:
        for i in range(cut):
            push(lib, i)
            if i >= start:
                lib.evaluate()
        rp.rp_save_state(lib.ctx, path)
    with rp.RetardedPotentials(doms, synth.C_AU, 0.05, **kw) as lib:
        rp.rp_load_state(lib.ctx, path)
        assert lib.query()["step"] == cut - 1
        for i in range(cut, T):
            push(lib, i)
            p_, a_ = lib.evaluate()
            got = [torch.cat([p_[d], a_[d]]).cpu().numpy() for d in range(3)]
            for d in range(3):
                np.testing.assert_array_equal(got[d], want[i][d], err_msg=f"cut {cut} step {i} domain {d}")
