"""Injected allocation failure (RP_ERR_OOM) and the profiling switch, on the GPU.

The device budget of rp_config makes an allocation that would pass it fail
on the host, before any allocator is called: a context whose plan does not
fit returns RP_ERR_OOM from rp_finalize, and one that fits finalize but not
the device staging of rp_evaluate_host gets RP_ERR_OOM from that call and
stays usable.  rp_set_profiling switches the per-launch events on and off
without changing results.
"""
import numpy as np
import pytest
import torch

from paper_2311_15429_gb300 import rp, synth

pytestmark = pytest.mark.gpu


def _inputs(w, T, dev):
    hists = [s.history(0, T, w.dt) for s in w.sources]
    rho = [[torch.from_numpy(np.ascontiguousarray(h[i, 0])).to(dev) for h in hists] for i in range(T)]
    J = [[torch.from_numpy(np.ascontiguousarray(h[i, 1:]).reshape(-1)).to(dev) for h in hists] for i in range(T)]
    return hists, rho, J


def test_budget_below_the_plan_fails_finalize():
    w = synth.workload("cfg1")
    with rp.RetardedPotentials(w.domains, w.c, w.dt) as lib:
        need = lib.query()["device_bytes"]
    ctx = rp.rp_create(w.c, w.dt, device_budget=need // 2)
    try:
        for d in w.domains:
            rp.rp_add_domain(ctx, d.origin, d.n, d.h)
        with pytest.raises(rp.RPError) as e:
            rp.rp_finalize(ctx)
        assert e.value.status == rp.RP_ERR_OOM
        assert "budget" in rp.rp_last_error(ctx)
    finally:
        rp.rp_destroy(ctx)


def test_budget_refuses_host_staging_and_the_context_stays_usable():
    """The budget is what finalize needs: rp_evaluate_host, which allocates
    its staging on first use, gets RP_ERR_OOM; rp_evaluate into caller
    buffers then still runs and matches a context without a budget."""
    w = synth.workload("cfg1")
    dev = torch.device("cuda", 0)
    T = 8
    _, rho, J = _inputs(w, T, dev)
    with rp.RetardedPotentials(w.domains, w.c, w.dt, flags=rp.RP_FLAG_GROUND_STATE_CLAMP) as ref:
        for i in range(T):
            ref.push_all(rho[i], J[i])
        ref.evaluate()
        ref.sync()
        need = ref.query()["device_bytes"]
        want = [torch.cat([ref.phi[t], ref.A[t]]).cpu().numpy() for t in range(2)]
    with rp.RetardedPotentials(w.domains, w.c, w.dt, flags=rp.RP_FLAG_GROUND_STATE_CLAMP,
                               device_budget=need) as lib:
        assert lib.query()["device_bytes"] <= need
        for i in range(T):
            lib.push_all(rho[i], J[i])
        hphi = [np.zeros(d.N, np.float32) for d in w.domains]
        hA = [np.zeros(3 * d.N, np.float32) for d in w.domains]
        with pytest.raises(rp.RPError) as e:
            rp.rp_evaluate_host(lib.ctx, hphi, hA)
        assert e.value.status == rp.RP_ERR_OOM
        lib.evaluate()
        lib.sync()
        for t in range(2):
            assert np.array_equal(torch.cat([lib.phi[t], lib.A[t]]).cpu().numpy(), want[t])


def test_profiling_switch():
    """Events on for the middle steps only: their launches are timed, the
    others counted; the outputs equal those of a context that never times."""
    w = synth.workload("cfg1")
    dev = torch.device("cuda", 0)
    T = 12
    _, rho, J = _inputs(w, T, dev)
    outs = []
    for switch in (False, True):
        with rp.RetardedPotentials(w.domains, w.c, w.dt, flags=rp.RP_FLAG_GROUND_STATE_CLAMP) as lib:
            rp.rp_kernel_stats(lib.ctx, 0, reset=True)
            for i in range(T):
                if switch and i == 4:
                    rp.rp_set_profiling(lib.ctx, 1)
                if switch and i == 8:
                    rp.rp_set_profiling(lib.ctx, 0)
                lib.push_all(rho[i], J[i])
                lib.evaluate()
            lib.sync()
            n_timed, ms = rp.rp_kernel_stats(lib.ctx, rp.RP_K_INV_PLANE)
            assert rp.rp_kernel_count(lib.ctx, rp.RP_K_INV_PLANE) == T
            assert n_timed == (4 if switch else 0)
            assert (ms > 0.0) == switch
            outs.append([torch.cat([lib.phi[t], lib.A[t]]).cpu().numpy() for t in range(2)])
    for a, b in zip(*outs):
        assert np.array_equal(a, b)
