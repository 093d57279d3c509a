"""GPU: the ground-state split of Eqs. 9-12 (RP_FLAG_GROUND_STATE_SPLIT).

rp_ground_potential gives P(0), the static potential of the first sample;
rp_evaluate gives the induced part sum_m G_m Delta S(l - m),
Delta S = S - S(0).  By the hat weights' partition of unity their sum is the
plain sum with samples before the first push equal to S(0) (the clamped
reading), so the oracle with clamp = True is the reference.
"""
import os
import tempfile

import numpy as np
import pytest

from paper_2311_15429_gb300 import rp, synth

from _harness import histories, oracle_values, rel_l2, run_library

pytestmark = pytest.mark.gpu
SPLIT = rp.RP_FLAG_GROUND_STATE_SPLIT
CLAMP = rp.RP_FLAG_GROUND_STATE_CLAMP


def run_split(domains, c, dt, hists, steps, mode=rp.RP_MODE_FFT):
    """{step: (induced [domain][4][N], static [domain][4][N])}."""
    import torch
    dev = torch.device("cuda", 0)
    out = {}
    with rp.RetardedPotentials(domains, c, dt, mode=mode, flags=SPLIT) as lib:
        ph = [torch.empty(d.N, device=dev) for d in domains]
        Ag = [torch.empty(3 * d.N, device=dev) for d in domains]
        for i in range(hists[0].shape[0]):
            lib.push_all([torch.from_numpy(np.ascontiguousarray(h[i, 0])).to(dev) for h in hists],
                         [torch.from_numpy(np.ascontiguousarray(h[i, 1:]).reshape(-1)).to(dev) for h in hists])
            if i in steps:
                phi, A = lib.evaluate()
                rp.rp_ground_potential(lib.ctx, ph, Ag)
                torch.cuda.synchronize()
                cat = lambda p, a: np.concatenate([p.cpu().numpy()[None], a.cpu().numpy().reshape(3, -1)])
                out[i] = ([cat(phi[d], A[d]) for d in range(len(domains))],
                          [cat(ph[d], Ag[d]) for d in range(len(domains))])
    return out


@pytest.mark.parametrize("mode", [rp.RP_MODE_FFT, rp.RP_MODE_DIRECT])
def test_split_matches_the_clamped_sum(mode):
    """P(0) + induced part against the clamped oracle from the first step on
    (steps before the deepest lag included); at step 0 the induced part is 0."""
    w = synth.workload("cfg1")
    T = 10
    hists = histories(w.sources, 0, T, w.dt)
    res = run_split(w.domains, w.c, w.dt, hists, {0, 1, 3, T - 1}, mode)
    for step, (ind, sta) in res.items():
        for t, d in enumerate(w.domains):
            want = oracle_values(w.domains, hists, 0, w.c, w.dt, t, step, np.arange(d.N), clamp=True)
            got = ind[t].astype(np.float64) + sta[t]
            assert max(rel_l2(got, want)) <= 1e-6, (step, t)
            if step == 0:
                assert np.all(ind[t] == 0)


def test_split_keeps_the_digits_of_a_small_response():
    """A static density 1000x the oscillating one: the induced part
    P(l) - P(0) comes out at FP32 accuracy relative to itself with the split,
    while the plain path's totals lose about three digits of it."""
    w = synth.workload("cfg1")
    T = 12
    hists = []
    for s, h in zip(w.sources, histories(w.sources, 0, T, w.dt)):
        big = (1000.0 * s.slice64(0.0)).astype(np.float32)   # a large static density and current
        hists.append((h + big[None]).astype(np.float32))
    split = run_split(w.domains, w.c, w.dt, hists, {T - 1})
    plain = run_library(w.domains, w.c, w.dt, hists, 0, [0, T - 1], flags=CLAMP)
    err_split, err_plain = 0.0, 0.0
    for t, d in enumerate(w.domains):
        nodes = np.arange(d.N)
        ref = (oracle_values(w.domains, hists, 0, w.c, w.dt, t, T - 1, nodes, clamp=True)
               - oracle_values(w.domains, hists, 0, w.c, w.dt, t, 0, nodes, clamp=True))
        err_split = max(err_split, max(rel_l2(split[T - 1][0][t].astype(np.float64), ref)))
        got = plain[T - 1][t].astype(np.float64) - plain[0][t].astype(np.float64)
        err_plain = max(err_plain, max(rel_l2(got, ref)))
    print("induced-part rel-L2: split %.2e, plain %.2e" % (err_split, err_plain))
    assert err_split <= 2e-6, (err_split, err_plain)
    assert err_plain >= 20 * err_split, (err_split, err_plain)


def test_split_state_round_trip_and_errors():
    """A saved split context resumes bit-identically (S(0) and P(0) travel
    with the histories); rp_ground_potential needs the flag and a first round."""
    import torch
    dev = torch.device("cuda", 0)
    w = synth.workload("cfg1")
    T = 9
    hists = histories(w.sources, 0, T, w.dt)
    sl = lambda i: ([torch.from_numpy(np.ascontiguousarray(h[i, 0])).to(dev) for h in hists],
                    [torch.from_numpy(np.ascontiguousarray(h[i, 1:]).reshape(-1)).to(dev) for h in hists])
    bufs = ([torch.empty(d.N, device=dev) for d in w.domains], [torch.empty(3 * d.N, device=dev) for d in w.domains])
    with rp.RetardedPotentials(w.domains, w.c, w.dt) as plain:
        with pytest.raises(rp.RPError) as e:
            rp.rp_ground_potential(plain.ctx, *bufs)
        assert e.value.status == rp.RP_ERR_STATE
    path = os.path.join(tempfile.mkdtemp(), "split.state")
    with rp.RetardedPotentials(w.domains, w.c, w.dt, flags=SPLIT) as a:
        with pytest.raises(rp.RPError) as e:
            rp.rp_ground_potential(a.ctx, *bufs)
        assert e.value.status == rp.RP_ERR_STATE
        for i in range(5):
            a.push_all(*sl(i))
        a.sync()
        rp.rp_save_state(a.ctx, path)
        for i in range(5, T):
            a.push_all(*sl(i))
        phi, A = a.evaluate()
        want = [(phi[d].cpu().numpy().copy(), A[d].cpu().numpy().copy()) for d in range(2)]
    with rp.RetardedPotentials(w.domains, w.c, w.dt, flags=SPLIT) as b:
        rp.rp_load_state(b.ctx, path)
        rp.rp_ground_potential(b.ctx, *bufs)
        for i in range(5, T):
            b.push_all(*sl(i))
        phi, A = b.evaluate()
        for d in range(2):
            np.testing.assert_array_equal(phi[d].cpu().numpy(), want[d][0])
            np.testing.assert_array_equal(A[d].cpu().numpy(), want[d][1])
