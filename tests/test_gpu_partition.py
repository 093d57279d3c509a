"""The source partition on one GPU: contexts that own complementary sets of
source domains (rp_own_sources), pushed with their own sources only; the sum
of their outputs must equal one context that owns every source.

Cases cover every writer of a target's output under a partition: an FFT
pass (self or cross pairs of equal spacing), the direct sum alone (pairs of
unequal spacing, no FFT pass), the far interpolation alone (a target reached
only by far pairs: written), and direct pairs with far pairs added (no FFT
pass: the interpolation adds after the direct sum).
"""
import numpy as np
import pytest
import torch

from paper_2311_15429_gb300 import rp, synth

from _harness import oracle_values, rel_l2

pytestmark = pytest.mark.gpu


def _run(doms, hists, owned, eval_at, **kw):
    dev = torch.device("cuda", 0)
    out = {}
    with rp.RetardedPotentials(doms, synth.C_AU, 0.05, owned_sources=owned, **kw) as lib:
        q = lib.query()
        for i in range(hists[0].shape[0]):
            r = [torch.from_numpy(np.ascontiguousarray(h[i, 0])).to(dev) if d in owned else None
                 for d, h in enumerate(hists)]
            J = [torch.from_numpy(np.ascontiguousarray(h[i, 1:]).reshape(-1)).to(dev) if d in owned else None
                 for d, h in enumerate(hists)]
            lib.push_all(r, J)
            if i in eval_at:
                lib.evaluate()
                out[i] = [torch.cat([lib.phi[d], lib.A[d]]).cpu().numpy() for d in range(len(doms))]
        lib.sync()
    return out, q


CASES = {
    "fft": ([synth.cubic((0.0, 0.0, 0.0), 12, 0.25), synth.cubic((8.0, 0.5, -0.3), 12, 0.25),
             synth.Domain((-6.0, 3.0, 1.0), (9, 7, 11), 0.25)], {}, [[0, 2], [1]]),
    "direct_alone": ([synth.cubic((0.0, 0.0, 0.0), 12, 0.3), synth.cubic((9.0, 2.0, -1.0), 10, 0.25),
                      synth.cubic((-8.0, 0.0, 3.0), 9, 0.3)], {}, [[1], [0, 2]]),
    "far_alone": ([synth.cubic((0.0, 0.0, 0.0), 12, 0.25), synth.cubic((8.0, 0.5, -0.3), 12, 0.25),
                   synth.cubic((600.0, 50.0, -30.0), 12, 0.25)],
                  dict(mode=rp.RP_MODE_LOWRANK, far_distance=100.0, far_batch=32, far_source_points=4), [[2], [0, 1]]),
    "direct_plus_far": ([synth.cubic((0.0, 0.0, 0.0), 12, 0.3), synth.cubic((9.0, 2.0, -1.0), 10, 0.25),
                         synth.cubic((600.0, 0.0, 0.0), 12, 0.3)],
                        dict(mode=rp.RP_MODE_LOWRANK, far_distance=100.0, far_batch=16), [[1, 2], [0]]),
}


@pytest.mark.parametrize("case", list(CASES))
def test_partial_outputs_add_up_to_the_whole(case):
    doms, kw, parts = CASES[case]
    srcs = synth.seeded_sources(doms)
    T = 104
    hists = [s.history(0, T, 0.05) for s in srcs]
    steps = [T - 5, T - 1]
    full, qf = _run(doms, hists, list(range(len(doms))), steps, **kw)
    partial = [_run(doms, hists, p, steps, **kw) for p in parts]
    for (_, q), p in zip(partial, parts):
        assert q["owned_sources"] == len(p) and q["npairs_other"] == len(doms) * (len(doms) - len(p))
    for step in steps:
        for t, d in enumerate(doms):
            total = sum(o[step][t].astype(np.float64) for o, _ in partial)
            ref = full[step][t].astype(np.float64)
            for f in range(4):
                sl = slice(f * d.N, (f + 1) * d.N)
                assert np.linalg.norm(total[sl] - ref[sl]) <= 1e-6 * np.linalg.norm(ref[sl]), (case, step, t, f)
            if not kw:   # and both against the FP64 oracle on the FP32 path
                want = oracle_values(doms, hists, 0, synth.C_AU, 0.05, t, step, np.arange(d.N))
                assert max(rel_l2(total.reshape(4, -1), want)) <= 1e-6


def test_push_of_a_domain_owned_elsewhere_is_refused():
    doms = CASES["fft"][0]
    with rp.RetardedPotentials(doms, synth.C_AU, 0.05, owned_sources=[0]) as lib:
        z = torch.zeros(doms[1].N, device="cuda"), torch.zeros(3 * doms[1].N, device="cuda")
        with pytest.raises(rp.RPError) as e:
            rp.rp_push(lib.ctx, 1, z[0], z[1])
        assert e.value.status == rp.RP_ERR_ARG
