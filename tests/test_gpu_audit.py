"""The FP64 error audit on the GPU (RP_FLAG_AUDIT, rp_audit, rp_audit_values).

rp_audit_values computes the plain direct retarded sum in FP64 on the GPU
from the context's own history; it must equal the CPU oracle (the same
definition, Neumaier-compensated in C) to 1e-12 at every node.  rp_audit
then scores an evaluation: within the FP32 bar on the FFT path, and it sees
an error planted in the output (so the comparison is not vacuous).
"""
import numpy as np
import pytest
import torch

from paper_2311_15429_gb300 import rp, synth

from _harness import histories, oracle_values

pytestmark = pytest.mark.gpu


def _drive(domains, c, dt, hists, flags, mode=rp.RP_MODE_FFT, **kw):
    dev = torch.device("cuda", 0)
    lib = rp.RetardedPotentials(domains, c, dt, mode=mode, flags=flags | rp.RP_FLAG_AUDIT, **kw)
    for i in range(hists[0].shape[0]):
        lib.push_all([torch.from_numpy(np.ascontiguousarray(h[i, 0])).to(dev) for h in hists],
                     [torch.from_numpy(np.ascontiguousarray(h[i, 1:]).reshape(-1)).to(dev) for h in hists])
    lib.evaluate()
    lib.sync()
    return lib


def _close(gpu, cpu, bar):
    for f in range(4):
        scale = np.max(np.abs(cpu[:, f]))
        assert np.max(np.abs(gpu[:, f] - cpu[:, f])) <= bar * scale, (f, np.max(np.abs(gpu[:, f] - cpu[:, f])) / scale)


def test_audit_values_match_the_cpu_oracle_on_cfg1():
    """2 x 16^3, 20 bohr apart, step 63 of a 64-step history: every node of
    both domains, FP64 on the GPU against the FP64 oracle on the host."""
    w = synth.workload("cfg1")
    T = 64
    hists = histories(w.sources, 0, T, w.dt)
    lib = _drive(w.domains, w.c, w.dt, hists, 0)
    try:
        for t, d in enumerate(w.domains):
            nodes = np.arange(d.N)
            gpu = rp.rp_audit_values(lib.ctx, t, nodes)
            cpu = oracle_values(w.domains, hists, 0, w.c, w.dt, t, T - 1, nodes)
            _close(gpu, cpu, 1e-12)
        rel = rp.rp_audit(lib.ctx, lib.phi, lib.A, 512, seed=3)
        assert rel.shape == (2, 4) and np.all(rel <= 1e-6) and np.all(rel > 0), rel
        q = lib.query()
        assert q["audit_rel_l2"] == pytest.approx(rel.max()) and q["audit_step"] == T - 1
        # a planted error of 1e-4 (relative, on domain 0's phi) is what the audit reports
        bad = lib.phi[0] * (1 + 1e-4)
        rel_bad = rp.rp_audit(lib.ctx, [bad, lib.phi[1]], lib.A, 512, seed=3)
        assert rel_bad[0, 0] == pytest.approx(1e-4, rel=0.05), rel_bad
        assert np.array_equal(rel_bad[1], rel[1]) and np.array_equal(rel_bad[0, 1:], rel[0, 1:])
    finally:
        lib.close()


def test_audit_values_clamped_mixed_spacing_and_ragged():
    """A direct pair of unequal spacing, a ragged grid, the clamped history
    (S(t <= 0) = S(0)) read from steps before the first push."""
    doms = [synth.cubic((0.0, 0.0, 0.0), 12, 0.3), synth.cubic((9.0, 2.0, -1.0), 10, 0.25),
            synth.Domain((-6.0, 3.0, 1.5), (11, 3, 7), 0.3)]
    srcs = synth.seeded_sources(doms)
    c, dt, T = 20.0, 0.05, 5   # slow light: lags up to ~12 steps reach back before the first push
    hists = histories(srcs, 0, T, dt)
    lib = _drive(doms, c, dt, hists, rp.RP_FLAG_GROUND_STATE_CLAMP)
    try:
        assert lib.query()["max_lag"] >= T
        for t, d in enumerate(doms):
            nodes = np.arange(0, d.N, 3)
            gpu = rp.rp_audit_values(lib.ctx, t, nodes)
            cpu = oracle_values(doms, hists, 0, c, dt, t, T - 1, nodes, clamp=True)
            _close(gpu, cpu, 1e-12)
        rel = rp.rp_audit(lib.ctx, lib.phi, lib.A, 256)
        assert np.all(rel <= 1e-6), rel
    finally:
        lib.close()


def test_audit_needs_its_flag_and_a_complete_step():
    w = synth.workload("cfg1")
    with rp.RetardedPotentials(w.domains, w.c, w.dt) as lib:
        with pytest.raises(rp.RPError) as e:
            rp.rp_audit_values(lib.ctx, 0, [0, 1])
        assert e.value.status == rp.RP_ERR_STATE
