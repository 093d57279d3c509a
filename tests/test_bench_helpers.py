"""CPU checks of bench.py's measurement arithmetic: the algorithmic bytes the
roofline divides by, the rule that takes ncu traffic from a committed
profile only when it was captured on the current kernel source, and the
plain path's flop count and ALU peak."""
import hashlib
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_2311_15429_gb300 import rp, synth  # noqa: E402


def _plan_info(w):
    ctx = rp.rp_create(w.c, w.dt, w.history, flags=rp.RP_FLAG_PLAN_ONLY)
    try:
        for d in w.domains:
            rp.rp_add_domain(ctx, d.origin, d.n, d.h)
        rp.rp_finalize(ctx)
        nd = len(w.domains)
        return {(t, s): rp.rp_pair_info(ctx, t, s) for t in range(nd) for s in range(nd)}
    finally:
        rp.rp_destroy(ctx)


def test_cfg2_algorithmic_bytes():
    """Per target (96^3 padded, 49 x 96 x 96 spectral cells): the T2 write
    (4 fields x 49 x 48 x 96 complex64), four self lags (real kernel + four
    field spectra) and five cross lags (complex kernel + four field
    spectra); twice.  The forward passes read the slices and write / read T1,
    the column pass writes the spectra; the inverse plane pass reads T2 and
    writes phi, A."""
    w = synth.workload("cfg2")
    b = bench.algorithmic_bytes(w, _plan_info(w))
    cells = 49 * 96 * 96
    t2 = 4 * 49 * 48 * 96 * 8
    per_target = t2 + 4 * (4 * cells + 32 * cells) + 5 * (8 * cells + 32 * cells)
    assert b["mac_inv_column"] == 2 * per_target == 325_140_480
    N = 48 ** 3
    assert b["inv_plane"] == 2 * (t2 + 16 * N)
    assert b["fwd_plane"] == 2 * (16 * N + t2)
    assert b["fwd_column"] == 2 * (t2 + 4 * cells * 8)


def _fake_tree(tmp_path, source_bytes, recorded_sha):
    (tmp_path / "profiles").mkdir()
    csrc = tmp_path / "paper_2311_15429_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "k.cu").write_bytes(source_bytes)
    (tmp_path / "profiles" / "kern_wl.md").write_text(
        "summary\ntraffic_bytes_per_launch: 2.5e8\nkernel_source: k.cu\n"
        f"kernel_source_sha256: {recorded_sha}\n")


def test_committed_traffic_only_for_the_current_source(tmp_path, monkeypatch):
    src = b"__global__ void k() {}\n"
    good = hashlib.sha256(src).hexdigest()
    _fake_tree(tmp_path, src, good)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.committed_traffic("kern", "wl") == 2.5e8
    assert bench.committed_traffic("kern", "other") is None          # no summary
    (tmp_path / "paper_2311_15429_gb300" / "csrc" / "k.cu").write_bytes(src + b"// changed\n")
    assert bench.committed_traffic("kern", "wl") is None             # kernel changed since


def test_committed_profiles_name_existing_sources():
    """Every committed summary that records a source hash names a kernel
    source of the package."""
    import re
    for name in os.listdir(os.path.join(ROOT, "profiles")):
        txt = open(os.path.join(ROOT, "profiles", name)).read()
        m = re.search(r"kernel_source:\s*(\S+)", txt)
        if m and "kernel_source_sha256" in txt:
            assert os.path.exists(os.path.join(ROOT, "paper_2311_15429_gb300", "csrc", m.group(1))), name


def test_plain_path_flops_and_alu_peak():
    assert bench.DIRECT_FLOPS_PER_PAIR_POINT == 34
    assert bench.FP32_PEAK_TFLOPS == pytest.approx(152 * 128 * 2 * 2.070e9 / 1e12)
    assert bench.kernel_pass_steps(5) == 20 and bench.kernel_pass_steps(20) == 20
    assert bench.kernel_pass_steps(10 ** 6) == bench.KERNEL_PASS_STEPS


def test_cfg2_far_gemm_bytes():
    """The cross pairs of the 2 x 48^3 workload on the factors (far distance
    1000 bohr, 4^3 nodes, batches of 32): per source one GEMM of W (5 lags x
    64 nodes = 320 rows, padded to 384) by X (4 fields x 32 slices = 128
    rows) over K = 110592, hi and lo bf16 planes (4 B per element), and the
    fp32 node values written: 170 + 56.6 + 0.2 MB."""
    w = synth.workload("cfg2")
    ctx = rp.rp_create(w.c, w.dt, w.history, rp.RP_MODE_LOWRANK, rp.RP_FLAG_PLAN_ONLY,
                       far_distance=1000.0, far_points=4, far_batch=32)
    try:
        for d in w.domains:
            rp.rp_add_domain(ctx, d.origin, d.n, d.h)
        rp.rp_finalize(ctx)
        info = {(t, s): rp.rp_pair_info(ctx, t, s) for t in range(2) for s in range(2)}
    finally:
        rp.rp_destroy(ctx)
    assert info[(1, 0)]["kind"] == rp.RP_PAIR_LOWRANK and info[(1, 0)]["lag_hi"] - info[(1, 0)]["lag_lo"] == 4
    K = 48 ** 3
    want = 384 * K * 4 + 128 * K * 4 + 384 * 128 * 4
    assert bench.far_gemm_bytes(w, info, 4, 32) == want
    assert 226e6 < want < 227e6   # 226.7 MB
