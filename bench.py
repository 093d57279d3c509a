#!/usr/bin/env python3
"""Benchmark: retarded phi, A grid-point updates per second per time step.

Workload (default): two 48^3 sub-domains, h = 0.25 bohr, centres 2000 bohr
apart on x (cross delays 290..294 steps), 320-step history ring, c = 137.036,
dt = 0.05 -- synthetic Gaussian sources with continuity-consistent currents.
One step = push (rho, Jx, Jy, Jz) of both domains + evaluate (phi, Ax, Ay, Az)
on both grids.  One update = all four fields complete at one grid point,
summed over every source domain including itself.

Prints ONE JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle
on this machine's host cores on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2311_15429_gb300 import synth  # noqa: E402

METRIC = "retarded phi,A grid updates/s per timestep vs plain path, at stated rel-L2 error"
UNIT = "updates/s"
# Per-kernel CUDA events sit between kernels and hold back the next launch
# (about 18 us a step on the 2 x 48^3 workload), so the timed steps run
# without them; the kernels are timed afterwards in a separate pass of
# KERNEL_PASS_STEPS steps on the same context, every launch bracketed.
KERNEL_PASS_STEPS = 100


def kernel_pass_steps(steps):
    """Steps of the separate kernel-timing pass."""
    return max(20, min(steps, KERNEL_PASS_STEPS))


L2_BYTES = 129 * 2 ** 20


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=2000)
    p.add_argument("--warmup", type=int, default=20)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", default="cfg2",
                   help="cfg1 | cfg2 | near48 (48^3 pair 200 bohr apart) | cfg3 | cfg5 | cfg5x8 (first 8 "
                        "domains of cfg5) | cfg4x8 (first 8 of cfg4: mixed sizes and spacings); cfg3, cfg4x8 and "
                        "cfg5* have thousands-deep histories and run the far path; "
                        "split: one enclosing domain against two sub-domains over a sweep of sizes (Eq. 13); "
                        "spill: cfg2 with and without the spectral history in host memory")
    p.add_argument("--no-plain", action="store_true", help="skip timing the plain direct path")
    p.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--oracle-nodes", type=int, default=8192, help="oracle sample per domain")
    p.add_argument("--mode", choices=["fft", "lowrank", "learned"], default="fft",
                   help="fft: every pair by FFT (FP32); lowrank: far pairs by bf16 tensor-core factors; "
                        "learned: far pairs by the trained stand-in (low-rank where the gate refuses)")
    p.add_argument("--learned-distance", type=float, default=2000.0)
    p.add_argument("--far-distance", type=float, default=1000.0)
    p.add_argument("--far-batch", type=int, default=32)
    p.add_argument("--source-points", type=int, default=4,
                   help="deep workloads: source nodes per axis of the two-sided far factors (0: source side exact)")
    p.add_argument("--no-deep", action="store_true", help="skip the deep workloads' lines in the default run")
    p.add_argument("--partition", choices=["replicas", "sources"], default="replicas",
                   help="N > 1: independent replicas (weak scaling), or the source partition: each rank owns some "
                        "source domains, and one reduce-scatter per step sums every target at its owner (strong "
                        "scaling)")
    return p.parse_args()


DEEP = ("cfg3", "cfg4", "cfg4x8", "cfg5", "cfg5x8", "farprobe")

# The direct sum's arithmetic per (target node, source node) pair: the offset
# (3 subtractions) and R^2 (one multiply, two FMAs: 5 flops), rsqrt, tau (two
# multiplies), floor and the hat weight (one subtraction), the 1/R volume
# factor (one multiply); per field the hat interpolation (one subtraction, one
# FMA: 3 flops), the scaling (one multiply) and the accumulation (one add),
# 5 flops x 4 fields.  Kahan compensation (3 more adds per field) is not
# counted: it is accuracy, not the sum.
DIRECT_FLOPS_PER_PAIR_POINT = 3 + 5 + 1 + 2 + 2 + 1 + 4 * 5     # = 34
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12              # 80.6


def get_workload(name):
    if name == "cfg5x8":
        w = synth.workload("cfg5")
        w.name = "cfg5x8"
        w.domains, w.sources = w.domains[:8], w.sources[:8]
        w.description = "first 8 of cfg5's 32 x 48^3 sub-domains (3000-38000 bohr apart)"
        return w
    if name == "cfg4x8":
        w = synth.workload("cfg4")
        w.name = "cfg4x8"
        w.domains, w.sources = w.domains[:8], w.sources[:8]
        w.description = ("first 8 of cfg4's 64 sub-domains: grids 24^3-96^3, spacings 0.225-0.33 bohr, "
                         "2600-16000 bohr apart")
        return w
    if name == "farprobe":
        # a small far-pair workload for profiling the far path: every cross
        # pair far (at least 300 bohr apart), a few hundred pushes before the
        # first batches of the gathered GEMM
        return synth.scattered("farprobe", 32, 32, 0.3, 1400.0, 300.0,
                               description="32 x 32^3, h=0.3 bohr, in a 1400 bohr cube at least 300 bohr apart "
                                           "(far path profiling)")
    if name == "near48":
        w = synth.two_domain(48, 0.25, 200.0, "near48", steps=100, history=40)
        w.description = "2 x 48^3, h=0.25 bohr, centres 200 bohr apart on x (small ring, for profiling)"
        return w
    return synth.workload(name)


def lag_window(w):
    """Largest lag any pair of the workload reads (for the pre-fill)."""
    from paper_2311_15429_gb300 import rp
    ctx = rp.rp_create(w.c, w.dt, flags=rp.RP_FLAG_PLAN_ONLY)
    try:
        for d in w.domains:
            rp.rp_add_domain(ctx, d.origin, d.n, d.h)
        rp.rp_finalize(ctx)
        return rp.rp_query(ctx)["max_lag"]
    finally:
        rp.rp_destroy(ctx)


# ----------------------------------------------------------------------------- dist

def dist_init(args):
    if args.gpus <= 1 and "RANK" not in os.environ:
        return 0, 1, 0
    import torch
    import torch.distributed as dist
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", args.gpus))
    local = int(os.environ.get("LOCAL_RANK", rank))
    backend = "nccl" if (args.impl == "ours" and torch.cuda.is_available()) else "gloo"
    if backend == "nccl":
        torch.cuda.set_device(local)
    dist.init_process_group(backend, rank=rank, world_size=world)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world, device=None):
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ----------------------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            import tempfile
            self.path = os.path.join(tempfile.gettempdir(), f"rp_clocks_{os.getpid()}.csv")
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ----------------------------------------------------------------------------- roofline

PER_STEP_KINDS = ("fwd_plane", "fwd_column", "mac_inv_column", "inv_plane")


def kernel_time_us(kind, ks, steps):
    """Device time matched to ``algorithmic_bytes``: per step for the kernels
    that run every step (one launch per size class, so several on mixed
    grids), per launch for the far GEMM."""
    if kind in PER_STEP_KINDS:
        return 1e3 * ks["total_ms"] / steps
    return ks["avg_us"]


def algorithmic_bytes(w, info):
    """Bytes each kernel class must move per step (all domains, every size
    class's launch), from the plan: spectra complex64, self kernels real
    float32.  The far GEMM's figure is per launch (``far_gemm_bytes``)."""
    nd = len(w.domains)
    out = {"fwd_plane": 0, "fwd_column": 0, "mac_inv_column": 0, "inv_plane": 0}
    for t in range(nd):
        m = info[(t, t)]["fft_m"]
        kx = m[0] // 2 + 1
        cells = kx * m[1] * m[2]
        Nt = w.domains[t].N
        nz = w.domains[t].n[2]
        t2 = 4 * kx * nz * m[1] * 8
        mac = t2                                          # write T2
        for s in range(nd):
            p = info[(t, s)]
            if p["kind"] != 0:
                continue
            nlag = p["lag_hi"] - p["lag_lo"] + 1
            g = cells * (4 if s == t else 8)
            mac += nlag * (g + 4 * cells * 8)
        out["mac_inv_column"] += mac
        out["inv_plane"] += t2 + 4 * Nt * 4
    for s in range(nd):
        m = info[(s, s)]["fft_m"]
        kx = m[0] // 2 + 1
        Ns = w.domains[s].N
        t1 = 4 * kx * w.domains[s].n[2] * m[1] * 8
        out["fwd_plane"] += 4 * Ns * 4 + t1
        out["fwd_column"] += t1 + 4 * kx * m[1] * m[2] * 8
    return out


def far_gemm_bytes(w, info, points, batch):
    """Bytes of one far GEMM launch (averaged over the far sources): the
    factor rows and batch matrix read (bf16 hi and lo planes, 4 bytes per
    element each), the fp32 node values written."""
    nd = len(w.domains)
    tot, n = 0, 0
    for s in range(nd):
        rows = 0
        for t in range(nd):
            p = info[(t, s)]
            if p["kind"] == 2:
                r = 1
                for a in range(3):
                    r *= min(points, w.domains[t].n[a])
                rows += (p["lag_hi"] - p["lag_lo"] + 1) * r
        if not rows:
            continue
        rows = (rows + 127) // 128 * 128
        ks = (w.domains[s].N + 63) // 64 * 64
        tot += rows * ks * 4 + 4 * batch * ks * 4 + rows * 4 * batch * 4
        n += 1
    return tot / max(n, 1)


def measured_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def committed_traffic(kernel, workload):
    """dram bytes per launch from the committed ncu summary, if it was taken
    on the current source of the kernel (the file its summary names under
    ``kernel_source:``), else None."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_{workload}.md")
    if not os.path.exists(path):
        return None
    txt = open(path).read()
    m1 = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", txt)
    m2 = re.search(r"kernel_source_sha256:\s*([0-9a-f]{64})", txt)
    m3 = re.search(r"kernel_source:\s*(\S+)", txt)
    if not m1 or not m2 or not m3:
        return None
    src = os.path.join(ROOT, "paper_2311_15429_gb300", "csrc", os.path.basename(m3.group(1)))
    if not os.path.exists(src) or hashlib.sha256(open(src, "rb").read()).hexdigest() != m2.group(1):
        return None
    return float(m1.group(1))


# ----------------------------------------------------------------------------- oracle

def oracle_sample(w, hists, j0, step, nodes_per_dom, seed=0):
    """Oracle at seeded sample nodes of every domain.  Returns (values per
    domain, nodes per domain, wall seconds, threads)."""
    import oracle
    rng = np.random.default_rng(seed)
    vals, nodes, threads = [], [], 1
    t0 = time.perf_counter()
    for t, d in enumerate(w.domains):
        sel = np.sort(rng.choice(d.N, size=min(nodes_per_dom, d.N), replace=False))
        v, threads = oracle.eval_points_parallel([x.origin for x in w.domains], [x.n for x in w.domains],
                                                 [x.h for x in w.domains], hists, j0, w.c, w.dt, t, step, sel)
        vals.append(v)
        nodes.append(sel)
    return vals, nodes, time.perf_counter() - t0, threads


# ----------------------------------------------------------------------------- reference arm

def run_reference(args, rank, world):
    if rank != 0:
        return
    import oracle
    w = get_workload(args.workload)
    lag = oracle.history_needed([d.origin for d in w.domains], [d.n for d in w.domains], [d.h for d in w.domains],
                                w.c, w.dt)
    W, K = args.warmup, args.steps
    hists = [s.history(-lag - 1, 1, w.dt) for s in w.sources]
    cores = os.cpu_count() or 1
    # calibrate with one node per thread per domain, then size the per-step
    # sample so that the whole run stays within ~90 s of wall time
    _, _, t_cal, _ = oracle_sample(w, hists, -lag - 1, 0, cores, seed=99)
    per_step_budget = 90.0 / max(1, K + W)
    nodes_per_dom = max(1, int(cores * per_step_budget / max(t_cal, 1e-9)))
    nodes_per_dom = min(nodes_per_dom, min(d.N for d in w.domains))
    for i in range(W):
        oracle_sample(w, hists, -lag - 1, 0, nodes_per_dom, seed=1000 + i)
    t_total = 0.0
    for i in range(K):
        _, _, dt_, threads = oracle_sample(w, hists, -lag - 1, 0, nodes_per_dom, seed=i)
        t_total += dt_
    pts = nodes_per_dom * len(w.domains)
    value = pts * K / t_total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": K, "warmup": W, "ms_per_step": 1e3 * t_total / K, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w.name, "description": w.description, "points_per_step": w.points},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": f"{nodes_per_dom} seeded target nodes per domain per step, "
                                   f"all {w.points} source nodes, FP64 direct retarded sum"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- our arm

def run_ours(args, rank, world, local):
    import torch
    from paper_2311_15429_gb300 import rp
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    w = get_workload(args.workload)
    lag = lag_window(w)
    W, K = args.warmup, args.steps
    ncycle = min(max(w.steps, 8), 100)
    pre = lag + 1
    depth = max(w.history, lag + 1)

    # host history: pre-fill (pre slices, t < 0) then ncycle slices; inputs on
    # the device for the timed region: ncycle slices per domain, cycled
    hists = [s.history(-pre, ncycle, w.dt) for s in w.sources]
    dev_in = [torch.from_numpy(h).to(dev) for h in hists]            # [T][4][N]
    rho = [[dev_in[d][i, 0] for d in range(len(w.domains))] for i in range(pre + ncycle)]
    J = [[dev_in[d][i, 1:].reshape(-1) for d in range(len(w.domains))] for i in range(pre + ncycle)]
    in_bytes = sum(x.numel() * 4 for x in dev_in)

    mode = rp.RP_MODE_LOWRANK if args.mode == "lowrank" else rp.RP_MODE_FFT
    # overlapped pushes: the inputs are complete device tensors when each push
    # is called, so rp_push_all_event lets step l+1's push run beside step l's
    # evaluation (same bits as sequential pushes, timed beside it below)
    lib = rp.RetardedPotentials(w.domains, w.c, w.dt, history_depth=depth, mode=mode, device=local, stream=stream,
                                far_distance=args.far_distance, far_batch=args.far_batch,
                                flags=rp.RP_FLAG_OVERLAP_PUSH)
    push = lambda r, j: rp.rp_push_all_event(lib.ctx, r, j)
    info = {(t, s): lib.pair_info(t, s) for t in range(len(w.domains)) for s in range(len(w.domains))}
    mac_warps = lib.query()["mac_warps"]
    for i in range(pre):
        push(rho[i], J[i])
    # warm-up on continuous time (t = 0, dt, ...), the accuracy check on the
    # last continuous step, then the rest of the warm-up on cycled inputs
    nwc = min(W, ncycle)
    for i in range(nwc):
        push(rho[pre + i], J[pre + i])
        lib.evaluate()
    lib.sync()
    check_step = nwc - 1
    acc = None
    cpu = None
    gpu_check = None
    if rank == 0 and check_step >= 0:
        gpu_check = [torch.cat([lib.phi[d], lib.A[d]]).cpu().numpy() for d in range(len(w.domains))]
    if rank == 0 and not args.no_cpu and check_step >= 0:
        gpu_vals = [torch.cat([lib.phi[d][None], lib.A[d].reshape(3, -1)]).cpu().numpy()
                    for d in range(len(w.domains))]
        ovals, onodes, t_or, threads = oracle_sample(w, hists, -pre, check_step, args.oracle_nodes)
        errs = []
        for d in range(len(w.domains)):
            g = gpu_vals[d][:, onodes[d]]
            for f in range(4):
                errs.append(float(np.linalg.norm(g[f] - ovals[d][:, f]) / np.linalg.norm(ovals[d][:, f])))
        npts = sum(len(n) for n in onodes)
        acc = {"rel_l2_max": max(errs), "rel_l2_per_field_domain": errs,
               "checked": f"{npts} sampled nodes at step t={check_step * w.dt:.2f} vs FP64 oracle"}
        if args.mode == "lowrank" and lib.query()["npairs_far"]:
            acc["far_field_only"] = far_only_error(args, w, hists, rho, J, pre, check_step, depth, local,
                                                   stream, info)
        pair_points = npts * w.points                 # every sampled target node sums every source node
        cpu = {"value": npts / t_or, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": f"{args.oracle_nodes} seeded target nodes per domain x all {w.points} "
                         f"source nodes at one step ({t_or:.1f} s wall)",
               "pair_points_per_s_per_core": pair_points / t_or / max(threads, 1),
               "full_step_s_extrapolated": w.points * w.points / (pair_points / t_or)}
    for i in range(W - nwc):
        k = pre + (nwc + i) % ncycle
        push(rho[k], J[k])
        lib.evaluate()
    lib.sync()

    # ---- timed region (device-resident inputs; no events between kernels)
    prho = {k: rp.pointer_array(rho[k]) for k in range(pre, pre + ncycle)}
    pJ = {k: rp.pointer_array(J[k]) for k in range(pre, pre + ncycle)}
    pphi, pA = rp.pointer_array(lib.phi), rp.pointer_array(lib.A)
    rp.rp_kernel_stats(lib.ctx, 0, reset=True)
    clocks = ClockSampler(local)
    barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.15)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(K):
        k = pre + (W + i) % ncycle
        rp.rp_push_all_event(lib.ctx, prho[k], pJ[k])
        rp.rp_evaluate(lib.ctx, pphi, pA)
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    barrier(world)
    ms = e0.elapsed_time(e1)
    ms_max = max_over_ranks(ms, world, dev)
    value = world * w.points * K / (ms_max / 1e3)
    launches = sum(rp.rp_kernel_count(lib.ctx, kind) for kind in range(rp.RP_K_COUNT))
    # ---- kernel times: a separate pass on the same context, every launch
    # bracketed by CUDA events on the context stream
    Kp = kernel_pass_steps(K)
    kstats = kernel_pass(lib, Kp, lambda i: (prho[pre + (W + K + i) % ncycle], pJ[pre + (W + K + i) % ncycle]),
                         pphi, pA)
    alg = algorithmic_bytes(w, info)
    alg["far_gemm"] = far_gemm_bytes(w, info, 4, args.far_batch)
    dom = max(kstats, key=lambda k: kstats[k]["total_ms"])
    peak, peak_kind = measured_peak()
    ach = alg[dom] / (kernel_time_us(dom, kstats[dom], Kp) * 1e-6) / 1e9
    roof = {"bound": "hbm", "kernel": dom, "achieved": ach, "peak": peak, "unit": "GB/s",
            "frac": ach / peak, "peak_source": f"{peak_kind} hbm_gbs (copy bandwidth)",
            "traffic": committed_traffic(dom, w.name),
            "algorithmic_bytes_per_launch": alg[dom],
            "time_basis": "per step (all launches of the step)" if dom in PER_STEP_KINDS else "per launch"}
    for k in kstats:
        if k in alg:
            kstats[k]["algorithmic_GBps"] = alg[k] / (kernel_time_us(k, kstats[k], Kp) * 1e-6) / 1e9

    # ---- the same step replayed as a CUDA graph (rp_graph_capture / rp_graph_step)
    # on a context without profiling; each step's slices are copied into the
    # captured input buffers first (device to device, on the stream)
    graph = None
    if rank == 0 and args.mode == "fft":
        nd = len(w.domains)
        with rp.RetardedPotentials(w.domains, w.c, w.dt, history_depth=depth, device=local, stream=stream) as gl:
            for i in range(pre):
                gl.push_all(rho[i], J[i])
            grho = [torch.empty(d.N, device=dev) for d in w.domains]
            gJ = [torch.empty(3 * d.N, device=dev) for d in w.domains]
            rp.rp_graph_capture(gl.ctx, grho, gJ, gl.phi, gl.A)
            def gstep(k):
                for d in range(nd):
                    grho[d].copy_(rho[k][d])
                    gJ[d].copy_(J[k][d])
                rp.rp_graph_step(gl.ctx)
            for i in range(W):
                gstep(pre + i % ncycle)
            torch.cuda.synchronize()
            ga, gb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ga.record(stream)
            for i in range(K):
                gstep(pre + (W + i) % ncycle)
            gb.record(stream)
            torch.cuda.synchronize()
            gms = ga.elapsed_time(gb) / K
        graph = {"ms_per_step": gms, "value": w.points / (gms / 1e3), "unit": UNIT, "steps": K,
                 "note": "one graph launch per step (step counter, forward passes, MAC, inverse passes) after "
                         "device-to-device copies of the step's slices into the captured buffers"}

    # ---- FP64 audit on the GPU, and the compensated pair sum: two more
    # contexts on the same inputs.  RP_FLAG_AUDIT only adds the raw history
    # ring, so its outputs must equal the headline context's bit for bit;
    # its audit is the headline's.  The compensated context is audited too,
    # and both are timed on the same K steps (their difference is the cost
    # of compensation).
    audit, comp = None, None
    if rank == 0 and args.mode == "fft" and check_step >= 0:
        legs = {}
        for name, fl in (("audit", rp.RP_FLAG_AUDIT), ("plain_sum", rp.RP_FLAG_AUDIT | rp.RP_FLAG_PLAIN_SUM)):
            with rp.RetardedPotentials(w.domains, w.c, w.dt, history_depth=depth, flags=fl, device=local,
                                       stream=stream) as al:
                for i in range(pre + nwc):
                    al.push_all(rho[i], J[i])
                    if i >= pre:
                        al.evaluate()
                al.sync()
                rel = rp.rp_audit(al.ctx, al.phi, al.A, 1024, seed=11)
                same = None
                if name == "audit":
                    same = all(torch.equal(torch.cat([al.phi[d], al.A[d]]), torch.from_numpy(gpu_check[d]).to(dev))
                               for d in range(len(w.domains))) if gpu_check is not None else None
                aphi, aA = rp.pointer_array(al.phi), rp.pointer_array(al.A)
                for i in range(3):
                    k = pre + (nwc + i) % ncycle
                    rp.rp_push_all(al.ctx, prho[k], pJ[k])
                    rp.rp_evaluate(al.ctx, aphi, aA)
                torch.cuda.synchronize()
                ta, tb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                ta.record(stream)
                for i in range(K):
                    k = pre + (W + i) % ncycle
                    rp.rp_push_all(al.ctx, prho[k], pJ[k])
                    rp.rp_evaluate(al.ctx, aphi, aA)
                tb.record(stream)
                torch.cuda.synchronize()
                legs[name] = {"ms_per_step": ta.elapsed_time(tb) / K, "rel_l2_max": float(rel.max()),
                              "rel_l2_per_domain_field": rel.tolist(), "bit_identical_to_headline": same}
        audit = {"rel_l2_max": legs["audit"]["rel_l2_max"],
                 "rel_l2_per_domain_field": legs["audit"]["rel_l2_per_domain_field"],
                 "checked": f"1024 seeded nodes per domain at step t={check_step * w.dt:.2f}: FP64 direct sum on the "
                            f"GPU from the context's own history (rp_audit, RP_FLAG_AUDIT)",
                 "outputs_bit_identical_to_headline": legs["audit"]["bit_identical_to_headline"],
                 "ms_per_step_with_audit_ring": legs["audit"]["ms_per_step"]}
        comp = {"headline_sum": "Kahan-compensated spectral sum over (source, lag) entries (the default)",
                "plain_sum": {"flag": "RP_FLAG_PLAIN_SUM", "ms_per_step": legs["plain_sum"]["ms_per_step"],
                              "value": w.points / (legs["plain_sum"]["ms_per_step"] / 1e3), "unit": UNIT,
                              "rel_l2_max_gpu_audit": legs["plain_sum"]["rel_l2_max"]},
                "compensated_rel_l2_max_gpu_audit": legs["audit"]["rel_l2_max"],
                "cost_of_compensation_ms_per_step": legs["audit"]["ms_per_step"] - legs["plain_sum"]["ms_per_step"],
                "note": "both legs keep the audit ring, so their step-time difference is the compensation alone"}

    # ---- the same step with sequential pushes (no RP_FLAG_OVERLAP_PUSH): each
    # push's kernels after the previous evaluation on the context stream
    sequential = None
    if rank == 0 and args.mode == "fft":
        with rp.RetardedPotentials(w.domains, w.c, w.dt, history_depth=depth, device=local, stream=stream) as sl:
            for i in range(pre):
                sl.push_all(rho[i], J[i])
            sphi, sA = rp.pointer_array(sl.phi), rp.pointer_array(sl.A)
            for i in range(W):
                k = pre + i % ncycle
                rp.rp_push_all(sl.ctx, prho[k], pJ[k])
                rp.rp_evaluate(sl.ctx, sphi, sA)
            torch.cuda.synchronize()
            sa, sb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            sa.record(stream)
            for i in range(K):
                k = pre + (W + i) % ncycle
                rp.rp_push_all(sl.ctx, prho[k], pJ[k])
                rp.rp_evaluate(sl.ctx, sphi, sA)
            sb.record(stream)
            torch.cuda.synchronize()
            sms = sa.elapsed_time(sb) / K
        sequential = {"ms_per_step": sms, "value": w.points / (sms / 1e3), "unit": UNIT,
                      "note": "rp_push_all + rp_evaluate on a context without RP_FLAG_OVERLAP_PUSH: every push "
                              "after the previous evaluation (the headline overlaps them; same bits)"}

    # ---- the fields of App. B from the last potentials (rp_fields), timed alone:
    # per point it reads phi and three A's (10 floats) and writes E and B (6)
    fields = None
    if rank == 0:
        nd = len(w.domains)
        A1 = [lib.A[d].clone() for d in range(nd)]
        A2 = [lib.A[d].clone() for d in range(nd)]
        E = [torch.empty_like(lib.A[d]) for d in range(nd)]
        B = [torch.empty_like(lib.A[d]) for d in range(nd)]
        reps = 200
        for _ in range(3):
            for d in range(nd):
                rp.rp_fields(lib.ctx, d, lib.phi[d], lib.A[d], A1[d], A2[d], E[d], B[d])
        torch.cuda.synchronize()
        fa, fb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        fa.record(stream)
        for _ in range(reps):
            for d in range(nd):
                rp.rp_fields(lib.ctx, d, lib.phi[d], lib.A[d], A1[d], A2[d], E[d], B[d])
        fb.record(stream)
        torch.cuda.synchronize()
        us = 1e3 * fa.elapsed_time(fb) / (reps * nd)
        fbytes = 64 * w.points / nd
        fields = {"kernel": "k_fields (E and B, one launch per domain)", "avg_us": us,
                  "algorithmic_bytes_per_launch": fbytes, "achieved_GBps": fbytes / (us * 1e-6) / 1e9,
                  "frac_of_peak": fbytes / (us * 1e-6) / 1e9 / peak, "launches": reps * nd,
                  "note": "timed alone after the step loop, 64 B per point (phi, 3 x A in; E, B out)"}

    # ---- plain path: direct FP32 sum of every pair
    plain = None
    if not args.no_plain and rank == 0:
        with rp.RetardedPotentials(w.domains, w.c, w.dt, history_depth=depth, mode=rp.RP_MODE_DIRECT,
                                   device=local, stream=stream) as dl:
            for i in range(pre):
                dl.push_all(rho[i], J[i])
            nplain = 3
            for i in range(1):
                dl.push_all(rho[pre], J[pre])
                dl.evaluate()
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for i in range(nplain):
                k = pre + 1 + i
                dl.push_all(rho[k], J[k])
                dl.evaluate()
            b.record(stream)
            torch.cuda.synchronize()
            pms = a.elapsed_time(b) / nplain
            # ALU roofline of the direct sum: pair-points per step (every
            # target node against every source node), 32 algorithmic flops
            # each, against the FP32 pipes' peak at the SM clock
            pp = sum(t.N for t in w.domains) * sum(s_.N for s_ in w.domains)
            achieved = pp * DIRECT_FLOPS_PER_PAIR_POINT / (pms * 1e-3) / 1e12
            plain = {"path": "direct FP32 retarded sum, every pair (Kahan-compensated)",
                     "value": w.points / (pms / 1e3), "unit": UNIT, "ms_per_step": pms, "steps": nplain,
                     "speedup_of_ours": (w.points / (ms / K / 1e3)) / (w.points / (pms / 1e3)),
                     "pair_points_per_s": pp / (pms * 1e-3),
                     "roofline": {"bound": "alu", "achieved": achieved, "peak": FP32_PEAK_TFLOPS,
                                  "unit": "TFLOP/s", "frac": achieved / FP32_PEAK_TFLOPS,
                                  "flops_per_pair_point": DIRECT_FLOPS_PER_PAIR_POINT,
                                  "peak_source": "152 SMs x 128 FP32 lanes x 2 flop (FMA) x 2070 MHz: nominal "
                                                 "unit counts at the maximum SM clock (derived, not measured)"}}

    # ---- end to end through the C-ABI with host buffers
    e2e = None
    if not args.no_e2e:
        ctx = lib.ctx
        nd = len(w.domains)
        hin = [torch.from_numpy(h).pin_memory() for h in hists]
        hout = [torch.empty(4 * d.N, dtype=torch.float32).pin_memory() for d in w.domains]
        hphi = [hout[d][: w.domains[d].N] for d in range(nd)]
        hA = [hout[d][w.domains[d].N:] for d in range(nd)]
        # per-step pointer arrays, made once (rho and J of a slice are adjacent: one copy each)
        prho = {k: rp.pointer_array([hin[d][k, 0] for d in range(nd)]) for k in range(pre, pre + ncycle)}
        pJ = {k: rp.pointer_array([hin[d][k, 1:].reshape(-1) for d in range(nd)]) for k in range(pre, pre + ncycle)}
        pphi, pA = rp.pointer_array(hphi), rp.pointer_array(hA)
        for i in range(3):
            k = pre + i % ncycle
            rp.rp_push_all_host(ctx, prho[k], pJ[k])
            rp.rp_evaluate_host(ctx, pphi, pA)
        rp.rp_sync(ctx)
        Ke = max(1, min(K, 500))
        barrier(world)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        a.record(stream)
        for i in range(Ke):
            k = pre + i % ncycle
            rp.rp_push_all_host(ctx, prho[k], pJ[k])
            rp.rp_evaluate_host(ctx, pphi, pA)
        # the last copies out run on the library's copy stream: wait for both
        # streams, then close the interval on the context stream
        rp.rp_sync(ctx)
        b.record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        ems = max_over_ranks(a.elapsed_time(b), world, dev)
        e2e = {"value": world * w.points * Ke / (ems / 1e3), "unit": UNIT,
               "h2d_bytes_per_step": sum(4 * 4 * d.N for d in w.domains),
               "d2h_bytes_per_step": sum(4 * 4 * d.N for d in w.domains),
               "steps": Ke, "host_wall_s": wall,
               "api": "rp_push_all_host + rp_evaluate_host, pinned host buffers (copies on the library's two copy "
                      "streams, overlapped with the kernels of neighbouring steps)"}
    lib.close()

    # ---- the deep workloads (every cross pair far, thousands-deep histories):
    # each chosen form timed on K steps beside its plain FP32 path (extrapolated)
    deep = None
    if rank == 0 and not args.no_deep and args.mode == "fft":
        deep = {}
        for key, name, mode, plain_leg in (("cfg3", "cfg3", "lowrank", True), ("cfg4", "cfg4", "lowrank", True),
                                           ("cfg5", "cfg5", "lowrank", True),
                                           ("cfg5_learned", "cfg5", "learned", False)):
            try:
                deep[key] = deep_leg(args, name, min(K, 64), max(W, 3), local, stream, mode=mode,
                                     source_points=args.source_points, check=not args.no_cpu, plain=plain_leg)
            except Exception as e:   # one workload's failure must not lose the line
                deep[key] = {"error": f"{type(e).__name__}: {e}"}
            torch.cuda.empty_cache()

    if rank != 0:
        return
    q_points = w.points
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": ms_max / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "pair_points_per_s": world * sum(t.N * s_.N for t in w.domains for s_ in w.domains) * K / (ms_max / 1e3),
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": w.name, "description": w.description, "points_per_step": q_points,
                   "path": ("FFT: Hockney self term + delay-binned cross pairs, spectral history ring, "
                            "Kahan-compensated spectral pair sum, overlapped pushes (rp_push_all_event)"
                            if args.mode == "fft" else
                            f"FFT self/near pairs; pairs >= {args.far_distance} bohr apart by bf16 tcgen05 "
                            f"low-rank factors (4^3 interpolation nodes, {args.far_batch}-step batches)"),
                   "l2": f"inputs larger than L2: {ncycle} distinct input slices per domain cycled "
                         f"({in_bytes / 2**20:.0f} MiB), spectral ring "
                         f"{lib_bytes_str(w, info, depth)} read per step",
                   "mac_consumer_warps": mac_warps,
                   "kernel_timing": f"timed steps without events between kernels; kernel times from a separate "
                                    f"pass of {Kp} steps right after it on the same context and inputs, CUDA events "
                                    f"around every launch on the context stream; gpu_launches counted in the timed "
                                    f"steps",
                   "parallelism": f"{world} independent replicas" if world > 1 else "1 GPU"},
        "accuracy": acc,
        "gpu_audit": audit,
        "pair_sum": comp,
        "sequential_push": sequential,
        "plain_path": plain,
        "roofline": roof,
        "kernels": kstats,
        "fields": fields,
        "graph_replay": graph,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clk,
        "deep_configs": deep,
    }
    print(json.dumps(line), flush=True)


def kernel_pass(lib, steps, inputs, pphi, pA):
    """Time every launch of `steps` more steps with CUDA events (the
    library's rp_set_profiling), then switch the events off again.  Returns
    per kernel class its launches, average and total device time."""
    from paper_2311_15429_gb300 import rp
    rp.rp_sync(lib.ctx)
    rp.rp_set_profiling(lib.ctx, 1)
    rp.rp_kernel_stats(lib.ctx, 0, reset=True)
    for i in range(steps):
        r, j = inputs(i)
        rp.rp_push_all(lib.ctx, r, j)
        rp.rp_evaluate(lib.ctx, pphi, pA)
    out = {}
    for kind in range(rp.RP_K_COUNT):
        n, t = rp.rp_kernel_stats(lib.ctx, kind)
        if n:
            out[rp.rp_kernel_name(kind)] = {"launches": n, "avg_us": 1e3 * t / n, "total_ms": t, "pass_steps": steps}
    rp.rp_set_profiling(lib.ctx, 0)
    rp.rp_kernel_stats(lib.ctx, 0, reset=True)
    return out


def far_only_error(args, w, hists, rho, J, pre, check_step, depth, local, stream, info):
    """rel-L2 of the far field alone: domain 0 the only active source, seen
    from the domains it reaches by the far path (sampled nodes, FP64 oracle)."""
    import torch
    from paper_2311_15429_gb300 import rp
    tg = [t for t in range(1, len(w.domains)) if info[(t, 0)]["kind"] == 2]
    if not tg:
        return None
    zr = [torch.zeros_like(x) for x in rho[0]]
    zJ = [torch.zeros_like(x) for x in J[0]]
    with rp.RetardedPotentials(w.domains, w.c, w.dt, history_depth=depth, mode=rp.RP_MODE_LOWRANK,
                               device=local, stream=stream, far_distance=args.far_distance,
                               far_batch=args.far_batch) as lf:
        for i in range(pre + check_step + 1):
            lf.push_all([rho[i][0]] + zr[1:], [J[i][0]] + zJ[1:])
        lf.evaluate()
        lf.sync()
        vals = [torch.cat([lf.phi[d][None], lf.A[d].reshape(3, -1)]).cpu().numpy() for d in tg]
    only = [hists[0]] + [np.zeros_like(h) for h in hists[1:]]
    ovals, onodes, _, _ = oracle_sample(w, only, -pre, check_step, 1024, seed=5)
    errs = []
    for k, t in enumerate(tg):
        g = vals[k][:, onodes[t]]
        for f in range(4):
            errs.append(float(np.linalg.norm(g[f] - ovals[t][:, f]) / np.linalg.norm(ovals[t][:, f])))
    return {"rel_l2_max": max(errs), "per_field": errs, "source": 0, "targets": tg}


def lib_bytes_str(w, info, depth):
    alg = algorithmic_bytes(w, info)
    return f"{alg['mac_inv_column'] / 2**20:.0f} MiB"


# Far distance of the low-rank pairs per deep workload: every cross pair of
# cfg4 is more than 250 bohr apart (cfg3 and cfg5: 500).
DEEP_FAR_DISTANCE = {"cfg3": 500.0, "cfg4": 250.0, "cfg4x8": 500.0, "cfg5": 500.0, "cfg5x8": 500.0,
                     "farprobe": 250.0}


def far_gather_work(lib, w, info, batch, source_points):
    """Algorithmic work of one gathered-GEMM launch (two-sided factors): per
    (target, far source, lag) block, 128 x BN x KS bf16 products three times
    (hi*hi, hi*lo, lo*hi); bytes: the factor blocks (bf16 hi and lo), the
    blocks' coefficient windows (128 rows x 2 KS bf16) and the partial sums
    written (128 x BN fp32 per CTA, an upper bound of 24 blocks per CTA)."""
    nd = len(w.domains)
    q = source_points
    KS = (q ** 3 + 63) // 64 * 64
    r = max(min(4, d.n[0]) * min(4, d.n[1]) * min(4, d.n[2]) for d in w.domains)
    BN = next(b for b in (32, 64, 128, 256) if r <= b)
    blocks = sum(info[(t, s)]["lag_hi"] - info[(t, s)]["lag_lo"] + 1 for t in range(nd) for s in range(nd)
                 if info[(t, s)]["kind"] == 2)
    flops = blocks * 3 * 2 * 128 * BN * KS
    by = blocks * (BN * 2 * KS * 2 + 128 * 2 * KS * 2) + (blocks // 24 + nd) * 128 * BN * 4
    return flops, by, blocks


def calibrate_fft_costs(w, local, stream, steps=24):
    """Measured costs of the plain FFT path per size class of w: two cubic
    n^3 domains of the class's spacing 3 box widths apart, FFT mode, every
    launch timed.  Returns {n: (forward passes us per source, inverse plane
    us per target, MAC us per (source, lag) entry)}."""
    import torch
    from paper_2311_15429_gb300 import rp
    dev = torch.device("cuda", local)
    out = {}
    for n in sorted({d.n[0] for d in w.domains}):
        h = next(d.h for d in w.domains if d.n[0] == n)
        cw = synth.two_domain(n, h, 3.0 * n * h, "cal")
        gen = synth.DeviceSlices(cw.sources, dev)
        with rp.RetardedPotentials(cw.domains, cw.c, cw.dt, flags=rp.RP_FLAG_GROUND_STATE_CLAMP, device=local,
                                   stream=stream) as lib:
            entries = sum(lib.pair_info(t, s)["lag_hi"] - lib.pair_info(t, s)["lag_lo"] + 1
                          for t in range(2) for s in range(2))
            sl = [gen.step(j, cw.dt) for j in range(4)]
            for j in range(4):
                lib.push_all(*sl[j])
                lib.evaluate()
            pphi, pA = rp.pointer_array(lib.phi), rp.pointer_array(lib.A)
            ps = [(rp.pointer_array(r), rp.pointer_array(J)) for r, J in sl]
            ks = kernel_pass(lib, steps, lambda i: ps[i % 4], pphi, pA)
        per = lambda k: 1e3 * ks[k]["total_ms"] / steps if k in ks else 0.0
        out[n] = ((per("fwd_plane") + per("fwd_column")) / 2, per("inv_plane") / 2, per("mac_inv_column") / entries)
    return out


def calibrate_direct_rate(local, stream, steps=3):
    """Pair-points per second of the plain direct FP32 sum (two 24^3 domains
    of unequal spacing in RP_MODE_DIRECT)."""
    import torch
    from paper_2311_15429_gb300 import rp
    dev = torch.device("cuda", local)
    doms = [synth.cubic((0.0, 0.0, 0.0), 24, 0.25), synth.cubic((30.0, 0.0, 0.0), 24, 0.3)]
    gen = synth.DeviceSlices(synth.seeded_sources(doms), dev)
    with rp.RetardedPotentials(doms, synth.C_AU, 0.05, mode=rp.RP_MODE_DIRECT, flags=rp.RP_FLAG_GROUND_STATE_CLAMP,
                               device=local, stream=stream) as lib:
        lib.push_all(*gen.step(0, 0.05))
        lib.evaluate()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for j in range(steps):
            lib.push_all(*gen.step(j + 1, 0.05))
            lib.evaluate()
        b.record(stream)
        torch.cuda.synchronize()
    return (2 * doms[0].N) ** 2 * steps / (a.elapsed_time(b) * 1e-3)


def plain_path_extrapolated(w, info, costs, direct_rate):
    """The plain FP32 path of every pair (the per-pair unbatched FFT path:
    self and equal-spacing cross pairs by FFT, one entry per lag; pairs of
    unequal spacing by the direct sum), whose histories do not fit the GPU
    for these workloads: its step time from the per-class costs measured by
    calibrate_fft_costs and the direct sum's measured rate, scaled by the
    workload's (pair, lag) count and pair-points."""
    nd = len(w.domains)
    t_us = 0.0
    entries, direct_pp = 0, 0
    for t in range(nd):
        fwd, inv, _ = costs[w.domains[t].n[0]]
        t_us += fwd + inv
        for s in range(nd):
            p = info[(t, s)]
            if t == s or abs(w.domains[t].h - w.domains[s].h) <= 1e-12 * w.domains[t].h:
                n = max(w.domains[t].n[0], w.domains[s].n[0])
                B = p["lag_hi"] - p["lag_lo"] + 1
                t_us += B * costs[n][2]
                entries += B
            else:
                direct_pp += w.domains[t].N * w.domains[s].N
    t_us += 1e6 * direct_pp / direct_rate
    return {"ms_per_step": t_us / 1e3, "value": w.points / (t_us * 1e-6), "unit": UNIT, "extrapolated": True,
            "fft_entries_per_step": entries, "direct_pair_points_per_step": direct_pp,
            "method": "per-class forward/inverse pass and per-(source, lag) MAC costs measured on two n^3 domains in "
                      "FFT mode, direct-sum pair-points/s measured in RP_MODE_DIRECT, scaled by this workload's "
                      "entries and pair-points (its full-depth spectral histories do not fit the GPU)"}


def deep_leg(args, name, K, W, local, stream, mode="lowrank", source_points=4, check=True, plain=True):
    """One deep workload (every cross pair far) on the chosen form: the timed
    steps (device-made inputs, no events between kernels), a kernel pass, the
    total and far-only error at sampled nodes against the FP64 oracle with a
    stored window per source, and the plain FP32 path extrapolated."""
    import torch
    import oracle
    from paper_2311_15429_gb300 import rp
    dev = torch.device("cuda", local)
    w = get_workload(name)
    flags = rp.RP_FLAG_DEFER_FAR if mode == "learned" else 0
    fd = DEEP_FAR_DISTANCE.get(name, args.far_distance)
    t0 = time.perf_counter()
    gen = synth.DeviceSlices(w.sources, dev)
    lib = rp.RetardedPotentials(w.domains, w.c, w.dt, mode=rp.RP_MODE_LOWRANK, flags=flags, device=local,
                                stream=stream, far_distance=fd, far_batch=args.far_batch,
                                far_source_points=source_points)
    train = lib.train_far_model(args.learned_distance) if mode == "learned" else None
    q = lib.query()
    nd = len(w.domains)
    info = {(t, s): lib.pair_info(t, s) for t in range(nd) for s in range(nd)}
    pre = q["max_lag"] + 1
    for j in range(pre + W):
        r, J = gen.step(j - pre, w.dt)
        lib.push_all(r, J)
        if j >= pre:
            lib.evaluate()
    lib.sync()
    setup_s = time.perf_counter() - t0
    step_t = W - 1                       # time index of the last continuous step
    acc = None
    if check:
        tgts = sorted({1, nd // 2, nd - 1})
        got = {t: torch.cat([lib.phi[t][None], lib.A[t].reshape(3, -1)]).cpu().numpy() for t in tgts}
        rng = np.random.default_rng(0)
        errs, far_errs = [], []
        tc = time.perf_counter()
        for t in tgts:
            hists, firsts = [], []
            for s in range(nd):
                p = info[(t, s)]
                lo, hi = step_t - p["lag_hi"] - 1, step_t - p["lag_lo"]
                hists.append(w.sources[s].history(lo, hi + 1, w.dt))
                firsts.append(lo)
            nodes = np.sort(rng.choice(w.domains[t].N, 48, replace=False))
            args_o = ([d.origin for d in w.domains], [d.n for d in w.domains], [d.h for d in w.domains])
            vals, _ = oracle.eval_points_windows_parallel(*args_o, hists, firsts, w.c, w.dt, t, step_t, nodes)
            own = [hh if s == t else np.zeros_like(hh) for s, hh in enumerate(hists)]
            selfv, _ = oracle.eval_points_windows_parallel(*args_o, own, firsts, w.c, w.dt, t, step_t, nodes)
            g = got[t][:, nodes]
            for f in range(4):
                errs.append(float(np.linalg.norm(g[f] - vals[:, f]) / np.linalg.norm(vals[:, f])))
                far_errs.append(float(np.linalg.norm(g[f] - vals[:, f]) / np.linalg.norm(vals[:, f] - selfv[:, f])))
        acc = {"rel_l2_max": max(errs), "total_error_over_far_field_max": max(far_errs),
               "checked": f"48 seeded nodes of domains {tgts} at t={step_t * w.dt:.2f} against the FP64 oracle "
                          f"({time.perf_counter() - tc:.1f} s); total_error_over_far_field: the total's error over "
                          f"the oracle's sum of the other domains alone (the self term's FP32 error included)"}
        acc["far_field_alone"] = far_alone_check(args, w, mode, source_points, fd, tgts, local, stream, lib)
    # timed region: cycled device inputs, no events between kernels
    ncycle = 16
    cyc = [gen.step(W + i, w.dt) for i in range(ncycle)]
    pcyc = [(rp.pointer_array(r), rp.pointer_array(J)) for r, J in cyc]
    pphi, pA = rp.pointer_array(lib.phi), rp.pointer_array(lib.A)
    rp.rp_kernel_stats(lib.ctx, 0, reset=True)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(K):
        r, J = pcyc[i % ncycle]
        rp.rp_push_all(lib.ctx, r, J)
        rp.rp_evaluate(lib.ctx, pphi, pA)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    launches = sum(rp.rp_kernel_count(lib.ctx, kind) for kind in range(rp.RP_K_COUNT))
    Kp = max(args.far_batch, kernel_pass_steps(K) // args.far_batch * args.far_batch)
    kstats = kernel_pass(lib, Kp, lambda i: pcyc[(K + i) % ncycle], pphi, pA)
    alg = algorithmic_bytes(w, info)
    peak, peak_kind = measured_peak()
    for k in kstats:
        if k in alg:
            kstats[k]["algorithmic_GBps"] = alg[k] / (kernel_time_us(k, kstats[k], Kp) * 1e-6) / 1e9
    dom = max(kstats, key=lambda k: kstats[k]["total_ms"])
    roof = None
    if dom in alg:
        ach = alg[dom] / (kernel_time_us(dom, kstats[dom], Kp) * 1e-6) / 1e9
        roof = {"bound": "hbm", "kernel": dom, "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                "peak_source": f"{peak_kind} hbm_gbs (copy bandwidth)", "traffic": committed_traffic(dom, w.name),
                "algorithmic_bytes_per_launch": alg[dom],
                "time_basis": "per step (all launches of the step)" if dom in PER_STEP_KINDS else "per launch"}
    far_roof = None
    if source_points and "far_gemm" in kstats:
        fl, by, blocks = far_gather_work(lib, w, info, args.far_batch, source_points)
        us = kstats["far_gemm"]["avg_us"]
        bf16 = bf16_peak()
        far_roof = {"kernel": "k_far_gather (tcgen05, bf16 hi/lo, three products)", "blocks": blocks,
                    "avg_us": us, "tflops": fl / (us * 1e-6) / 1e12, "tensor_peak": bf16[0],
                    "tensor_frac": fl / (us * 1e-6) / 1e12 / bf16[0], "gbps": by / (us * 1e-6) / 1e9,
                    "hbm_frac": by / (us * 1e-6) / 1e9 / peak, "flops_per_launch": fl, "bytes_per_launch": by,
                    "peak_source": bf16[1]}
    # the same step as one CUDA graph launch (two-sided factors): recorded on
    # one set of the cycled inputs, replayed K times with those inputs (the
    # work does not depend on the values; replays are checked bit for bit
    # against the plain calls by the GPU tests)
    graph = None
    if source_points and mode == "lowrank":
        r, J = cyc[0]
        rp.rp_graph_capture(lib.ctx, r, J, lib.phi, lib.A)
        rp.rp_graph_step(lib.ctx)
        torch.cuda.synchronize()
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        for i in range(K):
            rp.rp_graph_step(lib.ctx)
        g1.record(stream)
        torch.cuda.synchronize()
        gms = g0.elapsed_time(g1) / K
        graph = {"ms_per_step": gms, "value": w.points / (gms / 1e3), "unit": UNIT, "steps": K,
                 "host_launches_per_step": 1,
                 "note": "one graph launch per step: every push, FFT, MAC, far-path and interpolation kernel of the "
                         "step; inputs fixed between replays"}
    q = lib.query()
    lib.close()
    # two-sided factors: the same steps with overlapped pushes (each push on the
    # library's push stream beside the previous evaluation; the same bits as
    # the sequential context above, which keeps the accuracy check, the kernel
    # pass and the graph replay, which refuses overlapped contexts)
    sequential = None
    if source_points and mode == "lowrank":
        sequential = {"ms_per_step": ms / K, "value": w.points * K / (ms / 1e3), "unit": UNIT,
                      "note": "rp_push_all + rp_evaluate on a context without RP_FLAG_OVERLAP_PUSH"}
        with rp.RetardedPotentials(w.domains, w.c, w.dt, mode=rp.RP_MODE_LOWRANK,
                                   flags=flags | rp.RP_FLAG_OVERLAP_PUSH, device=local, stream=stream,
                                   far_distance=fd, far_batch=args.far_batch, far_source_points=source_points) as lo:
            for j in range(pre + W):
                r, J = gen.step(j - pre, w.dt)
                lo.push_all(r, J)
                if j >= pre:
                    lo.evaluate()
            lo.sync()
            ophi, oA = rp.pointer_array(lo.phi), rp.pointer_array(lo.A)
            torch.cuda.synchronize()
            o0, o1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            o0.record(stream)
            for i in range(K):
                r, J = pcyc[i % ncycle]
                rp.rp_push_all_event(lo.ctx, r, J)
                rp.rp_evaluate(lo.ctx, ophi, oA)
            o1.record(stream)
            torch.cuda.synchronize()
            ms = o0.elapsed_time(o1)
    plain_line = None
    if plain:
        costs = calibrate_fft_costs(w, local, stream)
        rate = calibrate_direct_rate(local, stream) if any(
            abs(a.h - b.h) > 1e-12 * a.h for a in w.domains for b in w.domains) else 1.0
        plain_line = plain_path_extrapolated(w, info, costs, rate)
        plain_line["speedup_of_chosen"] = plain_line["ms_per_step"] / (ms / K)
    return {"workload": name, "description": w.description, "points_per_step": w.points,
            "value": w.points * K / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / K, "steps": K, "warmup": W,
            "path": f"FFT self terms; far pairs {mode}" + (f", two-sided factors ({source_points}^3 source nodes), "
                                                          f"overlapped pushes"
                                                          if source_points and mode == "lowrank" else ""),
            "sequential_push": sequential,
            "far_pairs": q["npairs_far"], "learned_pairs": q["npairs_learned"], "far_bytes": q["far_bytes"],
            "device_bytes": q["device_bytes"], "training": train, "accuracy": acc, "roofline": roof,
            "far_gemm_roofline": far_roof, "kernels": kstats, "gpu_launches": launches, "plain_path": plain_line,
            "graph_replay": graph, "setup_s": setup_s}


def far_alone_check(args, w, mode, source_points, fd, tgts, local, stream, lib):
    """The far field alone: domain 0 the only source, its field on targets
    `tgts` against the FP64 oracle (sampled nodes, two steps).  Low-rank
    pairs are per pair, so the check runs each pair (target, 0) in a context
    of those two domains; learned pairs depend on the network the full
    context trained, so that context's run is repeated with the other
    sources zero."""
    import torch
    import oracle
    from paper_2311_15429_gb300 import rp
    dev = torch.device("cuda", local)
    gen = synth.DeviceSlices(w.sources[:1], dev)
    rng = np.random.default_rng(21)
    worst, steps = 0.0, None

    def score(t, dom_t, got, step, lag_lo, lag_hi):
        lo, hi = step - lag_hi - 1, step - lag_lo
        src = w.sources[0].history(lo, hi + 1, w.dt)
        tgt = np.zeros((16, 4, dom_t.N), dtype=np.float32)
        nodes = rng.integers(0, dom_t.N, 48)
        doms = [dom_t, w.domains[0]]
        vals, _ = oracle.eval_points_windows_parallel([d.origin for d in doms], [d.n for d in doms],
                                                      [d.h for d in doms], [tgt, src], [step - 15, lo], w.c, w.dt,
                                                      0, step, nodes)
        return max(float(np.linalg.norm(got[f, nodes] - vals[:, f]) / np.linalg.norm(vals[:, f])) for f in range(4))

    if mode == "lowrank":
        for t in tgts:
            doms = [w.domains[0], w.domains[t]]
            z = (torch.zeros(w.domains[t].N, device=dev), torch.zeros(3 * w.domains[t].N, device=dev))
            with rp.RetardedPotentials(doms, w.c, w.dt, mode=rp.RP_MODE_LOWRANK, device=local, stream=stream,
                                       far_distance=fd, far_batch=args.far_batch,
                                       far_source_points=source_points) as sub:
                p = sub.pair_info(1, 0)
                assert p["kind"] == rp.RP_PAIR_LOWRANK
                L = sub.query()["max_lag"] + 20
                steps = (L - 14, L - 1)
                for j in range(L):
                    r, J = gen.step(j, w.dt)
                    sub.push_all([r[0], z[0]], [J[0], z[1]])
                    if j in steps:
                        sub.evaluate()
                        got = torch.cat([sub.phi[1][None], sub.A[1].reshape(3, -1)]).cpu().numpy()
                        worst = max(worst, score(t, w.domains[t], got, j, p["lag_lo"], p["lag_hi"]))
        how = "each pair (target, 0) in a context of its two domains (the same factors)"
    else:
        nd = len(w.domains)
        zr = [torch.zeros(d.N, device=dev) for d in w.domains]
        zJ = [torch.zeros(3 * d.N, device=dev) for d in w.domains]
        info = {t: lib.pair_info(t, 0) for t in tgts}
        with rp.RetardedPotentials(w.domains, w.c, w.dt, mode=rp.RP_MODE_LOWRANK, flags=rp.RP_FLAG_DEFER_FAR,
                                   device=local, stream=stream, far_distance=fd, far_batch=args.far_batch,
                                   far_source_points=source_points) as full:
            full.train_far_model(args.learned_distance)
            L = full.query()["max_lag"] + 20
            steps = (L - 14, L - 1)
            for j in range(L):
                r, J = gen.step(j, w.dt)
                full.push_all([r[0]] + zr[1:], [J[0]] + zJ[1:])
                if j in steps:
                    full.evaluate()
                    for t in tgts:
                        got = torch.cat([full.phi[t][None], full.A[t].reshape(3, -1)]).cpu().numpy()
                        worst = max(worst, score(t, w.domains[t], got, j, info[t]["lag_lo"], info[t]["lag_hi"]))
        how = "the full context (same training seed) with only domain 0's source"
    return {"rel_l2_max": worst, "targets": list(tgts), "source": 0, "steps_from_end": [13, 0],
            "checked": f"48 seeded nodes per target per step against the FP64 oracle; {how}"}


def bf16_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(p))
        return float(d["bf16_tflops"]), "measured bf16_tflops (cuBLAS burst)"
    except Exception:
        return 1900.0, "fallback"


def run_deep(args, rank, world, local):
    """cfg3 / cfg4 / cfg5 on their own line: every cross pair is far."""
    import torch
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    mode = "lowrank" if args.mode == "fft" else args.mode
    clocks = ClockSampler(local)
    barrier(world)
    clocks.start()
    leg = deep_leg(args, args.workload, args.steps, args.warmup, local, stream, mode=mode,
                   source_points=args.source_points, check=not args.no_cpu, plain=not args.no_plain)
    clk = clocks.stop()
    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": world * leg["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": leg["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": leg["workload"], "description": leg["description"],
                   "points_per_step": leg["points_per_step"], "path": leg["path"], "far_pairs": leg["far_pairs"],
                   "learned_pairs": leg["learned_pairs"], "far_bytes": leg["far_bytes"],
                   "l2": "16 device-made input slices per domain cycled",
                   "parallelism": f"{world} independent replicas" if world > 1 else "1 GPU"},
        "training": leg["training"], "accuracy": leg["accuracy"], "roofline": leg["roofline"],
        "far_gemm_roofline": leg["far_gemm_roofline"], "kernels": leg["kernels"], "gpu_launches": leg["gpu_launches"],
        "plain_path": leg["plain_path"], "graph_replay": leg["graph_replay"], "clocks": clk, "e2e": None,
        "cpu_baseline": None,
    }
    print(json.dumps(line), flush=True)


def run_partitioned(args, rank, world, local):
    """The source partition across ranks (Sec. IV: one process per domain):
    rank r owns the source domains partition.owners gives it; a step is its
    pushes, its rp_evaluate (every target's share from its sources) and one
    reduce-scatter of the packed shares, after which each rank holds the
    totals of its own targets.  The work of the whole workload is fixed as
    ranks are added (strong scaling)."""
    import torch
    import torch.distributed as dist
    from paper_2311_15429_gb300 import partition, rp
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    w = get_workload(args.workload)
    lag = lag_window(w)
    W, K = args.warmup, args.steps
    nd = len(w.domains)
    sizes = [d.N for d in w.domains]
    own = partition.owners(sizes, world)
    mine = partition.owned_by(rank, own)
    ncycle = 16
    pre = lag + 1
    depth = max(w.history, lag + 1)
    gen = synth.DeviceSlices(w.sources, dev)
    cyc = [gen.step(j - pre, w.dt) for j in range(pre + ncycle)]
    ptr = lambda xs: rp.pointer_array([x if d in mine else 0 for d, x in enumerate(xs)])
    pins = [(ptr(r), ptr(J)) for r, J in cyc]
    if not mine:   # more ranks than domains: this rank only joins the exchange
        lib = None
    else:
        lib = rp.RetardedPotentials(w.domains, w.c, w.dt, history_depth=depth, device=local, stream=stream,
                                    owned_sources=mine)
        pphi, pA = rp.pointer_array(lib.phi), rp.pointer_array(lib.A)
        for i in range(pre):
            rp.rp_push_all(lib.ctx, *pins[i])
    zeros = [torch.zeros(4 * n, device=dev) for n in sizes]

    def step(i):
        if lib is not None:
            rp.rp_push_all(lib.ctx, *pins[pre + i % ncycle])
            rp.rp_evaluate(lib.ctx, pphi, pA)
            fields = [torch.cat([lib.phi[d], lib.A[d]]) for d in range(nd)]
        else:
            fields = zeros
        return partition.exchange(partition.pack(fields, sizes, own, world), world)

    for i in range(W):
        step(i)
    torch.cuda.synchronize()
    barrier(world)
    clocks = ClockSampler(local)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(K):
        step(W + i)
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    barrier(world)
    ms = max_over_ranks(e0.elapsed_time(e1), world, dev)
    if lib is not None:
        lib.close()
    if rank != 0:
        return
    line = {"metric": METRIC, "value": w.points * K / (ms / 1e3), "unit": UNIT, "n_gpus": world, "steps": K,
            "warmup": W, "ms_per_step": ms / K, "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": w.name, "description": w.description, "points_per_step": w.points,
                       "parallelism": f"source partition over {world} GPUs (owners {own}), one NCCL reduce-scatter "
                                      f"of the packed per-target shares per step",
                       "exchange_bytes_per_rank_per_step": 4 * world * partition.chunk_floats(sizes, own, world)},
            "clocks": clk, "e2e": None, "cpu_baseline": None}
    print(json.dumps(line), flush=True)


SPLIT_SWEEP = [(8, 32, 24), (8, 32, 48), (8, 32, 96), (8, 96, 24), (8, 96, 48), (8, 96, 96),
               (16, 96, 48), (16, 96, 96)]   # (W', L', d') in nodes, h = 0.25 bohr


def eq13_speedup(W, L, d):
    """Sec. III, Eq. 13: the paper's complexity ratio of one enclosing domain
    (W' d' L' nodes, N_R from its diagonal) to two W' x W' x L' sub-domains
    (cross pairs over Delta N_R = diagonal - (d' - 2W'), self terms over the
    sub-domain's diagonal), each lag costing N log N."""
    D = math.sqrt(d * d + L * L + W * W)
    sub = W * W * L * math.log(W * W * L)
    num = 2 * D * sub - 2 * (d - 2 * W) * sub + 2 * math.sqrt(2 * W * W + L * L) * sub
    den = D * W * d * L * math.log(W * d * L)
    return den / num


def run_split(args, rank, world, local):
    """Single enclosing domain against two sub-domains (Sec. III, Eq. 13):
    measured step times of both layouts on the FFT path, their ratio beside
    the paper's complexity ratio, both layouts checked against each other and
    against the FP64 oracle at seeded nodes."""
    import torch
    import oracle
    from paper_2311_15429_gb300 import rp
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    h, c, dt = 0.25, synth.C_AU, 0.01
    K, W = args.steps, max(args.warmup, 3)
    rows = []
    rng = np.random.default_rng(5)
    for (Wn, Ln, dn) in SPLIT_SWEEP:
        g = synth.split_geometry(Wn, Ln, dn, h)
        layouts = {"multi": g.subs, "single": [g.enclosing]}
        libs = {k: rp.RetardedPotentials(v, c, dt, device=local, stream=stream) for k, v in layouts.items()}
        lags = {k: lib.query()["max_lag"] for k, lib in libs.items()}
        T = max(lags.values()) + 1 + W
        hist = [s.history(0, T, dt) for s in g.sources]
        dev_in = {"multi": [torch.from_numpy(x).to(dev) for x in hist],
                  "single": [torch.from_numpy(g.embed(hist)).to(dev)]}
        out = {}
        for k, lib in libs.items():
            xs = dev_in[k]
            for i in range(T):
                lib.push_all([x[i, 0] for x in xs], [x[i, 1:].reshape(-1) for x in xs])
                if i >= T - W:
                    lib.evaluate()
            lib.sync()
            out[k] = [torch.cat([lib.phi[d][None], lib.A[d].reshape(3, -1)]).cpu().numpy()
                      for d in range(len(layouts[k]))]
        # agreement at the sub-domains' nodes, and the FP64 oracle at seeded nodes
        agree, err_multi, err_single = 0.0, 0.0, 0.0
        for k in range(2):
            a, b = out["single"][0][:, g.sub_nodes(k)], out["multi"][k]
            agree = max(agree, max(float(np.linalg.norm(a[f] - b[f]) / np.linalg.norm(b[f])) for f in range(4)))
            nodes = np.sort(rng.choice(g.subs[k].N, 32, replace=False))
            want = oracle.eval_points([x.origin for x in g.subs], [x.n for x in g.subs], [x.h for x in g.subs],
                                      hist, 0, c, dt, k, T - 1, nodes)
            for got, acc in ((b[:, nodes], "m"), (a[:, nodes], "s")):
                e = max(float(np.linalg.norm(got[f] - want[:, f]) / np.linalg.norm(want[:, f])) for f in range(4))
                if acc == "m":
                    err_multi = max(err_multi, e)
                else:
                    err_single = max(err_single, e)
        # timed: K steps each, cycled device inputs (the last W slices)
        ms = {}
        for k, lib in libs.items():
            xs = dev_in[k]
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for i in range(K):
                j = T - W + i % W
                lib.push_all([x[j, 0] for x in xs], [x[j, 1:].reshape(-1) for x in xs])
                lib.evaluate()
            e1.record(stream)
            torch.cuda.synchronize()
            ms[k] = e0.elapsed_time(e1) / K
        fft = {k: [tuple(lib.pair_info(t, s)["fft_m"]) for t in range(len(layouts[k])) for s in range(len(layouts[k]))]
               for k, lib in libs.items()}
        # this implementation's per-step MAC bytes: per (pair, lag) the kernel
        # spectrum (real for a self pair) and four field spectra, plus T2
        mac = {}
        for k, lib in libs.items():
            n = len(layouts[k])
            tot = 0
            for t in range(n):
                for s_ in range(n):
                    p = lib.pair_info(t, s_)
                    m = p["fft_m"]
                    cells = (m[0] // 2 + 1) * m[1] * m[2]
                    tot += (p["lag_hi"] - p["lag_lo"] + 1) * cells * ((4 if s_ == t else 8) + 4 * 8)
                tm = lib.pair_info(t, t)["fft_m"]
                tot += 4 * (tm[0] // 2 + 1) * tm[1] * layouts[k][t].n[2] * 8
            mac[k] = tot
        for lib in libs.values():
            lib.close()
        rows.append({"W": Wn, "L": Ln, "d": dn, "points_multi": 2 * g.subs[0].N, "points_single": g.enclosing.N,
                     "max_lag_multi": lags["multi"], "max_lag_single": lags["single"],
                     "fft_m_multi": fft["multi"][0], "fft_m_single": fft["single"][0],
                     "ms_multi": ms["multi"], "ms_single": ms["single"],
                     "speedup_measured": ms["single"] / ms["multi"], "speedup_eq13": eq13_speedup(Wn, Ln, dn),
                     "mac_bytes_multi": mac["multi"], "mac_bytes_single": mac["single"],
                     "speedup_mac_bytes": mac["single"] / mac["multi"],
                     "rel_l2_single_vs_multi": agree, "rel_l2_multi_vs_oracle": err_multi,
                     "rel_l2_single_vs_oracle": err_single})
    if rank != 0:
        return
    line = {"metric": "single-domain / two-sub-domain step time (Sec. III speedup, Eq. 13)", "unit": "ratio",
            "n_gpus": world, "steps": K, "warmup": W, "higher_is_better": True, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "split", "h": h, "dt": dt,
                       "description": "two W' x W' x L' sub-domains with outer faces d' nodes apart on x, against "
                                      "the d' x W' x L' domain enclosing them (zero sources in the gap); FFT path, "
                                      "device-resident inputs, CUDA events; oracle: 32 seeded nodes per sub-domain"},
            "rows": rows}
    print(json.dumps(line), flush=True)


def run_spill(args, rank, world, local):
    """History spill to host memory (Sec. IV, RP_FLAG_HISTORY_SPILL) on the
    2 x 48^3 workload: step time of the unspilled and the spilled context,
    device and pinned host bytes of each, bytes each step moves over the
    host link, and the two contexts' outputs compared bit for bit."""
    import torch
    from paper_2311_15429_gb300 import rp
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    w = get_workload("cfg2")
    K, W = args.steps, max(args.warmup, 3)
    src = synth.DeviceSlices(w.sources, dev)
    ncycle = 16
    slices = [src.step(j, w.dt) for j in range(ncycle)]
    flags = {"device": rp.RP_FLAG_GROUND_STATE_CLAMP,
             "spill": rp.RP_FLAG_GROUND_STATE_CLAMP | rp.RP_FLAG_HISTORY_SPILL}
    res, outs = {}, {}
    for name, fl in flags.items():
        with rp.RetardedPotentials(w.domains, w.c, w.dt, history_depth=w.history, flags=fl, device=local,
                                   stream=stream) as lib:
            q = lib.query()
            fill = q["max_lag"] + 2 * W   # past the deepest lag: every window in its steady state
            for i in range(fill):
                lib.push_all(*slices[i % ncycle])
                lib.evaluate()
            lib.sync()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for i in range(K):
                lib.push_all(*slices[(fill + i) % ncycle])
                lib.evaluate()
            lib.sync()   # the spill streams' last copies included
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / K
            outs[name] = [torch.cat([lib.phi[d], lib.A[d]]).clone() for d in range(len(w.domains))]
            # per step: each spilled source's slice to the host, each window's slice back
            link = (len(w.domains) + q["spill_windows"]) * 16 * w.domains[0].N if q["spill_windows"] else 0
            res[name] = {"ms_per_step": ms, "device_bytes": q["device_bytes"], "spectral_bytes": q["spectral_bytes"],
                         "host_bytes": q["host_bytes"], "spill_windows": q["spill_windows"],
                         "spectral_depth_device": q["spectral_depth"], "host_link_bytes_per_step": link,
                         "host_link_GBps": link / (ms * 1e-3) / 1e9 if link else 0.0}
    same = all(torch.equal(a, b) for a, b in zip(outs["device"], outs["spill"]))
    if rank != 0:
        return
    line = {"metric": "step time with the spectral history in host memory (Sec. IV history store)", "unit": "ms",
            "value": res["spill"]["ms_per_step"], "n_gpus": world, "steps": K, "warmup": W,
            "higher_is_better": False, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "cfg2-spill", "description": w.description + "; clamped history, every step "
                       "evaluated; the spilled context keeps the 290-294-step cross windows in 5-slot spectral "
                       "rings, fed one (rho, J) slice a step from a pinned host ring through the forward "
                       "passes", "ncycle_inputs": ncycle},
            "device": res["device"], "spill": res["spill"], "bit_identical": bool(same),
            "device_bytes_saved": res["device"]["device_bytes"] - res["spill"]["device_bytes"]}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank, world, local = dist_init(args)
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.workload == "split":
        run_split(args, rank, world, local)
    elif args.workload == "spill":
        run_spill(args, rank, world, local)
    elif args.partition == "sources" and world > 1:
        run_partitioned(args, rank, world, local)
    elif args.workload in DEEP:
        run_deep(args, rank, world, local)
    else:
        run_ours(args, rank, world, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
