"""Helpers shared by the GPU tests: drive the library through the C-ABI on
seeded synthetic histories and score it against the FP64 oracle."""
import numpy as np

import oracle
from paper_2311_15429_gb300 import rp


def histories(sources, j0, j1, dt):
    """Float32 samples [T][4][N] of each source for time indices j0..j1-1."""
    return [s.history(j0, j1, dt) for s in sources]


def run_library(domains, c, dt, hists, j0, eval_at, mode=rp.RP_MODE_FFT, flags=0, depth=0,
                push="all", mac_warps=0):
    """Push every sample of ``hists`` (time index j0 + i) and evaluate at the
    time indices in ``eval_at``.  Returns {time index: [domain][4][N] float32}."""
    if mac_warps:                   # the warp-count variants are those of the plain FP32 sum
        flags |= rp.RP_FLAG_PLAIN_SUM
    import torch
    dev = torch.device("cuda", 0)
    T = hists[0].shape[0]
    eval_at = set(eval_at)
    out = {}
    with rp.RetardedPotentials(domains, c, dt, history_depth=depth, mode=mode, flags=flags,
                               mac_warps=mac_warps) as lib:
        for i in range(T):
            j = j0 + i
            slices = [torch.from_numpy(np.ascontiguousarray(h[i])).to(dev) for h in hists]
            rhos = [s[0].contiguous() for s in slices]
            Js = [s[1:].contiguous().reshape(-1) for s in slices]
            if push == "all":
                lib.push_all(rhos, Js)
            elif push == "each":
                for d in reversed(range(len(domains))):
                    lib.push(d, rhos[d], Js[d])
            else:
                raise ValueError(push)
            if j in eval_at:
                phi, A = lib.evaluate()
                torch.cuda.synchronize()
                out[j] = [np.concatenate([phi[d].cpu().numpy()[None], A[d].cpu().numpy().reshape(3, -1)])
                          for d in range(len(domains))]
        lib.sync()
    return out


def oracle_values(domains, hists, j0, c, dt, target, step, nodes, clamp=False):
    args = ([d.origin for d in domains], [d.n for d in domains], [d.h for d in domains], hists, j0,
            c, dt, target, step, nodes)
    if len(nodes) * sum(d.N for d in domains) > 2e7:      # large checks: all host cores
        return oracle.eval_points_parallel(*args, clamp=clamp)[0]
    return oracle.eval_points(*args, clamp=clamp)


def rel_l2(got, want):
    """Per-field rel-L2 of got [4][n] against want [n][4]."""
    return [float(np.linalg.norm(got[f] - want[:, f]) / np.linalg.norm(want[:, f])) for f in range(4)]
