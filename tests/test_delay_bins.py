"""Why every lag is its own delay bin (the exact Eq. 11 form).

A bin of W > 1 lags would apply the bin's summed hat weights to the source
sample at the bin's centre delay: one kernel spectrum (or two) per bin
instead of one per lag.  On the 2 x 48^3 workload's cross pair (lags
290-294) this is computed here in FP64 at seeded target nodes, exactly and
binned.  The current, and so A, is all time dependence (J ~ dA/dt of the
breathing sources), so shifting its delay by up to W/2 steps costs about
omega dt W / 2 of it: the error is already percents of the cross field, and
above 1e-3 of the total potential, at W = 2.  An error-budgeted choice of
widths therefore keeps W = 1 for any budget of the FP32 (1e-6) or bf16 /
learned (1e-3) bars.
"""
import numpy as np

import oracle
from paper_2311_15429_gb300 import synth


def _binned_errors(widths, n_nodes=12):
    w = synth.workload("cfg2")
    t, s, step = 0, 1, 300
    hist = [src.history(0, step + 1, w.dt) for src in w.sources]

    def coords(d):
        i = np.arange(d.N)
        n = d.n
        return np.stack([d.origin[0] + d.h * (i % n[0]), d.origin[1] + d.h * ((i // n[0]) % n[1]),
                         d.origin[2] + d.h * (i // (n[0] * n[1]))], 1)

    xt, ys = coords(w.domains[t]), coords(w.domains[s])
    nodes = np.random.default_rng(0).choice(w.domains[t].N, n_nodes, replace=False)
    total = oracle.eval_points([d.origin for d in w.domains], [d.n for d in w.domains], [d.h for d in w.domains],
                               hist, 0, w.c, w.dt, t, step, nodes)
    S = hist[s].astype(np.float64)
    cols = np.arange(w.domains[s].N)
    vol, cdt, lo = w.domains[s].h ** 3, w.c * w.dt, 290

    def sample(delay):   # S(l - delay), linear between samples, per source node
        m = np.floor(delay).astype(int)
        f = delay - m
        return (1 - f)[None] * S[step - m, :, cols].T + f[None] * S[step - m - 1, :, cols].T

    out = {}
    for W in widths:
        err = np.zeros((n_nodes, 4))
        cross = np.zeros((n_nodes, 4))
        for a, k in enumerate(nodes):
            R = np.linalg.norm(ys - xt[k], axis=1)
            tau = R / cdt
            m = np.floor(tau).astype(int)
            f = tau - m
            exact = vol / R * sample(tau)
            centre = lambda lag: lo + W * ((lag - lo) // W) + (W - 1) / 2.0
            binned = vol / R * ((1 - f) * sample(centre(m)) + f * sample(centre(m + 1)))
            cross[a] = exact.sum(1)
            err[a] = (binned - exact).sum(1)
        out[W] = (max(np.linalg.norm(err[:, q]) / np.linalg.norm(cross[:, q]) for q in range(4)),
                  max(np.linalg.norm(err[:, q]) / np.linalg.norm(total[:, q]) for q in range(4)))
    return out


def test_one_lag_per_bin_is_exact_and_wider_bins_break_every_bar():
    e = _binned_errors([1, 2, 5])
    assert e[1] == (0.0, 0.0)                   # W = 1 is the Eq. 11 form itself
    for W in (2, 5):
        of_cross, of_total = e[W]
        assert of_cross > 1e-2 and of_total > 1e-3, (W, e[W])
