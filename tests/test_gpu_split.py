"""GPU: the single enclosing domain and the two-sub-domain path (Sec. III,
Eq. 13) through the C-ABI, against each other and the FP64 oracle.

Both run the FFT path (Hockney self term; for the two sub-domains also the
delay-binned cross pairs).  Non-cubic grids take the runtime-size kernels.
"""
import numpy as np
import pytest

import oracle
from paper_2311_15429_gb300 import rp, synth

from _harness import rel_l2, run_library

pytestmark = pytest.mark.gpu
TOL = 1e-6


@pytest.mark.parametrize("W,L,d", [(6, 24, 30), (8, 32, 48)])
def test_single_domain_matches_two_subdomains(W, L, d):
    g = synth.split_geometry(W, L, d, 0.25)
    c, dt, T = synth.C_AU, 0.01, 24
    hist = [s.history(0, T, dt) for s in g.sources]
    big = [g.embed(hist)]
    steps = range(T - 3, T)
    two = run_library(g.subs, c, dt, hist, 0, steps)
    one = run_library([g.enclosing], c, dt, big, 0, steps)
    rng = np.random.default_rng(7)
    for step in steps:
        for k in range(2):
            a = one[step][0][:, g.sub_nodes(k)]
            b = two[step][k]
            assert max(rel_l2(a, b.T.astype(np.float64))) <= TOL, (step, k)
    # both against the oracle at seeded nodes of each sub-domain, last step
    step = T - 1
    for k in range(2):
        nodes = np.sort(rng.choice(g.subs[k].N, 128, replace=False))
        want = oracle.eval_points([x.origin for x in g.subs], [x.n for x in g.subs], [x.h for x in g.subs],
                                  hist, 0, c, dt, k, step, nodes)
        assert max(rel_l2(two[step][k][:, nodes], want)) <= TOL
        assert max(rel_l2(one[step][0][:, g.sub_nodes(k)[nodes]], want)) <= TOL
