"""The learned far field's 16-sample delay window against the geometry of the
32 x 48^3 workload (cfg5).

The network reads, per pair, the source moments at the 16 times t - tau_c -
o (o = -7 .. 8 steps) around the centre-to-centre delay tau_c.  Every
retarded sample the pair's exact sum needs lies at a delay R / (c dt) with
|R - R_c| at most the two boxes' half diagonals (triangle inequality), and
the hat of Eq. 7 reads the two samples around it.  So the window holds every
sample a pair depends on when that spread plus one step stays inside it.
This checks it for all 992 ordered pairs (and that the bound is tight at the
box corners), the measurement behind keeping 16 samples rather than 64.
"""
import itertools

import numpy as np

from paper_2311_15429_gb300 import synth

WINDOW_OFFSETS = range(-7, 9)   # the 16 sample offsets the network reads


def _centre_and_half(d):
    half = d.h * (np.array(d.n) - 1) / 2.0
    return np.array(d.origin) + half, half


def test_cfg5_pairs_fit_the_16_sample_window():
    w = synth.workload("cfg5")
    cdt = w.c * w.dt
    worst_bound = worst_corner = 0.0
    npairs = 0
    for t, T in enumerate(w.domains):
        ct, ht = _centre_and_half(T)
        for s, S in enumerate(w.domains):
            if s == t:
                continue
            cs, hs = _centre_and_half(S)
            Rc = np.linalg.norm(ct - cs)
            assert Rc >= 500.0                 # every cfg5 pair is a far pair
            npairs += 1
            bound = (np.linalg.norm(ht) + np.linalg.norm(hs)) / cdt
            worst_bound = max(worst_bound, bound)
            for a in itertools.product((-1, 1), repeat=3):
                for b in itertools.product((-1, 1), repeat=3):
                    R = np.linalg.norm(ct + np.array(a) * ht - cs - np.array(b) * hs)
                    worst_corner = max(worst_corner, abs(R - Rc) / cdt)
    assert npairs == 992
    assert worst_corner <= worst_bound + 1e-9
    assert worst_bound > 0.9 * worst_corner   # the bound is nearly reached at the corners
    # the hat reads floor(tau) and floor(tau) + 1: one more step on each side
    reach = int(np.ceil(worst_bound)) + 1
    assert -reach >= min(WINDOW_OFFSETS) and reach <= max(WINDOW_OFFSETS), (worst_bound, reach)
    assert reach <= 4                          # 48^3 boxes at h = 0.25, c dt = 6.85 bohr: 2.97 steps + 1
