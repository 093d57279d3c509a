"""Pins for the FP64 oracle: closed forms, limits and brute-force forms.

None of these compares the oracle with a retyped copy of its own loop.  Each
check comes from somewhere else -- a closed-form potential, a known lattice
constant, the retarded phase of a monopole, the Lorenz gauge condition, or
the paper's own Delta-S / Green's-function form of the sum (Eq. 12) -- and is
chosen so that a plausible slip in the oracle (a dropped self term, a wrong
power of h, an advanced instead of retarded delay, the two interpolation
weights swapped, a missing 1/c, a mixed-up current component) fails one.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy import integrate
from scipy.special import erf

import oracle
from paper_2311_15429_gb300 import synth

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "constants.json")))
INF = float("inf")


def _geom(doms):
    return (np.array([d.origin for d in doms]), np.array([d.n for d in doms]),
            np.array([d.h for d in doms]))


def _node_of(dom, i, j, k):
    return i + dom.n[0] * (j + dom.n[1] * k)


# ---------------------------------------------------------------- constants

def test_cube_average_constant():
    """C of the self cell equals the cube integral of 1/|u|, by quadrature."""
    f = lambda z, y, x: 1.0 / math.sqrt(x * x + y * y + z * z)
    octant, _ = integrate.tplquad(f, 0, 0.5, 0, 0.5, 0, 0.5, epsabs=1e-12, epsrel=1e-12)
    assert abs(8 * octant - oracle.cube_average_constant()) < 1e-9
    assert abs(GOLDEN["cube_average_C"]["value"] - oracle.cube_average_constant()) < 1e-12


# ---------------------------------------------------------------- static limit (c -> inf)

def test_static_limit_matches_gaussian_potential():
    """c -> inf: only lag 0 survives (Eq. 2 with R/c -> 0), and the grid sum of a
    well-resolved unit Gaussian seen from outside it is erf(R/(sqrt2 sigma))/R."""
    sigma, h = 0.4, 0.2
    src = synth.cubic((0.0, 0.0, 0.0), 25, h)
    centre = np.array([0.013, -0.021, 0.007])          # off-node centre
    g = synth.BreathingGaussian(src, centre, sigma, eps=0.0, omega=0.0)
    hist_src = g.history(0, 1, 0.05)
    # target: a 2x2x2 grid outside the source box, 3..5 bohr from the centre
    tgt = synth.Domain((3.1, 0.4, -0.9), (2, 2, 2), 0.7)
    hist_tgt = np.zeros((1, 4, tgt.N))
    origins, ns, hs = _geom([src, tgt])
    out = oracle.eval_points(origins, ns, hs, [hist_src, hist_tgt], 0, INF, 0.05,
                             target=1, step=0, nodes=np.arange(tgt.N))
    x, y, z = tgt.coords()
    R = np.sqrt((x - centre[0]) ** 2 + (y - centre[1]) ** 2 + (z - centre[2]) ** 2)
    exact = erf(R / (math.sqrt(2.0) * sigma)) / R
    np.testing.assert_allclose(out[:, 0], exact, rtol=2e-8)
    assert np.all(out[:, 1:] == 0.0)          # A = (1/c) * ... vanishes as c -> inf


def test_self_cell_error_constant():
    """Self domain, c -> inf, target at the Gaussian's centre node.

    The lattice sum over k' != k of h^3 f/R misses int f/R by
    zeta*h^2*f(0) + O(h^4), zeta the simple-cubic lattice constant; the
    cell-averaged self weight adds C*h^2*f(0).  So the oracle's error is
    (C + zeta) h^2 rho(0): it pins both the h^2 scaling of the self weight and
    the value of C (a dropped self term would give zeta*h^2*rho(0))."""
    sigma = 1.0
    zeta = GOLDEN["sc_lattice_zeta"]["value"]
    C = GOLDEN["cube_average_C"]["value"]
    rho0 = (2 * math.pi * sigma ** 2) ** -1.5
    exact = math.sqrt(2.0 / math.pi) / sigma
    errs = {}
    for h, n in ((0.2, 61), (0.1, 121)):
        dom = synth.cubic((0.0, 0.0, 0.0), n, h)
        g = synth.BreathingGaussian(dom, (0.0, 0.0, 0.0), sigma, eps=0.0, omega=0.0)
        hist = g.history(0, 1, 0.05)
        origins, ns, hs = _geom([dom])
        mid = n // 2
        out = oracle.eval_points(origins, ns, hs, [hist], 0, INF, 0.05, target=0, step=0,
                                 nodes=[_node_of(dom, mid, mid, mid)])
        errs[h] = out[0, 0] - exact
    coef = errs[0.1] / (0.1 ** 2 * rho0)
    assert abs(coef - (C + zeta)) < 0.01 * abs(C + zeta), coef
    assert 3.8 < errs[0.2] / errs[0.1] < 4.2


# ---------------------------------------------------------------- retardation

def test_breathing_monopole_retarded_phase():
    """A monopole breathing at omega seen 2000 bohr away: phi(t) =
    Q [1 + eps sin(omega (t - R/c))]/R.  The fitted phase must be -omega R/c
    (the retardation of Eq. 2), the amplitude eps Q/R within the hat
    interpolation bound (omega dt)^2/8 (Eq. 7)."""
    c, dt, omega, eps, sigma, h = synth.C_AU, 0.05, 0.5, 0.1, 0.35, 0.2
    src = synth.cubic((0.0, 0.0, 0.0), 20, h)
    centre = src.center
    g = synth.BreathingGaussian(src, centre, sigma, eps=eps, omega=omega)
    direction = np.array([0.48, -0.6, 0.64])
    direction /= np.linalg.norm(direction)
    Rd = 2000.0
    tgt = synth.Domain(tuple(centre + Rd * direction), (1, 1, 1), 1.0)
    lag = int(Rd / (c * dt)) + 2
    period = int(round(2 * math.pi / omega / dt))
    j0, steps = 0, np.arange(lag, lag + period)
    hist_src = g.history(j0, lag + period, dt, dtype=np.float64)
    hist_tgt = np.zeros((lag + period, 4, 1))
    origins, ns, hs = _geom([src, tgt])
    phi = np.array([oracle.eval_points(origins, ns, hs, [hist_src, hist_tgt], j0, c, dt,
                                       target=1, step=int(l), nodes=[0])[0, 0] for l in steps])
    t = steps * dt
    M = np.stack([np.ones_like(t), np.sin(omega * t), np.cos(omega * t)], axis=1)
    a0, a1, a2 = np.linalg.lstsq(M, phi, rcond=None)[0]
    amp, phase = math.hypot(a1, a2), math.atan2(a2, a1)
    want_phase = -omega * Rd / c
    dphase = (phase - want_phase + math.pi) % (2 * math.pi) - math.pi
    assert abs(dphase) < 1e-4, dphase
    assert abs(a0 * Rd - 1.0) < 1e-6
    assert abs(amp * Rd / eps - 1.0) < (omega * dt) ** 2 / 8 + 1e-6


def _gauge_residual(dt):
    """|div A + (1/c) dphi/dt| / |(1/c) dphi/dt| at one point, for a moving Gaussian."""
    c = 5.0                                  # slow light: ~24-step delays
    sigma, amp, omega, h = 0.5, 0.3, 1.0, 0.2
    src = synth.cubic((0.0, 0.0, 0.0), 39, h)
    mg = synth.MovingGaussian(src, (0.0, 0.0, 0.0), sigma, amp, omega, axis=(1.0, 0.3, -0.2))
    ht = 0.05
    centre = np.array([4.0, 3.0, 2.5])
    tgt = synth.Domain(tuple(centre - 2 * ht), (5, 5, 5), ht)
    tmid = 1.7                               # evaluation time
    l = int(round(tmid / dt))
    first = l - int(14.0 / (c * dt)) - 4    # farthest source node is ~12.3 bohr away
    hist_src = mg.history(first, l + 3, dt)
    hist_tgt = np.zeros((l + 3 - first, 4, tgt.N))
    origins, ns, hs = _geom([src, tgt])

    def ev(step, nodes):
        return oracle.eval_points(origins, ns, hs, [hist_src, hist_tgt], first, c, dt,
                                  target=1, step=step, nodes=nodes)

    mid = _node_of(tgt, 2, 2, 2)
    phis = [ev(l + s, [mid])[0, 0] for s in (-2, -1, 1, 2)]
    dphi = (phis[0] - 8 * phis[1] + 8 * phis[2] - phis[3]) / (12 * dt)
    div = 0.0
    for axis in range(3):
        idx = []
        for s in (-2, -1, 1, 2):
            p = [2, 2, 2]
            p[axis] += s
            idx.append(_node_of(tgt, *p))
        A = ev(l, idx)[:, 1 + axis]
        div += (A[0] - 8 * A[1] + 8 * A[2] - A[3]) / (12 * ht)
    return abs(div + dphi / c) / abs(dphi / c)


def test_lorenz_gauge_condition():
    """div A + (1/c) dphi/dt = 0 (Appendix B, Eq. B3) for continuity-consistent
    sources.  Both terms are O(1) here and cancel to the hat-interpolation
    error of Eq. 7 (a few 1e-4): a sign or 1/c slip in A, a current component
    routed to the wrong output, or a lag that differs between phi and A leaves
    a residual of 1e-2 or more."""
    for dt in (0.05, 0.025):
        r = _gauge_residual(dt)
        assert r < 1e-3, (dt, r)


# ---------------------------------------------------------------- Eq. 12 brute force

def _hat(s):
    return np.maximum(0.0, 1.0 - np.abs(s))


def _eq12_brute_force(doms, hists, c, dt, target, l, C):
    """P(r_k, l dt) = sum_n [ P~_n(r_k, 0) + sum_k' sum_{l'=1..l} G_{l-l'}[k,k'] dS(k', l') ]
    with G_m[k,k'] = h^3 T(m dt - R/c)/R (Eq. 11), dS(l') = S(l') - S(0) (Eq. 9)
    and P~_n(0) the static potential of S(0) (Eq. 10).  Samples before t = 0
    are S(0), as Eq. 7 implies."""
    td = doms[target]
    xt, yt, zt = td.coords()
    out = np.zeros((td.N, 4))
    for n, dom in enumerate(doms):
        xs, ys, zs = dom.coords()
        R = np.sqrt((xt[:, None] - xs[None, :]) ** 2 + (yt[:, None] - ys[None, :]) ** 2
                    + (zt[:, None] - zs[None, :]) ** 2)
        self_pair = R == 0.0
        Rs = np.where(self_pair, 1.0, R)
        vol = dom.h ** 3
        # static part: instantaneous 1/R sum of S(0), cell average at R = 0
        W0 = np.where(self_pair, C * dom.h ** 2, vol / Rs)
        S0 = hists[n][0]
        out += W0 @ S0.T
        for lp in range(1, l + 1):
            m = l - lp
            Gm = np.where(self_pair, C * dom.h ** 2 * (1.0 if m == 0 else 0.0),
                          vol * _hat(m - R / (c * dt)) / Rs)
            dS = hists[n][lp] - S0
            out += Gm @ dS.T
    out[:, 1:] /= c
    return out


def test_eq12_delta_s_form_on_4cubed():
    """Brute force of Eq. 12 on two 4^3 grids with random histories equals the
    oracle (clamped history, S(t<0) = S(0)) to rounding."""
    rng = np.random.default_rng(7)
    doms = [synth.Domain((0.0, 0.0, 0.0), (4, 4, 4), 0.3),
            synth.Domain((1.6, 0.35, -0.2), (4, 4, 4), 0.3)]
    c, dt, L = 2.0, 0.1, 14           # delays up to ~13 steps
    hists = [rng.standard_normal((L, 4, 64)) for _ in doms]
    origins, ns, hs = _geom(doms)
    C = GOLDEN["cube_average_C"]["value"]
    for target in (0, 1):
        for l in (3, 13):
            want = _eq12_brute_force(doms, hists, c, dt, target, l, C)
            got = oracle.eval_points(origins, ns, hs, hists, 0, c, dt, target, l,
                                     np.arange(64), clamp=True)
            np.testing.assert_allclose(got, want, rtol=1e-11, atol=1e-11 * np.abs(want).max())


# ---------------------------------------------------------------- invariants

def _two_small():
    doms = [synth.Domain((0.0, 0.0, 0.0), (5, 4, 3), 0.25),
            synth.Domain((2.3, -0.4, 0.9), (3, 5, 4), 0.25)]
    return doms


def test_reciprocity_equal_spacing():
    """G_m[k,k'] = G_m[k',k] (Eq. 11 depends on |r_k - r_k'| only): an impulse
    at k' seen at k equals an impulse at k seen at k'."""
    doms = _two_small()
    c, dt, L = 3.0, 0.05, 30
    origins, ns, hs = _geom(doms)
    rng = np.random.default_rng(3)
    for _ in range(5):
        ka, kb = int(rng.integers(doms[0].N)), int(rng.integers(doms[1].N))
        j = 4
        h0 = np.zeros((L, 4, doms[0].N)); h1 = np.zeros((L, 4, doms[1].N))
        h1[j, 0, kb] = 1.0
        ab = oracle.eval_points(origins, ns, hs, [h0, h1], 0, c, dt, 0, L - 1, [ka])[0, 0]
        h1[:] = 0.0; h0[j, 0, ka] = 1.0
        ba = oracle.eval_points(origins, ns, hs, [h0, h1], 0, c, dt, 1, L - 1, [kb])[0, 0]
        assert ab == pytest.approx(ba, rel=1e-13, abs=1e-300)


def test_linearity_and_time_shift():
    doms = _two_small()
    c, dt, L = 3.0, 0.05, 40
    origins, ns, hs = _geom(doms)
    rng = np.random.default_rng(5)
    A = [rng.standard_normal((L, 4, d.N)) for d in doms]
    B = [rng.standard_normal((L, 4, d.N)) for d in doms]
    nodes = np.arange(doms[1].N)
    ea = oracle.eval_points(origins, ns, hs, A, 0, c, dt, 1, L - 1, nodes)
    eb = oracle.eval_points(origins, ns, hs, B, 0, c, dt, 1, L - 1, nodes)
    eab = oracle.eval_points(origins, ns, hs, [2.0 * a - 0.5 * b for a, b in zip(A, B)], 0, c,
                             dt, 1, L - 1, nodes)
    np.testing.assert_allclose(eab, 2.0 * ea - 0.5 * eb, rtol=1e-12, atol=1e-12)
    # the same history stored from time index 100 on and evaluated 100 steps later
    shifted = oracle.eval_points(origins, ns, hs, A, 100, c, dt, 1, L - 1 + 100, nodes)
    np.testing.assert_array_equal(shifted, ea)


def test_constant_source_equals_static_limit():
    """Sum_m T(m - tau) = 1 (partition of unity of the hats in Eq. 7): a
    time-constant source gives exactly the instantaneous (c -> inf) potential."""
    doms = _two_small()
    origins, ns, hs = _geom(doms)
    rng = np.random.default_rng(9)
    S = [rng.standard_normal((1, 4, d.N)) for d in doms]
    L = 120                           # delays up to ~80 steps at c = 0.9
    hist = [np.repeat(s, L, axis=0) for s in S]
    nodes = np.arange(doms[0].N)
    ret = oracle.eval_points(origins, ns, hs, hist, 0, 0.9, 0.05, 0, L - 1, nodes)
    sta = oracle.eval_points(origins, ns, hs, S, 0, INF, 0.05, 0, 0, nodes)
    np.testing.assert_allclose(ret[:, 0], sta[:, 0], rtol=1e-13, atol=1e-13)


def test_history_window_and_clamp():
    doms = _two_small()
    origins, ns, hs = _geom(doms)
    rng = np.random.default_rng(11)
    c, dt = 3.0, 0.05                 # delays up to ~20 steps
    L = 8
    hist = [rng.standard_normal((L, 4, d.N)) for d in doms]
    with pytest.raises(oracle.OracleError) as e:
        oracle.eval_points(origins, ns, hs, hist, 0, c, dt, 0, L - 1, [0])
    assert e.value.code == oracle.ERR_HISTORY
    # clamped == history explicitly extended backwards with the first sample
    got = oracle.eval_points(origins, ns, hs, hist, 0, c, dt, 0, L - 1, np.arange(10),
                             clamp=True)
    pad = 40
    ext = [np.concatenate([np.repeat(h[:1], pad, axis=0), h]) for h in hist]
    want = oracle.eval_points(origins, ns, hs, ext, -pad, c, dt, 0, L - 1, np.arange(10))
    np.testing.assert_array_equal(got, want)
    # a step beyond the stored samples is refused
    with pytest.raises(oracle.OracleError):
        oracle.eval_points(origins, ns, hs, hist, 0, c, dt, 0, L, [0], clamp=True)


def test_coincident_nodes_rejected():
    doms = [synth.Domain((0.0, 0.0, 0.0), (2, 2, 2), 0.5),
            synth.Domain((0.5, 0.5, 0.5), (2, 2, 2), 0.5)]
    origins, ns, hs = _geom(doms)
    hist = [np.ones((1, 4, 8)) for _ in doms]
    with pytest.raises(oracle.OracleError) as e:
        oracle.eval_points(origins, ns, hs, hist, 0, INF, 0.05, 0, 0, [7])
    assert e.value.code == oracle.ERR_COINCIDENT


def test_per_domain_windows_match_one_window():
    """Per-domain stored windows hold the same samples as one common window,
    so the sums agree exactly; a sample outside a domain's window is an error."""
    import oracle
    rng = np.random.default_rng(11)
    origins = [np.zeros(3), np.array([30.0, 2.0, -1.0])]
    ns, hs = [(4, 3, 3), (3, 3, 2)], [0.4, 0.5]
    c, dt, T, step = 137.036, 0.05, 40, 39
    hists = [rng.standard_normal((T, 4, 36)), rng.standard_normal((T, 4, 18))]
    nodes = np.arange(18)
    a = oracle.eval_points(origins, ns, hs, hists, 0, c, dt, 1, step, nodes)
    w = [hists[0][25:], hists[1][36:]]
    b = oracle.eval_points_windows(origins, ns, hs, w, [25, 36], c, dt, 1, step, nodes)
    assert np.array_equal(a, b)
    with pytest.raises(oracle.OracleError):
        oracle.eval_points_windows(origins, ns, hs, [hists[0][36:], hists[1][36:]], [36, 36], c, dt, 1, step, nodes)
