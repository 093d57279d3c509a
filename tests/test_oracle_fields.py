"""Pins of the field oracle (App. B: E = -grad phi - (1/c) dA/dt, B = curl A).

1. The difference stencils are exact on quadratics, in space (inside and on
   the faces) and in time, which a dropped term, a wrong sign or a swapped
   component would break.
2. Physics: the fields of the oracle's retarded potentials of an oscillating
   dipole match the oscillating-dipole field (Eq. 15's near, intermediate and
   far terms) on the dipole's broadside, from 90 to 7500 bohr, i.e. from the
   near zone into the radiation zone (c/omega = 1370 bohr).
"""
import math

import numpy as np
import pytest

import oracle
from oracle import fields as ofields
from paper_2311_15429_gb300 import synth


def test_stencils_exact_on_quadratics():
    n, h, c, dt = (5, 4, 6), 0.3, 137.036, 0.05
    dom = synth.Domain((0.1, -0.2, 0.3), n, h)
    x, y, z = dom.coords()
    phi = 1.5 * x * x - 0.7 * x * y + 2.0 * z * z + 0.3 * y - 4.0
    # A_a(r, t) quadratic in space and time at t = 2 dt, dt, 0
    def A(t):
        return np.stack([x * y + t * t * z, 0.5 * z * z - 3.0 * t * x, y * x * 0.25 + z * t + 2.0 * t * t])
    t = 2 * dt
    E, B = ofields.fields(phi, A(t), A(t - dt), A(t - 2 * dt), n, h, c, dt)
    gphi = np.stack([3.0 * x - 0.7 * y, -0.7 * x + 0.3, 4.0 * z])
    dAdt = np.stack([2.0 * t * z, -3.0 * x, z + 4.0 * t])
    np.testing.assert_allclose(E, -gphi - dAdt / c, rtol=1e-12, atol=1e-11)
    curl = np.stack([0.25 * x - z,                       # d_y Az - d_z Ay
                     t * t * 1.0 - 0.25 * y,             # d_z Ax - d_x Az
                     -3.0 * t - x])                      # d_x Ay - d_y Ax
    np.testing.assert_allclose(B, curl, rtol=1e-12, atol=1e-11)
    # first-order time difference without A_{l-2}: exact for A linear in t
    E1, _ = ofields.fields(phi, A(t), A(t - dt), None, n, h, c, dt)
    np.testing.assert_allclose(E1[1], -gphi[1] + 3.0 * x / c, rtol=1e-12, atol=1e-11)


def dipole_fields(p0, omega, d, t, c):
    """E_z and B_y on the broadside (d, 0, 0) of p(t) = p0 sin(omega t) z^
    at the origin: E_z = -[p/d^3 + p'/(c d^2) + p''/(c^2 d)],
    B_y = p'/(c d^2) + p''/(c^2 d), all at t - d/c (Eq. 15's three terms)."""
    tr = t - d / c
    p, pd, pdd = p0 * math.sin(omega * tr), p0 * omega * math.cos(omega * tr), -p0 * omega ** 2 * math.sin(omega * tr)
    return -(p / d ** 3 + pd / (c * d * d) + pdd / (c * c * d)), pd / (c * d * d) + pdd / (c * c * d)


def dipole_errors(d, dt):
    """Relative errors (to the amplitudes) of E_z and B_y from the oracle's
    potentials of an oscillating dipole against the closed form, at three
    times, plus the broadside E_x, E_y."""
    c, omega, Q, a, sigma, h = synth.C_AU, 0.1, 1.0, 0.2, 0.5, 0.25
    src = synth.cubic((0.0, 0.0, 0.0), 24, h)
    tgt = synth.cubic((d, 0.0, 0.0), 5, h)              # centre node (2, 2, 2) at (d, 0, 0)
    moving = synth.MovingGaussian(src, (0.0, 0.0, 0.0), sigma, a, omega, axis=(0.0, 0.0, 1.0), charge=Q)
    static = synth.BreathingGaussian(src, (0.0, 0.0, 0.0), sigma, 0.0, omega, charge=-Q)
    reach = 7.0                                          # half-diagonals of both boxes, bohr
    lag_lo = int(math.floor((d - reach) / (c * dt))) - 1
    lag_hi = int(math.ceil((d + reach) / (c * dt))) + 1
    k = 2 + 5 * (2 + 5 * 2)
    scaleE = Q * a * math.hypot(1 / d ** 3 - omega ** 2 / (c * c * d), omega / (c * d * d))
    scaleB = Q * a * math.hypot(-omega ** 2 / (c * c * d), omega / (c * d * d))
    eE, eB, side = [], [], []
    for t_end in (2.0, 4.85, 7.55):                      # three phases of the oscillation
        l = lag_hi + int(round(t_end / dt))
        first = l - 2 - lag_hi - 1                       # the source samples these three steps read
        hs = moving.history(first, l - lag_lo + 1, dt) + static.history(first, l - lag_lo + 1, dt)
        hz = np.zeros((12, 4, tgt.N))                    # the (source-free) target's own window
        pots = [oracle.eval_points_windows([src.origin, tgt.origin], [src.n, tgt.n], [h, h], [hs, hz],
                                           [first, l - 11], c, dt, 1, step, np.arange(tgt.N))
                for step in (l - 2, l - 1, l)]
        A_l, A_1, A_2 = (p[:, 1:].T for p in (pots[2], pots[1], pots[0]))
        E, B = ofields.fields(pots[2][:, 0], A_l, A_1, A_2, tgt.n, h, c, dt)
        Ez, By = dipole_fields(Q * a, omega, d, l * dt, c)
        eE.append(abs(E[2, k] - Ez) / scaleE)
        eB.append(abs(B[1, k] - By) / scaleB)
        side.append((abs(E[0, k]) / scaleE, abs(E[1, k]) / scaleE))
    return max(eE), max(eB), side, a / d


@pytest.mark.parametrize("d", [90.0, 500.0, 2000.0, 7500.0])
def test_oracle_fields_of_an_oscillating_dipole(d):
    """At dt = 0.0125 the fields match within 1e-4 of their amplitude; the
    gap is the time discretisation of the sampled sums (Eq. 7's hat
    interpolation, second order but with a phase-dependent constant): it is
    at least halved from dt = 0.05 (measured: up to 1.3e-3 at 0.05, 4e-4 at
    0.025, 3.3e-5 at 0.0125)."""
    eE, eB, side, a_over_d = dipole_errors(d, 0.0125)
    assert eE < 1e-4 and eB < 1e-4, (eE, eB)
    for ex, ey in side:   # broadside: E along z, up to the moving charge's quadrupole (~ a/d)
        assert ex < 3 * a_over_d and ey < 1e-6
    eE4, eB4, _, _ = dipole_errors(d, 0.05)
    assert eE < eE4 / 2 and eB < eB4 / 2, (eE, eE4, eB, eB4)
