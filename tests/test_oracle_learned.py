"""Pins of the learned far field's oracle steps and of the point evaluator
(CPU only).  Each check compares with something other than the oracle
itself: a closed form, brute force, finite differences or an exact property.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import learned as L


def _gauss_slice(n, h, origin, centre, sigma, Q=1.0, jvec=(0.0, 0.0, 0.0)):
    nx, ny, nz = n
    x = origin[0] + h * np.arange(nx)
    y = origin[1] + h * np.arange(ny)
    z = origin[2] + h * np.arange(nz)
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    r2 = (X - centre[0]) ** 2 + (Y - centre[1]) ** 2 + (Z - centre[2]) ** 2
    g = Q * np.exp(-r2 / (2 * sigma ** 2)) / (2 * np.pi * sigma ** 2) ** 1.5
    g = g.reshape(-1)
    return np.stack([g, jvec[0] * g, jvec[1] * g, jvec[2] * g])


# ---------------------------------------------------------------- point evaluator

def test_positions_static_limit_is_coulomb():
    """c -> infinity: a Gaussian of charge Q seen from far points is
    Q erf(R / sqrt2 sigma) / R (the grid sum of a smooth Gaussian is
    spectrally accurate)."""
    n, h, sigma = (32, 32, 32), 0.2, 0.45      # box half-width 7 sigma: no truncation
    origin = np.zeros(3)
    centre = origin + h * 15.5
    s = _gauss_slice(n, h, origin, centre, sigma, Q=2.0)
    hist = np.stack([s, s]).astype(np.float64)        # constant in time
    pts = centre + np.array([[40.0, 3.0, -2.0], [0.0, -25.0, 7.0], [11.0, 11.0, 11.0]])
    out = oracle.eval_positions([origin], [n], [h], [hist], 0, 1e15, 0.05, 1, pts)
    R = np.linalg.norm(pts - centre, axis=1)
    want = 2.0 * np.array([math.erf(r / (math.sqrt(2) * sigma)) for r in R]) / R
    assert np.max(np.abs(out[:, 0] - want) / want) < 1e-9


def test_positions_breathing_monopole_phase():
    """A monopole of amplitude 1 + 0.1 sin(w t) seen 300 bohr away lags by
    R/c: phi = Q(1 + 0.1 sin(w (t - R/c)))/R up to the hat interpolation's
    (w dt)^2/8 relative error on the oscillating part."""
    n, h, sigma, dt, c, w = (24, 24, 24), 0.25, 0.4, 0.05, 137.036, 0.9
    origin = np.zeros(3)
    centre = origin + h * 11.5
    g = _gauss_slice(n, h, origin, centre, sigma)
    pt = centre + np.array([300.0, 0.0, 0.0])
    R = 300.0
    lag = int(R / (c * dt)) + 3
    T = lag + 12
    hist = np.stack([g * (1 + 0.1 * np.sin(w * j * dt)) for j in range(T)])
    for step in (lag + 2, lag + 7):
        out = oracle.eval_positions([origin], [n], [h], [hist], 0, c, dt, step, pt[None])
        want = (1 + 0.1 * math.sin(w * (step * dt - R / c))) / R
        assert abs(out[0, 0] - want) < 0.1 / R * (w * dt) ** 2 / 8 * 1.5 + 1e-6 / R


def test_positions_match_nodes_of_an_empty_domain():
    """At the grid nodes of a domain holding no source, the point evaluator
    and the node evaluator sum the same terms."""
    src = dict(origin=np.zeros(3), n=(6, 5, 4), h=0.3)
    tgt = dict(origin=np.array([9.0, 1.0, -2.0]), n=(3, 3, 2), h=0.4)
    rng = np.random.default_rng(3)
    T = 40
    hs = rng.standard_normal((T, 4, 120))
    ht = np.zeros((T, 4, 18))
    origins = [src["origin"], tgt["origin"]]
    ns, hh = [src["n"], tgt["n"]], [src["h"], tgt["h"]]
    nodes = np.arange(18)
    a = oracle.eval_points(origins, ns, hh, [hs, ht], 0, 137.036, 0.01, 1, T - 1, nodes)
    pos = np.array([[tgt["origin"][0] + 0.4 * (k % 3), tgt["origin"][1] + 0.4 * ((k // 3) % 3),
                     tgt["origin"][2] + 0.4 * (k // 9)] for k in nodes])
    b = oracle.eval_positions([src["origin"]], [src["n"]], [src["h"]], [hs], 0, 137.036, 0.01, T - 1, pos)
    assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(b))


# ---------------------------------------------------------------- moments

def test_gaussian_moments_closed_form():
    """Moments of a Gaussian (charge Q, centre c0, width sigma) about a point
    x0: Q, Q d, Q (sigma^2 I + d d^T) with d = c0 - x0; and the current
    J = v g has the same moments times v."""
    n, h, sigma, Q = (32, 30, 28), 0.2, 0.4, 1.7
    origin = np.array([1.0, -2.0, 0.5])
    c0 = origin + h * np.array([15.3, 14.2, 13.9])
    x0 = origin + h * np.array([15.5, 14.5, 13.5])
    v = np.array([0.3, -1.2, 0.8])
    M = L.slice_moments(_gauss_slice(n, h, origin, c0, sigma, Q, v), origin, n, h, x0)
    d = c0 - x0
    q = Q * (sigma ** 2 * np.eye(3) + np.outer(d, d))
    want = np.concatenate([[Q], Q * d, [q[0, 0], q[0, 1], q[0, 2], q[1, 1], q[1, 2], q[2, 2]]])
    assert np.allclose(M[0], want, rtol=0, atol=1e-9)
    for k in range(3):
        assert np.allclose(M[1 + k], v[k] * want, rtol=0, atol=1e-9)


def test_moments_brute_force_two_cubed():
    rng = np.random.default_rng(0)
    s = rng.standard_normal((4, 8))
    origin, h = np.array([0.1, 0.2, 0.3]), 0.5
    x0 = np.array([0.3, 0.4, 0.1])
    M = L.slice_moments(s, origin, (2, 2, 2), h, x0)
    for f in range(4):
        acc = np.zeros(10)
        for q in range(8):
            d = origin + h * np.array([q % 2, (q // 2) % 2, q // 4]) - x0
            acc += s[f, q] * h ** 3 * np.array([1, d[0], d[1], d[2], d[0] * d[0], d[0] * d[1], d[0] * d[2],
                                                 d[1] * d[1], d[1] * d[2], d[2] * d[2]])
        assert np.allclose(M[f], acc, atol=1e-14)


# ---------------------------------------------------------------- frame

@pytest.mark.parametrize("n", [(1, 0, 0), (0.3, -0.4, 0.866), (-1, 1, 1), (0, 0, -2)])
def test_canonical_frame_is_a_rotation_onto_n(n):
    R = L.canonical_frame(n)
    assert np.allclose(R @ R.T, np.eye(3), atol=1e-14)
    assert abs(np.linalg.det(R) - 1.0) < 1e-14
    assert np.allclose(R[0], np.asarray(n) / np.linalg.norm(n))
    assert np.allclose(R @ np.asarray(n, float), [np.linalg.norm(n), 0, 0], atol=1e-14)


def test_rotated_moments_are_moments_of_the_rotated_source():
    """Rotating the source (positions and current vectors) and taking moments
    equals rotating the moments: checked on a Gaussian whose moments are known
    in closed form in both frames."""
    R = L.canonical_frame((0.2, -0.7, 0.4))
    sigma, Q = 0.6, 1.3
    d = np.array([0.4, -0.3, 0.2])
    v = np.array([0.5, 0.1, -0.9])
    def closed(dd, vv):
        q = Q * (sigma ** 2 * np.eye(3) + np.outer(dd, dd))
        row = np.concatenate([[Q], Q * dd, [q[0, 0], q[0, 1], q[0, 2], q[1, 1], q[1, 2], q[2, 2]]])
        return np.stack([row, vv[0] * row, vv[1] * row, vv[2] * row])
    assert np.allclose(L.rotate_moments(closed(d, v), R), closed(R @ d, R @ v), atol=1e-13)


# ---------------------------------------------------------------- window, features

def test_window_interpolates_linear_histories_exactly():
    A = np.arange(40.0).reshape(4, 10)
    B = np.linspace(-1, 2, 40).reshape(4, 10)
    win = L.sample_window(lambda j: A + B * j, 123.37, 16)
    for k, o in enumerate(L.window_offsets(16)):
        assert np.allclose(win[k], A + B * (123.37 - o), atol=1e-10)
    assert list(L.window_offsets(16)) == list(range(-7, 9))


def test_feature_scaling():
    rng = np.random.default_rng(1)
    win = rng.standard_normal((16, 4, 10))
    win[:, 2] = 0.0
    X, nu = L.features(win, 4000.0)
    for f in (0, 1, 3):
        base = X[f, :160]
        assert abs(np.sqrt(np.mean(base ** 2)) - 1.0) < 1e-14
        assert np.allclose(X[f, 160:], base * L.L0 / 4000.0)
        assert np.allclose(base * nu[f], win[:, f, :].reshape(-1))
    assert nu[2] == 0.0 and not X[2].any()


# ---------------------------------------------------------------- network

def test_mlp_gradients_match_finite_differences():
    rng = np.random.default_rng(2)
    sizes = [10, 7, 6, 5, 4]
    Ws = [rng.standard_normal((sizes[i + 1], sizes[i])) * 0.5 for i in range(4)]
    X = rng.standard_normal((9, 10))
    Y = rng.standard_normal((9, 4))
    loss, grads = L.mlp_loss_grad(Ws, X, Y)
    eps = 1e-6
    for li in range(4):
        num = np.zeros_like(Ws[li])
        for idx in np.ndindex(Ws[li].shape):
            Wp = [w.copy() for w in Ws]
            Wm = [w.copy() for w in Ws]
            Wp[li][idx] += eps
            Wm[li][idx] -= eps
            num[idx] = (L.mlp_loss_grad(Wp, X, Y)[0] - L.mlp_loss_grad(Wm, X, Y)[0]) / (2 * eps)
        assert np.max(np.abs(num - grads[li])) < 1e-7 * max(1.0, np.max(np.abs(num))), li


def test_mlp_is_positively_homogeneous():
    rng = np.random.default_rng(4)
    Ws = [rng.standard_normal((6, 8)), rng.standard_normal((6, 6)), rng.standard_normal((6, 6)),
          rng.standard_normal((3, 6))]
    X = rng.standard_normal((5, 8))
    a = L.mlp_forward(Ws, X)[1][-1]
    b = L.mlp_forward(Ws, 3.7 * X)[1][-1]
    assert np.allclose(b, 3.7 * a, rtol=1e-13)


def test_adam_first_step_moves_by_lr_sign():
    p = np.array([1.0, -2.0, 0.5])
    g = np.array([3.0, -0.01, 1e-3])
    q, m, v = L.adam_step(p, g, np.zeros(3), np.zeros(3), 1, 0.01, eps=0.0)
    assert np.allclose(q, p - 0.01 * np.sign(g), atol=1e-15)


# ---------------------------------------------------------------- nodes, output

def test_reinterpolation_is_exact_for_cubics():
    """Tensor-product cubics in canonical coordinates are reproduced exactly
    at the target's nodes, and assemble() rotates the vector fields back."""
    box = np.array([12.0, 12.0, 11.0])
    origin = np.array([1800.0, 300.0, -200.0])
    n, h = (48, 48, 44), 0.25
    c_t = origin + h * (np.array(n) - 1) / 2
    R = L.canonical_frame(c_t - np.array([0.0, 0.0, 0.0]))
    cn = L.canonical_nodes(box)
    tn = L.target_nodes(origin, n, h)
    P = L.reinterp_matrix(box, R, c_t, tn)
    f = lambda x: 1.0 + 0.3 * x[..., 0] - 0.02 * x[..., 1] ** 2 * x[..., 2] + 1e-3 * x[..., 0] ** 3 * x[..., 2] ** 3
    got = P @ f(cn)
    want = f((tn - c_t) @ R.T)
    assert np.max(np.abs(got - want)) < 1e-10
    # constant fields: phi = 2 and A' = R v give A = v at every node
    v = np.array([0.3, -0.5, 0.7])
    Rv = R @ v
    yhat = np.stack([np.full(64, 2.0), np.full(64, Rv[0]), np.full(64, Rv[1]), np.full(64, Rv[2])])
    out = L.assemble(yhat, np.ones(4), np.ones(64), P, R)
    assert np.allclose(out[:, 0], 2.0) and np.allclose(out[:, 1:], v[None, :])
