"""FP64 oracle of the learned far field (test infrastructure only).

The learned far field stands in for the retarded sum of Eq. 2 (sampled as in
Eqs. 7-8) between two well-separated sub-domains.  It is an approximation:
its result is judged by the direct sum (``oracle.eval_points`` /
``oracle.eval_positions``), not by this module.  What this module fixes is
each step's arithmetic, written plainly in NumPy FP64 so that the CUDA steps
can be compared with it one by one.  Only ``tests/`` may import it.

Steps, for a source domain s and a target domain t with box centres c_s, c_t:

1. Moments of a source slice (l <= 2) about c_s, per field f of
   (rho, Jx, Jy, Jz):  Q = sum S h^3,  p_i = sum S d_i h^3,
   q_ij = sum S d_i d_j h^3 (d = r - c_s; six entries xx xy xz yy yz zz).
   These are the monopole, dipole and (unreduced) quadrupole of the
   multipole expansion of the source (Sec. IV: the far interaction is
   carried by a few moments of the density).
2. Canonical frame: the rotation whose first row is the unit vector n from
   c_s to c_t; the second row is the component of the coordinate axis least
   aligned with n (lowest index on ties) orthogonal to n, normalised; the
   third is n x e2.  Moments rotate as scalars, vectors and rank-2 tensors;
   the current's components mix as a vector (J' = Rot J).
3. Delay window: the rotated moments sampled at the W fractional times
   l - tau_c - o_k, o_k = k - (W/2 - 1), k = 0..W-1, tau_c = |c_t - c_s|/(c dt),
   by the same hat (linear) interpolation in time as Eq. 7.
4. Features per field: the W x 10 window, followed by the same window times
   L0 / |c_t - c_s| (the 1/R scale of the dipole and quadrupole terms relative
   to the monopole); divided by nu, the RMS of the first half (nu = 0: zero
   row).
5. Network: x -> W1 -> leaky -> W2 -> leaky -> W3 -> leaky -> W4, no biases,
   leaky(z) = z (z >= 0), ALPHA z (z < 0).  Bias-free with a positively
   homogeneous activation, the network commutes with the scale nu > 0.
   Loss: (1 / 2B) sum over the B rows of |y_hat - y|^2.  Adam updates
   (Kingma and Ba, 2015).
6. Output per field: y_hat[a] = R_a value'(x_a) / nu at the 64 canonical
   nodes x_a (a 4 x 4 x 4 tensor grid of first-kind Chebyshev points on the
   cube [-hw, hw]^3 in canonical coordinates around c_t, hw = half the
   target box diagonal, x' fastest), R_a = |x_a - c_s|; value' is the raw
   retarded sum (phi, and J' sums without the 1/c of A).
7. Re-interpolation to the target's own interpolation nodes (the far path's
   per-axis Chebyshev nodes, x fastest): tensor-product Lagrange in canonical
   coordinates, then the vector fields rotated back (A = Rot^T A').

Parity status: steps 1-5 and 7 are pinned in ``tests/test_oracle_learned.py``
(closed-form Gaussian moments and brute force, rotation invariants, exact
interpolation of linear histories, finite-difference gradients, the Adam
first step, exact polynomial re-interpolation).  Step 6's labels come from
``oracle.eval_positions``, which is pinned there too.
"""
from __future__ import annotations

import numpy as np

NMOM = 10
ALPHA = 0.2
NODES = 4
L0 = 1000.0


# ---------------------------------------------------------------- 1. moments

def slice_moments(s4, origin, n, h, center):
    """[4][10] moments of one slice s4 [4][N] (x fastest) about ``center``."""
    nx, ny, nz = (int(v) for v in n)
    x = origin[0] + h * np.arange(nx) - center[0]
    y = origin[1] + h * np.arange(ny) - center[1]
    z = origin[2] + h * np.arange(nz) - center[2]
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    d = [X.reshape(-1), Y.reshape(-1), Z.reshape(-1)]
    vol = h ** 3
    out = np.zeros((4, NMOM))
    for f in range(4):
        S = np.asarray(s4[f], dtype=np.float64)
        out[f, 0] = S.sum() * vol
        for i in range(3):
            out[f, 1 + i] = (S * d[i]).sum() * vol
        k = 4
        for i in range(3):
            for j in range(i, 3):
                out[f, k] = (S * d[i] * d[j]).sum() * vol
                k += 1
    return out


# ---------------------------------------------------------------- 2. frame

def canonical_frame(nvec):
    n = np.asarray(nvec, dtype=np.float64)
    n = n / np.linalg.norm(n)
    e = np.zeros(3)
    e[int(np.argmin(np.abs(n)))] = 1.0        # argmin returns the lowest index on ties
    u = e - (e @ n) * n
    e2 = u / np.linalg.norm(u)
    e3 = np.cross(n, e2)
    return np.stack([n, e2, e3])


def _quad_matrix(q6):
    xx, xy, xz, yy, yz, zz = q6
    return np.array([[xx, xy, xz], [xy, yy, yz], [xz, yz, zz]])


def rotate_moments(M, R):
    """Moments [4][10] in the frame with rows R: spatial rotation, then the
    current components as a vector."""
    sp = np.zeros((4, NMOM))
    for f in range(4):
        sp[f, 0] = M[f, 0]
        sp[f, 1:4] = R @ M[f, 1:4]
        q = R @ _quad_matrix(M[f, 4:10]) @ R.T
        sp[f, 4:10] = [q[0, 0], q[0, 1], q[0, 2], q[1, 1], q[1, 2], q[2, 2]]
    out = sp.copy()
    out[1:4] = R @ sp[1:4]
    return out


# ---------------------------------------------------------------- 3-4. window, features

def window_offsets(W):
    return np.arange(W) - (W // 2 - 1)


def sample_window(moment_of_step, t_centre, W):
    """[W][4][10]: moment_of_step(j) -> [4][10] at integer step j, sampled at
    t_centre - o_k by linear interpolation."""
    out = np.zeros((W, 4, NMOM))
    for k, o in enumerate(window_offsets(W)):
        s = t_centre - o
        j = int(np.floor(s))
        w = s - j
        a = moment_of_step(j)
        out[k] = a if w == 0.0 else (1.0 - w) * a + w * moment_of_step(j + 1)
    return out


def features(win, Rc):
    """Rows [4][2*W*10] and scales nu [4] from a window [W][4][10]."""
    W = win.shape[0]
    X = np.zeros((4, 2 * W * NMOM))
    nu = np.zeros(4)
    for f in range(4):
        base = win[:, f, :].reshape(-1)
        r = np.sqrt(np.mean(base * base))
        nu[f] = r
        if r > 0.0:
            X[f] = np.concatenate([base, base * (L0 / Rc)]) / r
    return X, nu


# ---------------------------------------------------------------- 5. network

def leaky(z):
    return np.where(z >= 0.0, z, ALPHA * z)


def leaky_grad(z):
    return np.where(z >= 0.0, 1.0, ALPHA)


def mlp_forward(Ws, X, act16=False):
    """Ws: [W1 (d1 x d0), ..., W4]; X [B][d0].  Returns (z list, a list)
    with a[0] = X and a[-1] the output.  act16: each hidden activation is
    rounded to fp16 (the representation in which a tensor-core network
    passes it to the next layer's product), so that the slope each node
    takes (the sign of z) is decided on the same values as there; the
    arithmetic stays FP64."""
    a = [np.asarray(X, dtype=np.float64)]
    z = []
    for i, Wl in enumerate(Ws):
        zi = a[-1] @ np.asarray(Wl, dtype=np.float64).T
        z.append(zi)
        if i < len(Ws) - 1:
            ai = leaky(zi)
            a.append(ai.astype(np.float16).astype(np.float64) if act16 else ai)
        else:
            a.append(zi)
    return z, a


def mlp_loss_grad(Ws, X, Y, act16=False):
    """Loss (1/2B) sum |out - Y|^2 and its gradient with respect to each W
    (act16 as for mlp_forward)."""
    B = X.shape[0]
    z, a = mlp_forward(Ws, X, act16)
    r = a[-1] - np.asarray(Y, dtype=np.float64)
    loss = 0.5 * np.sum(r * r) / B
    grads = [None] * len(Ws)
    delta = r / B                                    # dL/dz of the last layer
    for i in reversed(range(len(Ws))):
        grads[i] = delta.T @ a[i]
        if i > 0:
            delta = (delta @ np.asarray(Ws[i], dtype=np.float64)) * leaky_grad(z[i - 1])
    return loss, grads


def adam_step(p, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update of parameter p with gradient g; t counts from 1."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** t)
    vh = v / (1.0 - b2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


# ---------------------------------------------------------------- 6-7. nodes, output

def chebyshev(lo, hi, p):
    a = np.arange(p)
    return 0.5 * (lo + hi) - 0.5 * (hi - lo) * np.cos((2.0 * a + 1.0) * np.pi / (2.0 * p))


def canonical_nodes(box_lengths):
    """[64][3] canonical coordinates (relative to c_t), x' fastest."""
    hw = 0.5 * float(np.linalg.norm(box_lengths))
    g = chebyshev(-hw, hw, NODES)
    out = []
    for c in range(NODES):
        for b in range(NODES):
            for a in range(NODES):
                out.append([g[a], g[b], g[c]])
    return np.array(out)


def target_nodes(origin, n, h, p=NODES):
    """The far path's interpolation nodes of a target box: per axis the grid
    nodes if n <= p, else p first-kind Chebyshev points of [o, o + h(n-1)];
    [P][3] world positions with x fastest."""
    axes = []
    for i in range(3):
        if n[i] <= p:
            axes.append(origin[i] + h * np.arange(n[i]))
        else:
            axes.append(chebyshev(origin[i], origin[i] + h * (n[i] - 1), p))
    out = []
    for zc in axes[2]:
        for yc in axes[1]:
            for xc in axes[0]:
                out.append([xc, yc, zc])
    return np.array(out)


def lagrange_weights(nodes, x):
    w = np.ones(len(nodes))
    for a in range(len(nodes)):
        for b in range(len(nodes)):
            if b != a:
                w[a] *= (x - nodes[b]) / (nodes[a] - nodes[b])
    return w


def reinterp_matrix(box_lengths, R, c_t, world_nodes):
    """P [len(world_nodes)][64]: values at the canonical nodes -> values at
    world_nodes, by tensor-product Lagrange interpolation in canonical
    coordinates."""
    hw = 0.5 * float(np.linalg.norm(box_lengths))
    g = chebyshev(-hw, hw, NODES)
    P = np.zeros((len(world_nodes), NODES ** 3))
    for i, xw in enumerate(world_nodes):
        xc = R @ (np.asarray(xw) - c_t)
        wa, wb, wc = (lagrange_weights(g, xc[k]) for k in range(3))
        P[i] = np.einsum("c,b,a->cba", wc, wb, wa).reshape(-1)
    return P


def assemble(yhat, nu, R_a, P, R):
    """Raw-sum values at the target nodes [len(P)][4] (phi and J sums, A
    without its 1/c) from the network output yhat [4][64]."""
    v = nu[:, None] * yhat / R_a[None, :]
    u = (P @ v.T)                                    # [nodes][4] canonical fields
    out = u.copy()
    out[:, 1:4] = u[:, 1:4] @ R                      # A_i = sum_k R_ki A'_k
    return out
