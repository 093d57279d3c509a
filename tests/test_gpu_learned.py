"""The learned far field on the GPU against its FP64 oracle.

Network: forward outputs and loss gradients of the CUDA kernels (fp16
operands, fp32 accumulation) against ``oracle.learned`` in FP64 on the same
fp16-rounded weights and inputs.  The CUDA path also rounds each hidden
activation (and each back-propagated gradient) to fp16, a relative error of
2^-11 per rounding; over four layers that stays below 5e-3 in rel-L2 for the
outputs and below 2e-2 for the gradients (which pass through fp16 twice per
layer), the bars used here.
"""
import numpy as np
import pytest

from oracle import learned as L
from paper_2311_15429_gb300 import rp

pytestmark = pytest.mark.gpu


def _net(seed):
    dims, nw = rp.rp_mlp_layout()
    rng = np.random.default_rng(seed)
    Ws = []
    for l in range(4):
        b = np.sqrt(6.0 / ((1 + L.ALPHA ** 2) * dims[l]))
        Ws.append(rng.uniform(-b, b, (dims[l + 1], dims[l])).astype(np.float16).astype(np.float64))
    flat = np.concatenate([w.reshape(-1) for w in Ws]).astype(np.float32)
    assert flat.size == nw
    return dims, Ws, flat, rng


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def test_layout_matches_the_oracle_network():
    dims, nw = rp.rp_mlp_layout()
    assert dims == [320, 256, 256, 256, 64]
    assert dims[0] == 2 * 16 * L.NMOM and dims[4] == L.NODES ** 3


@pytest.mark.parametrize("rows", [128, 512])
def test_forward_matches_oracle(rows):
    dims, Ws, flat, rng = _net(rows)
    X = rng.standard_normal((rows, dims[0])).astype(np.float16).astype(np.float64)
    y = rp.rp_mlp_forward(flat, X)
    want = L.mlp_forward(Ws, X)[1][-1]
    assert _rel(y, want) < 5e-3


@pytest.mark.parametrize("rows", [256, 1024])
def test_gradients_match_oracle(rows):
    dims, Ws, flat, rng = _net(7 + rows)
    X = rng.standard_normal((rows, dims[0])).astype(np.float16).astype(np.float64)
    T = rng.standard_normal((rows, dims[4]))
    loss, g = rp.rp_mlp_grad(flat, X, T)
    want_loss, want_g = L.mlp_loss_grad(Ws, X, T)
    assert abs(loss - want_loss) / want_loss < 5e-3
    o = 0
    for l in range(4):
        n = dims[l] * dims[l + 1]
        assert _rel(g[o:o + n].reshape(dims[l + 1], dims[l]), want_g[l]) < 2e-2, l
        o += n


def _history_slices(desc, n, h):
    """Source slices [64][4][N] (float64) of one generated history."""
    import math
    from paper_2311_15429_gb300 import synth
    nx, ny, nz = n
    x = h * np.arange(nx)
    y = h * np.arange(ny)
    z = h * np.arange(nz)
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    X, Y, Z = X.reshape(-1), Y.reshape(-1), Z.reshape(-1)
    G, T = 3, 64
    amp = desc[4 * G:4 * G + G * T].reshape(G, T)
    damp = desc[4 * G + G * T:4 * G + 2 * G * T].reshape(G, T)
    g = np.zeros((G, X.size))
    gp = np.zeros((G, 3, X.size))
    for k in range(G):
        cx, cy, cz, s = desc[4 * k:4 * k + 4]
        dx, dy, dz = X - cx, Y - cy, Z - cz
        g[k] = synth._unit_gaussian(dx * dx + dy * dy + dz * dz, s)
        gp[k] = np.stack(synth._grad_gaussian_potential(dx, dy, dz, s))
    out = np.zeros((T, 4, X.size))
    for j in range(T):
        out[j, 0] = amp[:, j] @ g
        out[j, 1:] = np.einsum("k,kfn->fn", damp[:, j], gp)
    return out


def test_dataset_rows_and_targets_match_oracle():
    """Network rows (moments -> canonical frame -> delay window -> scaling)
    and targets (the direct retarded sum at the canonical nodes, scaled) of
    the GPU data path against oracle.learned + the oracle's point evaluator."""
    import oracle
    n, h = (16, 14, 12), 0.25
    Lt = (3.75, 3.75, 3.0)
    direction = np.array([0.6, -0.3, 0.74])
    direction /= np.linalg.norm(direction)
    Rc, c, dt = 300.0, 137.036, 0.05
    H, S = 2, 8
    X, Y, D = rp.rp_learned_dataset(n, h, Lt, direction, Rc, 123, H, S, c, dt)
    R = L.canonical_frame(direction)
    cs = h * (np.array(n) - 1) / 2
    cn = L.canonical_nodes(np.array(Lt))
    pos = cs + Rc * direction + cn @ R                 # canonical node -> world
    Dn = np.linalg.norm(pos - cs, axis=1)
    worst_x, worst_y = 0.0, 0.0
    for i in range(H):
        desc = D[i]
        t0 = desc[-5]
        assert np.allclose(desc[-4:-1], direction) and desc[-1] == Rc
        sl = _history_slices(desc, n, h)
        mom = np.stack([L.rotate_moments(L.slice_moments(sl[j], np.zeros(3), n, h, cs), R) for j in range(64)])
        tau_c = Rc / (c * dt)
        assert abs((t0 + tau_c) - round(t0 + tau_c)) < 1e-9
        for k in range(S):
            win = L.sample_window(lambda j: mom[j], t0 + k, 16)
            xo, nu = L.features(win, Rc)
            row = (i * S + k) * 4
            for f in range(4):
                worst_x = max(worst_x, np.linalg.norm(X[row + f] - xo[f]) / np.linalg.norm(xo[f]))
            step = int(round(t0 + tau_c)) + k
            val = oracle.eval_positions([np.zeros(3)], [n], [h], [sl], 0, c, dt, step, pos)
            raw = val.copy()
            raw[:, 1:] *= c
            canon = raw.copy()
            canon[:, 1:] = raw[:, 1:] @ R.T
            for f in range(4):
                want = Dn * canon[:, f] / nu[f]
                worst_y = max(worst_y, np.linalg.norm(Y[row + f] - want) / np.linalg.norm(want))
    assert worst_x < 2e-3, worst_x      # fp16 rows
    assert worst_y < 1e-4, worst_y      # fp32 sums of the direct retarded sum
