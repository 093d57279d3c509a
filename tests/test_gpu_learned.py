"""The learned far field on the GPU against its FP64 oracle.

Network: forward outputs and loss gradients of the CUDA kernels (fp16
operands, fp32 accumulation) against ``oracle.learned`` in FP64 on the same
fp16-rounded weights and inputs, with its hidden activations carried as
fp16 too (act16: the tensor cores take them as fp16 operands, and the slope
of each leaky node, the sign of z, is then decided on the same values).  The
CUDA path further rounds each back-propagated gradient to fp16, a relative
error of 2^-11 per rounding; over four layers that stays below 5e-3 in
rel-L2 for the outputs and the gradients, the bars used here.
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
    want = L.mlp_forward(Ws, X, act16=True)[1][-1]
    assert _rel(y, want) < 5e-3


@pytest.mark.parametrize("rows", [256, 1024])
def test_gradients_match_oracle(rows):
    dims, Ws, flat, rng = _net(7 + rows)
    X = rng.standard_normal((rows, dims[0])).astype(np.float16).astype(np.float64)
    T = rng.standard_normal((rows, dims[4]))
    loss, g = rp.rp_mlp_grad(flat, X, T)
    want_loss, want_g = L.mlp_loss_grad(Ws, X, T, act16=True)
    assert abs(loss - want_loss) / want_loss < 5e-3
    o = 0
    errs = []
    for l in range(4):
        n = dims[l] * dims[l + 1]
        errs.append(_rel(g[o:o + n].reshape(dims[l + 1], dims[l]), want_g[l]))
        o += n
    print(f"\ngradient rel-L2 per layer ({rows} rows): " + ", ".join(f"{e:.2e}" for e in errs))
    assert max(errs) < 5e-3, errs


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


def _far_setup(n=16, dist=3000.0):
    from paper_2311_15429_gb300 import synth
    doms = [synth.cubic((0.0, 0.0, 0.0), n, 0.25), synth.cubic((8.0, 0.5, -0.3), n, 0.25),
            synth.cubic((dist * 0.6, dist * 0.48, -dist * 0.64), n, 0.25)]
    return doms, synth.seeded_sources(doms)


def _run_far(doms, hists, train, **kw):
    import torch
    from paper_2311_15429_gb300 import synth
    dev = torch.device("cuda", 0)
    with rp.RetardedPotentials(doms, synth.C_AU, 0.05, mode=rp.RP_MODE_LOWRANK, far_distance=500.0,
                               far_batch=16) as lib:
        report = lib.train_far_model(500.0, **kw) if train else None
        q = lib.query()
        kinds = {(t, s): lib.pair_info(t, s)["kind"] for t in range(3) for s in range(3)}
        T = hists[0].shape[0]
        for i in range(T):
            lib.push_all([torch.from_numpy(h[i, 0].copy()).to(dev) for h in hists],
                         [torch.from_numpy(h[i, 1:].copy().reshape(-1)).to(dev) for h in hists])
        phi, A = lib.evaluate()
        lib.sync()
        out = [np.concatenate([phi[d].cpu().numpy()[None], A[d].cpu().numpy().reshape(3, -1)]) for d in range(3)]
    return out, report, q, kinds


def test_trained_far_pairs_match_oracle():
    """rp_train_far_model moves the four far pairs onto the network (the
    linear skip plus the MLP); the far field alone (only the far domain
    active) and the total field then match the FP64 oracle within 1e-3."""
    from paper_2311_15429_gb300 import synth
    from _harness import oracle_values, rel_l2
    doms, srcs = _far_setup()
    with rp.RetardedPotentials(doms, synth.C_AU, 0.05, mode=rp.RP_MODE_LOWRANK, far_distance=500.0,
                               far_batch=16) as lib:
        T = lib.query()["max_lag"] + 24
    hists = [s.history(0, T, 0.05) for s in srcs]
    zero = [np.zeros_like(hists[0]), np.zeros_like(hists[1]), hists[2]]
    out, rep, q, kinds = _run_far(doms, zero, True)
    assert rep["candidates"] == 4 and rep["learned"] == 4, rep
    assert q["npairs_learned"] == 4 and q["npairs_far"] == 0
    for (t, s), k in kinds.items():
        assert k == (rp.RP_PAIR_LEARNED if (t == 2) != (s == 2) else rp.RP_PAIR_FFT), (t, s, k)
    nodes = np.arange(0, doms[0].N, 5)
    for t in (0, 1):
        want = oracle_values(doms, zero, 0, synth.C_AU, 0.05, t, T - 1, nodes)
        errs = rel_l2(out[t][:, nodes], want)
        assert max(errs) <= 1e-3, ("far only", t, errs)
    out, rep, q, _ = _run_far(doms, hists, True)
    for t in range(3):
        want = oracle_values(doms, hists, 0, synth.C_AU, 0.05, t, T - 1, nodes)
        errs = rel_l2(out[t][:, nodes], want)
        assert max(errs) <= 1e-3, ("total", t, errs)


def test_learned_gain_over_the_low_rank_path():
    """What the trained stand-in gains over the method without it (the
    low-rank far path of the same pairs): the far path's device memory drops
    from the factor matrices to a few kB of moment rings and node tables,
    at a far-field error inside the same 1e-3 bar; the training report gives
    the validation error of the linear skip alone and with the network."""
    from paper_2311_15429_gb300 import synth
    doms, _ = _far_setup(24, 3000.0)
    with rp.RetardedPotentials(doms, synth.C_AU, 0.05, mode=rp.RP_MODE_LOWRANK, far_distance=500.0,
                               far_batch=16) as lib:
        before = lib.query()["far_bytes"]
        rep = lib.train_far_model(500.0)
        after = lib.query()["far_bytes"]
    assert rep["learned"] == 4, rep
    assert after * 100 < before, (before, after)
    assert rep["val_max"] <= 1e-3 and rep["val_linear_max"] <= 1e-3, rep
    print("far-path bytes low-rank %d -> learned %d; validation rel-L2 linear skip %.3g, with network %.3g"
          % (before, after, rep["val_linear_max"], rep["val_max"]))


def test_training_errors_and_state():
    from paper_2311_15429_gb300 import synth
    doms, _ = _far_setup()
    with rp.RetardedPotentials(doms, synth.C_AU, 0.05) as lib:     # FFT mode
        with pytest.raises(rp.RPError) as e:
            lib.train_far_model(500.0)
        assert e.value.status == rp.RP_ERR_UNSUPPORTED
    with rp.RetardedPotentials(doms, synth.C_AU, 0.05, mode=rp.RP_MODE_LOWRANK, far_distance=500.0,
                               far_batch=16) as lib:
        with pytest.raises(rp.RPError) as e:
            lib.train_far_model(500.0, batch=100)                   # not a multiple of 128
        assert e.value.status == rp.RP_ERR_ARG
        rep = lib.train_far_model(1e6)                               # no candidates
        assert rep["candidates"] == 0 and rep["learned"] == 0
        with pytest.raises(rp.RPError) as e:
            lib.train_far_model(500.0)                               # only once
        assert e.value.status == rp.RP_ERR_STATE


def test_learned_pairs_beside_low_rank_pairs():
    """Learned and low-rank far pairs in one context: domains 0 and 1 are
    1000 bohr apart (low-rank), the rest at least 2000 bohr from every other
    domain (learned).  Only domain 2 carries a source; every other domain's
    field is its far field, whether the target also has low-rank pairs (its
    coefficient slot is added to) or only learned ones (the slot is set)."""
    import torch
    from paper_2311_15429_gb300 import synth
    from _harness import oracle_values, rel_l2
    dev = torch.device("cuda", 0)
    doms = [synth.cubic((0.0, 0.0, 0.0), 16, 0.25), synth.cubic((1000.0, 0.0, 0.0), 16, 0.25),
            synth.cubic((300.0, 2600.0, -500.0), 16, 0.25), synth.cubic((-2400.0, 900.0, 1700.0), 16, 0.25)]
    srcs = synth.seeded_sources(doms)
    with rp.RetardedPotentials(doms, synth.C_AU, 0.05, mode=rp.RP_MODE_LOWRANK, far_distance=500.0,
                               far_batch=16) as lib:
        rep = lib.train_far_model(2000.0)
        q = lib.query()
        kinds = [[lib.pair_info(t, s)["kind"] for s in range(4)] for t in range(4)]
        T = q["max_lag"] + 20
        hist = srcs[2].history(0, T, 0.05)
        zero = [torch.zeros(d.N, device=dev) for d in doms]
        zJ = [torch.zeros(3 * d.N, device=dev) for d in doms]
        for i in range(T):
            r = list(zero)
            J = list(zJ)
            r[2] = torch.from_numpy(hist[i, 0].copy()).to(dev)
            J[2] = torch.from_numpy(hist[i, 1:].copy().reshape(-1)).to(dev)
            lib.push_all(r, J)
        phi, A = lib.evaluate()
        lib.sync()
        out = [np.concatenate([phi[d].cpu().numpy()[None], A[d].cpu().numpy().reshape(3, -1)]) for d in range(4)]
    assert kinds[0][1] == rp.RP_PAIR_LOWRANK and kinds[1][0] == rp.RP_PAIR_LOWRANK
    assert rep["learned"] == 10 and q["npairs_learned"] == 10 and q["npairs_far"] == 2, (rep, q)
    hists = [np.zeros_like(hist), np.zeros_like(hist), hist, np.zeros_like(hist)]
    nodes = np.arange(0, doms[0].N, 9)
    for t in (0, 1, 3):
        want = oracle_values(doms, hists, 0, synth.C_AU, 0.05, t, T - 1, nodes)
        errs = rel_l2(out[t][:, nodes], want)
        assert max(errs) <= 1e-3, (t, errs)
