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
