"""GPU: rp_fields (App. B: E = -grad phi - (1/c) dA/dt, B = curl A) against
the field oracle, and end to end on an oscillating dipole."""
import math

import numpy as np
import pytest

from oracle import fields as ofields
from paper_2311_15429_gb300 import rp, synth

from _harness import run_library

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("with_a2,with_b", [(True, True), (False, True), (True, False)])
def test_fields_kernel_matches_oracle(with_a2, with_b):
    """Random potentials on a 7 x 5 x 9 grid (faces and interior): the CUDA
    stencils against the FP64 oracle's, within FP32 rounding."""
    import torch
    dev = torch.device("cuda", 0)
    dom = synth.Domain((0.0, 0.0, 0.0), (7, 5, 9), 0.3)
    rng = np.random.default_rng(3)
    N = dom.N
    phi = rng.standard_normal(N).astype(np.float32)
    A = [rng.standard_normal(3 * N).astype(np.float32) for _ in range(3)]
    c, dt = synth.C_AU, 0.05
    ctx = rp.rp_create(c, dt)
    try:
        rp.rp_add_domain(ctx, dom.origin, dom.n, dom.h)
        rp.rp_finalize(ctx)
        t = lambda x: torch.from_numpy(x).to(dev)
        E = torch.zeros(3 * N, device=dev)
        B = torch.zeros(3 * N, device=dev) if with_b else None
        rp.rp_fields(ctx, 0, t(phi), t(A[0]), t(A[1]), t(A[2]) if with_a2 else None, E, B)
        rp.rp_sync(ctx)
        wantE, wantB = ofields.fields(phi, A[0].reshape(3, N), A[1].reshape(3, N),
                                      A[2].reshape(3, N) if with_a2 else None, dom.n, dom.h, c, dt)
        gotE = E.cpu().numpy().reshape(3, N)
        np.testing.assert_allclose(gotE, wantE, rtol=2e-6, atol=2e-6 * np.abs(wantE).max())
        if with_b:
            gotB = B.cpu().numpy().reshape(3, N)
            np.testing.assert_allclose(gotB, wantB, rtol=2e-6, atol=2e-6 * np.abs(wantB).max())
    finally:
        rp.rp_destroy(ctx)


def test_fields_argument_errors():
    import torch
    dev = torch.device("cuda", 0)
    ctx = rp.rp_create(synth.C_AU, 0.05)
    try:
        rp.rp_add_domain(ctx, (0.0, 0.0, 0.0), (2, 4, 4), 0.3)
        rp.rp_finalize(ctx)
        x = torch.zeros(3 * 32, device=dev)
        for args in ((0, x, x, x, None, x), (1, x, x, x, None, x), (0, None, x, x, None, x)):
            with pytest.raises(rp.RPError) as e:
                rp.rp_fields(ctx, *args)
            assert e.value.status == rp.RP_ERR_ARG
    finally:
        rp.rp_destroy(ctx)


def test_dipole_field_end_to_end():
    """An oscillating dipole (a +Q Gaussian moving along z over a static -Q
    one) seen 90 bohr away on its broadside: the library's potentials (FFT
    path) through rp_fields give E_z and B_y of the oscillating-dipole field.
    The FP32 potentials resolve the broadside field -- the small difference
    of the dipole's two lobes -- to about 1e-3; the FP64 oracle does the same
    check to 1e-4 out to 7500 bohr."""
    import torch
    dev = torch.device("cuda", 0)
    c, dt, omega, Q, a, sigma, h, d = synth.C_AU, 0.0125, 0.1, 1.0, 0.2, 0.5, 0.25, 90.0
    src = synth.cubic((0.0, 0.0, 0.0), 24, h)
    tgt = synth.cubic((d, 0.0, 0.0), 5, h)
    moving = synth.MovingGaussian(src, (0.0, 0.0, 0.0), sigma, a, omega, axis=(0.0, 0.0, 1.0), charge=Q)
    static = synth.BreathingGaussian(src, (0.0, 0.0, 0.0), sigma, 0.0, omega, charge=-Q)
    lag = int(math.ceil((d + 7.0) / (c * dt))) + 2
    j0, T = -lag - 2, lag + 2 + 200
    hs = (moving.history(j0, j0 + T, dt) + static.history(j0, j0 + T, dt)).astype(np.float32)
    hz = np.zeros((T, 4, tgt.N), np.float32)
    steps = [j0 + T - 3, j0 + T - 2, j0 + T - 1]
    out = run_library([src, tgt], c, dt, [hs, hz], j0, steps)
    N = tgt.N
    k = 2 + 5 * (2 + 5 * 2)
    A2, A1, A0 = (torch.from_numpy(np.ascontiguousarray(out[s][1][1:].reshape(-1))).to(dev) for s in steps)
    phi = torch.from_numpy(np.ascontiguousarray(out[steps[2]][1][0])).to(dev)
    E = torch.zeros(3 * N, device=dev)
    B = torch.zeros(3 * N, device=dev)
    ctx = rp.rp_create(c, dt)
    try:
        for dd in (src, tgt):
            rp.rp_add_domain(ctx, dd.origin, dd.n, dd.h)
        rp.rp_finalize(ctx)
        rp.rp_fields(ctx, 1, phi, A0, A1, A2, E, B)
        rp.rp_sync(ctx)
    finally:
        rp.rp_destroy(ctx)
    E, B = E.cpu().numpy().reshape(3, N), B.cpu().numpy().reshape(3, N)
    t = steps[2] * dt
    tr = t - d / c
    p, pd, pdd = Q * a * math.sin(omega * tr), Q * a * omega * math.cos(omega * tr), -Q * a * omega ** 2 * math.sin(omega * tr)
    Ez = -(p / d ** 3 + pd / (c * d * d) + pdd / (c * c * d))
    By = pd / (c * d * d) + pdd / (c * c * d)
    sE = Q * a * math.hypot(1 / d ** 3 - omega ** 2 / (c * c * d), omega / (c * d * d))
    sB = Q * a * math.hypot(omega ** 2 / (c * c * d), omega / (c * d * d))
    assert abs(E[2, k] - Ez) < 3e-3 * sE, (E[2, k], Ez)
    assert abs(B[1, k] - By) < 3e-3 * sB, (B[1, k], By)
