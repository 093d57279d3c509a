"""Oracle: the fields from the potentials (App. B, Eqs. B1a and B1b).

Test infrastructure, like the rest of ``oracle/``: only the tests,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU baseline call it; the
CUDA path shares nothing with it.

App. B gives the gauge-free fields from the Lorenz-gauge potentials (atomic
units):

    E = -grad v - (1/c) dA/dt,        B = curl A.

The paper works with the continuous fields; on the sampled grid this module
takes the readings below, written out plainly in FP64 numpy:

* d/dx (and y, z) at an interior node: (f[i+1] - f[i-1]) / (2h); at the first
  node (-3 f[0] + 4 f[1] - f[2]) / (2h), at the last (3 f[n-1] - 4 f[n-2] +
  f[n-3]) / (2h) -- all second order;
* d/dt at step l: (3 A_l - 4 A_{l-1} + A_{l-2}) / (2 dt), second order, or
  (A_l - A_{l-1}) / dt when A_{l-2} is not given.

Arrays are node-ordered as everywhere else: node id = x + nx (y + ny z).
"""
from __future__ import annotations

import numpy as np


def d_axis(f: np.ndarray, n, h: float, axis: int) -> np.ndarray:
    """d f / d(x, y or z) of one field f[N] on an (nx, ny, nz) grid, second
    order inside and on the faces (the reading stated above)."""
    nx, ny, nz = (int(v) for v in n)
    g = np.asarray(f, dtype=np.float64).reshape(nz, ny, nx)
    ax = {0: 2, 1: 1, 2: 0}[axis]          # x is the fastest (last) array axis
    m = g.shape[ax]
    out = np.empty_like(g)
    sl = lambda i: tuple(i if a == ax else slice(None) for a in range(3))
    for i in range(m):
        if i == 0:
            v = -3.0 * g[sl(0)] + 4.0 * g[sl(1)] - g[sl(2)]
        elif i == m - 1:
            v = 3.0 * g[sl(m - 1)] - 4.0 * g[sl(m - 2)] + g[sl(m - 3)]
        else:
            v = g[sl(i + 1)] - g[sl(i - 1)]
        out[sl(i)] = v / (2.0 * h)
    return out.reshape(-1)


def fields(phi, A, A1, A2, n, h: float, c: float, dt: float):
    """(E [3][N], B [3][N]) from phi [N] and A, A1, A2 [3][N] at steps l, l-1,
    l-2 (A2 None: first-order time difference), Eqs. B1a and B1b."""
    N = int(n[0]) * int(n[1]) * int(n[2])
    A = np.asarray(A, dtype=np.float64).reshape(3, N)
    A1 = np.asarray(A1, dtype=np.float64).reshape(3, N)
    if A2 is None:
        dAdt = (A - A1) / dt
    else:
        A2 = np.asarray(A2, dtype=np.float64).reshape(3, N)
        dAdt = (3.0 * A - 4.0 * A1 + A2) / (2.0 * dt)
    E = np.stack([-d_axis(phi, n, h, a) - dAdt[a] / c for a in range(3)])
    B = np.stack([d_axis(A[2], n, h, 1) - d_axis(A[1], n, h, 2),
                  d_axis(A[0], n, h, 2) - d_axis(A[2], n, h, 0),
                  d_axis(A[1], n, h, 0) - d_axis(A[0], n, h, 1)])
    return E, B
