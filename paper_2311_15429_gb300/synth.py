"""Seeded synthetic inputs: sub-domain geometry and (rho, J) time slices.

This module only makes inputs.  It holds none of the arithmetic of the
retarded sum; both the CUDA path and the FP64 oracle consume what it returns.

Stand-ins for the paper's molecular densities (Sec. IV runs C12H4 and N2
dimers in PARSEC, which cannot be run here):

* each sub-domain carries three unit-integral Gaussians g_k with widths
  sigma_k ~ U[0.5, 1.0] bohr and centres uniform over the central half of the
  box, with amplitudes A_k(t) = a_k (1 + 0.1 sin(0.3 t + phi_k)),
  a_k ~ U[0.5, 1.5], phi_k ~ U[0, 2 pi);
* the current is J = sum_k (dA_k/dt / 4 pi) grad Phi_k with
  Phi_k = erf(r / (sqrt2 sigma_k)) / r, the potential of the unit Gaussian, so
  that laplacian(Phi_k) = -4 pi g_k and the continuity equation
  d(rho)/dt + div J = 0 holds at every point (Eqs. 14a/14b of Appendix A
  define rho and j from orbitals; this is a continuity-consistent stand-in).

Slices are laid out [4][N] = (rho, Jx, Jy, Jz), x fastest within a field,
node id = x + nx*(y + ny*z), node (i,j,k) at origin + h*(i,j,k).
Geometry seed 0, source seed 1.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Sequence, Tuple

import numpy as np
from scipy.special import erf

C_AU = 137.036  # speed of light in atomic units
GEOMETRY_SEED = 0
SOURCE_SEED = 1


@dataclass(frozen=True)
class Domain:
    origin: Tuple[float, float, float]
    n: Tuple[int, int, int]
    h: float

    @property
    def N(self) -> int:
        return int(self.n[0] * self.n[1] * self.n[2])

    @property
    def center(self) -> np.ndarray:
        return np.asarray(self.origin) + self.h * (np.asarray(self.n) - 1) / 2.0

    def coords(self) -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
        """Node coordinates, each of shape [N] in node-id order (x fastest)."""
        nx, ny, nz = self.n
        z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
        ox, oy, oz = self.origin
        return (ox + self.h * x.reshape(-1), oy + self.h * y.reshape(-1),
                oz + self.h * z.reshape(-1))


def cubic(center: Sequence[float], n: int, h: float) -> Domain:
    """A cubic grid of n^3 nodes with spacing h centred on ``center``."""
    half = h * (n - 1) / 2.0
    return Domain(tuple(float(c) - half for c in center), (n, n, n), float(h))


def _unit_gaussian(r2: np.ndarray, sigma: float) -> np.ndarray:
    return np.exp(-r2 / (2.0 * sigma * sigma)) / (2.0 * math.pi * sigma * sigma) ** 1.5


def _grad_gaussian_potential(dx, dy, dz, sigma: float):
    """grad of Phi(r) = erf(r/(sqrt2 sigma))/r, the potential of a unit Gaussian."""
    r = np.sqrt(dx * dx + dy * dy + dz * dz)
    s2 = math.sqrt(2.0) * sigma
    small = r < 1e-6 * sigma
    rs = np.where(small, 1.0, r)
    dphidr = (math.sqrt(2.0 / math.pi) / sigma * np.exp(-rs * rs / (2 * sigma * sigma)) * rs
              - erf(rs / s2)) / (rs * rs)
    # series near the centre: dPhi/dr = -sqrt(2/pi) r / (3 sigma^3)
    dphidr = np.where(small, -math.sqrt(2.0 / math.pi) * r / (3.0 * sigma ** 3), dphidr)
    over_r = np.where(small, 0.0, dphidr / rs)
    return dx * over_r, dy * over_r, dz * over_r


class GaussianSources:
    """rho = sum_k A_k(t) g_k(r);  J = sum_k (dA_k/dt)/(4 pi) grad Phi_k(r).

    Precomputes g_k and grad Phi_k per node so that any time slice costs one
    small matrix product.
    """

    def __init__(self, dom: Domain, sigma, centres, a, phase, omega: float = 0.3,
                 depth: float = 0.1):
        self.dom = dom
        self.sigma = np.asarray(sigma, dtype=np.float64)
        self.centres = np.asarray(centres, dtype=np.float64).reshape(-1, 3)
        self.a = np.asarray(a, dtype=np.float64)
        self.phase = np.asarray(phase, dtype=np.float64)
        self.omega = float(omega)
        self.depth = float(depth)
        x, y, z = dom.coords()
        K = self.sigma.size
        self.g = np.empty((K, dom.N))
        self.gradphi = np.empty((K, 3, dom.N))
        for k in range(K):
            dx, dy, dz = x - self.centres[k, 0], y - self.centres[k, 1], z - self.centres[k, 2]
            self.g[k] = _unit_gaussian(dx * dx + dy * dy + dz * dz, self.sigma[k])
            gx, gy, gz = _grad_gaussian_potential(dx, dy, dz, self.sigma[k])
            self.gradphi[k, 0], self.gradphi[k, 1], self.gradphi[k, 2] = gx, gy, gz

    def amplitudes(self, t: float):
        arg = self.omega * t + self.phase
        A = self.a * (1.0 + self.depth * np.sin(arg))
        dA = self.a * self.depth * self.omega * np.cos(arg)
        return A, dA

    def slice64(self, t: float) -> np.ndarray:
        A, dA = self.amplitudes(t)
        out = np.empty((4, self.dom.N))
        out[0] = A @ self.g
        out[1:] = np.einsum("k,kfn->fn", dA / (4.0 * math.pi), self.gradphi)
        return out

    def slice(self, t: float, dtype=np.float32) -> np.ndarray:
        return self.slice64(t).astype(dtype)

    def history(self, j0: int, j1: int, dt: float, dtype=np.float32) -> np.ndarray:
        """Samples at t_j = j*dt for j0 <= j < j1, shape [j1-j0][4][N]."""
        out = np.empty((j1 - j0, 4, self.dom.N), dtype=dtype)
        for i, j in enumerate(range(j0, j1)):
            out[i] = self.slice(j * dt, dtype)
        return out


def random_gaussians(dom: Domain, rng: np.random.Generator, count: int = 3,
                     omega: float = 0.3) -> GaussianSources:
    lo = np.asarray(dom.origin) + 0.25 * dom.h * (np.asarray(dom.n) - 1)
    hi = np.asarray(dom.origin) + 0.75 * dom.h * (np.asarray(dom.n) - 1)
    sigma = rng.uniform(0.5, 1.0, count)
    centres = rng.uniform(lo, hi, (count, 3))
    a = rng.uniform(0.5, 1.5, count)
    phase = rng.uniform(0.0, 2.0 * math.pi, count)
    return GaussianSources(dom, sigma, centres, a, phase, omega=omega)


class MovingGaussian:
    """rho = Q g(r - d(t)), J = rho * d'(t), d(t) = amp sin(omega t) * axis.

    Compact and continuity-consistent (d rho/dt = -div(rho d')) -- the input
    for the Lorenz-gauge check.
    """

    def __init__(self, dom: Domain, centre, sigma: float, amp: float, omega: float,
                 axis=(1.0, 0.0, 0.0), charge: float = 1.0):
        self.dom, self.sigma, self.amp, self.omega, self.q = dom, sigma, amp, omega, charge
        self.centre = np.asarray(centre, dtype=np.float64)
        self.axis = np.asarray(axis, dtype=np.float64) / np.linalg.norm(axis)
        self.x, self.y, self.z = dom.coords()

    def slice64(self, t: float) -> np.ndarray:
        d = self.centre + self.amp * math.sin(self.omega * t) * self.axis
        v = self.amp * self.omega * math.cos(self.omega * t) * self.axis
        dx, dy, dz = self.x - d[0], self.y - d[1], self.z - d[2]
        rho = self.q * _unit_gaussian(dx * dx + dy * dy + dz * dz, self.sigma)
        return np.stack([rho, rho * v[0], rho * v[1], rho * v[2]])

    def history(self, j0: int, j1: int, dt: float, dtype=np.float64) -> np.ndarray:
        return np.stack([self.slice64(j * dt).astype(dtype) for j in range(j0, j1)])


class BreathingGaussian:
    """rho = Q g(r) (1 + eps sin(omega t + phi0)), J = 0.

    Only phi is used from this source (the retarded phase of a monopole).
    """

    def __init__(self, dom: Domain, centre, sigma: float, eps: float, omega: float,
                 phi0: float = 0.0, charge: float = 1.0):
        self.dom, self.sigma, self.eps, self.omega, self.phi0, self.q = \
            dom, sigma, eps, omega, phi0, charge
        x, y, z = dom.coords()
        c = np.asarray(centre, dtype=np.float64)
        self.g = _unit_gaussian((x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2, sigma)

    def amplitude(self, t):
        return self.q * (1.0 + self.eps * np.sin(self.omega * np.asarray(t) + self.phi0))

    def history(self, j0: int, j1: int, dt: float, dtype=np.float64) -> np.ndarray:
        out = np.zeros((j1 - j0, 4, self.dom.N), dtype=dtype)
        for i, j in enumerate(range(j0, j1)):
            out[i, 0] = (self.amplitude(j * dt) * self.g).astype(dtype)
        return out


# ----------------------------------------------------------------------------
# Workloads shaped like the five configurations of the method's evaluation
# ----------------------------------------------------------------------------

@dataclass
class Workload:
    name: str
    domains: List[Domain]
    c: float
    dt: float
    history: int           # samples the harness keeps before the first evaluated step
    steps: int             # evaluated steps
    description: str = ""
    sources: List[GaussianSources] = field(default_factory=list)

    @property
    def points(self) -> int:
        return sum(d.N for d in self.domains)


def seeded_sources(domains: Sequence[Domain], seed: int = SOURCE_SEED) -> List[GaussianSources]:
    """Three random Gaussians per domain (``random_gaussians``), each domain
    drawing from its own child of one seed sequence."""
    ss = np.random.SeedSequence(seed)
    return [random_gaussians(d, np.random.default_rng(s))
            for d, s in zip(domains, ss.spawn(len(domains)))]


def _scatter_centres(count: int, side: float, min_sep: float, rng, max_tries: int = 1_000_000) -> np.ndarray:
    pts: List[np.ndarray] = []
    tries = 0
    while len(pts) < count:
        tries += 1
        if tries > max_tries:
            raise ValueError(f"cannot place {count} centres {min_sep} apart in a cube of side {side}")
        p = rng.uniform(-side / 2, side / 2, 3)
        if all(np.linalg.norm(p - q) >= min_sep for q in pts):
            pts.append(p)
    return np.asarray(pts)


def scattered(name: str, count: int, n: int, h: float, side: float, min_sep: float, seed: int = GEOMETRY_SEED,
              description: str = "") -> Workload:
    """``count`` cubic n^3 domains whose centres are drawn uniformly in a cube
    of the given side with a minimum separation (seeded), with seeded sources."""
    cs = _scatter_centres(count, side, min_sep, np.random.default_rng(seed))
    doms = [cubic(c, n, h) for c in cs]
    return Workload(name, doms, C_AU, 0.05, 0, 100, description, seeded_sources(doms))


def two_domain(n: int, h: float, distance: float, name: str = "custom", steps: int = 8,
               c: float = C_AU, dt: float = 0.05, history: int = 0,
               offset=(0.0, 0.0)) -> Workload:
    """Two cubic n^3 domains whose centres lie ``distance`` apart along x."""
    doms = [cubic((-distance / 2, 0.0, 0.0), n, h),
            cubic((distance / 2, offset[0], offset[1]), n, h)]
    return Workload(name, doms, c, dt, history, steps,
                    f"2 x {n}^3, h={h}, {distance} bohr apart", seeded_sources(doms))


@dataclass
class SplitGeometry:
    """Two elongated sub-domains of W' x W' x L' nodes whose outer faces are
    d' nodes apart along x (the gap between them is d' - 2W'), and the single
    domain of d' x W' x L' nodes that encloses both (Sec. III's comparison of a
    multi-domain and a single large domain, Eq. 13).  The enclosing domain's
    nodes include every node of both sub-domains."""
    W: int
    L: int
    d: int
    h: float
    subs: List[Domain]
    enclosing: Domain
    sources: List[GaussianSources]

    def embed(self, slices: Sequence[np.ndarray]) -> np.ndarray:
        """The enclosing domain's slice [..., 4, N]: each sub-domain's slice
        (shape [..., 4, N_sub]) at its own nodes, zero elsewhere."""
        lead = slices[0].shape[:-2]
        W, L, d = self.W, self.L, self.d
        out = np.zeros(lead + (4, L, W, d), dtype=slices[0].dtype)
        for k, sl in enumerate(slices):
            x0 = 0 if k == 0 else d - W
            out[..., x0:x0 + W] = sl.reshape(lead + (4, L, W, W))
        return out.reshape(lead + (4, L * W * d))

    def sub_nodes(self, k: int) -> np.ndarray:
        """Node ids, in the enclosing domain, of sub-domain k's nodes (in its
        own node order)."""
        W, L, d = self.W, self.L, self.d
        x0 = 0 if k == 0 else d - W
        z, y, x = np.meshgrid(np.arange(L), np.arange(W), np.arange(W), indexing="ij")
        return ((x + x0) + d * (y + W * z)).reshape(-1)


def split_geometry(W: int, L: int, d: int, h: float, seed: int = SOURCE_SEED) -> SplitGeometry:
    """Sub-domains of W x W x L nodes (x, y, z) at x-node offsets 0 and d - W
    of a d x W x L enclosing domain; three seeded Gaussians in each."""
    if not 2 * W <= d:
        raise ValueError("the sub-domains must not overlap: need 2W <= d")
    subs = [Domain((0.0, 0.0, 0.0), (W, W, L), h), Domain((h * (d - W), 0.0, 0.0), (W, W, L), h)]
    enclosing = Domain((0.0, 0.0, 0.0), (d, W, L), h)
    return SplitGeometry(W, L, d, h, subs, enclosing, seeded_sources(subs, seed))


def workload(name: str) -> Workload:
    """The named synthetic workload.

    cfg1  2 x 16^3, h=0.3, 20 bohr apart on x, 64-step history, last 8 steps out
    cfg2  2 x 48^3, h=0.25, 2000 bohr apart (delay ~292 steps), 320-step ring, 100 steps
    cfg3  8 x 64^3, h=0.25, centres in a 20000 bohr cube, min separation 100, 200 steps
    cfg4  64 domains, n from {24,32,48,64,96}, h in [0.2,0.35], cube side 20000/sqrt3,
          min separation 50, 500 steps
    cfg5  32 x 48^3, h=0.25, cube side 50000/sqrt3, min separation 500, 1000 steps
    """
    rng = np.random.default_rng(GEOMETRY_SEED)
    if name == "cfg1":
        w = two_domain(16, 0.3, 20.0, "cfg1", steps=8, history=56)
        w.description = "2 x 16^3, h=0.3 bohr, centres 20 bohr apart on x, 64-step history"
        return w
    if name == "cfg2":
        w = two_domain(48, 0.25, 2000.0, "cfg2", steps=100, history=320)
        w.description = ("2 x 48^3, h=0.25 bohr, centres 2000 bohr apart on x, "
                         "320-step ring, 100 steps")
        return w
    if name == "cfg3":
        cs = _scatter_centres(8, 20000.0, 100.0, rng)
        doms = [cubic(c, 64, 0.25) for c in cs]
        return Workload("cfg3", doms, C_AU, 0.05, 0, 200,
                        "8 x 64^3, h=0.25, 20000 bohr cube, min separation 100", seeded_sources(doms))
    if name == "cfg4":
        cs = _scatter_centres(64, 20000.0 / math.sqrt(3.0), 50.0, rng)
        ns = rng.choice([24, 32, 48, 64, 96], 64)
        hs = rng.uniform(0.2, 0.35, 64)
        doms = [cubic(c, int(n), float(h)) for c, n, h in zip(cs, ns, hs)]
        return Workload("cfg4", doms, C_AU, 0.05, 0, 500,
                        "64 mixed domains, n in {24..96}^3, h in [0.2,0.35]", seeded_sources(doms))
    if name == "cfg5":
        cs = _scatter_centres(32, 50000.0 / math.sqrt(3.0), 500.0, rng)
        doms = [cubic(c, 48, 0.25) for c in cs]
        return Workload("cfg5", doms, C_AU, 0.05, 0, 1000,
                        "32 x 48^3, 500-50000 bohr apart", seeded_sources(doms))
    raise KeyError(name)


class DeviceSlices:
    """The same slices as ``GaussianSources.slice``, made on a CUDA device:
    the per-node basis (g_k and grad Phi_k) is uploaded once as float32 and a
    slice is one small contraction with the amplitudes at t, so that histories
    thousands of steps deep need not pass through host memory."""

    def __init__(self, sources: Sequence[GaussianSources], device):
        import torch
        self.torch = torch
        self.sources = list(sources)
        self.device = device
        self.basis = []
        for s in self.sources:
            b = np.concatenate([s.g[:, None, :], s.gradphi], axis=1)        # [K][4][N]
            self.basis.append(torch.from_numpy(b.astype(np.float32)).to(device))
        same = len({(s.dom.N, s.sigma.size) for s in self.sources}) == 1
        self.stacked = torch.stack(self.basis) if same else None          # [D][K][4][N]

    def _weights(self, d: int, t: float):
        A, dA = self.sources[d].amplitudes(t)
        return np.concatenate([A[:, None], np.repeat((dA / (4.0 * math.pi))[:, None], 3, axis=1)], axis=1)

    def slice(self, d: int, t: float):
        """[4][N] float32 device tensor of domain d at time t."""
        wt = self.torch.from_numpy(self._weights(d, t).astype(np.float32)).to(self.device)   # [K][4]
        return (wt[:, :, None] * self.basis[d]).sum(0)

    def step(self, j: int, dt: float):
        """(rho list, J list) of every domain at t = j dt."""
        if self.stacked is not None:
            w = np.stack([self._weights(d, j * dt) for d in range(len(self.sources))])      # [D][K][4]
            wt = self.torch.from_numpy(w.astype(np.float32)).to(self.device)
            x = (wt[:, :, :, None] * self.stacked).sum(1)                                   # [D][4][N]
            return [x[d, 0] for d in range(x.shape[0])], [x[d, 1:].reshape(-1) for d in range(x.shape[0])]
        rho, J = [], []
        for d in range(len(self.sources)):
            x = self.slice(d, j * dt)
            rho.append(x[0].contiguous())
            J.append(x[1:].reshape(-1).contiguous())
        return rho, J
