"""Seeded synthetic inputs: wave-speed fields and point-like sources.

This module holds input generation only (no step of the solver's arithmetic); both the GPU
path's tests/benchmarks and the CPU oracle's tests draw their inputs from it.

Grid convention: n_a cell-centred interior nodes per axis, x_p = (p + 1/2) h on [0, n_a h];
fields are numpy arrays of shape n[::-1] (x1 fastest).  Every generator is deterministic in
its seed (numpy.random.default_rng).
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


def node_coords(n_a: int, h: float):
    return (np.arange(n_a) + 0.5) * h


def gaussian_source(n, h, centre, width, cutoff: float = 6.0):
    """Unit-mass Gaussian exp(-|x-x0|^2 / (2 w^2)) / (2 pi w^2)^(d/2), set to 0 beyond cutoff*w.

    The truncation makes the support compact, so subdomains away from the source see an exactly
    zero local source.
    """
    d = len(n)
    coords = [node_coords(n[a], h) for a in range(d)]
    grids = np.meshgrid(*coords[::-1], indexing="ij")       # grids[k] varies along x_{d-k}
    r2 = np.zeros(tuple(n[::-1]))
    for a in range(d):
        r2 = r2 + (grids[d - 1 - a] - centre[a]) ** 2
    f = np.exp(-r2 / (2.0 * width * width)) / (2.0 * math.pi * width * width) ** (d / 2.0)
    f[r2 > (cutoff * width) ** 2] = 0.0
    return f


def gaussian_source_patch(n, h, centre, width, cutoff: float = 6.0):
    """The nonzero part of gaussian_source(n, h, centre, width, cutoff): (slices into the
    n[::-1]-shaped field, values there).  Same formula on the same nodes, evaluated only inside
    the bounding box of the cutoff sphere."""
    d = len(n)
    lo, hi = [], []
    for a in range(d):
        lo.append(max(0, int(math.floor((centre[a] - cutoff * width) / h - 0.5))))
        hi.append(min(n[a], int(math.ceil((centre[a] + cutoff * width) / h - 0.5)) + 1))
    coords = [(np.arange(lo[a], hi[a]) + 0.5) * h for a in range(d)]
    grids = np.meshgrid(*coords[::-1], indexing="ij")
    r2 = np.zeros(tuple(hi[a] - lo[a] for a in range(d))[::-1])
    for a in range(d):
        r2 = r2 + (grids[d - 1 - a] - centre[a]) ** 2
    f = np.exp(-r2 / (2.0 * width * width)) / (2.0 * math.pi * width * width) ** (d / 2.0)
    f[r2 > (cutoff * width) ** 2] = 0.0
    return tuple(slice(lo[a], hi[a]) for a in range(d))[::-1], f


def uniform_centres(rng, count: int, dim: int, lo: float, hi: float):
    return rng.uniform(lo, hi, size=(count, dim))


def gaussian_sources(n, h, centres, width):
    """One Gaussian per right-hand side: array of shape (R, *n[::-1]), complex128."""
    return np.stack([gaussian_source(n, h, c, width) for c in centres]).astype(np.complex128)


def delta_sources(n, h, points):
    """Approximated delta sources (Eq. 5.4): a unit mass 1/(h1 h2) per point, spread bilinearly
    over the cell-centred nodes around the point.  All points sum into one field."""
    d = len(n)
    f = np.zeros(tuple(n[::-1]))
    for pt in points:
        idx, wts = [], []
        for a in range(d):
            s = pt[a] / h - 0.5                   # node coordinate: x_p = (p + 1/2) h
            p0 = int(math.floor(s))
            t = s - p0
            idx.append((p0, p0 + 1))
            wts.append((1.0 - t, t))
        for corner in range(1 << d):
            pos, w = [], 1.0
            for a in range(d):
                bit = (corner >> a) & 1
                pos.append(idx[a][bit])
                w *= wts[a][bit]
            if w == 0.0 or any(q < 0 or q >= n[a] for a, q in enumerate(pos)):
                continue
            f[tuple(pos[::-1])] += w / h ** d
    return f


# Table 5: subdomains of 300^2 nodes with a 30-point PML, N x N partitions, frequencies as printed
TABLE5_FREQ = {2: 65.9, 4: 126.0, 8: 246.0, 16: 486.0, 32: 966.0}
TABLE5_POINTS = [(0.25, 0.25), (0.25, 0.75), (0.75, 0.25), (0.75, 0.75)]


def medium_constant(n, c0: float = 1.0):
    return np.full(tuple(n[::-1]), c0, dtype=np.float64)


def medium_two_layer(n, h, interface: float = 0.37, c_below: float = 1.0,
                     c_above: float = 1.5, axis: int = 1):
    """Sharp two-layer medium (Eq. 3.11): c_below where x_{axis+1} < interface, else c_above."""
    d = len(n)
    x = node_coords(n[axis], h)
    shp = [1] * d
    shp[d - 1 - axis] = n[axis]
    layer = np.where(x < interface, c_below, c_above).reshape(shp)
    return np.broadcast_to(layer, tuple(n[::-1])).astype(np.float64).copy()


def medium_random(n, h, seed: int, corr_len: float = 0.1, c_min: float = 1.0,
                  c_max: float = 2.0):
    """Smooth random medium: c = c_min + (c_max - c_min) Phi(g), g a unit-variance Gaussian
    random field with Gaussian covariance of length corr_len (spectral filtering of seeded white
    noise with numpy's FFT), Phi the standard normal CDF."""
    rng = np.random.default_rng(seed)
    shape = tuple(n[::-1])
    noise = rng.standard_normal(shape)
    freqs = np.meshgrid(*[np.fft.fftfreq(s, d=h) for s in shape], indexing="ij")
    k2 = sum((2 * math.pi * f) ** 2 for f in freqs)
    filt = np.exp(-k2 * corr_len ** 2 / 4.0)
    g = np.real(np.fft.ifftn(np.fft.fftn(noise) * filt))
    g = (g - g.mean()) / g.std()
    phi = 0.5 * (1.0 + np.vectorize(math.erf)(g / math.sqrt(2.0)))
    return c_min + (c_max - c_min) * phi


# Convergence tests of Section 5.1: the computational box B_L = [0, 1]^2 holds the interior box
# (side 8/9 of it, cells 240 / 270 at the coarsest mesh) surrounded by a PML of 1/18 of the box on
# every side, partitioned 4 x 4; kappa = 50 pi below the smooth two-layer interface.
CONV_OFFSET = 1.0 / 18.0                 # interior-box origin in B_L coordinates
CONV_KAPPA_DOWN = 50.0 * math.pi
CONV_KAPPA_UP = 62.5 * math.pi
CONV_ETA, CONV_EPS = 0.65, 0.01
CONV_SOURCE = (0.28, 0.27)               # centre of Eq. (5.1)'s smooth source, B_L coordinates


def conv_mesh(total: int):
    """(interior nodes per axis, PML cells, h) of a Section 5.1 mesh of total^2 cells on B_L."""
    if total % 18:
        raise ValueError("the total mesh must be a multiple of 18 cells")
    return total * 8 // 9, total // 18, 1.0 / total


def medium_smooth_two_layer(n, h, offset: float = CONV_OFFSET):
    """Wave speed of the smooth two-layer medium of Section 5.1 for omega = kappa_down:
    kappa = kappa_down below eta, kappa_up above eta + eps, kappa_down (1 - w) + kappa_up w
    in between with w = (x2 - eta) / eps (x2 in B_L coordinates); c = kappa_down / kappa."""
    x2 = node_coords(n[1], h) + offset
    w = np.clip((x2 - CONV_ETA) / CONV_EPS, 0.0, 1.0)
    kappa = CONV_KAPPA_DOWN * (1.0 - w) + CONV_KAPPA_UP * w
    c = (CONV_KAPPA_DOWN / kappa).reshape(n[1], 1)
    return np.broadcast_to(c, (n[1], n[0])).astype(np.float64).copy()


def smooth_source(n, h, kappa: float = CONV_KAPPA_DOWN, centre=CONV_SOURCE,
                  offset: float = CONV_OFFSET, symmetric: bool = False):
    """Eq. (5.1): f = 16 kappa^2 / pi^3 exp(-(4 kappa / pi)^2 |x - r|^2) at the interior nodes
    (r in B_L coordinates); symmetric=True adds its mirror images in x1 -> 1 - x1, x2 -> 1 - x2
    and both (the four-source case)."""
    x1 = node_coords(n[0], h) + offset
    x2 = node_coords(n[1], h) + offset
    X2, X1 = np.meshgrid(x2, x1, indexing="ij")
    a = (4.0 * kappa / math.pi) ** 2
    amp = 16.0 * kappa * kappa / math.pi ** 3
    cs = [centre]
    if symmetric:
        r1, r2 = centre
        cs += [(1.0 - r1, r2), (r1, 1.0 - r2), (1.0 - r1, 1.0 - r2)]
    f = np.zeros((n[1], n[0]))
    for r1, r2 in cs:
        f += amp * np.exp(-a * ((X1 - r1) ** 2 + (X2 - r2) ** 2))
    return f


@dataclass
class Workload:
    """A named synthetic workload: problem parameters plus its seeded right-hand sides."""
    name: str
    n: tuple
    parts: tuple
    omega: float
    pml_cells: int
    pml_strength: float
    c: np.ndarray
    f: np.ndarray                      # (R, *n[::-1]) complex sources on interior nodes
    precision: str = "fp64"
    rounds: int = 1
    tol: float = 1e-6
    meta: dict = field(default_factory=dict)

    @property
    def h(self):
        return 1.0 / self.n[0]


def workload(name: str, nrhs: int | None = None) -> Workload:
    """The synthetic workloads (sizes, media and source recipes) used by tests and benchmarks.

    const2d_128   2D, 128^2 interior, h = 1/128, kappa = 2 pi 8, 2x2 subdomains, 16-cell PML,
                  one Gaussian (w = 2h) at (0.5, 0.5), direct FP64 DDM, one round.
    const2d_640   2D, 640^2, kappa = 2 pi 40, 8x8 subdomains of 80^2, 12-cell PML, 16 Gaussians
                  at seeded uniform centres, mixed precision + FGMRES to 1e-6 with two rounds of
                  sweeps per preconditioner application.
    layer2d_1024  2D two-layer (c = 1 below y = 0.37, 1.5 above), omega = 2 pi 50, 1024^2,
                  16x16 subdomains, 12-cell PML, 64 seeded Gaussians, FGMRES to 1e-6 with three
                  rounds of sweeps per preconditioner application.  One round leaves FGMRES
                  stalled near 0.25 relative residual at this size: the interface reflections
                  need the extra round of Theorem 3.10.  Two rounds converge in 3 iterations,
                  three in 2, and in the trace-operator plan a round adds only trace solves, so
                  three is the fastest (measured).
    const3d_128   3D, 128^3, kappa = 2 pi 10, 4x4x4 subdomains of 32^3, 8-cell PML, 8 Gaussians.
    table5_N      the weak-scaling series of Table 5: N x N subdomains of 300^2 nodes, 30-point
                  PML, omega / 2 pi as printed for N = 2, 4, 8, 16, 32, one right-hand side of four
                  approximated delta sources at (1/4, 1/4), (1/4, 3/4), (3/4, 1/4), (3/4, 3/4)
                  (Eq. 5.4), FGMRES to 1e-6 with one round of sweeps.
    """
    if name == "const2d_128":
        n = (128, 128)
        h = 1.0 / 128
        f = gaussian_sources(n, h, [(0.5, 0.5)], 2 * h)
        return Workload(name, n, (2, 2), 2 * math.pi * 8, 16, 30.0, medium_constant(n), f,
                        "fp64", 1, 1e-6)
    if name == "const2d_640":
        n = (640, 640)
        h = 1.0 / 640
        R = 16 if nrhs is None else nrhs
        w = 2 * h
        cen = uniform_centres(np.random.default_rng(2), R, 2, 6 * w, 1 - 6 * w)
        return Workload(name, n, (8, 8), 2 * math.pi * 40, 12, 30.0, medium_constant(n),
                        gaussian_sources(n, h, cen, w), "mixed", 2, 1e-6)
    if name == "layer2d_1024":
        n = (1024, 1024)
        h = 1.0 / 1024
        R = 64 if nrhs is None else nrhs
        w = 2 * h
        cen = uniform_centres(np.random.default_rng(3), R, 2, 6 * w, 1 - 6 * w)
        return Workload(name, n, (16, 16), 2 * math.pi * 50, 12, 30.0,
                        medium_two_layer(n, h), gaussian_sources(n, h, cen, w), "mixed", 3,
                        1e-6)
    if name == "const3d_128":
        n = (128, 128, 128)
        h = 1.0 / 128
        R = 8 if nrhs is None else nrhs
        w = 2 * h
        cen = uniform_centres(np.random.default_rng(4), R, 3, 6 * w, 1 - 6 * w)
        return Workload(name, n, (4, 4, 4), 2 * math.pi * 10, 8, 30.0, medium_constant(n),
                        gaussian_sources(n, h, cen, w), "mixed", 1, 1e-6)
    if name.startswith("table5_"):
        N = int(name.split("_")[1])
        n = (300 * N, 300 * N)
        h = 1.0 / n[0]
        f = delta_sources(n, h, TABLE5_POINTS)[None].astype(np.complex128)
        return Workload(name, n, (N, N), 2 * math.pi * TABLE5_FREQ[N], 30, 30.0,
                        medium_constant(n), f, "mixed", 1, 1e-6,
                        {"paper_freq": TABLE5_FREQ[N]})
    raise KeyError(name)
