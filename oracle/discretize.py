"""Discretisation of the PML problem: Eq. 2.1 (profile), Eq. 2.3 / 4.1 (PML equation), Eq. 2.8.

Test infrastructure only (see the package docstring).

Grid convention (the paper leaves it open; Section 5 only names 5/7-point second-order FD):
  * cell-centred nodes x_p = (p + 1/2) h, p = 0..n_a-1, on the physical box [0, n_a h] per axis;
  * E = H + P extra nodes per side: H un-stretched halo lines, then P PML lines;
  * homogeneous Dirichlet just outside the last extended node.
Arrays over a grid are numpy arrays of shape (G_{n-1}, ..., G_0): axis x1 is the fastest
(last numpy dimension).  ``axis a`` below always means the paper's x_{a+1}.

Operator (J-scaled form of Eq. 2.3 / 4.1, multiplied through by J = prod_b alpha_b so that the
matrix is complex symmetric; the sign convention is L = Delta + kappa^2 as in Section 2.1):
  (A u)_p = sum_a (prod_{b != a} alpha_b(p)) / h^2 *
                [ (u_{p+e_a} - u_p) / alpha_a(p + e_a/2) - (u_p - u_{p-e_a}) / alpha_a(p - e_a/2) ]
            + kappa(p)^2 * J(p) * u_p,
and the discrete PML problem is A u = J f.  alpha_a = 1 + i sigma_a is evaluated at nodes and
at half points.
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp


@dataclass
class Problem:
    """One Helmholtz PML problem on a checkerboard partition (Section 2.3 / Section 4).

    n            interior nodes per axis (x1, x2[, x3]); the physical box is [0, n_a h].
    h            mesh width.
    omega        angular frequency; kappa = omega / c (Section 1).
    c            wave speed at the interior nodes, shape n[::-1].
    parts        N1, N2[, N3] subdomains per axis (Section 2.3); n_a % N_a == 0.
    pml_cells    P, PML thickness in cells.
    pml_strength S, profile sigma(t) = S ((t - H h)/(P h))^power beyond the halo.
    pml_power    profile exponent (2 = quadratic).
    halo         H, un-stretched lines between a box edge and its PML (overlap, Section 1).
    """

    n: tuple
    h: float
    omega: float
    c: np.ndarray
    parts: tuple
    pml_cells: int
    pml_strength: float
    pml_power: int = 2
    halo: int = 0
    _cache: dict = field(default_factory=dict, repr=False, compare=False)

    def __post_init__(self):
        self.n = tuple(int(v) for v in self.n)
        self.parts = tuple(int(v) for v in self.parts)
        self.c = np.asarray(self.c, dtype=np.float64)
        if len(self.n) not in (2, 3) or len(self.parts) != len(self.n):
            raise ValueError("dimension must be 2 or 3 with one part count per axis")
        if self.c.shape != self.n[::-1]:
            raise ValueError(f"c must have shape {self.n[::-1]}, got {self.c.shape}")
        for na, Na in zip(self.n, self.parts):
            if na % Na:
                raise ValueError("n must be divisible by parts on every axis")

    @property
    def dim(self) -> int:
        return len(self.n)

    @property
    def E(self) -> int:
        return self.halo + self.pml_cells

    @property
    def m(self) -> tuple:
        """Own nodes per subdomain per axis."""
        return tuple(na // Na for na, Na in zip(self.n, self.parts))

    @property
    def M(self) -> tuple:
        """Extended local grid size per axis (own nodes plus E on each side)."""
        return tuple(ma + 2 * self.E for ma in self.m)

    @property
    def G(self) -> tuple:
        """Global extended grid size per axis."""
        return tuple(na + 2 * self.E for na in self.n)

    def subdomains(self):
        """All subdomain multi-indices (0-based, axis order x1, x2[, x3])."""
        return [tuple(int(v) for v in idx[::-1])
                for idx in np.ndindex(*self.parts[::-1])]


def sigma_profile(t, prob: Problem):
    """Eq. 2.1 with the profile sigma_hat left open by the paper (reading: power law).

    t is the distance beyond the box edge.  sigma = 0 inside the box and in the H halo lines;
    beyond them sigma = S ((t - H h) / (P h))^power.
    """
    t = np.asarray(t, dtype=np.float64)
    start = prob.halo * prob.h
    width = prob.pml_cells * prob.h
    s = np.zeros_like(t)
    beyond = t > start
    s[beyond] = prob.pml_strength * ((t[beyond] - start) / width) ** prob.pml_power
    return s


def _axis_alpha(prob: Problem, x_first: float, count: int, lo: float, hi: float):
    """alpha = 1 + i sigma on one axis of an extended grid (Eq. 2.1-2.2).

    Node p sits at x_first + p h; half point q (q = 0..count) sits at x_first + (q - 1/2) h,
    i.e. half point q lies between nodes q-1 and q.  The box on this axis is [lo, hi].
    """
    h = prob.h
    xn = x_first + h * np.arange(count)
    xh = x_first + h * (np.arange(count + 1) - 0.5)

    def dist(x):
        return np.maximum(np.maximum(lo - x, x - hi), 0.0)

    # round away the last bits of the coordinate arithmetic so that sigma is exactly 0 on edges
    an = 1.0 + 1j * sigma_profile(np.round(dist(xn) / h, 9) * h, prob)
    ah = 1.0 + 1j * sigma_profile(np.round(dist(xh) / h, 9) * h, prob)
    return an, ah


def global_axes(prob: Problem):
    """Per-axis (alpha at nodes, alpha at half points) of the global extended grid."""
    out = []
    for a in range(prob.dim):
        x_first = (-prob.E + 0.5) * prob.h
        out.append(_axis_alpha(prob, x_first, prob.G[a], 0.0, prob.n[a] * prob.h))
    return out


def local_axes(prob: Problem, sub):
    """Per-axis alphas of the extended subdomain sub (own box [k m h, (k+1) m h] per axis).

    Local node l on axis a is global extended node k_a m_a + l.  The subdomain PML is measured
    from the subdomain's own box with the same profile as the global PML (reading of the
    uniaxial PML of the proof of Lemma 2.3), so on exterior sides it equals the global PML.
    """
    out = []
    for a in range(prob.dim):
        k, m = sub[a], prob.m[a]
        x_first = (k * m - prob.E + 0.5) * prob.h
        out.append(_axis_alpha(prob, x_first, prob.M[a], k * m * prob.h, (k + 1) * m * prob.h))
    return out


def kappa_interior(prob: Problem):
    return prob.omega / prob.c


def kappa_global(prob: Problem):
    """kappa on the global extended grid: kappa at the nearest interior node (clamp)."""
    kin = kappa_interior(prob)
    idx = [np.clip(np.arange(prob.G[a]) - prob.E, 0, prob.n[a] - 1) for a in range(prob.dim)]
    return kin[np.ix_(*idx[::-1])]


def kappa_local(prob: Problem, sub):
    """Eq. 2.8: kappa_{ij}(x) = kappa(x') with x' the nearest point of the own box Omega_ij.

    Discretely: the value at the nearest own interior node (clamp of the node index into the
    own range on every axis).
    """
    kin = kappa_interior(prob)
    idx = []
    for a in range(prob.dim):
        k, m = sub[a], prob.m[a]
        g_int = k * m + np.arange(prob.M[a]) - prob.E
        idx.append(np.clip(g_int, k * m, (k + 1) * m - 1))
    return kin[np.ix_(*idx[::-1])]


def _grid_product(vecs, shape_dims):
    """Outer product of per-axis vectors laid out as (x_{n-1}, ..., x_0)."""
    n = len(vecs)
    out = np.ones(shape_dims, dtype=np.complex128)
    for a, v in enumerate(vecs):
        shp = [1] * n
        shp[n - 1 - a] = v.shape[0]
        out = out * v.reshape(shp)
    return out


def assemble(axes, kappa, h):
    """Assemble the J-scaled operator A and J on one extended grid (Eq. 2.3 / 4.1).

    axes   list over a of (alpha at nodes [G_a], alpha at half points [G_a + 1])
    kappa  wave number on the grid, shape (G_{n-1}, ..., G_0)
    Returns (A as scipy CSR, J as a grid-shaped array).
    """
    n = len(axes)
    dims = tuple(ax[0].shape[0] for ax in axes)[::-1]
    J = _grid_product([ax[0] for ax in axes], dims)
    N = int(np.prod(dims))
    lin = np.arange(N).reshape(dims)
    rows, cols, vals = [], [], []
    diag = kappa.astype(np.complex128) ** 2 * J
    for a in range(n):
        ax_dim = n - 1 - a
        Ga = dims[ax_dim]
        tang = [axes[b][0] if b != a else np.ones(Ga, dtype=np.complex128) for b in range(n)]
        T = _grid_product(tang, dims) / h ** 2            # prod_{b != a} alpha_b / h^2
        ah = axes[a][1]
        shp = [1] * n
        shp[ax_dim] = Ga
        inv_lo = (1.0 / ah[:-1]).reshape(shp)              # half point p - 1/2
        inv_hi = (1.0 / ah[1:]).reshape(shp)               # half point p + 1/2
        diag = diag - T * (inv_lo + inv_hi)
        # coupling p <-> p + e_a through half point p + 1/2
        sl_lo = [slice(None)] * n
        sl_hi = [slice(None)] * n
        sl_lo[ax_dim] = slice(0, Ga - 1)
        sl_hi[ax_dim] = slice(1, Ga)
        coup = (T * inv_hi)[tuple(sl_lo)]
        i0 = lin[tuple(sl_lo)].ravel()
        i1 = lin[tuple(sl_hi)].ravel()
        rows += [i0, i1]
        cols += [i1, i0]
        vals += [coup.ravel(), coup.ravel()]
    rows.append(lin.ravel())
    cols.append(lin.ravel())
    vals.append(diag.ravel())
    A = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(N, N))
    return A, J


def assemble_global(prob: Problem):
    """Global J-scaled PML operator and J on the global extended grid."""
    key = ("global",)
    if key not in prob._cache:
        prob._cache[key] = assemble(global_axes(prob), kappa_global(prob), prob.h)
    return prob._cache[key]


def assemble_local(prob: Problem, sub):
    """Operator, J and per-axis alphas of the extended subdomain problem P_{Omega_ij, kappa_ij}."""
    axes = local_axes(prob, sub)
    A, J = assemble(axes, kappa_local(prob, sub), prob.h)
    return A, J, axes


def extend_interior(prob: Problem, f_int):
    """Place an interior-node field (shape n[::-1] or (R, *n[::-1])) on the extended grid."""
    f_int = np.asarray(f_int)
    lead = f_int.shape[:-prob.dim]
    out = np.zeros(lead + prob.G[::-1], dtype=np.complex128)
    sl = tuple(slice(prob.E, prob.E + na) for na in prob.n[::-1])
    out[(Ellipsis,) + sl] = f_int
    return out


def interior_view(prob: Problem, u_ext):
    sl = tuple(slice(prob.E, prob.E + na) for na in prob.n[::-1])
    return np.asarray(u_ext)[(Ellipsis,) + sl]


def rhs_from_source(prob: Problem, f_ext):
    """Right-hand side of the J-scaled system: b = J f (J = 1 in the physical box)."""
    _, J = assemble_global(prob)
    return J * f_ext


def own_ranges(prob: Problem, sub):
    """Owned nodes of subdomain sub, per axis, as (global extended range, local range).

    Own nodes are the nodes of Omega_ij (cut-off mu_ij = 1).  Interfaces lie on half points,
    so no node carries the value 1/2 of the discontinuous cut-off (Section 2.2).  Exterior
    sides are not cut (mu^(1)_{-1;1} = 1 etc., Section 2.3), so the global PML nodes beyond an
    exterior side belong to the boundary subdomain.
    """
    out = []
    for a in range(prob.dim):
        k, m, E, Na = sub[a], prob.m[a], prob.E, prob.parts[a]
        lo = 0 if k == 0 else E
        hi = prob.M[a] if k == Na - 1 else E + m
        out.append(((k * m + lo, k * m + hi), (lo, hi)))
    return out
