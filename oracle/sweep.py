"""Algorithm 2.1 (2D) and Algorithm 4.1 (3D): trace-transfer diagonal sweeping DDM.

Test infrastructure only (see the package docstring).

Discrete reading of the trace potential (the paper only says the line integrals are
"discretized as solutions to the subdomain problem with particular sources", Section 2.3):

  * the interface between Omega_i and its neighbour lies on the half point between the last own
    line of one and the first own line of the other;
  * a trace held by a receiver R on its side D is a pair of lines (a, b): a on R's *outer* line
    (the neighbour's last own line), b on R's *inner* line (R's first own line);
  * the potential of the trace (Eq. 2.5 with the subdomain Green's function, Lemma 2.3) is the
    local solve with the commutator source [A_R, chi_H] t, chi_H the indicator of R's side:
        rhs[outer] += c * b,      rhs[inner] -= c * a,
    where c = prod_{b != axis} alpha_b / h^2 is the coupling of the two lines in A_R (the
    normal alpha is 1 on the interface).  This makes A_R^{-1}[A_R, chi_H] t = chi_H t -
    A_R^{-1} chi_H A_R t, the discrete form of Lemma 2.2; the unit normal of the continuous
    formula is absorbed into the commutator.
  * all potentials and the own source go into one right-hand side and one solve (Section 2.3);
  * the outgoing trace on side D of a solved subdomain X is (x[inner_D] - b_in_D, x[outer_D]),
    where b_in_D is the b-line of the trace X itself received on side D in this sweep.  The
    subtraction is the discrete form of the one-sided-limit convention after Lemma 2.2: the
    field that came in through D has no limit on the far side of D and must not be sent back.
  * u_DDM = sum over sweeps of x on the owned nodes (mu_ij = indicator of Omega_ij, exterior
    sides not cut).
"""

from __future__ import annotations

import hashlib
from concurrent.futures import ThreadPoolExecutor
from itertools import product

import numpy as np

from .discretize import Problem, assemble_local, kappa_local, local_axes, own_ranges
from .linsolve import factor


# --------------------------------------------------------------------------------------------
# Sweep order, step sets and routing
# --------------------------------------------------------------------------------------------

def sweep_directions(dim: int):
    """Sweep order of Eq. 2.9 (2D) and Eq. 4.2 (3D); x1 flips fastest, then x2, then x3."""
    if dim == 2:
        return [(+1, +1), (-1, +1), (+1, -1), (-1, -1)]
    if dim == 3:
        return [(+1, +1, +1), (-1, +1, +1), (+1, -1, +1), (-1, -1, +1),
                (+1, +1, -1), (-1, +1, -1), (+1, -1, -1), (-1, -1, -1)]
    raise ValueError(dim)


def num_steps(parts) -> int:
    """Steps per sweep: N1 + N2 - 1 in 2D, N1 + N2 + N3 - 2 in 3D (Sections 2.3 and 4)."""
    return sum(parts) - len(parts) + 1


def step_index(sub, d, parts) -> int:
    """Eq. 2.10-2.11 / 4.3-4.4 with 0-based indices: s = sum_a hat_a(k_a) + 1."""
    s = 1
    for k, da, Na in zip(sub, d, parts):
        s += k if da == 1 else Na - 1 - k
    return s


def step_set(d, s: int, parts):
    """Subdomains solved in step s of the sweep with direction d, in lexicographic order."""
    out = []
    for idx in product(*[range(Na) for Na in parts]):
        if step_index(idx, d, parts) == s:
            out.append(tuple(idx))
    return out


def similar_direction(v1, v2) -> bool:
    """Similar direction: v1.v2 > 0 (2D, Section 2.3); in 3D also v1(k) v2(k) >= 0 for all k
    (Section 4)."""
    dot = sum(a * b for a, b in zip(v1, v2))
    if len(v1) == 2:
        return dot > 0
    return dot > 0 and all(a * b >= 0 for a, b in zip(v1, v2))


def _opposite_rule(D, d_gen, d_use) -> bool:
    """True if a trace of direction D made in sweep d_gen is barred from a later sweep d_use.

    2D, Rule 2.5: the two sweeps have opposite directions.
    3D, Rule 4.2: under some coordinate-plane projection the trace direction has exactly one
    zero component and the projections of the two sweep directions are opposite.
    """
    if len(D) == 2:
        return all(a == -b for a, b in zip(d_gen, d_use))
    for p, q in ((0, 1), (0, 2), (1, 2)):
        proj = (D[p], D[q])
        if sum(1 for v in proj if v == 0) != 1:
            continue
        if d_gen[p] == -d_use[p] and d_gen[q] == -d_use[q]:
            return True
    return False


def sweep_usable(D, l_gen: int, l_use: int, dirs) -> bool:
    """May a trace of direction D generated in sweep l_gen be used in sweep l_use >= l_gen?

    Rule 2.4 / 4.1 (similar directions) and Rule 2.5 / 4.2 (opposite directions).  Sweeps are
    numbered over the whole list of rounds; sweep l has direction dirs[l % len(dirs)].
    """
    d_gen = dirs[l_gen % len(dirs)]
    d_use = dirs[l_use % len(dirs)]
    if not similar_direction(D, d_use):
        return False
    if l_use > l_gen and _opposite_rule(D, d_gen, d_use):
        return False
    return True


def route(D, l_gen: int, n_sweeps: int, dirs):
    """Smallest sweep l' >= l_gen in which the trace may be used, or None (dropped)."""
    for lp in range(l_gen, n_sweeps):
        if sweep_usable(D, l_gen, lp, dirs):
            return lp
    return None


def sides(dim: int):
    """The 2n cardinal directions as (axis, sign); axis 0 is x1."""
    return [(a, s) for a in range(dim) for s in (+1, -1)]


def side_vector(side, dim):
    a, s = side
    v = [0] * dim
    v[a] = s
    return tuple(v)


def strip_sweeps(parts, nsweeps: int):
    """Sweep list of the one-dimensional sweeping DDM for a strip partition (Section 3.2): only
    one axis a has N_a > 1, and the sweeps run along it alternately forward (+) and backward
    (-), starting forward.  nsweeps = 2 is the forward/backward pair, the degenerate form of
    Algorithm 2.1 on a strip; nsweeps = 3 adds the extra forward sweep of Theorem 3.6.  The
    other components of every direction are +1 (no neighbours lie along them)."""
    axes = [a for a, Na in enumerate(parts) if Na > 1]
    if len(axes) > 1:
        raise ValueError("strip sweeps need a partition with one axis of more than 1 part")
    if nsweeps < 1:
        raise ValueError("nsweeps must be >= 1")
    a = axes[0] if axes else len(parts) - 1
    out = []
    for k in range(nsweeps):
        v = [1] * len(parts)
        v[a] = 1 if k % 2 == 0 else -1
        out.append(tuple(v))
    return out


def route_table(dim: int, rounds: int = 1):
    """route[l][side] over all 2^n * rounds sweeps (None = dropped), generated from the Rules."""
    dirs = sweep_directions(dim)
    L = len(dirs) * rounds
    return [{sd: route(side_vector(sd, dim), l, L, dirs) for sd in sides(dim)} for l in range(L)]


# --------------------------------------------------------------------------------------------
# Algorithm 2.1 / 4.1
# --------------------------------------------------------------------------------------------

class LocalProblems:
    """Extended subdomain operators P_{Omega_ij, kappa_ij}, factored once and shared between
    subdomains whose extended wave number fields are identical (all alphas are translation
    invariant, so kappa_ij determines the operator)."""

    def __init__(self, prob: Problem):
        self.prob = prob
        self.factors = {}
        self.key_of = {}
        self.axes = {}
        for sub in prob.subdomains():
            kap = kappa_local(prob, sub)
            key = hashlib.sha1(np.ascontiguousarray(kap).tobytes()).hexdigest()
            self.key_of[sub] = key
            if key not in self.factors:
                A, _, _ = assemble_local(prob, sub)
                self.factors[key] = factor(A, prob.M[::-1])
            self.axes[sub] = local_axes(prob, sub)

    def solve(self, sub, rhs):
        """Solve A_R x = rhs for a batch of right-hand sides of shape (R, *M[::-1])."""
        R = rhs.shape[0]
        B = rhs.reshape(R, -1).T
        X = self.factors[self.key_of[sub]].solve(np.ascontiguousarray(B))
        return np.asarray(X).T.reshape(rhs.shape)

    @property
    def n_distinct(self):
        return len(self.factors)


def _line_index(prob: Problem, side, which: str) -> int:
    """Local index, along the side's axis, of the inner (first own) or outer line."""
    a, s = side
    E, m = prob.E, prob.m[a]
    if s == +1:
        return E + m - 1 if which == "inner" else E + m
    return E if which == "inner" else E - 1


def _line_slice(prob: Problem, side, which: str):
    a, _ = side
    n = prob.dim
    sl = [slice(None)] * (n + 1)          # leading batch dimension
    sl[1 + (n - 1 - a)] = _line_index(prob, side, which)
    return tuple(sl)


def _coupling(prob: Problem, axes, side):
    """c = prod_{b != a} alpha_b / h^2 on the interface line of the receiver (shape of a line)."""
    a, _ = side
    n = prob.dim
    out = np.ones([prob.M[b] for b in range(n) if b != a][::-1], dtype=np.complex128)
    tang = [b for b in range(n) if b != a]
    for j, b in enumerate(tang):
        shp = [1] * (n - 1)
        shp[n - 2 - j] = prob.M[b]
        out = out * axes[b][0].reshape(shp)
    return out / prob.h ** 2


def neighbour(sub, side, parts):
    a, s = side
    k = sub[a] + s
    if k < 0 or k >= parts[a]:
        return None
    nb = list(sub)
    nb[a] = k
    return tuple(nb)


def ddm_solve(prob: Problem, b_ext, rounds: int = 1, local: LocalProblems | None = None,
              workers: int = 1, record: list | None = None, sweeps=None):
    """Run Algorithm 2.1 (2D) / 4.1 (3D) with `rounds` rounds of 2^n sweeps.

    sweeps  optional explicit list of sweep directions replacing the `rounds` rounds of Eq. 2.9
            / 4.2 (e.g. strip_sweeps(parts, 3), the one-dimensional sweeping DDM of Section 3.2
            with its extra forward sweep); steps, routing (Rules 2.4/2.5, 4.1/4.2 over this
            list) and accumulation are unchanged.

    b_ext   J-scaled right-hand side(s) on the global extended grid, shape (*G[::-1]) or
            (R, *G[::-1]) (for a physical source f, b = J f = f in the box).
    Returns u_DDM with the shape of b_ext.

    The own source is consumed the first time a subdomain is solved (f_ij := 0).  A local solve
    whose assembled right-hand side is exactly zero is skipped (u_ij = 0), as the algorithm's
    "if f_ij != 0 ... else set u_ij = 0" step allows.  `record`, if given, receives one dict per
    local solve with the incoming sides and the outgoing trace norms and routes.
    """
    b = np.asarray(b_ext, dtype=np.complex128)
    single = b.ndim == prob.dim
    if single:
        b = b[None]
    R = b.shape[0]
    n = prob.dim
    if sweeps is None:
        dirs = sweep_directions(n)
        L = len(dirs) * rounds
    else:
        dirs = [tuple(d) for d in sweeps]
        L = len(dirs)
    if local is None:
        local = LocalProblems(prob)
    u = np.zeros_like(b)
    g = {}                                    # (l, sub, side) -> [a, b] batched lines
    consumed = set()
    loc_dims = prob.M[::-1]

    def assemble_rhs(l, sub):
        rhs = np.zeros((R,) + loc_dims, dtype=np.complex128)
        if sub not in consumed:
            (gr, lr) = zip(*own_ranges(prob, sub))
            gsl = (slice(None),) + tuple(slice(*r) for r in gr[::-1])
            lsl = (slice(None),) + tuple(slice(*r) for r in lr[::-1])
            rhs[lsl] += b[gsl]
        incoming = []
        for side in sides(n):
            tr = g.get((l, sub, side))
            if tr is None:
                continue
            if np.any(tr[0]) or np.any(tr[1]):
                incoming.append(side)
            c = _coupling(prob, local.axes[sub], side)
            rhs[_line_slice(prob, side, "outer")] += c * tr[1]
            rhs[_line_slice(prob, side, "inner")] -= c * tr[0]
        return rhs, incoming

    def solve(sub, rhs):
        x = np.zeros_like(rhs)
        nz = np.array([rhs[r].any() for r in range(R)])
        if nz.any():
            x[nz] = local.solve(sub, rhs[nz])
        return x

    pool = ThreadPoolExecutor(workers) if workers > 1 else None
    try:
        for l in range(L):
            d = dirs[l % len(dirs)]
            for s in range(1, num_steps(prob.parts) + 1):
                group = step_set(d, s, prob.parts)
                prepared = []
                for sub in group:
                    rhs, incoming = assemble_rhs(l, sub)
                    consumed.add(sub)
                    prepared.append((sub, rhs, incoming))
                if pool is not None:
                    xs = list(pool.map(lambda t: solve(t[0], t[1]), prepared))
                else:
                    xs = [solve(sub, rhs) for sub, rhs, _ in prepared]
                for (sub, rhs, incoming), x in zip(prepared, xs):
                    (gr, lr) = zip(*own_ranges(prob, sub))
                    gsl = (slice(None),) + tuple(slice(*r) for r in gr[::-1])
                    lsl = (slice(None),) + tuple(slice(*r) for r in lr[::-1])
                    u[gsl] += x[lsl]
                    out_log = {}
                    for side in sides(n):
                        nb = neighbour(sub, side, prob.parts)
                        if nb is None:
                            continue
                        tr_in = g.get((l, sub, side))
                        a_line = x[_line_slice(prob, side, "inner")].copy()
                        if tr_in is not None:
                            a_line -= tr_in[1]
                        b_line = x[_line_slice(prob, side, "outer")].copy()
                        lp = route(side_vector(side, n), l, L, dirs)
                        out_log[side] = (lp, float(np.sqrt(np.sum(np.abs(a_line) ** 2)
                                                           + np.sum(np.abs(b_line) ** 2))))
                        if lp is None:
                            continue
                        back = (side[0], -side[1])
                        key = (lp, nb, back)
                        if key in g:
                            g[key][0] += a_line
                            g[key][1] += b_line
                        else:
                            g[key] = [a_line, b_line]
                    if record is not None:
                        record.append({"sweep": l, "step": s, "sub": sub, "incoming": incoming,
                                       "outgoing": out_log,
                                       "solved": bool(np.any(rhs != 0))})
    finally:
        if pool is not None:
            pool.shutdown()
    return u[0] if single else u
