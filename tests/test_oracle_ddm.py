"""Pins for the oracle's sweeps, routing and FGMRES (CPU only).

The routing is pinned by the paper's walk-throughs (proof of Lemma 3.2) and, more strongly, by
the theorems it makes true: exactness in a constant medium (Theorem 3.3) and at most one extra
round in two-layer media (Theorem 3.10).  Exactness "up to PML reflection" is checked by the
gap shrinking as the PML thickens; a single subdomain must reproduce the global solve exactly.
"""

import os

import numpy as np
import pytest
import scipy.sparse as sp

from oracle.discretize import (Problem, assemble_global, assemble_local, extend_interior,
                               rhs_from_source)
from oracle.fgmres import fgmres
from oracle.linsolve import global_solve
from oracle.sweep import (LocalProblems, _coupling, _line_slice, ddm_solve, num_steps, route,
                          route_table, side_vector, similar_direction, step_index, step_set,
                          strip_sweeps, sweep_directions)
from paper_2003_02585_gb300 import synth


def _problem(n, parts, P, kappa, c=None, H=0):
    h = 1.0 / n[0]
    if c is None:
        c = synth.medium_constant(n)
    return Problem(n, h, kappa, c, parts, P, 30.0, 2, H)


def _rhs(prob, centres, width=None):
    h = prob.h
    w = 2 * h if width is None else width
    f = synth.gaussian_sources(prob.n, h, centres, w)
    return rhs_from_source(prob, extend_interior(prob, f))


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


# ------------------------------------------------------------------ step sets and routing ----

def test_step_sets_cover_each_subdomain_once():
    """Eq. 2.10-2.11: each sweep has N1 + N2 - 1 steps and visits every subdomain once; in the
    first sweep Omega_{i,j} (1-based) is solved at step i + j - 1 (proof of Lemma 3.2)."""
    parts = (5, 3)
    assert num_steps(parts) == 7
    for d in sweep_directions(2):
        seen = []
        for s in range(1, num_steps(parts) + 1):
            seen += step_set(d, s, parts)
        assert sorted(seen) == sorted((i, j) for i in range(5) for j in range(3))
    for i in range(5):
        for j in range(3):
            assert step_index((i, j), (1, 1), parts) == (i + 1) + (j + 1) - 1
    # 3D: N1 + N2 + N3 - 2 steps
    assert num_steps((4, 4, 4)) == 10


def test_similar_direction_3d_needs_componentwise_agreement():
    """Section 4: in 3D, d1 . d2 > 0 and d1(k) d2(k) >= 0 for every k."""
    assert similar_direction((1, 0, 0), (1, -1, -1))
    assert not similar_direction((1, 1, 0), (1, -1, 1))
    assert not similar_direction((1, 1, -1), (1, 1, 1))        # dot > 0 but a sign conflict
    assert similar_direction((1, 1), (1, -1)) is False          # 2D: dot = 0
    assert similar_direction((1, 0), (1, -1))


def _golden_rows(name):
    path = os.path.join(os.path.dirname(__file__), "golden", name)
    with open(path) as fh:
        return [ln.split() for ln in fh if ln.strip() and not ln.startswith("#")]


def test_routing_matches_the_paper_walkthrough():
    """Section 3.1 walkthrough of sweeps 2-4 (tests/golden/routing_2d.txt), sweep order
    (+,+),(-,+),(+,-),(-,-): which later sweep uses a trace made in a sweep, by its direction."""
    dirs = sweep_directions(2)
    L = 4
    rows = _golden_rows("routing_2d.txt")
    assert len(rows) == 7
    for frm, d1, d2, to in rows:
        want = None if to == "-" else int(to) - 1
        assert route((int(d1), int(d2)), int(frm) - 1, L, dirs) == want, (frm, d1, d2, to)
    # with an extra round (Theorem 3.10) the barred trace waits for the next (+,+)-type use
    assert route((1, 0), 1, 8, dirs) == 4


def test_route_table_3d_uses_projection_rule():
    """Rule 4.2: a +x trace from sweep (-,+,+) may not be used in (+,-,+) (x-y projections
    opposite) nor in (+,+,-) (x-z projections opposite) nor in (+,-,-)."""
    t = route_table(3, 1)
    assert t[1][(0, +1)] is None
    assert t[0][(0, -1)] == 1 and t[0][(1, -1)] == 2 and t[0][(2, -1)] == 4
    for l in range(8):
        for side, lp in t[l].items():
            if lp is not None:
                d_use = sweep_directions(3)[lp % 8]
                assert lp >= l and d_use[side[0]] == side[1]


def test_route_every_trace_forward_in_its_own_sweep():
    """A trace leaving in the sweep's own direction is consumed later in the same sweep, which
    is what makes one step set depend only on the previous one."""
    for dim in (2, 3):
        dirs = sweep_directions(dim)
        for l, d in enumerate(dirs):
            for a in range(dim):
                D = tuple(d[a] if b == a else 0 for b in range(dim))
                assert route(D, l, len(dirs), dirs) == l


# ------------------------------------------------------------------ local potential ----------

def test_commutator_source_identity():
    """The trace source reproduces A_R^{-1}[A_R, chi_H] t = chi_H t - A_R^{-1} chi_H A_R t for an
    arbitrary t; the commutator here is built from the sparse matrix, not from the oracle's
    line formula."""
    prob = _problem((24, 24), (3, 3), 4, 2 * np.pi * 3, H=1)
    sub = (1, 1)
    A, _, axes = assemble_local(prob, sub)
    dims = prob.M[::-1]
    rng = np.random.default_rng(0)
    t = rng.standard_normal(dims) + 1j * rng.standard_normal(dims)
    for side in [(0, 1), (0, -1), (1, 1), (1, -1)]:
        a_ax, s = side
        # chi_H: the receiver's side of the interface on `side` (own + beyond on the far side)
        ax_dim = 1 - a_ax
        idx = np.arange(prob.M[a_ax])
        inner = prob.E + prob.m[a_ax] - 1 if s == 1 else prob.E
        chi1 = (idx <= inner) if s == 1 else (idx >= inner)
        shp = [1, 1]
        shp[ax_dim] = prob.M[a_ax]
        chi = np.broadcast_to(chi1.reshape(shp), dims).astype(float)
        C = sp.diags(chi.ravel())
        comm = (A @ C - C @ A) @ t.ravel()
        # the oracle's line formula: rhs[outer] += c b, rhs[inner] -= c a
        rhs = np.zeros((1,) + dims, dtype=complex)
        c = _coupling(prob, axes, side)
        a_line = t[None][_line_slice(prob, side, "outer")]
        b_line = t[None][_line_slice(prob, side, "inner")]
        rhs[_line_slice(prob, side, "outer")] += c * b_line
        rhs[_line_slice(prob, side, "inner")] -= c * a_line
        assert np.max(np.abs(rhs[0].ravel() - comm)) < 1e-10 * np.max(np.abs(comm))
        # and the identity itself
        lhs = sp.linalg.spsolve(A.tocsc(), comm)
        rhs_id = chi.ravel() * t.ravel() - sp.linalg.spsolve(A.tocsc(), chi.ravel() * (A @ t.ravel()))
        assert np.linalg.norm(lhs - rhs_id) / np.linalg.norm(rhs_id) < 1e-12


# ------------------------------------------------------------------ whole DDM ----------------

@pytest.mark.parametrize("n,parts", [((40, 40), (1, 1)), ((12, 12, 12), (1, 1, 1)),
                                     ((48, 32), (1, 1))])
def test_single_subdomain_is_the_global_solve(n, parts):
    prob = _problem(n, parts, 6, 2 * np.pi * 3)
    b = _rhs(prob, [(0.4, 0.55, 0.5)[:len(n)]])
    assert _rel(ddm_solve(prob, b[0]), global_solve(prob, b[0])) < 1e-13


def test_theorem_3_3_constant_medium_gap_shrinks_with_pml():
    """Theorem 3.3: in a constant medium one round reproduces the global PML solution; the
    discrete gap is PML reflection and must shrink as the PML thickens."""
    gaps = []
    for P in (8, 16, 24):
        prob = _problem((64, 64), (2, 2), P, 8 * np.pi)
        b = _rhs(prob, [(0.5, 0.5)])
        gaps.append(_rel(ddm_solve(prob, b[0]), global_solve(prob, b[0])))
    assert gaps[0] < 2e-3 and gaps[1] < gaps[0] / 3 and gaps[2] < gaps[1]
    prob = _problem((64, 64), (4, 4), 16, 8 * np.pi)
    b = _rhs(prob, [(0.3, 0.6)])
    assert _rel(ddm_solve(prob, b[0]), global_solve(prob, b[0])) < 1e-3


def test_theorem_3_3_in_3d():
    gaps = []
    for P in (5, 8):
        prob = _problem((16, 16, 16), (2, 2, 2), P, 4 * np.pi)
        b = _rhs(prob, [(0.45, 0.5, 0.55)], width=1.5 / 16)
        gaps.append(_rel(ddm_solve(prob, b[0]), global_solve(prob, b[0])))
    assert gaps[1] < 5e-3 and gaps[1] < gaps[0] / 2


@pytest.mark.parametrize("axis", [1, 0])
def test_theorem_3_10_two_layer_needs_at_most_one_extra_round(axis):
    """Theorem 3.10 (and the vertical-interface rule after Lemma 3.9): a source below (left of)
    the interface needs one round; a source above (right of) it needs one extra round."""
    n = (64, 64)
    c = synth.medium_two_layer(n, 1.0 / 64, 0.37, 1.0, 1.5, axis=axis)
    prob = _problem(n, (4, 4), 16, 8 * np.pi, c=c)
    below = (0.3, 0.2) if axis == 1 else (0.2, 0.3)
    above = (0.3, 0.8) if axis == 1 else (0.8, 0.3)
    loc = LocalProblems(prob)
    assert loc.n_distinct == 3                       # below, straddling, above
    bb = _rhs(prob, [below])[0]
    assert _rel(ddm_solve(prob, bb, 1, loc), global_solve(prob, bb)) < 1e-3
    ba = _rhs(prob, [above])[0]
    ga = global_solve(prob, ba)
    e1 = _rel(ddm_solve(prob, ba, 1, loc), ga)
    e2 = _rel(ddm_solve(prob, ba, 2, loc), ga)
    assert e1 > 1e-2 and e2 < 1e-4


def test_walkthrough_5x5_trace_counts():
    """Section 3.1 walkthrough (tests/golden/walkthrough_5x5.txt): 5x5 partition, source inside
    Omega_{3,3}; in the first sweep, which subdomains solve at steps 5-7, how many traces each
    takes and how many it generates.  The trace sent back to the sender is zero up to PML
    reflection, so "generated" counts the significant outgoing traces."""
    prob = _problem((80, 80), (5, 5), 16, 8 * np.pi)
    b = _rhs(prob, [(0.5, 0.5)], width=1.0 / 80)       # support well inside Omega_{3,3}
    rec = []
    ddm_solve(prob, b[0], record=rec)
    s1 = [r for r in rec if r["sweep"] == 0]
    by_step = {}
    for r in s1:
        if r["solved"]:
            by_step.setdefault(r["step"], []).append(r)
    assert all(s >= 5 for s in by_step)                 # steps 1..4 have zero solutions
    ref = max(v[1] for v in by_step[5][0]["outgoing"].values())

    def significant(r):
        return sum(1 for v in r["outgoing"].values() if v[1] > 1e-2 * ref)

    rows = _golden_rows("walkthrough_5x5.txt")
    assert len(rows) == 4
    for step, i, j, taken, made in (map(int, row) for row in rows):
        # the oracle's step numbers are the paper's; its subdomain indices are 0-based
        subs = {r["sub"]: r for r in by_step[step]}
        r = subs[(i - 1, j - 1)]
        assert len(r["incoming"]) == taken, (step, i, j)
        assert significant(r) == made, (step, i, j)
    assert [r["sub"] for r in by_step[5]] == [(2, 2)]   # only Omega_{3,3} at step 5


def test_ddm_is_linear_and_batch_invariant():
    prob = _problem((48, 48), (3, 3), 8, 6 * np.pi)
    b = _rhs(prob, [(0.3, 0.4), (0.7, 0.6)])
    loc = LocalProblems(prob)
    u_batch = ddm_solve(prob, b, local=loc)
    u0 = ddm_solve(prob, b[0], local=loc)
    u1 = ddm_solve(prob, b[1], local=loc)
    assert _rel(u_batch[0], u0) < 1e-14 and _rel(u_batch[1], u1) < 1e-14
    ulin = ddm_solve(prob, b[0] + 2 * b[1], local=loc)
    assert _rel(ulin, u0 + 2 * u1) < 1e-13


def test_global_reciprocity():
    """G(x, y) = G(y, x) for the J-scaled symmetric system (Eq. 2.4 with J = 1 in the box)."""
    prob = _problem((40, 40), (1, 1), 8, 6 * np.pi, c=synth.medium_random((40, 40), 1 / 40, 7))
    G = prob.G
    e = np.zeros((2,) + G[::-1], dtype=complex)
    x, y = (prob.E + 5, prob.E + 9), (prob.E + 30, prob.E + 22)
    e[0][x[1], x[0]] = 1.0
    e[1][y[1], y[0]] = 1.0
    u = global_solve(prob, e)
    assert abs(u[0][y[1], y[0]] - u[1][x[1], x[0]]) < 1e-12 * abs(u[0][y[1], y[0]])


# ------------------------------------------------------------------ FGMRES -------------------

def _fgmres_case(prob, centre, rounds=1, tol=1e-10):
    A, _ = assemble_global(prob)
    b = _rhs(prob, [centre])[0]
    loc = LocalProblems(prob)
    shape = b.shape
    x, it, hist = fgmres(lambda v: A @ v,
                         lambda v: ddm_solve(prob, v.reshape(shape), rounds, loc).ravel(),
                         b.ravel(), tol=tol, maxit=40)
    return x.reshape(shape), it, hist, global_solve(prob, b)


def test_fgmres_constant_medium_converges_to_global_solution():
    prob = _problem((64, 64), (4, 4), 12, 8 * np.pi)
    x, it, hist, ug = _fgmres_case(prob, (0.35, 0.6))
    assert hist[-1] < 1e-10
    assert it <= 6                                      # Table 5: 3-4 iterations to 1e-6
    assert _rel(x, ug) < 1e-8


def test_fgmres_two_layer_and_exact_preconditioner():
    c = synth.medium_two_layer((64, 64), 1 / 64)
    prob = _problem((64, 64), (4, 4), 12, 8 * np.pi, c=c)
    x, it, hist, ug = _fgmres_case(prob, (0.5, 0.8), tol=1e-8)
    assert hist[-1] < 1e-8 and it <= 15 and _rel(x, ug) < 1e-6
    # two rounds make the preconditioner (nearly) exact in a two-layer medium (Theorem 3.10)
    x2, it2, _, _ = _fgmres_case(prob, (0.5, 0.8), rounds=2, tol=1e-8)
    assert it2 < it
    # one subdomain: the DDM is the exact inverse, one iteration suffices
    p1 = _problem((32, 32), (1, 1), 8, 4 * np.pi)
    _, it1, hist1, _ = _fgmres_case(p1, (0.5, 0.5))
    assert it1 == 1 and hist1[-1] < 1e-12


# ------------------------------------------------------------------ strip partitions ----------

def _strip_case(n, parts, P, interface, centre):
    h = 1.0 / n[0]
    c = (synth.medium_constant(n) if interface is None
         else synth.medium_two_layer(n, h, interface=interface))
    prob = _problem(n, parts, P, 2 * np.pi * 4, c=c)
    b = _rhs(prob, [centre])[0]
    return prob, b, global_solve(prob, b)


def test_strip_sweep_list_alternates_along_the_cut_axis():
    """Section 3.2: forward, backward, forward ... along the one cut axis."""
    assert strip_sweeps((1, 4), 3) == [(1, 1), (1, -1), (1, 1)]
    assert strip_sweeps((4, 1), 2) == [(1, 1), (-1, 1)]
    assert strip_sweeps((1, 1, 3), 3) == [(1, 1, 1), (1, 1, -1), (1, 1, 1)]
    with pytest.raises(ValueError):
        strip_sweeps((2, 2), 3)


@pytest.mark.parametrize("parts", [(1, 3), (3, 1)])
def test_strip_two_sweeps_are_algorithm_2_1_on_the_strip(parts):
    """The one-dimensional sweeping DDM is the degenerate form of Algorithm 2.1 on a 1 x N (or
    N x 1) partition (Section 3.2): its forward/backward pair gives exactly the field of one round
    of the four diagonal sweeps, two of which receive nothing."""
    prob, b, _ = _strip_case((48, 48), parts, 8, 0.4, (0.45, 0.6))
    loc = LocalProblems(prob)
    two = ddm_solve(prob, b, local=loc, sweeps=strip_sweeps(parts, 2))
    diag = ddm_solve(prob, b, 1, loc)
    assert np.array_equal(two, diag)


def test_strip_lemma_3_4_two_sweeps_suffice_below_the_interface():
    """Lemma 3.4 (1 x 2, horizontal interface above the subdomain interface, source in the lower
    subdomain): forward + backward already give the PML solution (up to PML reflection); one
    sweep alone does not."""
    prob, b, ug = _strip_case((48, 48), (1, 2), 10, 0.7, (0.5, 0.25))
    loc = LocalProblems(prob)
    gaps = [_rel(ddm_solve(prob, b, local=loc, sweeps=strip_sweeps((1, 2), k)), ug)
            for k in (1, 2)]
    assert gaps[0] > 1e-2 and gaps[1] < 3e-4, gaps


@pytest.mark.parametrize("n,parts,centre", [((48, 48), (1, 2), (0.5, 0.75)),
                                           ((64, 64), (1, 4), (0.5, 0.875))])
def test_strip_extra_forward_sweep_theorem_3_6(n, parts, centre):
    """Lemma 3.5 / Theorem 3.6: with the interface below the source's subdomain the reflection
    back into the upper subdomains needs a third (forward) sweep.  Two sweeps leave an O(1e-1)
    gap to the global PML solve; three sweeps reach PML-reflection level, and that gap shrinks
    as the PML thickens."""
    gaps = {}
    for P in (10, 16):
        prob, b, ug = _strip_case(n, parts, P, 0.3, centre)
        loc = LocalProblems(prob)
        gaps[P] = [_rel(ddm_solve(prob, b, local=loc, sweeps=strip_sweeps(parts, k)), ug)
                   for k in (2, 3)]
    assert gaps[10][0] > 3e-2 and gaps[16][0] > 3e-2, gaps
    assert gaps[10][1] < 2e-4 and gaps[16][1] < 0.7 * gaps[10][1], gaps
