"""Pins for the oracle's discretisation and direct solvers (CPU only).

Each test checks the oracle against something other than itself: a textbook matrix built from
library routines, a closed-form plane wave, the free-space Green's function, brute force, or a
structural property the method relies on.
"""

import numpy as np
import pytest
import scipy.sparse as sp
from scipy.special import hankel1

from oracle.discretize import (Problem, assemble_global, assemble_local, extend_interior,
                               interior_view, kappa_local, own_ranges, rhs_from_source)
from oracle.linsolve import BandedLU, SparseLU, dense_solve, global_solve
from paper_2003_02585_gb300 import synth


def _prob(n, parts, P=4, S=30.0, kappa=2 * np.pi * 2, c=None, H=0):
    d = len(n)
    h = 1.0 / n[0]
    if c is None:
        c = np.ones(tuple(n[::-1]))
    return Problem(n, h, kappa, c, parts, P, S, 2, H)


def _rand_c(n, seed=0):
    rng = np.random.default_rng(seed)
    return 1.0 + 0.5 * rng.random(tuple(n[::-1]))


@pytest.mark.parametrize("n", [(6, 6), (4, 6, 5)])
def test_operator_complex_symmetric(n):
    """The J-scaled form of Eq. 2.3 / 4.1 is complex symmetric (A = A^T, not Hermitian)."""
    prob = _prob(n, (1,) * len(n), P=3, c=_rand_c(n))
    A, _ = assemble_global(prob)
    assert abs(A - A.T).max() == 0.0
    assert abs(A - A.conj().T).max() > 1e-3


def _dirichlet_second_difference(G, h):
    return sp.diags([np.ones(G - 1), -2 * np.ones(G), np.ones(G - 1)], [-1, 0, 1]) / h ** 2


@pytest.mark.parametrize("n", [(7, 5), (4, 5, 6)])
def test_operator_without_pml_is_textbook_laplacian(n):
    """With sigma = 0 the operator is the Kronecker-sum 5/7-point Laplacian plus kappa^2."""
    c = _rand_c(n, 1)
    prob = _prob(n, (1,) * len(n), P=2, S=0.0, c=c)
    A, J = assemble_global(prob)
    assert np.all(J == 1.0)
    G = prob.G
    h = prob.h
    lap = None
    for a in range(len(n)):
        # numpy layout (x_{d-1}, ..., x_0): axis a is kron position d-1-a
        mats = [sp.identity(G[b]) for b in range(len(n))][::-1]
        mats[len(n) - 1 - a] = _dirichlet_second_difference(G[a], h)
        term = mats[0]
        for mtx in mats[1:]:
            term = sp.kron(term, mtx)
        lap = term if lap is None else lap + term
    kap = prob.omega / c
    # kappa in the halo/PML is the nearest interior value
    idx = [np.clip(np.arange(G[a]) - prob.E, 0, n[a] - 1) for a in range(len(n))]
    kext = kap[np.ix_(*idx[::-1])]
    ref = lap + sp.diags(kext.ravel() ** 2)
    assert abs(A - ref).max() < 1e-9 * abs(ref).max()


def test_plane_wave_dispersion_closed_form():
    """A discrete plane wave exp(i(t1 p + t2 q)) with 2cos t1 + 2cos t2 - 4 + kappa^2 h^2 = 0
    is annihilated by every row of A that sees only un-stretched nodes."""
    n = (24, 24)
    prob = _prob(n, (1, 1), P=4, S=30.0, kappa=2 * np.pi * 3)
    A, _ = assemble_global(prob)
    kh2 = (prob.omega * prob.h) ** 2
    t1 = 0.7
    t2 = np.arccos((4 - kh2 - 2 * np.cos(t1)) / 2)
    G = prob.G
    q, p = np.meshgrid(np.arange(G[1]), np.arange(G[0]), indexing="ij")
    u = np.exp(1j * (t1 * p + t2 * q))
    r = (A @ u.ravel()).reshape(G[::-1])
    E = prob.E
    inner = r[E + 1:E + n[1] - 1, E + 1:E + n[0] - 1]
    scale = 4.0 / prob.h ** 2                     # size of an interior diagonal entry
    assert np.max(np.abs(inner)) < 1e-12 * scale
    # a mismatched angle is not annihilated
    r2 = (A @ np.exp(1j * (t1 * p + 1.1 * t2 * q)).ravel()).reshape(G[::-1])
    assert np.max(np.abs(r2[E + 1:E + n[1] - 1, E + 1:E + n[0] - 1])) > 1e-3 * scale


def test_free_space_green_2d_second_order():
    """Global PML solve vs -(i/4) H0(kappa r) (L = Delta + kappa^2, L G = -delta), for a
    unit-mass Gaussian (spectral factor exp(-kappa^2 w^2 / 2)); error ~1e-2 and second order."""
    errs = []
    for n in (128, 256):
        h = 1.0 / n
        w = 2 * h
        kap = 8 * np.pi
        prob = Problem((n, n), h, kap, np.ones((n, n)), (1, 1), 16, 30.0)
        f = synth.gaussian_source((n, n), h, (0.5, 0.5), w)
        u = interior_view(prob, global_solve(prob, rhs_from_source(prob, extend_interior(prob, f))))
        x = (np.arange(n) + 0.5) * h
        X2, X1 = np.meshgrid(x, x, indexing="ij")
        r = np.hypot(X1 - 0.5, X2 - 0.5)
        mask = (r > 0.15) & (r < 0.45)
        ex = -0.25j * hankel1(0, kap * r[mask]) * np.exp(-kap ** 2 * w ** 2 / 2)
        errs.append(np.linalg.norm(u[mask] - ex) / np.linalg.norm(ex))
    assert errs[0] < 0.02
    assert 3.0 < errs[0] / errs[1] < 5.0          # second-order convergence (Table 1: rate 2.0)


def test_free_space_green_3d():
    """Global 7-point PML solve vs -exp(i kappa r) / (4 pi r)."""
    n = 32
    h = 1.0 / n
    w = 1.5 * h
    kap = 4 * np.pi
    prob = Problem((n, n, n), h, kap, np.ones((n, n, n)), (1, 1, 1), 8, 30.0)
    f = synth.gaussian_source((n, n, n), h, (0.5, 0.5, 0.5), w)
    u = interior_view(prob, global_solve(prob, rhs_from_source(prob, extend_interior(prob, f))))
    x = (np.arange(n) + 0.5) * h
    X3, X2, X1 = np.meshgrid(x, x, x, indexing="ij")
    r = np.sqrt((X1 - .5) ** 2 + (X2 - .5) ** 2 + (X3 - .5) ** 2)
    mask = (r > 0.2) & (r < 0.45)
    ex = -np.exp(1j * kap * r[mask]) / (4 * np.pi * r[mask]) * np.exp(-kap ** 2 * w ** 2 / 2)
    assert np.linalg.norm(u[mask] - ex) / np.linalg.norm(ex) < 0.04


def test_pml_sign_matters():
    """A PML with the wrong sign of sigma amplifies instead of absorbing (fails the Green pin)."""
    n = 64
    h = 1.0 / n
    w = 2 * h
    kap = 4 * np.pi
    errs = {}
    for S in (30.0, -30.0):
        prob = Problem((n, n), h, kap, np.ones((n, n)), (1, 1), 12, S)
        f = synth.gaussian_source((n, n), h, (0.5, 0.5), w)
        u = interior_view(prob, global_solve(prob, rhs_from_source(prob, extend_interior(prob, f))))
        x = (np.arange(n) + 0.5) * h
        X2, X1 = np.meshgrid(x, x, indexing="ij")
        r = np.hypot(X1 - 0.5, X2 - 0.5)
        mask = (r > 0.15) & (r < 0.45)
        ex = -0.25j * hankel1(0, kap * r[mask]) * np.exp(-kap ** 2 * w ** 2 / 2)
        errs[S] = np.linalg.norm(u[mask] - ex) / np.linalg.norm(ex)
    assert errs[30.0] < 0.05 and errs[-30.0] > 0.3


@pytest.mark.parametrize("n", [(8, 7), (5, 4, 6)])
def test_banded_lu_matches_dense(n):
    prob = _prob(n, (1,) * len(n), P=2, c=_rand_c(n, 2))
    A, _ = assemble_global(prob)
    rng = np.random.default_rng(0)
    b = rng.standard_normal(A.shape[0]) + 1j * rng.standard_normal(A.shape[0])
    xd = dense_solve(A, b)
    bw = int(np.prod(prob.G[::-1][1:]))
    xb = BandedLU(A, bw, bw).solve(b)
    xs = SparseLU(A).solve(b)
    assert np.linalg.norm(xb - xd) / np.linalg.norm(xd) < 1e-12
    assert np.linalg.norm(xs - xd) / np.linalg.norm(xd) < 1e-12


def test_global_solve_residual():
    n = (40, 40)
    prob = _prob(n, (1, 1), P=8, c=_rand_c(n, 3), kappa=2 * np.pi * 4)
    A, _ = assemble_global(prob)
    rng = np.random.default_rng(1)
    b = rng.standard_normal(prob.G[::-1]) + 0j
    u = global_solve(prob, b)
    assert np.linalg.norm(A @ u.ravel() - b.ravel()) / np.linalg.norm(b) < 1e-12


def test_kappa_extension_nearest_point_brute_force():
    """Eq. 2.8: kappa_ij at every extended node equals kappa at the nearest own node
    (brute-force nearest search over all own nodes)."""
    n = (12, 12)
    c = _rand_c(n, 4)
    prob = _prob(n, (3, 2), P=3, c=c)
    kin = prob.omega / c
    for sub in [(0, 0), (1, 1), (2, 0)]:
        kl = kappa_local(prob, sub)
        m = prob.m
        own = [(i, j) for j in range(sub[1] * m[1], (sub[1] + 1) * m[1])
               for i in range(sub[0] * m[0], (sub[0] + 1) * m[0])]
        own = np.array(own, dtype=float)
        for (lq, lp) in [(0, 0), (1, prob.M[0] - 1), (prob.M[1] - 1, 3), (4, 5)]:
            gi = sub[0] * m[0] + lp - prob.E
            gj = sub[1] * m[1] + lq - prob.E
            dist = (own[:, 0] - gi) ** 2 + (own[:, 1] - gj) ** 2
            bi, bj = own[np.argmin(dist)].astype(int)
            assert kl[lq, lp] == kin[bj, bi]


@pytest.mark.parametrize("n,parts", [((12, 8), (3, 2)), ((6, 6, 4), (2, 3, 2))])
def test_local_rows_equal_global_rows_on_own_nodes(n, parts):
    """The extended subdomain operator reproduces the global operator on every own node (the
    subdomain PML starts at its box, J = 1 there, and exterior PMLs coincide)."""
    prob = _prob(n, parts, P=3, c=_rand_c(n, 5), H=1)
    Ag, _ = assemble_global(prob)
    Gdims = prob.G[::-1]
    for sub in prob.subdomains():
        Al, _, _ = assemble_local(prob, sub)
        Ldims = prob.M[::-1]
        (gr, lr) = zip(*own_ranges(prob, sub))
        gidx = np.ix_(*[np.arange(*r) for r in gr[::-1]])
        lidx = np.ix_(*[np.arange(*r) for r in lr[::-1]])
        glin = np.arange(np.prod(Gdims)).reshape(Gdims)[gidx].ravel()
        llin = np.arange(np.prod(Ldims)).reshape(Ldims)[lidx].ravel()
        # map local column indices to global ones (local node l <-> global k m + l)
        offs = [sub[a] * prob.m[a] for a in range(len(n))]
        lcoords = np.array(np.unravel_index(np.arange(np.prod(Ldims)), Ldims))
        gcoords = lcoords + np.array(offs[::-1])[:, None]
        l2g = np.ravel_multi_index(gcoords, Gdims)
        Al = Al.tocsr()
        for gl, ll in zip(glin[::7], llin[::7]):
            row_l = Al.getrow(ll)
            row_g = Ag.getrow(gl)
            ref = dict(zip(row_g.indices, row_g.data))
            got = dict(zip(l2g[row_l.indices], row_l.data))
            assert set(ref) == set(got)
            for k in ref:
                assert abs(ref[k] - got[k]) <= 1e-12 * abs(ref[k])
