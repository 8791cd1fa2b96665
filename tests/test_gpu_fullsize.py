"""Full-size parity: the GPU solver in the launch configuration bench.py times, against the
CPU oracle at the workloads' full sizes.

At these sizes the oracle cannot run its DDM for every right-hand side, so two checks are made:
  * sampled right-hand sides against the oracle's global sparse solve of the whole PML problem
    (a plain LU of the assembled global operator, no domain decomposition), rel. L2 <= 1e-6;
  * every right-hand side through a property that holds at any size: the residual of the GPU
    field under the oracle's own assembled operator, ||J f - A u|| / ||J f||, at the solver
    tolerance (1e-6) up to a factor 2.
Degenerate inputs: a zero source gives exactly zero, and an empty batch is rejected.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.discretize import Problem, assemble_global, extend_interior, rhs_from_source
from oracle.linsolve import global_solve
from paper_2003_02585_gb300 import synth

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def _dds():
    from paper_2003_02585_gb300 import dds
    return dds


def _solve_workload(name, nrhs=None):
    wl = synth.workload(name, nrhs)
    dds = _dds()
    ctx = dds.Context(wl.n, wl.h, wl.omega, wl.c, wl.parts, wl.pml_cells, wl.pml_strength,
                      precision=wl.precision)
    fe = ctx.extend(wl.f)
    u, it, rel = ctx.solve(torch.from_numpy(fe).to(DEV), tol=wl.tol, maxit=30, rounds=wl.rounds)
    prob = Problem(wl.n, wl.h, wl.omega, wl.c, wl.parts, wl.pml_cells, wl.pml_strength)
    return wl, prob, u.cpu().numpy(), it, rel


def _check(wl, prob, u, rel, sample):
    A, _ = assemble_global(prob)
    b = rhs_from_source(prob, extend_interior(prob, wl.f))
    assert np.all(np.asarray(rel) < wl.tol)
    for r in range(b.shape[0]):
        res = A @ u[r].ravel() - b[r].ravel()
        assert np.linalg.norm(res) / np.linalg.norm(b[r]) < 2 * wl.tol
    ref = global_solve(prob, b[list(sample)])
    for i, r in enumerate(sample):
        err = np.linalg.norm(u[r] - ref[i]) / np.linalg.norm(ref[i])
        assert err < 1e-6, (r, err)


def test_const2d_640_full_size_matches_oracle():
    """640^2, 8x8 subdomains, 16 RHS, 3xTF32 sweeps + FP64 FGMRES to 1e-6, two rounds: the
    benchmark workload, solved exactly as bench.py times it."""
    wl, prob, u, it, rel = _solve_workload("const2d_640")
    assert u.shape[0] == 16
    _check(wl, prob, u, rel, sample=(0, 11))


def test_layer2d_1024_full_size_matches_oracle():
    """1024^2 two-layer medium, 16x16 subdomains, 64 RHS, FGMRES to 1e-6 with three rounds of
    sweeps per preconditioner application: the benchmark workload, solved as bench.py times it."""
    wl, prob, u, it, rel = _solve_workload("layer2d_1024")
    assert u.shape[0] == 64
    _check(wl, prob, u, rel, sample=(5,))


def test_table5_2x2_mixed_fgmres_matches_global_solve():
    """Table 5's smallest workload (Section 5.2, Eq. 5.4): 600^2 interior, 2x2 subdomains of
    300^2 with a 30-point PML (lines of 360 nodes: the stage-parallel tensor-core substitutions),
    four approximated delta sources in one right-hand side, omega / 2 pi = 65.9, mixed sweeps with
    FP64 FGMRES to 1e-6: the field against the oracle's global solve of the whole PML problem."""
    wl, prob, u, it, rel = _solve_workload("table5_2")
    assert prob.M[0] == 360
    _check(wl, prob, u, rel, sample=(0,))
    assert it <= 4, it     # the paper needs 3 iterations on this workload


def test_const2d_128_direct_solver_one_round():
    """The 128^2 / 2x2 case: the DDM as a direct solver (one round, FP64) against the oracle's
    DDM and, Theorem 3.3, within PML level of the global solve."""
    from oracle.sweep import ddm_solve
    wl = synth.workload("const2d_128")
    dds = _dds()
    ctx = dds.Context(wl.n, wl.h, wl.omega, wl.c, wl.parts, wl.pml_cells, wl.pml_strength,
                      precision="fp64")
    prob = Problem(wl.n, wl.h, wl.omega, wl.c, wl.parts, wl.pml_cells, wl.pml_strength)
    b = rhs_from_source(prob, extend_interior(prob, wl.f))
    u = ctx.sweep(torch.from_numpy(ctx.extend(wl.f)).to(DEV), 1).cpu().numpy()
    ref = ddm_solve(prob, b, 1)
    assert np.linalg.norm(u - ref) / np.linalg.norm(ref) < 1e-10
    ug = global_solve(prob, b)
    assert np.linalg.norm(u - ug) / np.linalg.norm(ug) < 3e-4


@pytest.mark.parametrize("precision", ["fp64", "mixed", "mixed_bf16"])
def test_zero_source_gives_zero_and_empty_batch_is_rejected(precision):
    dds = _dds()
    n = (64, 64)
    ctx = dds.Context(n, 1.0 / 64, 2 * np.pi * 4, synth.medium_constant(n), (4, 4), 8, 30.0,
                      precision=precision)
    G = ctx.info()["G"][:2]
    z = torch.zeros((2, G[1], G[0]), dtype=torch.complex128, device=DEV)
    u = ctx.sweep(z).cpu().numpy()
    assert np.count_nonzero(u) == 0
    u, it, rel = ctx.solve(z, tol=1e-6, maxit=5)
    assert np.count_nonzero(u.cpu().numpy()) == 0
    with pytest.raises(dds.DDSError):
        ctx.sweep(torch.zeros((0, G[1], G[0]), dtype=torch.complex128, device=DEV))


def test_const3d_128_full_size_residual_under_oracle_operator():
    """128^3, 4x4x4 subdomains (plane blocks of 2304 nodes: stage-parallel tensor-core
    substitutions), 8 RHS, FGMRES to 1e-6: every field's residual under the oracle's own 7-point
    operator.  (The oracle's global LU at 144^3 is too large to sample here.)"""
    wl, prob, u, it, rel = _solve_workload("const3d_128")
    assert u.shape[0] == 8
    A, _ = assemble_global(prob)
    b = rhs_from_source(prob, extend_interior(prob, wl.f))
    assert np.all(np.asarray(rel) < wl.tol)
    for r in range(8):
        res = A @ u[r].ravel() - b[r].ravel()
        assert np.linalg.norm(res) / np.linalg.norm(b[r]) < 2 * wl.tol
