"""GPU parity: libdds (through its C ABI) against the CPU oracle.

Tolerances.  FP64 mode: the GPU path factors line blocks instead of the oracle's banded LU and
sums in another order, so results agree to rounding of a well-conditioned chain; 1e-10 relative
L2 is asserted (observed ~1e-13).  Single-precision modes: substitutions and trace transfer in complex FP32
(unit roundoff 6e-8; 3xTF32 split products ~1e-6 and 3xBF16 ~4e-6 per block product on the
tensor cores, amplified by the local solve's conditioning); the raw DDM output is checked to
1e-4 relative (1e-3 for 3xBF16), and after FP64 FGMRES refinement the field must match the oracle's
global solve to 1e-6 (the accuracy target of the mixed mode).
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.discretize import (Problem, assemble_global, assemble_local, extend_interior,
                               rhs_from_source)
from oracle.linsolve import global_solve
from oracle.sweep import LocalProblems, ddm_solve
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


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _case(n, parts, P, kappa, c=None, centres=None, H=0, width=None):
    h = 1.0 / n[0]
    c = synth.medium_constant(n) if c is None else c
    centres = centres or [tuple(0.5 for _ in n)]
    f = synth.gaussian_sources(n, h, centres, 2 * h if width is None else width)
    prob = Problem(n, h, kappa, c, parts, P, 30.0, 2, H)
    return prob, f


def _ctx(prob, precision="fp64", plan="auto"):
    return _dds().Context(prob.n, prob.h, prob.omega, prob.c, prob.parts, prob.pml_cells,
                          prob.pml_strength, prob.pml_power, prob.halo, precision, plan)


def _on_dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to(DEV)


# ----------------------------------------------------------------------------- operator ------

@pytest.mark.parametrize("n,parts,H,P", [((40, 32), (2, 2), 0, 4), ((8, 12, 8), (2, 3, 2), 1, 2)])
def test_apply_matches_oracle_operator(n, parts, H, P):
    rng = np.random.default_rng(0)
    c = 1.0 + 0.5 * rng.random(n[::-1])
    prob, _ = _case(n, parts, P, 2 * np.pi * 3, c=c, H=H)
    ctx = _ctx(prob)
    A, J = assemble_global(prob)
    u = rng.standard_normal((2,) + prob.G[::-1]) + 1j * rng.standard_normal((2,) + prob.G[::-1])
    got = ctx.apply(_on_dev(u)).cpu().numpy()
    for r in range(2):
        ref = (A @ u[r].ravel()).reshape(prob.G[::-1]) / J
        assert _rel(got[r], ref) < 1e-13


# ----------------------------------------------------------------------------- local solve ---

SINGLE_TOL = {"mixed": 1e-4, "mixed_bf16": 1e-3, "mixed_fp32": 1e-4}


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-11)] + list(SINGLE_TOL.items()))
def test_local_solve_matches_banded_lu(precision, tol):
    """K2/K3 (block substitutions with the FP64 Schur factors) vs the oracle's banded LU on one
    extended subdomain, random right-hand sides (ragged: M = 50 is no multiple of a tile)."""
    rng = np.random.default_rng(1)
    prob, _ = _case((52, 52), (2, 2), 12, 2 * np.pi * 6)
    ctx = _ctx(prob, precision)
    loc = LocalProblems(prob)
    dims = prob.M[::-1]
    b = rng.standard_normal((3,) + dims) + 1j * rng.standard_normal((3,) + dims)
    for sub_lin, sub in [(0, (0, 0)), (3, (1, 1))]:
        x = ctx.local_solve(sub_lin, _on_dev(b)).cpu().numpy()
        ref = loc.solve(sub, b)
        assert _rel(x, ref) < tol


# ----------------------------------------------------------------------------- DDM parity ----

DDM_CASES = [
    # (n, parts, P, kappa, medium, centres, rounds, H)
    ((128, 128), (2, 2), 16, 2 * np.pi * 8, "const", [(0.5, 0.5)], 1, 0),   # 128^2 2x2, k=16 pi
    ((60, 36), (3, 2), 6, 2 * np.pi * 3, "const", [(0.3, 0.6), (0.8, 0.2)], 1, 0),
    ((48, 48), (4, 3), 5, 2 * np.pi * 3, "layer", [(0.4, 0.8)], 2, 1),
    ((40, 40), (1, 4), 6, 2 * np.pi * 3, "layer", [(0.5, 0.3)], 1, 0),        # 1 x N strip
    ((32, 32), (1, 1), 6, 2 * np.pi * 3, "const", [(0.5, 0.5)], 1, 0),        # one subdomain
    ((12, 12, 12), (2, 2, 2), 2, 2 * np.pi * 1.5, "const", [(0.4, 0.5, 0.6)], 1, 0),
    ((12, 12, 16), (2, 2, 4), 2, 2 * np.pi * 1.5, "layer", [(0.5, 0.4, 0.8)], 2, 0),
]


def _medium(kind, n):
    if kind == "const":
        return synth.medium_constant(n)
    return synth.medium_two_layer(n, 1.0 / n[0], axis=len(n) - 1)


@pytest.mark.parametrize("plan", ["direct", "trace"])
@pytest.mark.parametrize("case", DDM_CASES,
                         ids=lambda c: "x".join(map(str, c[0])) + f"-{c[1]}-r{c[6]}")
def test_ddm_fp64_matches_oracle(case, plan):
    n, parts, P, kappa, med, centres, rounds, H = case
    prob, f = _case(n, parts, P, kappa, c=_medium(med, n), centres=centres, H=H)
    b = rhs_from_source(prob, extend_interior(prob, f))
    ref = ddm_solve(prob, b, rounds)
    ctx = _ctx(prob, "fp64", plan)
    got = ctx.sweep(_on_dev(ctx.extend(f)), rounds).cpu().numpy()
    for r in range(len(centres)):
        assert _rel(got[r], ref[r]) < 1e-10


@pytest.mark.parametrize("precision", list(SINGLE_TOL))
@pytest.mark.parametrize("plan", ["direct", "trace"])
def test_ddm_mixed_matches_oracle(plan, precision):
    """Single-precision sweeps: 3xTF32 and 3xBF16 tensor-core substitutions and the FP32
    CUDA-core substitutions, raw DDM output against the FP64 oracle."""
    n = (96, 96)
    prob, f = _case(n, (3, 3), 12, 2 * np.pi * 6, c=_medium("layer", n), centres=[(0.3, 0.3)])
    b = rhs_from_source(prob, extend_interior(prob, f))
    ref = ddm_solve(prob, b, 1)
    ctx = _ctx(prob, precision, plan)
    got = ctx.sweep(_on_dev(ctx.extend(f))).cpu().numpy()
    assert _rel(got[0], ref[0]) < SINGLE_TOL[precision]


@pytest.mark.parametrize("precision", ["mixed", "mixed_bf16"])
@pytest.mark.parametrize("case", [DDM_CASES[1], DDM_CASES[2], DDM_CASES[5], DDM_CASES[6]],
                         ids=lambda c: "x".join(map(str, c[0])) + f"-{c[1]}-r{c[6]}")
def test_tensor_core_trace_solves_match_oracle(case, precision):
    """The trace solves of the trace plan on the tensor cores (k_trace_tc: the map as 128-row
    tiles of split pieces, 32-column tiles of (subdomain, RHS), FP32 accumulation in TMEM) on
    ragged geometry: sides of 60 and 64 inputs (padded to 16), 2D and 3D, two rounds, a halo;
    the raw DDM against the oracle's DDM."""
    n, parts, P, kappa, med, centres, rounds, H = case
    prob, f = _case(n, parts, P, kappa, c=_medium(med, n), centres=centres, H=H)
    b = rhs_from_source(prob, extend_interior(prob, f))
    ref = ddm_solve(prob, b, rounds)
    ctx = _ctx(prob, precision, "trace")
    got = ctx.sweep(_on_dev(ctx.extend(f)), rounds).cpu().numpy()
    for r in range(len(centres)):
        assert _rel(got[r], ref[r]) < SINGLE_TOL[precision], r


@pytest.mark.parametrize("precision", ["mixed", "mixed_bf16"])
@pytest.mark.parametrize("nrhs", [20, 40])
def test_tensor_core_wide_panels_match_oracle(nrhs, precision):
    """64 subdomains x 20 (40) right-hand sides put 1280 (2560) columns into one substitution
    launch, so the tensor-core kernel runs panels of 16 (32) columns; the mixed DDM must agree
    with the oracle's DDM (Algorithm 2.1, banded-LU local solves) right-hand side by right-hand
    side."""
    n = (128, 128)
    rng = np.random.default_rng(7)
    centres = [tuple(x) for x in rng.uniform(0.1, 0.9, size=(nrhs, 2))]
    prob, f = _case(n, (8, 8), 4, 2 * np.pi * 5, c=_medium("layer", n), centres=centres)
    b = rhs_from_source(prob, extend_interior(prob, f))
    ref = ddm_solve(prob, b, 1)
    ctx = _ctx(prob, precision, "trace")
    got = ctx.sweep(_on_dev(ctx.extend(f))).cpu().numpy()
    for r in range(nrhs):
        assert _rel(got[r], ref[r]) < SINGLE_TOL[precision], r


@pytest.mark.parametrize("precision", ["mixed", "mixed_bf16"])
def test_mixed_wide_lines_2d_match_oracle(precision):
    """2D lines of 136 nodes (> 128: the stage-parallel tensor-core substitutions, direct plan):
    the raw mixed DDM against the oracle's DDM, and mixed FGMRES against the oracle's global
    solve."""
    n = (240, 240)
    prob, f = _case(n, (2, 2), 8, 2 * np.pi * 6, c=_medium("layer", n),
                    centres=[(0.4, 0.3), (0.7, 0.8)])
    assert prob.M[0] == 136
    bb = rhs_from_source(prob, extend_interior(prob, f))
    ref = ddm_solve(prob, bb, 1)
    ctx = _ctx(prob, precision)
    assert ctx.info()["plan"] == 1   # the automatic plan is the direct one for wide lines
    fe = _on_dev(ctx.extend(f))
    got = ctx.sweep(fe).cpu().numpy()
    for r in range(2):
        assert _rel(got[r], ref[r]) < SINGLE_TOL[precision], r
    u, it, rel = ctx.solve(fe, tol=1e-9, maxit=30)
    ug = global_solve(prob, bb)
    u = u.cpu().numpy()
    assert np.all(rel < 1e-9), rel
    for r in range(2):
        assert _rel(u[r], ug[r]) < 1e-6, r


STRIP_CASES = [
    # (n, parts, P, interface, centre)
    ((64, 64), (1, 4), 10, 0.3, (0.5, 0.875)),     # Theorem 3.6: interface below the source
    ((48, 48), (3, 1), 8, 0.4, (0.7, 0.45)),       # strip along x1
    ((12, 12, 18), (1, 1, 3), 3, 0.4, (0.5, 0.5, 0.8)),
]


@pytest.mark.parametrize("nsweeps", [2, 3])
@pytest.mark.parametrize("plan", ["direct", "trace"])
@pytest.mark.parametrize("case", STRIP_CASES, ids=lambda c: "x".join(map(str, c[1])))
def test_strip_sweeps_match_oracle(case, plan, nsweeps):
    """dds_sweep_strip (the one-dimensional sweeping DDM of Section 3.2, with the extra forward
    sweep of Theorem 3.6 at nsweeps = 3) against the oracle's strip sweeps: FP64 to 1e-10, the
    3xTF32 tensor-core path to the single-precision tolerance."""
    from oracle.sweep import strip_sweeps
    n, parts, P, interface, centre = case
    h = 1.0 / n[0]
    c = synth.medium_two_layer(n, h, interface=interface, axis=len(n) - 1)
    prob, f = _case(n, parts, P, 2 * np.pi * 3, c=c, centres=[centre])
    b = rhs_from_source(prob, extend_interior(prob, f))
    ref = ddm_solve(prob, b, sweeps=strip_sweeps(parts, nsweeps))
    for precision, tol in (("fp64", 1e-10), ("mixed", SINGLE_TOL["mixed"])):
        ctx = _ctx(prob, precision, plan)
        got = ctx.sweep_strip(_on_dev(ctx.extend(f)), nsweeps).cpu().numpy()
        assert _rel(got[0], ref[0]) < tol, precision


def test_strip_sweeps_reject_a_checkerboard():
    dds = _dds()
    prob, f = _case((32, 32), (2, 2), 4, 2 * np.pi * 2)
    ctx = _ctx(prob)
    with pytest.raises(dds.DDSError):
        ctx.sweep_strip(_on_dev(ctx.extend(f)), 3)


ZERO_SKIP_CASES = [
    # (n, parts, P, centres, plan): sources that leave most own-source solves zero
    ((128, 128), (8, 8), 4, [(0.2, 0.3), (0.7, 0.6), (0.5, 0.85)], "trace"),
    ((128, 128), (8, 8), 4, [(0.2, 0.3), (0.7, 0.6), (0.5, 0.85)], "direct"),
    ((240, 240), (2, 2), 8, [(0.3, 0.3)], "direct"),                   # 136-node lines
    ((24, 24, 24), (2, 2, 2), 4, [(0.3, 0.3, 0.3)], "direct"),         # 400-node planes
]


@pytest.mark.parametrize("case", ZERO_SKIP_CASES,
                         ids=lambda c: "x".join(map(str, c[1])) + "-" + c[4] + f"-{c[0][0]}")
def test_zero_work_skipping_drops_zero_solves_and_keeps_the_field(case):
    """Algorithm 2.1's 'if f_ij != 0 solve, else u_ij = 0': with skipping on, the local problems
    whose assembled right-hand side is zero are not solved (fewer solves counted), and the field
    is bit-identical in FP64 to the one with skipping off (direct plan; the trace plan's atomic
    slot accumulation has no fixed order, so there to rounding); the mixed path agrees with its
    unskipped self to single-precision rounding and with the oracle's DDM (which skips the same
    solves)."""
    n, parts, P, centres, plan = case
    prob, f = _case(n, parts, P, 2 * np.pi * 4, c=_medium("layer", n), centres=centres)
    b = rhs_from_source(prob, extend_interior(prob, f))
    record = []
    ref = ddm_solve(prob, b, 1, record=record)
    oracle_solved = sum(1 for rec in record if rec["solved"])
    for precision in ("fp64", "mixed"):
        ctx = _ctx(prob, precision, plan)
        fe = _on_dev(ctx.extend(f))
        ctx.local_solve_counts(reset=True)
        on = ctx.sweep(fe).cpu().numpy()
        solved, assembled = ctx.local_solve_counts(reset=True)
        ctx.set_zero_skip(False)
        off = ctx.sweep(fe).cpu().numpy()
        assert ctx.local_solve_counts() == (0, 0)
        assert 0 < solved < assembled, (solved, assembled)
        if precision == "fp64" and plan == "trace":
            # the trace slots are accumulated with atomics in no fixed order: rounding only
            for r in range(len(centres)):
                assert _rel(on[r], off[r]) < 1e-13
        elif precision == "fp64":
            assert np.array_equal(on, off)
            if len(centres) == 1:
                # one assembled local problem per (sweep, subdomain): the skipped ones are
                # exactly those the oracle finds zero
                assert assembled == len(record) and solved == oracle_solved, \
                    (assembled, len(record), solved, oracle_solved)
        else:
            for r in range(len(centres)):
                assert _rel(on[r], off[r]) < 1e-6
        for r in range(len(centres)):
            assert _rel(on[r], ref[r]) < (1e-10 if precision == "fp64" else SINGLE_TOL["mixed"])


def test_ddm_host_buffers_equal_device_buffers():
    prob, f = _case((48, 48), (2, 2), 8, 2 * np.pi * 3)
    ctx = _ctx(prob)
    fe = ctx.extend(f)
    u_dev = ctx.sweep(_on_dev(fe)).cpu().numpy()
    u_host = ctx.sweep(fe)
    assert isinstance(u_host, np.ndarray)
    assert np.array_equal(u_dev, u_host)


def test_ddm_batch_invariance_and_linearity():
    prob, f = _case((64, 64), (4, 4), 8, 2 * np.pi * 4, centres=[(0.2, 0.3), (0.7, 0.6), (0.5, 0.9)])
    # single precision: the trace step accumulates with float atomics (order not fixed), and a
    # 1-ulp change is amplified by the local solves' conditioning to ~1e-6 of the field
    for precision, tol in (("fp64", 1e-13), ("mixed", 1e-5), ("mixed_bf16", 1e-5),
                           ("mixed_fp32", 1e-5)):
        ctx = _ctx(prob, precision)
        fe = ctx.extend(f)
        batch = ctx.sweep(_on_dev(fe)).cpu().numpy()
        for r in range(3):
            alone = ctx.sweep(_on_dev(fe[r:r + 1])).cpu().numpy()[0]
            assert _rel(alone, batch[r]) < tol
        lin = ctx.sweep(_on_dev(fe[0:1] + 2 * fe[1:2])).cpu().numpy()[0]
        assert _rel(lin, batch[0] + 2 * batch[1]) < max(tol, 1e-12) * 10


def test_ddm_constant_medium_reproduces_global_solution():
    """Theorem 3.3 on the GPU: the DDM gap to the global PML solve is PML-level."""
    prob, f = _case((128, 128), (2, 2), 16, 2 * np.pi * 8)
    ctx = _ctx(prob, "fp64")
    u = ctx.sweep(_on_dev(ctx.extend(f))).cpu().numpy()[0]
    ug = global_solve(prob, rhs_from_source(prob, extend_interior(prob, f))[0])
    assert _rel(u, ug) < 3e-4


# ----------------------------------------------------------------------------- FGMRES --------

@pytest.mark.parametrize("precision", ["fp64", "mixed", "mixed_bf16", "mixed_fp32"])
def test_fgmres_matches_global_solve(precision):
    n = (96, 96)
    prob, f = _case(n, (4, 4), 10, 2 * np.pi * 6, c=_medium("layer", n),
                    centres=[(0.3, 0.7), (0.6, 0.2)])
    ctx = _ctx(prob, precision)
    u, it, rel = ctx.solve(_on_dev(ctx.extend(f)), tol=1e-9, maxit=40)
    ug = global_solve(prob, rhs_from_source(prob, extend_interior(prob, f)))
    u = u.cpu().numpy()
    assert np.all(rel < 1e-9), rel
    assert it <= 25
    for r in range(2):
        assert _rel(u[r], ug[r]) < 1e-6


def test_fgmres_one_subdomain_converges_in_one_iteration():
    prob, f = _case((40, 40), (1, 1), 8, 2 * np.pi * 3)
    ctx = _ctx(prob, "fp64")
    _, it, rel = ctx.solve(_on_dev(ctx.extend(f)), tol=1e-10, maxit=5)
    assert it == 1 and rel[0] < 1e-10


# ----------------------------------------------------------------------------- errors --------

def test_invalid_problem_is_rejected():
    dds = _dds()
    with pytest.raises(dds.DDSError):
        dds.Context((30, 30), 1 / 30, 10.0, np.ones((30, 30)), (4, 4), 4)   # 30 % 4 != 0
    with pytest.raises(dds.DDSError):
        dds.Context((30, 30), 1 / 30, 10.0, -np.ones((30, 30)), (3, 3), 4)  # c <= 0


# ----------------------------------------------------------------------------- large blocks --

def test_large_block_local_solve_and_ddm_2d():
    """Line blocks too large for the in-shared-memory factorisation (Mb = 136): the global-memory
    Schur / Gauss-Jordan path, checked by a local solve and a whole FP64 DDM."""
    n = (240, 240)
    prob, f = _case(n, (2, 2), 8, 2 * np.pi * 6, c=_medium("layer", n), centres=[(0.4, 0.3)])
    assert prob.M[0] == 136
    ctx = _ctx(prob, "fp64", "direct")
    rng = np.random.default_rng(3)
    dims = prob.M[::-1]
    b = rng.standard_normal((2,) + dims) + 1j * rng.standard_normal((2,) + dims)
    loc = LocalProblems(prob)
    x = ctx.local_solve(3, _on_dev(b)).cpu().numpy()
    assert _rel(x, loc.solve((1, 1), b)) < 1e-11
    bb = rhs_from_source(prob, extend_interior(prob, f))
    ref = ddm_solve(prob, bb, 1, loc)
    got = ctx.sweep(_on_dev(ctx.extend(f))).cpu().numpy()
    assert _rel(got[0], ref[0]) < 1e-10


def test_large_block_3d_ddm_and_fgmres():
    """3D with plane blocks of 400 nodes (7-point stencil, 2x2x2): FP64 DDM vs the oracle, and
    mixed FGMRES vs the global solve."""
    n = (24, 24, 24)
    prob, f = _case(n, (2, 2, 2), 4, 2 * np.pi * 2, centres=[(0.45, 0.55, 0.5)])
    assert prob.M[0] * prob.M[1] == 400
    ctx = _ctx(prob, "fp64", "direct")
    bb = rhs_from_source(prob, extend_interior(prob, f))
    ref = ddm_solve(prob, bb, 1)
    got = ctx.sweep(_on_dev(ctx.extend(f))).cpu().numpy()
    assert _rel(got[0], ref[0]) < 1e-10
    ctxm = _ctx(prob, "mixed", "direct")
    u, it, rel = ctxm.solve(_on_dev(ctx.extend(f)), tol=1e-9, maxit=30)
    ug = global_solve(prob, bb)
    assert rel[0] < 1e-9 and _rel(u.cpu().numpy()[0], ug[0]) < 1e-6


# ----------------------------------------------------------------------------- autotuner -----

def test_autotune_picks_a_valid_shape_and_keeps_results():
    """dds_autotune times every candidate launch shape and keeps the fastest; the DDM output
    after tuning equals the output before it to single-precision rounding."""
    n = (128, 128)
    prob, f = _case(n, (8, 8), 4, 2 * np.pi * 5, c=_medium("layer", n),
                    centres=[(0.2, 0.3), (0.7, 0.6), (0.5, 0.8)])
    ctx = _ctx(prob, "mixed", "trace")
    fe = _on_dev(ctx.extend(f))
    before = ctx.sweep(fe, 2).cpu().numpy()
    t = ctx.autotune(3, 2)
    assert t["panel_width"] in (8, 16, 32) and t["trace_ctas_per_sm"] in (0, 1, 2)
    assert t["panels_per_cta"] in (1, 2)
    assert {row[2] for row in t["table"]} == {0, 1, 2}   # CUDA-core 1/SM, 2/SM, tensor cores
    assert {row[1] for row in t["table"]} == {1, 2}      # one or two panels per CTA
    assert len(t["table"]) >= 2 and all(row[3] > 0 for row in t["table"])
    after = ctx.sweep(fe, 2).cpu().numpy()
    for r in range(3):
        assert _rel(after[r], before[r]) < 1e-5


def test_pinned_launch_shape_keeps_results():
    """dds_set_launch_shape pins each shape dds_autotune could choose; every pinned shape gives
    the oracle's DDM output to single-precision rounding, and a shape the context cannot run is
    rejected with DDS_EINVAL."""
    n = (128, 128)
    prob, f = _case(n, (8, 8), 4, 2 * np.pi * 5, c=_medium("layer", n),
                    centres=[(0.2, 0.3), (0.7, 0.6)])
    ctx = _ctx(prob, "mixed", "trace")
    fe = _on_dev(ctx.extend(f))
    want = ddm_solve(prob, rhs_from_source(prob, extend_interior(prob, f)), 2)
    for shape in ((8, 1, 1), (16, 2, 2), (32, 1, 0), (0, 1, 2)):
        ctx.set_launch_shape(*shape)
        got = ctx.sweep(fe, 2).cpu().numpy()
        for r in range(2):
            assert _rel(got[r], want[r]) < 1e-4, shape
    for bad in ((12, 1, 1), (0, 2, 1), (16, 1, 3)):
        with pytest.raises(_dds().DDSError):
            ctx.set_launch_shape(*bad)
