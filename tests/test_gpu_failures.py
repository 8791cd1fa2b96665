"""Failure detection without a GPU fault: bounded waits that give up, a device-memory budget
that is exceeded, and a right-hand side that carries a NaN.

  * A small poll limit (dds_set_wait_limit) makes the level-completion waits of the cooperative
    trace launch run out: the call returns DDS_ETIMEOUT promptly, the launch ends (no hang, no
    fault), and after the default limit is restored the next call returns DDS_OK with the oracle's
    field.  Both trace kernels (tensor-core and CUDA-core) are exercised.
  * A budget below what a call needs (dds_set_memory_budget) makes the call return DDS_ENOMEM;
    the context stays usable for calls that fit.
  * A NaN in one right-hand side of a batch leaves every other right-hand side's field as it is
    without the NaN (the columns of every kernel are independent), and the bad right-hand side
    comes back as a NaN field (dds_sweep) or with a NaN relative residual (dds_solve).
"""

import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.discretize import Problem, extend_interior, rhs_from_source
from oracle.sweep import ddm_solve
from paper_2003_02585_gb300 import synth

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def _case(nrhs=3, n=(128, 128), parts=(8, 8), P=4):
    h = 1.0 / n[0]
    rng = np.random.default_rng(11)
    centres = [tuple(x) for x in rng.uniform(0.15, 0.85, size=(nrhs, 2))]
    c = synth.medium_two_layer(n, h)
    f = synth.gaussian_sources(n, h, centres, 2 * h)
    prob = Problem(n, h, 2 * np.pi * 5, c, parts, P, 30.0)
    return prob, f


def _ctx(prob, precision, plan="trace"):
    from paper_2003_02585_gb300 import dds
    return dds.Context(prob.n, prob.h, prob.omega, prob.c, prob.parts, prob.pml_cells,
                       prob.pml_strength, precision=precision, plan=plan)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("precision,tol", [("mixed", 1e-4), ("fp64", 1e-10)])
def test_level_wait_timeout_is_reported_and_the_context_recovers(precision, tol):
    from paper_2003_02585_gb300 import dds
    prob, f = _case()
    b = rhs_from_source(prob, extend_interior(prob, f))
    ref = ddm_solve(prob, b, 2)
    ctx = _ctx(prob, precision)
    fe = torch.from_numpy(ctx.extend(f)).to(DEV)
    ctx.set_wait_limit(1)              # one poll: the 43 level waits of two rounds run out
    statuses = []
    for _ in range(3):
        t0 = time.perf_counter()
        try:
            ctx.sweep(fe, 2)
            statuses.append(0)
        except dds.DDSError as e:
            statuses.append(e.status)
        assert time.perf_counter() - t0 < 30.0
        if statuses[-1] == 5:
            break
    assert 5 in statuses, statuses     # DDS_ETIMEOUT
    ctx.set_wait_limit(0)              # the default limit
    got = ctx.sweep(fe, 2).cpu().numpy()
    for r in range(f.shape[0]):
        assert _rel(got[r], ref[r]) < tol, r


def test_memory_budget_gives_enomem_and_the_context_stays_usable():
    from paper_2003_02585_gb300 import dds
    prob, f = _case(nrhs=2)
    ctx = _ctx(prob, "mixed")
    fe = torch.from_numpy(ctx.extend(f)).to(DEV)
    u_small, _, rel = ctx.solve(fe, tol=1e-8, maxit=20, rounds=2)
    held = ctx.info()["device_bytes"]
    assert held > 0
    assert ctx.set_memory_budget(held + (1 << 20)) == held
    big = torch.from_numpy(ctx.extend(np.repeat(f, 16, axis=0))).to(DEV)   # 32 RHS
    with pytest.raises(dds.DDSError) as e:
        ctx.solve(big, tol=1e-8, maxit=20, rounds=2)
    assert e.value.status == 2          # DDS_ENOMEM
    assert ctx.info()["device_bytes"] <= held + (1 << 20)
    u2, _, rel2 = ctx.solve(fe, tol=1e-8, maxit=20, rounds=2)   # fits again
    assert np.all(rel2 < 1e-8)
    for r in range(2):
        assert _rel(u2[r].cpu().numpy(), u_small[r].cpu().numpy()) < 1e-6
    ctx.set_memory_budget(0)
    u3, _, rel3 = ctx.solve(big, tol=1e-8, maxit=20, rounds=2)
    assert np.all(rel3 < 1e-8)


@pytest.mark.parametrize("precision", ["fp64", "mixed", "mixed_bf16"])
def test_nan_right_hand_side_leaves_the_others_intact(precision):
    prob, f = _case(nrhs=3)
    ctx = _ctx(prob, precision)
    fe = ctx.extend(f)
    clean = torch.from_numpy(fe).to(DEV)
    dirty = fe.copy()
    G = ctx.G
    dirty[1, G[1] // 2, G[0] // 3] = complex(np.nan, 0.0)
    dirty = torch.from_numpy(dirty).to(DEV)
    tol = 1e-12 if precision == "fp64" else 1e-5
    u_clean = ctx.sweep(clean, 2).cpu().numpy()
    u_dirty = ctx.sweep(dirty, 2).cpu().numpy()
    assert np.all(np.isnan(u_dirty[1]))        # the bad right-hand side is reported as NaN
    for r in (0, 2):
        assert np.all(np.isfinite(u_dirty[r]))
        assert _rel(u_dirty[r], u_clean[r]) < tol, r
    # FGMRES: the NaN column never converges (DDS_ENOCONV after maxit), the others do, with the
    # fields they have alone
    s_clean, _, rel_c = ctx.solve(clean, tol=1e-8, maxit=12, rounds=2)
    s_dirty, _, rel_d = ctx.solve(dirty, tol=1e-8, maxit=12, rounds=2)
    s_clean, s_dirty = s_clean.cpu().numpy(), s_dirty.cpu().numpy()
    assert np.isnan(rel_d[1]) and np.all(np.isnan(s_dirty[1]))
    for r in (0, 2):
        assert rel_d[r] < 1e-8
        assert _rel(s_dirty[r], s_clean[r]) < 1e-7, r
