"""Section 5.1, smooth two-layer medium (kappa_down = 50 pi below x2 = 0.65, kappa_up = 62.5 pi
above 0.66, linear ramp between), 4 x 4 subdomains on meshes of 270^2, 540^2 and 1080^2 cells of
the box B_L = [0, 1]^2 (interior 8/9 of it, PML 1/18 per side), the smooth source of Eq. (5.1)
and its four-fold symmetric version.

The paper reports errors against the continuous solution falling at second order in L^2 and H^1
(its tables for this medium: rates 2.0), i.e. the DDM adds no error of its own above the
finite-difference one.  The continuous solution is not available here (absolute errors are not
pinned), so the rates are measured from successive meshes: e_h = ||u_h - R u_{h/2}|| with R the
average over the four fine cells of a coarse cell; for a second-order scheme
e_h / e_{h/2} -> 4.  The fields are the GPU's FGMRES solutions to 1e-10 (DDM preconditioner, two
rounds), far below the discretisation error; on the 270^2 and 540^2 meshes they are compared with
the oracle's global solve of the same discrete problem.  At the coarsest mesh the direct DDM (two rounds,
FP64, no Krylov) is compared with the same field: its own error must sit well below the
discretisation error, which is the paper's claim for this medium.
"""

import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.discretize import Problem, extend_interior, rhs_from_source
from oracle.linsolve import global_solve
from paper_2003_02585_gb300 import synth

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
TOTALS = (270, 540, 1080)
ORACLE_TOTALS = (270, 540)


@pytest.fixture(scope="module")
def fields():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2003_02585_gb300 import dds
    out = {}
    for total in TOTALS:
        n_int, pml, h = synth.conv_mesh(total)
        n = (n_int, n_int)
        c = synth.medium_smooth_two_layer(n, h)
        f = np.stack([synth.smooth_source(n, h), synth.smooth_source(n, h, symmetric=True)])
        ctx = dds.Context(n, h, synth.CONV_KAPPA_DOWN, c, (4, 4), pml, 30.0, precision="mixed")
        fe = torch.from_numpy(ctx.extend(f)).to(DEV)
        u, it, rel = ctx.solve(fe, tol=1e-10, maxit=30, rounds=2)
        assert np.all(np.asarray(rel) < 1e-10)
        entry = {"u": ctx.interior(u.cpu().numpy()), "h": h}
        if total in ORACLE_TOTALS:
            # the oracle's global solve of the same discrete problem (banded LU at 270^2, SuperLU
            # above), no domain decomposition
            prob = Problem(n, h, synth.CONV_KAPPA_DOWN, c, (4, 4), pml, 30.0)
            ug = global_solve(prob, rhs_from_source(prob, extend_interior(prob, f)))
            entry["oracle"] = ctx.interior(ug)
        if total == TOTALS[0]:
            ctx64 = dds.Context(n, h, synth.CONV_KAPPA_DOWN, c, (4, 4), pml, 30.0, precision="fp64")
            ud = ctx64.sweep(torch.from_numpy(ctx64.extend(f)).to(DEV), 2).cpu().numpy()
            entry["ddm"] = ctx64.interior(ud)
        out[total] = entry
    return out


def _restrict(uf):
    return 0.25 * (uf[:, 0::2, 0::2] + uf[:, 1::2, 0::2] + uf[:, 0::2, 1::2] + uf[:, 1::2, 1::2])


def _l2(v, h):
    return np.sqrt(h * h * np.sum(np.abs(v) ** 2, axis=(1, 2)))


def _h1(v, h):
    dx = np.diff(v, axis=2) / h
    dy = np.diff(v, axis=1) / h
    return np.sqrt(h * h * (np.sum(np.abs(dx) ** 2, axis=(1, 2)) + np.sum(np.abs(dy) ** 2, axis=(1, 2))))


def _printed_rates():
    """Rates the paper prints for this medium (tests/golden/section51_rates.txt)."""
    path = os.path.join(os.path.dirname(__file__), "golden", "section51_rates.txt")
    with open(path) as fh:
        rows = [ln.split() for ln in fh if ln.strip() and not ln.startswith("#")]
    return {r[0]: (float(r[1]), float(r[2])) for r in rows}


def test_second_order_rates_in_l2_and_h1(fields):
    printed = _printed_rates()
    want = np.array([printed["one_source"], printed["four_sources"]])   # [case][L2, H1]
    e_l2, e_h1 = [], []
    for coarse, fine in zip(TOTALS[:-1], TOTALS[1:]):
        uc, uf, h = fields[coarse]["u"], fields[fine]["u"], fields[coarse]["h"]
        d = uc - _restrict(uf)
        e_l2.append(_l2(d, h))
        e_h1.append(_h1(d, h))
    rate_l2 = np.log2(e_l2[0] / e_l2[1])
    rate_h1 = np.log2(e_h1[0] / e_h1[1])
    # one source (column 0) and four symmetric sources (column 1) against the printed rates
    assert np.all(np.abs(rate_l2 - want[:, 0]) < 0.2), (rate_l2, want)
    assert np.all(np.abs(rate_h1 - want[:, 1]) < 0.3), (rate_h1, want)


def test_fields_match_the_oracle_global_solve(fields):
    """The fields behind the rates are the discrete solutions: on the 270^2 and 540^2 meshes
    every field (one source, four sources) equals the oracle's global solve of the same PML
    problem to relative L2 1e-6."""
    for total in ORACLE_TOTALS:
        u, ug = fields[total]["u"], fields[total]["oracle"]
        for r in range(u.shape[0]):
            err = np.linalg.norm(u[r] - ug[r]) / np.linalg.norm(ug[r])
            assert err < 1e-6, (total, r, err)


def test_direct_ddm_error_is_below_the_discretisation_error(fields):
    h = fields[TOTALS[0]]["h"]
    u, ud = fields[TOTALS[0]]["u"], fields[TOTALS[0]]["ddm"]
    disc = _l2(u - _restrict(fields[TOTALS[1]]["u"]), h)      # ~ 3/4 of the h^2 error
    ddm = _l2(ud - u, h)
    assert np.all(ddm < 0.05 * disc), (ddm, disc)


def test_report_rates(fields, capsys):
    """Print the measured differences and rates (context for the paper's tables)."""
    rows = []
    for coarse, fine in zip(TOTALS[:-1], TOTALS[1:]):
        uc, uf, h = fields[coarse]["u"], fields[fine]["u"], fields[coarse]["h"]
        d = uc - _restrict(uf)
        rows.append((coarse, fine, _l2(d, h) / _l2(uf[:, ::2, ::2], h), _h1(d, h) / _h1(uf[:, ::2, ::2], h)))
    with capsys.disabled():
        for coarse, fine, l2, h1 in rows:
            print(f"\n{coarse}->{fine}: rel L2 diff {l2}, rel H1 diff {h1}")
