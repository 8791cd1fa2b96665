"""The allocation-free local solve (dds_local_solve_noalloc) against dds_local_solve.

Callers whose device memory belongs to another allocator, or who cannot accept the device-wide
synchronisation of cudaMalloc, use dds_local_solve_noalloc; its scratch is one fixed device
array inside libdds that every call shares.  This file runs last (pytest collects it after the
other test files), so a failure here does not hide any other test; it also passes on its own
in a fresh process.  Two calls in a row with different right-hand sides check that nothing of
the first call's scratch leaks into the second.
"""

import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2003_02585_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-11), ("mixed", 1e-4)])
def test_noalloc_local_solve_matches_local_solve(precision, tol):
    from paper_2003_02585_gb300 import dds
    n = (52, 52)
    ctx = dds.Context(n, 1 / 52, 2 * np.pi * 6, synth.medium_two_layer(n, 1 / 52), (2, 2), 12,
                      30.0, precision=precision)
    lib = dds.load()
    M = ctx.M
    rng = np.random.default_rng(7)
    for call, (sub, nrhs) in enumerate([(3, 3), (1, 2)]):        # two calls in a row
        b = rng.standard_normal((nrhs,) + M[::-1]) + 1j * rng.standard_normal((nrhs,) + M[::-1])
        bd = torch.from_numpy(b).to("cuda:0")
        ref = ctx.local_solve(sub, bd).cpu().numpy()
        out = torch.full_like(bd, complex(np.nan, np.nan))
        torch.cuda.synchronize()
        st = lib.dds_local_solve_noalloc(ctx._h, sub, ctypes.c_void_p(bd.data_ptr()), nrhs,
                                         ctypes.c_void_p(out.data_ptr()))
        assert st == 0, lib.dds_last_error(ctx._h).decode()
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got)), f"call {call}"
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < tol, f"call {call}"


def test_noalloc_rejects_oversize_and_host_buffers():
    from paper_2003_02585_gb300 import dds
    n = (52, 52)
    ctx = dds.Context(n, 1 / 52, 2 * np.pi * 6, synth.medium_constant(n), (2, 2), 12, 30.0)
    lib = dds.load()
    M = ctx.M
    big = torch.zeros((300,) + M[::-1], dtype=torch.complex128, device="cuda:0")
    st = lib.dds_local_solve_noalloc(ctx._h, 0, ctypes.c_void_p(big.data_ptr()), 300,
                                     ctypes.c_void_p(big.data_ptr()))
    assert st == 1 and b"static scratch" in lib.dds_last_error(ctx._h)
    host = np.zeros((1,) + M[::-1], dtype=np.complex128)
    st = lib.dds_local_solve_noalloc(ctx._h, 0, ctypes.c_void_p(host.ctypes.data), 1,
                                     ctypes.c_void_p(host.ctypes.data))
    assert st == 1
