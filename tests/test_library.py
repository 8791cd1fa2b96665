"""The C-ABI library builds, loads and exports every entry point include/dds.h declares.

No compute call is made here (no GPU needed).
"""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "dds.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dds_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ["dds_setup", "dds_sweep", "dds_solve", "dds_apply", "dds_destroy",
              "dds_last_error", "dds_set_stream", "dds_local_solve"]:
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2003_02585_gb300 import build, dds
    try:
        path = build.build()
    except RuntimeError as e:  # pragma: no cover - toolkit missing
        pytest.skip(f"cannot build libdds: {e}")
    lib = ctypes.CDLL(path)
    for name in _declared():
        assert hasattr(lib, name), name
    assert sorted(dds.EXPORTS) == _declared()


def test_binding_rejects_missing_library(tmp_path):
    from paper_2003_02585_gb300 import dds
    with pytest.raises(RuntimeError):
        dds.load(str(tmp_path / "nope.so")) if dds._lib is None else (_ for _ in ()).throw(
            RuntimeError("already loaded"))


def test_local_solve_arguments_are_checked_before_the_call():
    """The binding refuses local-solve buffers whose dtype, shape or memory kind would make the
    library read or write past them (it touches nrhs * prod(M) * 16 bytes at each address)."""
    import numpy as np
    torch = pytest.importorskip("torch")
    from paper_2003_02585_gb300 import dds
    M, dim = (30, 28), 2
    ok = torch.zeros((3, 28, 30), dtype=torch.complex128)
    assert dds.local_field_count(ok, M, dim) == 3
    assert dds.local_field_count(ok[0], M, dim) == 1
    assert dds.local_field_count(np.zeros((28, 30), np.complex128), M, dim) == 1
    with pytest.raises(TypeError):
        dds.local_field_count(ok.to(torch.complex64), M, dim)
    with pytest.raises(TypeError):
        dds.local_field_count(np.zeros((28, 30), np.complex64), M, dim)
    with pytest.raises(ValueError):
        dds.local_field_count(torch.zeros((3, 30, 28), dtype=torch.complex128), M, dim)
    with pytest.raises(ValueError):
        dds.local_field_count(torch.zeros((3, 28, 60), dtype=torch.complex128)[:, :, ::2],
                              M, dim)
    with pytest.raises(ValueError):
        dds.local_field_count(torch.zeros((0, 28, 30), dtype=torch.complex128), M, dim)
    # allocation-free entry point: device memory only, and out must match b
    with pytest.raises(TypeError):
        dds.check_noalloc_pair(ok, ok.clone(), M, dim, 0)
    with pytest.raises(TypeError):
        dds.check_noalloc_pair(np.zeros((28, 30), np.complex128),
                               np.zeros((28, 30), np.complex128), M, dim, 0)
