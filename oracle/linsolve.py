"""Direct solvers for the global and local PML problems.

Test infrastructure only (see the package docstring).

The paper solves every local problem with a sparse direct solver (MUMPS, Section 5).  The
oracle uses textbook library factorisations instead, none of which shares an algorithm with the
GPU path (which factors line blocks):
  * banded LU with partial pivoting (LAPACK zgbtrf / zgbtrs) on the natural ordering, whose
    bandwidth is the product of the tangential grid sizes;
  * SuperLU (scipy.sparse.linalg.splu) where the band storage would not fit in memory;
  * dense LU (numpy.linalg.solve) on tiny grids, used only to pin the other two.
"""

from __future__ import annotations

import numpy as np
import scipy.linalg.lapack as lapack
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .discretize import Problem, assemble_global

BAND_BYTES_LIMIT = 3 << 30  # above this the band storage is swapped for SuperLU


def band_width(grid_dims):
    """Half bandwidth of the natural (x1 fastest) ordering: product of all but the slowest dim."""
    return int(np.prod(grid_dims[1:]))


class BandedLU:
    """LU factorisation with partial pivoting of a banded matrix (LAPACK gbtrf)."""

    def __init__(self, A: sp.spmatrix, kl: int, ku: int):
        A = sp.coo_matrix(A)
        N = A.shape[0]
        ab = np.zeros((2 * kl + ku + 1, N), dtype=np.complex128)
        if np.any(A.row - A.col > kl) or np.any(A.col - A.row > ku):
            raise ValueError("matrix entries outside the declared band")
        ab[kl + ku + A.row - A.col, A.col] = A.data
        self.lu, self.piv, info = lapack.zgbtrf(ab, kl, ku)
        if info != 0:
            raise np.linalg.LinAlgError(f"zgbtrf failed, info={info}")
        self.kl, self.ku, self.N = kl, ku, N

    def solve(self, B):
        B = np.asarray(B, dtype=np.complex128)
        vec = B.ndim == 1
        B2 = B.reshape(self.N, -1)
        X, info = lapack.zgbtrs(self.lu, self.kl, self.ku, B2, self.piv)
        if info != 0:
            raise np.linalg.LinAlgError(f"zgbtrs failed, info={info}")
        return X[:, 0] if vec else X


class SparseLU:
    """SuperLU factorisation (used where the band storage would be too large)."""

    def __init__(self, A: sp.spmatrix):
        self.f = spla.splu(sp.csc_matrix(A))
        self.N = A.shape[0]

    def solve(self, B):
        B = np.asarray(B, dtype=np.complex128)
        return self.f.solve(B)


def factor(A: sp.spmatrix, grid_dims, method: str = "auto"):
    """Factor A on a grid of numpy shape grid_dims with the banded LU, or SuperLU if too big."""
    bw = band_width(grid_dims)
    N = A.shape[0]
    if method == "auto":
        method = "band" if (3 * bw + 1) * N * 16 <= BAND_BYTES_LIMIT else "splu"
    if method == "band":
        return BandedLU(A, bw, bw)
    if method == "splu":
        return SparseLU(A)
    raise ValueError(method)


def dense_solve(A: sp.spmatrix, b):
    """Brute force: dense LU of the full matrix (tiny grids only)."""
    return np.linalg.solve(A.toarray(), b)


def global_solve(prob: Problem, b_ext, method: str = "auto"):
    """Solve the global discrete PML problem A u = b (b is J-scaled) for one or more RHS.

    b_ext has shape (*G[::-1]) or (R, *G[::-1]); the result has the same shape.
    """
    A, _ = assemble_global(prob)
    dims = prob.G[::-1]
    key = ("global_factor", method)
    if key not in prob._cache:
        prob._cache[key] = factor(A, dims, method)
    fac = prob._cache[key]
    b = np.asarray(b_ext, dtype=np.complex128)
    lead = b.shape[:-prob.dim]
    B = b.reshape(-1, int(np.prod(dims))).T
    X = fac.solve(np.ascontiguousarray(B))
    return X.T.reshape(lead + dims)
