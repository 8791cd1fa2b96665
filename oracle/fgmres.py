"""Flexible GMRES with the DDM as right preconditioner (Section 5.2).

Test infrastructure only (see the package docstring).

The paper uses GMRES with one application of the diagonal sweeping DDM (2^n sweeps) as the
preconditioner and stops when the relative residual drops below 1e-6.  The oracle uses the
flexible variant (right preconditioning, Z stored) so that the same routine also serves an
inexact (mixed-precision) preconditioner: x0 = 0, classical Gram-Schmidt applied twice, Givens
rotations, no restart.
"""

from __future__ import annotations

import numpy as np


def fgmres(apply_A, apply_M, b, tol: float = 1e-6, maxit: int = 50):
    """Solve A x = b.  Returns (x, iterations, relative residual history).

    apply_A, apply_M map a 1-D complex vector to a 1-D complex vector.  The reported residual
    is the true relative residual ||b - A x|| / ||b|| of the returned x.
    """
    b = np.asarray(b, dtype=np.complex128).ravel()
    beta = np.linalg.norm(b)
    if beta == 0.0:
        return np.zeros_like(b), 0, [0.0]
    V = [b / beta]
    Z = []
    H = np.zeros((maxit + 1, maxit), dtype=np.complex128)
    cs = np.zeros(maxit, dtype=np.complex128)
    sn = np.zeros(maxit, dtype=np.complex128)
    g = np.zeros(maxit + 1, dtype=np.complex128)
    g[0] = beta
    hist = [1.0]
    k = 0
    for j in range(maxit):
        z = apply_M(V[j])
        Z.append(z)
        w = apply_A(z)
        for _ in range(2):                        # classical Gram-Schmidt, twice
            Vm = np.array(V)
            coef = Vm.conj() @ w
            w = w - coef @ Vm
            H[: j + 1, j] += coef
        H[j + 1, j] = np.linalg.norm(w)
        # apply previous rotations to the new column
        for i in range(j):
            t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
            H[i + 1, j] = -np.conj(sn[i]) * H[i, j] + np.conj(cs[i]) * H[i + 1, j]
            H[i, j] = t
        r = np.hypot(abs(H[j, j]), abs(H[j + 1, j]))
        if r == 0.0:
            cs[j], sn[j] = 1.0, 0.0
        else:
            cs[j] = H[j, j] / r
            sn[j] = H[j + 1, j] / r
            # choose the rotation so that H[j, j] becomes the real nonnegative r
            cs[j], sn[j] = np.conj(cs[j]), np.conj(sn[j])
        H[j, j] = cs[j] * H[j, j] + sn[j] * H[j + 1, j]
        H[j + 1, j] = 0.0
        g[j + 1] = -np.conj(sn[j]) * g[j]
        g[j] = cs[j] * g[j]
        k = j + 1
        hist.append(abs(g[j + 1]) / beta)
        if hist[-1] < tol:
            break
        nrm = np.linalg.norm(w)
        if nrm == 0.0:                            # lucky breakdown: the solution is exact
            break
        V.append(w / nrm)
    y = np.linalg.solve(np.triu(H[:k, :k]), g[:k])
    x = np.array(Z[:k]).T @ y
    res = np.linalg.norm(b - apply_A(x)) / beta
    hist[-1] = res
    return x, k, hist
