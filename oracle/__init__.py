"""CPU FP64 oracle for the trace-transfer diagonal sweeping DDM (Leng & Ju, arXiv 2003.02585).

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow, obviously correct reference the
GPU path is checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s
``cpu_baseline`` / ``--impl reference`` legs may import it.  The product library
(``paper_2003_02585_gb300`` and its CUDA sources) never imports, links or calls anything here,
and this package imports nothing from the product.

Modules
-------
discretize  PML profile (Eq. 2.1), complex stretching, the J-scaled 5/7-point operator of the
            PML equation (Eq. 2.3 in 2D, Eq. 4.1 in 3D), subdomain boxes and the wave-number
            extension (Eq. 2.8).
linsolve    Banded LU (LAPACK gbtrf/gbtrs), SuperLU and dense solves; used for the global PML
            problem and for every local subdomain problem.
sweep       Step sets (Eq. 2.10-2.11, 4.3-4.4), the trace routing of Rules 2.4/2.5 and 4.1/4.2,
            and Algorithm 2.1 / Algorithm 4.1 written out step by step.
fgmres      Right-preconditioned flexible GMRES with the DDM as preconditioner (Section 5.2).

All arithmetic is complex128.  Every reading of a point where the paper is silent or ambiguous
is stated in the docstring of the function that makes it.

Parity status: every function here is pinned by a ``-m "not gpu"`` test against a closed form,
a library routine, a theorem of the paper or brute force (see tests/test_oracle_*.py).
"""

from .discretize import Problem, assemble_global, assemble_local, rhs_from_source  # noqa: F401
from .sweep import (sweep_directions, step_set, route_table, ddm_solve,  # noqa: F401
                    similar_direction, sweep_usable)
from .linsolve import global_solve  # noqa: F401
from .fgmres import fgmres  # noqa: F401
