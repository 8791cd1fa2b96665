"""GB300-native trace-transfer diagonal sweeping DDM for the Helmholtz equation.

Leng & Ju, "Trace transfer-based diagonal sweeping domain decomposition method for the
Helmholtz equation" (arXiv 2003.02585): Algorithm 2.1 (2D) and Algorithm 4.1 (3D), used as a
direct solver or as a GMRES preconditioner (Section 5.2).

The compute path is the C-ABI library ``libdds.so`` (hand-written CUDA for sm_103a, declared in
``include/dds.h``); :mod:`paper_2003_02585_gb300.dds` is its thin ctypes binding.  Importing this
package does not load the library; :func:`paper_2003_02585_gb300.dds.load` does, and fails loudly
if it has not been built.
"""

__all__ = ["dds", "synth"]
