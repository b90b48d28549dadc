"""CPU FP64 oracle for the matrix-free shifted boundary method operator.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import this
package: only the tests, ``__graft_entry__.smoke()`` and the benchmark's
CPU-baseline / reference arm use it.  It shares no code with the CUDA library
(its own 1D tables, geometry, numbering and local matrices), and the library
never calls it.

What it computes is the plain definition of the operator written out: dense
element-by-element (EBE) local matrices from the quadrature formulas of the
weak form (Section 2, "Shifting boundary conditions" weak form; Section 3,
Algorithms 1-3), summed into y = A x, plus a CSR-assembled global matrix on
small meshes.  Every module cites the passage it follows.

Pinned by tests/test_oracle_*.py (closed forms, exact symbolic integrals,
invariants, brute force on tiny meshes, patch tests, convergence rates).
Parity unpinned: none -- every function carries at least one pin.
"""
