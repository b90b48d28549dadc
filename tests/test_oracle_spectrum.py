"""Spectra of the SBM matrices behind the batched-solve workload.

The operator is nonsymmetric (shifted trial functions, Section 2.1) and need
not be positive definite: on coarse meshes the exact extension evaluates
degree-p polynomials well outside the cell and, with the penalty 10 p^2 / h,
the spectrum can reach into the left half-plane.  The batched solver runs
BiCGStab, so the batched-solve workload keeps the problems where it works;
these tests pin the selection with library routines (LAPACK eigenvalues of
the oracle's assembled matrix, SciPy's BiCGStab) and that the excluded cases
are real (an indefinite problem; a positive-real one on which BiCGStab
diverges)."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import synthetic as S
from oracle.operator import Problem


def _matrix(w):
    return Problem.from_workload(w).assemble()


@pytest.mark.parametrize("w", S.solve_batch(), ids=lambda w: w.name)
def test_solve_batch_is_positive_real_and_bicgstab_converges(w):
    A = _matrix(w)
    assert np.linalg.eigvals(A.toarray()).real.min() > 0.0
    b = S.random_vector(w.seed + 7, A.shape[0], "uniform")
    x, info = spla.bicgstab(A.tocsr(), b, rtol=1e-10, maxiter=5000)
    assert info == 0
    assert np.linalg.norm(b - A @ x) <= 1e-10 * np.linalg.norm(b) * 1.01


def test_excluded_problems():
    ws = S.batched_ellipsoids(nprob=24, n_range=(8, 14), p_range=(2, 3))
    w = ws[2]                               # p = 3, N = 8: indefinite
    assert (w.degree, w.cells) == (3, 8)
    ev = np.linalg.eigvals(_matrix(w).toarray())
    assert (ev.real < 0).sum() >= 10
    w = ws[21]                              # p = 3, N = 8: positive real, BiCGStab diverges
    A = _matrix(w)
    assert np.linalg.eigvals(A.toarray()).real.min() > 0.0
    b = S.random_vector(w.seed + 7, A.shape[0], "uniform")
    x, info = spla.bicgstab(A.tocsr(), b, rtol=1e-10, maxiter=2000)
    assert info != 0
    assert not (np.linalg.norm(b - A @ x) <= 1e-6 * np.linalg.norm(b))
