"""Pins of the oracle's first-order Taylor extension (Section 2.1).

E1 u(x~) = u(x~) + d . grad u(x~), the Taylor series of the extension
truncated after the gradient term.  Pinned independently of the oracle's
quadrature: exact rational face integrals for constant shifts, exactness of
E1 on affine functions (where it must agree with the exact point evaluation,
itself pinned in test_oracle_local/test_oracle_operator), identity when the
shift is zero, and the patch test for affine solutions, with negative
controls for quadratics.
"""
from fractions import Fraction

import numpy as np
import pytest
import scipy.sparse.linalg as spla

import synthetic as S
from oracle import basis1d, local
from oracle.operator import Problem

from test_oracle_local import integ01, kron_lex, lagrange_polys


def _face_ref_taylor(p, d, k, s, delta, h, sigma):
    """Exact A_F with E1 psi_j = psi_j(x~) + sum_l delta_l d/dxi_l psi_j(x~)
    (reference shift delta, physical d = h delta): every term a Kronecker
    product of exact 1D factors."""
    L = lagrange_polys(basis1d.gll_nodes(p))
    n = p + 1
    xs = Fraction(s)
    sign = 2 * s - 1
    Mt = np.array([[integ01(L[i] * L[j]) for j in range(n)] for i in range(n)])
    Md = np.array([[integ01(L[i] * L[j].deriv()) for j in range(n)] for i in range(n)])
    v = np.array([float(L[i](xs)) for i in range(n)])
    dv = np.array([float(L[i].deriv()(xs)) for i in range(n)])
    dn = dv * sign / h                                   # dn psi at the face (physical)

    def kr(normal, tang):
        return kron_lex([normal if l == k else tang[l] for l in range(d)])

    tang = {l: Mt for l in range(d) if l != k}
    T1 = kr(np.outer(v, dn), tang)                       # psi_i dn psi_j
    out = np.zeros_like(T1)
    for test_n, coef in ((dn, -1.0), (v, sigma)):        # -dn psi_i E1 psi_j, sigma psi_i E1 psi_j
        E = kr(np.outer(test_n, v), tang)                # psi_j(x~)
        E = E + delta[k] * kr(np.outer(test_n, dv), tang)
        for m in tang:
            tm = dict(tang)
            tm[m] = Md
            E = E + delta[m] * kr(np.outer(test_n, v), tm)
        out += coef * E
    return h ** (d - 1) * (-T1 + out)


@pytest.mark.parametrize("d,p", [(2, 1), (2, 2), (2, 4), (3, 1), (3, 2), (3, 3)])
def test_taylor_face_matrix_exact_for_constant_shift(d, p):
    nodes = basis1d.gll_nodes(p)
    gq, gw = basis1d.gauss_rule(p + 1)
    h, sigma = 0.25, 37.5
    n = p + 1
    rng = np.random.default_rng(11)
    tmi = local.tensor_index(n, d - 1)
    w = np.prod(gw[tmi], axis=1)
    for k in range(d):
        for s in (0, 1):
            delta = rng.uniform(-0.6, 0.6, size=d)
            xt = np.zeros((1, n ** (d - 1), d))
            tang = [l for l in range(d) if l != k]
            for a, l in enumerate(tang):
                xt[0, :, l] = gq[tmi[:, a]]
            xt[0, :, k] = s
            shift = np.broadcast_to(h * delta, xt.shape).copy()
            A = local.face_matrices(nodes, xt, xt + delta, w, np.array([k]),
                                    np.array([float(s)]), h, sigma, shift=shift)[0]
            ref = _face_ref_taylor(p, d, k, s, delta, h, sigma)
            np.testing.assert_allclose(A, ref, atol=1e-11 * np.abs(ref).max())


CURVED = [
    (2, 2, 8, "ball", (0.05, -0.03, 0.73)),
    (2, 3, 6, "ball", (0.1, 0.0, 0.8)),
    (3, 2, 5, "ball", (0.02, 0.01, -0.03, 0.71)),
    (3, 3, 4) + S.ellipsoid((0.8, 0.6, 0.5), S.rotation_from_quaternion((1, 0.3, -0.2, 0.5))),
]


def _pair(case, dg=False):
    d, p, N, kind, geom = case
    return (Problem(d, p, N, kind, geom, dg=dg),
            Problem(d, p, N, kind, geom, dg=dg, extension="taylor1"))


@pytest.mark.parametrize("case", CURVED)
def test_taylor_equals_exact_on_affine_functions(case):
    """E1 is exact for affine u, so A_taylor u = A_exact u there; for a
    quadratic the two differ (the truncation is real)."""
    Pe, Pt = _pair(case)
    d = case[0]
    X = Pe.dof_coordinates()
    rng = np.random.default_rng(2)
    a, b = rng.normal(size=d), rng.normal()
    u = X @ a + b
    ye, yt = Pe.apply(u), Pt.apply(u)
    np.testing.assert_allclose(yt, ye, atol=1e-12 * np.abs(ye).max())
    q = X[:, 0] ** 2 + 0.5 * X[:, -1] ** 2
    ye, yt = Pe.apply(q), Pt.apply(q)
    assert np.abs(yt - ye).max() > 1e-6 * np.abs(ye).max()


def test_taylor_equals_exact_without_shift():
    """A box on mesh planes: d = 0, E1 = E = identity, the same operator."""
    for d in (2, 3):
        box = S.box((0.0,) * d, (0.5,) * d)
        Pe = Problem(d, 2, 8, *box)
        Pt = Problem(d, 2, 8, *box, extension="taylor1")
        Ae, At = Pe.assemble().toarray(), Pt.assemble().toarray()
        np.testing.assert_allclose(At, Ae, atol=1e-13 * np.abs(Ae).max())


def test_taylor_dg_equals_exact_on_affine_functions():
    Pe, Pt = _pair((3, 2, 5, "torus", (0.6, 0.25)), dg=True)
    X = Pe.dof_coordinates()
    u = 0.3 * X[:, 0] - 1.1 * X[:, 1] + 0.7 * X[:, 2] + 0.2
    ye, yt = Pe.apply(u), Pt.apply(u)
    np.testing.assert_allclose(yt, ye, atol=1e-12 * np.abs(ye).max())


@pytest.mark.parametrize("case", CURVED[:3])
def test_taylor_patch_test_affine(case):
    """Affine u*, f = 0, g = u*(x_q): E1 u* = u*(x_q) exactly, so the SBM
    solution with the first-order extension reproduces u*; a quadratic u*
    (which the exact extension reproduces for p >= 2) is not reproduced."""
    d = case[0]
    _, Pt = _pair(case)
    a = np.linspace(0.4, -0.9, d)
    u = lambda X: X @ a + 0.25
    f = lambda X: np.zeros(X.shape[:-1])
    A = Pt.assemble().tocsc()
    uh = spla.spsolve(A, Pt.rhs(f, u))
    ref = Pt.interpolate(u)
    assert np.abs(uh - ref).max() < 1e-9 * max(1.0, np.abs(ref).max())
    uq = lambda X: X[..., 0] ** 2 - X[..., 1] ** 2          # harmonic
    uh = spla.spsolve(A, Pt.rhs(f, uq))
    assert np.abs(uh - Pt.interpolate(uq)).max() > 1e-7
