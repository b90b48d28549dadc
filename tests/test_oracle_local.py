"""Pins of the oracle's local matrices against exact integrals and textbook forms.

The reference values here never use the oracle's quadrature loops: they come
from exact rational polynomial integration (Fraction coefficients, or sympy)
of the weak-form terms, written in tensor-product form.
"""
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import basis1d, local

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


class RPoly:
    """Polynomial with exact rational (Fraction) coefficients, lowest degree first."""

    def __init__(self, c):
        self.c = [Fraction(v) for v in c] or [Fraction(0)]

    def __mul__(self, o):
        if not isinstance(o, RPoly):
            return RPoly([v * Fraction(o) for v in self.c])
        out = [Fraction(0)] * (len(self.c) + len(o.c) - 1)
        for i, a in enumerate(self.c):
            for j, b in enumerate(o.c):
                out[i + j] += a * b
        return RPoly(out)

    def __call__(self, x):
        x = Fraction(x)
        acc = Fraction(0)
        for v in reversed(self.c):
            acc = acc * x + v
        return acc

    def deriv(self):
        return RPoly([i * v for i, v in enumerate(self.c)][1:])

    def shifted(self, delta):
        """t -> P(t + delta)."""
        out = RPoly([0])
        power = RPoly([1])
        lin = RPoly([Fraction(delta), 1])
        for v in self.c:
            out = RPoly([a + b for a, b in zip(out.c + [Fraction(0)] * len(power.c),
                                               (power * v).c + [Fraction(0)] * len(out.c))])
            power = power * lin
        return out


def lagrange_polys(nodes):
    """Exact Lagrange polynomials of the (double) nodes, in rational arithmetic."""
    fn = [Fraction(float(x)) for x in nodes]
    out = []
    for i, xi in enumerate(fn):
        P = RPoly([1])
        for m, xm in enumerate(fn):
            if m != i:
                P = P * RPoly([-xm / (xi - xm), 1 / (xi - xm)])
        out.append(P)
    return out


def integ01(P):
    return float(sum(v / (k + 1) for k, v in enumerate(P.c)))


def mass_stiff_1d(p):
    L = lagrange_polys(basis1d.gll_nodes(p))
    n = p + 1
    M = np.array([[integ01(L[i] * L[j]) for j in range(n)] for i in range(n)])
    K = np.array([[integ01(L[i].deriv() * L[j].deriv()) for j in range(n)] for i in range(n)])
    return M, K


def kron_lex(mats):
    """Kronecker product for lexicographic index with axis 0 fastest."""
    out = mats[0]
    for m in mats[1:]:
        out = np.kron(m, out)
    return out


def _setup(p):
    nodes = basis1d.gll_nodes(p)
    gq, gw = basis1d.gauss_rule(p + 1)
    return nodes, gq, gw


@pytest.mark.parametrize("d", [2, 3])
@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6])
def test_cell_matrix_equals_exact_tensor_laplacian(d, p):
    if d == 3 and p > 5:
        pytest.skip("size")
    h = 0.37
    nodes, gq, gw = _setup(p)
    A = local.cell_matrix(nodes, gq, gw, d, h)
    M, K = mass_stiff_1d(p)
    ref = np.zeros_like(A)
    for k in range(d):
        ref += kron_lex([K if l == k else M for l in range(d)])
    ref *= h ** (d - 2)
    np.testing.assert_allclose(A, ref, atol=2e-13 * np.abs(ref).max())
    # invariants: annihilates constants, symmetric, positive semidefinite, 1D kernel
    assert np.abs(A @ np.ones(len(A))).max() < 1e-12 * np.abs(A).max()
    np.testing.assert_allclose(A, A.T, atol=1e-14 * np.abs(A).max())
    ev = np.linalg.eigvalsh(A)
    assert ev[0] > -1e-12 * ev[-1] and ev[1] > 1e-8 * ev[-1]


def _golden_q1():
    rows = {}
    for line in open(os.path.join(GOLDEN, "q1_stiffness.txt")):
        if line.startswith("#") or not line.strip():
            continue
        parts = line.split()
        rows[int(parts[0])] = [float(Fraction(v)) for v in parts[2:]]
    return rows


@pytest.mark.parametrize("d", [2, 3])
def test_q1_textbook(d):
    h = 0.5
    nodes, gq, gw = _setup(1)
    A = local.cell_matrix(nodes, gq, gw, d, h)
    vals = _golden_q1()[d]
    mi = local.tensor_index(2, d)
    scale = h ** (d - 2)
    for i in range(2 ** d):
        for j in range(2 ** d):
            ndiff = int(np.sum(mi[i] != mi[j]))
            assert abs(A[i, j] - scale * vals[ndiff]) < 1e-14


def _face_ref(p, d, k, s, delta, h, sigma):
    """Exact A_F for a face whose shifted points are x~_q + delta (constant).

    Tensor form: product over axes of 1D exact integrals (tangential axes) or
    1D values at the face coordinate (normal axis).
    """
    nodes = basis1d.gll_nodes(p)
    L = lagrange_polys(nodes)
    n = p + 1
    sign = 2 * s - 1
    xs = float(s)
    # tangential 1D factors
    Mt = {}
    Ms = {}
    for l in range(d):
        if l == k:
            continue
        Mt[l] = np.array([[integ01(L[i] * L[j]) for j in range(n)] for i in range(n)])
        Ms[l] = np.array([[integ01(L[i] * L[j].shifted(delta[l]))
                           for j in range(n)] for i in range(n)])
    v = np.array([float(L[i](xs)) for i in range(n)])
    dv = np.array([float(L[i].deriv()(xs)) for i in range(n)]) * sign / h
    vs = np.array([float(L[j](Fraction(xs) + Fraction(delta[k]))) for j in range(n)])
    # three terms, each a Kronecker product over axes
    def kr(normal, tang):
        return kron_lex([normal if l == k else tang[l] for l in range(d)])
    T1 = kr(np.outer(v, dv), Mt)          # psi_i(x~) dn psi_j(x~)
    T2 = kr(np.outer(dv, vs), Ms)         # dn psi_i(x~) psi_j(x~ + delta)
    T3 = kr(np.outer(v, vs), Ms)          # psi_i(x~) psi_j(x~ + delta)
    return h ** (d - 1) * (-T1 - T2 + sigma * T3)


@pytest.mark.parametrize("d,p", [(2, 1), (2, 2), (2, 4), (2, 6), (3, 1), (3, 2), (3, 4)])
def test_face_matrix_exact_for_constant_shift(d, p):
    nodes, gq, gw = _setup(p)
    h, sigma = 0.25, 37.5
    n = p + 1
    rng = np.random.default_rng(5)
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
            A = local.face_matrices(nodes, xt, xt + delta, w, np.array([k]),
                                    np.array([float(s)]), h, sigma)[0]
            ref = _face_ref(p, d, k, s, delta, h, sigma)
            np.testing.assert_allclose(A, ref, atol=1e-11 * np.abs(ref).max())


def test_face_matrix_sympy_rational_p2():
    """Exact rational check (p = 2, GLL nodes 0, 1/2, 1) of A_F in 2D."""
    sympy = pytest.importorskip("sympy")
    t = sympy.Symbol("t")
    R = sympy.Rational
    nodes = [R(0), R(1, 2), R(1)]

    def lag(i, x):
        e = R(1)
        for m, xm in enumerate(nodes):
            if m != i:
                e *= (x - xm) / (nodes[i] - xm)
        return e

    h, sigma = R(1, 4), R(75, 2)
    dx, dy = R(3, 10), R(-1, 5)          # shift, face k = 0, s = 1 (x = 1)
    n = 3
    ref = np.zeros((9, 9))
    for i in range(9):
        i0, i1 = i % 3, i // 3
        for j in range(9):
            j0, j1 = j % 3, j // 3
            x = sympy.Symbol("x")
            psi_i = lag(i0, x) * lag(i1, t)
            psi_j = lag(j0, x) * lag(j1, t)
            dn_i = sympy.diff(psi_i, x) / h
            dn_j = sympy.diff(psi_j, x) / h
            psi_j_shift = psi_j.subs({x: 1 + dx, t: t + dy}, simultaneous=True)
            integrand = (-psi_i * dn_j - dn_i * psi_j_shift.subs(x, 1)
                         + sigma * psi_i * psi_j_shift).subs(x, 1)
            ref[i, j] = float(h * sympy.integrate(sympy.expand(integrand), (t, 0, 1)))
    nodes_f = basis1d.gll_nodes(2)
    gq, gw = basis1d.gauss_rule(3)
    xt = np.zeros((1, 3, 2))
    xt[0, :, 0] = 1.0
    xt[0, :, 1] = gq
    A = local.face_matrices(nodes_f, xt, xt + np.array([0.3, -0.2]), gw, np.array([0]),
                            np.array([1.0]), 0.25, 37.5)[0]
    np.testing.assert_allclose(A, ref, atol=1e-12 * np.abs(ref).max())


@pytest.mark.parametrize("d,p", [(2, 1), (2, 3), (3, 2), (3, 3)])
def test_dg_face_block_exact(d, p):
    nodes, gq, gw = _setup(p)
    h, sf = 0.5, 9.0
    L = lagrange_polys(nodes)
    n = p + 1
    M = np.array([[integ01(L[i] * L[j]) for j in range(n)] for i in range(n)])
    v1 = np.array([float(L[i](1)) for i in range(n)])   # K1 sees the face at xi_k = 1
    v2 = np.array([float(L[i](0)) for i in range(n)])
    d1 = np.array([float(L[i].deriv()(1)) for i in range(n)]) / h
    d2 = np.array([float(L[i].deriv()(0)) for i in range(n)]) / h
    J = [v1, -v2]
    Av = [0.5 * d1, 0.5 * d2]
    for k in range(d):
        B = local.dg_face_matrix(nodes, gq, gw, d, k, h, sf)
        nd = n ** d
        for a in range(2):
            for b in range(2):
                normal = sf * np.outer(J[a], J[b]) - np.outer(J[a], Av[b]) - np.outer(Av[a], J[b])
                ref = h ** (d - 1) * kron_lex([normal if l == k else M for l in range(d)])
                blk = B[a * nd:(a + 1) * nd, b * nd:(b + 1) * nd]
                np.testing.assert_allclose(blk, ref, atol=1e-11 * np.abs(ref).max())
        np.testing.assert_allclose(B, B.T, atol=1e-12 * np.abs(B).max())
        assert np.abs(B @ np.ones(2 * nd)).max() < 1e-11 * np.abs(B).max()
