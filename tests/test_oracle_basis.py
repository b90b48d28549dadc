"""Pins of the oracle's 1D tables: closed forms, exactness, interpolation identities."""
import math
import os

import numpy as np
import pytest

from oracle import basis1d

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_gll():
    out = {}
    for line in open(os.path.join(GOLDEN, "gll_nodes.txt")):
        if line.startswith("#") or not line.strip():
            continue
        p, *expr = line.split()
        out[int(p)] = [eval(e, {"sqrt": math.sqrt}) for e in expr]
    return out


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_gll_closed_forms(p):
    ref = _golden_gll()[p]
    np.testing.assert_allclose(basis1d.gll_nodes(p), ref, rtol=0, atol=1e-15)


def _legendre_recurrence(p, t):
    """P_p(t) and P_p'(t) by the three-term (Bonnet) recurrence."""
    P0, P1 = np.ones_like(t), t
    if p == 0:
        return P0, np.zeros_like(t)
    for k in range(1, p):
        P0, P1 = P1, ((2 * k + 1) * t * P1 - k * P0) / (k + 1)
    with np.errstate(divide="ignore", invalid="ignore"):
        dP = p * (t * P1 - P0) / (t * t - 1.0)
    return P1, dP


@pytest.mark.parametrize("p", range(2, 9))
def test_gll_are_roots_of_legendre_derivative(p):
    x = basis1d.gll_nodes(p)
    t = 2 * x[1:-1] - 1
    _, dP = _legendre_recurrence(p, t)
    assert np.max(np.abs(dP)) < 1e-12
    assert np.all(np.diff(x) > 0) and x[0] == 0.0 and x[-1] == 1.0


@pytest.mark.parametrize("p", range(1, 9))
def test_gll_lobatto_rule_exact(p):
    # Lobatto weights 2/(p(p+1) P_p(t_i)^2) integrate degree 2p-1 exactly
    t = 2 * basis1d.gll_nodes(p) - 1
    P, _ = _legendre_recurrence(p, t)
    w = 2.0 / (p * (p + 1) * P * P)
    for k in range(2 * p):
        exact = (1 - (-1) ** (k + 1)) / (k + 1)
        assert abs(np.sum(w * t ** k) - exact) < 1e-13


@pytest.mark.parametrize("n", range(1, 10))
def test_gauss_exactness(n):
    x, w = basis1d.gauss_rule(n)
    assert abs(w.sum() - 1.0) < 4e-15
    for k in range(2 * n):
        assert abs(np.sum(w * x ** k) - 1.0 / (k + 1)) < 4e-15
    # degree 2n: the error is exactly the Gauss remainder (n!)^4/((2n+1)((2n)!)^2)
    # on [0,1] (f^(2n) = (2n)! constant), which also fixes the rule's size
    err = 1.0 / (2 * n + 1) - np.sum(w * x ** (2 * n))
    rem = math.factorial(n) ** 4 / ((2 * n + 1) * math.factorial(2 * n) ** 2)
    assert abs(err - rem) < 1e-6 * rem + 4e-15


@pytest.mark.parametrize("p", range(1, 8))
def test_lagrange_identities(p):
    nodes = basis1d.gll_nodes(p)
    np.testing.assert_allclose(basis1d.lagrange(nodes, nodes), np.eye(p + 1), atol=1e-14)
    t = np.linspace(-1.0, 2.0, 37)      # includes extrapolation outside [0,1]
    phi = basis1d.lagrange(nodes, t)
    dphi = basis1d.lagrange_deriv(nodes, t)
    for k in range(p + 1):
        # exact reproduction of every polynomial of degree <= p, also outside [0,1]
        np.testing.assert_allclose(phi @ nodes ** k, t ** k, atol=1e-11)
        dk = k * t ** (k - 1) if k else np.zeros_like(t)
        np.testing.assert_allclose(dphi @ nodes ** k, dk, atol=1e-9)
    # degree p+1 is not reproduced (the basis has the right size)
    assert np.max(np.abs(phi @ nodes ** (p + 1) - t ** (p + 1))) > 1e-3


def test_lagrange_derivative_matches_difference_quotient():
    nodes = basis1d.gll_nodes(5)
    t = np.array([-0.3, 0.1, 0.77, 1.4])
    e = 1e-6
    fd = (basis1d.lagrange(nodes, t + e) - basis1d.lagrange(nodes, t - e)) / (2 * e)
    np.testing.assert_allclose(basis1d.lagrange_deriv(nodes, t), fd, atol=1e-6)


@pytest.mark.parametrize("p", range(1, 7))
def test_face_gauss_round_trip_is_the_exact_mass(p):
    """With p+1 Gauss points the round trip 'interpolate nodal values to the
    Gauss points, weight, interpolate back' is the exact 1D mass matrix
    S^T diag(w) S = M, M_ij = int_0^1 phi_i phi_j: the identity the face
    kernels use to integrate the face terms that are linear in nodal traces
    in mass form.  M is computed independently by a (2p+4)-point Gauss rule;
    with p points instead of p+1 the identity fails (degree 2p exceeds
    2p-1)."""
    nodes = basis1d.gll_nodes(p)
    g, w = basis1d.gauss_rule(p + 1)
    S = basis1d.lagrange(nodes, g)                     # [q][j] = phi_j(g_q)
    gh, wh = basis1d.gauss_rule(2 * p + 4)
    Sh = basis1d.lagrange(nodes, gh)
    M = Sh.T @ np.diag(wh) @ Sh
    np.testing.assert_allclose(S.T @ np.diag(w) @ S, M, atol=1e-14)
    gl, wl = basis1d.gauss_rule(p)
    Sl = basis1d.lagrange(nodes, gl)
    assert np.abs(Sl.T @ np.diag(wl) @ Sl - M).max() > 1e-6
