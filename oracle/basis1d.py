"""1D ingredients of the tensor-product Q_p basis and Gauss quadrature (oracle).

Section 3.1 (tensor-product structure): basis functions on the reference
cell [0,1]^d are products of 1D polynomials of degree p; Gauss quadrature with
p+1 points per direction.  The paper does not name the 1D nodes; the reading
taken here is the Gauss--Lobatto--Legendre (GLL) points mapped to [0,1].

Independent of the library: nodes and Gauss points come from numpy's Legendre
routines (companion-matrix roots / Golub--Welsch), basis values from the
Lagrange product formula.
"""
from __future__ import annotations

import numpy as np
from numpy.polynomial import legendre as L


def gll_nodes(p: int) -> np.ndarray:
    """p+1 Gauss--Lobatto--Legendre nodes on [0,1]: 0, 1 and the roots of P_p'."""
    if p < 1:
        raise ValueError("degree must be >= 1")
    if p == 1:
        t = np.array([-1.0, 1.0])
    else:
        inner = np.sort(np.real(L.Legendre.basis(p).deriv().roots()))
        # one Newton polish step per root on P_p' (roots are simple)
        dp = L.Legendre.basis(p).deriv()
        d2p = dp.deriv()
        for _ in range(3):
            inner = inner - dp(inner) / d2p(inner)
        inner = 0.5 * (inner - inner[::-1])          # exact symmetry about 0
        t = np.concatenate([[-1.0], inner, [1.0]])
    return 0.5 * (t + 1.0)


def gauss_rule(n: int) -> tuple[np.ndarray, np.ndarray]:
    """n-point Gauss--Legendre rule on [0,1] (points, weights)."""
    t, w = L.leggauss(n)
    return 0.5 * (t + 1.0), 0.5 * w


def lagrange(nodes: np.ndarray, x) -> np.ndarray:
    """phi[..., i] = Lagrange polynomial i of ``nodes`` evaluated at x.

    Plain product formula prod_{m != i} (x - x_m)/(x_i - x_m); valid for x
    anywhere on the real line (extrapolation is needed at shifted points).
    """
    x = np.asarray(x, dtype=np.float64)
    n = len(nodes)
    out = np.ones(x.shape + (n,))
    for i in range(n):
        for m in range(n):
            if m != i:
                out[..., i] *= (x - nodes[m]) / (nodes[i] - nodes[m])
    return out


def lagrange_deriv(nodes: np.ndarray, x) -> np.ndarray:
    """dphi[..., i] = d/dx of Lagrange polynomial i at x (product rule)."""
    x = np.asarray(x, dtype=np.float64)
    n = len(nodes)
    out = np.zeros(x.shape + (n,))
    for i in range(n):
        for k in range(n):
            if k == i:
                continue
            term = np.full(x.shape, 1.0 / (nodes[i] - nodes[k]))
            for m in range(n):
                if m != i and m != k:
                    term = term * (x - nodes[m]) / (nodes[i] - nodes[m])
            out[..., i] += term
    return out
