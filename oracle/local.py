"""Dense local matrices of the SBM operator, straight from the quadrature (oracle).

Notation: n = p+1, local DoF index i = i_1 + n i_2 (+ n^2 i_3), i_1 fastest
(Section 3.1, lexicographic numbering; the figure's label formula is garbled
and read as this).  psi_i(xi) = prod_l phi_{i_l}(xi_l) on [0,1]^d, physical
x = x_K^lo + h xi, so grad = (1/h) grad_xi.

Cell (Algorithm 1, Section 3.1):
    A_K[i,j] = sum_q h^d w_q (1/h^2) grad_xi psi_i(g_q) . grad_xi psi_j(g_q)

Surrogate face F of cell K with outward normal n~ = (2s-1) e_k (Algorithm 3,
Section 3.3; weak form of Section 2.1), test index i, trial index j,
face Gauss points xi~_q (on F) and shifted reference points xi_q (closest
point on Gamma, in K's frame):
    A_F[i,j] = sum_q h^{d-1} w_q [ - psi_i(xi~_q) dn psi_j(xi~_q)
                                   - dn psi_i(xi~_q) psi_j(xi_q)
                                   + sigma psi_i(xi~_q) psi_j(xi_q) ]
i.e. I_value = -grad u.n~ + sigma E u tested against v, and I_grad = -E u
tested against grad v . n~, with E u(x~_q) = u_K(x_q) evaluated from cell K's
polynomial at the shifted point (exact point evaluation: the reading of the
Taylor extension applied to the discrete polynomial).  The first-order
variant truncates that series after the gradient term:
    E1 psi_j(x~_q) = psi_j(xi~_q) + (1/h) d_q . grad_xi psi_j(xi~_q),
d_q = x_q - x~_q (physical), in place of psi_j(xi_q).

DG interior face between K1 (lower side along axis k) and K2, n = +e_k
(Algorithm 2, Section 3.2, SIPG form):
    int_F sigma_F [u][v] - {dn u}[v] - [u]{dn v},  [u] = u1 - u2,
    {dn u} = (dn u1 + dn u2)/2.
"""
from __future__ import annotations

import numpy as np

from . import basis1d


def tensor_index(n: int, d: int) -> np.ndarray:
    """[n^d, d] multi-indices, component 0 fastest."""
    return np.indices((n,) * d)[::-1].reshape(d, -1).T


def tensor_values(nodes, pts):
    """Basis values psi_i(x) and reference gradients at points pts[..., d].

    Returns V[..., i] and G[..., i, l] = d psi_i / d xi_l.
    """
    pts = np.asarray(pts, dtype=np.float64)
    d = pts.shape[-1]
    n = len(nodes)
    mi = tensor_index(n, d)                              # [n^d, d]
    phi = basis1d.lagrange(nodes, pts)                   # [..., d, n]
    dphi = basis1d.lagrange_deriv(nodes, pts)            # [..., d, n]
    V = np.ones(pts.shape[:-1] + (n ** d,))
    G = np.ones(pts.shape[:-1] + (n ** d, d))
    for l in range(d):
        V = V * phi[..., l, mi[:, l]]
        for m in range(d):
            fac = dphi[..., l, mi[:, l]] if m == l else phi[..., l, mi[:, l]]
            G[..., m] = G[..., m] * fac
    return V, G


def cell_quadrature(gq, gw, d):
    """Tensor Gauss points [n^d, d] and weights [n^d] on [0,1]^d."""
    n = len(gq)
    mi = tensor_index(n, d)
    return gq[mi], np.prod(gw[mi], axis=1)


def cell_matrix(nodes, gq, gw, d: int, h: float) -> np.ndarray:
    """A_K for the Laplacian term; identical for every cell of a uniform mesh."""
    pts, w = cell_quadrature(gq, gw, d)
    _, G = tensor_values(nodes, pts)                     # [Q, nd, d]
    A = np.zeros((G.shape[1], G.shape[1]))
    for l in range(d):
        A += G[:, :, l].T @ (w[:, None] * G[:, :, l])
    return h ** (d - 2) * A


def face_matrices(nodes, xi_t, xi_s, w, k, s, h, sigma, shift=None):
    """A_F for a batch of surrogate faces.

    xi_t [F, Q, d] face points, xi_s [F, Q, d] shifted points (cell frame),
    w [Q] tangential weights, k [F] normal axis, s [F] side (0 or 1).
    The trial side is the extension E psi_j at x~_q (Section 2.1): with
    shift = None the exact one, psi_j(x_q) (the whole Taylor series of the
    polynomial); with shift = d [F, Q, d] (physical, d = x - x~) the
    first-order truncation psi_j(x~_q) + d_q . grad psi_j(x~_q).
    Returns [F, nd, nd] (row = test i, column = trial j).
    """
    d = xi_t.shape[-1]
    Vt, Gt = tensor_values(nodes, xi_t)                  # [F, Q, nd], [F, Q, nd, d]
    if shift is None:
        Vs, _ = tensor_values(nodes, xi_s)               # [F, Q, nd]
    else:
        Vs = Vt + np.einsum("fql,fqjl->fqj", shift, Gt) / h
    sign = (2.0 * s - 1.0)                               # outward normal +/- e_k
    Nt = np.take_along_axis(Gt, k[:, None, None, None], axis=3)[..., 0]
    Nt = Nt * (sign / h)[:, None, None]                  # dn psi at x~_q (physical)
    W = (h ** (d - 1) * w)[None, :, None]                # [1, Q, 1]
    VtT = np.swapaxes(W * Vt, 1, 2)                      # [F, nd, Q]
    NtT = np.swapaxes(W * Nt, 1, 2)
    A = -(VtT @ Nt)                  # - psi_i(x~) dn psi_j(x~)
    A -= NtT @ Vs                    # - dn psi_i(x~) psi_j(x)
    A += sigma * (VtT @ Vs)          # + sigma psi_i(x~) psi_j(x)
    return A


def dg_face_matrix(nodes, gq, gw, d: int, k: int, h: float, sigma_f: float):
    """2 n^d x 2 n^d SIPG block [[A11, A12], [A21, A22]] for a face normal to
    axis k; K1 sees the face at xi_k = 1, K2 at xi_k = 0, n = +e_k."""
    n = len(nodes)
    Q = n ** (d - 1)
    tmi = tensor_index(n, d - 1)
    tang = [l for l in range(d) if l != k]
    pts1 = np.zeros((Q, d))
    pts2 = np.zeros((Q, d))
    for a, l in enumerate(tang):
        pts1[:, l] = gq[tmi[:, a]]
        pts2[:, l] = gq[tmi[:, a]]
    pts1[:, k] = 1.0
    pts2[:, k] = 0.0
    w = np.prod(gw[tmi], axis=1) * h ** (d - 1)
    V1, G1 = tensor_values(nodes, pts1)
    V2, G2 = tensor_values(nodes, pts2)
    D1 = G1[:, :, k] / h
    D2 = G2[:, :, k] / h
    J = [V1, -V2]                    # jump of the test/trial function of side a
    Av = [0.5 * D1, 0.5 * D2]        # average normal derivative of side a
    nd = n ** d
    B = np.zeros((2 * nd, 2 * nd))
    for a in range(2):               # test side
        for b in range(2):           # trial side
            blk = sigma_f * J[a].T @ (w[:, None] * J[b])
            blk -= J[a].T @ (w[:, None] * Av[b])      # - {dn u}[v]
            blk -= Av[a].T @ (w[:, None] * J[b])      # - [u]{dn v}
            B[a * nd:(a + 1) * nd, b * nd:(b + 1) * nd] = blk
    return B
