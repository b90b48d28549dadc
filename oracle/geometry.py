"""Background mesh, active cells, surrogate faces and closest points (oracle).

Follows Section 2 (SBM formulation) of the paper: the surrogate domain is the
union of active background cells; the surrogate boundary consists of the faces
of active cells that are not shared with another active cell; each surrogate
quadrature point x~ is mapped to its closest point x on the true boundary and
d = x - x~ (Section 2.1, "Shifting boundary conditions").  For each such point
the reference coordinates of x in the frame of the owning cell K are kept
(Section 3.4, data structures), xi = (x - x_K^lo)/h.

Readings taken where the paper leaves a choice open:
* mesh [-1,1]^d, N cells per side, h = 2/N, cell lower corner -1 + h*i;
* a cell is active iff the level set at its centre is strictly negative
  (default), or -- the volume-fraction criterion the paper cites (Section 2)
  -- iff at least a fraction theta of the midpoints of its 8^d sub-cells
  have a strictly negative level set;
* a face between an active cell and the box boundary is a surrogate face;
* ellipsoid closest point: root of the Lagrange-multiplier equation
  sum_i (a_i y_i / (a_i^2 + t))^2 = 1 found by plain bisection (the paper
  says only that a Newton solve is used; any convergent root finder reaches
  the same point);
* union of balls (the multiple-ball benchmark of Section 4.3): phi =
  min_i (|x - c_i| - r_i); the closest point on the union's boundary is the
  nearest of the candidates that lie on it -- the projection onto each
  sphere, the nearest point of each pairwise intersection circle (3D), and
  the vertices where three spheres (3D) or two circles (2D) meet -- a
  candidate lying strictly inside another ball being discarded; ties go to
  the first candidate in that order.
Formulas are written with an explicit, fixed summation order so that the
integer decisions (active or not) are reproducible.
"""
from __future__ import annotations

import numpy as np

from . import basis1d


class LevelSet:
    """phi < 0 inside the true domain Omega."""

    def __init__(self, kind: str, geom, dim: int):
        self.kind, self.dim = kind, dim
        g = np.asarray(geom, dtype=np.float64)
        d = dim
        if kind == "ball":
            self.c, self.r = g[:d], g[d]
        elif kind == "ellipsoid":
            self.a = g[:d]
            self.R = g[d:d + d * d].reshape(d, d)
            self.c = g[d + d * d:d + d * d + d]
        elif kind == "torus":
            if d != 3:
                raise ValueError("torus needs d = 3")
            self.Rmaj, self.rmin = g[0], g[1]
        elif kind == "box":
            self.c, self.half = g[:d], g[d:2 * d]
        elif kind == "balls":
            B = g.reshape(-1, d + 1)
            self.bc, self.br = B[:, :d].copy(), B[:, d].copy()
            self._balls_setup()
        else:
            raise ValueError(kind)

    # -- level set -----------------------------------------------------------
    def _frame(self, x):
        """Ellipsoid frame coordinates y = R^T (x - c), summed j = 0..d-1."""
        d = self.dim
        y = np.zeros_like(x)
        for i in range(d):
            acc = np.zeros(x.shape[:-1])
            for j in range(d):
                acc = acc + self.R[j, i] * (x[..., j] - self.c[j])
            y[..., i] = acc
        return y

    def phi(self, x):
        x = np.asarray(x, dtype=np.float64)
        d = self.dim
        if self.kind == "ball":
            s = np.zeros(x.shape[:-1])
            for i in range(d):
                s = s + (x[..., i] - self.c[i]) * (x[..., i] - self.c[i])
            return np.sqrt(s) - self.r
        if self.kind == "ellipsoid":
            y = self._frame(x)
            s = np.zeros(x.shape[:-1])
            for i in range(d):
                s = s + (y[..., i] / self.a[i]) * (y[..., i] / self.a[i])
            return s - 1.0
        if self.kind == "torus":
            rho = np.sqrt(x[..., 0] * x[..., 0] + x[..., 1] * x[..., 1])
            return (rho - self.Rmaj) * (rho - self.Rmaj) + x[..., 2] * x[..., 2] \
                - self.rmin * self.rmin
        if self.kind == "box":
            m = np.abs(x[..., 0] - self.c[0]) - self.half[0]
            for i in range(1, d):
                m = np.maximum(m, np.abs(x[..., i] - self.c[i]) - self.half[i])
            return m
        if self.kind == "balls":
            m = None
            for b in range(len(self.br)):
                v = _dist(x, self.bc[b]) - self.br[b]
                m = v if m is None else np.minimum(m, v)
            return m
        raise AssertionError

    # -- closest point on Gamma ------------------------------------------------
    def closest_point(self, x):
        x = np.asarray(x, dtype=np.float64)
        if self.kind == "ball":
            v = x - self.c
            return self.c + self.r * v / np.linalg.norm(v, axis=-1, keepdims=True)
        if self.kind == "torus":
            rho = np.sqrt(x[..., 0] ** 2 + x[..., 1] ** 2)
            q = np.zeros_like(x)
            q[..., 0] = self.Rmaj * x[..., 0] / rho
            q[..., 1] = self.Rmaj * x[..., 1] / rho
            v = x - q
            return q + self.rmin * v / np.linalg.norm(v, axis=-1, keepdims=True)
        if self.kind == "box":
            return self._box_closest(x)
        if self.kind == "ellipsoid":
            return self._ellipsoid_closest(x)
        if self.kind == "balls":
            return self._balls_closest(x)
        raise AssertionError

    # -- union of balls ----------------------------------------------------------
    def _outside_others(self, p, skip):
        """p lies on the union's boundary side of every ball not in skip:
        |p - c_l| >= r_l."""
        ok = np.ones(p.shape[:-1], dtype=bool)
        for l in range(len(self.br)):
            if l not in skip:
                ok &= _dist(p, self.bc[l]) >= self.br[l]
        return ok

    def _balls_setup(self):
        """Pairwise intersection circles (3D) and boundary vertices."""
        d, C, R = self.dim, self.bc, self.br
        nb = len(R)
        self.circles = []                       # (i, j, m, u, rho)
        verts = []                              # (point, defining balls)
        for i in range(nb):
            for j in range(i + 1, nb):
                dv = C[j] - C[i]
                D = _norm(dv)
                if not (D < R[i] + R[j] and D > abs(R[i] - R[j])):
                    continue
                u = dv / D
                a = (D * D + R[i] * R[i] - R[j] * R[j]) / (2.0 * D)
                m = C[i] + a * u
                rho = np.sqrt(R[i] * R[i] - a * a)
                if d == 3:
                    self.circles.append((i, j, m, u, rho))
                else:
                    perp = np.array([-u[1], u[0]])
                    for sg in (1.0, -1.0):
                        verts.append((m + sg * rho * perp, (i, j)))
        if d == 3:
            for i in range(nb):
                for j in range(i + 1, nb):
                    for k in range(j + 1, nb):
                        for p in _three_spheres(C[i], R[i], C[j], R[j], C[k], R[k]):
                            verts.append((p, (i, j, k)))
        self.vertices = [p for p, s in verts if self._outside_others(p, s)]

    def _balls_closest(self, x):
        best = np.full(x.shape[:-1], np.inf)
        out = np.full(x.shape, np.nan)

        def take(p, ok):
            d2 = _dist2(p, x)
            upd = ok & (d2 < best)
            best[upd] = d2[upd]
            out[upd] = p[upd]

        for i in range(len(self.br)):            # projections onto each sphere
            v = x - self.bc[i]
            s = _norm(v)
            with np.errstate(invalid="ignore", divide="ignore"):
                p = self.bc[i] + self.br[i] * v / s[..., None]
            take(p, (s > 0) & self._outside_others(p, (i,)))
        for i, j, m, u, rho in self.circles:     # nearest points of the circles
            w = x - m
            t = w[..., 0] * u[0] + w[..., 1] * u[1] + w[..., 2] * u[2]
            wp = w - t[..., None] * u
            s = _norm(wp)
            with np.errstate(invalid="ignore", divide="ignore"):
                p = m + rho * wp / s[..., None]
            take(p, (s > 0) & self._outside_others(p, (i, j)))
        for p in self.vertices:                  # vertices
            take(np.broadcast_to(p, x.shape), np.ones(x.shape[:-1], dtype=bool))
        return out

    def _box_closest(self, x):
        v = x - self.c
        out = x.copy()
        inside = np.all(np.abs(v) <= self.half, axis=-1)
        # outside: clamp to the box
        clamped = self.c + np.clip(v, -self.half, self.half)
        out[~inside] = clamped[~inside]
        # inside: move to the nearest face along its normal
        gap = self.half - np.abs(v)                   # distance to each face pair
        k = np.argmin(gap, axis=-1)
        idx = np.nonzero(inside)
        kk = k[idx]
        sgn = np.where(v[idx + (kk,)] >= 0, 1.0, -1.0)
        out[idx + (kk,)] = self.c[kk] + sgn * self.half[kk]
        return out

    def _ellipsoid_closest(self, x):
        y = self._frame(x)
        a2 = self.a * self.a
        F = lambda t: np.sum((self.a * y / (a2 + t[..., None])) ** 2, axis=-1) - 1.0
        phi0 = np.sum((y / self.a) ** 2, axis=-1) - 1.0
        outside = phi0 > 0
        amin2 = np.min(a2)
        ynorm = np.linalg.norm(y, axis=-1)
        lo = np.where(outside, 0.0, -amin2)
        hi = np.where(outside, np.max(self.a) * ynorm, 0.0)
        # plain bisection on the monotone function F on (-a_min^2, inf)
        for _ in range(2000):
            mid = 0.5 * (lo + hi)
            if np.all((mid == lo) | (mid == hi)):
                break                   # no double strictly inside any bracket
            go_up = F(mid) > 0          # F decreasing: root lies above mid
            lo = np.where(go_up, mid, lo)
            hi = np.where(go_up, hi, mid)
        t = 0.5 * (lo + hi)
        z = a2 * y / (a2 + t[..., None])
        # back to the mesh frame: x = c + R z
        out = np.zeros_like(x)
        for i in range(self.dim):
            acc = np.zeros(x.shape[:-1])
            for j in range(self.dim):
                acc = acc + self.R[i, j] * z[..., j]
            out[..., i] = self.c[i] + acc
        return out


def _norm(v):
    s = np.zeros(np.shape(v)[:-1])
    for l in range(np.shape(v)[-1]):
        s = s + v[..., l] * v[..., l]
    return np.sqrt(s)


def _dist(x, c):
    return _norm(x - c)


def _dist2(p, x):
    s = np.zeros(np.shape(x)[:-1])
    for l in range(np.shape(x)[-1]):
        s = s + (p[..., l] - x[..., l]) * (p[..., l] - x[..., l])
    return s


def _three_spheres(c1, r1, c2, r2, c3, r3):
    """The 0 or 2 points common to three spheres (trilateration in the frame
    e_x along c2 - c1, e_y in the plane of the centres)."""
    dv = c2 - c1
    D = _norm(dv)
    ex = dv / D
    w = c3 - c1
    i = ex[0] * w[0] + ex[1] * w[1] + ex[2] * w[2]
    ey = w - i * ex
    ny = _norm(ey)
    if not ny > 1e-12 * D:
        return []                               # centres on one line
    ey = ey / ny
    ez = np.array([ex[1] * ey[2] - ex[2] * ey[1], ex[2] * ey[0] - ex[0] * ey[2],
                   ex[0] * ey[1] - ex[1] * ey[0]])
    j = ey[0] * w[0] + ey[1] * w[1] + ey[2] * w[2]
    X = (r1 * r1 - r2 * r2 + D * D) / (2.0 * D)
    Y = (r1 * r1 - r3 * r3 + i * i + j * j) / (2.0 * j) - (i / j) * X
    z2 = r1 * r1 - X * X - Y * Y
    if not z2 > 0:
        return []
    Z = np.sqrt(z2)
    base = c1 + X * ex + Y * ey
    return [base + Z * ez, base - Z * ez]


VF_SAMPLES = 8          # sub-cells per axis of the volume-fraction estimate


class Mesh:
    """Active cells, surrogate faces, interior faces and face quadrature data."""

    def __init__(self, dim: int, degree: int, cells: int, levelset: LevelSet,
                 activity: str = "centre", vf_threshold: float = 0.5):
        self.d, self.p, self.N = dim, degree, cells
        self.n = degree + 1
        self.h = 2.0 / cells
        self.ls = levelset
        d, N, h = dim, cells, self.h
        # all background cells in lexicographic order (axis 0 fastest)
        grid = np.indices((N,) * d)[::-1].reshape(d, -1).T     # [N^d, d], col 0 fastest
        if activity == "centre":
            centres = -1.0 + h * (grid + 0.5)
            active = levelset.phi(centres) < 0.0
        elif activity == "volume":
            # volume fraction of Omega in the cell by the midpoint rule on
            # VF_SAMPLES^d sub-cells; active iff >= vf_threshold
            m = VF_SAMPLES
            sub = np.indices((m,) * d)[::-1].reshape(d, -1).T   # [m^d, d]
            count = np.zeros(len(grid), dtype=np.int64)
            for s in sub:
                pts = -1.0 + h * (grid + (s + 0.5) / m)
                count += levelset.phi(pts) < 0.0
            active = count >= vf_threshold * m ** d
        else:
            raise ValueError(f"unknown activity criterion {activity!r}")
        self.active = active                                     # [N^d] background mask
        self.cells = grid[active]                                # [Nc, d] multi-indices
        self.cell_lin = np.nonzero(active)[0]                    # background index
        lookup = -np.ones(N ** d, dtype=np.int64)
        lookup[self.cell_lin] = np.arange(len(self.cell_lin))
        self._lookup = lookup

        # faces: per active cell, axis k ascending, side 0 then 1
        sf, inf = [], []
        strides = N ** np.arange(d)
        for c, idx in enumerate(self.cells):
            for k in range(d):
                for s in (0, 1):
                    j = idx[k] + (1 if s == 1 else -1)
                    nb = -1
                    if 0 <= j < N:
                        nb = lookup[self.cell_lin[c] + (1 if s == 1 else -1) * strides[k]]
                    if nb < 0:
                        sf.append((c, k, s))
                    elif s == 1:
                        inf.append((c, k, nb))
        self.sfaces = np.array(sf, dtype=np.int64).reshape(-1, 3)
        self.ifaces = np.array(inf, dtype=np.int64).reshape(-1, 3)   # (K1, k, K2)

        # quadrature
        self.nodes = basis1d.gll_nodes(degree)
        self.gq, self.gw = basis1d.gauss_rule(self.n)
        self._face_points()

    def cell_lo(self, c):
        return -1.0 + self.h * self.cells[c].astype(np.float64)

    def _face_points(self):
        """Surrogate face Gauss points x~_q, closest points x_q, reference xi_q.

        Tangential axes in increasing order, first tangential index fastest.
        """
        d, n, h = self.d, self.n, self.h
        F = len(self.sfaces)
        Q = n ** (d - 1)
        tang_idx = np.indices((n,) * (d - 1))[::-1].reshape(d - 1, -1).T   # [Q, d-1]
        self.face_weights = np.prod(self.gw[tang_idx], axis=1)               # [Q]
        xi_t = np.zeros((F, Q, d))
        for f, (c, k, s) in enumerate(self.sfaces):
            tang = [l for l in range(d) if l != k]
            xi_t[f, :, k] = float(s)
            for a, l in enumerate(tang):
                xi_t[f, :, l] = self.gq[tang_idx[:, a]]
        lo = -1.0 + h * self.cells[self.sfaces[:, 0]].astype(np.float64)     # [F, d]
        self.face_xt = lo[:, None, :] + h * xi_t                             # x~_q
        self.face_xi_t = xi_t
        if F:
            self.face_x = self.ls.closest_point(self.face_xt)                # x_q on Gamma
        else:
            self.face_x = np.zeros((0, Q, d))
        self.face_shift = self.face_x - self.face_xt                         # d = x - x~
        self.face_xi = (self.face_x - lo[:, None, :]) / h                    # xi_q, cell K frame
