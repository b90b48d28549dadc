"""Global SBM operator: DoF numbering, EBE apply, CSR assembly, RHS (oracle).

Section 3.5 (operator workflow): y = 0, add every cell's contribution
(Algorithm 1), then every face's (Algorithm 2 for DG interior faces,
Algorithm 3 for surrogate faces).  Here each contribution is a dense local
matrix times the gathered local vector, scattered back (element by element).

Readings:
* CG numbering: the global Gauss--Lobatto lattice of (pN+1)^d nodes, axis 0
  fastest; active DoFs are the lattice nodes touched by an active cell,
  numbered in increasing lattice order.
* DG numbering: active cells in lexicographic order, n^d DoFs each,
  local lexicographic order inside.
* Penalties (the paper leaves the constants open): CG sigma = C p^2/h,
  DG surrogate sigma = C (p+1)^2/h, DG interior sigma_F = C_F (p+1)^2/h.
* Extension operator E (Section 2.1): "exact" evaluates the cell polynomial
  at the true-boundary point x_q (the whole Taylor series); "taylor1" keeps
  the first-order term, u(x~_q) + d_q . grad u(x~_q).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp

from . import basis1d, geometry, local

_FACE_CACHE_BYTES = 1 << 30


class Problem:
    def __init__(self, dim, degree, cells, kind, geom, dg=False, pen_shift=10.0,
                 pen_interior=1.0, extension="exact", activity="centre", vf_threshold=0.5):
        if extension not in ("exact", "taylor1"):
            raise ValueError(f"unknown extension {extension!r}")
        self.extension = extension
        self.d, self.p, self.N = dim, degree, cells
        self.n = degree + 1
        self.nd = self.n ** dim
        self.dg = bool(dg)
        self.ls = geometry.LevelSet(kind, geom, dim)
        self.mesh = geometry.Mesh(dim, degree, cells, self.ls, activity, vf_threshold)
        self.h = self.mesh.h
        p, h = degree, self.h
        if self.dg:
            self.sigma = pen_shift * (p + 1) ** 2 / h
            self.sigma_f = pen_interior * (p + 1) ** 2 / h
        else:
            self.sigma = pen_shift * p * p / h
            self.sigma_f = 0.0
        self._number_dofs()
        self.A_cell = local.cell_matrix(self.mesh.nodes, self.mesh.gq, self.mesh.gw, dim, h)
        self._face_cache = None
        self._dg_blocks = None

    @classmethod
    def from_workload(cls, w):
        return cls(w.dim, w.degree, w.cells, w.kind, w.geom, dg=w.dg,
                   pen_shift=w.pen_shift, pen_interior=w.pen_interior,
                   extension=getattr(w, "extension", "exact"),
                   activity=getattr(w, "activity", "centre"),
                   vf_threshold=getattr(w, "vf_threshold", 0.5))

    # -- numbering -----------------------------------------------------------
    def _number_dofs(self):
        d, n, p, N = self.d, self.n, self.p, self.N
        cells = self.mesh.cells
        mi = local.tensor_index(n, d)                          # [nd, d]
        if self.dg:
            self.dofmap = (np.arange(len(cells))[:, None] * self.nd
                           + np.arange(self.nd)[None, :])
            self.n_dofs = len(cells) * self.nd
            self.lattice = None
            return
        M = p * N + 1
        strides = M ** np.arange(d)
        lat = (p * cells[:, None, :] + mi[None, :, :]) @ strides  # [Nc, nd]
        self.lattice = np.unique(lat)                              # sorted active nodes
        self.dofmap = np.searchsorted(self.lattice, lat)
        self.n_dofs = len(self.lattice)

    def dof_coordinates(self):
        """Physical coordinates of every DoF [n_dofs, d]."""
        d, n = self.d, self.n
        X = np.zeros((self.n_dofs, d))
        mi = local.tensor_index(n, d)
        for c in range(len(self.mesh.cells)):
            lo = self.mesh.cell_lo(c)
            X[self.dofmap[c]] = lo + self.h * self.mesh.nodes[mi]
        return X

    # -- local matrices ------------------------------------------------------
    def face_matrices(self, sel=slice(None)):
        m = self.mesh
        f = m.sfaces[sel]
        shift = m.face_shift[sel] if self.extension == "taylor1" else None
        return local.face_matrices(m.nodes, m.face_xi_t[sel], m.face_xi[sel],
                                   m.face_weights, f[:, 1], f[:, 2].astype(np.float64),
                                   self.h, self.sigma, shift=shift)

    def _face_chunks(self, chunk=1024):
        F = len(self.mesh.sfaces)
        if self._face_cache is None and F * self.nd * self.nd * 8 <= _FACE_CACHE_BYTES:
            self._face_cache = self.face_matrices() if F else np.zeros((0, self.nd, self.nd))
        if self._face_cache is not None:
            yield slice(0, F), self._face_cache
            return
        for s in range(0, F, chunk):
            sel = slice(s, min(F, s + chunk))
            yield sel, self.face_matrices(sel)

    def dg_blocks(self):
        if self._dg_blocks is None:
            m = self.mesh
            self._dg_blocks = [local.dg_face_matrix(m.nodes, m.gq, m.gw, self.d, k, self.h,
                                                    self.sigma_f) for k in range(self.d)]
        return self._dg_blocks

    # -- apply ---------------------------------------------------------------
    def apply(self, x):
        """y = A x, element by element (cells, surrogate faces, DG faces)."""
        x = np.asarray(x, dtype=np.float64)
        dm = self.dofmap
        Y = x[dm] @ self.A_cell.T
        y = np.bincount(dm.ravel(), weights=Y.ravel(), minlength=self.n_dofs)
        fc = self.mesh.sfaces[:, 0]
        for sel, Af in self._face_chunks():
            fd = dm[fc[sel]]
            Yf = np.einsum("fij,fj->fi", Af, x[fd])
            y += np.bincount(fd.ravel(), weights=Yf.ravel(), minlength=self.n_dofs)
        if self.dg and len(self.mesh.ifaces):
            B = self.dg_blocks()
            for k in range(self.d):
                sel = self.mesh.ifaces[:, 1] == k
                k1 = self.mesh.ifaces[sel, 0]
                k2 = self.mesh.ifaces[sel, 2]
                dd = np.concatenate([dm[k1], dm[k2]], axis=1)
                Yi = x[dd] @ B[k].T
                y += np.bincount(dd.ravel(), weights=Yi.ravel(), minlength=self.n_dofs)
        return y

    def apply_cells(self, x, cells):
        """The contributions of the given active cells (and their surrogate and
        DG interior faces) to y = A x: the same EBE arithmetic as apply(),
        restricted to a subset of the cells (a bounded sample of the work)."""
        x = np.asarray(x, dtype=np.float64)
        cells = np.asarray(cells)
        dm = self.dofmap
        Y = x[dm[cells]] @ self.A_cell.T
        y = np.bincount(dm[cells].ravel(), weights=Y.ravel(), minlength=self.n_dofs)
        own = np.zeros(len(dm), dtype=bool)
        own[cells] = True
        fsel = np.nonzero(own[self.mesh.sfaces[:, 0]])[0]
        for s in range(0, len(fsel), 1024):
            part = fsel[s:s + 1024]
            Af = self.face_matrices(part)
            fd = dm[self.mesh.sfaces[part, 0]]
            Yf = np.einsum("fij,fj->fi", Af, x[fd])
            y += np.bincount(fd.ravel(), weights=Yf.ravel(), minlength=self.n_dofs)
        if self.dg and len(self.mesh.ifaces):
            B = self.dg_blocks()
            for k in range(self.d):
                sel = (self.mesh.ifaces[:, 1] == k) & own[self.mesh.ifaces[:, 0]]
                dd = np.concatenate([dm[self.mesh.ifaces[sel, 0]],
                                     dm[self.mesh.ifaces[sel, 2]]], axis=1)
                Yi = x[dd] @ B[k].T
                y += np.bincount(dd.ravel(), weights=Yi.ravel(), minlength=self.n_dofs)
        return y

    def apply_rows(self, x, rows):
        """(A x)[rows] computed from the local matrices touching those rows only."""
        rows = np.asarray(rows)
        want = np.zeros(self.n_dofs, dtype=bool)
        want[rows] = True
        dm = self.dofmap
        y = np.zeros(self.n_dofs)
        cells = np.nonzero(want[dm].any(axis=1))[0]
        Y = x[dm[cells]] @ self.A_cell.T
        y += np.bincount(dm[cells].ravel(), weights=Y.ravel(), minlength=self.n_dofs)
        fsel = np.nonzero(want[dm[self.mesh.sfaces[:, 0]]].any(axis=1))[0]
        if len(fsel):
            Af = self.face_matrices(fsel)
            fd = dm[self.mesh.sfaces[fsel, 0]]
            Yf = np.einsum("fij,fj->fi", Af, x[fd])
            y += np.bincount(fd.ravel(), weights=Yf.ravel(), minlength=self.n_dofs)
        if self.dg and len(self.mesh.ifaces):
            B = self.dg_blocks()
            for k in range(self.d):
                sel = self.mesh.ifaces[:, 1] == k
                k1 = self.mesh.ifaces[sel, 0]
                k2 = self.mesh.ifaces[sel, 2]
                dd = np.concatenate([dm[k1], dm[k2]], axis=1)
                keep = want[dd].any(axis=1)
                Yi = x[dd[keep]] @ B[k].T
                y += np.bincount(dd[keep].ravel(), weights=Yi.ravel(), minlength=self.n_dofs)
        return y[rows]

    # -- assembled forms -------------------------------------------------------
    def assemble(self):
        """Global CSR matrix from the same local matrices (small meshes)."""
        dm = self.dofmap
        nd = self.nd
        rows, cols, vals = [], [], []
        Nc = len(dm)
        rows.append(np.repeat(dm, nd, axis=1).ravel())
        cols.append(np.tile(dm, (1, nd)).ravel())
        vals.append(np.broadcast_to(self.A_cell.ravel(), (Nc, nd * nd)).ravel())
        fc = self.mesh.sfaces[:, 0]
        for sel, Af in self._face_chunks():
            fd = dm[fc[sel]]
            rows.append(np.repeat(fd, nd, axis=1).ravel())
            cols.append(np.tile(fd, (1, nd)).ravel())
            vals.append(Af.reshape(len(fd), -1).ravel())
        if self.dg and len(self.mesh.ifaces):
            B = self.dg_blocks()
            for k in range(self.d):
                sel = self.mesh.ifaces[:, 1] == k
                dd = np.concatenate([dm[self.mesh.ifaces[sel, 0]],
                                     dm[self.mesh.ifaces[sel, 2]]], axis=1)
                rows.append(np.repeat(dd, 2 * nd, axis=1).ravel())
                cols.append(np.tile(dd, (1, 2 * nd)).ravel())
                vals.append(np.broadcast_to(B[k].ravel(), (len(dd), 4 * nd * nd)).ravel())
        A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                          shape=(self.n_dofs, self.n_dofs))
        return A.tocsr()

    def diagonal(self):
        dm = self.dofmap
        nd = self.nd
        diag = np.bincount(dm.ravel(), weights=np.tile(np.diag(self.A_cell), len(dm)),
                           minlength=self.n_dofs)
        fc = self.mesh.sfaces[:, 0]
        for sel, Af in self._face_chunks():
            fd = dm[fc[sel]]
            diag += np.bincount(fd.ravel(), weights=np.diagonal(Af, axis1=1, axis2=2).ravel(),
                                minlength=self.n_dofs)
        if self.dg and len(self.mesh.ifaces):
            B = self.dg_blocks()
            for k in range(self.d):
                sel = self.mesh.ifaces[:, 1] == k
                dd = np.concatenate([dm[self.mesh.ifaces[sel, 0]],
                                     dm[self.mesh.ifaces[sel, 2]]], axis=1)
                diag += np.bincount(dd.ravel(), weights=np.tile(np.diag(B[k]), len(dd)),
                                    minlength=self.n_dofs)
        return diag

    # -- right-hand side and errors ------------------------------------------
    def rhs(self, f, g):
        """b_i = int f v_i - int_F (grad v_i . n~) g(x) + int_F sigma g(x) v_i.

        f, g are callables on physical points [..., d]; g is evaluated at the
        true-boundary points x_q (weak form of Section 2.1, right-hand side).
        """
        m = self.mesh
        d, h = self.d, self.h
        pts, w = local.cell_quadrature(m.gq, m.gw, d)
        V, _ = local.tensor_values(m.nodes, pts)                    # [Q, nd]
        lo = -1.0 + h * m.cells.astype(np.float64)                  # [Nc, d]
        X = lo[:, None, :] + h * pts[None, :, :]                    # [Nc, Q, d]
        F = f(X) * (h ** d * w)[None, :]                            # [Nc, Q]
        B = F @ V                                                   # [Nc, nd]
        b = np.bincount(self.dofmap.ravel(), weights=B.ravel(), minlength=self.n_dofs)
        if len(m.sfaces):
            Vt, Gt = local.tensor_values(m.nodes, m.face_xi_t)      # [F, Q, nd(, d)]
            k = m.sfaces[:, 1]
            sign = 2.0 * m.sfaces[:, 2] - 1.0
            Nt = np.take_along_axis(Gt, k[:, None, None, None], axis=3)[..., 0]
            Nt = Nt * (sign / h)[:, None, None]
            G = g(m.face_x) * (h ** (d - 1) * m.face_weights)[None, :]   # [F, Q]
            Bf = np.einsum("fq,fqi->fi", G, self.sigma * Vt - Nt)
            fd = self.dofmap[m.sfaces[:, 0]]
            b += np.bincount(fd.ravel(), weights=Bf.ravel(), minlength=self.n_dofs)
        return b

    def interpolate(self, u):
        """Nodal interpolant of a callable u (DoF values at the GLL nodes)."""
        return u(self.dof_coordinates())

    def l2_error(self, uh, u, extra=2):
        """||u_h - u||_{L2(surrogate domain)} with n+extra Gauss points per axis."""
        m = self.mesh
        d, h = self.d, self.h
        gq, gw = basis1d.gauss_rule(self.n + extra)
        pts, w = local.cell_quadrature(gq, gw, d)
        V, _ = local.tensor_values(m.nodes, pts)
        lo = -1.0 + h * m.cells.astype(np.float64)
        X = lo[:, None, :] + h * pts[None, :, :]
        U = uh[self.dofmap] @ V.T                                   # [Nc, Q]
        err = (U - u(X)) ** 2 * (h ** d * w)[None, :]
        return math.sqrt(err.sum())


def sin_solution(d):
    """u = prod sin(pi x_i), f = d pi^2 u."""
    def u(X):
        out = np.ones(X.shape[:-1])
        for i in range(d):
            out = out * np.sin(math.pi * X[..., i])
        return out

    def f(X):
        return d * math.pi ** 2 * u(X)
    return u, f
