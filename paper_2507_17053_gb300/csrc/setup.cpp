// Host-side FP64 set-up of an SBM problem (see setup.hpp).
//
// Compiled with -ffp-contract=off so that the level-set tests that decide
// which cells are active are evaluated exactly as written (no fused
// multiply-add reassociation), on x86 and Arm alike.
#include "setup.hpp"

#include <algorithm>
#include <cmath>
#include <cstring>

namespace sbm {

// ---------------------------------------------------------------------------
// 1D tables
// ---------------------------------------------------------------------------

// Legendre P_m(t) and P_m'(t) by the three-term recurrence.
static void legendre(int m, double t, double* P, double* dP) {
  double p0 = 1.0, p1 = t;
  if (m == 0) { *P = 1.0; *dP = 0.0; return; }
  for (int k = 1; k < m; ++k) {
    double p2 = ((2.0 * k + 1.0) * t * p1 - k * p0) / (k + 1.0);
    p0 = p1;
    p1 = p2;
  }
  *P = p1;
  // (1 - t^2) P_m' = m (P_{m-1} - t P_m); only used away from t = +-1
  *dP = m * (p0 - t * p1) / (1.0 - t * t);
}

// Eigenbasis of the symmetric-definite pencil (K, M): Cholesky M = C C^T,
// cyclic Jacobi rotations on the symmetric C^-1 K C^-T = Q diag(lam) Q^T,
// V = C Q.  Then M = V V^T and K = V diag(lam) V^T.  Each column of V is
// made exactly even or odd, and the columns are reordered (even modes, then
// odd modes, each by increasing eigenvalue).
static void pencil_eigenbasis(Tables1D* t) {
  const int n = t->n;
  double C[kMaxN][kMaxN] = {};
  for (int j = 0; j < n; ++j) {
    double d = t->M[j][j];
    for (int k = 0; k < j; ++k) d -= C[j][k] * C[j][k];
    C[j][j] = std::sqrt(d);
    for (int i = j + 1; i < n; ++i) {
      double s = t->M[i][j];
      for (int k = 0; k < j; ++k) s -= C[i][k] * C[j][k];
      C[i][j] = s / C[j][j];
    }
  }
  // B = C^-1 K C^-T: forward substitution on the columns of K, then on the rows
  double Y[kMaxN][kMaxN], B[kMaxN][kMaxN];
  for (int c = 0; c < n; ++c)
    for (int i = 0; i < n; ++i) {
      double s = t->K[i][c];
      for (int k = 0; k < i; ++k) s -= C[i][k] * Y[k][c];
      Y[i][c] = s / C[i][i];
    }
  for (int r = 0; r < n; ++r)
    for (int i = 0; i < n; ++i) {
      double s = Y[r][i];
      for (int k = 0; k < i; ++k) s -= C[i][k] * B[r][k];
      B[r][i] = s / C[i][i];
    }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < i; ++j) B[i][j] = B[j][i] = 0.5 * (B[i][j] + B[j][i]);
  double Q[kMaxN][kMaxN] = {};
  for (int i = 0; i < n; ++i) Q[i][i] = 1.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, diag = 0.0;
    for (int i = 0; i < n; ++i) {
      diag += B[i][i] * B[i][i];
      for (int j = i + 1; j < n; ++j) off += B[i][j] * B[i][j];
    }
    if (off <= 1e-34 * diag) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        if (B[p][q] == 0.0) continue;
        // rotation zeroing B[p][q] (the symmetric Schur step)
        const double theta = (B[q][q] - B[p][p]) / (2.0 * B[p][q]);
        const double tt = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double cs = 1.0 / std::sqrt(tt * tt + 1.0), sn = tt * cs;
        for (int k = 0; k < n; ++k) {
          const double bp = B[k][p], bq = B[k][q];
          B[k][p] = cs * bp - sn * bq;
          B[k][q] = sn * bp + cs * bq;
        }
        for (int k = 0; k < n; ++k) {
          const double bp = B[p][k], bq = B[q][k];
          B[p][k] = cs * bp - sn * bq;
          B[q][k] = sn * bp + cs * bq;
        }
        for (int k = 0; k < n; ++k) {
          const double qp = Q[k][p], qq = Q[k][q];
          Q[k][p] = cs * qp - sn * qq;
          Q[k][q] = sn * qp + cs * qq;
        }
      }
  }
  double V0[kMaxN][kMaxN];
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < n; ++k) {
      double s = 0.0;
      for (int m = 0; m <= i; ++m) s += C[i][m] * Q[m][k];
      V0[i][k] = s;
    }
  // parity of each column, exact symmetry, order
  int order[kMaxN], parity[kMaxN];
  for (int k = 0; k < n; ++k) {
    double de = 0.0, dodd = 0.0;
    for (int j = 0; j < n; ++j) {
      de += std::fabs(V0[j][k] - V0[n - 1 - j][k]);
      dodd += std::fabs(V0[j][k] + V0[n - 1 - j][k]);
    }
    parity[k] = (de <= dodd) ? 0 : 1;
    for (int j = 0; j < n / 2; ++j) {
      const double a = V0[j][k], b = V0[n - 1 - j][k];
      const double m = parity[k] ? 0.5 * (a - b) : 0.5 * (a + b);
      V0[j][k] = m;
      V0[n - 1 - j][k] = parity[k] ? -m : m;
    }
    if ((n & 1) && parity[k]) V0[n / 2][k] = 0.0;
    order[k] = k;
  }
  for (int a = 0; a < n; ++a)
    for (int b = a + 1; b < n; ++b) {
      const int ka = order[a], kb = order[b];
      const bool swap = parity[kb] < parity[ka] ||
                        (parity[kb] == parity[ka] && B[kb][kb] < B[ka][ka]);
      if (swap) std::swap(order[a], order[b]);
    }
  double lmax = 0.0;
  for (int k = 0; k < n; ++k) lmax = std::max(lmax, std::fabs(B[k][k]));
  for (int k = 0; k < n; ++k) {
    t->lam[k] = B[order[k]][order[k]];
    // the constant mode: K annihilates constants, its eigenvalue is 0
    if (std::fabs(t->lam[k]) <= 1e-12 * lmax) t->lam[k] = 0.0;
    for (int j = 0; j < n; ++j) t->V[j][k] = V0[j][order[k]];
  }
  double em = 0.0, ek = 0.0, sm = 0.0, sk = 0.0;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double m = 0.0, kk = 0.0;
      for (int k = 0; k < n; ++k) {
        m += t->V[i][k] * t->V[j][k];
        kk += t->V[i][k] * t->lam[k] * t->V[j][k];
      }
      em = std::max(em, std::fabs(m - t->M[i][j]));
      ek = std::max(ek, std::fabs(kk - t->K[i][j]));
      sm = std::max(sm, std::fabs(t->M[i][j]));
      sk = std::max(sk, std::fabs(t->K[i][j]));
    }
  t->fd_residual = em / sm + ek / sk;
}

void build_tables(int p, Tables1D* t) {
  const int n = p + 1;
  *t = Tables1D();
  t->n = n;
  const double pi = 3.14159265358979323846;
  // GLL nodes: +-1 and the roots of P_p'; Newton on P_p' with
  // P_p'' = (2 t P_p' - p(p+1) P_p) / (1 - t^2) (Legendre's equation).
  double tn[kMaxN];
  tn[0] = -1.0;
  tn[p] = 1.0;
  for (int i = 1; i < p; ++i) {
    double x = -std::cos(pi * i / p);
    for (int it = 0; it < 100; ++it) {
      double P, dP;
      legendre(p, x, &P, &dP);
      double d2P = (2.0 * x * dP - p * (p + 1.0) * P) / (1.0 - x * x);
      double dx = dP / d2P;
      x -= dx;
      if (std::fabs(dx) < 1e-16) break;
    }
    tn[i] = x;
  }
  for (int i = 0; i < n; ++i) {          // exact symmetry about 0
    double s = 0.5 * (tn[i] - tn[p - i]);
    t->nodes[i] = 0.5 * (s + 1.0);
  }
  t->nodes[0] = 0.0;
  t->nodes[p] = 1.0;
  // Gauss points: roots of P_n, weights 2 / ((1 - t^2) P_n'(t)^2)
  double tg[kMaxN], wg[kMaxN];
  for (int i = 0; i < n; ++i) {
    double x = -std::cos(pi * (i + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; ++it) {
      double P, dP;
      legendre(n, x, &P, &dP);
      double dx = P / dP;
      x -= dx;
      if (std::fabs(dx) < 1e-16) break;
    }
    double P, dP;
    legendre(n, x, &P, &dP);
    tg[i] = x;
    wg[i] = 2.0 / ((1.0 - x * x) * dP * dP);
  }
  for (int i = 0; i < n; ++i) {          // exact symmetry about 0
    double s = 0.5 * (tg[i] - tg[n - 1 - i]);
    double w = 0.5 * (wg[i] + wg[n - 1 - i]);
    t->gpts[i] = 0.5 * (s + 1.0);
    t->gwts[i] = 0.5 * w;
  }
  for (int q = 0; q < n; ++q) {
    lagrange_values(*t, t->gpts[q], t->S[q]);
    lagrange_derivs(*t, t->gpts[q], t->Dg[q]);
  }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double m = 0.0, k = 0.0;
      for (int q = 0; q < n; ++q) {
        m += t->gwts[q] * t->S[q][i] * t->S[q][j];
        k += t->gwts[q] * t->Dg[q][i] * t->Dg[q][j];
      }
      t->M[i][j] = m;
      t->K[i][j] = k;
    }
  lagrange_derivs(*t, 0.0, t->D0);
  lagrange_derivs(*t, 1.0, t->D1);
  pencil_eigenbasis(t);
}

// Barycentric weights lambda_j = 1 / prod_{m != j} (x_j - x_m).
static void bary_weights(const Tables1D& t, double* lam) {
  for (int j = 0; j < t.n; ++j) {
    double prod = 1.0;
    for (int m = 0; m < t.n; ++m)
      if (m != j) prod *= (t.nodes[j] - t.nodes[m]);
    lam[j] = 1.0 / prod;
  }
}

// First (modified Lagrange) barycentric form: phi_j(x) = l(x) lambda_j / (x - x_j),
// l(x) = prod_m (x - x_m); exact Kronecker delta at the nodes.  Stable for
// extrapolation outside [0,1].
void lagrange_values(const Tables1D& t, double x, double* phi) {
  double lam[kMaxN];
  bary_weights(t, lam);
  for (int j = 0; j < t.n; ++j)
    if (x == t.nodes[j]) {
      for (int m = 0; m < t.n; ++m) phi[m] = (m == j) ? 1.0 : 0.0;
      return;
    }
  double l = 1.0;
  for (int m = 0; m < t.n; ++m) l *= (x - t.nodes[m]);
  for (int j = 0; j < t.n; ++j) phi[j] = l * lam[j] / (x - t.nodes[j]);
}

// Derivatives: at a node x_i the differentiation-matrix entries
// (lambda_j/lambda_i)/(x_i - x_j) and minus their row sum on the diagonal;
// elsewhere phi_j'(x) = sum_{k != j} lambda_j prod_{m != j,k} (x - x_m).
void lagrange_derivs(const Tables1D& t, double x, double* dphi) {
  double lam[kMaxN];
  bary_weights(t, lam);
  for (int i = 0; i < t.n; ++i)
    if (x == t.nodes[i]) {
      double diag = 0.0;
      for (int j = 0; j < t.n; ++j) {
        if (j == i) continue;
        dphi[j] = (lam[j] / lam[i]) / (t.nodes[i] - t.nodes[j]);
        diag -= dphi[j];
      }
      dphi[i] = diag;
      return;
    }
  for (int j = 0; j < t.n; ++j) {
    double s = 0.0;
    for (int k = 0; k < t.n; ++k) {
      if (k == j) continue;
      double prod = lam[j];
      for (int m = 0; m < t.n; ++m)
        if (m != j && m != k) prod *= (x - t.nodes[m]);
      s += prod;
    }
    dphi[j] = s;
  }
}

// ---------------------------------------------------------------------------
// Level sets and closest points (Section 2.1: closest-point projection onto
// Gamma, d = x - x~).  Fixed summation orders (axis 0 first).
// ---------------------------------------------------------------------------

int LevelSet::init(int k, int d, const double* g, std::string* err) {
  kind = k;
  dim = d;
  switch (k) {
    case SBM_GEOM_BALL:
      for (int i = 0; i < d; ++i) c[i] = g[i];
      r = g[d];
      if (!(r > 0)) { *err = "ball radius must be > 0"; return SBM_ERR_ARG; }
      return SBM_OK;
    case SBM_GEOM_ELLIPSOID:
      for (int i = 0; i < d; ++i) {
        a[i] = g[i];
        if (!(a[i] > 0)) { *err = "ellipsoid semi-axes must be > 0"; return SBM_ERR_ARG; }
      }
      for (int i = 0; i < d * d; ++i) R[i] = g[d + i];
      for (int i = 0; i < d; ++i) c[i] = g[d + d * d + i];
      return SBM_OK;
    case SBM_GEOM_TORUS:
      if (d != 3) { *err = "torus needs dim = 3"; return SBM_ERR_ARG; }
      Rmaj = g[0];
      rmin = g[1];
      if (!(rmin > 0 && Rmaj > rmin)) { *err = "torus needs R > r > 0"; return SBM_ERR_ARG; }
      return SBM_OK;
    case SBM_GEOM_BOX:
      for (int i = 0; i < d; ++i) {
        c[i] = g[i];
        half[i] = g[d + i];
        if (!(half[i] > 0)) { *err = "box half-widths must be > 0"; return SBM_ERR_ARG; }
      }
      return SBM_OK;
  }
  *err = "unknown geometry kind";
  return SBM_ERR_ARG;
}

// ---- union of balls ----------------------------------------------------------
// The same formulas, in the same operation order, as the oracle's, so that the
// two geometries agree to the last bit.

GeomView LevelSet::view() const {
  GeomView g;
  g.kind = kind;
  g.dim = dim;
  for (int i = 0; i < 3; ++i) {
    g.c[i] = c[i];
    g.a[i] = a[i];
    g.half[i] = half[i];
  }
  for (int i = 0; i < 9; ++i) g.R[i] = R[i];
  g.r = r;
  g.Rmaj = Rmaj;
  g.rmin = rmin;
  g.nb = (int)br.size();
  g.ncirc = (int)circles.size();
  g.nvert = (int)(verts.size() / 3);
  g.bc = bc.data();
  g.br = br.data();
  g.circ = circles.data();
  g.verts = verts.data();
  return g;
}

// the 0 or 2 points common to three spheres (trilateration)
static int three_spheres(const double* c1, double r1, const double* c2, double r2,
                         const double* c3, double r3, double out[2][3]) {
  double dv[3], ex[3], w[3], ey[3], ez[3];
  for (int l = 0; l < 3; ++l) dv[l] = c2[l] - c1[l];
  const double D = gv_norm(dv, 3);
  for (int l = 0; l < 3; ++l) ex[l] = dv[l] / D;
  for (int l = 0; l < 3; ++l) w[l] = c3[l] - c1[l];
  const double i = ex[0] * w[0] + ex[1] * w[1] + ex[2] * w[2];
  for (int l = 0; l < 3; ++l) ey[l] = w[l] - i * ex[l];
  const double ny = gv_norm(ey, 3);
  if (!(ny > 1e-12 * D)) return 0;
  for (int l = 0; l < 3; ++l) ey[l] = ey[l] / ny;
  ez[0] = ex[1] * ey[2] - ex[2] * ey[1];
  ez[1] = ex[2] * ey[0] - ex[0] * ey[2];
  ez[2] = ex[0] * ey[1] - ex[1] * ey[0];
  const double j = ey[0] * w[0] + ey[1] * w[1] + ey[2] * w[2];
  const double X = (r1 * r1 - r2 * r2 + D * D) / (2.0 * D);
  const double Y = (r1 * r1 - r3 * r3 + i * i + j * j) / (2.0 * j) - (i / j) * X;
  const double z2 = r1 * r1 - X * X - Y * Y;
  if (!(z2 > 0)) return 0;
  const double Z = std::sqrt(z2);
  for (int l = 0; l < 3; ++l) {
    const double base = c1[l] + X * ex[l] + Y * ey[l];
    out[0][l] = base + Z * ez[l];
    out[1][l] = base - Z * ez[l];
  }
  return 2;
}

int LevelSet::init_balls(int d, int nb, const double* b, std::string* err) {
  kind = SBM_GEOM_BALLS;
  dim = d;
  if (nb < 1 || !b) { *err = "balls: nballs >= 1 and a balls array are needed"; return SBM_ERR_ARG; }
  bc.assign(3 * (size_t)nb, 0.0);
  br.assign(nb, 0.0);
  for (int i = 0; i < nb; ++i) {
    for (int l = 0; l < d; ++l) bc[3 * i + l] = b[(d + 1) * i + l];
    br[i] = b[(d + 1) * i + d];
    if (!(br[i] > 0)) { *err = "ball radius must be > 0"; return SBM_ERR_ARG; }
  }
  circles.clear();
  verts.clear();
  std::vector<double> cand;            // vertex candidates with their defining balls
  std::vector<int> cdef;
  for (int i = 0; i < nb; ++i)
    for (int j = i + 1; j < nb; ++j) {
      double dv[3] = {0, 0, 0};
      for (int l = 0; l < d; ++l) dv[l] = bc[3 * j + l] - bc[3 * i + l];
      const double D = gv_norm(dv, d);
      if (!(D < br[i] + br[j] && D > std::fabs(br[i] - br[j]))) continue;
      GeomCircle C{};
      C.i = i;
      C.j = j;
      for (int l = 0; l < d; ++l) C.u[l] = dv[l] / D;
      const double aa = (D * D + br[i] * br[i] - br[j] * br[j]) / (2.0 * D);
      for (int l = 0; l < d; ++l) C.m[l] = bc[3 * i + l] + aa * C.u[l];
      C.rho = std::sqrt(br[i] * br[i] - aa * aa);
      if (d == 3) {
        circles.push_back(C);
      } else {
        const double perp[2] = {-C.u[1], C.u[0]};
        for (int sg = 0; sg < 2; ++sg) {
          const double sgn = sg ? -1.0 : 1.0;
          for (int l = 0; l < 2; ++l) cand.push_back(C.m[l] + sgn * C.rho * perp[l]);
          cand.push_back(0.0);
          cdef.push_back(i);
          cdef.push_back(j);
          cdef.push_back(-1);
        }
      }
    }
  if (d == 3)
    for (int i = 0; i < nb; ++i)
      for (int j = i + 1; j < nb; ++j)
        for (int k = j + 1; k < nb; ++k) {
          double pts[2][3];
          const int np = three_spheres(&bc[3 * i], br[i], &bc[3 * j], br[j], &bc[3 * k], br[k], pts);
          for (int q = 0; q < np; ++q) {
            for (int l = 0; l < 3; ++l) cand.push_back(pts[q][l]);
            cdef.push_back(i);
            cdef.push_back(j);
            cdef.push_back(k);
          }
        }
  const GeomView g = view();            // nb, bc, br set; no circles or vertices needed
  std::vector<double> kept;
  for (size_t q = 0; q * 3 < cand.size(); ++q)
    if (gv_outside_others(g, &cand[3 * q], cdef[3 * q], cdef[3 * q + 1], cdef[3 * q + 2]))
      for (int l = 0; l < 3; ++l) kept.push_back(cand[3 * q + l]);
  verts = kept;
  return SBM_OK;
}

// ---------------------------------------------------------------------------
// Mesh, faces, numbering
// ---------------------------------------------------------------------------

int setup_prepare(const sbm_desc& desc, HostProblem* hp, std::string* err) {
  HostProblem& P = *hp;
  P.desc = desc;
  const int d = desc.dim, p = desc.degree, N = desc.cells_per_side;
  if (d != 2 && d != 3) { *err = "dim must be 2 or 3"; return SBM_ERR_ARG; }
  if (p < 1 || p > 6) { *err = "degree must be in 1..6"; return SBM_ERR_UNSUPPORTED; }
  if (N < 1 || N > 4096) { *err = "cells_per_side must be in 1..4096"; return SBM_ERR_ARG; }
  if (!(desc.pen_shift > 0)) { *err = "pen_shift must be > 0"; return SBM_ERR_ARG; }
  if (desc.dg && !(desc.pen_interior > 0)) { *err = "pen_interior must be > 0"; return SBM_ERR_ARG; }
  if (desc.extension != SBM_EXT_EXACT && desc.extension != SBM_EXT_TAYLOR1) {
    *err = "unknown extension operator";
    return SBM_ERR_ARG;
  }
  if (desc.activity != SBM_ACTIVE_CENTRE && desc.activity != SBM_ACTIVE_VOLUME) {
    *err = "unknown activity criterion";
    return SBM_ERR_ARG;
  }
  if (desc.activity == SBM_ACTIVE_VOLUME && !(desc.vf_threshold > 0 && desc.vf_threshold <= 1)) {
    *err = "vf_threshold must be in (0, 1]";
    return SBM_ERR_ARG;
  }
  int st = (desc.geom_kind == SBM_GEOM_BALLS)
               ? P.ls.init_balls(d, desc.nballs, desc.balls, err)
               : P.ls.init(desc.geom_kind, d, desc.geom, err);
  P.desc.balls = nullptr;              // copied into the level set; the caller owns it
  if (st != SBM_OK) return st;
  P.d = d; P.p = p; P.n = p + 1; P.N = N;
  P.nd = 1; P.L = 1;
  for (int i = 0; i < d; ++i) P.nd *= P.n;
  P.L = P.nd / P.n;
  P.h = 2.0 / N;
  if (desc.dg) {
    P.sigma = desc.pen_shift * (p + 1.0) * (p + 1.0) / P.h;
    P.sigma_f = desc.pen_interior * (p + 1.0) * (p + 1.0) / P.h;
  } else {
    P.sigma = desc.pen_shift * p * p / P.h;
    P.sigma_f = 0.0;
  }
  build_tables(p, &P.tab);
  if (!(P.tab.fd_residual <= 1e-12)) {
    *err = "1D eigenbasis of the cell operator is inaccurate";
    return SBM_ERR_UNSUPPORTED;
  }
  return SBM_OK;
}

int setup_geometry_host(HostProblem* hp, std::string* err) {
  HostProblem& P = *hp;
  const sbm_desc& desc = P.desc;
  const int d = P.d, N = P.N;
  const double h = P.h;
  const GeomView gv = P.ls.view();

  // active cells: phi(centre) < 0, centre = -1 + h (i + 1/2); or the volume
  // fraction (sub-cell midpoints with phi < 0) >= vf_threshold
  int64_t nbg = 1;
  for (int i = 0; i < d; ++i) nbg *= N;
  P.bg_to_cell.assign(nbg, -1);
  P.cells.clear();
  P.cell_bg.clear();
  for (int64_t b = 0; b < nbg; ++b) {
    int idx[3] = {0, 0, 0};
    int64_t r = b;
    double xc[3];
    for (int i = 0; i < d; ++i) {
      idx[i] = (int)(r % N);
      r /= N;
      xc[i] = -1.0 + h * (idx[i] + 0.5);
    }
    bool active;
    if (desc.activity == SBM_ACTIVE_VOLUME) {
      // volume fraction by the midpoint rule on kVfSamples^d sub-cells
      constexpr int m = kVfSamples;
      int count = 0, tot = 1;
      for (int i = 0; i < d; ++i) tot *= m;
      for (int s = 0; s < tot; ++s) {
        double xs[3];
        int rs = s;
        for (int i = 0; i < d; ++i) {
          xs[i] = -1.0 + h * ((double)idx[i] + ((rs % m) + 0.5) / m);
          rs /= m;
        }
        if (geom_phi(gv, xs) < 0.0) ++count;
      }
      active = (double)count >= desc.vf_threshold * (double)tot;
    } else {
      active = geom_phi(gv, xc) < 0.0;
    }
    if (active) {
      P.bg_to_cell[b] = (int32_t)P.cell_bg.size();
      P.cell_bg.push_back(b);
      for (int i = 0; i < d; ++i) P.cells.push_back(idx[i]);
    }
  }
  const int64_t Nc = (int64_t)P.cell_bg.size();
  if (Nc == 0) { *err = "no active cell"; return SBM_ERR_EMPTY_DOMAIN; }

  // faces
  int64_t stride[3] = {1, N, (int64_t)N * N};
  P.sfaces.clear();
  P.ifaces.clear();
  for (int64_t c = 0; c < Nc; ++c) {
    for (int k = 0; k < d; ++k)
      for (int s = 0; s < 2; ++s) {
        int j = P.cells[c * d + k] + (s ? 1 : -1);
        int32_t nb = -1;
        if (j >= 0 && j < N) nb = P.bg_to_cell[P.cell_bg[c] + (s ? 1 : -1) * stride[k]];
        if (nb < 0) {
          P.sfaces.push_back((int32_t)c); P.sfaces.push_back(k); P.sfaces.push_back(s);
        } else if (s == 1) {
          P.ifaces.push_back((int32_t)c); P.ifaces.push_back(k); P.ifaces.push_back(nb);
        }
      }
  }

  // surrogate face Gauss points, closest points, reference coordinates
  const int64_t F = (int64_t)P.sfaces.size() / 3;
  const int Q = P.L, n = P.n;
  P.face_x.assign(F * Q * d, 0.0);
  P.face_xi.assign(F * Q * d, 0.0);
  P.face_d.assign(F * Q * d, 0.0);
  for (int64_t f = 0; f < F; ++f) {
    const int c = P.sfaces[3 * f], k = P.sfaces[3 * f + 1], s = P.sfaces[3 * f + 2];
    int tang[2], nt = 0;
    for (int l = 0; l < d; ++l) if (l != k) tang[nt++] = l;
    double lo[3];
    for (int l = 0; l < d; ++l) lo[l] = -1.0 + h * (double)P.cells[c * d + l];
    for (int q = 0; q < Q; ++q) {
      int qa = q % n, qb = q / n;
      double xi[3], xt[3], xq[3];
      xi[k] = (double)s;
      xi[tang[0]] = P.tab.gpts[qa];
      if (d == 3) xi[tang[1]] = P.tab.gpts[qb];
      for (int l = 0; l < d; ++l) xt[l] = lo[l] + h * xi[l];
      if (!geom_closest(gv, xt, xq)) {
        *err = "closest-point projection undefined for a surrogate quadrature point";
        return SBM_ERR_GEOMETRY;
      }
      for (int l = 0; l < d; ++l) {
        P.face_x[(f * Q + q) * d + l] = xq[l];
        P.face_xi[(f * Q + q) * d + l] = (xq[l] - lo[l]) / h;
        P.face_d[(f * Q + q) * d + l] = xq[l] - xt[l];
      }
    }
  }

  return SBM_OK;
}

int setup_numbering(HostProblem* hp, std::string* err) {
  HostProblem& P = *hp;
  const sbm_desc& desc = P.desc;
  const int d = P.d, p = P.p, n = P.n, N = P.N;
  const int64_t Nc = (int64_t)P.cell_bg.size();
  if (desc.dg) {
    P.n_dofs = Nc * P.nd;
    if (P.n_dofs >= (int64_t(1) << 31)) { *err = "too many DoFs for int32 indices"; return SBM_ERR_ARG; }
    P.lines.clear();
  } else {
    const int64_t M = (int64_t)p * N + 1;
    int64_t nlat = 1;
    for (int i = 0; i < d; ++i) nlat *= M;
    std::vector<int32_t> idx(nlat, 0);
    const int64_t ms[3] = {1, M, M * M};
    for (int64_t c = 0; c < Nc; ++c) {
      int64_t base = 0;
      for (int l = 0; l < d; ++l) base += (int64_t)p * P.cells[c * d + l] * ms[l];
      for (int r = 0; r < P.nd; ++r) {
        int64_t off = 0, rr = r;
        for (int l = 0; l < d; ++l) { off += (rr % n) * ms[l]; rr /= n; }
        idx[base + off] = 1;
      }
    }
    int64_t cnt = 0;
    for (int64_t i = 0; i < nlat; ++i) {
      if (idx[i]) {
        if (cnt >= (int64_t(1) << 31) - 1) { *err = "too many DoFs for int32 indices"; return SBM_ERR_ARG; }
        idx[i] = (int32_t)cnt++;
      } else {
        idx[i] = -1;
      }
    }
    P.n_dofs = cnt;
    P.lines.assign(Nc * P.L, 0);
    for (int64_t c = 0; c < Nc; ++c) {
      int64_t base = 0;
      for (int l = 0; l < d; ++l) base += (int64_t)p * P.cells[c * d + l] * ms[l];
      for (int line = 0; line < P.L; ++line) {
        int64_t off = (d == 2) ? line * ms[1] : (line % n) * ms[1] + (line / n) * ms[2];
        P.lines[c * P.L + line] = idx[base + off];
      }
    }
  }
  return SBM_OK;
}

int build_host_problem(const sbm_desc& desc, HostProblem* hp, std::string* err) {
  int st = setup_prepare(desc, hp, err);
  if (st == SBM_OK) st = setup_geometry_host(hp, err);
  if (st == SBM_OK) st = setup_numbering(hp, err);
  return st;
}

// ---------------------------------------------------------------------------
// Manufactured data, right-hand side, interpolant
// ---------------------------------------------------------------------------

bool manufactured_ok(int id, int dim) { return id == 0 || (id == 1 && dim == 2); }

double manufactured_u(int id, int dim, const double* x) {
  const double pi = 3.14159265358979323846;
  if (id == 0) {
    double u = 1.0;
    for (int i = 0; i < dim; ++i) u *= std::sin(pi * x[i]);
    return u;
  }
  return 2.0 * std::cos(x[0]) * std::sin(x[1]);
}

double manufactured_f(int id, int dim, const double* x) {
  const double pi = 3.14159265358979323846;
  if (id == 0) return dim * pi * pi * manufactured_u(id, dim, x);
  return 2.0 * manufactured_u(id, dim, x);
}

// global index of local DoF j of active cell c
static int64_t global_dof(const HostProblem& P, int64_t c, int j) {
  if (P.desc.dg) return c * P.nd + j;
  return (int64_t)P.lines[c * P.L + j / P.n] + (j % P.n);
}

void build_rhs(const HostProblem& P, int id, double* b) {
  const int d = P.d, n = P.n, nd = P.nd, L = P.L;
  const double h = P.h;
  const Tables1D& T = P.tab;
  for (int64_t i = 0; i < P.n_dofs; ++i) b[i] = 0.0;
  const int64_t Nc = (int64_t)P.cell_bg.size();
  std::vector<double> Fq(nd), t1(nd), t2(nd);
  const double hd = std::pow(h, d);
  for (int64_t c = 0; c < Nc; ++c) {
    double lo[3];
    for (int l = 0; l < d; ++l) lo[l] = -1.0 + h * (double)P.cells[c * d + l];
    // f h^d w_q at the tensor Gauss points, q = q0 + n q1 (+ n^2 q2)
    for (int q = 0; q < nd; ++q) {
      int qq[3] = {q % n, (q / n) % n, q / (n * n)};
      double x[3], w = hd;
      for (int l = 0; l < d; ++l) {
        x[l] = lo[l] + h * T.gpts[qq[l]];
        w *= T.gwts[qq[l]];
      }
      Fq[q] = w * manufactured_f(id, d, x);
    }
    // b_K[j] = sum_q Fq[q] prod_l S[q_l][j_l]: one transposed sweep per axis
    std::vector<double>* src = &Fq;
    std::vector<double>* dst = &t1;
    int stride = 1;
    for (int l = 0; l < d; ++l) {
      for (int r = 0; r < nd; ++r) {
        const int jl = (r / stride) % n, base = r - jl * stride;
        double s = 0.0;
        for (int q = 0; q < n; ++q) s += T.S[q][jl] * (*src)[base + q * stride];
        (*dst)[r] = s;
      }
      src = dst;
      dst = (dst == &t1) ? &t2 : &t1;
      stride *= n;
    }
    for (int j = 0; j < nd; ++j) b[global_dof(P, c, j)] += (*src)[j];
  }
  // surrogate faces
  const int64_t F = (int64_t)P.sfaces.size() / 3;
  const double hd1 = std::pow(h, d - 1);
  for (int64_t f = 0; f < F; ++f) {
    const int c = P.sfaces[3 * f], k = P.sfaces[3 * f + 1], s = P.sfaces[3 * f + 2];
    int tang[2] = {0, 0}, nt = 0;
    for (int l = 0; l < d; ++l) if (l != k) tang[nt++] = l;
    const double sg = s ? 1.0 : -1.0;
    for (int q = 0; q < L; ++q) {
      const int qa = q % n, qb = q / n;
      const double W = hd1 * T.gwts[qa] * (d == 3 ? T.gwts[qb] : 1.0);
      const double g = manufactured_u(id, d, &P.face_x[(f * L + q) * d]);
      for (int j = 0; j < nd; ++j) {
        int jj[3] = {j % n, (j / n) % n, j / (n * n)};
        double tg = T.S[qa][jj[tang[0]]];
        if (d == 3) tg *= T.S[qb][jj[tang[1]]];
        const double v = (jj[k] == (s ? n - 1 : 0)) ? tg : 0.0;
        const double dn = sg / h * (s ? T.D1[jj[k]] : T.D0[jj[k]]) * tg;
        const double contrib = W * g * (P.sigma * v - dn);
        if (contrib != 0.0) b[global_dof(P, c, j)] += contrib;
      }
    }
  }
}

void build_interpolant(const HostProblem& P, int id, double* u) {
  const int d = P.d, n = P.n, nd = P.nd;
  const double h = P.h;
  const int64_t Nc = (int64_t)P.cell_bg.size();
  for (int64_t c = 0; c < Nc; ++c) {
    double lo[3];
    for (int l = 0; l < d; ++l) lo[l] = -1.0 + h * (double)P.cells[c * d + l];
    for (int j = 0; j < nd; ++j) {
      int jj[3] = {j % n, (j / n) % n, j / (n * n)};
      double x[3];
      for (int l = 0; l < d; ++l) x[l] = lo[l] + h * P.tab.nodes[jj[l]];
      u[global_dof(P, c, j)] = manufactured_u(id, d, x);
    }
  }
}

}  // namespace sbm
