// Level sets and closest points of the true boundary Gamma, shared by the
// host set-up (setup.cpp) and the device set-up (setup_gpu.cu): one source,
// compiled without fused multiply-adds on both sides (g++ -ffp-contract=off,
// nvcc --fmad=false), so the two produce the same active cells, faces and
// closest points to the last bit.
//
// phi < 0 inside Omega.  Closest points (Section 2.1: x = the closest-point
// projection of x~ onto Gamma):
//  * ball, torus: closed forms; box: clamp / nearest face;
//  * ellipsoid: in the frame y = R^T (x - c) the closest point is
//    z_i = a_i^2 y_i / (a_i^2 + t), t the root on (-a_min^2, inf) of
//    F(t) = sum_i (a_i y_i / (a_i^2 + t))^2 - 1 (D. Eberly, "Distance from a
//    point to an ellipse, an ellipsoid, or a hyperellipsoid"); F is convex and
//    decreasing there: safeguarded Newton (bisection whenever a Newton step
//    leaves the bracket);
//  * union of balls (Section 4.3): the nearest of the candidates that lie on
//    the union's boundary -- projections onto each sphere, nearest points of
//    the pairwise intersection circles (3D), the boundary vertices -- a
//    candidate strictly inside another ball being discarded; ties go to the
//    first candidate in that order.
#pragma once

#include <cmath>
#include <cstdint>

#include "sbm.h"

#ifdef __CUDACC__
#define SBM_HD __host__ __device__
#else
#define SBM_HD
#endif

namespace sbm {

struct GeomCircle {
  int i, j;               // the two balls
  double m[3], u[3], rho; // centre, unit axis, radius
};

// Plain view of a level set (host or device pointers for the ball data).
struct GeomView {
  int kind = 0, dim = 0;
  double c[3] = {0, 0, 0};
  double r = 0;
  double a[3] = {1, 1, 1};
  double R[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
  double Rmaj = 0, rmin = 0;
  double half[3] = {0, 0, 0};
  int nb = 0, ncirc = 0, nvert = 0;
  const double* bc = nullptr;          // [nb * 3] centres
  const double* br = nullptr;          // [nb] radii
  const GeomCircle* circ = nullptr;    // [ncirc]
  const double* verts = nullptr;       // [nvert * 3]
};

SBM_HD inline double gv_norm(const double* v, int d) {
  double s = 0.0;
  for (int l = 0; l < d; ++l) s = s + v[l] * v[l];
  return sqrt(s);
}

SBM_HD inline double gv_dist(const double* x, const double* c, int d) {
  double v[3];
  for (int l = 0; l < d; ++l) v[l] = x[l] - c[l];
  return gv_norm(v, d);
}

// p is not strictly inside any ball other than s0, s1, s2 (-1: unused)
SBM_HD inline bool gv_outside_others(const GeomView& g, const double* p, int s0, int s1, int s2) {
  for (int l = 0; l < g.nb; ++l) {
    if (l == s0 || l == s1 || l == s2) continue;
    if (!(gv_dist(p, g.bc + 3 * l, g.dim) >= g.br[l])) return false;
  }
  return true;
}

SBM_HD inline double geom_phi(const GeomView& g, const double* x) {
  const int dim = g.dim;
  switch (g.kind) {
    case SBM_GEOM_BALL: {
      double s = 0.0;
      for (int i = 0; i < dim; ++i) s = s + (x[i] - g.c[i]) * (x[i] - g.c[i]);
      return sqrt(s) - g.r;
    }
    case SBM_GEOM_ELLIPSOID: {
      double s = 0.0;
      for (int i = 0; i < dim; ++i) {
        double y = 0.0;
        for (int j = 0; j < dim; ++j) y = y + g.R[j * dim + i] * (x[j] - g.c[j]);
        s = s + (y / g.a[i]) * (y / g.a[i]);
      }
      return s - 1.0;
    }
    case SBM_GEOM_TORUS: {
      double rho = sqrt(x[0] * x[0] + x[1] * x[1]);
      return (rho - g.Rmaj) * (rho - g.Rmaj) + x[2] * x[2] - g.rmin * g.rmin;
    }
    case SBM_GEOM_BOX: {
      double m = fabs(x[0] - g.c[0]) - g.half[0];
      for (int i = 1; i < dim; ++i) {
        const double v = fabs(x[i] - g.c[i]) - g.half[i];
        m = (m < v) ? v : m;
      }
      return m;
    }
    case SBM_GEOM_BALLS: {
      double m = gv_dist(x, g.bc, dim) - g.br[0];
      for (int b = 1; b < g.nb; ++b) {
        const double v = gv_dist(x, g.bc + 3 * b, dim) - g.br[b];
        m = (v < m) ? v : m;
      }
      return m;
    }
  }
  return 1.0;
}

SBM_HD inline bool geom_ellipsoid_root(int d, const double* a, const double* y, double* tout) {
  double a2[3], amin2 = 1e300, amax = 0, yn = 0, f0 = -1.0;
  for (int i = 0; i < d; ++i) {
    a2[i] = a[i] * a[i];
    amin2 = (a2[i] < amin2) ? a2[i] : amin2;
    amax = (amax < a[i]) ? a[i] : amax;
    yn += y[i] * y[i];
    f0 += (y[i] / a[i]) * (y[i] / a[i]);
  }
  yn = sqrt(yn);
  if (f0 == 0.0) {
    *tout = 0.0;
    return true;
  }
  double lo, hi;
  if (f0 > 0) {
    lo = 0.0;
    hi = amax * yn;
  } else {
    lo = -amin2;
    hi = 0.0;
    // the root exists in (-a_min^2, 0) only if some y_i on a shortest axis is non-zero
    bool ok = false;
    for (int i = 0; i < d; ++i)
      if (a2[i] == amin2 && y[i] != 0.0) ok = true;
    if (!ok) return false;
  }
  double t = (f0 > 0) ? 0.0 : 0.5 * (lo + hi);
  for (int it = 0; it < 300; ++it) {
    double F = -1.0, dF = 0.0;
    for (int i = 0; i < d; ++i) {
      double q = a[i] * y[i] / (a2[i] + t);
      F += q * q;
      dF += -2.0 * q * q / (a2[i] + t);
    }
    if (F > 0) lo = t;
    else hi = t;
    if (F == 0.0) break;
    double tn = t - F / dF;
    if (!(tn > lo && tn < hi)) tn = 0.5 * (lo + hi);
    const double at = fabs(t);
    if (fabs(tn - t) <= 1e-16 * ((1.0 < at) ? at : 1.0) || tn == lo || tn == hi) {
      t = tn;
      break;
    }
    t = tn;
  }
  *tout = t;
  return true;
}

// closest point on Gamma; false if the projection is undefined
SBM_HD inline bool geom_closest(const GeomView& g, const double* x, double* out) {
  const int dim = g.dim;
  switch (g.kind) {
    case SBM_GEOM_BALL: {
      double v[3], s = 0.0;
      for (int i = 0; i < dim; ++i) {
        v[i] = x[i] - g.c[i];
        s += v[i] * v[i];
      }
      s = sqrt(s);
      if (!(s > 0)) return false;
      for (int i = 0; i < dim; ++i) out[i] = g.c[i] + g.r * v[i] / s;
      return true;
    }
    case SBM_GEOM_TORUS: {
      double rho = sqrt(x[0] * x[0] + x[1] * x[1]);
      if (!(rho > 0)) return false;
      double q[3] = {g.Rmaj * x[0] / rho, g.Rmaj * x[1] / rho, 0.0};
      double v[3], s = 0.0;
      for (int i = 0; i < 3; ++i) {
        v[i] = x[i] - q[i];
        s += v[i] * v[i];
      }
      s = sqrt(s);
      if (!(s > 0)) return false;
      for (int i = 0; i < 3; ++i) out[i] = q[i] + g.rmin * v[i] / s;
      return true;
    }
    case SBM_GEOM_BOX: {
      double v[3] = {0, 0, 0};
      bool inside = true;
      for (int i = 0; i < dim; ++i) {
        v[i] = x[i] - g.c[i];
        if (fabs(v[i]) > g.half[i]) inside = false;
      }
      if (!inside) {
        for (int i = 0; i < dim; ++i) {
          const double cl = (v[i] < -g.half[i]) ? -g.half[i] : ((v[i] > g.half[i]) ? g.half[i] : v[i]);
          out[i] = g.c[i] + cl;
        }
        return true;
      }
      int kmin = 0;
      double gmin = g.half[0] - fabs(v[0]);
      for (int i = 1; i < dim; ++i) {
        double gap = g.half[i] - fabs(v[i]);
        if (gap < gmin) {
          gmin = gap;
          kmin = i;
        }
      }
      for (int i = 0; i < dim; ++i) out[i] = x[i];
      out[kmin] = g.c[kmin] + (v[kmin] >= 0 ? g.half[kmin] : -g.half[kmin]);
      return true;
    }
    case SBM_GEOM_ELLIPSOID: {
      double y[3] = {0, 0, 0}, z[3] = {0, 0, 0}, t = 0.0;
      for (int i = 0; i < dim; ++i) {
        double s = 0.0;
        for (int j = 0; j < dim; ++j) s += g.R[j * dim + i] * (x[j] - g.c[j]);
        y[i] = s;
      }
      if (!geom_ellipsoid_root(dim, g.a, y, &t)) return false;
      for (int i = 0; i < dim; ++i) z[i] = g.a[i] * g.a[i] * y[i] / (g.a[i] * g.a[i] + t);
      for (int i = 0; i < dim; ++i) {
        double s = 0.0;
        for (int j = 0; j < dim; ++j) s += g.R[i * dim + j] * z[j];
        out[i] = g.c[i] + s;
      }
      return true;
    }
    case SBM_GEOM_BALLS: {
      double best = INFINITY;
      bool found = false;
      auto take = [&](const double* p) {
        double d2 = 0.0;
        for (int l = 0; l < dim; ++l) d2 = d2 + (p[l] - x[l]) * (p[l] - x[l]);
        if (d2 < best) {
          best = d2;
          for (int l = 0; l < dim; ++l) out[l] = p[l];
          found = true;
        }
      };
      for (int i = 0; i < g.nb; ++i) {                   // projections onto each sphere
        double v[3], p[3];
        for (int l = 0; l < dim; ++l) v[l] = x[l] - g.bc[3 * i + l];
        const double s = gv_norm(v, dim);
        if (!(s > 0)) continue;
        for (int l = 0; l < dim; ++l) p[l] = g.bc[3 * i + l] + g.br[i] * v[l] / s;
        if (gv_outside_others(g, p, i, -1, -1)) take(p);
      }
      for (int q = 0; q < g.ncirc; ++q) {                // nearest points of the circles
        const GeomCircle& C = g.circ[q];
        double w[3], wp[3], p[3];
        for (int l = 0; l < 3; ++l) w[l] = x[l] - C.m[l];
        const double t = w[0] * C.u[0] + w[1] * C.u[1] + w[2] * C.u[2];
        for (int l = 0; l < 3; ++l) wp[l] = w[l] - t * C.u[l];
        const double s = gv_norm(wp, 3);
        if (!(s > 0)) continue;
        for (int l = 0; l < 3; ++l) p[l] = C.m[l] + C.rho * wp[l] / s;
        if (gv_outside_others(g, p, C.i, C.j, -1)) take(p);
      }
      for (int q = 0; q < g.nvert; ++q) take(g.verts + 3 * q);
      return found;
    }
  }
  return false;
}

}  // namespace sbm
