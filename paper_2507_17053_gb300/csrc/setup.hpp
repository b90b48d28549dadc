// Host-side (FP64) set-up of an SBM problem: 1D tables, level sets and closest
// points, active cells, surrogate faces, DoF numbering and the per-face data
// the kernels read.  Plain C++; no CUDA in this file's interface.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "geom.hpp"
#include "sbm.h"

namespace sbm {

constexpr int kMaxN = 7;   // n = p + 1 <= 7 (degrees 1..6)

// 1D tables on the reference interval [0,1] for n = p+1 GLL nodes and n Gauss
// points (Section 3.1: tensor-product basis and Gauss quadrature).
struct Tables1D {
  int n = 0;
  double nodes[kMaxN] = {};        // GLL nodes x_j
  double gpts[kMaxN] = {};         // Gauss points g_q
  double gwts[kMaxN] = {};         // Gauss weights w_q
  double S[kMaxN][kMaxN] = {};     // S[q][j] = phi_j(g_q)       (nodes -> Gauss points)
  double Dg[kMaxN][kMaxN] = {};    // Dg[q][j] = phi_j'(g_q)
  double M[kMaxN][kMaxN] = {};     // 1D mass      sum_q w_q phi_i(g_q) phi_j(g_q)
  double K[kMaxN][kMaxN] = {};     // 1D stiffness sum_q w_q phi_i'(g_q) phi_j'(g_q)
  double D0[kMaxN] = {};           // phi_j'(0)
  double D1[kMaxN] = {};           // phi_j'(1)
  // Eigenbasis of the pencil (K, M): M = V V^T, K = V diag(lam) V^T.  The
  // columns of V are even or odd about the interval's midpoint (M and K are
  // centrosymmetric on symmetric nodes): the ceil(n/2) even modes first, then
  // the floor(n/2) odd ones, each group by increasing eigenvalue.
  double V[kMaxN][kMaxN] = {};
  double lam[kMaxN] = {};
  double fd_residual = 0.0;        // max |V V^T - M| + max |V lam V^T - K|, relative
};

// GLL nodes by Newton on (1-t^2) P_p'(t) with the Legendre recurrence, Gauss
// points by Newton on P_n(t); Lagrange values by the barycentric formula.
void build_tables(int p, Tables1D* t);
void lagrange_values(const Tables1D& t, double x, double* phi);     // phi[j], any real x
void lagrange_derivs(const Tables1D& t, double x, double* dphi);

constexpr int kVfSamples = 8;    // sub-cells per axis of the volume-fraction estimate

struct LevelSet {
  int kind = 0, dim = 0;
  double c[3] = {0, 0, 0};
  double r = 0;
  double a[3] = {1, 1, 1};
  double R[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
  double Rmaj = 0, rmin = 0;
  double half[3] = {0, 0, 0};
  // union of balls: centres, radii, pairwise intersection circles (3D) and
  // the boundary vertices
  std::vector<double> bc, br;          // [nb * 3] (dim used), [nb]
  std::vector<GeomCircle> circles;
  std::vector<double> verts;           // [nv * 3]

  int init(int kind, int dim, const double* g, std::string* err);
  int init_balls(int dim, int nballs, const double* balls, std::string* err);
  // a plain view (host pointers into this object) for geom_phi / geom_closest
  GeomView view() const;
  double phi(const double* x) const { return geom_phi(view(), x); }
  // closest point on Gamma; returns false if the projection is undefined
  bool closest(const double* x, double* out) const { return geom_closest(view(), x, out); }
};

struct HostProblem {
  sbm_desc desc{};
  int d = 0, p = 0, n = 0, N = 0;
  int nd = 0;        // n^d
  int L = 0;         // n^(d-1) lines per cell / points per face
  double h = 0, sigma = 0, sigma_f = 0;
  Tables1D tab;
  LevelSet ls;

  // active cells, lexicographic (axis 0 fastest)
  std::vector<int32_t> cells;       // [Nc * d]
  std::vector<int64_t> cell_bg;     // background linear index
  std::vector<int32_t> bg_to_cell;  // [N^d] -> rank or -1
  // surrogate faces (cell rank, k, s), by cell, then k, then s
  std::vector<int32_t> sfaces;      // [F * 3]
  std::vector<double> face_x;       // [F * L * d] closest points
  std::vector<double> face_xi;      // [F * L * d] reference coordinates in the cell's frame
  std::vector<double> face_d;       // [F * L * d] shift d = x_q - x~_q (physical)
  // DG interior faces (K1 rank, k, K2 rank), K2 = K1 + e_k
  std::vector<int32_t> ifaces;

  int64_t n_dofs = 0;
  // CG: per active cell, the global index of local node (0, j1, j2) for each
  // of the L x-lines (j1 + n j2); the n nodes of an x-line are consecutive.
  std::vector<int32_t> lines;       // [Nc * L]
};

// Build everything on the host.  Returns SBM_OK or an error code with *err set.
int build_host_problem(const sbm_desc& desc, HostProblem* hp, std::string* err);
// The three stages of it: checks, 1D tables and level set; active cells,
// surrogate faces and closest points; DoF numbering.  The middle stage has a
// device counterpart (setup_geometry_device, setup_gpu.cu) with identical
// results.
int setup_prepare(const sbm_desc& desc, HostProblem* hp, std::string* err);
int setup_geometry_host(HostProblem* hp, std::string* err);
int setup_numbering(HostProblem* hp, std::string* err);
int setup_geometry_device(HostProblem* hp, int device, std::string* err);
int setup_numbering_device(HostProblem* hp, int device, std::string* err);

// Manufactured solutions: 0 = prod_i sin(pi x_i) (f = d pi^2 u),
// 1 = 2 cos(x_0) sin(x_1) in 2D (f = 2 u).
bool manufactured_ok(int id, int dim);
double manufactured_u(int id, int dim, const double* x);
double manufactured_f(int id, int dim, const double* x);

// Right-hand side of the weak form (Section 2.1):
//   b_i = int f v_i - int_F (grad v_i . n~) g(x) + int_F sigma g(x) v_i,
// g = u at the true-boundary point x_q of each surrogate quadrature point.
void build_rhs(const HostProblem& hp, int id, double* b);
// Nodal interpolant of the manufactured solution (DoF values at the nodes).
void build_interpolant(const HostProblem& hp, int id, double* u);

}  // namespace sbm
