// Device building blocks shared by the apply kernels: tile shapes and the
// sum-factorised cell sweeps (Algorithm 1).
//
// Cell term.  With Gauss quadrature of n = p+1 points per axis the cell
// integral of grad u . grad v is exact, so on a Cartesian cell
//   A_K = h^(d-2) sum_k (M x ... x K_k x ... x M)
// with the exact 1D mass M and stiffness K on [0,1].  It is evaluated with 7
// one-dimensional sweeps in 3D (4 in 2D) instead of the 4d sweeps of
// interpolate / differentiate / integrate:
//   a = M_z u, e = K_z u;  b = M_y a, g = K_y a + M_y e;  y = h (K_x b + M_x g).
// Each thread owns one line of the (p+1)^d tile per sweep (registers); the
// tile is staged in shared memory between sweeps.
#pragma once

#include "internal.hpp"

namespace sbm {

template <int D, int N>
struct Shape {
  static constexpr int L = (D == 3) ? N * N : N;   // lines per cell, points per face
  static constexpr int ND = L * N;                  // DoFs per cell
  static constexpr int CPB = (128 / L) > 0 ? (128 / L) : 1;
};

// ---- cell term -------------------------------------------------------------

// 3D: three phases over z-, y- and x-lines.  `X` holds ncells tiles; the x-line
// result of line `tl` of cell `c` is returned in out[].
template <typename T, int N>
__device__ __forceinline__ void cell_sweeps_3d(const KTab<T>& t, const T* X, T* A, T* E, T* B,
                                               T* G, int c, int tl, bool act, T (&out)[N]) {
  constexpr int ND = N * N * N;
  if (act) {
    const int base = c * ND + (tl % N) + N * (tl / N);      // z-line (j0, j1)
    T v[N];
#pragma unroll
    for (int j = 0; j < N; ++j) v[j] = X[base + N * N * j];
#pragma unroll
    for (int m = 0; m < N; ++m) {
      T a = T(0), e = T(0);
#pragma unroll
      for (int j = 0; j < N; ++j) {
        a = fma(t.M[m][j], v[j], a);
        e = fma(t.K[m][j], v[j], e);
      }
      A[base + N * N * m] = a;
      E[base + N * N * m] = e;
    }
  }
  __syncthreads();
  if (act) {
    const int base = c * ND + (tl % N) + N * N * (tl / N);  // y-line (j0, j2)
    T va[N], ve[N];
#pragma unroll
    for (int j = 0; j < N; ++j) {
      va[j] = A[base + N * j];
      ve[j] = E[base + N * j];
    }
#pragma unroll
    for (int m = 0; m < N; ++m) {
      T b = T(0), g = T(0);
#pragma unroll
      for (int j = 0; j < N; ++j) {
        b = fma(t.M[m][j], va[j], b);
        g = fma(t.K[m][j], va[j], g);
        g = fma(t.M[m][j], ve[j], g);
      }
      B[base + N * m] = b;
      G[base + N * m] = g;
    }
  }
  __syncthreads();
  if (act) {
    const int base = c * ND + N * tl;                       // x-line (j1, j2) = line tl
    T vb[N], vg[N];
#pragma unroll
    for (int j = 0; j < N; ++j) {
      vb[j] = B[base + j];
      vg[j] = G[base + j];
    }
#pragma unroll
    for (int m = 0; m < N; ++m) {
      T o = T(0);
#pragma unroll
      for (int j = 0; j < N; ++j) {
        o = fma(t.Kh[m][j], vb[j], o);
        o = fma(t.Mh[m][j], vg[j], o);
      }
      out[m] = o;
    }
  }
}

// 2D: y-lines then x-lines.
template <typename T, int N>
__device__ __forceinline__ void cell_sweeps_2d(const KTab<T>& t, const T* X, T* A, T* E, int c,
                                               int tl, bool act, T (&out)[N]) {
  constexpr int ND = N * N;
  if (act) {
    const int base = c * ND + tl;                           // y-line j0 = tl
    T v[N];
#pragma unroll
    for (int j = 0; j < N; ++j) v[j] = X[base + N * j];
#pragma unroll
    for (int m = 0; m < N; ++m) {
      T a = T(0), e = T(0);
#pragma unroll
      for (int j = 0; j < N; ++j) {
        a = fma(t.M[m][j], v[j], a);
        e = fma(t.K[m][j], v[j], e);
      }
      A[base + N * m] = a;
      E[base + N * m] = e;
    }
  }
  __syncthreads();
  if (act) {
    const int base = c * ND + N * tl;                       // x-line j1 = tl
    T va[N], ve[N];
#pragma unroll
    for (int j = 0; j < N; ++j) {
      va[j] = A[base + j];
      ve[j] = E[base + j];
    }
#pragma unroll
    for (int m = 0; m < N; ++m) {
      T o = T(0);
#pragma unroll
      for (int j = 0; j < N; ++j) {
        o = fma(t.Kh[m][j], va[j], o);
        o = fma(t.Mh[m][j], ve[j], o);
      }
      out[m] = o;
    }
  }
}

}  // namespace sbm
