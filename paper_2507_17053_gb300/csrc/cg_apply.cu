// Matrix-free apply (FP64 or FP32) of the continuous Galerkin SBM operator on sm_103a.
//
// One launch per cell colour (2^d colours: cells whose indices have the same
// parity pattern share no DoF), so the scatter y += A_K x_K is a plain
// read-modify-write without atomics and repeated applies are bitwise equal.
// Inside a colour, blocks [0, nint_tiles) process CPB interior cells each;
// every further block processes one cell that owns surrogate faces: its cell
// term, then each of its faces (Algorithm 3), then the scatter.
//
// Cell term (Algorithm 1).  With Gauss quadrature of n = p+1 points per axis
// the cell integral of grad u . grad v is exact, so on a Cartesian cell
//   A_K = h^(d-2) sum_k (M x ... x K_k x ... x M)
// with the exact 1D mass M and stiffness K on [0,1].  The kernel evaluates it
// with 7 one-dimensional sweeps in 3D (4 in 2D) instead of the 4d sweeps of
// interpolate/differentiate/integrate:
//   a = M_z u, e = K_z u;  b = M_y a, g = K_y a + M_y e;  y = h (K_x b + M_x g).
// Each thread owns one line of the (p+1)^d tile per sweep (registers); the
// tile is staged in shared memory between sweeps.
#include "internal.hpp"

namespace sbm {

template <int D, int N>
struct Shape {
  static constexpr int L = (D == 3) ? N * N : N;   // lines per cell, points per face
  static constexpr int ND = L * N;                  // DoFs per cell
  static constexpr int CPB = (128 / L) > 0 ? (128 / L) : 1;
};

CellLaunch cell_launch_shape(int d, int n) {
  int L = (d == 3) ? n * n : n;
  int cpb = 128 / L;
  if (cpb < 1) cpb = 1;
  return CellLaunch{d, n, cpb, cpb * L};
}

template <typename T>
struct CgArgs {
  const T* __restrict__ x;
  T* __restrict__ y;
  const int32_t* __restrict__ lines;       // ordered cells x L
  const int32_t* __restrict__ face_start;  // ordered cells + 1
  const int32_t* __restrict__ face_kind;
  const T* __restrict__ face_phi;
  int cell0;        // first ordered cell of the colour
  int nint;         // interior cells of the colour (first in the colour's range)
  int nint_tiles;   // ceil(nint / CPB)
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

// ---- surrogate face (Algorithm 3) --------------------------------------------
//
// For the face (k, s) of the cell tile X: u and the reference normal
// derivative at the face Gauss points by sum factorisation (GLL nodes contain
// the end points, so the value trace is the face slice of X); u at the shifted
// points x_q by point evaluation with the stored 1D values phi_j(xi_{q,l});
//   val_q = W_q (sigma E_q - dn u(x~_q)),   grd_q = -W_q E_q,
// integrated against v and dn v at x~_q by transposed sum factorisation and
// added to R.  sc must hold 10 L doubles.  All threads of the block call it.
template <typename T, int D, int N>
__device__ void face_apply(const KTab<T>& t, const T* X, T* R, T* sc, const T* __restrict__ phi,
                           int k, int s) {
  constexpr int L = Shape<D, N>::L;
  const int tid = threadIdx.x;
  T* Tu = sc;
  T* Td = sc + L;
  T* Ua = sc + 2 * L;
  T* Da = sc + 3 * L;
  T* Ug = sc + 4 * L;
  T* Dg = sc + 5 * L;
  T* val = sc + 6 * L;
  T* grd = sc + 7 * L;
  T* Va = sc + 8 * L;
  T* Ga = sc + 9 * L;
  // strides of the normal axis and the tangential axes (ascending)
  int sk, sa, sb;
  if (D == 2) {
    sk = (k == 0) ? 1 : N;
    sa = (k == 0) ? N : 1;
    sb = 0;
  } else {
    sk = (k == 0) ? 1 : (k == 1 ? N : N * N);
    sa = (k == 0) ? N : 1;
    sb = (k == 2) ? N : N * N;
  }
  const int kend = s ? (N - 1) : 0;
  const T sg = s ? T(1) : T(-1);

  // 1. traces at the tangential nodes: value and reference normal derivative
  if (tid < L) {
    const int bt = (tid % N) * sa + (D == 3 ? (tid / N) * sb : 0);
    Tu[tid] = X[kend * sk + bt];
    T dsum = T(0);
#pragma unroll
    for (int j = 0; j < N; ++j) dsum = fma(s ? t.D1[j] : t.D0[j], X[j * sk + bt], dsum);
    Td[tid] = dsum;
  }
  __syncthreads();
  // 2. interpolate to the tangential Gauss points
  if (D == 3) {
    if (tid < L) {
      const int qa = tid % N, jb = tid / N;
      T u = T(0), dv = T(0);
#pragma unroll
      for (int j = 0; j < N; ++j) {
        u = fma(t.S[qa][j], Tu[j + N * jb], u);
        dv = fma(t.S[qa][j], Td[j + N * jb], dv);
      }
      Ua[tid] = u;
      Da[tid] = dv;
    }
    __syncthreads();
    if (tid < L) {
      const int qa = tid % N, qb = tid / N;
      T u = T(0), dv = T(0);
#pragma unroll
      for (int j = 0; j < N; ++j) {
        u = fma(t.S[qb][j], Ua[qa + N * j], u);
        dv = fma(t.S[qb][j], Da[qa + N * j], dv);
      }
      Ug[tid] = u;
      Dg[tid] = dv;
    }
  } else {
    if (tid < L) {
      T u = T(0), dv = T(0);
#pragma unroll
      for (int j = 0; j < N; ++j) {
        u = fma(t.S[tid][j], Tu[j], u);
        dv = fma(t.S[tid][j], Td[j], dv);
      }
      Ug[tid] = u;
      Dg[tid] = dv;
    }
  }
  __syncthreads();
  // 3. point evaluation at the shifted points and the pointwise integrands
  if (tid < L) {
    const T* pq = phi + (size_t)tid * D * N;
    T p0[N], p1[N];
#pragma unroll
    for (int j = 0; j < N; ++j) {
      p0[j] = __ldg(pq + j);
      p1[j] = __ldg(pq + N + j);
    }
    T e = T(0);
    if (D == 3) {
      T p2[N];
#pragma unroll
      for (int j = 0; j < N; ++j) p2[j] = __ldg(pq + 2 * N + j);
#pragma unroll
      for (int j2 = 0; j2 < N; ++j2) {
        T s1 = T(0);
#pragma unroll
        for (int j1 = 0; j1 < N; ++j1) {
          T s0 = T(0);
#pragma unroll
          for (int j0 = 0; j0 < N; ++j0) s0 = fma(p0[j0], X[j0 + N * j1 + N * N * j2], s0);
          s1 = fma(p1[j1], s0, s1);
        }
        e = fma(p2[j2], s1, e);
      }
    } else {
#pragma unroll
      for (int j1 = 0; j1 < N; ++j1) {
        T s0 = T(0);
#pragma unroll
        for (int j0 = 0; j0 < N; ++j0) s0 = fma(p0[j0], X[j0 + N * j1], s0);
        e = fma(p1[j1], s0, e);
      }
    }
    const T W = t.W[tid];
    const T dn = sg * t.h_inv * Dg[tid];
    val[tid] = W * (t.sigma * e - dn);
    grd[tid] = -W * e * sg * t.h_inv;
  }
  __syncthreads();
  // 4. transposed interpolation back to the tangential nodes, 5. add to R
  T rv = T(0), rg = T(0);
  if (D == 3) {
    if (tid < L) {
      const int ja = tid % N, qb = tid / N;
      T a = T(0), g = T(0);
#pragma unroll
      for (int q = 0; q < N; ++q) {
        a = fma(t.S[q][ja], val[q + N * qb], a);
        g = fma(t.S[q][ja], grd[q + N * qb], g);
      }
      Va[tid] = a;
      Ga[tid] = g;
    }
    __syncthreads();
    if (tid < L) {
      const int ja = tid % N, jb = tid / N;
#pragma unroll
      for (int q = 0; q < N; ++q) {
        rv = fma(t.S[q][jb], Va[ja + N * q], rv);
        rg = fma(t.S[q][jb], Ga[ja + N * q], rg);
      }
    }
  } else {
    if (tid < L) {
#pragma unroll
      for (int q = 0; q < N; ++q) {
        rv = fma(t.S[q][tid], val[q], rv);
        rg = fma(t.S[q][tid], grd[q], rg);
      }
    }
  }
  if (tid < L) {
    const int bt = (tid % N) * sa + (D == 3 ? (tid / N) * sb : 0);
    R[kend * sk + bt] += rv;
#pragma unroll
    for (int j = 0; j < N; ++j) R[j * sk + bt] = fma(s ? t.D1[j] : t.D0[j], rg, R[j * sk + bt]);
  }
  __syncthreads();
}

// ---- the kernel ----------------------------------------------------------------

template <typename T, int D, int N>
__global__ void __launch_bounds__(Shape<D, N>::CPB * Shape<D, N>::L)
cg_apply_kernel(const CgArgs<T> a, const __grid_constant__ KTab<T> t) {
  constexpr int L = Shape<D, N>::L, ND = Shape<D, N>::ND, CPB = Shape<D, N>::CPB;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* X = reinterpret_cast<T*>(smem_raw);
  T* A = X + CPB * ND;
  T* E = A + CPB * ND;
  T* B = E + CPB * ND;
  T* G = B + CPB * ND;
  T* sc = G + CPB * ND;
  const int tid = threadIdx.x;

  if ((int)blockIdx.x < a.nint_tiles) {
    // ---------------- interior tile: CPB cells, cell term only
    const int first = a.cell0 + blockIdx.x * CPB;
    const int ncells = min(CPB, a.nint - (int)blockIdx.x * CPB);
    for (int r = tid; r < ncells * ND; r += blockDim.x) {
      const int c = r / ND, loc = r - c * ND, line = loc / N, j0 = loc - line * N;
      X[r] = __ldg(a.x + __ldg(a.lines + (size_t)(first + c) * L + line) + j0);
    }
    __syncthreads();
    const int c = tid / L, tl = tid - c * L;
    const bool act = c < ncells;
    T out[N];
    if (D == 3) cell_sweeps_3d<T, N>(t, X, A, E, B, G, c, tl, act, out);
    else cell_sweeps_2d<T, N>(t, X, A, E, c, tl, act, out);
    if (act) {
      const int g0 = __ldg(a.lines + (size_t)(first + c) * L + tl);
#pragma unroll
      for (int m = 0; m < N; ++m) a.y[g0 + m] += out[m];
    }
    return;
  }

  // ---------------- one cell with surrogate faces
  const int cell = a.cell0 + a.nint + ((int)blockIdx.x - a.nint_tiles);
  for (int r = tid; r < ND; r += blockDim.x) {
    const int line = r / N, j0 = r - line * N;
    X[r] = __ldg(a.x + __ldg(a.lines + (size_t)cell * L + line) + j0);
  }
  __syncthreads();
  const bool act = tid < L;
  T out[N];
  if (D == 3) cell_sweeps_3d<T, N>(t, X, A, E, B, G, 0, tid, act, out);
  else cell_sweeps_2d<T, N>(t, X, A, E, 0, tid, act, out);
  __syncthreads();
  T* R = A;   // A is no longer read: it becomes the cell's result tile
  if (act) {
#pragma unroll
    for (int m = 0; m < N; ++m) R[N * tid + m] = out[m];
  }
  __syncthreads();
  const int fs = __ldg(a.face_start + cell), fe = __ldg(a.face_start + cell + 1);
  for (int f = fs; f < fe; ++f) {
    const int kind = __ldg(a.face_kind + f);
    face_apply<T, D, N>(t, X, R, sc, a.face_phi + (size_t)f * L * D * N, kind & 3, kind >> 2);
  }
  if (act) {
    const int g0 = __ldg(a.lines + (size_t)cell * L + tid);
#pragma unroll
    for (int m = 0; m < N; ++m) a.y[g0 + m] += R[N * tid + m];
  }
}

template <typename T, int D, int N>
static cudaError_t launch_t(const HostProblem& hp, const DeviceData& dd, const T* x, T* y,
                            cudaStream_t st, Profiler* prof) {
  constexpr int L = Shape<D, N>::L, ND = Shape<D, N>::ND, CPB = Shape<D, N>::CPB;
  const KTab<T> t = make_ktab<T>(hp);
  const size_t smem = (size_t)(5 * CPB * ND + 10 * L) * sizeof(T);
  cudaError_t err = cudaMemsetAsync(y, 0, (size_t)hp.n_dofs * sizeof(T), st);
  if (err != cudaSuccess) return err;
  if (prof && prof->on && (err = prof->begin(st)) != cudaSuccess) return err;
  int nlaunch = 0;
  for (int c = 0; c < dd.ncolours; ++c) {
    const int n = dd.col_start[c + 1] - dd.col_start[c];
    if (n == 0) continue;
    CgArgs<T> a;
    a.x = x;
    a.y = y;
    a.lines = dd.lines;
    a.face_start = dd.face_start;
    a.face_kind = dd.face_kind;
    a.face_phi = face_phi_of<T>(dd);
    a.cell0 = dd.col_start[c];
    a.nint = dd.col_nint[c];
    a.nint_tiles = (a.nint + CPB - 1) / CPB;
    const int grid = a.nint_tiles + (n - a.nint);
    cg_apply_kernel<T, D, N><<<grid, CPB * L, smem, st>>>(a, t);
    nlaunch++;
  }
  if ((err = cudaGetLastError()) != cudaSuccess) return err;
  if (prof && prof->on) return prof->end(st, nlaunch);
  return cudaSuccess;
}

template <typename T>
cudaError_t launch_cg_apply(const HostProblem& hp, const DeviceData& dd, const T* x, T* y,
                            cudaStream_t st, Profiler* prof) {
#define SBM_CASE(DD, NN) \
  if (hp.d == DD && hp.n == NN) return launch_t<T, DD, NN>(hp, dd, x, y, st, prof);
  SBM_CASE(2, 2) SBM_CASE(2, 3) SBM_CASE(2, 4) SBM_CASE(2, 5) SBM_CASE(2, 6) SBM_CASE(2, 7)
  SBM_CASE(3, 2) SBM_CASE(3, 3) SBM_CASE(3, 4) SBM_CASE(3, 5) SBM_CASE(3, 6) SBM_CASE(3, 7)
#undef SBM_CASE
  return cudaErrorInvalidValue;
}
template cudaError_t launch_cg_apply<double>(const HostProblem&, const DeviceData&,
                                             const double*, double*, cudaStream_t, Profiler*);
template cudaError_t launch_cg_apply<float>(const HostProblem&, const DeviceData&, const float*,
                                            float*, cudaStream_t, Profiler*);

}  // namespace sbm
