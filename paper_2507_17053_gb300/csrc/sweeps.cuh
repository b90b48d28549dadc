// Device building blocks shared by the apply kernels: tile shapes and the
// sum-factorised cell sweeps (Algorithm 1).
//
// Cell term.  With Gauss quadrature of n = p+1 points per axis the cell
// integral of grad u . grad v is exact, so on a Cartesian cell
//   A_K = h^(d-2) sum_k (M x ... x K_k x ... x M)
// with the exact 1D mass M and stiffness K on [0,1], instead of the 4d
// sweeps of interpolate / differentiate / integrate.  2D: 4 one-dimensional
// sweeps, a = M_y u, e = K_y u;  y = K_x a + M_x e.  3D: the eigenbasis form
// below (5 phases, 5 even/odd products per line).  Each thread owns one line of the
// (p+1)^d tile per phase (registers); the tile is staged in shared memory
// between phases.
#pragma once

#include "internal.hpp"

namespace sbm {

// Programmatic dependent launch (the single applies: face kernel -> cell
// kernel -> assembly).  A kernel lets the next one in the stream start once
// all of its blocks run (pdl_trigger); the next one does its independent work
// (the gather, the cell term) and waits for the previous grid's completion
// and memory (pdl_wait) only before it reads that grid's results (it reads
// them with coherent loads, not the read-only path).  Both are no-ops for a
// kernel launched without the attribute.
__device__ __forceinline__ void pdl_trigger() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }


template <int D, int N>
struct Shape {
  static constexpr int L = (D == 3) ? N * N : N;   // lines per cell, points per face
  static constexpr int ND = L * N;                  // DoFs per cell
  static constexpr int CPB = (128 / L) > 0 ? (128 / L) : 1;
};

// ---- 1D line operations ------------------------------------------------------
//
// For n >= 5 the 1D matrices are applied in even/odd form (see Folded): an
// n x n product costs (n/2)^2 + ((n+1)/2)^2 multiply-adds plus 2n additions
// instead of n^2, and the folding of an input line is shared by every matrix
// applied to it.  For n <= 4 the plain product is as cheap and is used.

template <typename T, int N>
struct LineFold {
  static constexpr int H = N / 2, HE = (N + 1) / 2;
  T e[HE];
  T o[H > 0 ? H : 1];
  __device__ __forceinline__ LineFold() {}
  __device__ __forceinline__ explicit LineFold(const T (&v)[N]) {
#pragma unroll
    for (int j = 0; j < H; ++j) {
      e[j] = v[j] + v[N - 1 - j];
      o[j] = v[j] - v[N - 1 - j];
    }
    if (N & 1) e[H] = v[H];
  }
  // modal coefficients (even modes first) are already split: no additions
  __device__ __forceinline__ static LineFold of_modes(const T (&w)[N]) {
    LineFold f;
#pragma unroll
    for (int i = 0; i < HE; ++i) f.e[i] = w[i];
#pragma unroll
    for (int i = 0; i < H; ++i) f.o[i] = w[HE + i];
    return f;
  }
};

template <typename T, int N>
struct LineAcc {
  static constexpr int H = N / 2, HE = (N + 1) / 2;
  T s[HE];
  T d[H > 0 ? H : 1];
  __device__ __forceinline__ LineAcc() {
#pragma unroll
    for (int i = 0; i < HE; ++i) s[i] = T(0);
#pragma unroll
    for (int i = 0; i < H; ++i) d[i] = T(0);
  }
  __device__ __forceinline__ void mac(const Folded<T>& A, const LineFold<T, N>& f) {
#pragma unroll
    for (int i = 0; i < HE; ++i)
#pragma unroll
      for (int j = 0; j < HE; ++j) s[i] = fma(A.E[i][j], f.e[j], s[i]);
#pragma unroll
    for (int i = 0; i < H; ++i)
#pragma unroll
      for (int j = 0; j < H; ++j) d[i] = fma(A.O[i][j], f.o[j], d[i]);
  }
  __device__ __forceinline__ void unfold(T (&y)[N]) const {
#pragma unroll
    for (int i = 0; i < H; ++i) {
      y[i] = s[i] + d[i];
      y[N - 1 - i] = s[i] - d[i];
    }
    if (N & 1) y[H] = s[H];
  }
};

template <int N>
struct UseFold {
  static constexpr bool value = N >= 5;
};

// y = A v
template <typename T, int N>
__device__ __forceinline__ void line_apply(const T (&A)[kMaxN][kMaxN], const Folded<T>& F,
                                           const T (&v)[N], T (&y)[N]) {
  if constexpr (UseFold<N>::value) {
    LineFold<T, N> f(v);
    LineAcc<T, N> acc;
    acc.mac(F, f);
    acc.unfold(y);
  } else {
#pragma unroll
    for (int m = 0; m < N; ++m) {
      T a = T(0);
#pragma unroll
      for (int j = 0; j < N; ++j) a = fma(A[m][j], v[j], a);
      y[m] = a;
    }
  }
}

// y1 = A1 v, y2 = A2 v
template <typename T, int N>
__device__ __forceinline__ void line_apply2(const T (&A1)[kMaxN][kMaxN], const Folded<T>& F1,
                                            const T (&A2)[kMaxN][kMaxN], const Folded<T>& F2,
                                            const T (&v)[N], T (&y1)[N], T (&y2)[N]) {
  if constexpr (UseFold<N>::value) {
    LineFold<T, N> f(v);
    LineAcc<T, N> a1, a2;
    a1.mac(F1, f);
    a2.mac(F2, f);
    a1.unfold(y1);
    a2.unfold(y2);
  } else {
#pragma unroll
    for (int m = 0; m < N; ++m) {
      T a = T(0), b = T(0);
#pragma unroll
      for (int j = 0; j < N; ++j) {
        a = fma(A1[m][j], v[j], a);
        b = fma(A2[m][j], v[j], b);
      }
      y1[m] = a;
      y2[m] = b;
    }
  }
}

// y = A1 v1 + A2 v2
template <typename T, int N>
__device__ __forceinline__ void line_apply_sum(const T (&A1)[kMaxN][kMaxN], const Folded<T>& F1,
                                               const T (&v1)[N], const T (&A2)[kMaxN][kMaxN],
                                               const Folded<T>& F2, const T (&v2)[N],
                                               T (&y)[N]) {
  if constexpr (UseFold<N>::value) {
    LineFold<T, N> f1(v1), f2(v2);
    LineAcc<T, N> acc;
    acc.mac(F1, f1);
    acc.mac(F2, f2);
    acc.unfold(y);
  } else {
#pragma unroll
    for (int m = 0; m < N; ++m) {
      T a = T(0);
#pragma unroll
      for (int j = 0; j < N; ++j) {
        a = fma(A1[m][j], v1[j], a);
        a = fma(A2[m][j], v2[j], a);
      }
      y[m] = a;
    }
  }
}

// w = V^T v: the modes of a nodal line (even modes first); the folded input
// feeds the even and the odd modes, and the output needs no unfolding.
template <typename T, int N>
__device__ __forceinline__ void line_to_modes(const Folded<T>& Vt, const T (&v)[N], T (&w)[N]) {
  LineFold<T, N> f(v);
  LineAcc<T, N> acc;
  acc.mac(Vt, f);
#pragma unroll
  for (int i = 0; i < LineAcc<T, N>::HE; ++i) w[i] = acc.s[i];
#pragma unroll
  for (int i = 0; i < LineAcc<T, N>::H; ++i) w[LineAcc<T, N>::HE + i] = acc.d[i];
}

// y = V w: a nodal line from its modes (no folding of the input).
template <typename T, int N>
__device__ __forceinline__ void modes_to_line(const Folded<T>& V, const T (&w)[N], T (&y)[N]) {
  const LineFold<T, N> f = LineFold<T, N>::of_modes(w);
  LineAcc<T, N> acc;
  acc.mac(V, f);
  acc.unfold(y);
}

// ---- 3D cell term in the eigenbasis of the 1D pencil ---------------------------
//
// With M = V V^T and K = V diag(lam) V^T (the generalised eigenvectors of
// (K, M), scaled), the exact cell operator factors as
//   A_K = h (V x V x V) diag(lam_i + lam_j + lam_k) (V x V x V)^T.
// After the z- and y-transforms, the x-line of y-mode a and z-mode b needs
//   V diag(h lam_i + h lam_a + h lam_b) V^T = h K + mu_ab M,  mu_ab = h (lam_a + lam_b),
// a symmetric matrix of the 1D pencil that is applied directly (XLineOp)
// instead of a transform, a scaling and a transform back.  Five line phases
// over one scalar tile per cell, in place (a thread reads its line, then
// writes the same nodes): z-lines to z-modes, y-lines to y-modes, x-lines
// through h K + mu_ab M, y-modes back, z-modes back.  Every 1D product is an
// even/odd split product (V's columns are even or odd, K and M are
// centrosymmetric), so a line costs 5 (ceil(n/2)^2 + floor(n/2)^2) FMAs and
// 6 folds or unfolds of 2 floor(n/2) additions each -- 89 operations per
// line at p = 4, against 131 for the 7-sweep form.  Tile layout: node (j0, j1, j2) at
// j0 + n j1 + n^2 j2.  The z-line (j0, j1) = line tl of cell c is read from
// X[xb + xs * j2]; xop is h K + mu_ab M for the thread's x-line of modes
// (a, b) = (tl % n, tl / n).  The z-line result of line tl is returned in
// out[] (nodal, j2 = 0..n-1); the tile then holds nothing useful.

// h K + mu M in even/odd form (both blocks symmetric), built once per thread.
template <typename T, int N>
struct XLineOp {
  static constexpr int H = N / 2, HE = (N + 1) / 2;
  T E[HE][HE];
  T O[H > 0 ? H : 1][H > 0 ? H : 1];
  __device__ __forceinline__ XLineOp(const KTab<T>& t, int a, int b) {
    const T mu = t.hlam[a] + t.hlam[b];
#pragma unroll
    for (int i = 0; i < HE; ++i)
#pragma unroll
      for (int j = i; j < HE; ++j) E[i][j] = E[j][i] = fma(mu, t.fM.E[i][j], t.fKh.E[i][j]);
#pragma unroll
    for (int i = 0; i < H; ++i)
#pragma unroll
      for (int j = i; j < H; ++j) O[i][j] = O[j][i] = fma(mu, t.fM.O[i][j], t.fKh.O[i][j]);
  }
  __device__ __forceinline__ void apply(const T (&v)[N], T (&y)[N]) const {
    const LineFold<T, N> f(v);
    LineAcc<T, N> acc;
#pragma unroll
    for (int i = 0; i < HE; ++i)
#pragma unroll
      for (int j = 0; j < HE; ++j) acc.s[i] = fma(E[i][j], f.e[j], acc.s[i]);
#pragma unroll
    for (int i = 0; i < H; ++i)
#pragma unroll
      for (int j = 0; j < H; ++j) acc.d[i] = fma(O[i][j], f.o[j], acc.d[i]);
    acc.unfold(y);
  }
  static constexpr int kSize = HE * HE + H * H;   // scalars of one line's operator
  // Shared-memory form: both blocks are symmetric, so only their upper
  // triangles are kept (row-major, E then O), and the operator of modes
  // (a, b) equals that of (b, a) (mu_ab = mu_ba), so one slot serves both:
  // n(n+1)/2 slots of kPacked scalars (an odd count: the threads of a warp
  // read different slots without bank conflicts).
  static constexpr int kPacked = (HE * (HE + 1) / 2 + H * (H + 1) / 2) | 1;
  static constexpr int kSlots = N * (N + 1) / 2;
  __host__ __device__ static constexpr int tri(int i, int j, int n) {   // i <= j < n
    return i * n - i * (i - 1) / 2 + (j - i);
  }
  __host__ __device__ static constexpr int sym(int i, int j, int n) {
    return i <= j ? tri(i, j, n) : tri(j, i, n);
  }
  __device__ static int slot(int a, int b) { return sym(a, b, N); }
  __device__ __forceinline__ void store(T* m) const {
#pragma unroll
    for (int i = 0; i < HE; ++i)
#pragma unroll
      for (int j = i; j < HE; ++j) m[tri(i, j, HE)] = E[i][j];
#pragma unroll
    for (int i = 0; i < H; ++i)
#pragma unroll
      for (int j = i; j < H; ++j) m[HE * (HE + 1) / 2 + tri(i, j, H)] = O[i][j];
  }
};

// The same operator read from shared memory at each use (no registers held
// across the kernel).
template <typename T, int N>
struct XLineShared {
  static constexpr int H = N / 2, HE = (N + 1) / 2;
  using Op = XLineOp<T, N>;
  const T* m;                       // the slot of the thread's modes (a, b)
  __device__ __forceinline__ void apply(const T (&v)[N], T (&y)[N]) const {
    const LineFold<T, N> f(v);
    LineAcc<T, N> acc;
#pragma unroll
    for (int i = 0; i < HE; ++i)
#pragma unroll
      for (int j = 0; j < HE; ++j) acc.s[i] = fma(m[Op::sym(i, j, HE)], f.e[j], acc.s[i]);
#pragma unroll
    for (int i = 0; i < H; ++i)
#pragma unroll
      for (int j = 0; j < H; ++j)
        acc.d[i] = fma(m[HE * (HE + 1) / 2 + Op::sym(i, j, H)], f.o[j], acc.d[i]);
    acc.unfold(y);
  }
};

// The 3D cell tile in shared memory: node (j0, j1, j2) of a cell at
// j0 + PX j1 + PX n j2, cells NDP apart.  For even n the x-stride is padded
// to PX = n + 1 (FP32, and FP64 at n = 4) so that the x-line phase (stride PX
// between threads) and the y-line phase (stride PX n) spread over the
// shared-memory banks; odd n are conflict-free unpadded.
template <typename T, int N>
struct TilePad {
  static constexpr int PX =
      (N % 2 == 0 && (std::is_same<T, float>::value || N == 4)) ? N + 1 : N;
  static constexpr int NDP = PX * N * N;
};

// The thread's z-line of x comes from load(j), j = 0..n-1 (staged runs in
// shared memory, or global memory directly).
// PAD = false: the unpadded layout (PX = n), for callers that address the
// tile themselves (the DG kernel).
template <typename T, int N, bool PAD = true, typename XOp, typename Load>
__device__ __forceinline__ void cell_fd_3d_l(const KTab<T>& t, const Load& load, T* tile, int c,
                                             int tl, bool act, const XOp& xop, T (&out)[N]) {
  constexpr int PX = PAD ? TilePad<T, N>::PX : N, NDP = PX * N * N, PL = PX * N;
  const int a = tl % N, b = tl / N;
  const int zl = (PX == N) ? tl : a + PX * b;     // the z-line's first node
  T* cell = tile + c * NDP;
  if (act) {                       // z-lines (j0, j1) = (a, b) -> z-modes
    T v[N], w[N];
#pragma unroll
    for (int j = 0; j < N; ++j) v[j] = load(j);
    line_to_modes<T, N>(t.fVt, v, w);
#pragma unroll
    for (int k = 0; k < N; ++k) cell[zl + PL * k] = w[k];
  }
  __syncthreads();
  if (act) {                       // y-lines (j0 = a, z-mode b) -> y-modes
    T v[N], w[N];
#pragma unroll
    for (int j = 0; j < N; ++j) v[j] = cell[a + PX * j + PL * b];
    line_to_modes<T, N>(t.fVt, v, w);
#pragma unroll
    for (int k = 0; k < N; ++k) cell[a + PX * k + PL * b] = w[k];
  }
  __syncthreads();
  if (act) {                       // x-lines (y-mode a, z-mode b): h K + mu_ab M
    T v[N], y[N];
#pragma unroll
    for (int j = 0; j < N; ++j) v[j] = cell[PX * tl + j];
    xop.apply(v, y);
#pragma unroll
    for (int j = 0; j < N; ++j) cell[PX * tl + j] = y[j];
  }
  __syncthreads();
  if (act) {                       // y-modes back (j0 = a, z-mode b)
    T w[N], y[N];
#pragma unroll
    for (int k = 0; k < N; ++k) w[k] = cell[a + PX * k + PL * b];
    modes_to_line<T, N>(t.fV, w, y);
#pragma unroll
    for (int j = 0; j < N; ++j) cell[a + PX * j + PL * b] = y[j];
  }
  __syncthreads();
  if (act) {                       // z-modes back (j0, j1) = (a, b)
    T w[N];
#pragma unroll
    for (int k = 0; k < N; ++k) w[k] = cell[zl + PL * k];
    modes_to_line<T, N>(t.fV, w, out);
  }
}

template <typename T, int N, bool PAD = true, typename XOp>
__device__ __forceinline__ void cell_fd_3d(const KTab<T>& t, const T* X, int xb, int xs, T* tile,
                                           int c, int tl, bool act, const XOp& xop,
                                           T (&out)[N]) {
  cell_fd_3d_l<T, N, PAD>(t, [&](int j) { return X[xb + xs * j]; }, tile, c, tl, act, xop, out);
}

// ---- cell term -------------------------------------------------------------
//
// Each phase produces two arrays for the next one ((a, e), then (b, g)); they
// are stored interleaved as pairs, so one 8-byte (FP32) or 16-byte (FP64)
// shared-memory access moves both values of a node.

template <typename T>
struct PairOf;
template <>
struct PairOf<float> {
  using type = float2;
};
template <>
struct PairOf<double> {
  using type = double2;
};

// 2D: y-lines then x-lines; the y-line j0 = tl of cell c is read from
// X[xb + xs * j1].
template <typename T, int N>
__device__ __forceinline__ void cell_sweeps_2d(const KTab<T>& t, const T* X, int xb, int xs,
                                               typename PairOf<T>::type* AE, int c, int tl,
                                               bool act, T (&out)[N]) {
  using P2 = typename PairOf<T>::type;
  constexpr int ND = N * N;
  if (act) {
    const int base = c * ND + tl;                           // y-line j0 = tl
    T v[N], a[N], e[N];
#pragma unroll
    for (int j = 0; j < N; ++j) v[j] = X[xb + xs * j];
    line_apply2<T, N>(t.M, t.fM, t.K, t.fK, v, a, e);
#pragma unroll
    for (int m = 0; m < N; ++m) AE[base + N * m] = P2{a[m], e[m]};
  }
  __syncthreads();
  if (act) {
    const int base = c * ND + N * tl;                       // x-line j1 = tl
    T va[N], ve[N];
#pragma unroll
    for (int j = 0; j < N; ++j) {
      const P2 p = AE[base + j];
      va[j] = p.x;
      ve[j] = p.y;
    }
    line_apply_sum<T, N>(t.Kh, t.fKh, va, t.Mh, t.fMh, ve, out);
  }
}

}  // namespace sbm
