// Matrix-free apply (FP64 or FP32) of the SIPG discontinuous Galerkin SBM operator.
//
// Cell-centric: every block owns CPB cells and writes their DoFs once (a DG
// cell's DoFs belong to it alone), so there is a single launch, no colouring
// and no atomics.  Per cell: the cell term (Algorithm 1; 3D in the eigenbasis
// of the 1D pencil, 2D by sweeps, as in the CG kernel), then its 2d faces in
// the order (k, s):
//  * interior face (neighbour active), Algorithm 2 from this cell's side:
//      [u] = u_K1 - u_K2, {dn u} = (dn u_K1 + dn u_K2)/2 with n = +e_k, K1 the
//      lower cell; the value test gets +T_v (K1) or -T_v (K2),
//      T_v = sigma_F [u] - {dn u}, and the normal-derivative test -[u]/2;
//    the neighbour's trace comes straight from global memory (each face is
//    evaluated from both sides: twice the face arithmetic, no write conflict);
//  * surrogate face: Algorithm 3, computed for all faces beforehand by the
//    face kernel (face_kernel.cu) and folded in here from its scratch.
// Interior-face arithmetic in nodal form: the face integrands are linear in
// the nodal traces and the face quadrature is exact, so interpolation to the
// Gauss points, weights and transposed interpolation collapse into the 1D
// mass matrices: nodal traces -> pointwise combination -> (M x M) -> added to
// the cell result.
#include "sweeps.cuh"

namespace sbm {

template <int D, int N>
struct DgShape {
  static constexpr int L = (D == 3) ? N * N : N;
  static constexpr int ND = L * N;
  static constexpr int CPB = (128 / L) > 0 ? (128 / L) : 1;
};

// The result tile A (3D FP32: the padded layout of TilePad, node (j0, j1, j2)
// at j0 + PX j1 + PX n j2, cells NDP apart; FP64 (pipe-bound, registers
// first) and 2D unpadded; 2D: the pair tile's two halves).
template <typename T, int D, int N>
struct DgTile {
  static constexpr bool kPad = D == 3 && std::is_same<T, float>::value;
  static constexpr int PX = kPad ? TilePad<T, N>::PX : N;
  static constexpr int NDP = kPad ? TilePad<T, N>::NDP : (D == 3 ? 1 : 2) * DgShape<D, N>::ND;
  static constexpr int elems = DgShape<D, N>::CPB * NDP;   // A, before the input tiles
};

template <typename T>
struct DgArgs {
  const T* __restrict__ x;
  T* __restrict__ y;
  const int32_t* __restrict__ cell_rank;   // ordered cell -> active-cell rank
  const int32_t* __restrict__ nbr;         // [rank][2k+s] neighbour rank or -1
  const int32_t* __restrict__ face_start;  // ordered cell -> surrogate-face range
  const T* __restrict__ face_out;          // [F][2L] from the face kernel
  int ncell;
  T sigma_f;
};

template <typename T, int D, int N>
__global__ void __launch_bounds__(DgShape<D, N>::CPB * DgShape<D, N>::L)
dg_apply_kernel(const DgArgs<T> a, const __grid_constant__ KTab<T> t) {
  constexpr int L = DgShape<D, N>::L, ND = DgShape<D, N>::ND, CPB = DgShape<D, N>::CPB;
  using Pair2 = typename PairOf<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // 3D: a scalar sweep tile (the eigenbasis phases run in place and leave the
  // cell results there); 2D: a pair tile for the sweeps, then the results
  using DT = DgTile<T, D, N>;
  T* A = reinterpret_cast<T*>(smem_raw);       // sweep tile, then the result tile
  Pair2* AE = reinterpret_cast<Pair2*>(smem_raw);
  T* X = A + DT::elems;                        // CPB input tiles (unpadded)
  T* U1 = X + CPB * ND;        // face scratch, CPB * L each
  T* U2 = U1 + CPB * L;
  T* P1 = U2 + CPB * L;
  T* P2 = P1 + CPB * L;
  const int tid = threadIdx.x;
  const int first = blockIdx.x * CPB;
  const int ncells = min(CPB, a.ncell - first);
  for (int r = tid; r < ncells * ND; r += blockDim.x) {
    const int c = r / ND;
    X[r] = __ldg(a.x + (size_t)__ldg(a.cell_rank + first + c) * ND + (r - c * ND));
  }
  __syncthreads();
  const int c = tid / L, tl = tid - c * L;
  const bool act = c < ncells;
  const int pos = first + (act ? c : 0);
  const int rank = __ldg(a.cell_rank + pos);
  T* Xc = X + c * ND;
  T* R = A + c * (D == 3 ? DT::NDP : ND);
  {
    // cell term (Algorithm 1), then the line result into R (node (j0, j1, j2)
    // at j0 + n j1 + n^2 j2): 3D the z-line tl, back to the nodes its last
    // phase read; 2D the x-line tl, once every thread is past the sweeps
    T out[N];
    if constexpr (D == 3) {
      const XLineOp<T, N> xop(t, tl % N, tl / N);
      cell_fd_3d<T, N, DT::kPad>(t, X, c * ND + tl, N * N, A, c, tl, act, xop, out);
      if (act) {
#pragma unroll
        for (int m = 0; m < N; ++m)
          R[DT::PX == N ? tl + N * N * m : tl % N + DT::PX * (tl / N + N * m)] = out[m];
      }
    } else {
      cell_sweeps_2d<T, N>(t, X, c * ND + tl, N, AE, c, tl, act, out);
      __syncthreads();
      if (act) {
#pragma unroll
        for (int m = 0; m < N; ++m) R[N * tl + m] = out[m];
      }
    }
  }
  __syncthreads();

  int fptr = act ? __ldg(a.face_start + pos) : 0;   // next surrogate face of this cell
  T* u1 = U1 + c * L;
  T* u2 = U2 + c * L;
  T* p1 = P1 + c * L;
  T* p2 = P2 + c * L;
  for (int k = 0; k < D; ++k) {
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
    const int bt = (tl % N) * sa + (D == 3 ? (tl / N) * sb : 0);
    // the same strides in the result tile (3D FP32: padded)
    int rk = sk, rbt = bt;
    if constexpr (DT::PX != N) {
      rk = (k == 0) ? 1 : (k == 1 ? DT::PX : DT::PX * N);
      rbt = (tl % N) * ((k == 0) ? DT::PX : 1) + (tl / N) * ((k == 2) ? DT::PX : DT::PX * N);
    }
    for (int s = 0; s < 2; ++s) {
      const int nb = act ? __ldg(a.nbr + (size_t)rank * 2 * D + 2 * k + s) : -1;
      const bool interior = nb >= 0;
      const int kend = s ? N - 1 : 0;
      const T sg = s ? T(1) : T(-1);
      const T* fo = nullptr;
      if (act && !interior) fo = a.face_out + (size_t)(fptr++) * 2 * L;
      // A. nodal traces (own side and, for interior faces, the neighbour's),
      // and the two integrands in nodal form: with Gauss quadrature exact on
      // the face, interpolating to the Gauss points, weighting and
      // interpolating back is h^(d-1) (M x M) (the exact 1D mass matrices), so
      //   value test:  h^(d-1) (M x M) sg (sigma_F [u] - h^-1 {d_k u}),
      //   normal-derivative test:  h^(d-1) (M x M) (-[u] / (2 h))
      if (act) {
        T um = Xc[kend * sk + bt], dm = T(0);
#pragma unroll
        for (int j = 0; j < N; ++j) dm = fma(s ? t.D1[j] : t.D0[j], Xc[j * sk + bt], dm);
        T a1 = T(0), a2 = T(0);
        if (interior) {
          const T* xn = a.x + (size_t)nb * ND;
          const int nend = s ? 0 : N - 1;
          T un = __ldg(xn + nend * sk + bt), dnb = T(0);
#pragma unroll
          for (int j = 0; j < N; ++j)
            dnb = fma(s ? t.D0[j] : t.D1[j], __ldg(xn + j * sk + bt), dnb);
          const T jump = s ? (um - un) : (un - um);        // [u] = u_K1 - u_K2
          const T avg = T(0.5) * (dm + dnb);               // {d_k u} (reference)
          a1 = (sg * t.hface) * (a.sigma_f * jump - t.h_inv * avg);
          a2 = (T(-0.5) * t.hface * t.h_inv) * jump;
        }
        p1[tl] = a1;
        p2[tl] = a2;
      }
      __syncthreads();
      // B. (M x M) on both integrands, the first axis, then the second
      T rv = T(0), rg = T(0);
      if (D == 3) {
        if (act) {
          const int ia = tl % N, jb = tl / N;
          T v1 = T(0), v2 = T(0);
#pragma unroll
          for (int j = 0; j < N; ++j) {
            v1 = fma(t.M[ia][j], p1[j + N * jb], v1);
            v2 = fma(t.M[ia][j], p2[j + N * jb], v2);
          }
          u1[tl] = v1;
          u2[tl] = v2;
        }
        __syncthreads();
        if (act) {
          const int ia = tl % N, ib = tl / N;
#pragma unroll
          for (int j = 0; j < N; ++j) {
            rv = fma(t.M[ib][j], u1[ia + N * j], rv);
            rg = fma(t.M[ib][j], u2[ia + N * j], rg);
          }
        }
      } else {
        if (act) {
#pragma unroll
          for (int j = 0; j < N; ++j) {
            rv = fma(t.M[tl][j], p1[j], rv);
            rg = fma(t.M[tl][j], p2[j], rg);
          }
        }
      }
      if (act && !interior) {           // surrogate face: results of the face kernel
        rv = __ldg(fo + tl);
        rg = __ldg(fo + L + tl);
      }
      if (act) {
        R[kend * rk + rbt] += rv;
#pragma unroll
        for (int j = 0; j < N; ++j)
          R[j * rk + rbt] = fma(s ? t.D1[j] : t.D0[j], rg, R[j * rk + rbt]);
      }
      __syncthreads();
    }
  }
  for (int r = tid; r < ncells * ND; r += blockDim.x) {
    const int cc = r / ND, q = r - cc * ND;
    const int ar = DT::PX != N ? cc * DT::NDP + q % N + DT::PX * (q / N) : r;
    a.y[(size_t)__ldg(a.cell_rank + first + cc) * ND + q] = A[ar];
  }
}

template <typename T, int D, int N>
static cudaError_t dg_t(const HostProblem& hp, const DeviceData& dd, const T* x, T* y,
                        cudaStream_t st, Profiler* prof, int face_mode) {
  constexpr int L = DgShape<D, N>::L, ND = DgShape<D, N>::ND, CPB = DgShape<D, N>::CPB;
  const KTab<T> t = make_ktab<T>(hp);
  const size_t smem = (size_t)(DgTile<T, D, N>::elems + CPB * ND + 4 * CPB * L) * sizeof(T);
  cudaError_t err;
  if (smem > 48 * 1024) {
    err = cudaFuncSetAttribute(dg_apply_kernel<T, D, N>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
  }
  DgArgs<T> a;
  a.x = x;
  a.y = y;
  a.cell_rank = dd.cell_rank;
  a.nbr = dd.nbr;
  a.face_start = dd.face_start;
  a.face_out = face_out_of<T>(dd);
  a.ncell = dd.col_start[dd.ncolours];
  a.sigma_f = (T)hp.sigma_f;
  const bool pr = prof && prof->on;
  if (pr && (err = prof->mark(st)) != cudaSuccess) return err;
  int nlaunch = 1;
  if (dd.nface > 0) {
    if ((err = launch_faces<T>(hp, dd, x, face_out_of<T>(dd), face_mode, st)) != cudaSuccess)
      return err;
    nlaunch++;
  }
  if (pr && (err = prof->mark(st)) != cudaSuccess) return err;
  const int grid = (a.ncell + CPB - 1) / CPB;
  dg_apply_kernel<T, D, N><<<grid, CPB * L, smem, st>>>(a, t);
  if ((err = cudaGetLastError()) != cudaSuccess) return err;
  if (pr) {
    prof->count(nlaunch);
    if ((err = prof->mark(st)) != cudaSuccess) return err;   // cell phase ends
    return prof->mark(st);                                   // no assembly phase
  }
  return cudaSuccess;
}

template <typename T>
cudaError_t launch_dg_apply(const HostProblem& hp, const DeviceData& dd, const T* x, T* y,
                            cudaStream_t st, Profiler* prof, int face_mode) {
#define SBM_CASE(DD, NN) \
  if (hp.d == DD && hp.n == NN) return dg_t<T, DD, NN>(hp, dd, x, y, st, prof, face_mode);
  SBM_CASE(2, 2) SBM_CASE(2, 3) SBM_CASE(2, 4) SBM_CASE(2, 5) SBM_CASE(2, 6) SBM_CASE(2, 7)
  SBM_CASE(3, 2) SBM_CASE(3, 3) SBM_CASE(3, 4) SBM_CASE(3, 5) SBM_CASE(3, 6) SBM_CASE(3, 7)
#undef SBM_CASE
  return cudaErrorInvalidValue;
}
template cudaError_t launch_dg_apply<double>(const HostProblem&, const DeviceData&,
                                             const double*, double*, cudaStream_t, Profiler*,
                                             int);
template cudaError_t launch_dg_apply<float>(const HostProblem&, const DeviceData&, const float*,
                                            float*, cudaStream_t, Profiler*, int);

}  // namespace sbm
