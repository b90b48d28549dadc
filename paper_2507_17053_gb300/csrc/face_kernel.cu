// Surrogate-boundary faces (Algorithm 3), all faces of a problem in one launch.
//
// For the face (k, s) of cell K (outward normal (2s-1) e_k):
//  1. traces of u and of the reference normal derivative at the face's
//     tangential nodes (GLL nodes contain the end points, so the value trace
//     is the face slice of the tile);
//  2. interpolation to the tangential Gauss points x~_q (sum factorisation);
//  3. E u(x~_q) = u_K(x_q): point evaluation of the cell polynomial at the
//     shifted point from the stored 1D values phi_j(xi_{q,l}) -- the
//     O((p+1)^(2d-1)) step -- or, for the first-order Taylor extension,
//     E u = u(x~_q) + d_q . grad u(x~_q) from the value and gradient traces
//     (interpolated to x~_q like the normal derivative) and the stored shift
//     d_q; then the pointwise integrands
//       val_q = W_q (sigma E_q - dn u(x~_q)),  grd_q = -W_q E_q dn-scale;
//  4. transposed interpolation back to the tangential nodes.
// The face's contribution to its cell is then fully described by two
// n^(d-1) vectors per face (value test rv, normal-derivative test rg); the
// cell kernels fold them into the cell result:
//   R[node (kend, jt)] += rv[jt],  R[node (j, jt)] += phi_j'(s) rg[jt].
// Output: out[f * 2L + jt] = rv[jt], out[f * 2L + L + jt] = rg[jt].  Faces
// write disjoint slots, so there is no ordering hazard and no atomics.
#include "face_body.cuh"

namespace sbm {

template <typename T, int D, int N, int EXT>
__global__ void __launch_bounds__(Shape<D, N>::CPB * Shape<D, N>::L)
sface_kernel(const FaceArgs<T> a, const __grid_constant__ KTab<T> t) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // FP32: the cell kernel may start (it waits before its folds)
  if constexpr (std::is_same<T, float>::value) pdl_trigger();
  face_group<T, D, N, EXT, Shape<D, N>::CPB>(a, t, t, smem_raw,
                                              a.face0 + blockIdx.x * Shape<D, N>::CPB, a.nface,
                                              blockIdx.y);
}

template <typename T, int D, int N, int EXT>
static cudaError_t face_t(const HostProblem& hp, const DeviceData& dd, const T* x, T* out,
                          cudaStream_t st, int64_t ldx, int nrhs, int fb, int fe) {
  constexpr int L = Shape<D, N>::L, FPB = Shape<D, N>::CPB;
  if (fe <= fb) return cudaSuccess;
  const KTab<T> t = make_ktab<T>(hp);
  FaceArgs<T> a;
  a.x = x;
  a.lines = dd.lines;
  a.cell_rank = dd.cell_rank;
  a.face_cell = dd.face_cell;
  a.face_kind = dd.face_kind;
  a.face_phi = face_phi_of<T>(dd);
  a.face_pp = face_pp_of<T>(dd);
  a.out = out;
  a.face0 = fb;
  a.nface = fe;
  a.dg = hp.desc.dg;
  a.ldx = ldx;
  a.ld_out = (int64_t)dd.nface * 2 * L;
  const size_t smem = face_group_smem<T, D, N, EXT, FPB>();
  sface_kernel<T, D, N, EXT><<<dim3((fe - fb + FPB - 1) / FPB, nrhs), FPB * L, smem, st>>>(a, t);
  return cudaGetLastError();
}

template <typename T, int D, int N>
static cudaError_t face_x(const HostProblem& hp, const DeviceData& dd, const T* x, T* out,
                          cudaStream_t st, int64_t ldx = 0, int nrhs = 1, int fb = 0,
                          int fe = -1) {
  if (fe < 0) fe = dd.nface;
  return hp.desc.extension == SBM_EXT_TAYLOR1
             ? face_t<T, D, N, 1>(hp, dd, x, out, st, ldx, nrhs, fb, fe)
             : face_t<T, D, N, 0>(hp, dd, x, out, st, ldx, nrhs, fb, fe);
}

template <typename T>
cudaError_t launch_face_kernel(const HostProblem& hp, const DeviceData& dd, const T* x, T* out,
                               cudaStream_t st, int fb, int fe) {
#define SBM_CASE(DD, NN) \
  if (hp.d == DD && hp.n == NN) return face_x<T, DD, NN>(hp, dd, x, out, st, 0, 1, fb, fe);
  SBM_CASE(2, 2) SBM_CASE(2, 3) SBM_CASE(2, 4) SBM_CASE(2, 5) SBM_CASE(2, 6) SBM_CASE(2, 7)
  SBM_CASE(3, 2) SBM_CASE(3, 3) SBM_CASE(3, 4) SBM_CASE(3, 5) SBM_CASE(3, 6) SBM_CASE(3, 7)
#undef SBM_CASE
  return cudaErrorInvalidValue;
}
template cudaError_t launch_face_kernel<double>(const HostProblem&, const DeviceData&,
                                                const double*, double*, cudaStream_t, int, int);

template cudaError_t launch_face_kernel<float>(const HostProblem&, const DeviceData&,
                                               const float*, float*, cudaStream_t, int, int);

}  // namespace sbm
