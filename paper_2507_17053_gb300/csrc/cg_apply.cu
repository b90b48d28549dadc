// Matrix-free apply (FP64 or FP32) of the continuous Galerkin SBM operator.
//
// One apply = three launches:
//  1. the surrogate-face kernel (face_kernel.cu): every face into per-face
//     scratch;
//  2. the cell kernel over ALL active cells: gather, cell sweeps
//     (Algorithm 1), fold in the cell's surrogate faces, and a plain store of
//     the local result into the accumulation buffer of the cell's colour.
//     Colours are the 2^d parity patterns of the cell indices; two cells of
//     one colour share no DoF, so every store has a single writer;
//  3. the assembly kernel: y_i = sum over the colours that touch DoF i (a
//     per-DoF bit mask) of buffer_c[i], in fixed colour order.
// No atomics, no read-modify-write, no y = 0 fill; repeated applies are
// bitwise equal.  One launch over all cells keeps many independent blocks in
// flight, so the gather latency of some overlaps the arithmetic of others.
#include <algorithm>

#include "sweeps.cuh"

namespace sbm {

CellLaunch cell_launch_shape(int d, int n) {
  int L = (d == 3) ? n * n : n;
  int cpb = 128 / L;
  if (cpb < 1) cpb = 1;
  return CellLaunch{d, n, cpb, cpb * L};
}

template <typename T>
struct CgArgs {
  const T* __restrict__ x;
  T* __restrict__ ycol;                    // [ncolours][n_dofs] accumulation buffers
  const int32_t* __restrict__ lines;       // ordered cells x L
  const int32_t* __restrict__ face_start;  // ordered cells + 1
  const int32_t* __restrict__ face_kind;
  const T* __restrict__ face_out;          // [F][2L] from the face kernel
  int64_t n_dofs;
  int ncell;                               // all active cells
  int col_start[9];                        // ordered cells are grouped by colour
  // right-hand side blockIdx.y of a multi-RHS launch: offsets of its x, its
  // colour buffers and its face results (0 for a single right-hand side)
  int64_t ldx, ld_ycol, ld_face;
};

// Add the contributions of surrogate face (k, s) to the x-line result out[]
// of line tl: R[node (kend, jt)] += rv[jt], R[node (j, jt)] += phi_j'(s) rg[jt].
template <typename T, int D, int N>
__device__ __forceinline__ void fold_face(const KTab<T>& t, const T* __restrict__ fo, int k, int s,
                                          int tl, T (&out)[N]) {
  constexpr int L = Shape<D, N>::L;
  const T* rv = fo;
  const T* rg = fo + L;
  const int kend = s ? N - 1 : 0;
  if (k == 0) {                       // tangential index = the line itself
    const T v = __ldg(rv + tl), g = __ldg(rg + tl);
#pragma unroll
    for (int m = 0; m < N; ++m) {
      out[m] = fma(s ? t.D1[m] : t.D0[m], g, out[m]);
      if (m == kend) out[m] += v;       // compile-time index: out stays in registers
    }
  } else {
    // k == 1: line tl = (j1, j2), tangential (m, j2);  k == 2: tangential (m, j1)
    const int jk = (D == 2 || k == 1) ? tl % N : tl / N;
    const int jo = (D == 2) ? 0 : (k == 1 ? tl / N : tl % N);
    const T dk = s ? t.D1[jk] : t.D0[jk];
#pragma unroll
    for (int m = 0; m < N; ++m) {
      const int jt = m + N * jo;
      T add = dk * __ldg(rg + jt);
      if (jk == kend) add += __ldg(rv + jt);
      out[m] += add;
    }
  }
}

// Every block walks over tiles of CPB cells (tile = blockIdx.x, then +
// gridDim.x, ...).  While a tile is in the sweeps, the x-lines of the block's
// next tile are already being loaded into registers, so the gather latency
// of one tile hides behind the arithmetic of the previous one.
template <typename T, int D, int N, int CPB = Shape<D, N>::CPB>
__global__ void __launch_bounds__(CPB * Shape<D, N>::L)
cg_apply_kernel(const CgArgs<T> a, const __grid_constant__ KTab<T> t) {
  constexpr int L = Shape<D, N>::L, ND = Shape<D, N>::ND;
  using P2 = typename PairOf<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  P2* AE = reinterpret_cast<P2*>(smem_raw);     // pair arrays first: 8/16-byte aligned
  P2* BG = AE + CPB * ND;
  T* X = reinterpret_cast<T*>(BG + CPB * ND);
  const int tid = threadIdx.x;
  const int c = tid / L, tl = tid - c * L;
  const int ntiles = (a.ncell + CPB - 1) / CPB;
  const T* __restrict__ xr = a.x + blockIdx.y * a.ldx;
  const T* fo = a.face_out + blockIdx.y * a.ld_face;
  T* ycb = a.ycol + blockIdx.y * a.ld_ycol;

  // registers of the tile in flight: its x-line, its index, its face range
  int tile = blockIdx.x;
  int cell = tile * CPB + c;
  bool act = tile < ntiles && cell < a.ncell;
  int g0 = 0, fs = 0, fe = 0;
  T v[N];
  if (act) {
    g0 = __ldg(a.lines + (size_t)cell * L + tl);
#pragma unroll
    for (int m = 0; m < N; ++m) v[m] = __ldg(xr + g0 + m);
    fs = __ldg(a.face_start + cell);
    fe = __ldg(a.face_start + cell + 1);
  }
  while (tile < ntiles) {
    if (act) {
#pragma unroll
      for (int m = 0; m < N; ++m) X[c * ND + N * tl + m] = v[m];
    }
    __syncthreads();
    // prefetch the next tile
    const int ntile = tile + gridDim.x;
    const int ncell_ = ntile * CPB + c;
    const bool nact = ntile < ntiles && ncell_ < a.ncell;
    int ng0 = 0, nfs = 0, nfe = 0;
    if (nact) {
      ng0 = __ldg(a.lines + (size_t)ncell_ * L + tl);
#pragma unroll
      for (int m = 0; m < N; ++m) v[m] = __ldg(xr + ng0 + m);
      nfs = __ldg(a.face_start + ncell_);
      nfe = __ldg(a.face_start + ncell_ + 1);
    }
    T out[N];
    if (D == 3) cell_sweeps_3d<T, N>(t, X, AE, BG, c, tl, act, out);
    else cell_sweeps_2d<T, N>(t, X, AE, c, tl, act, out);
    if (act) {
      for (int f = fs; f < fe; ++f) {
        const int kind = __ldg(a.face_kind + f);
        fold_face<T, D, N>(t, fo + (size_t)f * 2 * L, kind & 3, kind >> 2, tl, out);
      }
      int col = 0;             // cells are ordered by colour; unrolled: no local copy
#pragma unroll
      for (int k = 1; k < 8; ++k) col += (cell >= a.col_start[k]) ? 1 : 0;
      T* yc = ycb + (size_t)col * a.n_dofs + g0;
#pragma unroll
      for (int m = 0; m < N; ++m) yc[m] = out[m];
    }
    tile = ntile;
    cell = ncell_;
    act = nact;
    g0 = ng0;
    fs = nfs;
    fe = nfe;
  }
}

// Blocks of the cell kernel: enough to fill every SM at the kernel's
// occupancy (so each block walks over several tiles), capped by the tiles.
template <typename T, int D, int N, int CPB>
static int cell_grid(int ntiles, size_t smem) {
  static int per_sm = 0, sms = 0;
  if (per_sm == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cg_apply_kernel<T, D, N, CPB>,
                                                      CPB * Shape<D, N>::L, smem) != cudaSuccess ||
        per_sm < 1)
      per_sm = 1;
  }
  const int g = per_sm * sms;
  return ntiles < g ? ntiles : g;
}

// y_i = sum_{c in mask_i} ycol[c][i], colours in increasing order.  One DoF
// per thread (all of its loads in flight at once); the buffers are read once.
// Adding 0.0 is exact, so y_i equals the plain sum over the set colours; the
// additions of a colour that no lane of the warp has are skipped (on GB300
// every double addition costs an FP64-pipe slot).
template <typename T>
__global__ void assemble_kernel(const T* __restrict__ ycol, const uint8_t* __restrict__ mask,
                                T* __restrict__ y, int64_t n, int ncol, int64_t ld_ycol = 0,
                                int64_t ldy = 0) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  ycol += blockIdx.y * ld_ycol;
  y += blockIdx.y * ldy;
  const unsigned m = (i < n) ? (unsigned)__ldg(mask + i) : 0u;
  T v[8];
#pragma unroll
  for (int c = 0; c < 8; ++c)
    v[c] = (c < ncol && (m & (1u << c))) ? __ldcs(ycol + (size_t)c * n + i) : T(0);
  T acc = T(0);
#pragma unroll
  for (int c = 0; c < 8; ++c)
    if (__any_sync(0xffffffffu, (m >> c) & 1u)) acc += v[c];
  if (i < n) __stcs(y + i, acc);
}

template <typename T, int D, int N>
static cudaError_t launch_t(const HostProblem& hp, const DeviceData& dd, const T* x, T* y,
                            cudaStream_t st, Profiler* prof, int face_mode) {
  constexpr int L = Shape<D, N>::L, ND = Shape<D, N>::ND, CPB = Shape<D, N>::CPB;
  const KTab<T> t = make_ktab<T>(hp);
  const size_t smem = (size_t)(5 * CPB * ND) * sizeof(T);
  T* fo = face_out_of<T>(dd);
  T* ycol = ycol_of<T>(dd);
  cudaError_t err;
  const bool pr = prof && prof->on;
  if (pr && (err = prof->mark(st)) != cudaSuccess) return err;
  int nlaunch = 0;
  if (dd.nface > 0) {
    if ((err = launch_faces<T>(hp, dd, x, fo, face_mode, st)) != cudaSuccess) return err;
    nlaunch++;
  }
  if (pr && (err = prof->mark(st)) != cudaSuccess) return err;
  CgArgs<T> a;
  a.x = x;
  a.ycol = ycol;
  a.lines = dd.lines;
  a.face_start = dd.face_start;
  a.face_kind = dd.face_kind;
  a.face_out = fo;
  a.n_dofs = hp.n_dofs;
  a.ncell = dd.col_start[dd.ncolours];
  for (int c = 0; c < 9; ++c) a.col_start[c] = dd.col_start[c < dd.ncolours ? c : dd.ncolours];
  a.ldx = a.ld_ycol = a.ld_face = 0;
  cg_apply_kernel<T, D, N><<<cell_grid<T, D, N, CPB>((a.ncell + CPB - 1) / CPB, smem), CPB * L, smem,
                             st>>>(a, t);
  nlaunch++;
  if (pr && (err = prof->mark(st)) != cudaSuccess) return err;
  const int64_t n = hp.n_dofs;
  assemble_kernel<T><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(ycol, dd.dof_colours, y, n,
                                                                   dd.ncolours);
  nlaunch++;
  if ((err = cudaGetLastError()) != cudaSuccess) return err;
  if (pr) {
    prof->count(nlaunch);
    return prof->mark(st);
  }
  return cudaSuccess;
}

// The same three launches with caller-provided scratch: per-face results `fo`
// ([F][2L]) and colour buffers `ycol` ([ncolours][n_dofs]).
template <typename T, int D, int N>
static cudaError_t launch_scratch_t(const HostProblem& hp, const DeviceData& dd, const T* x, T* y,
                                    T* fo, T* ycol, cudaStream_t st) {
  constexpr int L = Shape<D, N>::L, ND = Shape<D, N>::ND, CPB = Shape<D, N>::CPB;
  const KTab<T> t = make_ktab<T>(hp);
  const size_t smem = (size_t)(5 * CPB * ND) * sizeof(T);
  cudaError_t err;
  if (dd.nface > 0 && (err = launch_face_kernel<T>(hp, dd, x, fo, st)) != cudaSuccess) return err;
  CgArgs<T> a;
  a.x = x;
  a.ycol = ycol;
  a.lines = dd.lines;
  a.face_start = dd.face_start;
  a.face_kind = dd.face_kind;
  a.face_out = fo;
  a.n_dofs = hp.n_dofs;
  a.ncell = dd.col_start[dd.ncolours];
  for (int c = 0; c < 9; ++c) a.col_start[c] = dd.col_start[c < dd.ncolours ? c : dd.ncolours];
  a.ldx = a.ld_ycol = a.ld_face = 0;
  cg_apply_kernel<T, D, N><<<cell_grid<T, D, N, CPB>((a.ncell + CPB - 1) / CPB, smem), CPB * L, smem,
                             st>>>(a, t);
  const int64_t n = hp.n_dofs;
  assemble_kernel<T><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(ycol, dd.dof_colours, y, n,
                                                                   dd.ncolours);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_cg_apply_scratch(const HostProblem& hp, const DeviceData& dd, const T* x, T* y,
                                    T* face_scratch, T* colour_scratch, cudaStream_t st) {
#define SBM_CASE(DD, NN)                                                                    \
  if (hp.d == DD && hp.n == NN)                                                             \
    return launch_scratch_t<T, DD, NN>(hp, dd, x, y, face_scratch, colour_scratch, st);
  SBM_CASE(2, 2) SBM_CASE(2, 3) SBM_CASE(2, 4) SBM_CASE(2, 5) SBM_CASE(2, 6) SBM_CASE(2, 7)
  SBM_CASE(3, 2) SBM_CASE(3, 3) SBM_CASE(3, 4) SBM_CASE(3, 5) SBM_CASE(3, 6) SBM_CASE(3, 7)
#undef SBM_CASE
  return cudaErrorInvalidValue;
}
template cudaError_t launch_cg_apply_scratch<double>(const HostProblem&, const DeviceData&,
                                                     const double*, double*, double*, double*,
                                                     cudaStream_t);

// nrhs right-hand sides in one set of launches (grid.y = right-hand side):
// x and y hold nrhs vectors of n_dofs each, ld apart; the scratch holds nrhs
// copies.  variant 0/1 picks the cells-per-block of the cell kernel (128 or
// 256 threads' worth of lines), chosen by the autotuner.
template <typename T, int D, int N, int CPB>
static cudaError_t multi_cell_t(const HostProblem& hp, const DeviceData& dd, const T* x, int64_t ld,
                                int nrhs, T* fo, T* ycol, cudaStream_t st) {
  constexpr int L = Shape<D, N>::L, ND = Shape<D, N>::ND;
  const KTab<T> t = make_ktab<T>(hp);
  const size_t smem = (size_t)(5 * CPB * ND) * sizeof(T);
  cudaError_t err;
  if (smem > 48 * 1024 &&
      (err = cudaFuncSetAttribute(cg_apply_kernel<T, D, N, CPB>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
          cudaSuccess)
    return err;
  CgArgs<T> a;
  a.x = x;
  a.ycol = ycol;
  a.lines = dd.lines;
  a.face_start = dd.face_start;
  a.face_kind = dd.face_kind;
  a.face_out = fo;
  a.n_dofs = hp.n_dofs;
  a.ncell = dd.col_start[dd.ncolours];
  for (int c = 0; c < 9; ++c) a.col_start[c] = dd.col_start[c < dd.ncolours ? c : dd.ncolours];
  a.ldx = ld;
  a.ld_ycol = (int64_t)dd.ncolours * hp.n_dofs;
  a.ld_face = (int64_t)dd.nface * 2 * L;
  cg_apply_kernel<T, D, N, CPB>
      <<<dim3(cell_grid<T, D, N, CPB>((a.ncell + CPB - 1) / CPB, smem), nrhs), CPB * L, smem, st>>>(
          a, t);
  return cudaGetLastError();
}

template <typename T, int D, int N>
static cudaError_t multi_t(const HostProblem& hp, const DeviceData& dd, const T* x, T* y,
                           int64_t ld, int nrhs, T* fo, T* ycol, int variant, cudaStream_t st) {
  constexpr int L = Shape<D, N>::L;
  cudaError_t err;
  if (dd.nface > 0 &&
      (err = launch_face_kernel_multi<T>(hp, dd, x, ld, nrhs, fo, st)) != cudaSuccess)
    return err;
  if (variant == 1 && 256 / L > Shape<D, N>::CPB)
    err = multi_cell_t<T, D, N, (256 / L > 0 ? 256 / L : 1)>(hp, dd, x, ld, nrhs, fo, ycol, st);
  else
    err = multi_cell_t<T, D, N, Shape<D, N>::CPB>(hp, dd, x, ld, nrhs, fo, ycol, st);
  if (err != cudaSuccess) return err;
  const int64_t n = hp.n_dofs;
  assemble_kernel<T><<<dim3((unsigned)((n + 255) / 256), nrhs), 256, 0, st>>>(
      ycol, dd.dof_colours, y, n, dd.ncolours, (int64_t)dd.ncolours * n, ld);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_cg_apply_multi(const HostProblem& hp, const DeviceData& dd, const T* x, T* y,
                                  int64_t ld, int nrhs, T* face_scratch, T* colour_scratch,
                                  int variant, cudaStream_t st) {
#define SBM_CASE(DD, NN)                                                                   \
  if (hp.d == DD && hp.n == NN)                                                            \
    return multi_t<T, DD, NN>(hp, dd, x, y, ld, nrhs, face_scratch, colour_scratch, variant, st);
  SBM_CASE(2, 2) SBM_CASE(2, 3) SBM_CASE(2, 4) SBM_CASE(2, 5) SBM_CASE(2, 6) SBM_CASE(2, 7)
  SBM_CASE(3, 2) SBM_CASE(3, 3) SBM_CASE(3, 4) SBM_CASE(3, 5) SBM_CASE(3, 6) SBM_CASE(3, 7)
#undef SBM_CASE
  return cudaErrorInvalidValue;
}
template cudaError_t launch_cg_apply_multi<double>(const HostProblem&, const DeviceData&,
                                                   const double*, double*, int64_t, int, double*,
                                                   double*, int, cudaStream_t);
template cudaError_t launch_cg_apply_multi<float>(const HostProblem&, const DeviceData&,
                                                  const float*, float*, int64_t, int, float*,
                                                  float*, int, cudaStream_t);

template <typename T>
cudaError_t launch_cg_apply(const HostProblem& hp, const DeviceData& dd, const T* x, T* y,
                            cudaStream_t st, Profiler* prof, int face_mode) {
#define SBM_CASE(DD, NN) \
  if (hp.d == DD && hp.n == NN) return launch_t<T, DD, NN>(hp, dd, x, y, st, prof, face_mode);
  SBM_CASE(2, 2) SBM_CASE(2, 3) SBM_CASE(2, 4) SBM_CASE(2, 5) SBM_CASE(2, 6) SBM_CASE(2, 7)
  SBM_CASE(3, 2) SBM_CASE(3, 3) SBM_CASE(3, 4) SBM_CASE(3, 5) SBM_CASE(3, 6) SBM_CASE(3, 7)
#undef SBM_CASE
  return cudaErrorInvalidValue;
}
template cudaError_t launch_cg_apply<double>(const HostProblem&, const DeviceData&,
                                             const double*, double*, cudaStream_t, Profiler*,
                                             int);
template cudaError_t launch_cg_apply<float>(const HostProblem&, const DeviceData&, const float*,
                                            float*, cudaStream_t, Profiler*, int);

}  // namespace sbm
