// Matrix-free apply (FP64 or FP32) of the continuous Galerkin SBM operator.
//
// One apply = three launches:
//  1. the surrogate-face kernel (face_kernel.cu, or tc_face.cu on the tensor
//     cores): every face into per-face scratch;
//  2. the chunk kernel.  Active cells are cut into chunks: up to R
//     consecutive active cells of one x-row of the mesh.  In the compact DoF
//     numbering the x-lines of consecutive active cells continue each other,
//     so the chunk's line (j1, j2) is one contiguous run of p*nc + 1 values:
//     the block gathers those runs coalesced, runs the cell sweeps
//     (Algorithm 1) for each cell, folds in the cells' surrogate faces, sums
//     the values of the x-face nodes its consecutive cells share in shared
//     memory, and writes each run once, coalesced: a DoF that no other chunk
//     touches goes straight to y, any other into the accumulation buffer of
//     the chunk's colour.  A chunk's colour is (its parity within its row
//     run, cy mod 2[, cz mod 2]); chunks of one colour share no DoF, so every
//     element of y and of the buffers has a single writer;
//  3. the assembly kernel, over the DoFs that two colours or more touch:
//     y_i = sum over those colours (a per-DoF bit mask) of buffer_c[i], in
//     fixed colour order.
// No atomics, no read-modify-write, no y = 0 fill; repeated applies are
// bitwise equal.
#include <algorithm>
#include <type_traits>

#include "chunk_body.cuh"

namespace sbm {

template <int D, int N>
struct ChunkShape {
  static constexpr int L = Shape<D, N>::L;
  static constexpr int R = (256 / L) > 0 ? (256 / L) : 1;     // cells per chunk
};

int chunk_cells(int d, int n) {
  const int L = (d == 3) ? n * n : n;
  return (256 / L) > 0 ? (256 / L) : 1;
}

CellLaunch cell_launch_shape(int d, int n) {
  const int r = chunk_cells(d, n);
  return CellLaunch{d, n, r, r * ((d == 3) ? n * n : n)};
}


template <typename T, int D, int N, int R>
__global__ void __launch_bounds__(R * Shape<D, N>::L)
cg_chunk_kernel(const ChunkArgs<T> a, const __grid_constant__ KTab<T> t) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // FP32: launched as a programmatic dependent of the face kernel (coherent
  // face loads, a wait before the first fold); FP64 launches plainly
  constexpr bool kPdl = std::is_same<T, float>::value;
  if constexpr (kPdl) pdl_trigger();
  chunk_xline_build<T, D, N, R>(smem_raw, t, threadIdx.x);
  chunk_loop<T, D, N, R, kPdl, R * Shape<D, N>::L, kPdl>(a, t, smem_raw, blockIdx.y,
                                                         a.q0 + blockIdx.x, a.q1, gridDim.x);
}

// The same chunks with colour-ordered stores (chunk_loop, ORD): a
// persistent grid taking chunks from the ticket counter, no assembly pass.
template <typename T, int D, int N, int R>
__global__ void __launch_bounds__(R * Shape<D, N>::L)
cg_chunk_ord_kernel(const ChunkArgs<T> a, const __grid_constant__ KTab<T> t,
                    const __grid_constant__ OrdArgs o) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  chunk_xline_build<T, D, N, R>(smem_raw, t, threadIdx.x);
  chunk_loop_ord<T, D, N, R>(a, t, smem_raw, o);
}

// Tile shape 3 (3D): the chunks of shape 0 without staged runs.  Resident
// blocks asked of the compiler: FP32 6 (40 registers, no spills); FP64 5 up
// to p = 4 (48 registers), 4 above (64 registers; 5 would spill).
template <typename T, int N>
constexpr int direct_min_blocks() {
  return std::is_same<T, float>::value ? 6 : (N <= 5 ? 5 : 4);
}

template <typename T, int N, int R>
__global__ void __launch_bounds__(R * N * N, (direct_min_blocks<T, N>()))
cg_direct_kernel(const ChunkArgs<T> a, const __grid_constant__ KTab<T> t) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr bool kPdl = std::is_same<T, float>::value;     // as cg_chunk_kernel
  if constexpr (kPdl) pdl_trigger();
  chunk_loop_direct<T, N, R, kPdl, false, kPdl>(a, t, t, smem_raw, blockIdx.y,
                                                a.q0 + blockIdx.x, a.q1, gridDim.x);
}

template <typename T, int N, int R>
__global__ void __launch_bounds__(R * N * N, (direct_min_blocks<T, N>()))
cg_direct_ord_kernel(const ChunkArgs<T> a, const __grid_constant__ KTab<T> t,
                     const __grid_constant__ OrdArgs o) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  chunk_loop_direct<T, N, R, false, true>(a, t, t, smem_raw, 0, 0, 0, 0, &o);
}

// Resident blocks per SM x SMs of a kernel (the persistent grid of the
// colour-ordered launches), once per kernel.
template <typename K>
static cudaError_t resident_grid(K kernel, int threads, size_t smem, int* cache, int* grid) {
  if (*cache == 0) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess && smem > 48 * 1024)
      e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem);
    if (e != cudaSuccess) return e;
    *cache = std::max(1, per_sm) * sms;
  }
  *grid = *cache;
  return cudaSuccess;
}

template <typename T, int N, int R>
static cudaError_t direct_prepare(int* grid_cap) {
  static int per_sm = 0, sms = 0;
  static cudaError_t attr = cudaSuccess;
  constexpr size_t smem = DirectSmem<T, N, R>::bytes;
  if (per_sm == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (smem > 48 * 1024)
      attr = cudaFuncSetAttribute(cg_direct_kernel<T, N, R>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (attr != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cg_direct_kernel<T, N, R>,
                                                      R * N * N, smem) != cudaSuccess ||
        per_sm < 1)
      per_sm = 1;
  }
  *grid_cap = 4 * per_sm * sms;
  return attr;
}

// The DoFs that several colours touch (assemble_warp), one per thread;
// grid.y = right-hand side.
template <typename T>
__global__ void assemble_kernel(const T* __restrict__ ycol, const int32_t* __restrict__ multi,
                                const uint8_t* __restrict__ multi_mask, T* __restrict__ y,
                                int64_t n, int64_t nmulti, int ncol, int64_t ld_ycol = 0,
                                int64_t ldy = 0) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  assemble_warp<T, false>(ycol + blockIdx.y * ld_ycol, multi, multi_mask, y + blockIdx.y * ldy, n,
                          nmulti, ncol, t);
}

// Single right-hand side: two shared DoFs per thread (entries b + tid and
// b + 256 + tid of a 512-entry tile; assemble_pair).  FP32: Q4 sphere 41 ->
// 37.5 us, p = 3 20.6 -> 16.7 us against one per thread (four: 41 / 20.6).
// The tiles go in reverse list order (block 0 takes the last tile), so that
// the first blocks read the colour values the cell kernel stored last (the
// list ascends in DoF number, as its stores do).  Every DoF's sum is
// independent of the order.  Measured: Q4 sphere FP32 35.6 -> 33.1 us, FP64
// 50.0 -> 46.3 us in a loop of applies, and also faster with cold caches
// (ncu, FP64 39.0 -> 34.7 us), so L2 reuse is not the whole reason.
template <typename T>
__global__ void __launch_bounds__(256)
assemble_set_kernel(const T* __restrict__ ycol, const int32_t* __restrict__ multi,
                    const uint8_t* __restrict__ multi_mask, T* __restrict__ y, int64_t n,
                    int64_t nmulti, int ncol) {
  const int64_t tile = (int64_t)(gridDim.x - 1u - blockIdx.x);
  assemble_pair<T, false, std::is_same<T, float>::value>(ycol, multi, multi_mask, y, n, nmulti,
                                                         ncol, tile * 512 + threadIdx.x, 256);
}

// Blocks of the chunk kernel: 4 x (resident blocks per SM) x SMs at most
// (each block walks over several chunks), capped by the number of chunks.
template <typename T, int D, int N, int R>
static cudaError_t chunk_prepare(int* grid_cap) {
  static int per_sm = 0, sms = 0;
  static cudaError_t attr = cudaSuccess;
  constexpr size_t smem = ChunkSmem<T, D, N, R>::bytes;
  if (per_sm == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (smem > 48 * 1024)
      attr = cudaFuncSetAttribute(cg_chunk_kernel<T, D, N, R>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (attr != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cg_chunk_kernel<T, D, N, R>,
                                                      R * Shape<D, N>::L, smem) != cudaSuccess ||
        per_sm < 1)
      per_sm = 1;
  }
  *grid_cap = 4 * per_sm * sms;
  return attr;
}

// Which part of the operator one apply_r call runs: surrogate faces
// [f0, f1), chunks [q0, q1), shared DoFs [m0, m1) of the assembly list (all:
// f1 = q1 = m1 = -1).
struct Part {
  int f0 = 0, f1 = -1, q0 = 0, q1 = -1;
  int64_t m0 = 0, m1 = -1;
};

// face stage + chunk kernel + assembly, with explicit scratch and nrhs
// right-hand sides (x, y: nrhs vectors ld apart).
template <typename T, int D, int N, int R>
static cudaError_t apply_r(const HostProblem& hp, const DeviceData& dd, const ChunkTable& ct,
                           const T* x, T* y, int64_t ld, int nrhs, T* fo, T* ycol, int face_mode,
                           cudaStream_t st, Profiler* prof, Part part, bool reg,
                           bool direct, bool ord, bool allow_pdl) {
  constexpr int L = Shape<D, N>::L;
  const KTab<T> t = make_ktab<T>(hp);
  constexpr size_t smem = ChunkSmem<T, D, N, R>::bytes;
  if (part.f1 < 0) part.f1 = dd.nface;
  if (part.q1 < 0) part.q1 = ct.n;
  if (part.m1 < 0) part.m1 = ct.nmulti;
  cudaError_t err;
  const bool pr = prof && prof->on;
  int nlaunch = 0;
  if (pr && (err = prof->mark(st)) != cudaSuccess) return err;
  // programmatic dependent launches (FP32 whole applies, no profiling marks
  // between the kernels): the cell kernels (shapes 0, 2, 3) after the
  // CUDA-core face kernel (which x's producers precede in the stream), the
  // assembly after the cell kernel.  Measured (unprofiled applies, GB300):
  // FP32 p = 6 ellipsoid (shape 3) 62.7 -> 57.4 us, p = 3 / 4 spheres
  // (shapes 0, 3) 1-5 % faster, shape 2 1-8 % faster (cell_reg.cu); the
  // FP64 p = 4 sphere 2.3 % slower (1.026 ->
  // 1.049 ms), so FP64 launches without it.
  allow_pdl = allow_pdl && std::is_same<T, float>::value;
  bool pdl_cell = false;
  if (part.f1 > part.f0) {
    err = face_mode != 0 ? launch_faces<T>(hp, dd, x, fo, face_mode, st)
                         : launch_face_kernel<T>(hp, dd, x, fo, st, part.f0, part.f1);
    if (err != cudaSuccess) return err;
    nlaunch++;
    pdl_cell = allow_pdl && !pr && face_mode == 0;
  }
  if (pr && (err = prof->mark(st)) != cudaSuccess) return err;
  int cap = 0;
  if ((err = chunk_prepare<T, D, N, R>(&cap)) != cudaSuccess) return err;
  ChunkArgs<T> a;
  a.x = x;
  a.y = y;
  a.ycol = ycol;
  a.run_bits = ct.run_bits;
  a.bit_words = ct.bit_words;
  a.lines = dd.lines;
  a.face_start = dd.face_start;
  a.face_kind = dd.face_kind;
  a.face_out = fo;
  a.chunk_first = ct.first;
  a.chunk_col = ct.colour;
  a.n_dofs = hp.n_dofs;
  a.q0 = part.q0;
  a.q1 = part.q1;
  a.ldx = ld;
  a.ld_ycol = (int64_t)dd.ncolours * hp.n_dofs;
  a.ld_face = (int64_t)dd.nface * 2 * L;
  OrdArgs oa{ct.ord, ct.add_bits, ct.deps, ct.ndeps, ct.done, ct.tickets, dd.err_flag, ct.n,
             ct.dep_cap};
  const int nl0 = nlaunch;
  if (reg) {                 // tile shape 2: one thread per cell (cell_reg.cu)
    if ((err = launch_cell_reg<T>(hp, dd, x, y, fo, ycol, st, pdl_cell)) != cudaSuccess)
      return err;
    nlaunch++;
  } else if (ord && part.q1 > part.q0) {      // colour-ordered stores, no assembly
    if constexpr (R == ChunkShape<D, N>::R) {
      static int cache = 0;
      int grid = 0;
      if (direct) {
        if constexpr (D == 3) {
          if ((err = resident_grid(cg_direct_ord_kernel<T, N, R>, R * L,
                                   DirectSmem<T, N, R>::bytes, &cache, &grid)) != cudaSuccess)
            return err;
          if ((err = launch_maybe_pdl(cg_direct_ord_kernel<T, N, R>, dim3(std::min(grid, ct.n)),
                                      dim3(R * L), DirectSmem<T, N, R>::bytes, st, pdl_cell, a,
                                      t, oa)) != cudaSuccess)
            return err;
        }
      } else {
        static int cache0 = 0;
        if ((err = resident_grid(cg_chunk_ord_kernel<T, D, N, R>, R * L, smem, &cache0, &grid)) !=
            cudaSuccess)
          return err;
        if ((err = launch_maybe_pdl(cg_chunk_ord_kernel<T, D, N, R>, dim3(std::min(grid, ct.n)),
                                    dim3(R * L), smem, st, pdl_cell, a, t, oa)) != cudaSuccess)
          return err;
      }
      nlaunch++;
    }
  } else if (direct && part.q1 > part.q0) {   // tile shape 3: no staged runs (3D)
    if constexpr (D == 3 && R == ChunkShape<D, N>::R) {
      int dcap = 0;
      if ((err = direct_prepare<T, N, R>(&dcap)) != cudaSuccess) return err;
      const int grid = std::min(part.q1 - part.q0, dcap);
      if ((err = launch_maybe_pdl(cg_direct_kernel<T, N, R>, dim3(grid, nrhs), dim3(R * L),
                                  DirectSmem<T, N, R>::bytes, st, pdl_cell, a, t)) !=
          cudaSuccess)
        return err;
      nlaunch++;
    }
  } else if (part.q1 > part.q0) {
    const int grid = std::min(part.q1 - part.q0, cap);
    if ((err = launch_maybe_pdl(cg_chunk_kernel<T, D, N, R>, dim3(grid, nrhs), dim3(R * L), smem,
                                st, pdl_cell, a, t)) != cudaSuccess)
      return err;
    nlaunch++;
  }
  const bool pdl_asm = allow_pdl && !pr && nlaunch > nl0;
  if (pr && (err = prof->mark(st)) != cudaSuccess) return err;
  const int64_t n = hp.n_dofs, nm = ord ? 0 : part.m1 - part.m0;
  if (nm > 0 && nrhs == 1) {
    if ((err = launch_maybe_pdl(assemble_set_kernel<T>, dim3((unsigned)((nm + 511) / 512)),
                                dim3(256), 0, st, pdl_asm, (const T*)ycol,
                                (const int32_t*)(ct.multi + part.m0),
                                (const uint8_t*)(ct.multi_mask + part.m0), y, n, nm,
                                dd.ncolours)) != cudaSuccess)
      return err;
    nlaunch++;
  } else if (nm > 0) {
    assemble_kernel<T><<<dim3((unsigned)((nm + 255) / 256), nrhs), 256, 0, st>>>(
        ycol, ct.multi + part.m0, ct.multi_mask + part.m0, y, n, nm, dd.ncolours,
        (int64_t)dd.ncolours * n, ld);
    nlaunch++;
  }
  if ((err = cudaGetLastError()) != cudaSuccess) return err;
  if (pr) {
    prof->count(nlaunch);
    return prof->mark(st);
  }
  return cudaSuccess;
}

// variant 0: R cells per chunk; variant 1: R/2 (a second tile shape for the
// autotuner); variant 2: the cells of variant 0's chunks one thread each
// (cell_reg.cu; whole applies only -- a slab of the host pipeline runs
// variant 0, which gives the same bits); variant 3 (3D): variant 0's chunks
// without staged runs (chunk_loop_direct; slabs too).  Both chunkings are built at set-up
// with the same colouring rule, so the variants give bitwise-equal results.
template <typename T, int D, int N>
static cudaError_t apply_t(const HostProblem& hp, const DeviceData& dd, const T* x, T* y,
                           int64_t ld, int nrhs, T* fo, T* ycol, int face_mode, int variant,
                           bool ordered, cudaStream_t st, Profiler* prof, int slab, int stages) {
  constexpr int R = ChunkShape<D, N>::R;
  constexpr int RH = (R / 2) > 0 ? R / 2 : 1;
  const int v = (variant == 1 && RH < R) ? 1 : 0;
  const bool reg = variant == 2 && slab < 0 && nrhs == 1 &&
                   cell_reg_available(hp, std::is_same<T, float>::value);
  const bool direct = variant == 3 && D == 3;
  const ChunkTable& ct = dd.chunks[v];
  // colour-ordered stores: whole single applies of chunking 0 by the chunk
  // kernels (shapes 0 and 3; shape 2 keeps the colour buffers)
  const bool ord = ordered && v == 0 && !reg && slab < 0 && nrhs == 1 && ct.ordered;
  Part part;
  if (slab >= 0) {
    const bool faces = stages & 1, cells = stages & 2;
    part.f0 = dd.slab_face[slab];
    part.f1 = faces ? dd.slab_face[slab + 1] : part.f0;
    part.q0 = ct.slab_chunk[slab];
    part.q1 = cells ? ct.slab_chunk[slab + 1] : part.q0;
    part.m0 = ct.slab_multi[slab];
    part.m1 = cells ? ct.slab_multi[slab + 1] : part.m0;
  }
  if (v == 1)
    return apply_r<T, D, N, RH>(hp, dd, ct, x, y, ld, nrhs, fo, ycol, face_mode, st, prof, part,
                                false, false, false, slab < 0);
  return apply_r<T, D, N, R>(hp, dd, ct, x, y, ld, nrhs, fo, ycol, face_mode, st, prof, part,
                             reg, direct, ord, slab < 0);
}

template <typename T>
static cudaError_t dispatch(const HostProblem& hp, const DeviceData& dd, const T* x, T* y,
                            int64_t ld, int nrhs, T* fo, T* ycol, int face_mode, int variant,
                            bool ordered, cudaStream_t st, Profiler* prof, int slab = -1,
                            int stages = 3) {
#define SBM_CASE(DD, NN)                                                                   \
  if (hp.d == DD && hp.n == NN)                                                            \
    return apply_t<T, DD, NN>(hp, dd, x, y, ld, nrhs, fo, ycol, face_mode, variant, ordered, \
                              st, prof, slab, stages);
  SBM_CASE(2, 2) SBM_CASE(2, 3) SBM_CASE(2, 4) SBM_CASE(2, 5) SBM_CASE(2, 6) SBM_CASE(2, 7)
  SBM_CASE(3, 2) SBM_CASE(3, 3) SBM_CASE(3, 4) SBM_CASE(3, 5) SBM_CASE(3, 6) SBM_CASE(3, 7)
#undef SBM_CASE
  return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t launch_cg_apply(const HostProblem& hp, const DeviceData& dd, const T* x, T* y,
                            cudaStream_t st, Profiler* prof, int face_mode) {
  const int pi = std::is_same<T, float>::value ? 1 : 0;
  return dispatch<T>(hp, dd, x, y, 0, 1, face_out_of<T>(dd), ycol_of<T>(dd), face_mode,
                     dd.variant[pi], dd.ordered[pi], st, prof);
}
template cudaError_t launch_cg_apply<double>(const HostProblem&, const DeviceData&,
                                             const double*, double*, cudaStream_t, Profiler*,
                                             int);
template cudaError_t launch_cg_apply<float>(const HostProblem&, const DeviceData&, const float*,
                                            float*, cudaStream_t, Profiler*, int);

// Slab s of the FP64 apply (the pipelined host-buffer apply): stages 1 =
// the surrogate faces of the cells of slab s, 2 = their chunks and the shared
// DoFs the slab completes; after both, y is final on the DoFs [slab_y[s],
// slab_y[s+1]) given x on [0, slab_x[s]).
cudaError_t launch_cg_apply_slab(const HostProblem& hp, const DeviceData& dd, const double* x,
                                 double* y, int slab, int stages, cudaStream_t st) {
  return dispatch<double>(hp, dd, x, y, 0, 1, dd.face_out, dd.ycol, 0, dd.variant[0], false, st,
                          nullptr, slab, stages);
}

// The same launches with caller-provided scratch: per-face results
// ([F][2L]) and colour buffers ([ncolours][n_dofs]).
template <typename T>
cudaError_t launch_cg_apply_scratch(const HostProblem& hp, const DeviceData& dd, const T* x, T* y,
                                    T* face_scratch, T* colour_scratch, int variant,
                                    cudaStream_t st) {
  return dispatch<T>(hp, dd, x, y, 0, 1, face_scratch, colour_scratch, 0, variant, false, st,
                     nullptr);
}
template cudaError_t launch_cg_apply_scratch<double>(const HostProblem&, const DeviceData&,
                                                     const double*, double*, double*, double*,
                                                     int, cudaStream_t);

}  // namespace sbm
