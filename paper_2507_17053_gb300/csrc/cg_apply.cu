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

#include "sweeps.cuh"

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

template <typename T>
struct ChunkArgs {
  const T* __restrict__ x;
  T* __restrict__ y;                       // result (DoFs of a single colour)
  T* __restrict__ ycol;                    // [ncolours][n_dofs] accumulation buffers
  const uint32_t* __restrict__ run_bits;   // per chunk: bit l*S + kk set if that run
  int bit_words;                           //   element is a DoF of several colours
  const int32_t* __restrict__ lines;       // ordered cells x L
  const int32_t* __restrict__ face_start;  // ordered cells + 1
  const int32_t* __restrict__ face_kind;
  const T* __restrict__ face_out;          // [F][2L] from the face kernel
  const int32_t* __restrict__ chunk_first; // [nchunk + 1] first ordered cell of each chunk
  const uint8_t* __restrict__ chunk_col;   // [nchunk] colour of each chunk
  int64_t n_dofs;
  int q0, q1;                              // this launch: chunks [q0, q1)
  // right-hand side blockIdx.y of a multi-RHS launch: offsets of its x and y,
  // its colour buffers and its face results (0 for a single right-hand side)
  int64_t ldx, ld_ycol, ld_face;
};

// Add the contributions of surrogate face (k, s) to the z-line result out[]
// (nodes (a, b, m), m = 0..n-1) of a 3D cell: R[node with j_k = kend] +=
// rv[jt], R[node] += phi_{j_k}'(s) rg[jt], jt = the node's tangential index
// (the two other axes in increasing order, the first fastest).
template <typename T, int N>
__device__ __forceinline__ void fold_face_z(const KTab<T>& t, const T* __restrict__ fo, int k,
                                            int s, int a, int b, T (&out)[N]) {
  constexpr int L = N * N;
  const T* rv = fo;
  const T* rg = fo + L;
  const int kend = s ? N - 1 : 0;
  if (k == 2) {                       // normal along the line, tangential (a, b)
    const int jt = a + N * b;
    const T v = __ldg(rv + jt), g = __ldg(rg + jt);
#pragma unroll
    for (int m = 0; m < N; ++m) {
      out[m] = fma(s ? t.D1[m] : t.D0[m], g, out[m]);
      if (m == kend) out[m] += v;       // compile-time index: out stays in registers
    }
  } else {
    // k == 0: j_k = a, tangential (j1, j2) = (b, m);  k == 1: j_k = b, (j0, j2) = (a, m)
    const int jk = (k == 0) ? a : b;
    const int jo = (k == 0) ? b : a;
    const T dk = s ? t.D1[jk] : t.D0[jk];
#pragma unroll
    for (int m = 0; m < N; ++m) {
      const int jt = jo + N * m;
      T add = dk * __ldg(rg + jt);
      if (jk == kend) add += __ldg(rv + jt);
      out[m] += add;
    }
  }
}

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

// Shared memory of a chunk: one pair tile (R cells; the second sweep phase
// overwrites its own y-lines in place) and one scalar area that holds the
// gathered x-line runs until the first phase has read them and the per-cell
// x-line results after the last one.
// 3D: one scalar tile of R cells (the eigenbasis sweeps run in place and
// leave the cells' results there) and the gathered runs.  2D: one pair tile
// (the second sweep phase overwrites its own lines in place) and one area
// that holds the gathered runs until the first phase has read them and the
// per-cell x-line results after the last one.  Both: + the L run starts and
// the chunk's run-element bits (several colours or not).
template <typename T, int D, int N, int R>
struct ChunkSmem {
  static constexpr int L = Shape<D, N>::L, ND = Shape<D, N>::ND;
  static constexpr int SM0 = (N - 1) * R + 1;
  static constexpr int SM = (SM0 % 2) ? SM0 : SM0 + 1;        // odd row stride of the runs
  static constexpr int XZ = (L * SM > R * L * N) ? L * SM : R * L * N;
  static constexpr int TILE = (D == 3) ? R * ND : 2 * R * ND;  // scalars before the runs
  static constexpr int XS = (D == 3) ? L * SM : XZ;
  static constexpr int WORDS = (L * SM + 31) / 32;              // run-element bits
  static constexpr int XL = (D == 3) ? L * XLineOp<T, N>::kSize : 0;  // x-line operators
  // two run areas and two run-start tables: the next chunk's runs are copied
  // in (cp.async) while the current chunk is computed
  static constexpr size_t bytes =
      (size_t)(TILE + 2 * XS + XL) * sizeof(T) + (size_t)(2 * L + WORDS) * 4;
};

// Asynchronous global -> shared copy of one element (cp.async, no register
// round trip); the copies of a thread are grouped by commit and waited for
// by group.
template <typename T>
__device__ __forceinline__ void cp_async_elem(T* smem, const T* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  if constexpr (sizeof(T) == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int Pending>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(Pending) : "memory");
}

// Issue the copies of a chunk's L x-line runs (S values each, run l from
// Ls[l]) into Xs (row stride SM).  idx -> (run l, position kk) without an
// integer division: idx < L*S <= 1600, so (idx + 1/2)/S in FP32 is within
// 1e-5 of the exact quotient, far inside its distance 1/(2S) >= 0.0038 from
// an integer.
template <typename T, int L, int SM>
__device__ __forceinline__ void gather_runs_async(const T* __restrict__ xr, const int* Ls, T* Xs,
                                                  int S, int tid, int nthr) {
  const float invS = 1.0f / (float)S;
  for (int idx = tid; idx < L * S; idx += nthr) {
    const int l = __float2int_rz(((float)idx + 0.5f) * invS), kk = idx - l * S;
    cp_async_elem(Xs + l * SM + kk, xr + (int64_t)Ls[l] + kk);
  }
}

template <typename T, int D, int N, int R>
__global__ void __launch_bounds__(R * Shape<D, N>::L)
cg_chunk_kernel(const ChunkArgs<T> a, const __grid_constant__ KTab<T> t) {
  constexpr int L = Shape<D, N>::L, ND = Shape<D, N>::ND, P = N - 1;
  constexpr int SM = ChunkSmem<T, D, N, R>::SM;
  using P2 = typename PairOf<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  using CS = ChunkSmem<T, D, N, R>;
  T* tile = reinterpret_cast<T*>(smem_raw);   // 3D: [R][ND] scalar tile
  P2* AE = reinterpret_cast<P2*>(smem_raw);   // 2D: pair tile (8/16-byte aligned); phase 2
  P2* BG = AE;                                //     runs in place
  T* Xbuf = tile + CS::TILE;                  // [2][L][SM] x-line runs (current, next)
  T* XLs = Xbuf + 2 * CS::XS;                                // 3D: [L] x-line operators
  int* Lbuf = reinterpret_cast<int*>(XLs + CS::XL);          // [2][L] run starts
  uint32_t* Bs = reinterpret_cast<uint32_t*>(Lbuf + 2 * L);  // run-element bits
  const int tid = threadIdx.x;
  const int c = tid / L, tl = tid - c * L;
  // 3D: h K + mu M for the x-line of modes (a, b) = (tl % n, tl / n), in
  // shared memory (visible after the first chunk's first barrier)
  if (D == 3 && c == 0) XLineOp<T, N>(t, tl % N, tl / N).store(XLs + tl * XLineOp<T, N>::kSize);
  const XLineShared<T, N> xop{XLs + tl * XLineOp<T, N>::kSize};
  const T* __restrict__ xr = a.x + blockIdx.y * a.ldx;
  const T* fo = a.face_out + blockIdx.y * a.ld_face;
  T* ycb = a.ycol + blockIdx.y * a.ld_ycol;
  T* yb = a.y + blockIdx.y * a.ldx;

  // prologue: the first chunk's run starts, then its runs in flight
  int ch = a.q0 + blockIdx.x, buf = 0;
  if (ch < a.q1) {
    const int first = __ldg(a.chunk_first + ch);
    const int S = P * (__ldg(a.chunk_first + ch + 1) - first) + 1;
    for (int i = tid; i < L; i += blockDim.x) Lbuf[i] = __ldg(a.lines + (size_t)first * L + i);
    __syncthreads();
    gather_runs_async<T, L, SM>(xr, Lbuf, Xbuf, S, tid, R * L);
  }
  cp_async_commit();
  for (; ch < a.q1; ch += gridDim.x, buf ^= 1) {
    T* Xs = Xbuf + buf * CS::XS;              // this chunk's runs
    const int* Ls = Lbuf + buf * L;
    // per-cell results, node (j0, j1, j2) of cell c at c ND + j0 + n j1 +
    // n^2 j2 (3D: the tile; 2D: the run area, free after the first phase)
    T* Z = (D == 3) ? tile : Xs;
    const int first = __ldg(a.chunk_first + ch);
    const int nc = __ldg(a.chunk_first + ch + 1) - first;
    const int S = P * nc + 1;                 // values per x-line run
    const float invS = 1.0f / (float)S;
    // the next chunk's run starts, then its runs into the other buffer (the
    // previous iteration's last barrier freed it); they land while this
    // chunk is computed
    const int nx = ch + gridDim.x;
    if (nx < a.q1) {
      const int f2 = __ldg(a.chunk_first + nx);
      const int S2 = P * (__ldg(a.chunk_first + nx + 1) - f2) + 1;
      int* Ln = Lbuf + (buf ^ 1) * L;
      for (int i = tid; i < L; i += blockDim.x) Ln[i] = __ldg(a.lines + (size_t)f2 * L + i);
      __syncthreads();
      gather_runs_async<T, L, SM>(xr, Ln, Xbuf + (buf ^ 1) * CS::XS, S2, tid, R * L);
    }
    cp_async_commit();
    {
      const uint32_t* bits = a.run_bits + (size_t)ch * a.bit_words;
      for (int i = tid; i < (L * S + 31) / 32; i += blockDim.x) Bs[i] = __ldg(bits + i);
    }
    cp_async_wait<1>();                       // this chunk's runs (this thread's copies) ...
    __syncthreads();                          // ... and everyone's
    const bool act = c < nc;
    T out[N];
    if constexpr (D == 3)
      cell_fd_3d<T, N>(t, Xs, (tl / N) * SM + P * c + (tl % N), N * SM, tile, c, tl, act, xop,
                       out);
    else
      cell_sweeps_2d<T, N>(t, Xs, P * c + tl, SM, AE, c, tl, act, out);
    if (act) {
      const int pos = first + c;
      const int fs = __ldg(a.face_start + pos), fe = __ldg(a.face_start + pos + 1);
      for (int f = fs; f < fe; ++f) {
        const int kind = __ldg(a.face_kind + f);
        if constexpr (D == 3)
          fold_face_z<T, N>(t, fo + (size_t)f * 2 * L, kind & 3, kind >> 2, tl % N, tl / N, out);
        else
          fold_face<T, D, N>(t, fo + (size_t)f * 2 * L, kind & 3, kind >> 2, tl, out);
      }
      // 3D: z-line (j0, j1) = tl, back to the nodes it was read from
#pragma unroll
      for (int m = 0; m < N; ++m) {
        if constexpr (D == 3) Z[c * ND + tl + L * m] = out[m];
        else Z[(c * L + tl) * N + m] = out[m];
      }
    }
    __syncthreads();
    // runs of the result: the node shared by cells c-1 and c is the sum of
    // their two values (fixed order), then one coalesced store per run, into
    // y where this chunk is the DoF's only writer
    T* yc = ycb + (size_t)__ldg(a.chunk_col + ch) * a.n_dofs;
    for (int idx = tid; idx < L * S; idx += blockDim.x) {
      const int l = __float2int_rz(((float)idx + 0.5f) * invS), kk = idx - l * S;
      const int cc = kk / P, m = kk - cc * P;
      T v;
      if (cc == nc) v = Z[((nc - 1) * L + l) * N + P];
      else if (m == 0 && cc > 0) v = Z[((cc - 1) * L + l) * N + P] + Z[(cc * L + l) * N];
      else v = Z[(cc * L + l) * N + m];
      const int64_t g = (int64_t)Ls[l] + kk;
      if ((Bs[idx >> 5] >> (idx & 31)) & 1u) yc[g] = v;
      else yb[g] = v;
    }
    __syncthreads();                          // Xs / Z / Ls / Bs are reused
  }
  cp_async_wait<0>();
}

// For the DoFs i = multi[t] that several colours touch:
// y_i = sum_{c in mask_i} ycol[c][i], colours in increasing order.  Lane by
// lane the j-th step adds the value of the lane's j-th colour (0 past its
// count), for j up to the warp's largest colour count.  FP64: a loop with a
// warp-uniform, run-time trip count, so the additions a warp issues are its
// own count minus one (on GB300 a double addition costs an FP64-pipe slot
// per warp instruction, whatever its active lanes; the list is grouped by
// colour count, so most warps need one).  FP32: all loads first, then the
// unrolled sum (the additions are cheap, the load latency is not).  Adding
// a 0 leaves a sum unchanged.
template <typename T>
__global__ void assemble_kernel(const T* __restrict__ ycol, const int32_t* __restrict__ multi,
                                const uint8_t* __restrict__ multi_mask, T* __restrict__ y,
                                int64_t n, int64_t nmulti, int ncol, int64_t ld_ycol = 0,
                                int64_t ldy = 0) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  ycol += blockIdx.y * ld_ycol;
  y += blockIdx.y * ldy;
  int64_t i = 0;
  unsigned m = 0u;
  if (t < nmulti) {
    i = __ldg(multi + t);
    m = (unsigned)__ldg(multi_mask + t);
  }
  if (ncol < 8) m &= (1u << ncol) - 1u;
  const unsigned kmax = __reduce_max_sync(0xffffffffu, (unsigned)__popc(m));
  T acc = T(0);
  if constexpr (std::is_same<T, double>::value) {
    if (m) {
      acc = __ldcs(ycol + (size_t)(__ffs(m) - 1) * n + i);
      m &= m - 1u;
    }
    for (unsigned j = 1; j < kmax; ++j) {
      T v = T(0);
      if (m) {
        v = __ldcs(ycol + (size_t)(__ffs(m) - 1) * n + i);
        m &= m - 1u;
      }
      acc += v;
    }
  } else {
    T v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      v[j] = m ? __ldcs(ycol + (size_t)(__ffs(m) - 1) * n + i) : T(0);
      m &= m - 1u;
    }
    acc = v[0];
#pragma unroll
    for (int j = 1; j < 8; ++j)
      if ((unsigned)j < kmax) acc += v[j];
  }
  if (t < nmulti) __stcs(y + i, acc);
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
                           cudaStream_t st, Profiler* prof, Part part) {
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
  if (part.f1 > part.f0) {
    err = (nrhs == 1) ? (face_mode != 0 ? launch_faces<T>(hp, dd, x, fo, face_mode, st)
                                        : launch_face_kernel<T>(hp, dd, x, fo, st, part.f0,
                                                                part.f1))
                      : launch_face_kernel_multi<T>(hp, dd, x, ld, nrhs, fo, st);
    if (err != cudaSuccess) return err;
    nlaunch++;
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
  if (part.q1 > part.q0) {
    const int grid = std::min(part.q1 - part.q0, cap);
    cg_chunk_kernel<T, D, N, R><<<dim3(grid, nrhs), R * L, smem, st>>>(a, t);
    nlaunch++;
  }
  if (pr && (err = prof->mark(st)) != cudaSuccess) return err;
  const int64_t n = hp.n_dofs, nm = part.m1 - part.m0;
  if (nm > 0) {
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
// autotuner).  Both chunkings are built at set-up with the same colouring
// rule, so the two variants give bitwise-equal results.
template <typename T, int D, int N>
static cudaError_t apply_t(const HostProblem& hp, const DeviceData& dd, const T* x, T* y,
                           int64_t ld, int nrhs, T* fo, T* ycol, int face_mode, int variant,
                           cudaStream_t st, Profiler* prof, int slab, int stages) {
  constexpr int R = ChunkShape<D, N>::R;
  constexpr int RH = (R / 2) > 0 ? R / 2 : 1;
  const int v = (variant == 1 && RH < R) ? 1 : 0;
  const ChunkTable& ct = dd.chunks[v];
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
    return apply_r<T, D, N, RH>(hp, dd, ct, x, y, ld, nrhs, fo, ycol, face_mode, st, prof, part);
  return apply_r<T, D, N, R>(hp, dd, ct, x, y, ld, nrhs, fo, ycol, face_mode, st, prof, part);
}

template <typename T>
static cudaError_t dispatch(const HostProblem& hp, const DeviceData& dd, const T* x, T* y,
                            int64_t ld, int nrhs, T* fo, T* ycol, int face_mode, int variant,
                            cudaStream_t st, Profiler* prof, int slab = -1,
                            int stages = 3) {
#define SBM_CASE(DD, NN)                                                                  \
  if (hp.d == DD && hp.n == NN)                                                           \
    return apply_t<T, DD, NN>(hp, dd, x, y, ld, nrhs, fo, ycol, face_mode, variant, st, prof, \
                              slab, stages);
  SBM_CASE(2, 2) SBM_CASE(2, 3) SBM_CASE(2, 4) SBM_CASE(2, 5) SBM_CASE(2, 6) SBM_CASE(2, 7)
  SBM_CASE(3, 2) SBM_CASE(3, 3) SBM_CASE(3, 4) SBM_CASE(3, 5) SBM_CASE(3, 6) SBM_CASE(3, 7)
#undef SBM_CASE
  return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t launch_cg_apply(const HostProblem& hp, const DeviceData& dd, const T* x, T* y,
                            cudaStream_t st, Profiler* prof, int face_mode) {
  return dispatch<T>(hp, dd, x, y, 0, 1, face_out_of<T>(dd), ycol_of<T>(dd), face_mode,
                     dd.variant[std::is_same<T, float>::value ? 1 : 0], st, prof);
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
  return dispatch<double>(hp, dd, x, y, 0, 1, dd.face_out, dd.ycol, 0, dd.variant[0], st,
                          nullptr, slab, stages);
}

// The same launches with caller-provided scratch: per-face results
// ([F][2L]) and colour buffers ([ncolours][n_dofs]).
template <typename T>
cudaError_t launch_cg_apply_scratch(const HostProblem& hp, const DeviceData& dd, const T* x, T* y,
                                    T* face_scratch, T* colour_scratch, int variant,
                                    cudaStream_t st) {
  return dispatch<T>(hp, dd, x, y, 0, 1, face_scratch, colour_scratch, 0, variant, st, nullptr);
}
template cudaError_t launch_cg_apply_scratch<double>(const HostProblem&, const DeviceData&,
                                                     const double*, double*, double*, double*,
                                                     int, cudaStream_t);

// nrhs right-hand sides in one set of launches (grid.y = right-hand side);
// variant 0/1: R or R/2 cells per chunk (chosen by the autotuner).
template <typename T>
cudaError_t launch_cg_apply_multi(const HostProblem& hp, const DeviceData& dd, const T* x, T* y,
                                  int64_t ld, int nrhs, T* face_scratch, T* colour_scratch,
                                  int variant, cudaStream_t st) {
  return dispatch<T>(hp, dd, x, y, ld, nrhs, face_scratch, colour_scratch, 0, variant, st,
                     nullptr);
}
template cudaError_t launch_cg_apply_multi<double>(const HostProblem&, const DeviceData&,
                                                   const double*, double*, int64_t, int, double*,
                                                   double*, int, cudaStream_t);
template cudaError_t launch_cg_apply_multi<float>(const HostProblem&, const DeviceData&,
                                                  const float*, float*, int64_t, int, float*,
                                                  float*, int, cudaStream_t);

}  // namespace sbm
