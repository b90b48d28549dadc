// Cell term of the continuous Galerkin apply with one thread per cell and
// the cell's whole (p+1)^3 tile in registers (3D; FP32 for p <= 4, FP64 for
// p <= 3): tile shape 2 of the single applies.
//
// The chunk kernel (cg_apply.cu) spends most of its issue slots outside the
// arithmetic: staging runs in shared memory, splitting run indices, five
// barriers per chunk.  Here every line phase of the eigenbasis cell term
// (Algorithm 1 in the exact form sweeps.cuh describes) runs on registers
// with compile-time indices, so almost every instruction is a load, a store
// or an operation of the method.  Each thread
//  1. loads its cell's nodes from x (lines of the ordered cell table),
//  2. runs the five line phases (z- and y-transforms, the x-line operators
//     h K + mu_ab M, transforms back) -- the same per-line arithmetic as the
//     chunk kernel,
//  3. folds in its surrogate faces' results, in the chunk kernel's order
//     (under a programmatic dependent launch only the threads of cells with
//     surrogate faces wait for the face kernel),
//  4. adds the x-face values of the previous cell of its chunk (shared
//     memory; a block holds whole chunks), prev + own as the chunk kernel,
//  5. stores every node it owns (the last node of a line belongs to the next
//     cell of the chunk) into y or into its chunk's colour buffer, by the
//     chunk colouring of tile shape 0.
// The results are bitwise those of tile shape 0; the assembly kernel of that
// shape completes the DoFs several colours share.
#include <algorithm>
#include <cmath>

#include "chunk_body.cuh"

namespace sbm {

namespace {

// Threads (cells) per block, a block holding whole chunks of R = 256 / n^2
// cells: 96 at p = 4, 32 at p = 2, 3, 64 at p = 1 (a chunk of 64 cells).
// A thread lives one cell, about 25 us at p = 4, so the grid's last,
// partly filled wave costs up to that much; the sizes were measured
// (unprofiled FP32 applies, spheres of 96^3 cells, 128^3 at p = 2; 64
// threads before): p = 4 0.1352 -> 0.1331 ms (96; 32: 0.1429, 128:
// 0.1351), p = 3 0.0577 -> 0.0562 ms (32; 96: 0.0597), p = 2 0.0469 ->
// 0.0458 ms (32).  (Earlier, without the programmatic launch, 64-cell
// blocks beat 128-cell ones at p = 4: 0.096 -> 0.083 ms.)
constexpr int reg_threads(int n) { return n == 5 ? 96 : (n == 2 ? 64 : 32); }

// Resident blocks asked of the compiler, as warps per SM: FP32 p <= 3, 16
// (128 registers, no spills; p = 3 cell term 41.2 -> 37.9 us against 12 at
// 148 registers); p = 4 and FP64, 12 (168 registers; 14 or 16 warps spill
// the p = 4 tile: 83 -> 102 us).
template <typename T, int N>
constexpr int reg_min_blocks() {
  return ((std::is_same<T, float>::value && N <= 4) ? 16 : 12) * 32 / reg_threads(N);
}

template <int N>
constexpr int reg_words() {
  return (N * N * N + 31) / 32;
}

// h K + mu_ab M of every x-line of modes (a, b), index a + n b, in the
// even/odd layout of XLineOp::store, computed on the host with the same
// arithmetic as XLineOp (fused multiply-add, correctly rounded on both).
template <typename T, int N>
struct XOps {
  T m[N * N][XLineOp<T, N>::kSize];
};

template <typename T, int N>
XOps<T, N> make_xops(const KTab<T>& t) {
  constexpr int H = N / 2, HE = (N + 1) / 2;
  XOps<T, N> o;
  for (int b = 0; b < N; ++b)
    for (int a = 0; a < N; ++a) {
      T* m = o.m[a + N * b];
      const T mu = t.hlam[a] + t.hlam[b];
      for (int i = 0; i < HE; ++i)
        for (int j = i; j < HE; ++j)
          m[i * HE + j] = m[j * HE + i] = std::fma(mu, t.fM.E[i][j], t.fKh.E[i][j]);
      for (int i = 0; i < H; ++i)
        for (int j = i; j < H; ++j)
          m[HE * HE + i * H + j] = m[HE * HE + j * H + i] = std::fma(mu, t.fM.O[i][j],
                                                                      t.fKh.O[i][j]);
    }
  return o;
}

template <typename T>
struct RegArgs {
  const T* __restrict__ x;
  T* __restrict__ y;
  T* __restrict__ ycol;                     // [ncolours][n_dofs]
  const int32_t* __restrict__ lines;        // ordered cells x L
  const int32_t* __restrict__ face_start;
  const int32_t* __restrict__ face_kind;
  const T* __restrict__ face_out;           // [F][2L]
  const int32_t* __restrict__ chunk_first;  // tile shape 0
  const uint8_t* __restrict__ chunk_col;
  const int32_t* __restrict__ cell_chunk;   // ordered cell -> its chunk
  const uint32_t* __restrict__ mask;        // [Nc][W]: node shared by several colours
  const int32_t* __restrict__ block_first;  // [nblocks + 1] first chunk of each block
  int64_t n_dofs;
};

// the x-line operator h K + mu_ab M (even/odd layout) on one register line
template <typename T, int N>
__device__ __forceinline__ void xline_apply(const T* m, const T (&v)[N], T (&y)[N]) {
  constexpr int H = N / 2, HE = (N + 1) / 2;
  const LineFold<T, N> f(v);
  LineAcc<T, N> acc;
#pragma unroll
  for (int i = 0; i < HE; ++i)
#pragma unroll
    for (int j = 0; j < HE; ++j) acc.s[i] = fma(m[i * HE + j], f.e[j], acc.s[i]);
#pragma unroll
  for (int i = 0; i < H; ++i)
#pragma unroll
    for (int j = 0; j < H; ++j) acc.d[i] = fma(m[HE * HE + i * H + j], f.o[j], acc.d[i]);
  acc.unfold(y);
}

// the five line phases on the tile (node j0 + n j1 + n^2 j2)
template <typename T, int N>
__device__ __forceinline__ void cell_phases(const KTab<T>& t, const XOps<T, N>& xo,
                                            T (&u)[N * N * N]) {
  constexpr int L = N * N;
  T v[N], w[N];
#pragma unroll
  for (int l = 0; l < L; ++l) {          // z-lines (j0, j1) = (l % n, l / n) -> z-modes
#pragma unroll
    for (int j = 0; j < N; ++j) v[j] = u[l + L * j];
    line_to_modes<T, N>(t.fVt, v, w);
#pragma unroll
    for (int j = 0; j < N; ++j) u[l + L * j] = w[j];
  }
#pragma unroll
  for (int b = 0; b < N; ++b)            // y-lines (j0 = a, z-mode b) -> y-modes
#pragma unroll
    for (int a = 0; a < N; ++a) {
#pragma unroll
      for (int j = 0; j < N; ++j) v[j] = u[a + N * j + L * b];
      line_to_modes<T, N>(t.fVt, v, w);
#pragma unroll
      for (int j = 0; j < N; ++j) u[a + N * j + L * b] = w[j];
    }
#pragma unroll
  for (int l = 0; l < L; ++l) {          // x-lines (y-mode, z-mode) = (l % n, l / n)
#pragma unroll
    for (int j = 0; j < N; ++j) v[j] = u[N * l + j];
    xline_apply<T, N>(xo.m[l], v, w);
#pragma unroll
    for (int j = 0; j < N; ++j) u[N * l + j] = w[j];
  }
#pragma unroll
  for (int b = 0; b < N; ++b)            // y-modes back
#pragma unroll
    for (int a = 0; a < N; ++a) {
#pragma unroll
      for (int j = 0; j < N; ++j) w[j] = u[a + N * j + L * b];
      modes_to_line<T, N>(t.fV, w, v);
#pragma unroll
      for (int j = 0; j < N; ++j) u[a + N * j + L * b] = v[j];
    }
#pragma unroll
  for (int l = 0; l < L; ++l) {          // z-modes back
#pragma unroll
    for (int j = 0; j < N; ++j) w[j] = u[l + L * j];
    modes_to_line<T, N>(t.fV, w, v);
#pragma unroll
    for (int j = 0; j < N; ++j) u[l + L * j] = v[j];
  }
}

// surrogate face (k, s): the chunk kernel's fold_face_z on every z-line
// (j0, j1) of the tile, in the same operation order
template <typename T, int N, int K, int SD, bool COH>
__device__ __forceinline__ void fold_reg(const KTab<T>& t, const T* __restrict__ fo,
                                         T (&u)[N * N * N]) {
  constexpr int L = N * N, KEND = SD ? N - 1 : 0;
  const T* rv = fo;
  const T* rg = fo + L;
#pragma unroll
  for (int b = 0; b < N; ++b)
#pragma unroll
    for (int a = 0; a < N; ++a) {
      if (K == 2) {
        const T vv = ld_face<COH>(rv + a + N * b), g = ld_face<COH>(rg + a + N * b);
#pragma unroll
        for (int m = 0; m < N; ++m) {
          T& o = u[a + N * b + L * m];
          o = fma(SD ? t.D1[m] : t.D0[m], g, o);
          if (m == KEND) o = add_rn(o, vv);
        }
      } else {
        const int jk = (K == 0) ? a : b, jo = (K == 0) ? b : a;
        const T dk = SD ? t.D1[jk] : t.D0[jk];
#pragma unroll
        for (int m = 0; m < N; ++m) {
          T add = mul_rn(dk, ld_face<COH>(rg + jo + N * m));
          if (jk == KEND) add = add_rn(add, ld_face<COH>(rv + jo + N * m));
          u[a + N * b + L * m] = add_rn(u[a + N * b + L * m], add);
        }
      }
    }
}

template <typename T, int N, bool PDL>
__global__ void __launch_bounds__(reg_threads(N), (reg_min_blocks<T, N>()))
cg_cell_reg_kernel(const RegArgs<T> a, const __grid_constant__ KTab<T> t,
                   const __grid_constant__ XOps<T, N> xo) {
  constexpr int L = N * N, ND = L * N, P = N - 1, W = reg_words<N>();
  __shared__ T xface[reg_threads(N)][L + 1];    // j0 = P face of each cell (odd row stride)
  const int tid = threadIdx.x;
  const int b0 = a.block_first[blockIdx.x], b1 = a.block_first[blockIdx.x + 1];
  const int c0 = __ldg(a.chunk_first + b0), c1 = __ldg(a.chunk_first + b1);
  const int pos = c0 + tid;
  const bool act = pos < c1;
  T u[ND];
  int c = 0, nc = 0, ch = 0;
  const int32_t* ln = a.lines + (size_t)(act ? pos : 0) * L;
  if (act) {
    ch = __ldg(a.cell_chunk + pos);
    const int f = __ldg(a.chunk_first + ch);
    c = pos - f;
    nc = __ldg(a.chunk_first + ch + 1) - f;
#pragma unroll
    for (int l = 0; l < L; ++l) {
      const T* xl = a.x + __ldg(ln + l);
#pragma unroll
      for (int j0 = 0; j0 < N; ++j0) u[j0 + N * l] = __ldg(xl + j0);
    }
    cell_phases<T, N>(t, xo, u);
    const int fs = __ldg(a.face_start + pos), fe = __ldg(a.face_start + pos + 1);
    if constexpr (PDL) {
      if (fs < fe) pdl_wait();
    }
    for (int f2 = fs; f2 < fe; ++f2) {
      const int kind = __ldg(a.face_kind + f2);
      const T* fo = a.face_out + (size_t)f2 * 2 * L;
      switch (kind) {
        case 0: fold_reg<T, N, 0, 0, PDL>(t, fo, u); break;
        case 1: fold_reg<T, N, 1, 0, PDL>(t, fo, u); break;
        case 2: fold_reg<T, N, 2, 0, PDL>(t, fo, u); break;
        case 4: fold_reg<T, N, 0, 1, PDL>(t, fo, u); break;
        case 5: fold_reg<T, N, 1, 1, PDL>(t, fo, u); break;
        case 6: fold_reg<T, N, 2, 1, PDL>(t, fo, u); break;
        default: break;
      }
    }
#pragma unroll
    for (int l = 0; l < L; ++l) xface[tid][l] = u[P + N * l];
  }
  __syncthreads();
  if (!act) return;
  // the x-face node shared with the previous cell of the chunk: prev + own
  if (c > 0) {
#pragma unroll
    for (int l = 0; l < L; ++l) u[N * l] = add_rn(xface[tid - 1][l], u[N * l]);
  }
  uint32_t mk[W];
#pragma unroll
  for (int i = 0; i < W; ++i) mk[i] = __ldg(a.mask + (size_t)pos * W + i);
  T* yc = a.ycol + (size_t)__ldg(a.chunk_col + ch) * a.n_dofs;
  const bool last = c == nc - 1;     // only the chunk's last cell stores its j0 = P nodes
#pragma unroll
  for (int l = 0; l < L; ++l) {
    const int64_t base = __ldg(ln + l);
#pragma unroll
    for (int j0 = 0; j0 < N; ++j0) {
      const int node = j0 + N * l;
      if (j0 == P && !last) continue;
      T* dst = ((mk[node >> 5] >> (node & 31)) & 1u) ? yc : a.y;
      dst[base + j0] = u[node];
    }
  }
}

// per-cell multi-colour bits from the chunk run bits (tile shape 0): node
// (j0, line l) of cell c of chunk ch is element l S + P c + j0 of the
// chunk's runs, S = P nc + 1
__global__ void k_reg_mask(const int32_t* __restrict__ cell_chunk,
                           const int32_t* __restrict__ chunk_first,
                           const uint32_t* __restrict__ run_bits, int bit_words, int n, int nc_all,
                           int words, uint32_t* __restrict__ mask) {
  const int pos = blockIdx.x * blockDim.x + threadIdx.x;
  if (pos >= nc_all) return;
  const int P = n - 1, L = n * n, ND = L * n;
  const int ch = cell_chunk[pos];
  const int f = chunk_first[ch], nc = chunk_first[ch + 1] - f, c = pos - f;
  const int S = P * nc + 1;
  const uint32_t* bits = run_bits + (size_t)ch * bit_words;
  for (int w = 0; w < words; ++w) {
    uint32_t m = 0u;
    for (int b = 0; b < 32; ++b) {
      const int node = 32 * w + b;
      if (node >= ND) break;
      const int j0 = node % n, l = node / n;
      const int e = l * S + P * c + j0;
      if ((bits[e >> 5] >> (e & 31)) & 1u) m |= 1u << b;
    }
    mask[(size_t)pos * words + w] = m;
  }
}

template <typename T, int N>
cudaError_t launch_reg(const HostProblem& hp, const DeviceData& dd, const T* x, T* y,
                       const T* fo, T* ycol, cudaStream_t st, bool pdl) {
  RegArgs<T> a;
  a.x = x;
  a.y = y;
  a.ycol = ycol;
  a.lines = dd.lines;
  a.face_start = dd.face_start;
  a.face_kind = dd.face_kind;
  a.face_out = fo;
  a.chunk_first = dd.chunks[0].first;
  a.chunk_col = dd.chunks[0].colour;
  a.cell_chunk = dd.reg_cell_chunk;
  a.mask = dd.reg_mask;
  a.block_first = dd.reg_block_first;
  a.n_dofs = hp.n_dofs;
  const KTab<T> t = make_ktab<T>(hp);
  const XOps<T, N> xo = make_xops<T, N>(t);
  // pdl (FP32 applies after the CUDA-core face kernel): a programmatic
  // dependent launch; a thread waits for the face kernel only when its cell
  // has surrogate faces (the other cells need nothing from it) and then reads
  // the face results with coherent loads.  The kernel does not trigger its
  // own dependents early (the assembly starts as its blocks finish): an early
  // trigger cost 0.5-1 %.  Measured, unprofiled FP32 applies on GB300,
  // spheres with 96^3 cells (128^3 at p = 2): p = 4 0.1427 -> 0.1409 ms,
  // p = 3 0.0623 -> 0.0577 ms, p = 2 0.0520 -> 0.0480 ms; results bitwise
  // unchanged.
  cudaError_t e = pdl ? launch_maybe_pdl(cg_cell_reg_kernel<T, N, true>, dim3(dd.reg_nblocks),
                                         dim3(reg_threads(N)), 0, st, true, a, t, xo)
                      : launch_maybe_pdl(cg_cell_reg_kernel<T, N, false>, dim3(dd.reg_nblocks),
                                         dim3(reg_threads(N)), 0, st, false, a, t, xo);
  return e != cudaSuccess ? e : cudaGetLastError();
}

}  // namespace

bool cell_reg_available(const HostProblem& hp, bool fp32) {
  return hp.d == 3 && !hp.desc.dg && hp.n >= 2 && hp.n <= (fp32 ? 5 : 4);
}

// The per-cell tables of tile shape 2 (3D continuous Galerkin, n <= 5): the
// chunk of every ordered cell, blocks of whole chunks (at most
// reg_threads(n) cells; a chunk has at most 256 / n^2 <= reg_threads(n)),
// and the per-cell multi-colour bits (from the device run bits of tile
// shape 0).
cudaError_t build_cell_reg_tables(const HostProblem& hp, const std::vector<int32_t>& ch_first,
                                  DeviceData* dd) {
  if (!cell_reg_available(hp, true)) return cudaSuccess;
  const int nch = (int)ch_first.size() - 1;
  const int nc_all = ch_first.back();
  const int threads = reg_threads(hp.n);
  std::vector<int32_t> cell_chunk(nc_all), block_first;
  for (int q = 0; q < nch; ++q) {
    if (ch_first[q + 1] - ch_first[q] > threads) return cudaErrorInvalidValue;
    for (int i = ch_first[q]; i < ch_first[q + 1]; ++i) cell_chunk[i] = q;
  }
  for (int q = 0; q < nch;) {
    block_first.push_back(q);
    int q1 = q;
    while (q1 < nch && ch_first[q1 + 1] - ch_first[q] <= threads) ++q1;
    q = std::max(q1, q + 1);
  }
  block_first.push_back(nch);
  const int words = (hp.nd + 31) / 32;
  cudaError_t e = cudaMalloc((void**)&dd->reg_cell_chunk, cell_chunk.size() * sizeof(int32_t));
  if (e == cudaSuccess)
    e = cudaMemcpy(dd->reg_cell_chunk, cell_chunk.data(), cell_chunk.size() * sizeof(int32_t),
                   cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMalloc((void**)&dd->reg_block_first, block_first.size() * sizeof(int32_t));
  if (e == cudaSuccess)
    e = cudaMemcpy(dd->reg_block_first, block_first.data(), block_first.size() * sizeof(int32_t),
                   cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMalloc((void**)&dd->reg_mask, (size_t)nc_all * words * sizeof(uint32_t));
  if (e == cudaSuccess && nc_all > 0) {
    k_reg_mask<<<(nc_all + 255) / 256, 256>>>(dd->reg_cell_chunk, dd->chunks[0].first,
                                             dd->chunks[0].run_bits, dd->chunks[0].bit_words,
                                             hp.n, nc_all, words, dd->reg_mask);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
  }
  dd->reg_nblocks = (int)block_first.size() - 1;
  return e;
}

template <typename T>
cudaError_t launch_cell_reg(const HostProblem& hp, const DeviceData& dd, const T* x, T* y,
                            const T* fo, T* ycol, cudaStream_t st, bool pdl) {
  if (!cell_reg_available(hp, std::is_same<T, float>::value) || !dd.reg_mask)
    return cudaErrorInvalidValue;
  switch (hp.n) {
    case 2: return launch_reg<T, 2>(hp, dd, x, y, fo, ycol, st, pdl);
    case 3: return launch_reg<T, 3>(hp, dd, x, y, fo, ycol, st, pdl);
    case 4: return launch_reg<T, 4>(hp, dd, x, y, fo, ycol, st, pdl);
    case 5:
      if constexpr (std::is_same<T, float>::value)
        return launch_reg<T, 5>(hp, dd, x, y, fo, ycol, st, pdl);
      return cudaErrorInvalidValue;
    default: return cudaErrorInvalidValue;
  }
}
template cudaError_t launch_cell_reg<double>(const HostProblem&, const DeviceData&, const double*,
                                             double*, const double*, double*, cudaStream_t,
                                             bool);
template cudaError_t launch_cell_reg<float>(const HostProblem&, const DeviceData&, const float*,
                                            float*, const float*, float*, cudaStream_t,
                                            bool);

}  // namespace sbm
