// The continuous Galerkin chunk kernel's building blocks, shared by the
// single-problem apply (cg_apply.cu) and the persistent batched apply
// (batch_kernel.cuh): the chunk arguments, the face folds, the shared-memory
// layout, the cp.async gather, the chunk loop (gather, cell term of
// Algorithm 1, surrogate-face folds, x-face sums, single-writer stores) and
// the assembly of the DoFs several colours share.
#pragma once

#include "sweeps.cuh"

namespace sbm {

// Loads of the per-face results and of the colour buffers.  COH = false:
// read-only-path loads (the data was written by an earlier launch); COH =
// true: loads at the L2 (ld.global.cg), for data another block of the same
// launch wrote (the persistent batched kernel), which the read-only path
// does not keep coherent.
template <bool COH, typename T>
__device__ __forceinline__ T ld_face(const T* p) {
  if constexpr (COH) return __ldcg(p);
  else return __ldg(p);
}

// Separately rounded product and sum (never contracted into a fused
// multiply-add): the face folds round the same way in every kernel that
// applies them, whatever the compiler knows about their operands.
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }

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

// ---- colour-ordered stores ----------------------------------------------------
//
// The alternative to colour buffers and the assembly pass (single applies):
// the chunks run in ascending colour order, taken from a ticket counter.  A
// DoF several colours share is stored by its lowest colour's chunk, then
// read, added to and stored back by each higher colour's chunk in colour
// order -- the sum and the order of the assembly, so y is bitwise the same.
// Before its stores a chunk waits (bounded) for the lower-colour chunks it
// shares a DoF with: per-chunk completion counts that every launch raises by
// one, the target being the chunk's own count + 1 (no reset between
// launches).  Every dependency has a smaller ticket, taken by a block that
// is running, so the order cannot deadlock; on expiry the block records
// SBM_ERR_TIMEOUT and still stores and counts its chunk, so the counts stay
// in step.  The last block to finish resets the ticket counters.
struct OrdArgs {
  const int32_t* __restrict__ ord;       // ticket -> chunk (colours ascending)
  const uint32_t* __restrict__ add_bits; // per chunk: run elements to read-add-write
  const int32_t* __restrict__ deps;      // [nchunk][cap] lower-colour neighbours
  const int32_t* __restrict__ ndeps;
  int* done;                             // [nchunk] completion counts
  unsigned* tickets;                     // [0] next ticket, [1] blocks finished
  int* err;
  int nch, cap;
};
constexpr long long kOrdPolls = 1ll << 20;     // about a second of polling

__device__ __forceinline__ int ld_acquire_gpu(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
// relaxed (no ordering of later accesses: the first look at a count is
// issued before the compute and must not hold it up); fence_acquire_gpu
// after the counts were seen orders the reads of y that follow
__device__ __forceinline__ int ld_relaxed_gpu(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void fence_acquire_gpu() {
  asm volatile("fence.acq_rel.gpu;" ::: "memory");
}
__device__ __forceinline__ void st_release_gpu(int* p, int v) {
  asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
// wrap-safe count comparison
__device__ __forceinline__ bool count_reached(int v, int target) {
  return (int)((unsigned)v - (unsigned)target) >= 0;
}

// The first look at chunk ch's lower-colour neighbours, issued early (one
// per thread, blockDim >= cap) and checked by ord_wait after the compute.
__device__ __forceinline__ int ord_peek(const OrdArgs& o, int ch, int target) {
  const int nd = __ldg(o.ndeps + ch);
  return (int)threadIdx.x < nd
             ? ld_relaxed_gpu(o.done + __ldg(o.deps + (size_t)ch * o.cap + threadIdx.x))
             : target;
}

// Block-wide: wait until chunk ch's lower-colour neighbours are done
// (count >= target), bounded; peek: this thread's ord_peek.  All threads
// call it.
__device__ __forceinline__ void ord_wait(const OrdArgs& o, int ch, int target, int peek) {
  if (__syncthreads_and(count_reached(peek, target))) {
    if ((int)threadIdx.x < __ldg(o.ndeps + ch)) fence_acquire_gpu();
    __syncthreads();
    return;
  }
  const int nd = __ldg(o.ndeps + ch);
  const int32_t* dl = o.deps + (size_t)ch * o.cap;
  for (long long it = 0;; ++it) {
    int ok = 1;
    for (int i = threadIdx.x; i < nd; i += blockDim.x)
      if (!count_reached(ld_acquire_gpu(o.done + __ldg(dl + i)), target)) ok = 0;
    if (__syncthreads_and(ok)) return;
    if (it >= kOrdPolls) {
      if (threadIdx.x == 0) atomicExch(o.err, SBM_ERR_TIMEOUT);
      return;
    }
    __nanosleep(128);
  }
}

// The block's last act: count it out; the last one resets the counters for
// the next launch.
__device__ __forceinline__ void ord_exit(const OrdArgs& o) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned nb = gridDim.x * gridDim.y * gridDim.z;
    if (atomicAdd(o.tickets + 1, 1u) == nb - 1u) {
      atomicExch(o.tickets, 0u);
      atomicExch(o.tickets + 1, 0u);
    }
  }
}

// a ticket's chunk, or -1 past the last
__device__ __forceinline__ int ord_chunk(const OrdArgs& o, int tk) {
  return tk < o.nch ? __ldg(o.ord + tk) : -1;
}

// Add the contributions of surrogate face (k, s) to the z-line result out[]
// (nodes (a, b, m), m = 0..n-1) of a 3D cell: R[node with j_k = kend] +=
// rv[jt], R[node] += phi_{j_k}'(s) rg[jt], jt = the node's tangential index
// (the two other axes in increasing order, the first fastest).
template <typename T, int N, bool COH>
__device__ __forceinline__ void fold_face_z(const KTab<T>& t, const T* __restrict__ fo, int k,
                                            int s, int a, int b, T (&out)[N]) {
  constexpr int L = N * N;
  const T* rv = fo;
  const T* rg = fo + L;
  const int kend = s ? N - 1 : 0;
  if (k == 2) {                       // normal along the line, tangential (a, b)
    const int jt = a + N * b;
    const T v = ld_face<COH>(rv + jt), g = ld_face<COH>(rg + jt);
#pragma unroll
    for (int m = 0; m < N; ++m) {
      out[m] = fma(s ? t.D1[m] : t.D0[m], g, out[m]);
      if (m == kend) out[m] = add_rn(out[m], v);  // compile-time index: out stays in registers
    }
  } else {
    // k == 0: j_k = a, tangential (j1, j2) = (b, m);  k == 1: j_k = b, (j0, j2) = (a, m)
    const int jk = (k == 0) ? a : b;
    const int jo = (k == 0) ? b : a;
    const T dk = s ? t.D1[jk] : t.D0[jk];
#pragma unroll
    for (int m = 0; m < N; ++m) {
      const int jt = jo + N * m;
      T add = mul_rn(dk, ld_face<COH>(rg + jt));
      if (jk == kend) add = add_rn(add, ld_face<COH>(rv + jt));
      out[m] = add_rn(out[m], add);
    }
  }
}

// Add the contributions of surrogate face (k, s) to the x-line result out[]
// of line tl: R[node (kend, jt)] += rv[jt], R[node (j, jt)] += phi_j'(s) rg[jt].
template <typename T, int D, int N, bool COH>
__device__ __forceinline__ void fold_face(const KTab<T>& t, const T* __restrict__ fo, int k, int s,
                                          int tl, T (&out)[N]) {
  constexpr int L = Shape<D, N>::L;
  const T* rv = fo;
  const T* rg = fo + L;
  const int kend = s ? N - 1 : 0;
  if (k == 0) {                       // tangential index = the line itself
    const T v = ld_face<COH>(rv + tl), g = ld_face<COH>(rg + tl);
#pragma unroll
    for (int m = 0; m < N; ++m) {
      out[m] = fma(s ? t.D1[m] : t.D0[m], g, out[m]);
      if (m == kend) out[m] = add_rn(out[m], v);  // compile-time index: out stays in registers
    }
  } else {
    // k == 1: line tl = (j1, j2), tangential (m, j2);  k == 2: tangential (m, j1)
    const int jk = (D == 2 || k == 1) ? tl % N : tl / N;
    const int jo = (D == 2) ? 0 : (k == 1 ? tl / N : tl % N);
    const T dk = s ? t.D1[jk] : t.D0[jk];
#pragma unroll
    for (int m = 0; m < N; ++m) {
      const int jt = m + N * jo;
      T add = mul_rn(dk, ld_face<COH>(rg + jt));
      if (jk == kend) add = add_rn(add, ld_face<COH>(rv + jt));
      out[m] = add_rn(out[m], add);
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
  static constexpr int TILE =                                   // scalars before the runs
      (D == 3) ? R * TilePad<T, N>::NDP : 2 * R * ND;
  static constexpr int XS = (D == 3) ? L * SM : XZ;
  static constexpr int WORDS = (L * SM + 31) / 32;              // run-element bits
  static constexpr int XL =                                     // x-line operators
      (D == 3) ? XLineOp<T, N>::kSlots * XLineOp<T, N>::kPacked : 0;
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
  for (int idx = tid; idx < L * S; idx += blockDim.x) {
    const int l = __float2int_rz(((float)idx + 0.5f) * invS), kk = idx - l * S;
    cp_async_elem(Xs + l * SM + kk, xr + (int64_t)Ls[l] + kk);
  }
}


// Position of node (j0 = m, x-line l) of chunk cell cc among the per-cell
// results: 3D, the padded tile (TilePad); 2D, the run area ((cc L + l) n + m).
template <typename T, int D, int N>
__device__ __forceinline__ int zix(int cc, int l, int m) {
  if constexpr (D == 3) return cc * TilePad<T, N>::NDP + TilePad<T, N>::PX * l + m;
  else return (cc * Shape<D, N>::L + l) * N + m;
}

// h K + mu M of the 3D x-lines into the chunk's shared memory (one operator
// per x-line of modes (a, b) = (tl % n, tl / n), built by the threads of
// cell 0); visible after the caller's next barrier.  tx supplies hlam, fM
// and fKh (the problem's h-scaled tables).
template <typename T, int D, int N, int R>
__device__ __forceinline__ T* chunk_xline_smem(unsigned char* smem_raw) {
  using CS = ChunkSmem<T, D, N, R>;
  return reinterpret_cast<T*>(smem_raw) + CS::TILE + 2 * CS::XS;
}
template <typename T, int D, int N, int R>
__device__ __forceinline__ void chunk_xline_build(unsigned char* smem_raw, const KTab<T>& tx,
                                                  int tid) {
  constexpr int L = Shape<D, N>::L;
  if (D == 3 && tid < L && tid % N <= tid / N)
    XLineOp<T, N>(tx, tid % N, tid / N)
        .store(chunk_xline_smem<T, D, N, R>(smem_raw) +
               XLineOp<T, N>::slot(tid % N, tid / N) * XLineOp<T, N>::kPacked);
}

// Chunks ch, ch + step, ... (< q1) of right-hand side rhs, by the whole block
// of NTHR >= R L threads (threads beyond R L only help with the copies).
// t supplies the h-independent tables (eigenbasis transforms, face-fold
// derivatives; 2D: the 1D mass and stiffness, h^(d-2) = 1); the x-line
// operators are already in shared memory (chunk_xline_build).  The next
// chunk's runs are copied in (cp.async) while the current one is computed.
template <typename T, int D, int N, int R, bool COH, int NTHR, bool PDL = false>
__device__ __forceinline__ void chunk_loop(const ChunkArgs<T>& a, const KTab<T>& t,
                                           unsigned char* smem_raw, int rhs, int ch, int q1,
                                           int step) {
  constexpr int L = Shape<D, N>::L, P = N - 1;
  constexpr int SM = ChunkSmem<T, D, N, R>::SM;
  using P2 = typename PairOf<T>::type;
  using CS = ChunkSmem<T, D, N, R>;
  T* tile = reinterpret_cast<T*>(smem_raw);   // 3D: [R][ND] scalar tile
  P2* AE = reinterpret_cast<P2*>(smem_raw);   // 2D: pair tile (8/16-byte aligned); phase 2
                                              //     runs in place
  T* Xbuf = tile + CS::TILE;                  // [2][L][SM] x-line runs (current, next)
  T* XLs = Xbuf + 2 * CS::XS;                                // 3D: [L] x-line operators
  int* Lbuf = reinterpret_cast<int*>(XLs + CS::XL);          // [2][L] run starts
  uint32_t* Bs = reinterpret_cast<uint32_t*>(Lbuf + 2 * L);  // run-element bits
  const int tid = threadIdx.x;
  // the copy loop steps by the compile-time block size, the other loops by
  // blockDim.x (the same value; this split keeps the FP64 kernels at 32-40
  // registers)
  constexpr int nthr = NTHR;
  const int c = tid / L, tl = tid - c * L;
  const XLineShared<T, N> xop{XLs + XLineOp<T, N>::slot(tl % N, tl / N) *
                                         XLineOp<T, N>::kPacked};
  const T* __restrict__ xr = a.x + rhs * a.ldx;
  const T* fo = a.face_out + rhs * a.ld_face;
  T* ycb = a.ycol + rhs * a.ld_ycol;
  T* yb = a.y + rhs * a.ldx;

  // prologue: the first chunk's run starts, then its runs in flight
  int buf = 0;
  if (ch < q1) {
    const int first = __ldg(a.chunk_first + ch);
    const int S = P * (__ldg(a.chunk_first + ch + 1) - first) + 1;
    for (int i = tid; i < L; i += blockDim.x) Lbuf[i] = __ldg(a.lines + (size_t)first * L + i);
    __syncthreads();
    gather_runs_async<T, L, SM>(xr, Lbuf, Xbuf, S, tid, nthr);
  }
  cp_async_commit();
  // PDL: the first chunk's runs are in flight; the face kernel's results
  // are read from here on
  if (PDL) pdl_wait();
  for (; ch < q1; ch += step, buf ^= 1) {
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
    const int nx = ch + step;
    if (nx < q1) {
      const int f2 = __ldg(a.chunk_first + nx);
      const int S2 = P * (__ldg(a.chunk_first + nx + 1) - f2) + 1;
      int* Ln = Lbuf + (buf ^ 1) * L;
      for (int i = tid; i < L; i += blockDim.x) Ln[i] = __ldg(a.lines + (size_t)f2 * L + i);
      __syncthreads();
      gather_runs_async<T, L, SM>(xr, Ln, Xbuf + (buf ^ 1) * CS::XS, S2, tid, nthr);
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
          fold_face_z<T, N, COH>(t, fo + (size_t)f * 2 * L, kind & 3, kind >> 2, tl % N, tl / N,
                                 out);
        else
          fold_face<T, D, N, COH>(t, fo + (size_t)f * 2 * L, kind & 3, kind >> 2, tl, out);
      }
      // 3D: z-line (j0, j1) = tl, back to the nodes it was read from
#pragma unroll
      for (int m = 0; m < N; ++m) {
        if constexpr (D == 3)
          Z[c * TilePad<T, N>::NDP + tl % N + TilePad<T, N>::PX * (tl / N + N * m)] = out[m];
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
      if (cc == nc) v = Z[zix<T, D, N>(nc - 1, l, P)];
      else if (m == 0 && cc > 0) v = Z[zix<T, D, N>(cc - 1, l, P)] + Z[zix<T, D, N>(cc, l, 0)];
      else v = Z[zix<T, D, N>(cc, l, m)];
      const int64_t g = (int64_t)Ls[l] + kk;
      if ((Bs[idx >> 5] >> (idx & 31)) & 1u) yc[g] = v;
      else yb[g] = v;
    }
    __syncthreads();                          // Xs / Z / Ls / Bs are reused
  }
  cp_async_wait<0>();
}

// chunk_loop with colour-ordered stores (single applies, one right-hand
// side, a block of exactly R L threads): the chunks come from the ticket
// counter, the next ticket taken one chunk ahead; a chunk peeks at its
// lower-colour neighbours' counts before its compute and waits, if it must,
// before its stores.
__shared__ int s_ord_next;
template <typename T, int D, int N, int R>
__device__ __forceinline__ void chunk_loop_ord(const ChunkArgs<T>& a, const KTab<T>& t,
                                               unsigned char* smem_raw, const OrdArgs& o) {
  constexpr int L = Shape<D, N>::L, P = N - 1;
  constexpr int SM = ChunkSmem<T, D, N, R>::SM;
  using P2 = typename PairOf<T>::type;
  using CS = ChunkSmem<T, D, N, R>;
  T* tile = reinterpret_cast<T*>(smem_raw);
  P2* AE = reinterpret_cast<P2*>(smem_raw);
  T* Xbuf = tile + CS::TILE;
  T* XLs = Xbuf + 2 * CS::XS;
  int* Lbuf = reinterpret_cast<int*>(XLs + CS::XL);
  uint32_t* Bs = reinterpret_cast<uint32_t*>(Lbuf + 2 * L);
  const int tid = threadIdx.x;
  const int c = tid / L, tl = tid - c * L;
  const XLineShared<T, N> xop{XLs + XLineOp<T, N>::slot(tl % N, tl / N) *
                                         XLineOp<T, N>::kPacked};
  const T* __restrict__ xr = a.x;
  T* yb = a.y;

  if (tid == 0) s_ord_next = (int)atomicAdd(o.tickets, 1u);
  __syncthreads();
  int ch = ord_chunk(o, s_ord_next);
  __syncthreads();                            // s_ord_next read by all
  int buf = 0;
  if (ch >= 0) {
    const int first = __ldg(a.chunk_first + ch);
    const int S = P * (__ldg(a.chunk_first + ch + 1) - first) + 1;
    for (int i = tid; i < L; i += blockDim.x) Lbuf[i] = __ldg(a.lines + (size_t)first * L + i);
    __syncthreads();
    if (tid == 0) s_ord_next = (int)atomicAdd(o.tickets, 1u);
    gather_runs_async<T, L, SM>(xr, Lbuf, Xbuf, S, tid, R * L);
  }
  cp_async_commit();
  __syncthreads();                            // s_ord_next written
  for (; ch >= 0; buf ^= 1) {
    T* Xs = Xbuf + buf * CS::XS;
    const int* Ls = Lbuf + buf * L;
    T* Z = (D == 3) ? tile : Xs;
    const int first = __ldg(a.chunk_first + ch);
    const int nc = __ldg(a.chunk_first + ch + 1) - first;
    const int S = P * nc + 1;
    const float invS = 1.0f / (float)S;
    const int target = __ldcg(o.done + ch) + 1;
    const int peek = ord_peek(o, ch, target);
    const int nx = ord_chunk(o, s_ord_next);
    // the ticket after nx, taken now and published after the compute (its
    // latency hidden behind this chunk)
    unsigned tk2 = 0u;
    if (nx >= 0) {
      const int f2 = __ldg(a.chunk_first + nx);
      const int S2 = P * (__ldg(a.chunk_first + nx + 1) - f2) + 1;
      int* Ln = Lbuf + (buf ^ 1) * L;
      for (int i = tid; i < L; i += blockDim.x) Ln[i] = __ldg(a.lines + (size_t)f2 * L + i);
      if (tid == 0) tk2 = atomicAdd(o.tickets, 1u);
      __syncthreads();
      gather_runs_async<T, L, SM>(xr, Ln, Xbuf + (buf ^ 1) * CS::XS, S2, tid, R * L);
    }
    cp_async_commit();
    {
      const uint32_t* bits = o.add_bits + (size_t)ch * a.bit_words;
      for (int i = tid; i < (L * S + 31) / 32; i += blockDim.x) Bs[i] = __ldg(bits + i);
    }
    cp_async_wait<1>();
    __syncthreads();
    const bool act = c < nc;
    T out[N];
    if constexpr (D == 3)
      cell_fd_3d<T, N>(t, Xs, (tl / N) * SM + P * c + (tl % N), N * SM, tile, c, tl, act, xop,
                       out);
    else
      cell_sweeps_2d<T, N>(t, Xs, P * c + tl, SM, AE, c, tl, act, out);
    pdl_wait();                               // the face kernel's results
    if (act) {
      const int pos = first + c;
      const int fs = __ldg(a.face_start + pos), fe = __ldg(a.face_start + pos + 1);
      for (int f = fs; f < fe; ++f) {
        const int kind = __ldg(a.face_kind + f);
        if constexpr (D == 3)
          fold_face_z<T, N, true>(t, a.face_out + (size_t)f * 2 * L, kind & 3, kind >> 2,
                                  tl % N, tl / N, out);
        else
          fold_face<T, D, N, true>(t, a.face_out + (size_t)f * 2 * L, kind & 3, kind >> 2, tl,
                                   out);
      }
#pragma unroll
      for (int m = 0; m < N; ++m) {
        if constexpr (D == 3)
          Z[c * TilePad<T, N>::NDP + tl % N + TilePad<T, N>::PX * (tl / N + N * m)] = out[m];
        else Z[(c * L + tl) * N + m] = out[m];
      }
    }
    __syncthreads();
    ord_wait(o, ch, target, peek);
    // a thread's run elements (at most n of them: L S <= L (P R + 1) <=
    // n R L): first the earlier colours' partial sums where the bit is set,
    // loaded together, then the values (again from shared memory, the node
    // shared by cells c-1 and c summed in chunk_loop's order) and the stores
    T old[N];
#pragma unroll
    for (int k = 0; k < N; ++k) {
      const int idx = tid + k * R * L;
      old[k] = T(0);
      if (idx < L * S && ((Bs[idx >> 5] >> (idx & 31)) & 1u)) {
        const int l = __float2int_rz(((float)idx + 0.5f) * invS);
        old[k] = __ldcg(yb + Ls[l] + (idx - l * S));
      }
    }
#pragma unroll
    for (int k = 0; k < N; ++k) {
      const int idx = tid + k * R * L;
      if (idx < L * S) {
        const int l = __float2int_rz(((float)idx + 0.5f) * invS), kk = idx - l * S;
        const int cc = kk / P, m = kk - cc * P;
        T v;
        if (cc == nc) v = Z[zix<T, D, N>(nc - 1, l, P)];
        else if (m == 0 && cc > 0)
          v = Z[zix<T, D, N>(cc - 1, l, P)] + Z[zix<T, D, N>(cc, l, 0)];
        else v = Z[zix<T, D, N>(cc, l, m)];
        yb[(int64_t)Ls[l] + kk] = ((Bs[idx >> 5] >> (idx & 31)) & 1u) ? old[k] + v : v;
      }
    }
    if (tid == 0 && nx >= 0) s_ord_next = (int)tk2;
    __syncthreads();                          // Xs / Z / Ls / Bs are reused
    if (tid == 0) st_release_gpu(o.done + ch, target);
    ch = nx;
  }
  cp_async_wait<0>();
  ord_exit(o);
}

// For the DoFs i = multi[t], t in [t0, t0 + 32) of one warp (lanes past
// nmulti idle): y_i = sum_{c in mask_i} ycol[c][i], colours in increasing
// order.  Lane by lane the j-th step adds the value of the lane's j-th colour
// (0 past its count), for j up to the warp's largest colour count.  FP64: a
// loop with a warp-uniform, run-time trip count, so the additions a warp
// issues are its own count minus one (on GB300 a double addition costs an
// FP64-pipe slot per warp instruction, whatever its active lanes; the list
// is grouped by colour count, so most warps need one).  FP32: all loads
// first, then the unrolled sum over the lane's own colours (the additions
// are cheap, the load latency is not).  All 32 lanes of the warp call
// this together.  COH: colour buffers written by other blocks of the same
// launch (L2 loads instead of the streaming ones).
template <typename T, bool COH>
__device__ __forceinline__ void assemble_warp(const T* __restrict__ ycol,
                                              const int32_t* __restrict__ multi,
                                              const uint8_t* __restrict__ multi_mask,
                                              T* __restrict__ y, int64_t n, int64_t nmulti,
                                              int ncol, int64_t t) {
  int64_t i = 0;
  unsigned m = 0u;
  if (t < nmulti) {
    i = __ldg(multi + t);
    m = (unsigned)__ldg(multi_mask + t);
  }
  if (ncol < 8) m &= (1u << ncol) - 1u;
  const unsigned kmax = __reduce_max_sync(0xffffffffu, (unsigned)__popc(m));
  auto ld = [&](unsigned mm) -> T {
    const T* p = ycol + (size_t)(__ffs(mm) - 1) * n + i;
    if constexpr (COH) return __ldcg(p);
    else return __ldcs(p);
  };
  T acc = T(0);
  if constexpr (std::is_same<T, double>::value) {
    if (m) {
      acc = ld(m);
      m &= m - 1u;
    }
    for (unsigned j = 1; j < kmax; ++j) {
      T v = T(0);
      if (m) {
        v = ld(m);
        m &= m - 1u;
      }
      acc += v;
    }
  } else {
    const unsigned cnt = __popc(m);
    T v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      v[j] = m ? ld(m) : T(0);
      m &= m - 1u;
    }
    acc = v[0];
#pragma unroll
    for (int j = 1; j < 8; ++j)
      if ((unsigned)j < cnt) acc += v[j];
  }
  if (t < nmulti) __stcs(y + i, acc);
}

// Two shared DoFs per thread, entries t0 and t0 + stride: all colour values
// of both loaded before either is summed, the loads unrolled to the warp's
// largest colour count K (the list is grouped by count).  The sums are
// assemble_warp's -- in colour order, FP32 over the lane's own colours,
// FP64 over the warp's largest count (zeros past the lane's own) -- so the
// results are bitwise the same.  All 32 lanes of the warp call this.
template <typename T, bool COH, int K>
__device__ __forceinline__ void assemble_pair_k(const T* __restrict__ ycol,
                                                const int64_t (&i)[2], unsigned (&m)[2],
                                                const int64_t (&t)[2], unsigned kmax,
                                                T* __restrict__ y, int64_t n, int64_t nmulti) {
  T v[2][K];
  unsigned cnt[2];
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    cnt[e] = std::is_same<T, float>::value ? __popc(m[e]) : kmax;
#pragma unroll
    for (int j = 0; j < K; ++j) {
      const T* p = ycol + (size_t)(__ffs(m[e]) - 1) * n + i[e];
      v[e][j] = m[e] ? (COH ? __ldcg(p) : __ldcs(p)) : T(0);
      m[e] &= m[e] - 1u;
    }
  }
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    T acc = v[e][0];
#pragma unroll
    for (int j = 1; j < K; ++j)
      if ((unsigned)j < cnt[e]) acc += v[e][j];
    if (t[e] < nmulti) __stcs(y + i[e], acc);
  }
}

template <typename T, bool COH, bool PDL = false>
__device__ __forceinline__ void assemble_pair(const T* __restrict__ ycol,
                                              const int32_t* __restrict__ multi,
                                              const uint8_t* __restrict__ multi_mask,
                                              T* __restrict__ y, int64_t n, int64_t nmulti,
                                              int ncol, int64_t t0, int stride) {
  const int64_t t[2] = {t0, t0 + stride};
  int64_t i[2];
  unsigned m[2], kmax = 0u;
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    i[e] = t[e] < nmulti ? __ldg(multi + t[e]) : 0;
    m[e] = t[e] < nmulti ? (unsigned)__ldg(multi_mask + t[e]) : 0u;
    if (ncol < 8) m[e] &= (1u << ncol) - 1u;
    kmax = max(kmax, (unsigned)__popc(m[e]));
  }
  kmax = __reduce_max_sync(0xffffffffu, kmax);
  if (PDL) pdl_wait();                        // the cell kernel's colour buffers
  if (kmax <= 2) assemble_pair_k<T, COH, 2>(ycol, i, m, t, kmax, y, n, nmulti);
  else if (kmax <= 4) assemble_pair_k<T, COH, 4>(ycol, i, m, t, kmax, y, n, nmulti);
  else assemble_pair_k<T, COH, 8>(ycol, i, m, t, kmax, y, n, nmulti);
}


// ---- tile shape 3: the chunk loop without staged runs (3D) ------------------------
//
// The same chunks, phases, folds, x-face sums and single-writer stores as
// chunk_loop, but each thread loads its own z-line (j0, j1) of x straight
// from global memory (the chunk's runs start at its first cell's lines, cell
// c P c further) and stores its own z-line result straight to y or to the
// chunk's colour buffer; only the x-face nodes two cells of the chunk share
// pass through shared memory (prev + own, as chunk_loop sums them).  Without
// the run staging and its index splitting a chunk costs a third of the
// instructions; the arithmetic and the summation order are unchanged, so the
// results are bitwise those of tile shape 0.
template <typename T, int N, int R>
struct DirectSmem {
  static constexpr int L = N * N, ND = L * N, P = N - 1;
  static constexpr int TILE = R * TilePad<T, N>::NDP;    // the cells' tiles
  static constexpr int XL = XLineOp<T, N>::kSlots * XLineOp<T, N>::kPacked;  // x-line ops
  static constexpr int XF = R * L;                       // j0 = P faces of the cells
  static constexpr int WORDS = (L * (P * R + 1) + 31) / 32;
  static constexpr size_t bytes = (size_t)(TILE + XL + XF) * sizeof(T) + (size_t)(L + WORDS) * 4;
};

template <typename T, int N, int R, bool COH, bool ORD = false, bool PDL = false>
__device__ __forceinline__ void chunk_loop_direct(const ChunkArgs<T>& a, const KTab<T>& t,
                                                  const KTab<T>& tx, unsigned char* smem_raw,
                                                  int rhs, int ch, int q1, int step,
                                                  const OrdArgs* o = nullptr) {
  constexpr int L = N * N, P = N - 1;
  using DS = DirectSmem<T, N, R>;
  T* tile = reinterpret_cast<T*>(smem_raw);
  T* XLs = tile + DS::TILE;
  T* XF = XLs + DS::XL;
  int* Ls = reinterpret_cast<int*>(XF + DS::XF);
  uint32_t* Bs = reinterpret_cast<uint32_t*>(Ls + L);
  const int tid = threadIdx.x;
  const int c = tid / L, tl = tid - c * L;
  const int j0 = tl % N, j1 = tl / N;
  if (tid < L && tid % N <= tid / N)
    XLineOp<T, N>(tx, tid % N, tid / N)
        .store(XLs + XLineOp<T, N>::slot(tid % N, tid / N) * XLineOp<T, N>::kPacked);
  const XLineShared<T, N> xop{XLs + XLineOp<T, N>::slot(tl % N, tl / N) *
                                         XLineOp<T, N>::kPacked};
  const T* __restrict__ xr = a.x + rhs * a.ldx;
  const T* fo = a.face_out + rhs * a.ld_face;
  T* ycb = a.ycol + rhs * a.ld_ycol;
  T* yb = a.y + rhs * a.ldx;
  if constexpr (ORD) {
    if (tid == 0) s_ord_next = (int)atomicAdd(o->tickets, 1u);
    __syncthreads();
    ch = ord_chunk(*o, s_ord_next);
  }
  while (ORD ? ch >= 0 : ch < q1) {
    const int first = __ldg(a.chunk_first + ch);
    const int nc = __ldg(a.chunk_first + ch + 1) - first;
    const int S = P * nc + 1;
    int target = 0, peek = 0;
    if constexpr (ORD) {
      target = __ldcg(o->done + ch) + 1;
      peek = ord_peek(*o, ch, target);
    }
    for (int i = tid; i < L; i += blockDim.x) Ls[i] = __ldg(a.lines + (size_t)first * L + i);
    {
      const uint32_t* bits = (ORD ? o->add_bits : a.run_bits) + (size_t)ch * a.bit_words;
      for (int i = tid; i < (L * S + 31) / 32; i += blockDim.x) Bs[i] = __ldg(bits + i);
    }
    // the next ticket, taken now and published before the last barrier
    unsigned tk2 = 0u;
    if constexpr (ORD) {
      if (tid == 0) tk2 = atomicAdd(o->tickets, 1u);
    }
    __syncthreads();                          // Ls, Bs; the x-line operators (first chunk)
    const bool act = c < nc;
    T out[N];
    cell_fd_3d_l<T, N>(
        t, [&](int j) { return __ldg(xr + Ls[j1 + N * j] + P * c + j0); }, tile, c, tl, act, xop,
        out);
    if (act) {
      const int pos = first + c;
      const int fs = __ldg(a.face_start + pos), fe = __ldg(a.face_start + pos + 1);
      if (PDL && fs < fe) pdl_wait();         // the face kernel's results
      for (int f = fs; f < fe; ++f) {
        const int kind = __ldg(a.face_kind + f);
        fold_face_z<T, N, COH>(t, fo + (size_t)f * 2 * L, kind & 3, kind >> 2, j0, j1, out);
      }
      if (j0 == P && c < nc - 1) {
#pragma unroll
        for (int m = 0; m < N; ++m) XF[c * L + j1 + N * m] = out[m];
      }
    }
    __syncthreads();
    if constexpr (ORD) ord_wait(*o, ch, target, peek);
    if (act && !(j0 == P && c < nc - 1)) {
      if (j0 == 0 && c > 0) {
#pragma unroll
        for (int m = 0; m < N; ++m) out[m] = add_rn(XF[(c - 1) * L + j1 + N * m], out[m]);
      }
      if constexpr (ORD) {       // the earlier colours' partial sums, loaded together
        T old[N];
#pragma unroll
        for (int m = 0; m < N; ++m) {
          const int e = (j1 + N * m) * S + P * c + j0;
          old[m] = ((Bs[e >> 5] >> (e & 31)) & 1u) ? __ldcg(yb + Ls[j1 + N * m] + P * c + j0)
                                                   : T(0);
        }
#pragma unroll
        for (int m = 0; m < N; ++m) {
          const int e = (j1 + N * m) * S + P * c + j0;
          yb[(int64_t)Ls[j1 + N * m] + P * c + j0] =
              ((Bs[e >> 5] >> (e & 31)) & 1u) ? old[m] + out[m] : out[m];
        }
      } else {
        T* yc = ycb + (size_t)__ldg(a.chunk_col + ch) * a.n_dofs;
#pragma unroll
        for (int m = 0; m < N; ++m) {
          const int l = j1 + N * m, e = l * S + P * c + j0;
          const bool bit = (Bs[e >> 5] >> (e & 31)) & 1u;
          (bit ? yc : yb)[(int64_t)Ls[l] + P * c + j0] = out[m];
        }
      }
    }
    if constexpr (ORD) {
      if (tid == 0) s_ord_next = (int)tk2;
    }
    __syncthreads();                          // Ls, Bs, XF and the tile are reused
    if constexpr (ORD) {
      if (tid == 0) st_release_gpu(o->done + ch, target);
      ch = ord_chunk(*o, s_ord_next);
    } else {
      ch += step;
    }
  }
  if constexpr (ORD) ord_exit(*o);
}

}  // namespace sbm
