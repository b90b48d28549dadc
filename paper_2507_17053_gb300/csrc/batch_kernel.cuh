// The persistent batched apply: every problem, right-hand side and phase of
// a batch of continuous Galerkin problems in ONE kernel launch.
//
// Work list.  The host cuts each system (problem k, right-hand side r) into
// items: surrogate-face items (a range of faces, Algorithm 3), chunk items
// (a range of cell chunks: gather, cell term of Algorithm 1, face folds,
// single-writer stores) and assembly items (a range of the DoFs several
// colours share).  Items are sized and ordered by the paper's load-balancing
// weights (Section 3.5: 10 per cell, plus 40 per surrogate face in 3D, 20 in
// 2D), scaled across degrees by the per-cell sum-factorisation cost
// (p+1)^(d+1): all face items first, then all chunk items, then all assembly
// items, each group heaviest first.
//
// Scheduling.  Blocks stay resident and take the next item from a global
// ticket counter (atomicAdd).  A chunk item needs every face item of its
// system done (it folds their results), an assembly item every chunk item:
// per-system counters, incremented after an item (block barrier, fence,
// atomic add) and polled by the consumer before it starts.  Every dependency
// points to a smaller ticket, whose block is already running and never waits
// on a later one, so the schedule cannot deadlock; still, every poll is
// bounded: on expiry the block records SBM_ERR_TIMEOUT in the batch's error
// word and returns.  Data written by other blocks of the launch (face
// results, colour buffers) is read at the L2 (ld.global.cg).
//
// Tables.  The h-independent 1D tables of degree p (eigenbasis transforms,
// 1D mass and stiffness, Gauss interpolation, end-point derivatives) are one
// copy per degree in constant memory, so the inner products take them as
// constant-bank operands as in the single-problem kernels; the h-scaled
// values (x-line operators h K + mu M, face weights, sigma, 1/h) come from
// the problem's own table in global memory.  Arithmetic and summation order
// are those of the single-problem kernels: a batch apply equals the single
// applies bitwise for the same tile shape.
#pragma once

#include "chunk_body.cuh"
#include "face_body.cuh"

namespace sbm {
namespace bk {

constexpr int kThreads = 256;
enum { kFace = 0, kChunk = 1, kAsm = 2 };
constexpr long long kWaitPolls = 1ll << 21;   // bounded dependency waits (about a second)

struct Item {
  int32_t prob;
  int32_t kr;       // kind | (rhs << 2)
  int32_t b, e;     // faces / chunks / shared-DoF list entries [b, e)
};

// dispatch code of a problem: dimension, degree, tile shape (0: R cells per
// chunk, 1: R/2), face batch (0: 256/L faces per pass, 1: 128/L), extension
__host__ __device__ constexpr int code_of(int d, int n, int v, int fh, int ext) {
  return d * 1000 + n * 100 + v * 10 + fh * 2 + ext;
}

// Problems of one launch (a batch of more is split into several launches).
constexpr int kLaunchProbs = 96;

template <typename T>
struct Prob {
  ChunkArgs<T> ca;          // chunk tables of the problem's tile shape; vectors of rhs 0
  FaceArgs<T> fa;           // face tables; vectors of rhs 0
  const KTab<T>* kt;        // the problem's full table (global memory)
  const int32_t* multi;     // shared-DoF list of the tile shape, its colour masks
  const uint8_t* mask;
  int64_t ld_asm_ycol;      // colour buffers of one right-hand side
  int code;
  int ncol;
  int n_face_items, n_chunk_items;
};

// The launch's problem descriptors, passed by value as one kernel parameter
// (parameter space: every field is a constant-bank read, as in the
// single-problem kernels, not a dependent global load).
template <typename T>
struct ProbTable {
  Prob<T> p[kLaunchProbs];
};
static_assert(sizeof(ProbTable<double>) <= 31 * 1024, "kernel parameter space");

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Thread 0 polls *c until it reaches target (bounded); the block agrees on
// the outcome.  On expiry: SBM_ERR_TIMEOUT into *err, false for every thread.
__device__ __forceinline__ bool wait_count(const int* c, int target, int* err, int* s_flag) {
  if (threadIdx.x == 0) {
    int ok = 0;
    for (long long it = 0; it < kWaitPolls; ++it) {
      if (ld_acquire(c) >= target) {
        ok = 1;
        break;
      }
      __nanosleep(256);
    }
    if (!ok) atomicExch(err, SBM_ERR_TIMEOUT);
    __threadfence();
    *s_flag = ok;
  }
  __syncthreads();
  return *s_flag != 0;
}

// The block's writes of an item are done: count the item.
__device__ __forceinline__ void signal_done(int* c) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(c, 1);
  }
}

// Item functions are inlined into the kernel (its problem table stays in
// parameter space, which separately compiled functions could only reach
// through generic pointers: 11 % slower in FP32); SBM_BK_NOINLINE compiles
// them as separate functions instead.
#ifdef SBM_BK_NOINLINE
#define SBM_BK_ITEM __noinline__
#else
#define SBM_BK_ITEM __forceinline__
#endif
// the launch's dynamic shared memory, named here (not passed as a pointer)
// so that the separately compiled item functions address it as shared
// memory rather than through generic pointers
extern __shared__ __align__(16) unsigned char bk_smem[];

template <typename T, int D, int N, int EXT, int FPB>
__device__ SBM_BK_ITEM void face_item(const Prob<T>& P, const KTab<T>& tu, const Item& it,
                                       int rhs) {
  for (int f0 = it.b; f0 < it.e; f0 += FPB)
    face_group<T, D, N, EXT, FPB>(P.fa, tu, *P.kt, bk_smem, f0, it.e, rhs);
}

template <typename T, int D, int N, int R>
__device__ SBM_BK_ITEM void chunk_item(const Prob<T>& P, const KTab<T>& tu, const Item& it,
                                        int rhs) {
  chunk_xline_build<T, D, N, R>(bk_smem, *P.kt, threadIdx.x);
  chunk_loop<T, D, N, R, true, kThreads>(P.ca, tu, bk_smem, rhs, it.b, it.e, 1);
}

template <typename T>
__device__ SBM_BK_ITEM void asm_item(const Prob<T>& P, const Item& it, int rhs) {
  const T* ycol = P.ca.ycol + rhs * P.ld_asm_ycol;
  T* y = P.ca.y + rhs * P.ca.ldx;
  for (int64_t t0 = it.b; t0 < it.e; t0 += kThreads)
    assemble_warp<T, true>(ycol, P.multi, P.mask, y, P.ca.n_dofs, it.e, P.ncol,
                           t0 + threadIdx.x);
}

// One (dimension, degree) combination: its face and chunk variants.
template <typename T, int D, int N>
__device__ __forceinline__ void run_dn(const Prob<T>& P, const KTab<T>& tu, const Item& it,
                                       int kind, int rhs, int code) {
  constexpr int L = Shape<D, N>::L;
  constexpr int R = (256 / L) > 0 ? (256 / L) : 1;
  constexpr int RH = (R / 2) > 0 ? R / 2 : 1;
  constexpr int FF = kThreads / L;                    // faces per pass, full block
  constexpr int FHALF = (FF / 2) > 0 ? FF / 2 : 1;
  const int rest = code - (D * 1000 + N * 100);
  const int v = rest / 10, fh = (rest % 10) / 2, ext = rest % 2;
  if (kind == kFace) {
    if (ext) face_item<T, D, N, 1, FF>(P, tu, it, rhs);
    else if (fh) face_item<T, D, N, 0, FHALF>(P, tu, it, rhs);
    else face_item<T, D, N, 0, FF>(P, tu, it, rhs);
  } else {
    if (v) chunk_item<T, D, N, RH>(P, tu, it, rhs);
    else chunk_item<T, D, N, R>(P, tu, it, rhs);
  }
}

// Shared-memory bytes a problem's items need (host side, for the launch).
template <typename T, int D, int N>
size_t smem_dn(int v, int fh, int ext) {
  constexpr int L = Shape<D, N>::L;
  constexpr int R = (256 / L) > 0 ? (256 / L) : 1;
  constexpr int RH = (R / 2) > 0 ? R / 2 : 1;
  constexpr int FF = kThreads / L;
  constexpr int FHALF = (FF / 2) > 0 ? FF / 2 : 1;
  const size_t c = v ? ChunkSmem<T, D, N, RH>::bytes : ChunkSmem<T, D, N, R>::bytes;
  const size_t f = ext ? face_group_smem<T, D, N, 1, FF>()
                       : (fh ? face_group_smem<T, D, N, 0, FHALF>()
                             : face_group_smem<T, D, N, 0, FF>());
  return c > f ? c : f;
}


// The persistent kernel.  U::tab<N>() is the constant-memory unit table of
// degree N - 1 (one per translation unit and precision).
// Resident blocks per SM the register budget is sized for: FP64 5 (48
// registers, no spills in the item loops), FP32 6 (40; its kernels are
// latency-bound and gain from the extra warps).
#ifndef SBM_BK_F32_MINB
#define SBM_BK_F32_MINB 6
#endif
template <typename T>
constexpr int min_blocks() {
  return sizeof(T) == 4 ? SBM_BK_F32_MINB : 5;
}

template <typename T, typename U>
__global__ void __launch_bounds__(kThreads, min_blocks<T>())
batch_kernel(const __grid_constant__ ProbTable<T> tab, const Item* __restrict__ items, int nitems,
             int nsys, int nrhs, int* __restrict__ cnt, int* __restrict__ err) {
  __shared__ int s_ticket, s_flag;
  for (;;) {
    __syncthreads();              // the previous item is done with shared memory and s_ticket
    if (threadIdx.x == 0) s_ticket = atomicAdd(cnt, 1);
    __syncthreads();
    const int ti = s_ticket;
    if (ti >= nitems) return;
    const Item it = items[ti];
    const Prob<T>& P = tab.p[it.prob];
    const int kind = it.kr & 3, rhs = it.kr >> 2;
    int* fdone = cnt + 1 + it.prob * nrhs + rhs;
    int* cdone = fdone + nsys;
    if (kind == kAsm) {
      if (!wait_count(cdone, P.n_chunk_items, err, &s_flag)) return;
      asm_item<T>(P, it, rhs);
      continue;
    }
    if (kind == kChunk && !wait_count(fdone, P.n_face_items, err, &s_flag)) return;
    const int code = P.code;
    switch (code / 100) {
#define SBM_DN(DD, NN) \
  case DD * 10 + NN: run_dn<T, DD, NN>(P, U::template tab<NN>(), it, kind, rhs, code); break;
      SBM_DN(2, 2) SBM_DN(2, 3) SBM_DN(2, 4) SBM_DN(2, 5) SBM_DN(2, 6) SBM_DN(2, 7)
      SBM_DN(3, 2) SBM_DN(3, 3) SBM_DN(3, 4) SBM_DN(3, 5) SBM_DN(3, 6) SBM_DN(3, 7)
#undef SBM_DN
      default: break;
    }
    signal_done(kind == kFace ? fdone : cdone);
  }
}

// Host side of one precision: launch attributes and the launch.
template <typename T, typename U>
struct Launcher {
  static size_t smem(int d, int n, int v, int fh, int ext) {
#define SBM_DN(DD, NN) \
  if (d == DD && n == NN) return smem_dn<T, DD, NN>(v, fh, ext);
    SBM_DN(2, 2) SBM_DN(2, 3) SBM_DN(2, 4) SBM_DN(2, 5) SBM_DN(2, 6) SBM_DN(2, 7)
    SBM_DN(3, 2) SBM_DN(3, 3) SBM_DN(3, 4) SBM_DN(3, 5) SBM_DN(3, 6) SBM_DN(3, 7)
#undef SBM_DN
    return 0;
  }
  // resident blocks per SM for this dynamic shared memory size
  static cudaError_t occupancy(size_t smem_bytes, int* per_sm) {
    cudaError_t e = cudaFuncSetAttribute(batch_kernel<T, U>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem_bytes);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, batch_kernel<T, U>, kThreads,
                                                         smem_bytes);
  }
  static cudaError_t launch(const ProbTable<T>& tab, const Item* items, int nitems, int nsys,
                            int nrhs, int* cnt, int* err, size_t smem_bytes, int grid,
                            cudaStream_t st) {
    batch_kernel<T, U><<<grid, kThreads, smem_bytes, st>>>(tab, items, nitems, nsys, nrhs, cnt,
                                                           err);
    return cudaGetLastError();
  }
};

}  // namespace bk
}  // namespace sbm
