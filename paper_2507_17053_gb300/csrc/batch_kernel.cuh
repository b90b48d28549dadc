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
#include "tc_common.cuh"

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
// chunk, 1: R/2, 3: R cells without staged runs, 3D FP32), tensor-core
// faces (0: CUDA cores, 1: TF32 tcgen05), face batch (0: 256/L faces per
// pass, 1: 128/L), extension
__host__ __device__ constexpr int code_of(int d, int n, int v, int fh, int ext, int tc = 0) {
  return ((d * 10 + n) * 10 + v) * 100 + tc * 10 + fh * 2 + ext;
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

// tile shape 3 (3D FP32): the same chunks without staged runs
template <typename T, int N, int R>
__device__ SBM_BK_ITEM void direct_item(const Prob<T>& P, const KTab<T>& tu, const Item& it,
                                         int rhs) {
  chunk_loop_direct<T, N, R, true>(P.ca, tu, *P.kt, bk_smem, rhs, it.b, it.e, 1);
}

template <typename T>
__device__ SBM_BK_ITEM void asm_item(const Prob<T>& P, const Item& it, int rhs) {
  const T* ycol = P.ca.ycol + rhs * P.ld_asm_ycol;
  T* y = P.ca.y + rhs * P.ca.ldx;
  for (int64_t t0 = it.b; t0 < it.e; t0 += 2 * kThreads)
    assemble_pair<T, true>(ycol, P.multi, P.mask, y, P.ca.n_dofs, it.e, P.ncol,
                           t0 + threadIdx.x, kThreads);
}

// ---- tensor-core face items (FP32 applies, 3D) ---------------------------------
//
// The face's shifted point evaluation with its first contraction on the
// tensor cores, as in tc_face.cu: T[q][l] = sum_j0 phi_j0(xi_q0) u[j0][l] is
// one tcgen05.mma (TF32, M = 128 points, N = 64 x-lines, K = 8, FP32
// accumulator in the block's 64 tensor-memory columns) per face, issued by
// one thread while the others compute the normal-derivative trace; the two
// warps that own TMEM lanes 0..63 read T back 16 columns at a time and
// finish the point evaluation; the integrands and the transposed
// interpolation run on the CUDA cores.  The MMA's completion wait is bounded:
// on expiry SBM_ERR_TIMEOUT, and the item reports failure.  A separate
// function, so that its registers do not weigh on the other paths.
struct TcState {
  uint32_t tmem;     // the block's accumulator columns
  uint32_t mbar;     // shared address of the MMA completion barrier
  uint32_t phase;    // parity of the next completion
};

// shared-memory bytes of a tensor-core face item (operands on 1024-byte
// boundaries, the tile, six arrays of L values)
template <int N>
constexpr size_t tc_item_smem() {
  return 1024 + tc::kM / 8 * tc::kGroupBytes + tc::kN / 8 * tc::kGroupBytes +
         (size_t)(N * N * N + 6 * N * N) * sizeof(float);
}

#ifdef SBM_BK_TC_INLINE
#define SBM_BK_TC_ITEM __forceinline__
#else
#define SBM_BK_TC_ITEM __noinline__
#endif
template <int N>
__device__ SBM_BK_TC_ITEM bool tc_face_item(const Prob<float>& P, const KTab<float>& t,
                                         const Item& it, int rhs, TcState& ts, int* err,
                                         int* s_flag) {
  constexpr int D = 3, L = N * N, ND = L * N, ES = 4;
  const KTab<float>& tsc = *P.kt;
  const uint32_t sbase = smem_u32(bk_smem);
  unsigned char* opA = bk_smem + (((sbase + 1023u) & ~1023u) - sbase);
  unsigned char* opB = opA + tc::kM / 8 * tc::kGroupBytes;
  float* X = reinterpret_cast<float*>(opB + tc::kN / 8 * tc::kGroupBytes);
  float* Td = X + ND;
  float* Da = Td + L;
  float* val = Da + L;
  float* grd = val + L;
  float* Va = grd + L;
  float* Ga = Va + L;
  const int tid = threadIdx.x, warp = tid / 32;
  // padding rows and columns of both operands stay zero for the whole item
  for (int i = tid; i < (tc::kM + tc::kN) / 8 * tc::kGroupBytes / 4; i += kThreads)
    reinterpret_cast<uint32_t*>(opA)[i] = 0u;
  __syncthreads();
  const uint32_t idesc = tc_instr_desc(2, tc::kM, tc::kN);
  const uint64_t adesc = tc_smem_desc(smem_u32(opA), tc::kLBO, tc::kSBO);
  const uint64_t bdesc = tc_smem_desc(smem_u32(opB), tc::kLBO, tc::kSBO);
  const float* xr = P.fa.x + rhs * P.fa.ldx;
  float* outr = P.fa.out + rhs * P.fa.ld_out;
  const int tl = tid;
  const bool act = tl < L;
  for (int f = it.b; f < it.e; ++f) {
    const int cell = __ldg(P.fa.face_cell + f);
    const int kind = __ldg(P.fa.face_kind + f);
    const int k = kind & 3, s = kind >> 2;
    // the tile and the operands: B[l][j0] = u[j0][l], A[q][j0] = phi_j0(xi_q0)
    for (int r = tid; r < ND; r += kThreads) {
      const float v = __ldg(xr + __ldg(P.fa.lines + (size_t)cell * L + r / N) + (r % N));
      X[r] = v;
      *reinterpret_cast<uint32_t*>(opB + tc::opnd_offset(r / N, r % N, ES)) = to_tf32(v);
    }
    for (int r = tid; r < L * N; r += kThreads) {
      const int q = r / N, j0 = r % N;
      *reinterpret_cast<uint32_t*>(opA + tc::opnd_offset(q, j0, ES)) =
          to_tf32(__ldg(P.fa.face_phi + ((size_t)f * L + q) * D * N + j0));
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (tid == 0) {
      asm volatile(
          "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
          "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(ts.tmem),
          "l"(adesc), "l"(bdesc), "r"(idesc), "r"(0));
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              ts.mbar)
          : "memory");
    }
    // meanwhile: normal-derivative trace and its tangential interpolation
    const int sk = (k == 0) ? 1 : (k == 1 ? N : N * N);
    const int sa = (k == 0) ? N : 1;
    const int sb = (k == 2) ? N : N * N;
    const int bt = act ? (tl % N) * sa + (tl / N) * sb : 0;
    if (act) {
      float dsum = 0.f;
#pragma unroll
      for (int j = 0; j < N; ++j) dsum = fmaf(s ? t.D1[j] : t.D0[j], X[j * sk + bt], dsum);
      Td[tl] = dsum;
    }
    __syncthreads();
    if (act) {
      const int qa = tl % N, jb = tl / N;
      float dv = 0.f;
#pragma unroll
      for (int j = 0; j < N; ++j) dv = fmaf(t.S[qa][j], Td[j + N * jb], dv);
      Da[tl] = dv;
    }
    if (tid == 0) {       // the MMA's completion (bounded wait)
      uint32_t ok = 0;
      for (long long w = 0; w < tc::kWaitLimit && !ok; ++w)
        asm volatile(
            "{\n\t.reg .pred P1;\n\tmbarrier.try_wait.parity.shared::cta.b64 P1, [%1], %2;\n\t"
            "selp.b32 %0, 1, 0, P1;\n\t}\n"
            : "=r"(ok)
            : "r"(ts.mbar), "r"(ts.phase)
            : "memory");
      if (!ok) atomicExch(err, SBM_ERR_TIMEOUT);
      *s_flag = ok;
    }
    ts.phase ^= 1u;
    __syncthreads();
    if (!*s_flag) return false;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    float dg = 0.f;
    if (act) {
      const int qa = tl % N, qb = tl / N;
#pragma unroll
      for (int j = 0; j < N; ++j) dg = fmaf(t.S[qb][j], Da[qa + N * j], dg);
    }
    if (warp < 2) {
      // row q = tl of T, 16 columns (x-lines l = j1 + n j2) at a time
      const float* pq = P.fa.face_phi + ((size_t)f * L + (act ? tl : 0)) * D * N;
      float s1[N];
#pragma unroll
      for (int j = 0; j < N; ++j) s1[j] = 0.f;
#pragma unroll
      for (int c0 = 0; c0 < tc::kN; c0 += 16) {
        uint32_t r[16];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, "
            "%10, %11, %12, %13, %14, %15}, [%16];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
              "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),
              "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
            : "r"(ts.tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (act) {
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            const int c = c0 + i;
            if (c < L) s1[c / N] = fmaf(__ldg(pq + N + c % N), __uint_as_float(r[i]), s1[c / N]);
          }
        }
      }
      if (act) {
        float e = 0.f;
#pragma unroll
        for (int j2 = 0; j2 < N; ++j2) e = fmaf(__ldg(pq + 2 * N + j2), s1[j2], e);
        const float sg = s ? 1.f : -1.f;
        const float W = tsc.W[tl];
        val[tl] = W * (tsc.sigma * e - sg * tsc.h_inv * dg);
        grd[tl] = -W * e * sg * tsc.h_inv;
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (act) {        // transposed interpolation back to the tangential nodes
      const int ja = tl % N, qb = tl / N;
      float v1 = 0.f, v2 = 0.f;
#pragma unroll
      for (int q = 0; q < N; ++q) {
        v1 = fmaf(t.S[q][ja], val[q + N * qb], v1);
        v2 = fmaf(t.S[q][ja], grd[q + N * qb], v2);
      }
      Va[tl] = v1;
      Ga[tl] = v2;
    }
    __syncthreads();
    if (act) {
      const int ja = tl % N, jb = tl / N;
      float rv = 0.f, rg = 0.f;
#pragma unroll
      for (int q = 0; q < N; ++q) {
        rv = fmaf(t.S[q][jb], Va[ja + N * q], rv);
        rg = fmaf(t.S[q][jb], Ga[ja + N * q], rg);
      }
      outr[(size_t)f * 2 * L + tl] = rv;
      outr[(size_t)f * 2 * L + L + tl] = rg;
    }
    __syncthreads();      // the next face rewrites the operands and the accumulator
  }
  return true;
}

// One (dimension, degree) combination: its face and chunk variants.
template <typename T, bool TC, int D, int N>
__device__ __forceinline__ bool run_dn(const Prob<T>& P, const KTab<T>& tu, const Item& it,
                                       int kind, int rhs, int code, TcState& ts, int* err,
                                       int* s_flag) {
  constexpr int L = Shape<D, N>::L;
  constexpr int R = (256 / L) > 0 ? (256 / L) : 1;
  constexpr int RH = (R / 2) > 0 ? R / 2 : 1;
  constexpr int FF = kThreads / L;                    // faces per pass, full block
  constexpr int FHALF = (FF / 2) > 0 ? FF / 2 : 1;
  const int v = (code / 100) % 10, tc = (code / 10) % 10, fh = (code % 10) / 2, ext = code % 2;
  if (kind == kFace) {
    if constexpr (TC && std::is_same<T, float>::value && D == 3) {
      if (tc) return tc_face_item<N>(P, tu, it, rhs, ts, err, s_flag);
    }
    if (ext) face_item<T, D, N, 1, FF>(P, tu, it, rhs);
    else if (fh) face_item<T, D, N, 0, FHALF>(P, tu, it, rhs);
    else face_item<T, D, N, 0, FF>(P, tu, it, rhs);
  } else {
    if constexpr (D == 3 && std::is_same<T, float>::value) {
      if (v == 3) {
        direct_item<T, N, R>(P, tu, it, rhs);
        return true;
      }
    }
    if (v == 1) chunk_item<T, D, N, RH>(P, tu, it, rhs);
    else chunk_item<T, D, N, R>(P, tu, it, rhs);
  }
  return true;
}

// Shared-memory bytes a problem's items need (host side, for the launch).
template <typename T, int D, int N>
size_t smem_dn(int v, int fh, int ext, int tc) {
  constexpr int L = Shape<D, N>::L;
  constexpr int R = (256 / L) > 0 ? (256 / L) : 1;
  constexpr int RH = (R / 2) > 0 ? R / 2 : 1;
  constexpr int FF = kThreads / L;
  constexpr int FHALF = (FF / 2) > 0 ? FF / 2 : 1;
  size_t c = v == 1 ? ChunkSmem<T, D, N, RH>::bytes : ChunkSmem<T, D, N, R>::bytes;
  if constexpr (D == 3) {
    if (v == 3) c = DirectSmem<T, N, R>::bytes;
  }
  const size_t f = ext ? face_group_smem<T, D, N, 1, FF>()
                       : (fh ? face_group_smem<T, D, N, 0, FHALF>()
                             : face_group_smem<T, D, N, 0, FF>());
  const size_t g = tc ? tc_item_smem<N>() : 0;
  return std::max(std::max(c, f), g);
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

// TC: the variant with the tensor-core face items (FP32).  It is a separate
// instantiation: on GB300 a kernel that merely contains tcgen05 instructions
// ran every other path about 3x slower (64 x 8 batch, FP32 5.9 -> 19.4 ms,
// FP64 32.6 -> 49.3 ms, tensor-core items never executed), so the variant
// without them has none.
template <typename T, typename U, bool TC>
__global__ void __launch_bounds__(kThreads, min_blocks<T>())
batch_kernel(const __grid_constant__ ProbTable<T> tab, const Item* __restrict__ items, int nitems,
             int nsys, int nrhs, int* __restrict__ cnt, int* __restrict__ err, int tc_cols) {
  __shared__ int s_ticket, s_flag;
  __shared__ __align__(8) uint64_t s_mbar;
  __shared__ uint32_t s_tmem;
  TcState ts{0u, 0u, 0u};
  if constexpr (TC) {         // tensor memory and the MMA barrier for tensor-core face items
    if (threadIdx.x == 0) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&s_mbar)));
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (threadIdx.x < 32) {
      asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                       smem_u32(&s_tmem)),
                   "r"(tc_cols));
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    ts.tmem = s_tmem;
    ts.mbar = smem_u32(&s_mbar);
  }
  for (;;) {
    __syncthreads();              // the previous item is done with shared memory and s_ticket
    if (threadIdx.x == 0) s_ticket = atomicAdd(cnt, 1);
    __syncthreads();
    const int ti = s_ticket;
    if (ti >= nitems) break;
    const Item it = items[ti];
    const Prob<T>& P = tab.p[it.prob];
    const int kind = it.kr & 3, rhs = it.kr >> 2;
    int* fdone = cnt + 1 + it.prob * nrhs + rhs;
    int* cdone = fdone + nsys;
    if (kind == kAsm) {
      if (!wait_count(cdone, P.n_chunk_items, err, &s_flag)) break;
      asm_item<T>(P, it, rhs);
      continue;
    }
    if (kind == kChunk && !wait_count(fdone, P.n_face_items, err, &s_flag)) break;
    const int code = P.code;
    bool ok = true;
    switch (code / 1000) {
#define SBM_DN(DD, NN)                                                                    \
  case DD * 10 + NN:                                                                      \
    ok = run_dn<T, TC, DD, NN>(P, U::template tab<NN>(), it, kind, rhs, code, ts, err,    \
                               &s_flag);                                                  \
    break;
      SBM_DN(2, 2) SBM_DN(2, 3) SBM_DN(2, 4) SBM_DN(2, 5) SBM_DN(2, 6) SBM_DN(2, 7)
      SBM_DN(3, 2) SBM_DN(3, 3) SBM_DN(3, 4) SBM_DN(3, 5) SBM_DN(3, 6) SBM_DN(3, 7)
#undef SBM_DN
      default: break;
    }
    if (!ok) break;               // a bounded wait expired (recorded in err)
    signal_done(kind == kFace ? fdone : cdone);
  }
  if constexpr (TC) {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (threadIdx.x < 32)
      asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(ts.tmem),
                   "r"(tc_cols));
  }
}

// Host side of one precision: launch attributes and the launch.
template <typename T, typename U>
struct Launcher {
  static size_t smem(int d, int n, int v, int fh, int ext, int tc) {
#define SBM_DN(DD, NN) \
  if (d == DD && n == NN) return smem_dn<T, DD, NN>(v, fh, ext, tc);
    SBM_DN(2, 2) SBM_DN(2, 3) SBM_DN(2, 4) SBM_DN(2, 5) SBM_DN(2, 6) SBM_DN(2, 7)
    SBM_DN(3, 2) SBM_DN(3, 3) SBM_DN(3, 4) SBM_DN(3, 5) SBM_DN(3, 6) SBM_DN(3, 7)
#undef SBM_DN
    return 0;
  }
  // resident blocks per SM for this dynamic shared memory size (tc: the
  // variant with tensor-core face items)
  template <bool TC>
  static cudaError_t occ(size_t smem_bytes, int* per_sm) {
    cudaError_t e = cudaFuncSetAttribute(batch_kernel<T, U, TC>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem_bytes);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, batch_kernel<T, U, TC>,
                                                         kThreads, smem_bytes);
  }
  static cudaError_t occupancy(size_t smem_bytes, bool tc, int* per_sm) {
    if constexpr (std::is_same<T, float>::value)
      if (tc) return occ<true>(smem_bytes, per_sm);
    return occ<false>(smem_bytes, per_sm);
  }
  static cudaError_t launch(const ProbTable<T>& tab, const Item* items, int nitems, int nsys,
                            int nrhs, int* cnt, int* err, size_t smem_bytes, int grid,
                            int tc_cols, cudaStream_t st) {
    if constexpr (std::is_same<T, float>::value) {
      if (tc_cols) {
        batch_kernel<T, U, true><<<grid, kThreads, smem_bytes, st>>>(tab, items, nitems, nsys,
                                                                     nrhs, cnt, err, tc_cols);
        return cudaGetLastError();
      }
    }
    batch_kernel<T, U, false><<<grid, kThreads, smem_bytes, st>>>(tab, items, nitems, nsys, nrhs,
                                                                  cnt, err, 0);
    return cudaGetLastError();
  }
};

}  // namespace bk
}  // namespace sbm
