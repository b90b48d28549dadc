// Surrogate-boundary faces with the shifted point evaluation on the 5th-
// generation tensor cores (tcgen05), for the FP32 apply in TF32 or BF16 mode.
//
// The O((p+1)^(2d-1)) step of Algorithm 3 is, per face, the contraction
//   T[q][l] = sum_{j0} phi_{j0}(xi_{q,0}) u[j0][l]       (q: face point, l: x-line)
// followed by per-point weighted sums over the remaining axes.  The first
// contraction is a dense (points x n) . (n x lines) product: one
//   tcgen05.mma.cta_group::1.kind::{tf32, f16}  M = 128, N = 64, K = 8 | 16
// per face (points padded to 128 rows, the (p+1)^2 x-lines to 64 columns, the
// x-direction to K), both operands in shared memory in the canonical
// K-major, no-swizzle core-matrix layout (8 rows x 16 bytes per core matrix;
// core matrices adjacent in K 128 bytes apart, 8-row groups 256 bytes apart),
// the FP32 accumulator in tensor memory (row q = TMEM lane q, column l), read
// back by the two warps that own lanes 0..63 with tcgen05.ld.  Everything
// else (normal-derivative trace, the remaining two contractions, the
// integrands, the transposed interpolation) runs on the CUDA cores in FP32,
// exactly as in face_kernel.cu, and the output has the same format.
//
// Waits on the MMA's mbarrier are bounded: on expiry the kernel records
// SBM_ERR_TIMEOUT in the problem's device error word, stops, frees its tensor
// memory and returns.
#include <algorithm>

#include "sweeps.cuh"
#include "tc_common.cuh"

namespace sbm {

template <typename T>
struct TcArgs {
  const float* __restrict__ x;
  const int32_t* __restrict__ lines;       // CG gather (null for DG)
  const int32_t* __restrict__ cell_rank;   // DG gather
  const int32_t* __restrict__ face_cell;
  const int32_t* __restrict__ face_kind;
  const float* __restrict__ face_phi;      // [F][L][3][N] FP32
  float* __restrict__ out;                 // [F][2L]
  int* __restrict__ err;                   // device error word
  int nface;
  int dg;
};

// KIND: 0 = TF32 (K = 8), 1 = BF16 (K = 16)
template <int KIND, int N>
__global__ void __launch_bounds__(tc::kThreads)
tc_face_kernel(const TcArgs<float> a, const __grid_constant__ KTab<float> t) {
  constexpr int D = 3, L = N * N, ND = L * N;
  constexpr int KMMA = KIND == 0 ? 8 : 16;
  constexpr int ES = KIND == 0 ? 4 : 2;
  __shared__ __align__(1024) unsigned char opA[tc::kM / 8 * tc::kGroupBytes];   // 4 KB
  __shared__ __align__(1024) unsigned char opB[tc::kN / 8 * tc::kGroupBytes];   // 2 KB
  __shared__ float X[ND];
  __shared__ float Td[L], Da[L], val[L], grd[L], Va[L], Ga[L];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;

  // zero both operands once (padding rows/columns stay zero), set up the
  // mbarrier, allocate tensor memory (warp 0)
  for (int i = tid; i < (int)sizeof(opA) / 4; i += tc::kThreads) ((uint32_t*)opA)[i] = 0u;
  for (int i = tid; i < (int)sizeof(opB) / 4; i += tc::kThreads) ((uint32_t*)opB)[i] = 0u;
  if (tid == 0) {
    abort_flag = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_base)),
                 "r"(tc::kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  const uint32_t idesc = tc_instr_desc(KIND == 0 ? 2 : 1, tc::kM, tc::kN);
  const uint64_t adesc = tc_smem_desc(smem_u32(opA), tc::kLBO, tc::kSBO);
  const uint64_t bdesc = tc_smem_desc(smem_u32(opB), tc::kLBO, tc::kSBO);
  uint32_t phase = 0;

  for (int f = blockIdx.x; f < a.nface; f += gridDim.x) {
    const int cell = __ldg(a.face_cell + f);
    const int kind = __ldg(a.face_kind + f);
    const int k = kind & 3, s = kind >> 2;
    // tile, and the MMA operands: B[l][j0] = u[j0][l], A[q][j0] = phi_{j0}(xi_{q,0})
    for (int r = tid; r < ND; r += tc::kThreads) {
      size_t g;
      if (a.dg) g = (size_t)__ldg(a.cell_rank + cell) * ND + r;
      else g = (size_t)__ldg(a.lines + (size_t)cell * L + r / N) + (r % N);
      const float v = __ldg(a.x + g);
      X[r] = v;
      const int l = r / N, j0 = r % N;
      if (KIND == 0) *(uint32_t*)(opB + tc::opnd_offset(l, j0, ES)) = to_tf32(v);
      else *(uint16_t*)(opB + tc::opnd_offset(l, j0, ES)) = to_bf16(v);
    }
    for (int r = tid; r < L * N; r += tc::kThreads) {
      const int q = r / N, j0 = r % N;
      const float v = __ldg(a.face_phi + ((size_t)f * L + q) * D * N + j0);
      if (KIND == 0) *(uint32_t*)(opA + tc::opnd_offset(q, j0, ES)) = to_tf32(v);
      else *(uint16_t*)(opA + tc::opnd_offset(q, j0, ES)) = to_bf16(v);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (tid == 0) {
      // D = A . B (enable-input-d false: no accumulation into old contents)
      if constexpr (KIND == 0)
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(0));
      else
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(0));
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              smem_u32(&mbar))
          : "memory");
    }
    // meanwhile on the CUDA cores: normal-derivative trace at the tangential
    // nodes and its interpolation to the tangential Gauss points
    int sk, sa, sb;
    sk = (k == 0) ? 1 : (k == 1 ? N : N * N);
    sa = (k == 0) ? N : 1;
    sb = (k == 2) ? N : N * N;
    const int tl = tid;
    const bool act = tl < L;
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
    // wait for the MMA (bounded)
    {
      uint32_t ok = 0;
      for (long long it = 0; it < tc::kWaitLimit && !ok; ++it) {
        asm volatile(
            "{\n\t.reg .pred P1;\n\tmbarrier.try_wait.parity.shared::cta.b64 P1, [%1], %2;\n\t"
            "selp.b32 %0, 1, 0, P1;\n\t}\n"
            : "=r"(ok)
            : "r"(smem_u32(&mbar)), "r"(phase)
            : "memory");
      }
      if (!ok) {
        abort_flag = 1;
        if (tid == 0) atomicExch(a.err, SBM_ERR_TIMEOUT);
      }
    }
    phase ^= 1u;
    __syncthreads();
    if (abort_flag) break;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    float dg = 0.f;
    if (act) {
      const int qa = tl % N, qb = tl / N;
#pragma unroll
      for (int j = 0; j < N; ++j) dg = fmaf(t.S[qb][j], Da[qa + N * j], dg);
    }
    // the two warps that own TMEM lanes 0..63 read their rows of T and finish
    // the point evaluation for their point q = tid
    if (warp < 2) {
      float Tq[tc::kN];
#pragma unroll
      for (int c0 = 0; c0 < tc::kN; c0 += 16) {
        uint32_t r[16];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, "
            "%10, %11, %12, %13, %14, %15}, [%16];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
              "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),
              "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
            : "r"(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int i = 0; i < 16; ++i) Tq[c0 + i] = __uint_as_float(r[i]);
      }
      if (act) {
        const float* pq = a.face_phi + ((size_t)f * L + tl) * D * N;
        float e = 0.f;
#pragma unroll
        for (int j2 = 0; j2 < N; ++j2) {
          float s1 = 0.f;
#pragma unroll
          for (int j1 = 0; j1 < N; ++j1) s1 = fmaf(__ldg(pq + N + j1), Tq[j1 + N * j2], s1);
          e = fmaf(__ldg(pq + 2 * N + j2), s1, e);
        }
        const float sg = s ? 1.f : -1.f;
        const float W = t.W[tl];
        val[tl] = W * (t.sigma * e - sg * t.h_inv * dg);
        grd[tl] = -W * e * sg * t.h_inv;
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    // transposed interpolation back to the tangential nodes
    if (act) {
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
      a.out[(size_t)f * 2 * L + tl] = rv;
      a.out[(size_t)f * 2 * L + L + tl] = rg;
    }
    // the next face overwrites the operands and the accumulator: everyone is
    // past its reads (operands were consumed: the mbarrier completed)
    __syncthreads();
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(tc::kTmemCols));
}

// Diagnostic: wait (bounded, `limit` polls) on an mbarrier that nothing ever
// arrives on, so the wait expires and the device error word gets
// SBM_ERR_TIMEOUT -- the same path the tensor-core kernel takes when an MMA
// never completes.  Exercises failure detection without faulting the GPU.
__global__ void timeout_selftest_kernel(int* err, long long limit) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar)));
    uint32_t ok = 0;
    for (long long it = 0; it < limit && !ok; ++it)
      asm volatile(
          "{\n\t.reg .pred P1;\n\tmbarrier.try_wait.parity.shared::cta.b64 P1, [%1], %2;\n\t"
          "selp.b32 %0, 1, 0, P1;\n\t}\n"
          : "=r"(ok)
          : "r"(smem_u32(&bar)), "r"(0u)
          : "memory");
    if (!ok) atomicExch(err, SBM_ERR_TIMEOUT);
  }
}

cudaError_t launch_timeout_selftest(int* err, cudaStream_t st) {
  timeout_selftest_kernel<<<1, 32, 0, st>>>(err, 1ll << 14);
  return cudaGetLastError();
}

template <int KIND, int N>
static cudaError_t tc_t(const HostProblem& hp, const DeviceData& dd, const float* x, float* out,
                        cudaStream_t st) {
  if (dd.nface == 0) return cudaSuccess;
  const KTab<float> t = make_ktab<float>(hp);
  TcArgs<float> a;
  a.x = x;
  a.lines = dd.lines;
  a.cell_rank = dd.cell_rank;
  a.face_cell = dd.face_cell;
  a.face_kind = dd.face_kind;
  a.face_phi = dd.face_phi32;
  a.out = out;
  a.err = dd.err_flag;
  a.nface = dd.nface;
  a.dg = hp.desc.dg;
  int sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = std::min(dd.nface, 4 * sms);   // at most 4 x 64 of 512 TMEM columns per SM
  tc_face_kernel<KIND, N><<<grid, tc::kThreads, 0, st>>>(a, t);
  return cudaGetLastError();
}

cudaError_t launch_tc_face_kernel(const HostProblem& hp, const DeviceData& dd, const float* x,
                                  float* out, int face_mode, cudaStream_t st) {
  if (hp.d != 3) return cudaErrorInvalidValue;
  const int kind = (face_mode == SBM_FACE_TF32) ? 0 : 1;
#define SBM_CASE(NN)                                                  \
  if (hp.n == NN)                                                     \
    return kind == 0 ? tc_t<0, NN>(hp, dd, x, out, st) : tc_t<1, NN>(hp, dd, x, out, st);
  SBM_CASE(2) SBM_CASE(3) SBM_CASE(4) SBM_CASE(5) SBM_CASE(6) SBM_CASE(7)
#undef SBM_CASE
  return cudaErrorInvalidValue;
}

}  // namespace sbm
