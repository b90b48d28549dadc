// tcgen05 building blocks shared by the tensor-core surrogate-face kernel
// (tc_face.cu) and the persistent batched apply (batch_kernel.cuh): the
// operand layout in shared memory, the shared-memory and instruction
// descriptors, TF32 / BF16 rounding.
#pragma once

#include <cstdint>

namespace sbm {

namespace tc {

constexpr int kThreads = 128;
constexpr int kM = 128;          // MMA rows (face points, padded)
constexpr int kN = 64;           // MMA columns (x-lines of the tile, padded)
constexpr int kTmemCols = 64;    // FP32 accumulator columns
constexpr int kRowBytes = 32;    // one operand row: 8 tf32 or 16 bf16
constexpr int kGroupBytes = 256; // 8 rows x 32 bytes
constexpr uint32_t kLBO = 128;   // K-adjacent core matrices
constexpr uint32_t kSBO = 256;   // M/N-adjacent core matrices (8-row groups)
constexpr long long kWaitLimit = 1ll << 26;

// byte offset of element k of operand row r (4-byte tf32 or 2-byte bf16)
__host__ __device__ constexpr uint32_t opnd_offset(int r, int k, int esize) {
  return (uint32_t)((r / 8) * kGroupBytes + ((k * esize) / 16) * kLBO + (r % 8) * 16 +
                    (k * esize) % 16);
}

}  // namespace tc

// Shared-memory matrix descriptor (tcgen05): start address, leading (K) and
// stride (M/N) byte offsets, all >> 4; bits 46..48 = 0b001; no swizzle.
__host__ __device__ constexpr uint64_t tc_smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}

// Instruction descriptor for .kind::tf32 / .kind::f16: D = F32 (bits 4-5 = 1),
// A and B format (bits 7-9, 10-12: 1 = BF16, 2 = TF32), both K-major, N >> 3
// at bits 17-22, M >> 4 at bits 24-28, dense.
__host__ __device__ constexpr uint32_t tc_instr_desc(int ab_format, int m, int n) {
  return (1u << 4) | ((uint32_t)ab_format << 7) | ((uint32_t)ab_format << 10) |
         ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint32_t to_tf32(float v) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
  return r;
}

// BF16: FP32 -> BF16 round to nearest even (finite inputs)
__device__ __forceinline__ uint16_t to_bf16(float v) {
  uint32_t u = __float_as_uint(v);
  u += 0x7FFFu + ((u >> 16) & 1u);
  return (uint16_t)(u >> 16);
}

}  // namespace sbm
