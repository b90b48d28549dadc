// The persistent batched apply in FP64: the kernel instantiation,
// its constant-memory unit tables and the host entry points (batch_kernel.cuh).
#include "batch.hpp"
#include "batch_kernel.cuh"

namespace sbm {
namespace bk {

// h-independent 1D tables of degree n - 1 at index n
__constant__ KTab<double> c_unit_f64[kMaxN + 1];

struct U_f64 {
  template <int N>
  __device__ __forceinline__ static const KTab<double>& tab() {
    return c_unit_f64[N];
  }
};

using L_f64 = Launcher<double, U_f64>;

cudaError_t set_unit_table(int n, const KTab<double>& t) {
  return cudaMemcpyToSymbol(c_unit_f64, &t, sizeof(t), (size_t)n * sizeof(t));
}
size_t item_smem_f64(int d, int n, int v, int fh, int ext, int tc) {
  return L_f64::smem(d, n, v, fh, ext, tc);
}
cudaError_t occupancy_f64(size_t smem, bool tc, int* per_sm) {
  return L_f64::occupancy(smem, tc, per_sm);
}
cudaError_t launch(const ProbTable<double>& tab, const Item* items, int nitems, int nsys, int nrhs,
                   int* cnt, int* err, size_t smem, int grid, int tc_cols, cudaStream_t st) {
  return L_f64::launch(tab, items, nitems, nsys, nrhs, cnt, err, smem, grid, tc_cols, st);
}

}  // namespace bk
}  // namespace sbm
