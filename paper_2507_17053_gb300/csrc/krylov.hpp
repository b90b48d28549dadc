// Krylov drivers on the matrix-free operator (implementation in krylov.cu).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <functional>
#include <vector>

#include "sbm.h"

namespace sbm {

constexpr int SBM_NOT_DONE = -1;

// y = A x on stream st (all work enqueued; no synchronisation)
template <typename T>
using ApplyFn = std::function<cudaError_t(const T* x, T* y, cudaStream_t st)>;

struct SolveInfo {
  int iters = 0;        // operator applications inside the Krylov iterations
  double relres = 0.0;  // true relative residual |b - A x| / |b| at exit (FP64 for IR)
  int restarts = 0;     // CG restarts / GMRES cycles / IR outer steps
};

struct SolveStatus {
  int status;
  cudaError_t cuda;
};

// Device scratch of one solve; released by the caller.
struct Workspace {
  std::vector<void*> bufs;
  void* host_state = nullptr;
  cudaStream_t cap = nullptr;
  cudaError_t alloc(void** p, size_t bytes);
  void release();
};

// Conjugate gradients (Jacobi-preconditioned when diag != nullptr), FP64.
SolveStatus solve_cg(const ApplyFn<double>& apply, int64_t n, const double* b, double* x,
                     const double* diag, double rtol, int maxit, cudaStream_t st, Workspace& ws,
                     SolveInfo* info);

// Restarted GMRES(restart) in precision T on x/b of precision TX.
template <typename T, typename TX>
SolveStatus solve_gmres(const ApplyFn<T>& apply, int64_t n, const TX* b, TX* x, double rtol,
                        int maxit, int restart, cudaStream_t st, Workspace& ws, SolveInfo* info,
                        const ApplyFn<TX>* apply_x);

// BiCGStab in precision T (FP64 scalars), bound to one right-hand side b and
// iterate x; setup allocates from ws and captures BI_CHUNK iterations as one
// CUDA graph, solve may run several times (e.g. as an inner solver), and
// destroy frees the graph, the capture stream and the pinned state.
template <typename T>
struct Bicgstab {
  ApplyFn<T> apply;
  int64_t n = 0;
  const T* b = nullptr;
  T* x = nullptr;
  T *r = nullptr, *rh = nullptr, *p = nullptr, *v = nullptr, *s = nullptr, *t = nullptr;
  T* xb = nullptr;   // iterate of least recursive residual so far
  double* part = nullptr;
  void* dstate = nullptr;
  void* hstate = nullptr;
  cudaStream_t cap = nullptr;
  cudaGraphExec_t exec = nullptr;
  // Reliable updates (set apply_hi): the iterations run on `apply` (e.g.
  // FP32 applies), and whenever the recursive residual has fallen by
  // reliable_factor since the last update it is replaced by the true
  // residual b - apply_hi(x); the first and the final residuals use
  // apply_hi too.
  ApplyFn<T> apply_hi;
  double reliable_factor = 0.1;
  int replacements = 0;
  cudaError_t setup(const ApplyFn<T>& apply, int64_t n, const T* b, T* x, Workspace& ws);
  // x_zero: x holds zeros on entry (skips the first residual's apply).
  // info->iters counts iterations (two operator applications each).
  SolveStatus solve(bool x_zero, double rtol, int maxit, cudaStream_t st, SolveInfo* info);
  void destroy();
};

// BiCGStab in FP64 vectors and scalars on the FP32 apply (converted in and
// out around every application) with reliable updates: the recursive
// residual is replaced by the true FP64 residual b - A64 x whenever it has
// fallen tenfold since the last replacement.
SolveStatus solve_bicgstab_reliable(const ApplyFn<double>& apply64,
                                    const ApplyFn<float>& apply32, int64_t n, const double* b,
                                    double* x, double rtol, int maxit, cudaStream_t st,
                                    Workspace& ws, SolveInfo* info, int* replacements);

// FP64 iterative refinement: r = b - A64 x in FP64, inner FP32 solve
// (GMRES(restart) or BiCGStab, SBM_INNER_*) of A32 c = r/|r| to inner_rtol,
// x += |r| c; maxit outer steps.
SolveStatus solve_ir(const ApplyFn<double>& apply64, const ApplyFn<float>& apply32, int64_t n,
                     const double* b, double* x, double rtol, int maxit, int restart,
                     double inner_rtol, int inner_maxit, int inner, cudaStream_t st,
                     Workspace& ws, SolveInfo* info);

}  // namespace sbm
