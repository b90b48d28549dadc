// A batch of independent continuous Galerkin problems (batch.cu: the
// persistent batched apply and its autotuner; batch_kernel.cuh: the kernel;
// batch_solve.cu: solves).
#pragma once

#include <map>
#include <vector>

#include "internal.hpp"

namespace sbm {
namespace bk {
struct Item;
template <typename T>
struct ProbTable;
// per precision (batch_f32.cu / batch_f64.cu)
cudaError_t set_unit_table(int n, const KTab<double>& t);
cudaError_t set_unit_table(int n, const KTab<float>& t);
size_t item_smem_f64(int d, int n, int v, int fh, int ext, int tc);
size_t item_smem_f32(int d, int n, int v, int fh, int ext, int tc);
cudaError_t occupancy_f64(size_t smem, bool tc, int* per_sm);
cudaError_t occupancy_f32(size_t smem, bool tc, int* per_sm);
cudaError_t launch(const ProbTable<double>& tab, const Item* items, int nitems, int nsys,
                   int nrhs, int* cnt, int* err, size_t smem, int grid, int tc_cols,
                   cudaStream_t st);
cudaError_t launch(const ProbTable<float>& tab, const Item* items, int nitems, int nsys, int nrhs,
                   int* cnt, int* err, size_t smem, int grid, int tc_cols, cudaStream_t st);
}  // namespace bk
}  // namespace sbm

// Device workspace of the batched solver, kept across solves so that the
// batched applies it issues reuse their cached graphs.
struct BatchSolveWs {
  int64_t n = 0;                   // elements of one concatenated vector
  int nsys = 0, ntile = 0;
  std::vector<void*> bufs;         // device allocations
  double *b = nullptr, *x = nullptr, *rout = nullptr, *d = nullptr;
  double *r = nullptr, *rh = nullptr, *p = nullptr, *v = nullptr, *s = nullptr, *t = nullptr,
         *xb = nullptr;
  float *a32 = nullptr, *b32 = nullptr;
  double* part = nullptr;          // [3][ntile] tile partial sums
  double* sums = nullptr;          // [2][nsys] per-system sums
  int32_t* use = nullptr;          // [nsys] refinement: keep this system's correction
  void* state = nullptr;           // [nsys] per-system BiCGStab state
  void* hstate = nullptr;          // pinned host copy
  int32_t *tsys = nullptr, *tlen = nullptr, *tfirst = nullptr;
  int64_t* tstart = nullptr;
  std::vector<int64_t> off;        // [nprob] first element of each problem
};

// Knobs of one degree for one precision, chosen by the autotuner: the cell
// kernel's tile shape (0: R cells per chunk, 1: R/2, 3: R cells without
// staged runs, 3D FP32), the face batch (0: 256/L faces per pass, 1:
// 128/L), tensor-core faces (FP32, 3D: 0 CUDA cores, 1 TF32 tcgen05), and
// the measured time of every option tried (ms of that degree's sub-batch;
// index shape + 2 face batch + 4 tensor cores for shapes 0 and 1, 8 + face
// batch for shape 3; < 0: not tried).
constexpr int kKnobOptions = 10;
struct DegreeKnobs {
  int shape = 0, face_batch = 0, tc = 0;
  float ms[kKnobOptions] = {-1.f, -1.f, -1.f, -1.f, -1.f, -1.f, -1.f, -1.f, -1.f, -1.f};
};

// The chunk table a tile shape uses (shape 3 runs shape 0's chunks).
inline int chunking(int shape) { return shape == 1 ? 1 : 0; }

// One launch of the persistent kernel: up to bk::kLaunchProbs problems of
// the batch (global indices in probs; the work list uses local ones), their
// work list for the current knobs, the launch shape and the offset of its
// dependency counters.
struct LaunchPlan {
  std::vector<int> probs;
  void* items = nullptr;             // device work list
  int nitems = 0;
  std::vector<int> nface_items, nchunk_items;   // [local problem] items per right-hand side
  size_t smem = 0;                   // dynamic shared memory per block
  int grid = 0;
  int tc_cols = 0;                   // tensor-memory columns per block (tensor-core faces)
  int cnt_off = 0;                   // ticket + 2 counters per system, from here
};

// Per-precision state of the batched apply: knobs, launch plans and the
// captured graphs (one per set of vector pointers).
struct BatchPrec {
  bool allow_tc = false;             // FP32: tensor-core (TF32) faces may be chosen
  std::vector<int> shape;            // [nprob] tile shape per problem
  std::map<int, DegreeKnobs> knobs;  // degree -> knobs
  bool dirty = true;                 // plans to rebuild
  std::vector<LaunchPlan> plans;
  int* cnt = nullptr;                // device counters of all plans
  std::vector<void*> face, col;      // [nprob] scratch: nrhs face results / colour buffers
  void* ktab = nullptr;              // [nprob] device copies of the problems' tables
  struct Graph {
    std::vector<const void*> ptrs;
    cudaGraphExec_t exec;
  };
  std::vector<Graph> graphs;
};

// Host copies of a problem's chunk boundaries, both tile shapes (for the
// work list).
struct ChunkHost {
  std::vector<int32_t> first[2];
};

struct sbm_batch {
  std::vector<sbm_problem*> probs;
  std::vector<ChunkHost> ch;         // [nprob]
  int nrhs = 0;
  int device = 0;
  cudaStream_t cap = nullptr;        // capture / tuning stream
  int* err = nullptr;                // device error word (SBM_ERR_TIMEOUT from bounded waits)
  BatchPrec prec[2];                 // [0] FP32, [1] FP64
  BatchSolveWs ws;
};

// Free the solver workspace (batch_solve.cu).
void batch_solve_release(sbm_batch* B);
