// A batch of independent continuous Galerkin problems (batch.cu: applies;
// batch_solve.cu: solves).
#pragma once

#include <map>
#include <vector>

#include "internal.hpp"

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

struct sbm_batch {
  std::vector<sbm_problem*> probs;
  int nrhs = 0;
  int device = 0;
  std::vector<int> order;           // problems, largest first
  std::vector<int> variant;         // cell-kernel tile shape per problem
  std::map<int, int> tuned;         // degree -> variant
  std::vector<cudaStream_t> streams;
  cudaStream_t cap = nullptr;
  cudaEvent_t fork = nullptr;
  std::vector<cudaEvent_t> join;
  std::vector<float*> face32, col32;
  std::vector<double*> face64, col64;
  struct Graph {
    std::vector<const void*> ptrs;
    int prec;
    cudaGraphExec_t exec;
  };
  std::vector<Graph> graphs;
  BatchSolveWs ws;
};

// Free the solver workspace (batch_solve.cu).
void batch_solve_release(sbm_batch* B);
