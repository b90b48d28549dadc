// Batched operator applies: many independent SBM problems of different size,
// degree and geometry, several right-hand sides each, in one CUDA-graph
// launch.
//
// Each problem's right-hand sides go through one set of its three kernels
// (face, cell, assembly) with grid.y = right-hand side.  Problems are spread
// over a pool of worker streams (largest first, round robin), forked from and
// joined back to a capture stream, and the whole fork/join is captured once
// into a CUDA graph per set of vector pointers; later calls only launch the
// graph.  The cell kernel's tile shape (cells per block) is chosen per degree
// by timing both shapes on the batch's largest problem of that degree.
#include <algorithm>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "batch.hpp"

using namespace sbm;

namespace {

constexpr int kStreams = 16;

size_t face_elems(const sbm_problem* p) { return (size_t)p->dd.nface * 2 * p->hp.L; }
size_t colour_elems(const sbm_problem* p) { return (size_t)p->dd.ncolours * p->hp.n_dofs; }

template <typename T>
cudaError_t ensure_scratch(sbm_batch* B, std::vector<T*>* face, std::vector<T*>* col) {
  if (!face->empty()) return cudaSuccess;
  face->assign(B->probs.size(), nullptr);
  col->assign(B->probs.size(), nullptr);
  for (size_t k = 0; k < B->probs.size(); ++k) {
    const size_t fe = std::max<size_t>(1, face_elems(B->probs[k])) * B->nrhs;
    const size_t ce = colour_elems(B->probs[k]) * B->nrhs;
    cudaError_t e = cudaMalloc((void**)&(*face)[k], fe * sizeof(T));
    if (e != cudaSuccess) return e;
    e = cudaMalloc((void**)&(*col)[k], ce * sizeof(T));
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <typename T>
cudaError_t enqueue(sbm_batch* B, const T* const* x, T* const* y, const std::vector<T*>& face,
                    const std::vector<T*>& col, cudaStream_t origin) {
  cudaError_t e = cudaEventRecord(B->fork, origin);
  if (e != cudaSuccess) return e;
  for (cudaStream_t s : B->streams)
    if ((e = cudaStreamWaitEvent(s, B->fork, 0)) != cudaSuccess) return e;
  for (size_t i = 0; i < B->order.size(); ++i) {
    const int k = B->order[i];
    const sbm_problem* p = B->probs[k];
    cudaStream_t s = B->streams[i % B->streams.size()];
    e = launch_cg_apply_multi<T>(p->hp, p->dd, x[k], y[k], p->hp.n_dofs, B->nrhs, face[k],
                                 col[k], B->variant[k], s);
    if (e != cudaSuccess) return e;
  }
  for (size_t s = 0; s < B->streams.size(); ++s) {
    if ((e = cudaEventRecord(B->join[s], B->streams[s])) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(origin, B->join[s], 0)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <typename T>
int batch_apply(sbm_batch* B, const T* const* x, T* const* y, void* stream, int prec,
                std::vector<T*>* face, std::vector<T*>* col) {
  if (!B || !x || !y) return sbm_fail_detail(SBM_ERR_ARG, "NULL argument");
  for (size_t k = 0; k < B->probs.size(); ++k)
    if (!x[k] || !y[k] || (const void*)x[k] == (const void*)y[k])
      return sbm_fail_detail(SBM_ERR_ARG, "bad vector pointer for problem " + std::to_string(k));
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return sbm_cuda_fail_detail(e, "cudaGetDevice");
  if (dev != B->device) return sbm_fail_detail(SBM_ERR_STATE, "current device is not the batch's");
  if ((e = ensure_scratch<T>(B, face, col)) != cudaSuccess)
    return e == cudaErrorMemoryAllocation ? sbm_fail_detail(SBM_ERR_OOM, "batch scratch")
                                          : sbm_cuda_fail_detail(e, "batch scratch");
  std::vector<const void*> key;
  for (size_t k = 0; k < B->probs.size(); ++k) {
    key.push_back(x[k]);
    key.push_back(y[k]);
  }
  cudaGraphExec_t exec = nullptr;
  for (auto& g : B->graphs)
    if (g.prec == prec && g.ptrs == key) exec = g.exec;
  if (!exec) {
    cudaGraph_t graph;
    if ((e = cudaStreamBeginCapture(B->cap, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
      return sbm_cuda_fail_detail(e, "capture");
    cudaError_t le = enqueue<T>(B, x, y, *face, *col, B->cap);
    e = cudaStreamEndCapture(B->cap, &graph);
    if (le != cudaSuccess) return sbm_cuda_fail_detail(le, "batch enqueue");
    if (e != cudaSuccess) return sbm_cuda_fail_detail(e, "capture end");
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return sbm_cuda_fail_detail(e, "graph instantiate");
    B->graphs.push_back({key, prec, exec});
  }
  if ((e = cudaGraphLaunch(exec, (cudaStream_t)stream)) != cudaSuccess)
    return sbm_cuda_fail_detail(e, "graph launch");
  return SBM_OK;
}

// Time both cell-kernel tile shapes on the largest problem of each degree.
int autotune(sbm_batch* B) {
  std::map<int, int> largest;   // degree -> problem index
  for (size_t k = 0; k < B->probs.size(); ++k) {
    const int p = B->probs[k]->hp.p;
    auto it = largest.find(p);
    if (it == largest.end() || B->probs[k]->hp.n_dofs > B->probs[it->second]->hp.n_dofs)
      largest[p] = (int)k;
  }
  cudaError_t e = ensure_scratch<float>(B, &B->face32, &B->col32);
  if (e != cudaSuccess) return sbm_cuda_fail_detail(e, "autotune scratch");
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  int status = SBM_OK;
  for (auto [deg, k] : largest) {
    const sbm_problem* p = B->probs[k];
    const size_t n = (size_t)p->hp.n_dofs * B->nrhs;
    float *x = nullptr, *y = nullptr;
    if (cudaMalloc((void**)&x, n * sizeof(float)) != cudaSuccess ||
        cudaMalloc((void**)&y, n * sizeof(float)) != cudaSuccess) {
      cudaFree(x);
      status = sbm_fail_detail(SBM_ERR_OOM, "autotune buffers");
      break;
    }
    cudaMemsetAsync(x, 0, n * sizeof(float), B->cap);
    float best = 1e30f;
    int bestv = 0;
    for (int v = 0; v < 2; ++v) {
      float tot = 0.f;
      for (int rep = 0; rep < 4; ++rep) {
        cudaEventRecord(e0, B->cap);
        e = launch_cg_apply_multi<float>(p->hp, p->dd, x, y, p->hp.n_dofs, B->nrhs, B->face32[k],
                                         B->col32[k], v, B->cap);
        cudaEventRecord(e1, B->cap);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0) tot += ms;      // first repetition warms up
      }
      if (e != cudaSuccess) {
        status = sbm_cuda_fail_detail(e, "autotune launch");
        break;
      }
      if (tot < best) {
        best = tot;
        bestv = v;
      }
    }
    cudaFree(x);
    cudaFree(y);
    if (status != SBM_OK) break;
    B->tuned[deg] = bestv;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  for (size_t k = 0; k < B->probs.size(); ++k) B->variant[k] = B->tuned[B->probs[k]->hp.p];
  return status;
}

void destroy(sbm_batch* B) {
  batch_solve_release(B);
  for (auto& g : B->graphs) cudaGraphExecDestroy(g.exec);
  for (auto* p : B->face32) cudaFree(p);
  for (auto* p : B->col32) cudaFree(p);
  for (auto* p : B->face64) cudaFree(p);
  for (auto* p : B->col64) cudaFree(p);
  for (cudaStream_t s : B->streams) cudaStreamDestroy(s);
  for (cudaEvent_t ev : B->join) cudaEventDestroy(ev);
  if (B->fork) cudaEventDestroy(B->fork);
  if (B->cap) cudaStreamDestroy(B->cap);
  delete B;
}

}  // namespace

extern "C" {

int sbm_batch_create(sbm_problem* const* probs, int nprob, int nrhs, int autotune_shapes,
                     sbm_batch** out) {
  if (!out) return sbm_fail_detail(SBM_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!probs || nprob < 1 || nrhs < 1 || nrhs > 65535)
    return sbm_fail_detail(SBM_ERR_ARG, "bad batch size");
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return sbm_cuda_fail_detail(e, "cudaGetDevice");
  for (int k = 0; k < nprob; ++k) {
    if (!probs[k]) return sbm_fail_detail(SBM_ERR_ARG, "NULL problem");
    if (!probs[k]->on_device || probs[k]->device != dev)
      return sbm_fail_detail(SBM_ERR_STATE, "problem not set up on the current device");
    if (probs[k]->hp.desc.dg)
      return sbm_fail_detail(SBM_ERR_UNSUPPORTED, "batches hold continuous Galerkin problems");
  }
  sbm_batch* B = new (std::nothrow) sbm_batch();
  if (!B) return sbm_fail_detail(SBM_ERR_OOM, "host allocation failed");
  B->probs.assign(probs, probs + nprob);
  B->nrhs = nrhs;
  B->device = dev;
  B->variant.assign(nprob, 0);
  B->order.resize(nprob);
  for (int k = 0; k < nprob; ++k) B->order[k] = k;
  std::stable_sort(B->order.begin(), B->order.end(), [&](int a, int b) {
    return B->probs[a]->hp.n_dofs * (int64_t)B->probs[a]->hp.nd >
           B->probs[b]->hp.n_dofs * (int64_t)B->probs[b]->hp.nd;
  });
  const int ns = std::min(kStreams, nprob);
  B->streams.assign(ns, nullptr);
  B->join.assign(ns, nullptr);
  bool ok = cudaStreamCreateWithFlags(&B->cap, cudaStreamNonBlocking) == cudaSuccess &&
            cudaEventCreateWithFlags(&B->fork, cudaEventDisableTiming) == cudaSuccess;
  for (int s = 0; ok && s < ns; ++s)
    ok = cudaStreamCreateWithFlags(&B->streams[s], cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&B->join[s], cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    destroy(B);
    return sbm_fail_detail(SBM_ERR_CUDA, "stream/event creation failed");
  }
  if (autotune_shapes) {
    int st = autotune(B);
    if (st != SBM_OK) {
      destroy(B);
      return st;
    }
  }
  *out = B;
  return SBM_OK;
}

int sbm_batch_apply_f32(sbm_batch* batch, const float* const* x, float* const* y, void* stream) {
  return batch_apply<float>(batch, x, y, stream, 32, batch ? &batch->face32 : nullptr,
                            batch ? &batch->col32 : nullptr);
}

int sbm_batch_apply_f64(sbm_batch* batch, const double* const* x, double* const* y,
                        void* stream) {
  return batch_apply<double>(batch, x, y, stream, 64, batch ? &batch->face64 : nullptr,
                             batch ? &batch->col64 : nullptr);
}

int sbm_batch_tile_shape(const sbm_batch* batch, int problem, int* variant) {
  if (!batch || !variant || problem < 0 || problem >= (int)batch->probs.size())
    return sbm_fail_detail(SBM_ERR_ARG, "bad argument");
  *variant = batch->variant[problem];
  return SBM_OK;
}

int sbm_batch_set_tile_shape(sbm_batch* batch, int problem, int variant) {
  if (!batch || problem < 0 || problem >= (int)batch->probs.size() || variant < 0 || variant > 1)
    return sbm_fail_detail(SBM_ERR_ARG, "bad argument");
  batch->variant[problem] = variant;
  for (auto& g : batch->graphs) cudaGraphExecDestroy(g.exec);
  batch->graphs.clear();
  return SBM_OK;
}

void sbm_batch_destroy(sbm_batch* batch) {
  if (batch) destroy(batch);
}

}  // extern "C"
