// Batched operator applies: many independent continuous Galerkin SBM
// problems of different size, degree and geometry, several right-hand sides
// each, in ONE persistent kernel launch (batch_kernel.cuh) captured into a
// CUDA graph.
//
// The host side: the work list (items sized and ordered by the paper's
// load-balancing weights, Section 3.5), the per-degree constant tables, the
// scratch, the graphs (one per set of vector pointers: a memset of the
// dependency counters and the kernel), and the autotuner that picks, per
// degree and precision, the cell kernel's tile shape and the face batch.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <new>
#include <numeric>
#include <string>
#include <vector>

#include "batch.hpp"
#include "batch_kernel.cuh"
#include "tc_common.cuh"

using namespace sbm;
using bk::Item;
using bk::Prob;

namespace {

constexpr int kItemsPerBlock = 6;      // work-list items per resident block and phase
constexpr int64_t kAsmEntries = 4096;  // shared-DoF list entries per assembly item
constexpr int kMaxGraphs = 8;          // cached pointer sets per precision

template <typename T>
constexpr int pidx() {
  return std::is_same<T, double>::value ? 1 : 0;
}

size_t item_smem(int pi, int d, int n, int v, int fh, int ext, int tc) {
  return pi ? bk::item_smem_f64(d, n, v, fh, ext, tc) : bk::item_smem_f32(d, n, v, fh, ext, tc);
}
cudaError_t occupancy(int pi, size_t smem, bool tc, int* per_sm) {
  return pi ? bk::occupancy_f64(smem, tc, per_sm) : bk::occupancy_f32(smem, tc, per_sm);
}

// Tile shape 3 in the batch: FP32 (precision index 0), 3D problems (the
// FP64 kernel's 48-register budget would make its loop spill).
bool direct_ok(int pi, const sbm_problem* p) { return pi == 0 && p->hp.d == 3; }

int face_batch_faces(int d, int n, int fh) {
  const int L = (d == 3) ? n * n : n;
  const int ff = bk::kThreads / L;
  return fh ? std::max(1, ff / 2) : ff;
}

// Tensor-core faces for problem k in precision pi: FP32, 3D, exact
// extension, allowed for the batch and chosen for the problem's degree.
int prob_tc(const sbm_batch* B, int pi, int k) {
  const BatchPrec& P = B->prec[pi];
  const sbm_problem* p = B->probs[k];
  if (pi != 0 || !P.allow_tc || p->hp.d != 3 || p->hp.desc.extension != SBM_EXT_EXACT) return 0;
  auto kn = P.knobs.find(p->hp.p);
  return kn == P.knobs.end() ? 0 : kn->second.tc;
}

// ---- scratch -----------------------------------------------------------------

size_t face_elems(const sbm_problem* p) { return (size_t)p->dd.nface * 2 * p->hp.L; }
size_t colour_elems(const sbm_problem* p) { return (size_t)p->dd.ncolours * p->hp.n_dofs; }

void free_scratch(BatchPrec& P) {
  for (void* q : P.face) cudaFree(q);
  for (void* q : P.col) cudaFree(q);
  P.face.clear();
  P.col.clear();
}

// nrhs copies of every problem's per-face results and colour buffers; all or
// nothing (a failed allocation frees what was allocated).
cudaError_t ensure_scratch(sbm_batch* B, int pi) {
  BatchPrec& P = B->prec[pi];
  if (!P.face.empty()) return cudaSuccess;
  const size_t es = pi ? sizeof(double) : sizeof(float);
  std::vector<void*> face(B->probs.size(), nullptr), col(B->probs.size(), nullptr);
  cudaError_t e = cudaSuccess;
  for (size_t k = 0; k < B->probs.size() && e == cudaSuccess; ++k) {
    const size_t fe = std::max<size_t>(1, face_elems(B->probs[k])) * B->nrhs;
    const size_t ce = colour_elems(B->probs[k]) * B->nrhs;
    e = cudaMalloc(&face[k], fe * es);
    if (e == cudaSuccess) e = cudaMalloc(&col[k], ce * es);
  }
  if (e != cudaSuccess) {
    for (void* q : face) cudaFree(q);
    for (void* q : col) cudaFree(q);
    cudaGetLastError();
    return e;
  }
  P.face = face;
  P.col = col;
  return cudaSuccess;
}

void drop_graphs(BatchPrec& P) {
  for (auto& g : P.graphs) cudaGraphExecDestroy(g.exec);
  P.graphs.clear();
}

// ---- the work list ------------------------------------------------------------

struct HostItem {
  Item it;
  double w;
  int deg;
};

// Work list of one launch plan for precision pi with the batch's current
// knobs: every system's faces in groups of whole face passes, its chunks,
// its shared-DoF list; sized so that each phase has about kItemsPerBlock
// items per resident block, then ordered face items, chunk items, assembly
// items, each by degree and heaviest first (weights: 10 per cell, 40 per
// surrogate face in 3D and 20 in 2D, times (p+1)^(d+1)).  Item problem
// indices are local to the plan.
void make_items(const sbm_batch* B, int pi, const std::vector<int>& probs, int grid,
                std::vector<Item>* out, std::vector<int>* nfi, std::vector<int>* nci) {
  const BatchPrec& P = B->prec[pi];
  const int np = (int)probs.size();
  nfi->assign(np, 0);
  nci->assign(np, 0);
  double wf_tot = 0.0, wc_tot = 0.0;
  for (int k : probs) {
    const sbm_problem* p = B->probs[k];
    const double cost = std::pow((double)p->hp.n, p->hp.d + 1);
    wf_tot += (p->hp.d == 3 ? 40.0 : 20.0) * cost * p->dd.nface;
    wc_tot += 10.0 * cost * (double)(p->hp.cells.size() / p->hp.d);
  }
  const double slots = (double)kItemsPerBlock * std::max(1, grid);
  const double tf = std::max(1.0, wf_tot * B->nrhs / slots);
  const double tc = std::max(1.0, wc_tot * B->nrhs / slots);
  std::vector<HostItem> F, C, A;
  for (int j = 0; j < np; ++j) {
    const int k = probs[j];
    const sbm_problem* p = B->probs[k];
    const int d = p->hp.d, n = p->hp.n;
    const double cost = std::pow((double)n, d + 1);
    const double wface = (d == 3 ? 40.0 : 20.0) * cost, wcell = 10.0 * cost;
    const int v = chunking(P.shape[k]);
    auto kn = P.knobs.find(p->hp.p);
    const int fh = (kn == P.knobs.end() || p->hp.desc.extension == SBM_EXT_TAYLOR1)
                       ? 0 : kn->second.face_batch;
    // a tensor-core face item runs its faces one at a time
    const int fpb = prob_tc(B, pi, k) ? 1 : face_batch_faces(d, n, fh);
    // faces: whole passes of fpb faces, about tf weight per item
    std::vector<std::pair<int, int>> fr;
    const int per = std::max(fpb, (int)std::lround(tf / wface / fpb) * fpb);
    for (int f = 0; f < p->dd.nface; f += per) fr.push_back({f, std::min(p->dd.nface, f + per)});
    // chunks: consecutive chunks up to about tc weight
    std::vector<std::pair<int, int>> cr;
    const std::vector<int32_t>& first = B->ch[k].first[v];
    const int nch = (int)first.size() - 1;
    for (int q = 0; q < nch;) {
      int q1 = q;
      double w = 0.0;
      while (q1 < nch && (q1 == q || w < tc)) {
        w += wcell * (first[q1 + 1] - first[q1]);
        ++q1;
      }
      cr.push_back({q, q1});
      q = q1;
    }
    const int64_t nm = p->dd.chunks[v].nmulti;
    (*nfi)[j] = (int)fr.size();
    (*nci)[j] = (int)cr.size();
    for (int r = 0; r < B->nrhs; ++r) {
      for (auto [a, b] : fr) F.push_back({{j, bk::kFace | (r << 2), a, b}, wface * (b - a), p->hp.p});
      for (auto [a, b] : cr)
        C.push_back({{j, bk::kChunk | (r << 2), a, b}, wcell * (first[b] - first[a]), p->hp.p});
      for (int64_t m = 0; m < nm; m += kAsmEntries) {
        const int64_t m1 = std::min(nm, m + kAsmEntries);
        A.push_back({{j, bk::kAsm | (r << 2), (int32_t)m, (int32_t)m1}, (double)(m1 - m), p->hp.p});
      }
    }
  }
  // within a phase: by degree (highest first), then heaviest first -- a
  // block's consecutive items then mostly run one degree's code, which keeps
  // the instruction caches warm (the kernel holds every degree's paths)
  auto heavy_first = [](const HostItem& a, const HostItem& b) {
    return a.deg != b.deg ? a.deg > b.deg : a.w > b.w;
  };
  std::stable_sort(F.begin(), F.end(), heavy_first);
  std::stable_sort(C.begin(), C.end(), heavy_first);
  std::stable_sort(A.begin(), A.end(), heavy_first);
  out->clear();
  for (auto* g : {&F, &C, &A})
    for (const HostItem& h : *g) out->push_back(h.it);
}

// Dynamic shared memory one problem's items need with the current knobs.
size_t prob_smem(const sbm_batch* B, int pi, int k) {
  const BatchPrec& P = B->prec[pi];
  const sbm_problem* p = B->probs[k];
  auto kn = P.knobs.find(p->hp.p);
  const int fh = kn == P.knobs.end() ? 0 : kn->second.face_batch;
  return item_smem(pi, p->hp.d, p->hp.n, P.shape[k], fh,
                   p->hp.desc.extension == SBM_EXT_TAYLOR1, prob_tc(B, pi, k));
}

void free_plans(std::vector<LaunchPlan>* plans) {
  for (LaunchPlan& L : *plans) cudaFree(L.items);
  plans->clear();
}

// Launch plans for the problems `probs` (in order, at most kLaunchProbs per
// launch): work lists on the device, launch shapes, counter offsets.
// smem_min raises every plan's shared memory (the autotuner times all
// options at one occupancy).
cudaError_t make_plans(const sbm_batch* B, int pi, const std::vector<int>& probs, size_t smem_min,
                       std::vector<LaunchPlan>* plans) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  int cnt_off = 0;
  for (size_t g = 0; g < probs.size(); g += bk::kLaunchProbs) {
    LaunchPlan L;
    L.probs.assign(probs.begin() + g,
                   probs.begin() + std::min(probs.size(), g + (size_t)bk::kLaunchProbs));
    L.smem = smem_min;
    for (int k : L.probs) {
      L.smem = std::max(L.smem, prob_smem(B, pi, k));
      if (prob_tc(B, pi, k)) L.tc_cols = tc::kTmemCols;
    }
    int per_sm = 0;
    if ((e = occupancy(pi, L.smem, L.tc_cols != 0, &per_sm)) != cudaSuccess) break;
    if (per_sm < 1) {
      e = cudaErrorInvalidConfiguration;
      break;
    }
    // every resident block holds tc_cols of the SM's 512 tensor-memory columns
    if (L.tc_cols) per_sm = std::min(per_sm, 512 / L.tc_cols);
    std::vector<Item> items;
    make_items(B, pi, L.probs, per_sm * sms, &items, &L.nface_items, &L.nchunk_items);
    L.nitems = (int)items.size();
    L.grid = std::min(per_sm * sms, L.nitems);
    L.cnt_off = cnt_off;
    cnt_off += 1 + 2 * (int)L.probs.size() * B->nrhs;
    if ((e = cudaMalloc(&L.items, items.size() * sizeof(Item))) != cudaSuccess) break;
    plans->push_back(L);
    if ((e = cudaMemcpy(L.items, items.data(), items.size() * sizeof(Item),
                        cudaMemcpyHostToDevice)) != cudaSuccess)
      break;
  }
  if (e != cudaSuccess) free_plans(plans);
  return e;
}

// counters of all plans (the batch's allocation covers any plan set)
size_t cnt_ints(const sbm_batch* B) {
  const size_t np = B->probs.size();
  return (np + bk::kLaunchProbs - 1) / bk::kLaunchProbs + 2 * np * B->nrhs;
}

// Plans of the whole batch for precision pi (after a knob change).
cudaError_t rebuild(sbm_batch* B, int pi) {
  BatchPrec& P = B->prec[pi];
  if (!P.dirty) return cudaSuccess;
  drop_graphs(P);
  free_plans(&P.plans);
  std::vector<int> all(B->probs.size());
  std::iota(all.begin(), all.end(), 0);
  cudaError_t e = make_plans(B, pi, all, 0, &P.plans);
  if (e == cudaSuccess) P.dirty = false;
  return e;
}

// The problem descriptors of one plan for one set of vectors (x[k], y[k]).
template <typename T>
void make_table(const sbm_batch* B, const LaunchPlan& L, const T* const* x, T* const* y,
                bk::ProbTable<T>* tab) {
  constexpr int pi = pidx<T>();
  const BatchPrec& P = B->prec[pi];
  std::memset((void*)tab, 0, sizeof(*tab));
  for (size_t j = 0; j < L.probs.size(); ++j) {
    const int k = L.probs[j];
    const sbm_problem* p = B->probs[k];
    const DeviceData& dd = p->dd;
    const int v = P.shape[k];
    const ChunkTable& ct = dd.chunks[chunking(v)];
    auto kn = P.knobs.find(p->hp.p);
    const int fh = kn == P.knobs.end() ? 0 : kn->second.face_batch;
    const int ext = p->hp.desc.extension == SBM_EXT_TAYLOR1;
    Prob<T>& q = tab->p[j];
    T* fo = static_cast<T*>(P.face[k]);
    T* yc = static_cast<T*>(P.col[k]);
    q.ca.x = x[k];
    q.ca.y = y[k];
    q.ca.ycol = yc;
    q.ca.run_bits = ct.run_bits;
    q.ca.bit_words = ct.bit_words;
    q.ca.lines = dd.lines;
    q.ca.face_start = dd.face_start;
    q.ca.face_kind = dd.face_kind;
    q.ca.face_out = fo;
    q.ca.chunk_first = ct.first;
    q.ca.chunk_col = ct.colour;
    q.ca.n_dofs = p->hp.n_dofs;
    q.ca.q0 = 0;
    q.ca.q1 = ct.n;
    q.ca.ldx = p->hp.n_dofs;
    q.ca.ld_ycol = (int64_t)dd.ncolours * p->hp.n_dofs;
    q.ca.ld_face = (int64_t)dd.nface * 2 * p->hp.L;
    q.fa.x = x[k];
    q.fa.lines = dd.lines;
    q.fa.cell_rank = dd.cell_rank;
    q.fa.face_cell = dd.face_cell;
    q.fa.face_kind = dd.face_kind;
    q.fa.face_phi = face_phi_of<T>(dd);
    q.fa.face_pp = face_pp_of<T>(dd);
    q.fa.out = fo;
    q.fa.face0 = 0;
    q.fa.nface = dd.nface;
    q.fa.dg = 0;
    q.fa.ldx = p->hp.n_dofs;
    q.fa.ld_out = (int64_t)dd.nface * 2 * p->hp.L;
    q.kt = static_cast<const KTab<T>*>(P.ktab) + k;
    q.multi = ct.multi;
    q.mask = ct.multi_mask;
    q.ld_asm_ycol = (int64_t)dd.ncolours * p->hp.n_dofs;
    q.code = bk::code_of(p->hp.d, p->hp.n, v, ext ? 0 : fh, ext, prob_tc(B, pi, k));
    q.ncol = dd.ncolours;
    q.n_face_items = L.nface_items[j];
    q.n_chunk_items = L.nchunk_items[j];
  }
}

int nsys(const sbm_batch* B) { return (int)B->probs.size() * B->nrhs; }

// A counter reset and one launch per plan, on st.
template <typename T>
cudaError_t enqueue(sbm_batch* B, const std::vector<LaunchPlan>& plans, const T* const* x,
                    T* const* y, cudaStream_t st) {
  constexpr int pi = pidx<T>();
  BatchPrec& P = B->prec[pi];
  cudaError_t e = cudaMemsetAsync(P.cnt, 0, cnt_ints(B) * sizeof(int), st);
  std::unique_ptr<bk::ProbTable<T>> tab(new (std::nothrow) bk::ProbTable<T>);
  if (!tab) return cudaErrorMemoryAllocation;
  for (const LaunchPlan& L : plans) {
    if (e != cudaSuccess) break;
    make_table<T>(B, L, x, y, tab.get());
    e = bk::launch(*tab, static_cast<const Item*>(L.items), L.nitems,
                   (int)L.probs.size() * B->nrhs, B->nrhs, P.cnt + L.cnt_off, B->err, L.smem,
                   L.grid, L.tc_cols, st);
  }
  return e;
}

template <typename T>
int batch_apply(sbm_batch* B, const T* const* x, T* const* y, void* stream) {
  constexpr int pi = pidx<T>();
  if (!B || !x || !y) return sbm_fail_detail(SBM_ERR_ARG, "NULL argument");
  for (size_t k = 0; k < B->probs.size(); ++k)
    if (!x[k] || !y[k] || (const void*)x[k] == (const void*)y[k])
      return sbm_fail_detail(SBM_ERR_ARG, "bad vector pointer for problem " + std::to_string(k));
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return sbm_cuda_fail_detail(e, "cudaGetDevice");
  if (dev != B->device) return sbm_fail_detail(SBM_ERR_STATE, "current device is not the batch's");
  if ((e = ensure_scratch(B, pi)) != cudaSuccess)
    return e == cudaErrorMemoryAllocation ? sbm_fail_detail(SBM_ERR_OOM, "batch scratch")
                                          : sbm_cuda_fail_detail(e, "batch scratch");
  BatchPrec& P = B->prec[pi];
  if ((e = rebuild(B, pi)) != cudaSuccess) return sbm_cuda_fail_detail(e, "batch work list");
  std::vector<const void*> key;
  for (size_t k = 0; k < B->probs.size(); ++k) {
    key.push_back(x[k]);
    key.push_back(y[k]);
  }
  cudaGraphExec_t exec = nullptr;
  for (auto& g : P.graphs)
    if (g.ptrs == key) exec = g.exec;
  if (!exec) {
    if ((int)P.graphs.size() >= kMaxGraphs) {
      cudaDeviceSynchronize();
      drop_graphs(P);
    }
    cudaGraph_t graph = nullptr;
    if ((e = cudaStreamBeginCapture(B->cap, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
      return sbm_cuda_fail_detail(e, "capture");
    const cudaError_t le = enqueue<T>(B, P.plans, x, y, B->cap);
    e = cudaStreamEndCapture(B->cap, &graph);
    if (le == cudaSuccess && e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (le != cudaSuccess || e != cudaSuccess) {
      cudaGetLastError();
      return sbm_cuda_fail_detail(le != cudaSuccess ? le : e, "batch graph");
    }
    P.graphs.push_back({key, exec});
  }
  if ((e = cudaGraphLaunch(exec, (cudaStream_t)stream)) != cudaSuccess)
    return sbm_cuda_fail_detail(e, "graph launch");
  return SBM_OK;
}

// ---- autotuner ------------------------------------------------------------------

// Time the problems of one degree with the current knobs, every launch at
// shared memory smem (one warm-up, then the best of three), in ms.
template <typename T>
cudaError_t time_subset(sbm_batch* B, const std::vector<int>& subset, size_t smem, T* xbuf,
                        T* ybuf, float* ms) {
  constexpr int pi = pidx<T>();
  std::vector<const T*> xs(B->probs.size(), xbuf);
  std::vector<T*> ys(B->probs.size(), ybuf);
  size_t off = 0;
  for (int k : subset) {
    xs[k] = xbuf + off;
    ys[k] = ybuf + off;
    off += (size_t)B->probs[k]->hp.n_dofs * B->nrhs;
  }
  std::vector<LaunchPlan> plans;
  cudaError_t e = make_plans(B, pi, subset, smem, &plans);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float best = 1e30f;
  for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
    e = cudaEventRecord(e0, B->cap);
    if (e == cudaSuccess) e = enqueue<T>(B, plans, xs.data(), ys.data(), B->cap);
    if (e == cudaSuccess) e = cudaEventRecord(e1, B->cap);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    if (e == cudaSuccess && rep > 0) best = std::min(best, t);     // the first one warms up
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaStreamSynchronize(B->cap);
  free_plans(&plans);
  *ms = best;
  return e;
}

// Per degree: every (tile shape, face batch) option on that degree's
// problems; the fastest is kept, the timings recorded.
template <typename T>
int autotune(sbm_batch* B) {
  constexpr int pi = pidx<T>();
  BatchPrec& P = B->prec[pi];
  cudaError_t e = ensure_scratch(B, pi);
  if (e != cudaSuccess) return sbm_cuda_fail_detail(e, "autotune scratch");
  std::map<int, std::vector<int>> by_deg;
  for (size_t k = 0; k < B->probs.size(); ++k) by_deg[B->probs[k]->hp.p].push_back((int)k);
  // shared memory: the largest any option of any problem needs, so every
  // option is timed at the occupancy of the final launch or below
  size_t smem = 0, most = 0;
  for (auto& [deg, ks] : by_deg) {
    size_t n = 0;
    for (int k : ks) {
      const sbm_problem* p = B->probs[k];
      for (int v : {0, 1, 3})
        for (int fh = 0; fh < 2; ++fh)
          if (v != 3 || direct_ok(pi, p))
            smem = std::max(smem, item_smem(pi, p->hp.d, p->hp.n, v, fh,
                                            p->hp.desc.extension == SBM_EXT_TAYLOR1,
                                            P.allow_tc && pi == 0 && p->hp.d == 3));
      n += (size_t)p->hp.n_dofs * B->nrhs;
    }
    most = std::max(most, n);
  }
  T *xbuf = nullptr, *ybuf = nullptr;
  if (cudaMalloc((void**)&xbuf, most * sizeof(T)) != cudaSuccess ||
      cudaMalloc((void**)&ybuf, most * sizeof(T)) != cudaSuccess) {
    cudaFree(xbuf);
    cudaGetLastError();
    return sbm_fail_detail(SBM_ERR_OOM, "autotune buffers");
  }
  int status = SBM_OK;
  if ((e = cudaMemsetAsync(xbuf, 0, most * sizeof(T), B->cap)) != cudaSuccess)
    status = sbm_cuda_fail_detail(e, "autotune buffers");
  for (auto& [deg, ks] : by_deg) {
    if (status != SBM_OK) break;
    DegreeKnobs& kn = P.knobs[deg];
    float best = 1e30f;
    int bv = 0, bf = 0, bt = 0;
    // tensor-core faces: FP32, when the batch allows them and the degree has
    // a 3D problem with the exact extension (they take one face at a time,
    // so the face batch is not varied with them)
    bool tc_ok = false;
    for (int k : ks)
      tc_ok |= B->probs[k]->hp.d == 3 && B->probs[k]->hp.desc.extension == SBM_EXT_EXACT;
    tc_ok = tc_ok && pi == 0 && P.allow_tc;
    // tile shape 3 (options 8, 9): FP32, when every problem of the degree is 3D
    bool direct = pi == 0;
    for (int k : ks) direct = direct && direct_ok(pi, B->probs[k]);
    for (int opt = 0; opt < kKnobOptions && status == SBM_OK; ++opt) {
      const int v = opt >= 8 ? 3 : (opt & 1), fh = opt >= 8 ? opt - 8 : (opt >> 1) & 1;
      const int tcv = opt >= 8 ? 0 : opt >> 2;
      if ((tcv && (!tc_ok || fh)) || (v == 3 && !direct)) continue;
      kn.shape = v;
      kn.face_batch = fh;
      kn.tc = tcv;
      for (int k : ks) P.shape[k] = v;
      float ms = 0.f;
      if ((e = time_subset<T>(B, ks, smem, xbuf, ybuf, &ms)) != cudaSuccess) {
        status = sbm_cuda_fail_detail(e, "autotune launch");
        break;
      }
      kn.ms[opt] = ms;
      if (ms < best) {
        best = ms;
        bv = v;
        bf = fh;
        bt = tcv;
      }
    }
    kn.shape = bv;
    kn.face_batch = bf;
    kn.tc = bt;
    for (int k : ks) P.shape[k] = bv;
  }
  cudaStreamSynchronize(B->cap);
  cudaFree(xbuf);
  cudaFree(ybuf);
  P.dirty = true;
  if (status == SBM_OK) {
    int h = 0;
    if ((e = cudaMemcpy(&h, B->err, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess)
      return sbm_cuda_fail_detail(e, "autotune status");
    if (h != 0) return sbm_fail_detail(h, "a bounded wait expired while autotuning");
  }
  return status;
}

void destroy(sbm_batch* B) {
  cudaDeviceSynchronize();      // no launch of this batch may still run
  batch_solve_release(B);
  for (BatchPrec& P : B->prec) {
    drop_graphs(P);
    free_scratch(P);
    free_plans(&P.plans);
    cudaFree(P.cnt);
    cudaFree(P.ktab);
  }
  cudaFree(B->err);
  if (B->cap) cudaStreamDestroy(B->cap);
  delete B;
}

// The h-independent tables of degree n - 1 for the constant bank: the
// problem's table with the h-scaled entries replaced by their unscaled
// values (the 2D cell term reads Mh, Kh, whose scale h^0 is exactly 1) and
// the per-problem scalars poisoned (the kernel takes those from the
// problem's own table).
template <typename T>
KTab<T> unit_table(const HostProblem& hp) {
  KTab<T> t = make_ktab<T>(hp);
  std::memcpy(t.Mh, t.M, sizeof(t.M));
  std::memcpy(t.Kh, t.K, sizeof(t.K));
  t.fMh = t.fM;
  t.fKh = t.fK;
  const T nan = std::numeric_limits<T>::quiet_NaN();
  for (auto& w : t.W) w = nan;
  for (auto& l : t.hlam) l = nan;
  t.h_inv = t.hface = t.sigma = nan;
  return t;
}

template <typename T>
int setup_tables(sbm_batch* B) {
  constexpr int pi = pidx<T>();
  const int nprob = (int)B->probs.size();
  std::vector<KTab<T>> kt(nprob);
  std::map<int, KTab<T>> unit;
  for (int k = 0; k < nprob; ++k) {
    const HostProblem& hp = B->probs[k]->hp;
    kt[k] = make_ktab<T>(hp);
    const KTab<T> u = unit_table<T>(hp);
    auto it = unit.find(hp.n);
    if (it == unit.end()) {
      unit[hp.n] = u;
    } else if (std::memcmp(&it->second, &u, sizeof(u)) != 0) {
      return sbm_fail_detail(SBM_ERR_STATE, "1D tables of one degree differ between problems");
    }
  }
  cudaError_t e = cudaMalloc(&B->prec[pi].ktab, nprob * sizeof(KTab<T>));
  if (e != cudaSuccess) return sbm_fail_detail(SBM_ERR_OOM, "batch tables");
  if ((e = cudaMemcpy(B->prec[pi].ktab, kt.data(), nprob * sizeof(KTab<T>),
                      cudaMemcpyHostToDevice)) != cudaSuccess)
    return sbm_cuda_fail_detail(e, "batch tables");
  for (auto& [n, u] : unit)
    if ((e = bk::set_unit_table(n, u)) != cudaSuccess)
      return sbm_cuda_fail_detail(e, "constant tables");
  return SBM_OK;
}

}  // namespace

extern "C" {

int sbm_batch_create(sbm_problem* const* probs, int nprob, int nrhs, int autotune_shapes,
                     sbm_batch** out) {
  if (!out) return sbm_fail_detail(SBM_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!probs || nprob < 1 || nrhs < 1 || nrhs > (1 << 20))
    return sbm_fail_detail(SBM_ERR_ARG, "bad batch size");
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return sbm_cuda_fail_detail(e, "cudaGetDevice");
  int64_t items_bound = 0;
  for (int k = 0; k < nprob; ++k) {
    if (!probs[k]) return sbm_fail_detail(SBM_ERR_ARG, "NULL problem");
    if (!probs[k]->on_device || probs[k]->device != dev)
      return sbm_fail_detail(SBM_ERR_STATE, "problem not set up on the current device");
    if (probs[k]->hp.desc.dg)
      return sbm_fail_detail(SBM_ERR_UNSUPPORTED, "batches hold continuous Galerkin problems");
    items_bound += (int64_t)nrhs * (probs[k]->dd.nface + probs[k]->dd.chunks[0].n +
                                    probs[k]->dd.chunks[0].nmulti / kAsmEntries + 3);
  }
  if (items_bound >= (int64_t)1 << 31 || (int64_t)nprob * nrhs * 2 + 1 >= (int64_t)1 << 31)
    return sbm_fail_detail(SBM_ERR_ARG, "batch too large for one work list");
  sbm_batch* B = new (std::nothrow) sbm_batch();
  if (!B) return sbm_fail_detail(SBM_ERR_OOM, "host allocation failed");
  B->probs.assign(probs, probs + nprob);
  B->nrhs = nrhs;
  B->device = dev;
  B->ch.resize(nprob);
  bool ok = cudaStreamCreateWithFlags(&B->cap, cudaStreamNonBlocking) == cudaSuccess &&
            cudaMalloc((void**)&B->err, sizeof(int)) == cudaSuccess &&
            cudaMemset(B->err, 0, sizeof(int)) == cudaSuccess;
  B->prec[0].allow_tc = (autotune_shapes & SBM_BATCH_TENSOR_CORES) != 0;
  for (int pi = 0; ok && pi < 2; ++pi) {
    B->prec[pi].shape.assign(nprob, 0);
    ok = cudaMalloc((void**)&B->prec[pi].cnt, cnt_ints(B) * sizeof(int)) == cudaSuccess;
  }
  for (int k = 0; ok && k < nprob; ++k)
    for (int v = 0; ok && v < 2; ++v) {
      const ChunkTable& ct = probs[k]->dd.chunks[v];
      B->ch[k].first[v].resize(ct.n + 1);
      ok = cudaMemcpy(B->ch[k].first[v].data(), ct.first, (ct.n + 1) * sizeof(int32_t),
                      cudaMemcpyDeviceToHost) == cudaSuccess;
    }
  if (!ok) {
    cudaGetLastError();
    destroy(B);
    return sbm_fail_detail(SBM_ERR_CUDA, "batch set-up (stream, counters, chunk tables)");
  }
  int st = setup_tables<float>(B);
  if (st == SBM_OK) st = setup_tables<double>(B);
  if (st == SBM_OK && (autotune_shapes & SBM_BATCH_AUTOTUNE)) {
    st = autotune<float>(B);
    if (st == SBM_OK) st = autotune<double>(B);
  }
  if (st != SBM_OK) {
    destroy(B);
    return st;
  }
  *out = B;
  return SBM_OK;
}

int sbm_batch_apply_f32(sbm_batch* batch, const float* const* x, float* const* y, void* stream) {
  return batch_apply<float>(batch, x, y, stream);
}

int sbm_batch_apply_f64(sbm_batch* batch, const double* const* x, double* const* y,
                        void* stream) {
  return batch_apply<double>(batch, x, y, stream);
}

int sbm_batch_tile_shape(const sbm_batch* batch, int problem, int* variant) {
  if (!batch || !variant || problem < 0 || problem >= (int)batch->probs.size())
    return sbm_fail_detail(SBM_ERR_ARG, "bad argument");
  *variant = batch->prec[0].shape[problem];
  return SBM_OK;
}

int sbm_batch_set_tile_shape(sbm_batch* batch, int problem, int variant) {
  if (!batch || problem < 0 || problem >= (int)batch->probs.size() || variant < 0 || variant > 1)
    return sbm_fail_detail(SBM_ERR_ARG, "bad argument");
  cudaDeviceSynchronize();
  for (BatchPrec& P : batch->prec) {
    P.shape[problem] = variant;
    P.dirty = true;
    drop_graphs(P);
  }
  return SBM_OK;
}

int sbm_batch_knobs(const sbm_batch* batch, int precision, int degree, int* tile_shape,
                    int* face_batch, int* tensor_cores, float* ms) {
  if (!batch || (precision != 32 && precision != 64))
    return sbm_fail_detail(SBM_ERR_ARG, "bad argument");
  const BatchPrec& P = batch->prec[precision == 64 ? 1 : 0];
  auto it = P.knobs.find(degree);
  if (it == P.knobs.end()) return sbm_fail_detail(SBM_ERR_ARG, "no tuned problem of that degree");
  if (tile_shape) *tile_shape = it->second.shape;
  if (face_batch) *face_batch = it->second.face_batch;
  if (tensor_cores) *tensor_cores = it->second.tc;
  if (ms)
    for (int i = 0; i < kKnobOptions; ++i) ms[i] = it->second.ms[i];
  return SBM_OK;
}

int sbm_batch_set_knobs(sbm_batch* batch, int precision, int degree, int tile_shape,
                        int face_batch, int tensor_cores) {
  if (!batch || (precision != 32 && precision != 64) || tile_shape < 0 || tile_shape > 3 ||
      tile_shape == 2 || face_batch < 0 || face_batch > 1 || tensor_cores < 0 ||
      tensor_cores > 1)
    return sbm_fail_detail(SBM_ERR_ARG, "bad argument");
  const int pi = precision == 64 ? 1 : 0;
  if (tensor_cores && (pi != 0 || !batch->prec[0].allow_tc))
    return sbm_fail_detail(SBM_ERR_UNSUPPORTED,
                           "tensor-core faces: FP32 batches created with SBM_BATCH_TENSOR_CORES");
  if (tile_shape == 3 && tensor_cores)
    return sbm_fail_detail(SBM_ERR_UNSUPPORTED, "tile shape 3 runs CUDA-core faces");
  bool any = false;
  for (size_t k = 0; k < batch->probs.size(); ++k)
    if (batch->probs[k]->hp.p == degree) {
      any = true;
      if (tile_shape == 3 && !direct_ok(pi, batch->probs[k]))
        return sbm_fail_detail(SBM_ERR_UNSUPPORTED, "tile shape 3: FP32 batches of 3D problems");
    }
  if (!any) return sbm_fail_detail(SBM_ERR_ARG, "no problem of that degree");
  cudaDeviceSynchronize();
  BatchPrec& P = batch->prec[pi];
  DegreeKnobs& kn = P.knobs[degree];
  kn.shape = tile_shape;
  kn.face_batch = face_batch;
  kn.tc = tensor_cores;
  for (size_t k = 0; k < batch->probs.size(); ++k)
    if (batch->probs[k]->hp.p == degree) P.shape[k] = tile_shape;
  P.dirty = true;
  drop_graphs(P);
  return SBM_OK;
}

int sbm_batch_device_status(sbm_batch* batch) {
  if (!batch) return sbm_fail_detail(SBM_ERR_ARG, "NULL batch");
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return sbm_cuda_fail_detail(e, "synchronize");
  int h = 0;
  if ((e = cudaMemcpy(&h, batch->err, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess)
    return sbm_cuda_fail_detail(e, "status read");
  if (h != 0) {
    cudaMemset(batch->err, 0, sizeof(int));
    return sbm_fail_detail(h, "a bounded device wait of the batched apply expired");
  }
  return SBM_OK;
}

void sbm_batch_destroy(sbm_batch* batch) {
  if (batch) destroy(batch);
}

}  // extern "C"

// Failure path of the persistent kernel (a diagnostic; no fault, no hang):
// one launch whose only item is a chunk item of a system that expects one
// face item that the work list does not contain, so its dependency wait
// can never be satisfied and expires (about a second); the kernel records
// SBM_ERR_TIMEOUT in the batch's error word and returns before touching any
// vector.  Synchronous; the status is then read by sbm_batch_device_status.
extern "C" int sbm_batch_selftest_timeout(sbm_batch* batch, void* stream) {
  if (!batch) return sbm_fail_detail(SBM_ERR_ARG, "NULL batch");
  std::unique_ptr<bk::ProbTable<float>> tab(new (std::nothrow) bk::ProbTable<float>);
  if (!tab) return sbm_fail_detail(SBM_ERR_OOM, "host allocation failed");
  std::memset((void*)tab.get(), 0, sizeof(*tab));
  tab->p[0].n_face_items = 1;   // never produced
  tab->p[0].code = bk::code_of(3, 5, 0, 0, 0);
  const Item it{0, bk::kChunk, 0, 1};
  void* di = nullptr;
  int* cnt = nullptr;
  cudaError_t e = cudaMalloc(&di, sizeof(it));
  if (e == cudaSuccess) e = cudaMalloc((void**)&cnt, 3 * sizeof(int));
  if (e == cudaSuccess) e = cudaMemcpy(di, &it, sizeof(it), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, 3 * sizeof(int), (cudaStream_t)stream);
  if (e == cudaSuccess)
    e = bk::launch(*tab, static_cast<const Item*>(di), 1, 1, 1, cnt, batch->err, 0, 1, 0,
                   (cudaStream_t)stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
  cudaFree(di);
  cudaFree(cnt);
  if (e != cudaSuccess) return sbm_cuda_fail_detail(e, "sbm_batch_selftest_timeout");
  return SBM_OK;
}
