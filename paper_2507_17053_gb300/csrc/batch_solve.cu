// Batched solves: every (problem, right-hand side) system of a batch runs its
// own BiCGStab iteration -- its own scalars, residual tests and stopping --
// but the iterations advance together, so that each step costs one batched
// apply (sbm_batch_apply_*: all problems and right-hand sides in one graph
// launch) and one launch per vector operation over the concatenated vectors.
//
// The paper states no solver (Section 4.2 only notes that the mat-vec
// dominates iterative solvers); this drives the batched operator.
//
// Layout: the systems' vectors are concatenated in problem order, right-hand
// side r of problem k at off[k] + r n_k -- the layout sbm_batch_apply takes
// per problem.  Reductions: each system's segment is cut into tiles of at
// most kTile elements (a tile never spans two systems); a block sums one
// tile in a fixed tree order and one warp per system adds its tiles' partial
// sums in order, so a solve is bitwise reproducible.  Per-system state
// (FP64 scalars, status) stays on the device; the host reads it once per
// kChunk iterations.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "batch.hpp"

using namespace sbm;

namespace {

constexpr int kTile = 4096;      // elements per reduction tile
constexpr int kThr = 256;        // threads per tile block
constexpr int kChunk = 8;        // iterations between host reads of the state
constexpr int kFinishRestarts = 20;
constexpr int kFinishMaxit = 20000;   // FP64 finish of the refinement, at most

// per-system BiCGStab state
struct BSys {
  double rho, alpha, omega, beta, rr, bb, tol2, best;
  int done;      // 0 running, 1 converged, 2 breakdown / divergence, 3 iteration cap, 4 idle
  int iters, maxit, improved;
};

struct Tiles {
  const int32_t* sys;     // [ntile] system of the tile
  const int64_t* start;   // [ntile] first element
  const int32_t* len;     // [ntile] elements
  const int32_t* first;   // [nsys + 1] first tile of each system
  int ntile, nsys;
};

// sum over the block (thread 0 gets it), fixed order
__device__ __forceinline__ double tile_sum(double v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < kThr / 32; ++w) r += sh[w];
  return r;
}

// the tiles' partial sums j = 0..ND-1 of system s, summed in tile order (all lanes)
template <int ND>
__device__ __forceinline__ void sys_sums(const double* __restrict__ part, const Tiles& m, int s,
                                         double (&v)[ND]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int j = 0; j < ND; ++j) {
    double a = 0.0;
    for (int t = m.first[s] + lane; t < m.first[s + 1]; t += 32) a += part[(size_t)j * m.ntile + t];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    v[j] = a;
  }
}

#define TILE_HEAD                                        \
  const int tile = blockIdx.x;                           \
  const int sy = m.sys[tile];                            \
  const int64_t i0 = m.start[tile], i1 = i0 + m.len[tile];
#define SYS_HEAD                                                                \
  const int s = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5); \
  if (s >= m.nsys) return;                                                      \
  const bool lead = (threadIdx.x & 31) == 0;

// r = b - q (q = A x; null for x = 0); r^ = r; p = r; partial (r, r), (b, b)
__global__ void k_init(const Tiles m, const double* __restrict__ b, const double* __restrict__ q,
                       double* __restrict__ r, double* __restrict__ rh, double* __restrict__ p,
                       const BSys* __restrict__ st, double* __restrict__ part) {
  __shared__ double sh[kThr / 32];
  TILE_HEAD
  if (st[sy].done) return;
  double rr = 0.0, bb = 0.0;
  for (int64_t i = i0 + threadIdx.x; i < i1; i += kThr) {
    const double ri = q ? b[i] - q[i] : b[i];
    r[i] = ri;
    rh[i] = ri;
    p[i] = ri;
    rr = fma(ri, ri, rr);
    bb = fma(b[i], b[i], bb);
  }
  rr = tile_sum(rr, sh);
  bb = tile_sum(bb, sh);
  if (threadIdx.x == 0) {
    part[tile] = rr;
    part[m.ntile + tile] = bb;
  }
}

__global__ void k_fin_init(const Tiles m, const double* __restrict__ part, BSys* st) {
  SYS_HEAD
  if (st[s].done) return;
  double v[2];
  sys_sums<2>(part, m, s, v);
  if (lead) {
    BSys& y = st[s];
    y.rr = v[0];
    y.bb = v[1];
    y.best = INFINITY;           // the first chunk end keeps this iterate
    y.rho = v[0];
    y.alpha = y.omega = 1.0;
    y.beta = 0.0;
    y.done = (v[0] <= y.tol2 * v[1]) ? 1 : 0;
    if (!isfinite(v[0])) y.done = 2;
    if (y.maxit <= 0 && !y.done) y.done = 3;
  }
}

// partial (r^, v)
__global__ void k_dot_rv(const Tiles m, const double* __restrict__ rh,
                         const double* __restrict__ v, const BSys* __restrict__ st,
                         double* __restrict__ part) {
  __shared__ double sh[kThr / 32];
  TILE_HEAD
  if (st[sy].done) return;
  double a = 0.0;
  for (int64_t i = i0 + threadIdx.x; i < i1; i += kThr) a = fma(rh[i], v[i], a);
  a = tile_sum(a, sh);
  if (threadIdx.x == 0) part[tile] = a;
}

// alpha = rho / (r^, v)
__global__ void k_fin_alpha(const Tiles m, const double* __restrict__ part, BSys* st) {
  SYS_HEAD
  if (st[s].done) return;
  double v[1];
  sys_sums<1>(part, m, s, v);
  if (lead) {
    if (!(v[0] != 0.0) || !isfinite(v[0])) st[s].done = 2;
    else st[s].alpha = st[s].rho / v[0];
  }
}

// s = r - alpha v
__global__ void k_sv(const Tiles m, const double* __restrict__ r, const double* __restrict__ v,
                     double* __restrict__ sv, const BSys* __restrict__ st) {
  TILE_HEAD
  if (st[sy].done) return;
  const double al = st[sy].alpha;
  for (int64_t i = i0 + threadIdx.x; i < i1; i += kThr) sv[i] = fma(-al, v[i], r[i]);
}

// partial (t, s), (t, t)
__global__ void k_dot_ts(const Tiles m, const double* __restrict__ t,
                         const double* __restrict__ sv, const BSys* __restrict__ st,
                         double* __restrict__ part) {
  __shared__ double sh[kThr / 32];
  TILE_HEAD
  if (st[sy].done) return;
  double ts = 0.0, tt = 0.0;
  for (int64_t i = i0 + threadIdx.x; i < i1; i += kThr) {
    ts = fma(t[i], sv[i], ts);
    tt = fma(t[i], t[i], tt);
  }
  ts = tile_sum(ts, sh);
  tt = tile_sum(tt, sh);
  if (threadIdx.x == 0) {
    part[tile] = ts;
    part[m.ntile + tile] = tt;
  }
}

// omega = (t, s) / (t, t)  (0 when t = 0)
__global__ void k_fin_omega(const Tiles m, const double* __restrict__ part, BSys* st) {
  SYS_HEAD
  if (st[s].done) return;
  double v[2];
  sys_sums<2>(part, m, s, v);
  if (lead) {
    st[s].omega = (v[1] > 0.0) ? v[0] / v[1] : 0.0;
    if (!isfinite(st[s].omega)) st[s].done = 2;
  }
}

// x += alpha p + omega s; r = s - omega t; partial (r^, r), (r, r)
__global__ void k_update(const Tiles m, double* __restrict__ x, double* __restrict__ r,
                         const double* __restrict__ p, const double* __restrict__ sv,
                         const double* __restrict__ t, const double* __restrict__ rh,
                         const BSys* __restrict__ st, double* __restrict__ part) {
  __shared__ double sh[kThr / 32];
  TILE_HEAD
  if (st[sy].done) return;
  const double al = st[sy].alpha, om = st[sy].omega;
  double a = 0.0, c = 0.0;
  for (int64_t i = i0 + threadIdx.x; i < i1; i += kThr) {
    const double si = sv[i];
    x[i] = fma(om, si, fma(al, p[i], x[i]));
    const double ri = fma(-om, t[i], si);
    r[i] = ri;
    a = fma(rh[i], ri, a);
    c = fma(ri, ri, c);
  }
  a = tile_sum(a, sh);
  c = tile_sum(c, sh);
  if (threadIdx.x == 0) {
    part[tile] = a;
    part[m.ntile + tile] = c;
  }
}

// rho' = (r^, r); tests; beta = (rho' / rho)(alpha / omega)
__global__ void k_fin_beta(const Tiles m, const double* __restrict__ part, BSys* st) {
  SYS_HEAD
  if (st[s].done) return;
  double v[2];
  sys_sums<2>(part, m, s, v);
  if (lead) {
    BSys& y = st[s];
    y.iters += 1;
    y.rr = v[1];
    if (v[1] <= y.tol2 * y.bb) y.done = 1;
    else if (!isfinite(v[1]) || v[1] > 1e24 * y.bb) y.done = 2;
    else if (!(v[0] != 0.0) || !(y.omega != 0.0)) y.done = 2;
    else if (y.iters >= y.maxit) y.done = 3;
    if (!y.done) {
      y.beta = (v[0] / y.rho) * (y.alpha / y.omega);
      y.rho = v[0];
    }
  }
}

// p = r + beta (p - omega v)
__global__ void k_pv(const Tiles m, double* __restrict__ p, const double* __restrict__ r,
                     const double* __restrict__ v, const BSys* __restrict__ st) {
  TILE_HEAD
  if (st[sy].done) return;
  const double be = st[sy].beta, om = st[sy].omega;
  for (int64_t i = i0 + threadIdx.x; i < i1; i += kThr) p[i] = fma(be, fma(-om, v[i], p[i]), r[i]);
}

// improved = (finite rr below the best so far); best = min(best, rr)
__global__ void k_mark_best(BSys* st, int nsys) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nsys) return;
  BSys& y = st[s];
  y.improved = (y.done != 4 && isfinite(y.rr) && y.rr < y.best) ? 1 : 0;
  if (y.improved) y.best = y.rr;
}

// xb = x on the systems whose residual improved
__global__ void k_keep_best(const Tiles m, const double* __restrict__ x, double* __restrict__ xb,
                            const BSys* __restrict__ st) {
  TILE_HEAD
  if (!st[sy].improved) return;
  for (int64_t i = i0 + threadIdx.x; i < i1; i += kThr) xb[i] = x[i];
}

// x = xb on the systems that stopped worse than their best iterate
__global__ void k_restore_best(const Tiles m, double* __restrict__ x,
                               const double* __restrict__ xb, const BSys* __restrict__ st) {
  TILE_HEAD
  const BSys& y = st[sy];
  if (y.done == 4 || y.done == 1 || y.rr <= y.best) return;
  for (int64_t i = i0 + threadIdx.x; i < i1; i += kThr) x[i] = xb[i];
}

// partial (b - q, b - q), (b, b)
__global__ void k_resid_dots(const Tiles m, const double* __restrict__ b,
                             const double* __restrict__ q, double* __restrict__ r,
                             double* __restrict__ part) {
  __shared__ double sh[kThr / 32];
  TILE_HEAD
  (void)sy;
  double rr = 0.0, bb = 0.0;
  for (int64_t i = i0 + threadIdx.x; i < i1; i += kThr) {
    const double ri = q ? b[i] - q[i] : b[i];
    if (r) r[i] = ri;
    rr = fma(ri, ri, rr);
    bb = fma(b[i], b[i], bb);
  }
  rr = tile_sum(rr, sh);
  bb = tile_sum(bb, sh);
  if (threadIdx.x == 0) {
    part[tile] = rr;
    part[m.ntile + tile] = bb;
  }
}

__global__ void k_fin_sums2(const Tiles m, const double* __restrict__ part,
                            double* __restrict__ out) {
  SYS_HEAD
  double v[2];
  sys_sums<2>(part, m, s, v);
  if (lead) {
    out[s] = v[0];
    out[m.nsys + s] = v[1];
  }
}

// x += d on the systems with use[s] != 0
__global__ void k_add_masked(const Tiles m, double* __restrict__ x, const double* __restrict__ d,
                             const int32_t* __restrict__ use) {
  TILE_HEAD
  if (!use[sy]) return;
  for (int64_t i = i0 + threadIdx.x; i < i1; i += kThr) x[i] += d[i];
}

__global__ void k_to_f32(const double* __restrict__ a, float* __restrict__ o, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    o[i] = (float)a[i];
}

__global__ void k_to_f64(const float* __restrict__ a, double* __restrict__ o, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    o[i] = (double)a[i];
}

int grid_of(int64_t n) { return (int)std::min<int64_t>((n + 255) / 256, 152 * 16); }
int sys_grid(int nsys) { return (nsys * 32 + 255) / 256; }

struct Ctx {
  sbm_batch* B;
  BatchSolveWs& w;
  Tiles m;
  cudaStream_t st;
  int nsys;
};

// pointer array of a concatenated vector, one entry per problem
template <typename T>
std::vector<T*> per_problem(const BatchSolveWs& w, T* base) {
  std::vector<T*> v(w.off.size());
  for (size_t k = 0; k < w.off.size(); ++k) v[k] = base + w.off[k];
  return v;
}

// out = A in for every system: FP64 applies, or FP32 applies on the rounded
// input (mixed)
int apply(Ctx& c, bool mixed, const double* in, double* out) {
  BatchSolveWs& w = c.w;
  if (mixed) {
    k_to_f32<<<grid_of(w.n), 256, 0, c.st>>>(in, w.a32, w.n);
    const std::vector<float*> xa = per_problem<float>(w, w.a32), ya = per_problem<float>(w, w.b32);
    std::vector<const float*> xc(xa.begin(), xa.end());
    int s = sbm_batch_apply_f32(c.B, xc.data(), ya.data(), c.st);
    if (s != SBM_OK) return s;
    k_to_f64<<<grid_of(w.n), 256, 0, c.st>>>(w.b32, out, w.n);
  } else {
    const std::vector<double*> xa = per_problem<double>(w, const_cast<double*>(in)),
                               ya = per_problem<double>(w, out);
    std::vector<const double*> xc(xa.begin(), xa.end());
    int s = sbm_batch_apply_f64(c.B, xc.data(), ya.data(), c.st);
    if (s != SBM_OK) return s;
  }
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SBM_OK : sbm_cuda_fail_detail(e, "batch solve");
}

#define CKS(x)                       \
  do {                               \
    int s_ = (x);                    \
    if (s_ != SBM_OK) return s_;     \
  } while (0)
#define CKC(x, where)                                          \
  do {                                                         \
    cudaError_t e_ = (x);                                      \
    if (e_ != cudaSuccess) return sbm_cuda_fail_detail(e_, where); \
  } while (0)

// BiCGStab on every system with active[s] != 0: A xs = bs to |r| <= rtol |bs|
// or maxit iterations, from xs = 0 (x_zero) or the given xs; the others are
// left alone.  Ends with each system at its iterate of least recursive
// residual among the chunk ends (unless converged).  Host copy of the final
// states in hs.
int bicgstab(Ctx& c, bool mixed, const double* bs, double* xs, bool x_zero, double rtol,
             int maxit, const std::vector<char>& active, std::vector<BSys>& hs) {
  BatchSolveWs& w = c.w;
  const Tiles& m = c.m;
  BSys* dst = (BSys*)w.state;
  hs.assign(c.nsys, BSys{});
  for (int s = 0; s < c.nsys; ++s) {
    hs[s].tol2 = rtol * rtol;
    hs[s].maxit = maxit;
    hs[s].done = active[s] ? 0 : 4;
  }
  CKC(cudaMemcpyAsync(dst, hs.data(), sizeof(BSys) * c.nsys, cudaMemcpyHostToDevice, c.st),
      "state upload");
  if (x_zero) CKC(cudaMemsetAsync(xs, 0, (size_t)w.n * 8, c.st), "memset");
  else CKS(apply(c, mixed, xs, w.v));
  k_init<<<m.ntile, kThr, 0, c.st>>>(m, bs, x_zero ? nullptr : w.v, w.r, w.rh, w.p, dst, w.part);
  k_fin_init<<<sys_grid(c.nsys), 256, 0, c.st>>>(m, w.part, dst);
  while (true) {
    k_mark_best<<<(c.nsys + 255) / 256, 256, 0, c.st>>>(dst, c.nsys);
    k_keep_best<<<m.ntile, kThr, 0, c.st>>>(m, xs, w.xb, dst);
    CKC(cudaMemcpyAsync(w.hstate, dst, sizeof(BSys) * c.nsys, cudaMemcpyDeviceToHost, c.st),
        "state read");
    CKC(cudaStreamSynchronize(c.st), "sync");
    const BSys* h = (const BSys*)w.hstate;
    bool running = false;
    for (int s = 0; s < c.nsys; ++s) running |= h[s].done == 0;
    if (!running) break;
    for (int it = 0; it < kChunk; ++it) {
      CKS(apply(c, mixed, w.p, w.v));
      k_dot_rv<<<m.ntile, kThr, 0, c.st>>>(m, w.rh, w.v, dst, w.part);
      k_fin_alpha<<<sys_grid(c.nsys), 256, 0, c.st>>>(m, w.part, dst);
      k_sv<<<m.ntile, kThr, 0, c.st>>>(m, w.r, w.v, w.s, dst);
      CKS(apply(c, mixed, w.s, w.t));
      k_dot_ts<<<m.ntile, kThr, 0, c.st>>>(m, w.t, w.s, dst, w.part);
      k_fin_omega<<<sys_grid(c.nsys), 256, 0, c.st>>>(m, w.part, dst);
      k_update<<<m.ntile, kThr, 0, c.st>>>(m, xs, w.r, w.p, w.s, w.t, w.rh, dst, w.part);
      k_fin_beta<<<sys_grid(c.nsys), 256, 0, c.st>>>(m, w.part, dst);
      k_pv<<<m.ntile, kThr, 0, c.st>>>(m, w.p, w.r, w.v, dst);
    }
    CKC(cudaGetLastError(), "bicgstab launch");
  }
  k_restore_best<<<m.ntile, kThr, 0, c.st>>>(m, xs, w.xb, dst);
  CKC(cudaMemcpyAsync(hs.data(), dst, sizeof(BSys) * c.nsys, cudaMemcpyDeviceToHost, c.st),
      "state read");
  CKC(cudaStreamSynchronize(c.st), "sync");
  return SBM_OK;
}

// true residuals: rr[s] = |b - A x|^2, bb[s] = |b|^2 (r = b - A x when r != null)
int residuals(Ctx& c, const double* x, double* r, std::vector<double>& rr,
              std::vector<double>& bb, bool x_zero) {
  BatchSolveWs& w = c.w;
  if (!x_zero) CKS(apply(c, false, x, w.v));
  k_resid_dots<<<c.m.ntile, kThr, 0, c.st>>>(c.m, w.b, x_zero ? nullptr : w.v, r, w.part);
  k_fin_sums2<<<sys_grid(c.nsys), 256, 0, c.st>>>(c.m, w.part, w.sums);
  std::vector<double> h(2 * c.nsys);
  CKC(cudaMemcpyAsync(h.data(), w.sums, 16 * (size_t)c.nsys, cudaMemcpyDeviceToHost, c.st),
      "residual read");
  CKC(cudaStreamSynchronize(c.st), "sync");
  rr.assign(h.begin(), h.begin() + c.nsys);
  bb.assign(h.begin() + c.nsys, h.end());
  return SBM_OK;
}

cudaError_t ensure_ws(sbm_batch* B) {
  BatchSolveWs& w = B->ws;
  if (!w.bufs.empty()) return cudaSuccess;
  const int nprob = (int)B->probs.size(), nrhs = B->nrhs;
  w.off.assign(nprob, 0);
  std::vector<int32_t> tsys, tlen, tfirst;
  std::vector<int64_t> tstart;
  int64_t n = 0;
  int sys = 0;
  for (int k = 0; k < nprob; ++k) {
    w.off[k] = n;
    const int64_t nk = B->probs[k]->hp.n_dofs;
    for (int r = 0; r < nrhs; ++r, ++sys) {
      tfirst.push_back((int32_t)tsys.size());
      for (int64_t i = 0; i < nk; i += kTile) {
        tsys.push_back(sys);
        tstart.push_back(n + i);
        tlen.push_back((int32_t)std::min<int64_t>(kTile, nk - i));
      }
      n += nk;
    }
  }
  tfirst.push_back((int32_t)tsys.size());
  w.n = n;
  w.nsys = sys;
  w.ntile = (int)tsys.size();
  auto alloc = [&](void** p, size_t bytes) {
    cudaError_t e = cudaMalloc(p, bytes > 0 ? bytes : 1);
    if (e == cudaSuccess) w.bufs.push_back(*p);
    return e;
  };
  double** v64[] = {&w.b, &w.x, &w.rout, &w.d, &w.r, &w.rh, &w.p, &w.v, &w.s, &w.t, &w.xb};
  cudaError_t e;
  for (double** p : v64)
    if ((e = alloc((void**)p, (size_t)n * 8)) != cudaSuccess) return e;
  if ((e = alloc((void**)&w.a32, (size_t)n * 4)) != cudaSuccess ||
      (e = alloc((void**)&w.b32, (size_t)n * 4)) != cudaSuccess ||
      (e = alloc((void**)&w.part, (size_t)3 * w.ntile * 8)) != cudaSuccess ||
      (e = alloc((void**)&w.sums, (size_t)2 * w.nsys * 8)) != cudaSuccess ||
      (e = alloc((void**)&w.use, (size_t)w.nsys * 4)) != cudaSuccess ||
      (e = alloc(&w.state, sizeof(BSys) * w.nsys)) != cudaSuccess ||
      (e = alloc((void**)&w.tsys, 4 * tsys.size())) != cudaSuccess ||
      (e = alloc((void**)&w.tlen, 4 * tlen.size())) != cudaSuccess ||
      (e = alloc((void**)&w.tstart, 8 * tstart.size())) != cudaSuccess ||
      (e = alloc((void**)&w.tfirst, 4 * tfirst.size())) != cudaSuccess)
    return e;
  if ((e = cudaMallocHost(&w.hstate, sizeof(BSys) * w.nsys)) != cudaSuccess) return e;
  if ((e = cudaMemcpy(w.tsys, tsys.data(), 4 * tsys.size(), cudaMemcpyHostToDevice)) !=
          cudaSuccess ||
      (e = cudaMemcpy(w.tlen, tlen.data(), 4 * tlen.size(), cudaMemcpyHostToDevice)) !=
          cudaSuccess ||
      (e = cudaMemcpy(w.tstart, tstart.data(), 8 * tstart.size(), cudaMemcpyHostToDevice)) !=
          cudaSuccess ||
      (e = cudaMemcpy(w.tfirst, tfirst.data(), 4 * tfirst.size(), cudaMemcpyHostToDevice)) !=
          cudaSuccess)
    return e;
  return cudaSuccess;
}

}  // namespace

void batch_solve_release(sbm_batch* B) {
  BatchSolveWs& w = B->ws;
  for (void* p : w.bufs) cudaFree(p);
  if (w.hstate) cudaFreeHost(w.hstate);
  w = BatchSolveWs();
}

extern "C" int sbm_batch_solve(sbm_batch* batch, const double* const* b, double* const* x,
                               int mode, double rtol, int maxit, double inner_rtol,
                               int inner_maxit, int* iters, double* relres, int* outer,
                               void* stream) {
  if (!batch || !b || !x) return sbm_fail_detail(SBM_ERR_ARG, "NULL argument");
  if (mode != SBM_BATCH_SOLVE_FP64 && mode != SBM_BATCH_SOLVE_MIXED)
    return sbm_fail_detail(SBM_ERR_ARG, "unknown batch solve mode");
  if (!(rtol > 0.0) || maxit < 1 ||
      (mode == SBM_BATCH_SOLVE_MIXED && (!(inner_rtol > 0.0) || inner_rtol >= 1.0 || inner_maxit < 1)))
    return sbm_fail_detail(SBM_ERR_ARG, "bad tolerance or iteration limit");
  const int nprob = (int)batch->probs.size();
  for (int k = 0; k < nprob; ++k)
    if (!b[k] || !x[k]) return sbm_fail_detail(SBM_ERR_ARG, "NULL vector");
  int dev = -1;
  cudaGetDevice(&dev);
  if (dev != batch->device) return sbm_fail_detail(SBM_ERR_STATE, "current device is not the batch's");
  cudaError_t e = ensure_ws(batch);
  if (e != cudaSuccess) {
    batch_solve_release(batch);
    return e == cudaErrorMemoryAllocation ? sbm_fail_detail(SBM_ERR_OOM, "batch solve workspace")
                                          : sbm_cuda_fail_detail(e, "batch solve workspace");
  }
  BatchSolveWs& w = batch->ws;
  Ctx c{batch, w, Tiles{w.tsys, w.tstart, w.tlen, w.tfirst, w.ntile, w.nsys},
        (cudaStream_t)stream, w.nsys};
  const int nrhs = batch->nrhs;
  for (int k = 0; k < nprob; ++k)
    CKC(cudaMemcpyAsync(w.b + w.off[k], b[k], (size_t)nrhs * batch->probs[k]->hp.n_dofs * 8,
                        cudaMemcpyDeviceToDevice, c.st),
        "rhs copy");
  std::vector<int> its(c.nsys, 0);
  std::vector<BSys> hs;
  std::vector<double> rr, bb;
  std::vector<char> conv(c.nsys, 0), active(c.nsys, 1);
  int nouter = 0;
  CKC(cudaMemsetAsync(w.x, 0, (size_t)w.n * 8, c.st), "memset");
  if (mode == SBM_BATCH_SOLVE_MIXED) {
    // FP64 refinement around inner BiCGStab solves with FP32 applies
    std::vector<double> prev(c.nsys, INFINITY);
    std::vector<int32_t> use(c.nsys, 0);
    for (int o = 0; o < maxit; ++o) {
      CKS(residuals(c, w.x, w.rout, rr, bb, o == 0));
      bool any = false;
      for (int s = 0; s < c.nsys; ++s) {
        const double rel = bb[s] > 0.0 ? std::sqrt(rr[s] / bb[s]) : 0.0;
        conv[s] = rel <= rtol;
        // a system whose residual no longer halves leaves the refinement
        if (!conv[s] && !(rel <= 0.5 * prev[s])) active[s] = 0;
        if (conv[s]) active[s] = 0;
        prev[s] = rel;
        any |= active[s] != 0;
      }
      if (!any) break;
      CKS(bicgstab(c, true, w.rout, w.d, true, inner_rtol, inner_maxit, active, hs));
      for (int s = 0; s < c.nsys; ++s) {
        its[s] += hs[s].iters;
        // keep the correction only where the inner solve reduced its residual
        use[s] = active[s] && std::isfinite(hs[s].best) && std::min(hs[s].rr, hs[s].best) < hs[s].bb;
      }
      CKC(cudaMemcpyAsync(w.use, use.data(), 4 * (size_t)c.nsys, cudaMemcpyHostToDevice, c.st),
          "mask upload");
      k_add_masked<<<c.m.ntile, kThr, 0, c.st>>>(c.m, w.x, w.d, w.use);
      CKC(cudaGetLastError(), "refinement update");
      nouter++;
    }
    CKS(residuals(c, w.x, nullptr, rr, bb, false));
    for (int s = 0; s < c.nsys; ++s)
      conv[s] = bb[s] == 0.0 || std::sqrt(rr[s] / bb[s]) <= rtol;
  }
  // FP64 BiCGStab on the systems not converged, from their current x;
  // after a breakdown or divergence it restarts from the best iterate
  for (int rs = 0; rs <= kFinishRestarts; ++rs) {
    bool any = false;
    for (int s = 0; s < c.nsys; ++s) {
      active[s] = conv[s] == 0;
      any |= active[s] != 0;
    }
    if (!any) break;
    const bool zero = mode == SBM_BATCH_SOLVE_FP64 && rs == 0;
    const int cap = mode == SBM_BATCH_SOLVE_FP64
                        ? maxit
                        : (int)std::min<int64_t>(kFinishMaxit, (int64_t)maxit * inner_maxit);
    CKS(bicgstab(c, false, w.b, w.x, zero, rtol, cap, active, hs));
    CKS(residuals(c, w.x, nullptr, rr, bb, false));
    // restart (fresh shadow residual, from the current iterate) a system
    // that broke down, or whose recursive residual met rtol but whose true
    // residual does not, while its iteration budget lasts
    bool retry = false;
    for (int s = 0; s < c.nsys; ++s) {
      if (!active[s]) continue;
      its[s] += hs[s].iters;
      if (bb[s] == 0.0 || std::sqrt(rr[s] / bb[s]) <= rtol) conv[s] = 1;
      else if (hs[s].done == 3 || its[s] >= cap) conv[s] = 2;     // budget spent
      else retry = true;
    }
    if (!retry) break;
  }
  CKS(residuals(c, w.x, nullptr, rr, bb, false));
  bool all = true;
  for (int s = 0; s < c.nsys; ++s) {
    const double rel = bb[s] > 0.0 ? std::sqrt(rr[s] / bb[s]) : 0.0;
    if (relres) relres[s] = rel;
    if (iters) iters[s] = its[s];
    all &= rel <= rtol;
  }
  if (outer) *outer = nouter;
  for (int k = 0; k < nprob; ++k)
    CKC(cudaMemcpyAsync(x[k], w.x + w.off[k], (size_t)nrhs * batch->probs[k]->hp.n_dofs * 8,
                        cudaMemcpyDeviceToDevice, c.st),
        "solution copy");
  CKC(cudaStreamSynchronize(c.st), "sync");
  return all ? SBM_OK : sbm_fail_detail(SBM_ERR_NOT_CONVERGED, "batch solve: a system above rtol");
}
