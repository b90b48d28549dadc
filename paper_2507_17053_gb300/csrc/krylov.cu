// Krylov drivers on the matrix-free operator: conjugate gradients, restarted
// GMRES, and FP64 iterative refinement around an FP32 inner solve.
//
// The paper gives no solver; it states that the mat-vec dominates iterative
// solvers (Section 4.2).  These drivers keep every vector on the device:
//  * reductions are deterministic (fixed grid, fixed tree order, FP64
//    accumulation), so a solve is bitwise reproducible;
//  * CG keeps its scalars on the device and runs CG_CHUNK iterations per
//    CUDA-graph launch; a converged/failed flag turns the remaining
//    iterations of a chunk into no-ops, and the host reads the state once
//    per chunk;
//  * GMRES(m) orthogonalises with classical Gram-Schmidt applied twice
//    (CGS2) and keeps the small Hessenberg least-squares problem (Givens
//    rotations) on the host, one short read per Arnoldi step.
#include <cmath>
#include <functional>
#include <vector>

#include "internal.hpp"
#include "krylov.hpp"

namespace sbm {

constexpr int RED_BLOCKS = 1216;   // 8 x 152 SMs
constexpr int RED_THREADS = 256;
constexpr int CG_CHUNK = 16;

// ---- deterministic reductions ---------------------------------------------

__device__ __forceinline__ double block_sum(double v, double* sh) {
  const int tid = threadIdx.x;
  sh[tid] = v;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (tid < s) sh[tid] += sh[tid + s];
    __syncthreads();
  }
  const double r = sh[0];
  __syncthreads();
  return r;
}

// part[j * RED_BLOCKS + block] = partial sum of a_j . b over this block's rows,
// a_j = a + j * lda (blockIdx.y = j).
template <typename T>
__global__ void k_multi_dot(const T* __restrict__ a, int64_t lda, const T* __restrict__ b,
                            int64_t n, double* __restrict__ part) {
  __shared__ double sh[RED_THREADS];
  const T* aj = a + (int64_t)blockIdx.y * lda;
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    s = fma((double)aj[i], (double)b[i], s);
  s = block_sum(s, sh);
  if (threadIdx.x == 0) part[blockIdx.y * RED_BLOCKS + blockIdx.x] = s;
}

// out[j] = sum of part[j * RED_BLOCKS + 0 .. RED_BLOCKS-1] (blockIdx.x = j)
__global__ void k_finalize(const double* __restrict__ part, double* __restrict__ out) {
  __shared__ double sh[RED_THREADS];
  double s = 0.0;
  for (int i = threadIdx.x; i < RED_BLOCKS; i += blockDim.x) s += part[blockIdx.x * RED_BLOCKS + i];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) out[blockIdx.x] = s;
}

// ---- CG -----------------------------------------------------------------

struct CgState {
  double rz, pq, alpha, beta, rr, bb, tol2;
  int done;     // 0 running, 1 converged (recursive residual), 2 breakdown/divergence, 3 maxit
  int iters;
  int maxit;
};

// r = b - q; z = dinv * r (or r); p = z; partials of r.z, r.r, b.b
__global__ void k_cg_init(const double* __restrict__ b, const double* __restrict__ q,
                          double* __restrict__ r, double* __restrict__ z, double* __restrict__ p,
                          const double* __restrict__ dinv, int64_t n, double* __restrict__ part) {
  __shared__ double sh[RED_THREADS];
  double srz = 0.0, srr = 0.0, sbb = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double ri = b[i] - q[i];
    const double zi = dinv ? ri * dinv[i] : ri;
    r[i] = ri;
    z[i] = zi;
    p[i] = zi;
    srz = fma(ri, zi, srz);
    srr = fma(ri, ri, srr);
    sbb = fma(b[i], b[i], sbb);
  }
  srz = block_sum(srz, sh);
  srr = block_sum(srr, sh);
  sbb = block_sum(sbb, sh);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = srz;
    part[RED_BLOCKS + blockIdx.x] = srr;
    part[2 * RED_BLOCKS + blockIdx.x] = sbb;
  }
}

__global__ void k_cg_init_fin(const double* __restrict__ part, CgState* st) {
  __shared__ double sh[RED_THREADS];
  double v[3];
  for (int j = 0; j < 3; ++j) {
    double s = 0.0;
    for (int i = threadIdx.x; i < RED_BLOCKS; i += blockDim.x) s += part[j * RED_BLOCKS + i];
    v[j] = block_sum(s, sh);
  }
  if (threadIdx.x == 0) {
    st->rz = v[0];
    st->rr = v[1];
    st->bb = v[2];
    st->done = (v[1] <= st->tol2 * v[2]) ? 1 : 0;
    if (!(v[0] == v[0]) || v[2] == 0.0) st->done = (v[2] == 0.0) ? 1 : 2;
  }
}

__global__ void k_cg_alpha(const double* __restrict__ part, CgState* st) {
  __shared__ double sh[RED_THREADS];
  double s = 0.0;
  for (int i = threadIdx.x; i < RED_BLOCKS; i += blockDim.x) s += part[i];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) {
    st->pq = s;
    if (st->done) {
      st->alpha = 0.0;
    } else if (!(s != 0.0) || !isfinite(s)) {
      st->alpha = 0.0;
      st->done = 2;
    } else {
      st->alpha = st->rz / s;
    }
  }
}

// x += alpha p; r -= alpha q; z = dinv r; partials of r.z, r.r
__global__ void k_cg_update(double* __restrict__ x, double* __restrict__ r, double* __restrict__ z,
                            const double* __restrict__ p, const double* __restrict__ q,
                            const double* __restrict__ dinv, int64_t n, const CgState* st,
                            double* __restrict__ part) {
  __shared__ double sh[RED_THREADS];
  const double al = st->alpha;
  double srz = 0.0, srr = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    x[i] = fma(al, p[i], x[i]);
    const double ri = fma(-al, q[i], r[i]);
    const double zi = dinv ? ri * dinv[i] : ri;
    r[i] = ri;
    z[i] = zi;
    srz = fma(ri, zi, srz);
    srr = fma(ri, ri, srr);
  }
  srz = block_sum(srz, sh);
  srr = block_sum(srr, sh);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = srz;
    part[RED_BLOCKS + blockIdx.x] = srr;
  }
}

__global__ void k_cg_beta(const double* __restrict__ part, CgState* st) {
  __shared__ double sh[RED_THREADS];
  double v[2];
  for (int j = 0; j < 2; ++j) {
    double s = 0.0;
    for (int i = threadIdx.x; i < RED_BLOCKS; i += blockDim.x) s += part[j * RED_BLOCKS + i];
    v[j] = block_sum(s, sh);
  }
  if (threadIdx.x == 0) {
    if (st->done) {
      st->beta = 0.0;
    } else {
      st->iters += 1;
      st->rr = v[1];
      if (v[1] <= st->tol2 * st->bb) st->done = 1;
      else if (!isfinite(v[1]) || v[1] > 1e24 * st->bb || !(v[0] != 0.0)) st->done = 2;
      else if (st->iters >= st->maxit) st->done = 3;
      st->beta = v[0] / st->rz;
      st->rz = v[0];
      if (st->done) st->beta = 0.0;
    }
  }
}

__global__ void k_cg_p(double* __restrict__ p, const double* __restrict__ z, int64_t n,
                       const CgState* st) {
  if (st->done) return;
  const double be = st->beta;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    p[i] = fma(be, p[i], z[i]);
}

// dinv = 1 / diag
__global__ void k_reciprocal(const double* __restrict__ d, double* __restrict__ o, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    o[i] = 1.0 / d[i];
}

// ---- generic vector kernels (GMRES, IR) ------------------------------------

// y = b - y (y holds A x on entry)
template <typename T>
__global__ void k_residual(const T* __restrict__ b, T* __restrict__ y, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] = b[i] - y[i];
}

// v = w * (1 / nrm[0]) with nrm a device scalar holding the squared norm
template <typename T>
__global__ void k_scale_inv_sqrt(T* __restrict__ v, const T* __restrict__ w,
                                 const double* __restrict__ nrm2, int64_t n) {
  const double s = 1.0 / sqrt(*nrm2);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    v[i] = (T)((double)w[i] * s);
}

// w -= sum_j h[j] V_j  (j < m)
template <typename T>
__global__ void k_multi_axpy(T* __restrict__ w, const T* __restrict__ V, int64_t ldv,
                             const double* __restrict__ h, int m, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double acc = (double)w[i];
    for (int j = 0; j < m; ++j) acc = fma(-h[j], (double)V[j * ldv + i], acc);
    w[i] = (T)acc;
  }
}

// x += sum_j y[j] V_j, accumulated in double (x may be T or double)
template <typename TX, typename T>
__global__ void k_update_x(TX* __restrict__ x, const T* __restrict__ V, int64_t ldv,
                           const double* __restrict__ y, int m, double scale, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int j = 0; j < m; ++j) acc = fma(y[j], (double)V[j * ldv + i], acc);
    x[i] = (TX)((double)x[i] + scale * acc);
  }
}

template <typename TO, typename TI>
__global__ void k_convert_scaled(TO* __restrict__ o, const TI* __restrict__ in, double scale,
                                 int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    o[i] = (TO)((double)in[i] * scale);
}

// x += s * c (c in FP32, x in FP64)
__global__ void k_add_scaled(double* __restrict__ x, const float* __restrict__ c, double s,
                             int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    x[i] = fma(s, (double)c[i], x[i]);
}

static inline int vec_grid(int64_t n) {
  int64_t g = (n + 255) / 256;
  return (int)(g < 4864 ? (g < 1 ? 1 : g) : 4864);
}

// ---- workspace ---------------------------------------------------------------

void Workspace::release() {
  for (void* p : bufs) cudaFree(p);
  bufs.clear();
  if (host_state) cudaFreeHost(host_state);
  host_state = nullptr;
  if (cap) cudaStreamDestroy(cap);
  cap = nullptr;
}

cudaError_t Workspace::alloc(void** p, size_t bytes) {
  cudaError_t e = cudaMalloc(p, bytes);
  if (e == cudaSuccess) bufs.push_back(*p);
  return e;
}

// dot products into dev scalars out[0..m-1] = a_j . b
template <typename T>
static cudaError_t multi_dot(const T* a, int64_t lda, const T* b, int64_t n, int m, double* part,
                             double* out, cudaStream_t st) {
  k_multi_dot<T><<<dim3(RED_BLOCKS, m), RED_THREADS, 0, st>>>(a, lda, b, n, part);
  k_finalize<<<m, RED_THREADS, 0, st>>>(part, out);
  return cudaGetLastError();
}

#define CK(x)                                   \
  do {                                          \
    cudaError_t e_ = (x);                       \
    if (e_ != cudaSuccess) return {SBM_ERR_CUDA, e_}; \
  } while (0)

// ---- CG --------------------------------------------------------------------

SolveStatus solve_cg(const ApplyFn<double>& apply, int64_t n, const double* b, double* x,
                     const double* diag, double rtol, int maxit, cudaStream_t st, Workspace& ws,
                     SolveInfo* info) {
  double *r, *z, *p, *q, *dinv = nullptr, *part;
  CgState* dst;
  CK(ws.alloc((void**)&r, n * 8));
  CK(ws.alloc((void**)&z, n * 8));
  CK(ws.alloc((void**)&p, n * 8));
  CK(ws.alloc((void**)&q, n * 8));
  CK(ws.alloc((void**)&part, 3 * RED_BLOCKS * 8));
  CK(ws.alloc((void**)&dst, sizeof(CgState)));
  if (diag) {
    CK(ws.alloc((void**)&dinv, n * 8));
    k_reciprocal<<<vec_grid(n), 256, 0, st>>>(diag, dinv, n);
    CK(cudaGetLastError());
  }
  if (!ws.host_state) CK(cudaMallocHost(&ws.host_state, 4096));
  CgState* hs = (CgState*)ws.host_state;
  if (!ws.cap) CK(cudaStreamCreateWithFlags(&ws.cap, cudaStreamNonBlocking));

  // one chunk of CG iterations, captured once
  cudaGraph_t graph;
  cudaGraphExec_t exec;
  CK(cudaStreamBeginCapture(ws.cap, cudaStreamCaptureModeThreadLocal));
  for (int it = 0; it < CG_CHUNK; ++it) {
    cudaError_t e = apply(p, q, ws.cap);
    if (e != cudaSuccess) {
      cudaStreamEndCapture(ws.cap, &graph);
      return {SBM_ERR_CUDA, e};
    }
    k_multi_dot<double><<<dim3(RED_BLOCKS, 1), RED_THREADS, 0, ws.cap>>>(p, 0, q, n, part);
    k_cg_alpha<<<1, RED_THREADS, 0, ws.cap>>>(part, dst);
    k_cg_update<<<RED_BLOCKS, RED_THREADS, 0, ws.cap>>>(x, r, z, p, q, dinv, n, dst, part);
    k_cg_beta<<<1, RED_THREADS, 0, ws.cap>>>(part, dst);
    k_cg_p<<<vec_grid(n), 256, 0, ws.cap>>>(p, z, n, dst);
  }
  CK(cudaStreamEndCapture(ws.cap, &graph));
  CK(cudaGraphInstantiate(&exec, graph, 0));
  cudaGraphDestroy(graph);

  int total = 0, restarts = 0, status = SBM_NOT_DONE;
  double relres = INFINITY;
  SolveStatus ret{SBM_OK, cudaSuccess};
  while (true) {
    // (re)start from the current x: r = b - A x
    CgState init{};
    init.tol2 = rtol * rtol;
    init.maxit = maxit - total;
    CK(cudaMemcpyAsync(dst, &init, sizeof(CgState), cudaMemcpyHostToDevice, st));
    CK(apply(x, q, st));
    k_cg_init<<<RED_BLOCKS, RED_THREADS, 0, st>>>(b, q, r, z, p, dinv, n, part);
    k_cg_init_fin<<<1, RED_THREADS, 0, st>>>(part, dst);
    CK(cudaGetLastError());
    int done = 0;
    while (true) {
      CK(cudaMemcpyAsync(hs, dst, sizeof(CgState), cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      done = hs->done;
      if (done || hs->maxit <= 0) break;
      CK(cudaGraphLaunch(exec, st));
    }
    total += hs->iters;
    // true residual
    CK(apply(x, q, st));
    k_residual<double><<<vec_grid(n), 256, 0, st>>>(b, q, n);
    CK(multi_dot<double>(q, 0, q, n, 1, part, part + 2 * RED_BLOCKS, st));
    double rr;
    CK(cudaMemcpyAsync(&rr, part + 2 * RED_BLOCKS, 8, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    const double bb = hs->bb;
    relres = (bb > 0) ? std::sqrt(rr / bb) : 0.0;
    if (relres <= rtol) { status = SBM_OK; break; }
    if (done == 2 || done == 3 || total >= maxit || ++restarts > 5 || !std::isfinite(relres)) {
      status = SBM_ERR_NOT_CONVERGED;
      break;
    }
  }
  cudaGraphExecDestroy(exec);
  info->iters = total;
  info->relres = relres;
  info->restarts = restarts;
  ret.status = status;
  return ret;
}

// ---- GMRES(m) --------------------------------------------------------------

// Givens-based least squares of the Arnoldi relation, host side
struct Hess {
  int m;
  std::vector<double> H, cs, sn, g;
  explicit Hess(int m_) : m(m_), H((m_ + 1) * m_, 0.0), cs(m_), sn(m_), g(m_ + 1) {}
  double& h(int i, int j) { return H[j * (m + 1) + i]; }
  // apply the previous rotations to column j, create rotation j; return |g[j+1]|
  double add_column(int j, const double* col) {
    for (int i = 0; i <= j + 1; ++i) h(i, j) = col[i];
    for (int i = 0; i < j; ++i) {
      const double a = cs[i] * h(i, j) + sn[i] * h(i + 1, j);
      const double bb = -sn[i] * h(i, j) + cs[i] * h(i + 1, j);
      h(i, j) = a;
      h(i + 1, j) = bb;
    }
    const double a = h(j, j), bb = h(j + 1, j);
    const double rr = std::hypot(a, bb);
    cs[j] = (rr == 0.0) ? 1.0 : a / rr;
    sn[j] = (rr == 0.0) ? 0.0 : bb / rr;
    h(j, j) = rr;
    h(j + 1, j) = 0.0;
    g[j + 1] = -sn[j] * g[j];
    g[j] = cs[j] * g[j];
    return std::fabs(g[j + 1]);
  }
  void solve(int k, double* y) {   // back substitution on the k x k triangle
    for (int i = k - 1; i >= 0; --i) {
      double s = g[i];
      for (int j = i + 1; j < k; ++j) s -= h(i, j) * y[j];
      y[i] = s / h(i, i);
    }
  }
};

template <typename T, typename TX>
SolveStatus solve_gmres(const ApplyFn<T>& apply, int64_t n, const TX* b, TX* x, double rtol,
                        int maxit, int restart, cudaStream_t st, Workspace& ws, SolveInfo* info,
                        const ApplyFn<TX>* apply_x) {
  // apply_x: operator in the precision of x/b for the outer residual (T == TX: same as apply)
  const int m = restart;
  T* V;
  TX* rx;
  double *part, *dsc;
  CK(ws.alloc((void**)&V, (size_t)(m + 1) * n * sizeof(T)));
  CK(ws.alloc((void**)&rx, (size_t)n * sizeof(TX)));
  CK(ws.alloc((void**)&part, (size_t)(m + 2) * RED_BLOCKS * 8));
  CK(ws.alloc((void**)&dsc, (m + 4) * 8));
  std::vector<double> col(m + 2), y(m + 1);
  int total = 0, cycles = 0;
  double relres = INFINITY, bnorm = 0.0;
  {
    CK(multi_dot<TX>(b, 0, b, n, 1, part, dsc, st));
    CK(cudaMemcpyAsync(&bnorm, dsc, 8, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    bnorm = std::sqrt(bnorm);
  }
  if (bnorm == 0.0) {
    CK(cudaMemsetAsync(x, 0, n * sizeof(TX), st));
    info->iters = 0;
    info->relres = 0.0;
    return {SBM_OK, cudaSuccess};
  }
  const ApplyFn<TX>& ax = *apply_x;
  int status = SBM_ERR_NOT_CONVERGED;
  while (total < maxit) {
    // r = b - A x, v0 = r / |r|
    CK(ax(x, rx, st));
    k_residual<TX><<<vec_grid(n), 256, 0, st>>>(b, rx, n);
    CK(multi_dot<TX>(rx, 0, rx, n, 1, part, dsc, st));
    double rr;
    CK(cudaMemcpyAsync(&rr, dsc, 8, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    relres = std::sqrt(rr) / bnorm;
    if (relres <= rtol) { status = SBM_OK; break; }
    if (!std::isfinite(relres)) break;
    k_convert_scaled<T, TX><<<vec_grid(n), 256, 0, st>>>(V, rx, 1.0 / std::sqrt(rr), n);
    Hess H(m);
    H.g[0] = std::sqrt(rr);
    int k = 0;
    bool conv = false;
    for (int j = 0; j < m && total < maxit; ++j) {
      T* vj = V + (size_t)j * n;
      T* w = V + (size_t)(j + 1) * n;
      CK(apply(vj, w, st));
      // CGS2: h = V^T w; w -= V h; twice
      CK(multi_dot<T>(V, n, w, n, j + 1, part, dsc, st));
      k_multi_axpy<T><<<vec_grid(n), 256, 0, st>>>(w, V, n, dsc, j + 1, n);
      CK(cudaMemcpyAsync(col.data(), dsc, (j + 1) * 8, cudaMemcpyDeviceToHost, st));
      CK(multi_dot<T>(V, n, w, n, j + 1, part, dsc, st));
      k_multi_axpy<T><<<vec_grid(n), 256, 0, st>>>(w, V, n, dsc, j + 1, n);
      std::vector<double> h2(j + 1);
      CK(cudaMemcpyAsync(h2.data(), dsc, (j + 1) * 8, cudaMemcpyDeviceToHost, st));
      CK(multi_dot<T>(w, 0, w, n, 1, part, dsc + m + 2, st));
      double hn2;
      CK(cudaMemcpyAsync(&hn2, dsc + m + 2, 8, cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      for (int i = 0; i <= j; ++i) col[i] += h2[i];
      col[j + 1] = std::sqrt(hn2);
      k_scale_inv_sqrt<T><<<vec_grid(n), 256, 0, st>>>(w, w, dsc + m + 2, n);
      const double res = H.add_column(j, col.data());
      ++total;
      k = j + 1;
      if (res / bnorm <= rtol * 0.5 || hn2 == 0.0 || !std::isfinite(res)) {
        conv = true;
        break;
      }
    }
    H.solve(k, y.data());
    CK(cudaMemcpyAsync(dsc, y.data(), k * 8, cudaMemcpyHostToDevice, st));
    k_update_x<TX, T><<<vec_grid(n), 256, 0, st>>>(x, V, n, dsc, k, 1.0, n);
    CK(cudaGetLastError());
    ++cycles;
    (void)conv;
  }
  if (status != SBM_OK) {
    // final true residual
    CK(ax(x, rx, st));
    k_residual<TX><<<vec_grid(n), 256, 0, st>>>(b, rx, n);
    CK(multi_dot<TX>(rx, 0, rx, n, 1, part, dsc, st));
    double rr;
    CK(cudaMemcpyAsync(&rr, dsc, 8, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    relres = std::sqrt(rr) / bnorm;
    if (relres <= rtol) status = SBM_OK;
  }
  info->iters = total;
  info->relres = relres;
  info->restarts = cycles;
  return {status, cudaSuccess};
}

template SolveStatus solve_gmres<double, double>(const ApplyFn<double>&, int64_t, const double*,
                                                 double*, double, int, int, cudaStream_t,
                                                 Workspace&, SolveInfo*, const ApplyFn<double>*);
template SolveStatus solve_gmres<float, float>(const ApplyFn<float>&, int64_t, const float*,
                                               float*, double, int, int, cudaStream_t, Workspace&,
                                               SolveInfo*, const ApplyFn<float>*);

// ---- FP64 iterative refinement around an FP32 inner GMRES ------------------

SolveStatus solve_ir(const ApplyFn<double>& apply64, const ApplyFn<float>& apply32, int64_t n,
                     const double* b, double* x, double rtol, int maxit, int restart,
                     double inner_rtol, int inner_maxit, cudaStream_t st, Workspace& ws,
                     SolveInfo* info) {
  double *r, *part, *dsc;
  float *r32, *c32;
  CK(ws.alloc((void**)&r, n * 8));
  CK(ws.alloc((void**)&r32, n * 4));
  CK(ws.alloc((void**)&c32, n * 4));
  CK(ws.alloc((void**)&part, RED_BLOCKS * 8));
  CK(ws.alloc((void**)&dsc, 8));
  double bb;
  CK(multi_dot<double>(b, 0, b, n, 1, part, dsc, st));
  CK(cudaMemcpyAsync(&bb, dsc, 8, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  const double bnorm = std::sqrt(bb);
  int outer = 0, inner_total = 0;
  double relres = INFINITY;
  int status = SBM_ERR_NOT_CONVERGED;
  Workspace inner_ws;
  while (outer <= maxit) {
    CK(apply64(x, r, st));
    k_residual<double><<<vec_grid(n), 256, 0, st>>>(b, r, n);
    CK(multi_dot<double>(r, 0, r, n, 1, part, dsc, st));
    double rr;
    CK(cudaMemcpyAsync(&rr, dsc, 8, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    relres = bnorm > 0 ? std::sqrt(rr) / bnorm : 0.0;
    if (relres <= rtol) { status = SBM_OK; break; }
    if (!std::isfinite(relres) || outer == maxit) break;
    // inner: A32 c = r / |r| to inner_rtol, c starts at 0
    const double rn = std::sqrt(rr);
    k_convert_scaled<float, double><<<vec_grid(n), 256, 0, st>>>(r32, r, 1.0 / rn, n);
    CK(cudaMemsetAsync(c32, 0, n * 4, st));
    SolveInfo ii{};
    SolveStatus s = solve_gmres<float, float>(apply32, n, r32, c32, inner_rtol, inner_maxit,
                                              restart, st, inner_ws, &ii, &apply32);
    inner_ws.release();
    if (s.status == SBM_ERR_CUDA) {
      info->iters = inner_total;
      return s;
    }
    inner_total += ii.iters;
    // x += |r| c
    k_add_scaled<<<vec_grid(n), 256, 0, st>>>(x, c32, rn, n);
    CK(cudaGetLastError());
    ++outer;
  }
  info->iters = inner_total;
  info->relres = relres;
  info->restarts = outer;
  return {status, cudaSuccess};
}

}  // namespace sbm
