// Krylov drivers on the matrix-free operator: conjugate gradients, restarted
// GMRES, BiCGStab, and FP64 iterative refinement around an FP32 inner solve.
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

// The BiCGStab chunk's vector and scalar kernels are launched as
// programmatic dependents of the kernel before them (their launch overlaps
// its end); each waits for it before touching memory, so the order is that
// of the stream.  A no-op when a kernel is launched without the attribute.
__device__ __forceinline__ void pdl_wait_all() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

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
  pdl_wait_all();
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

// x += s * c (FP64)
__global__ void k_axpy_d(double* __restrict__ x, const double* __restrict__ c, double s,
                         int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    x[i] = fma(s, c[i], x[i]);
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

// ---- BiCGStab ----------------------------------------------------------------
//
// van der Vorst's stabilised bi-conjugate gradients, two operator
// applications and three reductions per iteration.  Vectors are in T
// (FP64 or FP32); every scalar is FP64 and stays on the device, so a chunk of
// BI_CHUNK iterations is one CUDA-graph launch with no host round trip.  A
// breakdown (rho or (r^, v) vanishing, omega = 0) or a recursive residual that
// disagrees with the true one restarts from the current iterate with a fresh
// shadow residual r^ = r.

constexpr int BI_CHUNK = 8;
constexpr int kIrFinishMaxit = 20000;   // FP64 BiCGStab finish of the refinement, at most

struct BiState {
  double rho, alpha, omega, beta, rr, bb, tol2;
  int done;     // 0 running, 1 converged (recursive residual), 2 breakdown/divergence, 3 maxit
  int iters;
  int maxit;
};

// r = b - q (q = A x; q == nullptr for x = 0); r^ = r; p = r; partials r.r, b.b
template <typename T>
__global__ void k_bi_init(const T* __restrict__ b, const T* __restrict__ q, T* __restrict__ r,
                          T* __restrict__ rh, T* __restrict__ p, int64_t n,
                          double* __restrict__ part) {
  __shared__ double sh[RED_THREADS];
  double srr = 0.0, sbb = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const T ri = q ? (T)(b[i] - q[i]) : b[i];
    r[i] = ri;
    rh[i] = ri;
    p[i] = ri;
    srr = fma((double)ri, (double)ri, srr);
    sbb = fma((double)b[i], (double)b[i], sbb);
  }
  srr = block_sum(srr, sh);
  sbb = block_sum(sbb, sh);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = srr;
    part[RED_BLOCKS + blockIdx.x] = sbb;
  }
}

__global__ void k_bi_init_fin(const double* __restrict__ part, BiState* st) {
  __shared__ double sh[RED_THREADS];
  double v[2];
  for (int j = 0; j < 2; ++j) {
    double s = 0.0;
    for (int i = threadIdx.x; i < RED_BLOCKS; i += blockDim.x) s += part[j * RED_BLOCKS + i];
    v[j] = block_sum(s, sh);
  }
  if (threadIdx.x == 0) {
    st->rr = v[0];
    st->bb = v[1];
    st->rho = v[0];              // (r^, r) with r^ = r
    st->alpha = st->omega = 1.0;
    st->beta = 0.0;
    st->done = (v[0] <= st->tol2 * v[1]) ? 1 : 0;
    if (!isfinite(v[0])) st->done = 2;
    if (st->maxit <= 0 && !st->done) st->done = 3;
  }
}

// alpha = rho / (r^, v)
__global__ void k_bi_alpha(const double* __restrict__ part, BiState* st) {
  pdl_wait_all();
  __shared__ double sh[RED_THREADS];
  if (st->done) return;
  double s = 0.0;
  for (int i = threadIdx.x; i < RED_BLOCKS; i += blockDim.x) s += part[i];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) {
    if (!(s != 0.0) || !isfinite(s)) st->done = 2;
    else st->alpha = st->rho / s;
  }
}

// s = r - alpha v
template <typename T>
__global__ void k_bi_s(const T* __restrict__ r, const T* __restrict__ v, T* __restrict__ s,
                       int64_t n, const BiState* st) {
  pdl_wait_all();
  if (st->done) return;
  const double al = st->alpha;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    s[i] = (T)fma(-al, (double)v[i], (double)r[i]);
}

// partials of (t, s) and (t, t)
template <typename T>
__global__ void k_bi_dot2(const T* __restrict__ t, const T* __restrict__ s, int64_t n,
                          const BiState* st, double* __restrict__ part) {
  pdl_wait_all();
  __shared__ double sh[RED_THREADS];
  if (st->done) return;
  double sts = 0.0, stt = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double ti = (double)t[i];
    sts = fma(ti, (double)s[i], sts);
    stt = fma(ti, ti, stt);
  }
  sts = block_sum(sts, sh);
  stt = block_sum(stt, sh);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = sts;
    part[RED_BLOCKS + blockIdx.x] = stt;
  }
}

// omega = (t, s) / (t, t)  (0 when t = 0: the update then keeps r = s)
__global__ void k_bi_omega(const double* __restrict__ part, BiState* st) {
  pdl_wait_all();
  __shared__ double sh[RED_THREADS];
  if (st->done) return;
  double v[2];
  for (int j = 0; j < 2; ++j) {
    double s = 0.0;
    for (int i = threadIdx.x; i < RED_BLOCKS; i += blockDim.x) s += part[j * RED_BLOCKS + i];
    v[j] = block_sum(s, sh);
  }
  if (threadIdx.x == 0) {
    st->omega = (v[1] > 0.0) ? v[0] / v[1] : 0.0;
    if (!isfinite(st->omega)) st->done = 2;
  }
}

// x += alpha p + omega s; r = s - omega t; partials of (r^, r), (r, r)
template <typename T>
__global__ void k_bi_update(T* __restrict__ x, T* __restrict__ r, const T* __restrict__ p,
                            const T* __restrict__ s, const T* __restrict__ t,
                            const T* __restrict__ rh, int64_t n, const BiState* st,
                            double* __restrict__ part) {
  pdl_wait_all();
  __shared__ double sh[RED_THREADS];
  if (st->done) return;
  const double al = st->alpha, om = st->omega;
  double srh = 0.0, srr = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double si = (double)s[i];
    x[i] = (T)fma(om, si, fma(al, (double)p[i], (double)x[i]));
    const T ri = (T)fma(-om, (double)t[i], si);
    r[i] = ri;
    srh = fma((double)rh[i], (double)ri, srh);
    srr = fma((double)ri, (double)ri, srr);
  }
  srh = block_sum(srh, sh);
  srr = block_sum(srr, sh);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = srh;
    part[RED_BLOCKS + blockIdx.x] = srr;
  }
}

// rho' = (r^, r); convergence / breakdown tests; beta = (rho'/rho)(alpha/omega)
__global__ void k_bi_beta(const double* __restrict__ part, BiState* st) {
  pdl_wait_all();
  __shared__ double sh[RED_THREADS];
  if (st->done) return;
  double v[2];
  for (int j = 0; j < 2; ++j) {
    double s = 0.0;
    for (int i = threadIdx.x; i < RED_BLOCKS; i += blockDim.x) s += part[j * RED_BLOCKS + i];
    v[j] = block_sum(s, sh);
  }
  if (threadIdx.x == 0) {
    st->iters += 1;
    st->rr = v[1];
    if (v[1] <= st->tol2 * st->bb) st->done = 1;
    else if (!isfinite(v[1]) || v[1] > 1e24 * st->bb) st->done = 2;
    else if (!(v[0] != 0.0) || !(st->omega != 0.0)) st->done = 2;
    else if (st->iters >= st->maxit) st->done = 3;
    if (!st->done) {
      st->beta = (v[0] / st->rho) * (st->alpha / st->omega);
      st->rho = v[0];
    }
  }
}

// reliable update: r = b - q (q = A x with the accurate operator); partials
// of (r^, r), (r, r)
template <typename T>
__global__ void k_bi_replace(const T* __restrict__ b, const T* __restrict__ q,
                             T* __restrict__ r, const T* __restrict__ rh, int64_t n,
                             double* __restrict__ part) {
  __shared__ double sh[RED_THREADS];
  double srh = 0.0, srr = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const T ri = (T)((double)b[i] - (double)q[i]);
    r[i] = ri;
    srh = fma((double)rh[i], (double)ri, srh);
    srr = fma((double)ri, (double)ri, srr);
  }
  srh = block_sum(srh, sh);
  srr = block_sum(srr, sh);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = srh;
    part[RED_BLOCKS + blockIdx.x] = srr;
  }
}

// rho = (r^, r) and rr = (r, r) of the replaced residual; convergence test
__global__ void k_bi_replace_fin(const double* __restrict__ part, BiState* st) {
  __shared__ double sh[RED_THREADS];
  if (st->done) return;
  double v[2];
  for (int j = 0; j < 2; ++j) {
    double s = 0.0;
    for (int i = threadIdx.x; i < RED_BLOCKS; i += blockDim.x) s += part[j * RED_BLOCKS + i];
    v[j] = block_sum(s, sh);
  }
  if (threadIdx.x == 0) {
    st->rr = v[1];
    st->rho = v[0];
    if (v[1] <= st->tol2 * st->bb) st->done = 1;
    else if (!isfinite(v[1]) || !(v[0] != 0.0)) st->done = 2;
  }
}

// p = r + beta (p - omega v)
template <typename T>
__global__ void k_bi_p(T* __restrict__ p, const T* __restrict__ r, const T* __restrict__ v,
                       int64_t n, const BiState* st) {
  pdl_wait_all();
  if (st->done) return;
  const double be = st->beta, om = st->omega;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    p[i] = (T)fma(be, fma(-om, (double)v[i], (double)p[i]), (double)r[i]);
}

template <typename T>
cudaError_t Bicgstab<T>::setup(const ApplyFn<T>& apply_, int64_t n_, const T* b_, T* x_,
                               Workspace& ws) {
  apply = apply_;
  n = n_;
  b = b_;
  x = x_;
  cudaError_t e;
  T** vecs[7] = {&r, &rh, &p, &v, &s, &t, &xb};
  for (T** pv : vecs)
    if ((e = ws.alloc((void**)pv, (size_t)n * sizeof(T))) != cudaSuccess) return e;
  if ((e = ws.alloc((void**)&part, 2 * RED_BLOCKS * 8)) != cudaSuccess) return e;
  if ((e = ws.alloc(&dstate, sizeof(BiState))) != cudaSuccess) return e;
  if ((e = cudaMallocHost(&hstate, sizeof(BiState))) != cudaSuccess) return e;
  if ((e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking)) != cudaSuccess) return e;
  BiState* dst = (BiState*)dstate;
  cudaGraph_t graph;
  if ((e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
    return e;
  cudaError_t ae = cudaSuccess;
  for (int it = 0; it < BI_CHUNK && ae == cudaSuccess; ++it) {
    ae = apply(p, v, cap);
    if (ae != cudaSuccess) break;
    const T* crh = rh;
    const T* cv = v;
    const T* cr = r;
    const T* cs = s;
    const T* ct = t;
    const T* cp = p;
    if ((ae = launch_maybe_pdl(k_multi_dot<T>, dim3(RED_BLOCKS, 1), dim3(RED_THREADS), 0, cap,
                               true, crh, (int64_t)0, cv, n, part)) != cudaSuccess ||
        (ae = launch_maybe_pdl(k_bi_alpha, dim3(1), dim3(RED_THREADS), 0, cap, true,
                               (const double*)part, dst)) != cudaSuccess ||
        (ae = launch_maybe_pdl(k_bi_s<T>, dim3(vec_grid(n)), dim3(256), 0, cap, true, cr, cv, s,
                               n, (const BiState*)dst)) != cudaSuccess)
      break;
    ae = apply(s, t, cap);
    if (ae != cudaSuccess) break;
    if ((ae = launch_maybe_pdl(k_bi_dot2<T>, dim3(RED_BLOCKS), dim3(RED_THREADS), 0, cap, true,
                               ct, cs, n, (const BiState*)dst, part)) != cudaSuccess ||
        (ae = launch_maybe_pdl(k_bi_omega, dim3(1), dim3(RED_THREADS), 0, cap, true,
                               (const double*)part, dst)) != cudaSuccess ||
        (ae = launch_maybe_pdl(k_bi_update<T>, dim3(RED_BLOCKS), dim3(RED_THREADS), 0, cap,
                               true, x, r, cp, cs, ct, crh, n, (const BiState*)dst, part)) !=
            cudaSuccess ||
        (ae = launch_maybe_pdl(k_bi_beta, dim3(1), dim3(RED_THREADS), 0, cap, true,
                               (const double*)part, dst)) != cudaSuccess ||
        (ae = launch_maybe_pdl(k_bi_p<T>, dim3(vec_grid(n)), dim3(256), 0, cap, true, p, cr, cv,
                               n, (const BiState*)dst)) != cudaSuccess)
      break;
  }
  e = cudaStreamEndCapture(cap, &graph);
  if (ae != cudaSuccess) {
    if (e == cudaSuccess) cudaGraphDestroy(graph);
    return ae;
  }
  if (e != cudaSuccess) return e;
  e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  return e;
}

template <typename T>
void Bicgstab<T>::destroy() {
  if (exec) cudaGraphExecDestroy(exec);
  exec = nullptr;
  if (hstate) cudaFreeHost(hstate);
  hstate = nullptr;
  if (cap) cudaStreamDestroy(cap);
  cap = nullptr;
}

template <typename T>
SolveStatus Bicgstab<T>::solve(bool x_zero, double rtol, int maxit, cudaStream_t st,
                               SolveInfo* info) {
  BiState* dst = (BiState*)dstate;
  BiState* hs = (BiState*)hstate;
  int total = 0, restarts = 0, status = SBM_NOT_DONE;
  double relres = INFINITY, best = INFINITY;
  bool zero = x_zero;
  const bool reliable = (bool)apply_hi;
  const ApplyFn<T>& ap_true = reliable ? apply_hi : apply;   // first and final residuals
  while (true) {
    BiState init{};
    init.tol2 = rtol * rtol;
    init.maxit = maxit - total;
    CK(cudaMemcpyAsync(dst, &init, sizeof(BiState), cudaMemcpyHostToDevice, st));
    if (!zero) CK(ap_true(x, v, st));
    k_bi_init<T><<<RED_BLOCKS, RED_THREADS, 0, st>>>(b, zero ? nullptr : v, r, rh, p, n, part);
    k_bi_init_fin<<<1, RED_THREADS, 0, st>>>(part, dst);
    CK(cudaGetLastError());
    zero = false;
    int done = 0;
    double rr_ref = -1.0;        // recursive residual at the last reliable update
    double rr_true = INFINITY;   // true residual at the last reliable update
    bool replaced = false, stalled = false;
    while (true) {
      CK(cudaMemcpyAsync(hs, dst, sizeof(BiState), cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      done = hs->done;
      if (rr_ref < 0.0) {
        // a true residual (the first one, or just replaced)
        rr_ref = hs->rr;
        // one that no longer halves between updates: the reduced-precision
        // iteration has stalled (the caller finishes)
        if (replaced) stalled = !done && hs->rr > 0.25 * rr_true;
        rr_true = hs->rr;
        replaced = false;
        // with reliable updates: keep the iterate of least true residual
        if (reliable && std::isfinite(hs->rr) && hs->rr < best) {
          best = hs->rr;
          CK(cudaMemcpyAsync(xb, x, (size_t)n * sizeof(T), cudaMemcpyDeviceToDevice, st));
        }
      }
      if (stalled) {
        done = 3;
        break;
      }
      // reliable update: the true residual replaces the recursive one
      if (reliable && !done && std::isfinite(hs->rr) &&
          hs->rr < reliable_factor * reliable_factor * rr_ref) {
        CK(apply_hi(x, t, st));
        k_bi_replace<T><<<RED_BLOCKS, RED_THREADS, 0, st>>>(b, t, r, rh, n, part);
        k_bi_replace_fin<<<1, RED_THREADS, 0, st>>>(part, dst);
        CK(cudaGetLastError());
        ++replacements;
        rr_ref = -1.0;           // re-read: the reference is the replaced residual
        replaced = true;
        continue;
      }
      // keep the iterate of least (recursive) residual seen at a chunk end
      if (!reliable && std::isfinite(hs->rr) && hs->rr < best) {
        best = hs->rr;
        CK(cudaMemcpyAsync(xb, x, (size_t)n * sizeof(T), cudaMemcpyDeviceToDevice, st));
      }
      if (done) break;
      CK(cudaGraphLaunch(exec, st));
    }
    total += hs->iters;
    // after a breakdown, divergence, a stall or the iteration cap, continue
    // from the best iterate rather than the last one (reliable updates: the
    // best true residual; otherwise the best recursive one)
    if (done != 1 && (reliable || !(hs->rr <= best)))
      CK(cudaMemcpyAsync(x, xb, (size_t)n * sizeof(T), cudaMemcpyDeviceToDevice, st));
    if (hs->bb == 0.0) {
      relres = 0.0;
      status = SBM_OK;
      break;
    }
    // true residual of the current iterate
    CK(ap_true(x, v, st));
    k_residual<T><<<vec_grid(n), 256, 0, st>>>(b, v, n);
    CK(multi_dot<T>(v, 0, v, n, 1, part, part + RED_BLOCKS, st));
    double rr;
    CK(cudaMemcpyAsync(&rr, part + RED_BLOCKS, 8, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    relres = std::sqrt(rr / hs->bb);
    if (relres <= rtol) { status = SBM_OK; break; }
    if (done == 3 || total >= maxit || ++restarts > 50 || !std::isfinite(relres)) {
      status = SBM_ERR_NOT_CONVERGED;
      break;
    }
  }
  info->iters = total;
  info->relres = relres;
  info->restarts = restarts;
  return {status, cudaSuccess};
}

template struct Bicgstab<double>;
template struct Bicgstab<float>;

// ---- BiCGStab on the FP32 apply with FP64 reliable updates -------------------

SolveStatus solve_bicgstab_reliable(const ApplyFn<double>& apply64,
                                    const ApplyFn<float>& apply32, int64_t n, const double* b,
                                    double* x, double rtol, int maxit, cudaStream_t st,
                                    Workspace& ws, SolveInfo* info, int* replacements) {
  float *xa = nullptr, *ya = nullptr;
  CK(ws.alloc((void**)&xa, n * 4));
  CK(ws.alloc((void**)&ya, n * 4));
  ApplyFn<double> apply_mixed = [&](const double* xin, double* yout, cudaStream_t s) {
    k_convert_scaled<float, double><<<vec_grid(n), 256, 0, s>>>(xa, xin, 1.0, n);
    cudaError_t e = apply32(xa, ya, s);
    if (e != cudaSuccess) return e;
    k_convert_scaled<double, float><<<vec_grid(n), 256, 0, s>>>(yout, ya, 1.0, n);
    return cudaGetLastError();
  };
  Bicgstab<double> bi;
  bi.apply_hi = apply64;
  cudaError_t e = bi.setup(apply_mixed, n, b, x, ws);
  SolveStatus s{SBM_ERR_CUDA, e};
  if (e == cudaSuccess) s = bi.solve(false, rtol, maxit, st, info);
  if (replacements) *replacements = bi.replacements;
  bi.destroy();
  // FP64 finish when the reduced-precision iteration stalled (the FP32
  // operator's rounding, about kappa * 6e-8 of |b|, limits its corrections)
  if (s.status == SBM_ERR_NOT_CONVERGED && std::isfinite(info->relres) &&
      info->iters < maxit) {
    Bicgstab<double> bf;
    SolveInfo fi{};
    e = bf.setup(apply64, n, b, x, ws);
    SolveStatus f{SBM_ERR_CUDA, e};
    if (e == cudaSuccess) f = bf.solve(false, rtol, maxit - info->iters, st, &fi);
    bf.destroy();
    if (f.status == SBM_ERR_CUDA) return f;
    info->iters += fi.iters;
    info->relres = fi.relres;
    info->restarts += 1;
    s = f;
  }
  return s;
}

// ---- FP64 iterative refinement around an FP32 inner solve --------------------

SolveStatus solve_ir(const ApplyFn<double>& apply64, const ApplyFn<float>& apply32, int64_t n,
                     const double* b, double* x, double rtol, int maxit, int restart,
                     double inner_rtol, int inner_maxit, int inner, cudaStream_t st,
                     Workspace& ws, SolveInfo* info) {
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
  Bicgstab<float> bi;
  if (inner == SBM_INNER_BICGSTAB) {
    cudaError_t e = bi.setup(apply32, n, r32, c32, ws);
    if (e != cudaSuccess) {
      bi.destroy();
      return {SBM_ERR_CUDA, e};
    }
  }
  // mixed inner solver: FP64 vectors and scalars, the FP32 apply (converted
  // in and out around every application)
  Bicgstab<double> bm;
  double *r64 = nullptr, *c64 = nullptr;
  float *xa = nullptr, *ya = nullptr;
  ApplyFn<double> apply_mixed = [&](const double* xin, double* yout, cudaStream_t s) {
    k_convert_scaled<float, double><<<vec_grid(n), 256, 0, s>>>(xa, xin, 1.0, n);
    cudaError_t e = apply32(xa, ya, s);
    if (e != cudaSuccess) return e;
    k_convert_scaled<double, float><<<vec_grid(n), 256, 0, s>>>(yout, ya, 1.0, n);
    return cudaGetLastError();
  };
  if (inner == SBM_INNER_BICGSTAB_MIXED) {
    cudaError_t e;
    if ((e = ws.alloc((void**)&r64, n * 8)) != cudaSuccess ||
        (e = ws.alloc((void**)&c64, n * 8)) != cudaSuccess ||
        (e = ws.alloc((void**)&xa, n * 4)) != cudaSuccess ||
        (e = ws.alloc((void**)&ya, n * 4)) != cudaSuccess ||
        (e = bm.setup(apply_mixed, n, r64, c64, ws)) != cudaSuccess) {
      bm.destroy();
      return {SBM_ERR_CUDA, e};
    }
  }
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
    SolveInfo ii{};
    SolveStatus s;
    if (inner == SBM_INNER_BICGSTAB_MIXED) {
      k_convert_scaled<double, double><<<vec_grid(n), 256, 0, st>>>(r64, r, 1.0 / rn, n);
      CK(cudaMemsetAsync(c64, 0, n * 8, st));
      s = bm.solve(true, inner_rtol, inner_maxit, st, &ii);
      if (s.status == SBM_ERR_CUDA) {
        bm.destroy();
        bi.destroy();
        info->iters = inner_total;
        return s;
      }
      inner_total += ii.iters;
      if (s.status != SBM_OK && !(ii.relres < 1.0)) break;
      k_axpy_d<<<vec_grid(n), 256, 0, st>>>(x, c64, rn, n);       // x += |r| c
      CK(cudaGetLastError());
      ++outer;
      continue;
    }
    k_convert_scaled<float, double><<<vec_grid(n), 256, 0, st>>>(r32, r, 1.0 / rn, n);
    CK(cudaMemsetAsync(c32, 0, n * 4, st));
    if (inner == SBM_INNER_BICGSTAB) {
      s = bi.solve(true, inner_rtol, inner_maxit, st, &ii);
    } else {
      s = solve_gmres<float, float>(apply32, n, r32, c32, inner_rtol, inner_maxit, restart, st,
                                    inner_ws, &ii, &apply32);
      inner_ws.release();
    }
    if (s.status == SBM_ERR_CUDA) {
      bi.destroy();
      info->iters = inner_total;
      return s;
    }
    inner_total += ii.iters;
    // an inner solve that made no progress would only spoil x
    if (s.status != SBM_OK && !(ii.relres < 1.0)) break;
    // x += |r| c
    k_add_scaled<<<vec_grid(n), 256, 0, st>>>(x, c32, rn, n);
    CK(cudaGetLastError());
    ++outer;
  }
  bi.destroy();
  bm.destroy();
  // FP64 finish: when the reduced-precision corrections stall (an ill-conditioned
  // operator whose FP32 rounding, about kappa * 6e-8 of |b|, floors what an
  // inner solve can reach), BiCGStab on the FP64 operator continues from x
  if (status != SBM_OK && std::isfinite(relres) && bnorm > 0) {
    Bicgstab<double> bf;
    cudaError_t e = bf.setup(apply64, n, b, x, ws);
    SolveInfo fi{};
    SolveStatus s{SBM_ERR_CUDA, e};
    const int cap = (int)std::min<int64_t>(kIrFinishMaxit, (int64_t)maxit * inner_maxit);
    if (e == cudaSuccess) s = bf.solve(false, rtol, cap, st, &fi);
    bf.destroy();
    if (s.status == SBM_ERR_CUDA) {
      info->iters = inner_total;
      return s;
    }
    inner_total += fi.iters;
    relres = fi.relres;
    status = s.status;
    ++outer;
  }
  info->iters = inner_total;
  info->relres = relres;
  info->restarts = outer;
  return {status, cudaSuccess};
}

}  // namespace sbm
