// Geometry stage of the set-up on the GPU (the paper's operator
// initialisation, Section 4.4: active cells, surrogate faces, closest-point
// projections of the surrogate quadrature points).
//
// Same results as setup_geometry_host, bit for bit: the level set and the
// closest points come from the shared geom.hpp, this file is compiled without
// fused multiply-adds, and every index is produced in the host's order:
//  1. one thread per background cell: active or not (centre, or volume
//     fraction over 8^d sub-cell midpoints);
//  2. exclusive scan of the flags -> active-cell ranks in lexicographic order;
//  3. one thread per active cell: its multi-index, its surrogate faces and
//     (s = 1) interior faces counted, then (after a scan) written in the order
//     (axis k, side s);
//  4. one thread per surrogate quadrature point: x~, its closest point x_q,
//     the reference coordinates and the shift.
// The scans are deterministic two-level block scans.  The CG DoF numbering
// follows on the device too (setup_numbering_device: lattice marks, scan,
// line starts); its input cells and output line table go through the host,
// where the rest of the set-up continues.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>
#include <vector>

#include "internal.hpp"
#include "setup.hpp"

namespace sbm {

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;                        // per thread
constexpr int kScanTile = kScanThreads * kScanItems; // elements per block

struct GeoArgs {
  GeomView g;
  int d, N, activity;
  double h, vf_threshold;
};

__device__ __forceinline__ void cell_index(int64_t b, int d, int N, int* idx) {
  int64_t r = b;
  for (int i = 0; i < d; ++i) {
    idx[i] = (int)(r % N);
    r /= N;
  }
}

__global__ void k_active(const GeoArgs a, int64_t nbg, int32_t* __restrict__ flag) {
  for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < nbg;
       b += (int64_t)gridDim.x * blockDim.x) {
    int idx[3] = {0, 0, 0};
    cell_index(b, a.d, a.N, idx);
    bool active;
    if (a.activity == SBM_ACTIVE_VOLUME) {
      constexpr int m = kVfSamples;
      int count = 0, tot = 1;
      for (int i = 0; i < a.d; ++i) tot *= m;
      for (int s = 0; s < tot; ++s) {
        double xs[3];
        int rs = s;
        for (int i = 0; i < a.d; ++i) {
          xs[i] = -1.0 + a.h * ((double)idx[i] + ((rs % m) + 0.5) / m);
          rs /= m;
        }
        if (geom_phi(a.g, xs) < 0.0) ++count;
      }
      active = (double)count >= a.vf_threshold * (double)tot;
    } else {
      double xc[3];
      for (int i = 0; i < a.d; ++i) xc[i] = -1.0 + a.h * (idx[i] + 0.5);
      active = geom_phi(a.g, xc) < 0.0;
    }
    flag[b] = active ? 1 : 0;
  }
}

// ---- deterministic exclusive scan (int32 values, int64 offsets) ------------------

__device__ __forceinline__ int64_t block_exclusive(int64_t v, int64_t* sh, int64_t* total) {
  const int t = threadIdx.x;
  sh[t] = v;
  __syncthreads();
  for (int off = 1; off < blockDim.x; off <<= 1) {
    const int64_t add = (t >= off) ? sh[t - off] : 0;
    __syncthreads();
    sh[t] += add;
    __syncthreads();
  }
  const int64_t incl = sh[t];
  *total = sh[blockDim.x - 1];
  __syncthreads();
  return incl - v;
}

__global__ void k_tile_sums(const int32_t* __restrict__ in, int64_t n, int64_t* __restrict__ sums) {
  __shared__ int64_t sh[kScanThreads];
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  int64_t s = 0;
  for (int i = 0; i < kScanItems; ++i)
    if (base + i < n) s += in[base + i];
  int64_t tot;
  block_exclusive(s, sh, &tot);
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// one block: exclusive scan of the tile sums, in passes of blockDim values
__global__ void k_scan_sums(int64_t* __restrict__ sums, int64_t ntiles, int64_t* __restrict__ total) {
  __shared__ int64_t sh[kScanThreads];
  int64_t carry = 0;
  for (int64_t p = 0; p < ntiles; p += blockDim.x) {
    const int64_t i = p + threadIdx.x;
    const int64_t v = (i < ntiles) ? sums[i] : 0;
    int64_t tot;
    const int64_t ex = block_exclusive(v, sh, &tot);
    if (i < ntiles) sums[i] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0) *total = carry;
}

__global__ void k_scan_apply(const int32_t* __restrict__ in, int64_t n,
                             const int64_t* __restrict__ offs, int64_t* __restrict__ out) {
  __shared__ int64_t sh[kScanThreads];
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  int64_t s = 0;
  for (int i = 0; i < kScanItems; ++i)
    if (base + i < n) s += in[base + i];
  int64_t tot;
  int64_t run = offs[blockIdx.x] + block_exclusive(s, sh, &tot);
  for (int i = 0; i < kScanItems; ++i)
    if (base + i < n) {
      out[base + i] = run;
      run += in[base + i];
    }
}

// ---- cells and faces ----------------------------------------------------------------

__global__ void k_cells(const int32_t* __restrict__ flag, const int64_t* __restrict__ rank,
                        int64_t nbg, int d, int N, int32_t* __restrict__ cells,
                        int64_t* __restrict__ cell_bg, int32_t* __restrict__ bg_to_cell) {
  for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < nbg;
       b += (int64_t)gridDim.x * blockDim.x) {
    if (!flag[b]) {
      bg_to_cell[b] = -1;
      continue;
    }
    const int64_t r = rank[b];
    int idx[3] = {0, 0, 0};
    cell_index(b, d, N, idx);
    for (int i = 0; i < d; ++i) cells[r * d + i] = idx[i];
    cell_bg[r] = b;
    bg_to_cell[b] = (int32_t)r;
  }
}

// mode 0: counts per cell (surrogate, interior); mode 1: write at the offsets
__global__ void k_faces(int mode, int64_t nc, int d, int N, const int32_t* __restrict__ cells,
                        const int64_t* __restrict__ cell_bg, const int32_t* __restrict__ bg_to_cell,
                        int32_t* __restrict__ nsf, int32_t* __restrict__ nif,
                        const int64_t* __restrict__ osf, const int64_t* __restrict__ oif,
                        int32_t* __restrict__ sfaces, int32_t* __restrict__ ifaces) {
  const int64_t stride[3] = {1, N, (int64_t)N * N};
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nc;
       c += (int64_t)gridDim.x * blockDim.x) {
    int cs = 0, ci = 0;
    for (int k = 0; k < d; ++k)
      for (int s = 0; s < 2; ++s) {
        const int j = cells[c * d + k] + (s ? 1 : -1);
        int32_t nb = -1;
        if (j >= 0 && j < N) nb = bg_to_cell[cell_bg[c] + (s ? 1 : -1) * stride[k]];
        if (nb < 0) {
          if (mode == 1) {
            int32_t* o = sfaces + 3 * (osf[c] + cs);
            o[0] = (int32_t)c;
            o[1] = k;
            o[2] = s;
          }
          ++cs;
        } else if (s == 1) {
          if (mode == 1) {
            int32_t* o = ifaces + 3 * (oif[c] + ci);
            o[0] = (int32_t)c;
            o[1] = k;
            o[2] = nb;
          }
          ++ci;
        }
      }
    if (mode == 0) {
      nsf[c] = cs;
      nif[c] = ci;
    }
  }
}

struct PointArgs {
  GeomView g;
  int d, n, L;
  double h;
  double gpts[kMaxN];
};

__global__ void k_face_points(const PointArgs a, int64_t F, const int32_t* __restrict__ sfaces,
                              const int32_t* __restrict__ cells, double* __restrict__ face_x,
                              double* __restrict__ face_xi, double* __restrict__ face_d,
                              int* __restrict__ failed) {
  const int d = a.d, Q = a.L;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < F * Q;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t f = t / Q;
    const int q = (int)(t - f * Q);
    const int c = sfaces[3 * f], k = sfaces[3 * f + 1], s = sfaces[3 * f + 2];
    int tang[2] = {0, 0}, nt = 0;
    for (int l = 0; l < d; ++l)
      if (l != k) tang[nt++] = l;
    double lo[3];
    for (int l = 0; l < d; ++l) lo[l] = -1.0 + a.h * (double)cells[(int64_t)c * d + l];
    const int qa = q % a.n, qb = q / a.n;
    double xi[3], xt[3], xq[3];
    xi[k] = (double)s;
    xi[tang[0]] = a.gpts[qa];
    if (d == 3) xi[tang[1]] = a.gpts[qb];
    for (int l = 0; l < d; ++l) xt[l] = lo[l] + a.h * xi[l];
    if (!geom_closest(a.g, xt, xq)) {
      atomicOr(failed, 1);
      continue;
    }
    for (int l = 0; l < d; ++l) {
      face_x[t * d + l] = xq[l];
      face_xi[t * d + l] = (xq[l] - lo[l]) / a.h;
      face_d[t * d + l] = xq[l] - xt[l];
    }
  }
}

// RAII list of device buffers
struct DevBufs {
  std::vector<void*> p;
  ~DevBufs() {
    for (void* q : p) cudaFree(q);
  }
  template <typename T>
  cudaError_t alloc(T** out, size_t n) {
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, (n > 0 ? n : 1) * sizeof(T));
    if (e == cudaSuccess) {
      p.push_back(q);
      *out = static_cast<T*>(q);
    }
    return e;
  }
};

cudaError_t exclusive_scan(const int32_t* in, int64_t n, int64_t* out, int64_t* total_dev,
                           DevBufs& bufs) {
  const int64_t tiles = (n + kScanTile - 1) / kScanTile;
  int64_t* sums;
  cudaError_t e = bufs.alloc(&sums, (size_t)tiles);
  if (e != cudaSuccess) return e;
  if (tiles > 0) {
    k_tile_sums<<<(unsigned)tiles, kScanThreads>>>(in, n, sums);
    k_scan_sums<<<1, kScanThreads>>>(sums, tiles, total_dev);
    k_scan_apply<<<(unsigned)tiles, kScanThreads>>>(in, n, sums, out);
  } else {
    e = cudaMemset(total_dev, 0, sizeof(int64_t));
  }
  return e != cudaSuccess ? e : cudaGetLastError();
}

int grid_for(int64_t n) {
  const int64_t g = (n + 255) / 256;
  return (int)(g < 1 ? 1 : (g > 65535 * 8 ? 65535 * 8 : g));
}

// CG numbering: mark every lattice node an active cell touches (the same
// value from every writer), scan, then the global index of each cell's line
// starts (node (0, j1, j2)).
__global__ void k_mark(int64_t nc, int d, int p, int n, int nd, int64_t M,
                       const int32_t* __restrict__ cells, int32_t* __restrict__ mark) {
  const int64_t ms[3] = {1, M, M * M};
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nc * nd;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = t / nd;
    int r = (int)(t - c * nd);
    int64_t g = 0;
    for (int l = 0; l < d; ++l) {
      g += ((int64_t)p * cells[c * d + l] + (r % n)) * ms[l];
      r /= n;
    }
    mark[g] = 1;
  }
}

__global__ void k_lines(int64_t nc, int d, int p, int n, int L, int64_t M,
                        const int32_t* __restrict__ cells, const int64_t* __restrict__ num,
                        int32_t* __restrict__ lines) {
  const int64_t ms[3] = {1, M, M * M};
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nc * L;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = t / L;
    const int line = (int)(t - c * L);
    int64_t g = 0;
    for (int l = 0; l < d; ++l) g += (int64_t)p * cells[c * d + l] * ms[l];
    g += (d == 2) ? line * ms[1] : (line % n) * ms[1] + (line / n) * ms[2];
    lines[t] = (int32_t)num[g];
  }
}

}  // namespace

int setup_numbering_device(HostProblem* hp, int device, std::string* err) {
  HostProblem& P = *hp;
  if (P.desc.dg) return setup_numbering(hp, err);     // DG: cell-major, nothing to compute
  const int d = P.d, p = P.p, n = P.n;
  const int64_t Nc = (int64_t)P.cell_bg.size();
  const int64_t M = (int64_t)p * P.N + 1;
  int64_t nlat = 1;
  for (int i = 0; i < d; ++i) nlat *= M;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaError_t e = cudaSetDevice(device);
  int status = SBM_OK;
  if (e != cudaSuccess) {
    *err = std::string("cudaSetDevice: ") + cudaGetErrorString(e);
    return SBM_ERR_CUDA;
  }
  {
    DevBufs B;
    int32_t *cells, *mark, *lines;
    int64_t *num, *tot;
    int64_t nd = 0;
    if ((e = B.alloc(&cells, (size_t)Nc * d)) != cudaSuccess ||
        (e = B.alloc(&mark, (size_t)nlat)) != cudaSuccess ||
        (e = B.alloc(&num, (size_t)nlat)) != cudaSuccess ||
        (e = B.alloc(&tot, 1)) != cudaSuccess ||
        (e = B.alloc(&lines, (size_t)Nc * P.L)) != cudaSuccess ||
        (e = cudaMemcpy(cells, P.cells.data(), (size_t)Nc * d * 4, cudaMemcpyHostToDevice)) !=
            cudaSuccess ||
        (e = cudaMemset(mark, 0, (size_t)nlat * 4)) != cudaSuccess) {
      *err = std::string("numbering buffers: ") + cudaGetErrorString(e);
      status = (e == cudaErrorMemoryAllocation) ? SBM_ERR_OOM : SBM_ERR_CUDA;
    } else {
      k_mark<<<grid_for(Nc * P.nd), 256>>>(Nc, d, p, n, P.nd, M, cells, mark);
      if ((e = exclusive_scan(mark, nlat, num, tot, B)) == cudaSuccess &&
          (e = cudaMemcpy(&nd, tot, 8, cudaMemcpyDeviceToHost)) == cudaSuccess) {
        if (nd >= (int64_t(1) << 31) - 1) {
          *err = "too many DoFs for int32 indices";
          status = SBM_ERR_ARG;
        } else {
          k_lines<<<grid_for(Nc * P.L), 256>>>(Nc, d, p, n, P.L, M, cells, num, lines);
          P.lines.resize((size_t)Nc * P.L);
          if ((e = cudaGetLastError()) == cudaSuccess)
            e = cudaMemcpy(P.lines.data(), lines, P.lines.size() * 4, cudaMemcpyDeviceToHost);
          P.n_dofs = nd;
        }
      }
      if (status == SBM_OK && e != cudaSuccess) {
        *err = std::string("numbering kernels: ") + cudaGetErrorString(e);
        status = SBM_ERR_CUDA;
      }
    }
  }
  cudaSetDevice(prev);
  return status;
}

// ---- device tables of sbm_setup_face_data -------------------------------------

namespace {

// per chunk-ordered cell: the DoFs of its n^d nodes get the bit of its colour
__global__ void k_colour_masks(int64_t nc, int L, int n, const int32_t* __restrict__ lines,
                               const uint8_t* __restrict__ col, uint32_t* __restrict__ mask) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nc * L * n;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / ((int64_t)L * n);
    const int r = (int)(t - i * L * n);
    const int64_t g = (int64_t)lines[i * L + r / n] + (r % n);
    atomicOr(mask + g, 1u << col[i]);
  }
}

// Shared DoFs are listed slab by slab (DoF ranges [cut[s], cut[s+1])), and
// within a slab by colour count: group 0 = 2 colours, 1 = 3..4, 2 = 5..8
// (ascending DoF index within a group), so that a warp of the assembly
// kernel adds about as many values for each of its DoFs.
struct SlabCuts {
  int n;                         // slabs
  int64_t cut[kMaxSlabs + 1];    // DoF cut points
  int64_t base[kMaxSlabs][3];    // list offset of (slab, group)
  int64_t first[kMaxSlabs][3];   // group scan value at the slab's first DoF
};

__device__ __forceinline__ int multi_group(uint32_t m) {
  const int k = __popc(m);
  return k < 2 ? -1 : (k == 2 ? 0 : (k <= 4 ? 1 : 2));
}

__global__ void k_multi_flags(const uint32_t* __restrict__ mask, int64_t n, int group,
                              int32_t* __restrict__ flag) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n;
       g += (int64_t)gridDim.x * blockDim.x)
    flag[g] = (multi_group(mask[g]) == group) ? 1 : 0;
}

// pos: exclusive scan of the group's flags over all DoFs
__global__ void k_multi_write(const uint32_t* __restrict__ mask, const int32_t* __restrict__ flag,
                              const int64_t* __restrict__ pos, const SlabCuts sc, int group,
                              int64_t n, int32_t* __restrict__ multi,
                              uint8_t* __restrict__ multi_mask) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n;
       g += (int64_t)gridDim.x * blockDim.x)
    if (flag[g]) {
      int s = 0;
      while (s + 1 < sc.n && g >= sc.cut[s + 1]) ++s;
      const int64_t at = sc.base[s][group] + (pos[g] - sc.first[s][group]);
      multi[at] = (int32_t)g;
      multi_mask[at] = (uint8_t)mask[g];
    }
}

// out[s] = pos[cut[s]] (cut[s] < n) or total (cut[s] == n), s = 0..ns
__global__ void k_scan_at(const int64_t* __restrict__ pos, const int64_t* __restrict__ total,
                          const SlabCuts sc, int64_t n, int64_t* __restrict__ out) {
  const int s = threadIdx.x;
  if (s <= sc.n) out[s] = (sc.cut[s] < n) ? pos[sc.cut[s]] : *total;
}

// run element (l, kk) of chunk k shared by several colours -> bit l*S + kk
__global__ void k_run_bits(int nch, int L, int P, int R, int words, const int32_t* __restrict__ first,
                           const int32_t* __restrict__ lines, const uint32_t* __restrict__ mask,
                           uint32_t* __restrict__ bits) {
  const int Smax = P * R + 1;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < (int64_t)nch * L * Smax;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(t / ((int64_t)L * Smax));
    const int r = (int)(t - (int64_t)k * L * Smax);
    const int l = r / Smax, kk = r - l * Smax;
    const int S = P * (first[k + 1] - first[k]) + 1;
    if (kk >= S) continue;
    const int64_t g = (int64_t)lines[(int64_t)first[k] * L + l] + kk;
    if (__popc(mask[g]) >= 2) {
      const int b = l * S + kk;
      atomicOr(bits + (size_t)k * words + b / 32, 1u << (b % 32));
    }
  }
}

// ---- colour-ordered stores ----------------------------------------------------
constexpr int kDepCap = 64;       // lower-colour neighbours a chunk may have

// owner[g ncol + colour] = the chunk of that colour that touches DoF g, for
// the DoFs several colours share (the chunks of one colour are disjoint)
__global__ void k_dof_owner(int nch, int L, int P, int R, int ncol,
                            const int32_t* __restrict__ first, const int32_t* __restrict__ lines,
                            const uint8_t* __restrict__ col, const uint32_t* __restrict__ mask,
                            int32_t* __restrict__ owner) {
  const int Smax = P * R + 1;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < (int64_t)nch * L * Smax;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(t / ((int64_t)L * Smax));
    const int r = (int)(t - (int64_t)k * L * Smax);
    const int l = r / Smax, kk = r - l * Smax;
    if (kk >= P * (first[k + 1] - first[k]) + 1) continue;
    const int64_t g = (int64_t)lines[(int64_t)first[k] * L + l] + kk;
    if (__popc(mask[g]) >= 2) owner[g * ncol + col[k]] = k;
  }
}

// Per chunk: the run bits of the DoFs a lower colour also touches, and the
// set of lower-colour chunks it shares a DoF with (deps[k][0..ndeps[k]),
// deduplicated; more than kDepCap sets *overflow).
__global__ void k_chunk_deps(int nch, int L, int P, int R, int ncol, int words,
                             const int32_t* __restrict__ first, const int32_t* __restrict__ lines,
                             const uint8_t* __restrict__ col, const uint32_t* __restrict__ mask,
                             const int32_t* __restrict__ owner, int32_t* __restrict__ deps,
                             int32_t* __restrict__ ndeps, uint32_t* __restrict__ add_bits,
                             int* __restrict__ overflow) {
  const int Smax = P * R + 1;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < (int64_t)nch * L * Smax;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(t / ((int64_t)L * Smax));
    const int r = (int)(t - (int64_t)k * L * Smax);
    const int l = r / Smax, kk = r - l * Smax;
    const int S = P * (first[k + 1] - first[k]) + 1;
    if (kk >= S) continue;
    const int64_t g = (int64_t)lines[(int64_t)first[k] * L + l] + kk;
    const uint32_t m = mask[g];
    uint32_t lower = m & ((1u << col[k]) - 1u);
    if (__popc(m) < 2 || lower == 0u) continue;
    const int b = l * S + kk;
    atomicOr(add_bits + (size_t)k * words + b / 32, 1u << (b % 32));
    for (; lower; lower &= lower - 1u) {
      const int dep = owner[g * ncol + (__ffs(lower) - 1)];
      int32_t* list = deps + (size_t)k * kDepCap;
      int i = 0;
      for (; i < kDepCap; ++i) {
        const int old = atomicCAS(list + i, -1, dep);
        if (old == -1) {
          atomicAdd(ndeps + k, 1);
          break;
        }
        if (old == dep) break;
      }
      if (i == kDepCap) atomicExch(overflow, 1);
    }
  }
}

struct LagArgs {
  int n, d, L, taylor;
  double nodes[kMaxN], lam[kMaxN];
};

// the 1D Lagrange values at each shifted point (first barycentric form, exact
// Kronecker delta at the nodes), or (Taylor) the shift itself, in kernel face
// order
__global__ void k_face_phi(const LagArgs a, int64_t F, const int64_t* __restrict__ fsrc,
                           const double* __restrict__ xi, double* __restrict__ out,
                           float* __restrict__ out32) {
  const int per = a.taylor ? 1 : a.n;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < F * a.L * a.d;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t f = t / ((int64_t)a.L * a.d);
    const int r = (int)(t - f * a.L * a.d);              // q * d + l
    const double x = xi[(fsrc[f] * a.L) * a.d + r];
    double* o = out + t * per;
    float* o32 = out32 + t * per;
    if (a.taylor) {
      o[0] = x;
      o32[0] = (float)x;
      continue;
    }
    int hit = -1;
    for (int j = 0; j < a.n; ++j)
      if (x == a.nodes[j]) hit = j;
    double l = 1.0;
    for (int m = 0; m < a.n; ++m) l *= (x - a.nodes[m]);
    for (int j = 0; j < a.n; ++j) {
      const double v = (hit >= 0) ? ((j == hit) ? 1.0 : 0.0) : l * a.lam[j] / (x - a.nodes[j]);
      o[j] = v;
      o32[j] = (float)v;
    }
  }
}

}  // namespace

cudaError_t device_chunk_tables(const int32_t* lines, int64_t nc, int L, int n, int64_t n_dofs,
                                const std::vector<int32_t>& ch_first,
                                const std::vector<uint8_t>& ch_col, int R,
                                const int32_t* first_dev, const std::vector<int64_t>& ycut,
                                ChunkTable* ct, bool ordered) {
  DevBufs B;
  const int nch = (int)ch_col.size();
  std::vector<uint8_t> col(nc);
  for (int k = 0; k < nch; ++k)
    for (int i = ch_first[k]; i < ch_first[k + 1]; ++i) col[i] = ch_col[k];
  uint8_t* col_d;
  uint32_t* mask;
  int32_t* flag;
  int64_t *pos, *tot, *at;
  SlabCuts sc;
  sc.n = (int)ycut.size() - 1;
  if (sc.n < 1 || sc.n > kMaxSlabs) return cudaErrorInvalidValue;
  for (int s = 0; s <= sc.n; ++s) sc.cut[s] = ycut[s];
  cudaError_t e;
  if ((e = B.alloc(&col_d, (size_t)nc)) != cudaSuccess ||
      (e = B.alloc(&mask, (size_t)n_dofs)) != cudaSuccess ||
      (e = B.alloc(&flag, (size_t)n_dofs)) != cudaSuccess ||
      (e = B.alloc(&pos, (size_t)n_dofs)) != cudaSuccess || (e = B.alloc(&tot, 1)) != cudaSuccess ||
      (e = B.alloc(&at, (size_t)kMaxSlabs + 1)) != cudaSuccess ||
      (e = cudaMemcpy(col_d, col.data(), (size_t)nc, cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemset(mask, 0, (size_t)n_dofs * 4)) != cudaSuccess)
    return e;
  k_colour_masks<<<grid_for(nc * L * n), 256>>>(nc, L, n, lines, col_d, mask);
  // per group: the scan values at the slab cuts give the (slab, group) counts
  int64_t sv[3][kMaxSlabs + 1];
  for (int grp = 0; grp < 3; ++grp) {
    k_multi_flags<<<grid_for(n_dofs), 256>>>(mask, n_dofs, grp, flag);
    if ((e = exclusive_scan(flag, n_dofs, pos, tot, B)) != cudaSuccess) return e;
    k_scan_at<<<1, kMaxSlabs + 1>>>(pos, tot, sc, n_dofs, at);
    if ((e = cudaMemcpy(sv[grp], at, (size_t)(sc.n + 1) * 8, cudaMemcpyDeviceToHost)) !=
        cudaSuccess)
      return e;
  }
  int64_t nm = 0;
  ct->slab_multi.assign(sc.n + 1, 0);
  for (int s = 0; s < sc.n; ++s) {
    ct->slab_multi[s] = nm;
    for (int grp = 0; grp < 3; ++grp) {
      sc.base[s][grp] = nm;
      sc.first[s][grp] = sv[grp][s];
      nm += sv[grp][s + 1] - sv[grp][s];
    }
  }
  ct->slab_multi[sc.n] = nm;
  ct->nmulti = nm;
  if (nm > 0) {
    if ((e = cudaMalloc((void**)&ct->multi, (size_t)nm * 4)) != cudaSuccess ||
        (e = cudaMalloc((void**)&ct->multi_mask, (size_t)nm)) != cudaSuccess)
      return e;
    for (int grp = 0; grp < 3; ++grp) {
      if (sv[grp][sc.n] == sv[grp][0]) continue;
      k_multi_flags<<<grid_for(n_dofs), 256>>>(mask, n_dofs, grp, flag);
      if ((e = exclusive_scan(flag, n_dofs, pos, tot, B)) != cudaSuccess) return e;
      k_multi_write<<<grid_for(n_dofs), 256>>>(mask, flag, pos, sc, grp, n_dofs, ct->multi,
                                               ct->multi_mask);
    }
  }
  const int P = n - 1;
  const int words = (L * (P * R + 1) + 31) / 32;
  ct->bit_words = words;
  if ((e = cudaMalloc((void**)&ct->run_bits, (size_t)nch * words * 4)) != cudaSuccess ||
      (e = cudaMemset(ct->run_bits, 0, (size_t)nch * words * 4)) != cudaSuccess)
    return e;
  k_run_bits<<<grid_for((int64_t)nch * L * (P * R + 1)), 256>>>(nch, L, P, R, words, first_dev,
                                                                lines, mask, ct->run_bits);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (ordered && nch > 0) {
    // tickets in colour order (stable: row order within a colour)
    std::vector<int32_t> ord(nch);
    int at_ = 0;
    for (int c = 0; c < 8; ++c)
      for (int k = 0; k < nch; ++k)
        if (ch_col[k] == c) ord[at_++] = k;
    int ncol = 1;
    for (int k = 0; k < nch; ++k) ncol = std::max(ncol, (int)ch_col[k] + 1);
    int32_t* owner;
    int* overflow;
    const int64_t work = (int64_t)nch * L * (P * R + 1);
    if ((e = B.alloc(&owner, (size_t)n_dofs * ncol)) != cudaSuccess ||
        (e = B.alloc(&overflow, 1)) != cudaSuccess ||
        (e = cudaMemset(overflow, 0, sizeof(int))) != cudaSuccess ||
        (e = cudaMalloc((void**)&ct->ord, (size_t)nch * 4)) != cudaSuccess ||
        (e = cudaMemcpy(ct->ord, ord.data(), (size_t)nch * 4, cudaMemcpyHostToDevice)) !=
            cudaSuccess ||
        (e = cudaMalloc((void**)&ct->add_bits, (size_t)nch * words * 4)) != cudaSuccess ||
        (e = cudaMemset(ct->add_bits, 0, (size_t)nch * words * 4)) != cudaSuccess ||
        (e = cudaMalloc((void**)&ct->deps, (size_t)nch * kDepCap * 4)) != cudaSuccess ||
        (e = cudaMemset(ct->deps, 0xff, (size_t)nch * kDepCap * 4)) != cudaSuccess ||
        (e = cudaMalloc((void**)&ct->ndeps, (size_t)nch * 4)) != cudaSuccess ||
        (e = cudaMemset(ct->ndeps, 0, (size_t)nch * 4)) != cudaSuccess ||
        (e = cudaMalloc((void**)&ct->done, (size_t)nch * 4)) != cudaSuccess ||
        (e = cudaMemset(ct->done, 0, (size_t)nch * 4)) != cudaSuccess ||
        (e = cudaMalloc((void**)&ct->tickets, 2 * sizeof(uint32_t))) != cudaSuccess ||
        (e = cudaMemset(ct->tickets, 0, 2 * sizeof(uint32_t))) != cudaSuccess)
      return e;
    k_dof_owner<<<grid_for(work), 256>>>(nch, L, P, R, ncol, first_dev, lines, ct->colour, mask,
                                         owner);
    k_chunk_deps<<<grid_for(work), 256>>>(nch, L, P, R, ncol, words, first_dev, lines,
                                          ct->colour, mask, owner, ct->deps, ct->ndeps,
                                          ct->add_bits, overflow);
    int of = 0;
    if ((e = cudaGetLastError()) != cudaSuccess ||
        (e = cudaMemcpy(&of, overflow, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess)
      return e;
    ct->dep_cap = kDepCap;
    ct->ordered = of == 0;
  }
  return cudaDeviceSynchronize();
}

// pp[(f n^2 + j12) L + q] = phi[f][q][1][j1] phi[f][q][2][j2], j12 = j1 + n j2
__global__ void k_face_pp(int64_t F, int L, int n, const double* __restrict__ phi,
                          double* __restrict__ pp) {
  const int64_t nn = (int64_t)n * n;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < F * nn * L;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int q = (int)(t % L);
    const int64_t fj = t / L;
    const int j12 = (int)(fj % nn);
    const int64_t f = fj / nn;
    const int j1 = j12 % n, j2 = j12 / n;
    const double* pq = phi + ((size_t)f * L + q) * 3 * n;
    pp[t] = pq[n + j1] * pq[2 * n + j2];
  }
}

cudaError_t device_face_pp(int64_t F, int L, int n, const double* phi, double** pp) {
  *pp = nullptr;
  if (F == 0) return cudaSuccess;
  const size_t cnt = (size_t)F * n * n * L;
  cudaError_t e;
  if ((e = cudaMalloc((void**)pp, cnt * 8)) != cudaSuccess) return e;
  k_face_pp<<<grid_for((int64_t)cnt), 256>>>(F, L, n, phi, *pp);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  return cudaDeviceSynchronize();
}

cudaError_t device_face_phi(const HostProblem& hp, const std::vector<int64_t>& fsrc,
                            double** phi, float** phi32) {
  DevBufs B;
  const int64_t F = (int64_t)fsrc.size();
  const int d = hp.d, L = hp.L, n = hp.n;
  const bool taylor = hp.desc.extension == SBM_EXT_TAYLOR1;
  const size_t per = taylor ? 1 : n;
  const size_t cnt = (size_t)F * L * d * per;
  *phi = nullptr;
  *phi32 = nullptr;
  if (F == 0) return cudaSuccess;
  const std::vector<double>& src = taylor ? hp.face_d : hp.face_xi;
  int64_t* fsrc_d;
  double* xi_d;
  cudaError_t e;
  if ((e = B.alloc(&fsrc_d, (size_t)F)) != cudaSuccess ||
      (e = B.alloc(&xi_d, src.size())) != cudaSuccess ||
      (e = cudaMemcpy(fsrc_d, fsrc.data(), (size_t)F * 8, cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(xi_d, src.data(), src.size() * 8, cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMalloc((void**)phi, cnt * 8)) != cudaSuccess ||
      (e = cudaMalloc((void**)phi32, cnt * 4)) != cudaSuccess)
    return e;
  LagArgs la;
  la.n = n;
  la.d = d;
  la.L = L;
  la.taylor = taylor;
  for (int j = 0; j < kMaxN; ++j) {
    la.nodes[j] = hp.tab.nodes[j];
    la.lam[j] = 0.0;
  }
  for (int j = 0; j < n; ++j) {             // barycentric weights 1 / prod_{m != j} (x_j - x_m)
    double prod = 1.0;
    for (int m = 0; m < n; ++m)
      if (m != j) prod *= (hp.tab.nodes[j] - hp.tab.nodes[m]);
    la.lam[j] = 1.0 / prod;
  }
  k_face_phi<<<grid_for(F * L * d), 256>>>(la, F, fsrc_d, xi_d, *phi, *phi32);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  return cudaDeviceSynchronize();
}

int setup_geometry_device(HostProblem* hp, int device, std::string* err) {
  HostProblem& P = *hp;
  const int d = P.d, N = P.N, n = P.n, Q = P.L;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaError_t e = cudaSetDevice(device);
  if (e != cudaSuccess) {
    *err = std::string("cudaSetDevice: ") + cudaGetErrorString(e);
    return SBM_ERR_CUDA;
  }
  int status = SBM_OK;
  {
    DevBufs B;
    auto fail = [&](cudaError_t ce, const char* what) {
      *err = std::string(what) + ": " + cudaGetErrorString(ce);
      status = (ce == cudaErrorMemoryAllocation) ? SBM_ERR_OOM : SBM_ERR_CUDA;
    };
    // level set with device copies of the ball data
    GeomView gv = P.ls.view();
    double *bc = nullptr, *br = nullptr, *vt = nullptr;
    GeomCircle* circ = nullptr;
    if (gv.nb > 0) {
      if ((e = B.alloc(&bc, 3 * (size_t)gv.nb)) != cudaSuccess ||
          (e = B.alloc(&br, (size_t)gv.nb)) != cudaSuccess ||
          (e = B.alloc(&circ, (size_t)gv.ncirc)) != cudaSuccess ||
          (e = B.alloc(&vt, 3 * (size_t)gv.nvert)) != cudaSuccess ||
          (e = cudaMemcpy(bc, gv.bc, 3 * (size_t)gv.nb * 8, cudaMemcpyHostToDevice)) != cudaSuccess ||
          (e = cudaMemcpy(br, gv.br, (size_t)gv.nb * 8, cudaMemcpyHostToDevice)) != cudaSuccess ||
          (gv.ncirc > 0 && (e = cudaMemcpy(circ, gv.circ, gv.ncirc * sizeof(GeomCircle),
                                           cudaMemcpyHostToDevice)) != cudaSuccess) ||
          (gv.nvert > 0 && (e = cudaMemcpy(vt, gv.verts, 3 * (size_t)gv.nvert * 8,
                                           cudaMemcpyHostToDevice)) != cudaSuccess)) {
        fail(e, "geometry upload");
        goto done;
      }
      gv.bc = bc;
      gv.br = br;
      gv.circ = circ;
      gv.verts = vt;
    }
    {
      int64_t nbg = 1;
      for (int i = 0; i < d; ++i) nbg *= N;
      int32_t *flag, *bg_to_cell, *cells, *nsf, *nif, *sfaces = nullptr, *ifaces = nullptr;
      int64_t *rank, *cell_bg, *tot, *osf, *oif;
      int* failed;
      if ((e = B.alloc(&flag, nbg)) != cudaSuccess || (e = B.alloc(&rank, nbg)) != cudaSuccess ||
          (e = B.alloc(&bg_to_cell, nbg)) != cudaSuccess || (e = B.alloc(&tot, 3)) != cudaSuccess ||
          (e = B.alloc(&failed, 1)) != cudaSuccess ||
          (e = cudaMemset(failed, 0, sizeof(int))) != cudaSuccess) {
        fail(e, "device set-up buffers");
        goto done;
      }
      GeoArgs ga;
      ga.g = gv;
      ga.d = d;
      ga.N = N;
      ga.activity = P.desc.activity;
      ga.h = P.h;
      ga.vf_threshold = P.desc.vf_threshold;
      k_active<<<grid_for(nbg), 256>>>(ga, nbg, flag);
      if ((e = exclusive_scan(flag, nbg, rank, tot, B)) != cudaSuccess) {
        fail(e, "active-cell scan");
        goto done;
      }
      int64_t Nc = 0;
      if ((e = cudaMemcpy(&Nc, tot, sizeof(int64_t), cudaMemcpyDeviceToHost)) != cudaSuccess) {
        fail(e, "active-cell count");
        goto done;
      }
      if (Nc == 0) {
        *err = "no active cell";
        status = SBM_ERR_EMPTY_DOMAIN;
        goto done;
      }
      if ((e = B.alloc(&cells, (size_t)Nc * d)) != cudaSuccess ||
          (e = B.alloc(&cell_bg, (size_t)Nc)) != cudaSuccess ||
          (e = B.alloc(&nsf, (size_t)Nc)) != cudaSuccess ||
          (e = B.alloc(&nif, (size_t)Nc)) != cudaSuccess ||
          (e = B.alloc(&osf, (size_t)Nc)) != cudaSuccess ||
          (e = B.alloc(&oif, (size_t)Nc)) != cudaSuccess) {
        fail(e, "cell buffers");
        goto done;
      }
      k_cells<<<grid_for(nbg), 256>>>(flag, rank, nbg, d, N, cells, cell_bg, bg_to_cell);
      k_faces<<<grid_for(Nc), 256>>>(0, Nc, d, N, cells, cell_bg, bg_to_cell, nsf, nif, nullptr,
                                     nullptr, nullptr, nullptr);
      if ((e = exclusive_scan(nsf, Nc, osf, tot + 1, B)) != cudaSuccess ||
          (e = exclusive_scan(nif, Nc, oif, tot + 2, B)) != cudaSuccess) {
        fail(e, "face scans");
        goto done;
      }
      int64_t counts[3];
      if ((e = cudaMemcpy(counts, tot, 3 * sizeof(int64_t), cudaMemcpyDeviceToHost)) != cudaSuccess) {
        fail(e, "face counts");
        goto done;
      }
      const int64_t F = counts[1], FI = counts[2];
      if ((e = B.alloc(&sfaces, 3 * (size_t)F)) != cudaSuccess ||
          (e = B.alloc(&ifaces, 3 * (size_t)FI)) != cudaSuccess) {
        fail(e, "face buffers");
        goto done;
      }
      k_faces<<<grid_for(Nc), 256>>>(1, Nc, d, N, cells, cell_bg, bg_to_cell, nsf, nif, osf, oif,
                                     sfaces, ifaces);
      double *fx, *fxi, *fd;
      if ((e = B.alloc(&fx, (size_t)F * Q * d)) != cudaSuccess ||
          (e = B.alloc(&fxi, (size_t)F * Q * d)) != cudaSuccess ||
          (e = B.alloc(&fd, (size_t)F * Q * d)) != cudaSuccess) {
        fail(e, "face point buffers");
        goto done;
      }
      PointArgs pa;
      pa.g = gv;
      pa.d = d;
      pa.n = n;
      pa.L = Q;
      pa.h = P.h;
      for (int i = 0; i < kMaxN; ++i) pa.gpts[i] = P.tab.gpts[i];
      if (F > 0) k_face_points<<<grid_for(F * Q), 256>>>(pa, F, sfaces, cells, fx, fxi, fd, failed);
      if ((e = cudaGetLastError()) != cudaSuccess || (e = cudaDeviceSynchronize()) != cudaSuccess) {
        fail(e, "geometry kernels");
        goto done;
      }
      int bad = 0;
      if ((e = cudaMemcpy(&bad, failed, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess) {
        fail(e, "geometry status");
        goto done;
      }
      if (bad) {
        *err = "closest-point projection undefined for a surrogate quadrature point";
        status = SBM_ERR_GEOMETRY;
        goto done;
      }
      // back to the host problem
      P.cells.resize((size_t)Nc * d);
      P.cell_bg.resize((size_t)Nc);
      P.bg_to_cell.resize((size_t)nbg);
      P.sfaces.resize(3 * (size_t)F);
      P.ifaces.resize(3 * (size_t)FI);
      P.face_x.resize((size_t)F * Q * d);
      P.face_xi.resize((size_t)F * Q * d);
      P.face_d.resize((size_t)F * Q * d);
      struct {
        void* dst;
        const void* src;
        size_t bytes;
      } cp[] = {{P.cells.data(), cells, P.cells.size() * 4},
                {P.cell_bg.data(), cell_bg, P.cell_bg.size() * 8},
                {P.bg_to_cell.data(), bg_to_cell, P.bg_to_cell.size() * 4},
                {P.sfaces.data(), sfaces, P.sfaces.size() * 4},
                {P.ifaces.data(), ifaces, P.ifaces.size() * 4},
                {P.face_x.data(), fx, P.face_x.size() * 8},
                {P.face_xi.data(), fxi, P.face_xi.size() * 8},
                {P.face_d.data(), fd, P.face_d.size() * 8}};
      for (auto& c : cp)
        if (c.bytes && (e = cudaMemcpy(c.dst, c.src, c.bytes, cudaMemcpyDeviceToHost)) != cudaSuccess) {
          fail(e, "geometry download");
          goto done;
        }
    }
  done:;
  }
  cudaSetDevice(prev);
  return status;
}

}  // namespace sbm
