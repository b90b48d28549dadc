// C ABI of the SBM operator library (declarations and contracts in include/sbm.h).
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <string>

#include "internal.hpp"
#include "krylov.hpp"

namespace sbm {

static thread_local std::string g_detail;

static int fail(int code, const std::string& msg) {
  g_detail = msg;
  return code;
}

static int cuda_fail(cudaError_t e, const char* where) {
  g_detail = std::string(where) + ": " + cudaGetErrorString(e);
  return SBM_ERR_CUDA;
}

template <typename T>
KTab<T> make_ktab(const HostProblem& hp) {
  KTab<T> t;
  std::memset(&t, 0, sizeof(t));
  const Tables1D& tb = hp.tab;
  const int n = hp.n;
  const double hd2 = std::pow(hp.h, hp.d - 2);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      t.M[i][j] = (T)tb.M[i][j];
      t.K[i][j] = (T)tb.K[i][j];
      t.Mh[i][j] = (T)(hd2 * tb.M[i][j]);
      t.Kh[i][j] = (T)(hd2 * tb.K[i][j]);
      t.S[i][j] = (T)tb.S[i][j];
      t.Dg[i][j] = (T)tb.Dg[i][j];
    }
  for (int j = 0; j < n; ++j) {
    t.D0[j] = (T)tb.D0[j];
    t.D1[j] = (T)tb.D1[j];
  }
  const double hd1 = std::pow(hp.h, hp.d - 1);
  for (int q = 0; q < hp.L; ++q) {
    const int qa = q % n, qb = q / n;
    const double w = (hp.d == 3) ? tb.gwts[qa] * tb.gwts[qb] : tb.gwts[qa];
    t.W[q] = (T)(hd1 * w);
  }
  t.h_inv = (T)(1.0 / hp.h);
  t.hface = (T)hd1;
  t.sigma = (T)hp.sigma;
  auto fold = [n](const double (&A)[kMaxN][kMaxN], double scale, Folded<T>* f) {
    const int H = n / 2, HE = (n + 1) / 2;
    for (int i = 0; i < HE; ++i)
      for (int j = 0; j < HE; ++j) {
        const bool mid = (n & 1) && j == n / 2;
        f->E[i][j] = (T)(scale * (mid ? A[i][j] : 0.5 * (A[i][j] + A[i][n - 1 - j])));
        if (i < H && j < H) f->O[i][j] = (T)(scale * 0.5 * (A[i][j] - A[i][n - 1 - j]));
      }
  };
  fold(tb.M, 1.0, &t.fM);
  fold(tb.K, 1.0, &t.fK);
  fold(tb.M, hd2, &t.fMh);
  fold(tb.K, hd2, &t.fKh);
  // V^T on a folded line: even mode ke = sum_{j < HE} V[j][ke] e_j, odd mode
  // ko = sum_{j < H} V[j][ko] o_j; V on the modes: s_j = sum V[j][ke] w_ke,
  // d_j = sum V[j][ko] w_ko, then y_j = s_j + d_j, y_{n-1-j} = s_j - d_j
  {
    const int H = n / 2, HE = (n + 1) / 2;
    for (int i = 0; i < HE; ++i)
      for (int j = 0; j < HE; ++j) {
        t.fVt.E[i][j] = (T)tb.V[j][i];
        t.fV.E[j][i] = (T)tb.V[j][i];
      }
    for (int i = 0; i < H; ++i)
      for (int j = 0; j < H; ++j) {
        t.fVt.O[i][j] = (T)tb.V[j][HE + i];
        t.fV.O[j][i] = (T)tb.V[j][HE + i];
      }
    for (int k = 0; k < n; ++k) t.hlam[k] = (T)(hd2 * tb.lam[k]);
  }
  return t;
}
template KTab<double> make_ktab<double>(const HostProblem&);
template KTab<float> make_ktab<float>(const HostProblem&);

cudaError_t Profiler::mark(cudaStream_t st) {
  if (used + 1 > ev.size()) {
    for (int i = 0; i < 64 * kMarks; ++i) {
      cudaEvent_t e;
      cudaError_t err = cudaEventCreate(&e);
      if (err != cudaSuccess) return err;
      ev.push_back(e);
    }
  }
  return cudaEventRecord(ev[used++], st);
}

void Profiler::release() {
  for (cudaEvent_t e : ev) cudaEventDestroy(e);
  ev.clear();
  used = 0;
  launches = 0;
}

template <typename T>
static cudaError_t upload(T** dst, const T* src, size_t count) {
  *dst = nullptr;
  if (count == 0) return cudaSuccess;
  cudaError_t e = cudaMalloc((void**)dst, count * sizeof(T));
  if (e != cudaSuccess) return e;
  return cudaMemcpy(*dst, src, count * sizeof(T), cudaMemcpyHostToDevice);
}

static void free_device(DeviceData* dd) {
  cudaFree(dd->lines);
  cudaFree(dd->reg_cell_chunk);
  cudaFree(dd->reg_block_first);
  cudaFree(dd->reg_mask);
  cudaFree(dd->cell_rank);
  cudaFree(dd->face_start);
  cudaFree(dd->face_kind);
  cudaFree(dd->face_cell);
  cudaFree(dd->face_out);
  cudaFree(dd->face_out32);
  for (auto& ct : dd->chunks) {
    cudaFree(ct.first);
    cudaFree(ct.colour);
    cudaFree(ct.run_bits);
    cudaFree(ct.multi);
    cudaFree(ct.multi_mask);
    cudaFree(ct.ord);
    cudaFree(ct.add_bits);
    cudaFree(ct.deps);
    cudaFree(ct.ndeps);
    cudaFree(ct.done);
    cudaFree(ct.tickets);
  }
  cudaFree(dd->diag_pos);
  cudaFree(dd->err_flag);
  cudaFree(dd->ycol);
  cudaFree(dd->ycol32);
  cudaFree(dd->face_phi);
  cudaFree(dd->face_phi32);
  cudaFree(dd->face_pp);
  cudaFree(dd->nbr);
  cudaFree(dd->stage_x);
  cudaFree(dd->stage_y);
  for (cudaEvent_t ev : dd->ev_in)
    if (ev) cudaEventDestroy(ev);
  for (cudaEvent_t ev : dd->ev_face)
    if (ev) cudaEventDestroy(ev);
  for (cudaEvent_t ev : dd->ev_done)
    if (ev) cudaEventDestroy(ev);
  if (dd->face_st) cudaStreamDestroy(dd->face_st);
  if (dd->cap_st) cudaStreamDestroy(dd->cap_st);
  for (auto& g : dd->host_graphs) cudaGraphExecDestroy(g.exec);
  if (dd->ev_fork) cudaEventDestroy(dd->ev_fork);
  if (dd->ev_join) cudaEventDestroy(dd->ev_join);
  if (dd->copy_in) cudaStreamDestroy(dd->copy_in);
  if (dd->copy_out) cudaStreamDestroy(dd->copy_out);
  *dd = DeviceData();
}

// Order the cells for the kernels and upload the set-up data.
static int build_device(const HostProblem& hp, DeviceData* dd) {
  const int d = hp.d, n = hp.n, L = hp.L;
  const int64_t Nc = (int64_t)hp.cell_bg.size();
  const int64_t F = (int64_t)hp.sfaces.size() / 3;
  // faces per cell (surrogate faces are grouped by cell already)
  std::vector<int32_t> nf(Nc, 0), first_face(Nc, -1);
  for (int64_t f = 0; f < F; ++f) {
    const int c = hp.sfaces[3 * f];
    if (first_face[c] < 0) first_face[c] = (int32_t)f;
    nf[c]++;
  }
  dd->ncolours = hp.desc.dg ? 1 : (1 << d);
  dd->col_start.assign(dd->ncolours + 1, 0);
  dd->col_nint.assign(dd->ncolours, 0);
  dd->order.clear();
  dd->order.reserve(Nc);
  // CG chunk tables (host side): chunk start positions and colours
  std::vector<int32_t> ch_first[2];
  std::vector<uint8_t> ch_col[2];
  if (hp.desc.dg) {
    // DG: one launch over all cells, interior cells first
    for (int pass = 0; pass < 2; ++pass)
      for (int64_t c = 0; c < Nc; ++c)
        if ((pass == 0) == (nf[c] == 0)) dd->order.push_back((int32_t)c);
    int nint = 0;
    for (int64_t c = 0; c < Nc; ++c)
      if (nf[c] == 0) nint++;
    dd->col_nint[0] = nint;
  } else {
    // CG: cells in row-run order (rows lexicographic, x fastest); each run of
    // consecutive active cells along x is cut into chunks of R (resp. R/2)
    // cells; chunk colour = (index of the chunk within its run) mod 2 |
    // (cy mod 2) << 1 | (cz mod 2) << 2
    const int N = hp.N;
    const int Rs[2] = {chunk_cells(d, n), std::max(1, chunk_cells(d, n) / 2)};
    const int64_t nrows = (d == 3) ? (int64_t)N * N : N;
    for (int64_t row = 0; row < nrows; ++row) {
      const int cy = (int)(row % N), cz = (d == 3) ? (int)(row / N) : 0;
      int cx = 0;
      while (cx < N) {
        if (hp.bg_to_cell[row * N + cx] < 0) { ++cx; continue; }
        const int run0 = (int)dd->order.size();
        while (cx < N && hp.bg_to_cell[row * N + cx] >= 0) {
          dd->order.push_back(hp.bg_to_cell[row * N + cx]);
          ++cx;
        }
        const int runlen = (int)dd->order.size() - run0;
        for (int v = 0; v < 2; ++v)
          for (int k = 0; k * Rs[v] < runlen; ++k) {
            ch_first[v].push_back(run0 + k * Rs[v]);
            ch_col[v].push_back((uint8_t)((k & 1) | ((cy & 1) << 1) | ((cz & 1) << 2)));
          }
      }
    }
    for (int v = 0; v < 2; ++v) ch_first[v].push_back((int32_t)dd->order.size());
  }
  dd->col_start[dd->ncolours] = (int)dd->order.size();
  for (int col = 1; col < dd->ncolours; ++col) dd->col_start[col] = dd->col_start[dd->ncolours];

  std::vector<int32_t> lines_o, fstart(Nc + 1, 0), fkind, fcell;
  std::vector<int64_t> fsrc;             // kernel face order -> face index
  if (!hp.desc.dg) lines_o.resize(Nc * L);
  fkind.reserve(F);
  fsrc.reserve(F);
  for (int64_t i = 0; i < Nc; ++i) {
    const int c = dd->order[i];
    if (!hp.desc.dg)
      std::memcpy(&lines_o[i * L], &hp.lines[(int64_t)c * L], L * sizeof(int32_t));
    fstart[i] = (int32_t)fkind.size();
    for (int j = 0; j < nf[c]; ++j) {
      const int64_t f = first_face[c] + j;
      fkind.push_back(hp.sfaces[3 * f + 1] | (hp.sfaces[3 * f + 2] << 2));
      fcell.push_back((int32_t)i);
      fsrc.push_back(f);
    }
  }
  fstart[Nc] = (int32_t)fkind.size();

  // CG: slabs of the pipelined host-buffer apply -- whole cell layers along
  // the last axis (cells are ordered layer by layer, the DoF numbering is
  // monotone in the lattice plane along that axis), cut where the cell count
  // first reaches each share of kSlabCuts
  std::vector<int64_t> ycut{0, hp.n_dofs};
  std::vector<int> slab_cell{0, (int)Nc};
  if (!hp.desc.dg) {
    const int N = hp.N, p = hp.p, dl = d - 1;
    const int64_t M = (int64_t)p * N + 1;                 // lattice planes
    std::vector<int64_t> per(N, 0);
    for (int64_t i = 0; i < Nc; ++i) per[hp.cells[(int64_t)dd->order[i] * d + dl]]++;
    std::vector<int> zb{0};
    int64_t cum = 0, last = 0;
    const int ncut = (int)(sizeof(kSlabCuts) / sizeof(kSlabCuts[0]));
    for (int z = 0, k = 0; z + 1 < N && k < ncut; ++z) {
      cum += per[z];
      if (cum > last && (double)cum >= kSlabCuts[k] * (double)Nc) {
        zb.push_back(z + 1);
        last = cum;
        while (k < ncut && (double)cum >= kSlabCuts[k] * (double)Nc) ++k;
      }
    }
    zb.push_back(N);
    // first DoF of each lattice plane (of the next non-empty one if empty)
    std::vector<int64_t> pf(M + 1, INT64_MAX);
    pf[M] = hp.n_dofs;
    for (int64_t c = 0; c < Nc; ++c) {
      const int64_t cz = hp.cells[c * d + dl];
      for (int line = 0; line < L; ++line) {
        const int64_t kz = p * cz + ((d == 3) ? line / n : line);
        pf[kz] = std::min<int64_t>(pf[kz], hp.lines[c * L + line]);
      }
    }
    for (int64_t kz = M - 1; kz >= 0; --kz) pf[kz] = std::min(pf[kz], pf[kz + 1]);
    const int ns = (int)zb.size() - 1;
    dd->nslab = ns;
    ycut.assign(ns + 1, hp.n_dofs);
    slab_cell.assign(ns + 1, (int)Nc);
    dd->slab_x.assign(ns, hp.n_dofs);
    int64_t before = 0;
    for (int s = 0, z = 0; s < ns; ++s) {
      for (; z < zb[s]; ++z) before += per[z];
      slab_cell[s] = (int)before;
      ycut[s] = pf[(int64_t)p * zb[s]];
      dd->slab_x[s] = pf[std::min<int64_t>((int64_t)p * zb[s + 1] + 1, M)];
    }
    dd->slab_y = ycut;
    dd->slab_face.assign(ns + 1, 0);
    for (int s = 0; s <= ns; ++s) dd->slab_face[s] = fstart[slab_cell[s]];
    for (int v = 0; v < 2; ++v) {
      dd->chunks[v].slab_chunk.assign(ns + 1, 0);
      for (int s = 0; s <= ns; ++s)
        dd->chunks[v].slab_chunk[s] =
            (int)(std::lower_bound(ch_first[v].begin(), ch_first[v].end(), slab_cell[s]) -
                  ch_first[v].begin());
    }
  }

  std::vector<int32_t> nbr;
  if (hp.desc.dg) {
    nbr.assign(Nc * 2 * d, -1);
    const int N = hp.N;
    int64_t stride[3] = {1, N, (int64_t)N * N};
    for (int64_t c = 0; c < Nc; ++c)
      for (int k = 0; k < d; ++k)
        for (int s = 0; s < 2; ++s) {
          const int j = hp.cells[c * d + k] + (s ? 1 : -1);
          if (j < 0 || j >= N) continue;
          nbr[c * 2 * d + 2 * k + s] = hp.bg_to_cell[hp.cell_bg[c] + (s ? 1 : -1) * stride[k]];
        }
  }
  cudaError_t e;
  if ((e = upload(&dd->nbr, nbr.data(), nbr.size())) != cudaSuccess) goto err;
  if ((e = upload(&dd->lines, lines_o.data(), lines_o.size())) != cudaSuccess) goto err;
  if ((e = upload(&dd->cell_rank, dd->order.data(), dd->order.size())) != cudaSuccess) goto err;
  if ((e = upload(&dd->face_start, fstart.data(), fstart.size())) != cudaSuccess) goto err;
  if ((e = upload(&dd->face_kind, fkind.data(), fkind.size())) != cudaSuccess) goto err;
  if ((e = upload(&dd->face_cell, fcell.data(), fcell.size())) != cudaSuccess) goto err;
  dd->nface = (int)fkind.size();
  if ((e = cudaMalloc((void**)&dd->err_flag, sizeof(int))) != cudaSuccess) goto err;
  if ((e = cudaMemset(dd->err_flag, 0, sizeof(int))) != cudaSuccess) goto err;
  if (!hp.desc.dg) {
    // per chunking: chunk tables, then on the device the per-DoF colour sets,
    // the list of DoFs several colours share and the per-chunk run bits
    for (int v = 0; v < 2; ++v) {
      const int nch = (int)ch_col[v].size();
      dd->chunks[v].n = nch;
      if ((e = upload(&dd->chunks[v].first, ch_first[v].data(), ch_first[v].size())) !=
          cudaSuccess)
        goto err;
      if ((e = upload(&dd->chunks[v].colour, ch_col[v].data(), ch_col[v].size())) != cudaSuccess)
        goto err;
      const int R = v == 0 ? chunk_cells(d, n) : std::max(chunk_cells(d, n) / 2, 1);
      if ((e = device_chunk_tables(dd->lines, Nc, L, n, hp.n_dofs, ch_first[v], ch_col[v], R,
                                   dd->chunks[v].first, ycut, &dd->chunks[v], v == 0)) !=
          cudaSuccess)
        goto err;
    }
    if ((e = build_cell_reg_tables(hp, ch_first[0], dd)) != cudaSuccess) goto err;
    // ordered positions grouped by the parity colour of the cell (diagonal kernel)
    {
      std::vector<int32_t> pos;
      dd->diag_col_start.assign(dd->ncolours + 1, 0);
      for (int col = 0; col < dd->ncolours; ++col) {
        dd->diag_col_start[col] = (int)pos.size();
        for (int64_t i = 0; i < Nc; ++i) {
          const int c = dd->order[i];
          int cc = 0;
          for (int l = 0; l < d; ++l) cc |= (hp.cells[(int64_t)c * d + l] & 1) << l;
          if (cc == col) pos.push_back((int32_t)i);
        }
      }
      dd->diag_col_start[dd->ncolours] = (int)pos.size();
      if ((e = upload(&dd->diag_pos, pos.data(), pos.size())) != cudaSuccess) goto err;
    }
    const size_t nb = (size_t)dd->ncolours * hp.n_dofs;
    if ((e = cudaMalloc((void**)&dd->ycol, nb * sizeof(double))) != cudaSuccess) goto err;
    if ((e = cudaMalloc((void**)&dd->ycol32, nb * sizeof(float))) != cudaSuccess) goto err;
  }
  if (dd->nface > 0) {
    if ((e = cudaMalloc((void**)&dd->face_out, (size_t)dd->nface * 2 * L * sizeof(double))) !=
        cudaSuccess)
      goto err;
    if ((e = cudaMalloc((void**)&dd->face_out32, (size_t)dd->nface * 2 * L * sizeof(float))) !=
        cudaSuccess)
      goto err;
  }
  if ((e = device_face_phi(hp, fsrc, &dd->face_phi, &dd->face_phi32)) != cudaSuccess) goto err;
  if (d == 3 && hp.desc.extension == SBM_EXT_EXACT &&
      (e = device_face_pp((int64_t)fsrc.size(), L, n, dd->face_phi, &dd->face_pp)) !=
          cudaSuccess)
    goto err;
  if (dd->nslab > 1) {
    // copy streams and events of the pipelined host-buffer apply
    const unsigned fl = cudaEventDisableTiming;
    if ((e = cudaStreamCreateWithFlags(&dd->copy_in, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&dd->copy_out, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&dd->face_st, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&dd->cap_st, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&dd->ev_fork, fl)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&dd->ev_join, fl)) != cudaSuccess)
      goto err;
    dd->ev_in.assign(dd->nslab, nullptr);
    dd->ev_face.assign(dd->nslab, nullptr);
    dd->ev_done.assign(dd->nslab, nullptr);
    for (int s = 0; s < dd->nslab; ++s)
      if ((e = cudaEventCreateWithFlags(&dd->ev_in[s], fl)) != cudaSuccess ||
          (e = cudaEventCreateWithFlags(&dd->ev_face[s], fl)) != cudaSuccess ||
          (e = cudaEventCreateWithFlags(&dd->ev_done[s], fl)) != cudaSuccess)
        goto err;
  }
  return SBM_OK;
err:
  free_device(dd);
  return e == cudaErrorMemoryAllocation ? fail(SBM_ERR_OOM, "device allocation failed")
                                        : cuda_fail(e, "upload");
}

// The slab pipeline of the host-buffer apply, enqueued after the work on
// origin and joined back to it: per slab, the copy of its part of x
// (copy_in), its face kernel (face_st), its chunks and completed assembly
// (origin), the copy of the part of y it finishes (copy_out).
cudaError_t enqueue_host_pipeline(const HostProblem& hp, const DeviceData& dd, const double* x_host,
                                  double* y_host, cudaStream_t origin) {
  cudaError_t e;
  if ((e = cudaEventRecord(dd.ev_fork, origin)) != cudaSuccess ||
      (e = cudaStreamWaitEvent(dd.copy_in, dd.ev_fork, 0)) != cudaSuccess ||
      (e = cudaStreamWaitEvent(dd.face_st, dd.ev_fork, 0)) != cudaSuccess ||
      (e = cudaStreamWaitEvent(dd.copy_out, dd.ev_fork, 0)) != cudaSuccess)
    return e;
  int64_t xdone = 0;
  for (int s = 0; s < dd.nslab; ++s) {
    const int64_t x1 = dd.slab_x[s], y0 = dd.slab_y[s], y1 = dd.slab_y[s + 1];
    if (x1 > xdone &&
        (e = cudaMemcpyAsync(dd.stage_x + xdone, x_host + xdone, (size_t)(x1 - xdone) * 8,
                             cudaMemcpyHostToDevice, dd.copy_in)) != cudaSuccess)
      return e;
    xdone = std::max(xdone, x1);
    if ((e = cudaEventRecord(dd.ev_in[s], dd.copy_in)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(dd.face_st, dd.ev_in[s], 0)) != cudaSuccess)
      return e;
    if ((e = launch_cg_apply_slab(hp, dd, dd.stage_x, dd.stage_y, s, 1, dd.face_st)) !=
        cudaSuccess)
      return e;
    // the chunks of slab s wait for its faces (and so for its part of x)
    if ((e = cudaEventRecord(dd.ev_face[s], dd.face_st)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(origin, dd.ev_face[s], 0)) != cudaSuccess)
      return e;
    if ((e = launch_cg_apply_slab(hp, dd, dd.stage_x, dd.stage_y, s, 2, origin)) != cudaSuccess)
      return e;
    if ((e = cudaEventRecord(dd.ev_done[s], origin)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(dd.copy_out, dd.ev_done[s], 0)) != cudaSuccess)
      return e;
    if (y1 > y0 &&
        (e = cudaMemcpyAsync(y_host + y0, dd.stage_y + y0, (size_t)(y1 - y0) * 8,
                             cudaMemcpyDeviceToHost, dd.copy_out)) != cudaSuccess)
      return e;
  }
  // (face_st's work ends before the last slab's chunks, which copy_out waited for)
  if ((e = cudaEventRecord(dd.ev_join, dd.copy_out)) != cudaSuccess) return e;
  return cudaStreamWaitEvent(origin, dd.ev_join, 0);
}

int sbm_fail_detail(int code, const std::string& msg) { return fail(code, msg); }
int sbm_cuda_fail_detail(cudaError_t e, const char* where) { return cuda_fail(e, where); }

}  // namespace sbm

using namespace sbm;

extern "C" {

const char* sbm_error_string(int status) {
  switch (status) {
    case SBM_OK: return "ok";
    case SBM_ERR_ARG: return "invalid argument";
    case SBM_ERR_OOM: return "out of memory";
    case SBM_ERR_CUDA: return "CUDA error";
    case SBM_ERR_EMPTY_DOMAIN: return "empty domain (no active cell)";
    case SBM_ERR_NOT_CONVERGED: return "not converged";
    case SBM_ERR_TIMEOUT: return "device wait timed out";
    case SBM_ERR_STATE: return "invalid state";
    case SBM_ERR_UNSUPPORTED: return "unsupported configuration";
    case SBM_ERR_GEOMETRY: return "closest-point projection failed";
  }
  return "unknown status";
}

const char* sbm_last_error_detail(void) { return g_detail.c_str(); }

// device < 0: the whole set-up on the host; otherwise the geometry stage on
// that GPU
static int create_problem(const sbm_desc* desc, int device, sbm_problem** out) {
  if (!out) return fail(SBM_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!desc) return fail(SBM_ERR_ARG, "desc is NULL");
  sbm_problem* P = new (std::nothrow) sbm_problem();
  if (!P) return fail(SBM_ERR_OOM, "host allocation failed");
  std::string err;
  int st;
  try {
    if (device < 0) {
      st = build_host_problem(*desc, &P->hp, &err);
    } else {
      st = setup_prepare(*desc, &P->hp, &err);
      if (st == SBM_OK) st = setup_geometry_device(&P->hp, device, &err);
      if (st == SBM_OK) st = setup_numbering_device(&P->hp, device, &err);
    }
  } catch (const std::bad_alloc&) {
    st = SBM_ERR_OOM;
    err = "host allocation failed";
  }
  if (st != SBM_OK) {
    delete P;
    return fail(st, err);
  }
  *out = P;
  return SBM_OK;
}

int sbm_create(const sbm_desc* desc, sbm_problem** out) { return create_problem(desc, -1, out); }

int sbm_create_gpu(const sbm_desc* desc, int device, sbm_problem** out) {
  if (device < 0) return fail(SBM_ERR_ARG, "device must be >= 0");
  return create_problem(desc, device, out);
}

int sbm_setup_face_data(sbm_problem* prob) {
  if (!prob) return fail(SBM_ERR_ARG, "prob is NULL");
  if (prob->on_device) return fail(SBM_ERR_STATE, "device data already set up");
  cudaError_t e = cudaGetDevice(&prob->device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  int st;
  try {
    st = build_device(prob->hp, &prob->dd);
  } catch (const std::bad_alloc&) {
    st = fail(SBM_ERR_OOM, "host allocation failed");
  }
  if (st == SBM_OK) prob->on_device = true;
  return st;
}

void sbm_destroy(sbm_problem* prob) {
  if (!prob) return;
  prob->prof.release();
  if (prob->on_device) free_device(&prob->dd);
  delete prob;
}

int sbm_sizes(const sbm_problem* prob, int64_t* n_dofs, int64_t* n_cells, int64_t* n_sfaces,
              int64_t* n_ifaces) {
  if (!prob) return fail(SBM_ERR_ARG, "prob is NULL");
  if (n_dofs) *n_dofs = prob->hp.n_dofs;
  if (n_cells) *n_cells = (int64_t)prob->hp.cell_bg.size();
  if (n_sfaces) *n_sfaces = (int64_t)prob->hp.sfaces.size() / 3;
  if (n_ifaces) *n_ifaces = prob->hp.desc.dg ? (int64_t)prob->hp.ifaces.size() / 3 : 0;
  return SBM_OK;
}

int sbm_export_geometry(const sbm_problem* prob, int32_t* cells, int32_t* sfaces, double* face_x) {
  if (!prob) return fail(SBM_ERR_ARG, "prob is NULL");
  const HostProblem& hp = prob->hp;
  if (cells) std::memcpy(cells, hp.cells.data(), hp.cells.size() * sizeof(int32_t));
  if (sfaces) std::memcpy(sfaces, hp.sfaces.data(), hp.sfaces.size() * sizeof(int32_t));
  if (face_x) std::memcpy(face_x, hp.face_x.data(), hp.face_x.size() * sizeof(double));
  return SBM_OK;
}

int sbm_apply_f64(sbm_problem* prob, const double* x, double* y, void* stream) {
  if (!prob || !x || !y) return fail(SBM_ERR_ARG, "NULL argument");
  if (x == y) return fail(SBM_ERR_ARG, "x and y must not overlap");
  if (!prob->on_device) return fail(SBM_ERR_STATE, "sbm_setup_face_data not called");
  cudaError_t e = prob->hp.desc.dg
      ? launch_dg_apply<double>(prob->hp, prob->dd, x, y, (cudaStream_t)stream, &prob->prof)
      : launch_cg_apply<double>(prob->hp, prob->dd, x, y, (cudaStream_t)stream, &prob->prof);
  if (e != cudaSuccess) return cuda_fail(e, "sbm_apply_f64");
  return SBM_OK;
}

int sbm_apply_f64_host(sbm_problem* prob, const double* x_host, double* y_host, void* stream) {
  if (!prob || !x_host || !y_host) return fail(SBM_ERR_ARG, "NULL argument");
  if (!prob->on_device) return fail(SBM_ERR_STATE, "sbm_setup_face_data not called");
  DeviceData& dd = prob->dd;
  const size_t bytes = (size_t)prob->hp.n_dofs * sizeof(double);
  cudaError_t e;
  if (!dd.stage_x) {
    if ((e = cudaMalloc((void**)&dd.stage_x, bytes)) != cudaSuccess) return cuda_fail(e, "stage");
    if ((e = cudaMalloc((void**)&dd.stage_y, bytes)) != cudaSuccess) return cuda_fail(e, "stage");
  }
  cudaStream_t st = (cudaStream_t)stream;
  if (dd.nslab > 1) {
    // page-locked buffers: the pipeline is captured once per buffer pair and
    // replayed (its copies need page-locked memory inside a graph)
    cudaPointerAttributes ax{}, ay{};
    const bool locked = cudaPointerGetAttributes(&ax, x_host) == cudaSuccess &&
                        cudaPointerGetAttributes(&ay, y_host) == cudaSuccess &&
                        ax.type == cudaMemoryTypeHost && ay.type == cudaMemoryTypeHost;
    cudaGetLastError();    // clear a pageable-pointer query's error state
    if (locked) {
      cudaGraphExec_t exec = nullptr;
      for (const auto& g : dd.host_graphs)
        if (g.x == x_host && g.y == y_host && g.variant == dd.variant[0]) exec = g.exec;
      if (!exec) {
        cudaGraph_t graph;
        if ((e = cudaStreamBeginCapture(dd.cap_st, cudaStreamCaptureModeThreadLocal)) !=
            cudaSuccess)
          return cuda_fail(e, "capture");
        const cudaError_t le = enqueue_host_pipeline(prob->hp, dd, x_host, y_host, dd.cap_st);
        e = cudaStreamEndCapture(dd.cap_st, &graph);
        if (le != cudaSuccess) return cuda_fail(le, "sbm_apply_f64_host");
        if (e != cudaSuccess) return cuda_fail(e, "capture end");
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return cuda_fail(e, "graph instantiate");
        if (dd.host_graphs.size() >= 4) {           // keep the most recent buffer pairs
          cudaGraphExecDestroy(dd.host_graphs.front().exec);
          dd.host_graphs.erase(dd.host_graphs.begin());
        }
        dd.host_graphs.push_back({x_host, y_host, dd.variant[0], exec});
      }
      if ((e = cudaGraphLaunch(exec, st)) != cudaSuccess) return cuda_fail(e, "graph launch");
    } else if ((e = enqueue_host_pipeline(prob->hp, dd, x_host, y_host, st)) != cudaSuccess) {
      return cuda_fail(e, "sbm_apply_f64_host");
    }
  } else {
    if ((e = cudaMemcpyAsync(dd.stage_x, x_host, bytes, cudaMemcpyHostToDevice, st)) !=
        cudaSuccess)
      return cuda_fail(e, "H2D");
    int s = sbm_apply_f64(prob, dd.stage_x, dd.stage_y, stream);
    if (s != SBM_OK) return s;
    if ((e = cudaMemcpyAsync(y_host, dd.stage_y, bytes, cudaMemcpyDeviceToHost, st)) !=
        cudaSuccess)
      return cuda_fail(e, "D2H");
  }
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(e, "sync");
  return SBM_OK;
}

int sbm_diagonal(sbm_problem* prob, double* diag, void* stream) {
  if (!prob || !diag) return fail(SBM_ERR_ARG, "NULL argument");
  if (!prob->on_device) return fail(SBM_ERR_STATE, "sbm_setup_face_data not called");
  cudaError_t e = launch_diag_f64(prob->hp, prob->dd, diag, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "sbm_diagonal");
  return SBM_OK;
}

static int check_face_mode(const sbm_problem* prob, int face_mode) {
  if (face_mode != SBM_FACE_FP32 && face_mode != SBM_FACE_TF32 && face_mode != SBM_FACE_BF16)
    return fail(SBM_ERR_ARG, "unknown face mode");
  if (face_mode != SBM_FACE_FP32 && prob->hp.d != 3)
    return fail(SBM_ERR_UNSUPPORTED, "tensor-core face modes are built for 3D problems");
  if (face_mode != SBM_FACE_FP32 && prob->hp.desc.extension != SBM_EXT_EXACT)
    return fail(SBM_ERR_UNSUPPORTED,
                "tensor-core face modes evaluate the exact extension's point evaluation");
  return SBM_OK;
}

int sbm_apply_f32(sbm_problem* prob, const float* x, float* y, int face_mode, void* stream) {
  if (!prob || !x || !y) return fail(SBM_ERR_ARG, "NULL argument");
  if (x == y) return fail(SBM_ERR_ARG, "x and y must not overlap");
  if (!prob->on_device) return fail(SBM_ERR_STATE, "sbm_setup_face_data not called");
  const int fm = check_face_mode(prob, face_mode);
  if (fm != SBM_OK) return fm;
  cudaError_t e = prob->hp.desc.dg
      ? launch_dg_apply<float>(prob->hp, prob->dd, x, y, (cudaStream_t)stream, &prob->prof,
                               face_mode)
      : launch_cg_apply<float>(prob->hp, prob->dd, x, y, (cudaStream_t)stream, &prob->prof,
                               face_mode);
  if (e != cudaSuccess) return cuda_fail(e, "sbm_apply_f32");
  return SBM_OK;
}

static ApplyFn<double> apply64_fn(sbm_problem* prob) {
  return [prob](const double* x, double* y, cudaStream_t st) {
    return prob->hp.desc.dg ? launch_dg_apply<double>(prob->hp, prob->dd, x, y, st, nullptr)
                            : launch_cg_apply<double>(prob->hp, prob->dd, x, y, st, nullptr);
  };
}

static ApplyFn<float> apply32_fn(sbm_problem* prob, int face_mode = SBM_FACE_FP32) {
  return [prob, face_mode](const float* x, float* y, cudaStream_t st) {
    return prob->hp.desc.dg
               ? launch_dg_apply<float>(prob->hp, prob->dd, x, y, st, nullptr, face_mode)
               : launch_cg_apply<float>(prob->hp, prob->dd, x, y, st, nullptr, face_mode);
  };
}

static int solve_result(SolveStatus s, const SolveInfo& info, int* iters, double* relres,
                        const char* what) {
  if (iters) *iters = info.iters;
  if (relres) *relres = info.relres;
  if (s.status == SBM_ERR_CUDA) return cuda_fail(s.cuda, what);
  if (s.status == SBM_ERR_NOT_CONVERGED)
    return fail(SBM_ERR_NOT_CONVERGED, std::string(what) + ": relative residual " +
                                           std::to_string(info.relres) + " after " +
                                           std::to_string(info.iters) + " iterations");
  return s.status;
}

int sbm_cg(sbm_problem* prob, const double* b, double* x, double rtol, int maxit, int precond,
           int* iters, double* relres, void* stream) {
  if (!prob || !b || !x || b == x) return fail(SBM_ERR_ARG, "bad vector argument");
  if (!prob->on_device) return fail(SBM_ERR_STATE, "sbm_setup_face_data not called");
  if (!(rtol > 0) || maxit < 1 || (precond != SBM_PRECOND_NONE && precond != SBM_PRECOND_JACOBI))
    return fail(SBM_ERR_ARG, "bad solver parameter");
  cudaStream_t st = (cudaStream_t)stream;
  Workspace ws;
  double* diag = nullptr;
  SolveInfo info;
  SolveStatus s{SBM_OK, cudaSuccess};
  if (precond == SBM_PRECOND_JACOBI) {
    cudaError_t e = ws.alloc((void**)&diag, prob->hp.n_dofs * sizeof(double));
    if (e == cudaSuccess) e = launch_diag_f64(prob->hp, prob->dd, diag, st);
    if (e != cudaSuccess) s = {SBM_ERR_CUDA, e};
  }
  if (s.status == SBM_OK)
    s = solve_cg(apply64_fn(prob), prob->hp.n_dofs, b, x, diag, rtol, maxit, st, ws, &info);
  cudaStreamSynchronize(st);
  ws.release();
  return solve_result(s, info, iters, relres, "sbm_cg");
}

int sbm_gmres(sbm_problem* prob, const double* b, double* x, double rtol, int maxit, int restart,
              int* iters, double* relres, void* stream) {
  if (!prob || !b || !x || b == x) return fail(SBM_ERR_ARG, "bad vector argument");
  if (!prob->on_device) return fail(SBM_ERR_STATE, "sbm_setup_face_data not called");
  if (!(rtol > 0) || maxit < 1 || restart < 1 || restart > 1000)
    return fail(SBM_ERR_ARG, "bad solver parameter");
  cudaStream_t st = (cudaStream_t)stream;
  Workspace ws;
  SolveInfo info;
  ApplyFn<double> ap = apply64_fn(prob);
  SolveStatus s = solve_gmres<double, double>(ap, prob->hp.n_dofs, b, x, rtol, maxit, restart, st,
                                              ws, &info, &ap);
  cudaStreamSynchronize(st);
  ws.release();
  return solve_result(s, info, iters, relres, "sbm_gmres");
}

extern "C++" template <typename T>
int run_bicgstab(sbm_problem* prob, const ApplyFn<T>& ap, const T* b, T* x, double rtol,
                        int maxit, int* iters, double* relres, cudaStream_t st,
                        const char* what) {
  Workspace ws;
  SolveInfo info;
  Bicgstab<T> bi;
  SolveStatus s{SBM_OK, cudaSuccess};
  cudaError_t e = bi.setup(ap, prob->hp.n_dofs, b, x, ws);
  if (e != cudaSuccess) s = {SBM_ERR_CUDA, e};
  else s = bi.solve(false, rtol, maxit, st, &info);
  cudaStreamSynchronize(st);
  bi.destroy();
  ws.release();
  return solve_result(s, info, iters, relres, what);
}

int sbm_bicgstab(sbm_problem* prob, const double* b, double* x, double rtol, int maxit,
                 int* iters, double* relres, void* stream) {
  if (!prob || !b || !x || b == x) return fail(SBM_ERR_ARG, "bad vector argument");
  if (!prob->on_device) return fail(SBM_ERR_STATE, "sbm_setup_face_data not called");
  if (!(rtol > 0) || maxit < 1) return fail(SBM_ERR_ARG, "bad solver parameter");
  return run_bicgstab<double>(prob, apply64_fn(prob), b, x, rtol, maxit, iters, relres,
                              (cudaStream_t)stream, "sbm_bicgstab");
}

int sbm_bicgstab_f32(sbm_problem* prob, const float* b, float* x, double rtol, int maxit,
                     int face_mode, int* iters, double* relres, void* stream) {
  if (!prob || !b || !x || b == x) return fail(SBM_ERR_ARG, "bad vector argument");
  if (!prob->on_device) return fail(SBM_ERR_STATE, "sbm_setup_face_data not called");
  if (!(rtol > 0) || maxit < 1) return fail(SBM_ERR_ARG, "bad solver parameter");
  const int fm = check_face_mode(prob, face_mode);
  if (fm != SBM_OK) return fm;
  return run_bicgstab<float>(prob, apply32_fn(prob, face_mode), b, x, rtol, maxit, iters, relres, (cudaStream_t)stream, "sbm_bicgstab_f32");
}

int sbm_solve_ir(sbm_problem* prob, const double* b, double* x, double rtol, int max_outer,
                 int restart, double inner_rtol, int inner_maxit, int face_mode,
                 int inner_solver, int* iters, int* outer, double* relres, void* stream) {
  if (!prob || !b || !x || b == x) return fail(SBM_ERR_ARG, "bad vector argument");
  if (!prob->on_device) return fail(SBM_ERR_STATE, "sbm_setup_face_data not called");
  if (!(rtol > 0) || max_outer < 0 || restart < 1 || restart > 1000 || !(inner_rtol > 0) ||
      inner_maxit < 1 || (inner_solver != SBM_INNER_GMRES && inner_solver != SBM_INNER_BICGSTAB &&
                          inner_solver != SBM_INNER_BICGSTAB_MIXED))
    return fail(SBM_ERR_ARG, "bad solver parameter");
  const int fm = check_face_mode(prob, face_mode);
  if (fm != SBM_OK) return fm;
  cudaStream_t st = (cudaStream_t)stream;
  Workspace ws;
  SolveInfo info;
  SolveStatus s = solve_ir(apply64_fn(prob), apply32_fn(prob, face_mode), prob->hp.n_dofs, b, x, rtol,
                           max_outer, restart, inner_rtol, inner_maxit, inner_solver, st, ws,
                           &info);
  cudaStreamSynchronize(st);
  ws.release();
  if (outer) *outer = info.restarts;
  return solve_result(s, info, iters, relres, "sbm_solve_ir");
}

int sbm_bicgstab_mixed(sbm_problem* prob, const double* b, double* x, double rtol, int maxit,
                       int face_mode, int* iters, int* replacements, double* relres,
                       void* stream) {
  if (!prob || !b || !x || b == x) return fail(SBM_ERR_ARG, "bad vector argument");
  if (!prob->on_device) return fail(SBM_ERR_STATE, "sbm_setup_face_data not called");
  if (!(rtol > 0) || maxit < 1) return fail(SBM_ERR_ARG, "bad solver parameter");
  const int fm = check_face_mode(prob, face_mode);
  if (fm != SBM_OK) return fm;
  cudaStream_t st = (cudaStream_t)stream;
  Workspace ws;
  SolveInfo info;
  SolveStatus s = solve_bicgstab_reliable(apply64_fn(prob), apply32_fn(prob, face_mode),
                                          prob->hp.n_dofs, b, x, rtol, maxit, st, ws, &info,
                                          replacements);
  cudaStreamSynchronize(st);
  ws.release();
  return solve_result(s, info, iters, relres, "sbm_bicgstab_mixed");
}

int sbm_rhs(const sbm_problem* prob, int manufactured, double* b_host) {
  if (!prob || !b_host) return fail(SBM_ERR_ARG, "NULL argument");
  if (!manufactured_ok(manufactured, prob->hp.d)) return fail(SBM_ERR_ARG, "unknown solution id");
  build_rhs(prob->hp, manufactured, b_host);
  return SBM_OK;
}

int sbm_rhs_device(const sbm_problem* prob, int manufactured, double* b, void* stream) {
  if (!prob || !b) return fail(SBM_ERR_ARG, "NULL argument");
  if (!manufactured_ok(manufactured, prob->hp.d)) return fail(SBM_ERR_ARG, "unknown solution id");
  if (!prob->on_device) return fail(SBM_ERR_STATE, "sbm_setup_face_data not called");
  std::vector<double> h((size_t)prob->hp.n_dofs);
  build_rhs(prob->hp, manufactured, h.data());
  // from pageable memory the call returns once h is staged for the copy
  cudaError_t e = cudaMemcpyAsync(b, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice,
                                  (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "sbm_rhs_device copy");
  return SBM_OK;
}

int sbm_interpolate(const sbm_problem* prob, int manufactured, double* u_host) {
  if (!prob || !u_host) return fail(SBM_ERR_ARG, "NULL argument");
  if (!manufactured_ok(manufactured, prob->hp.d)) return fail(SBM_ERR_ARG, "unknown solution id");
  build_interpolant(prob->hp, manufactured, u_host);
  return SBM_OK;
}

int sbm_device_status(sbm_problem* prob) {
  if (!prob) return fail(SBM_ERR_ARG, "prob is NULL");
  if (!prob->on_device) return SBM_OK;
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceSynchronize");
  int v = 0;
  if ((e = cudaMemcpy(&v, prob->dd.err_flag, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess)
    return cuda_fail(e, "read device error word");
  if (v != 0) {
    cudaMemset(prob->dd.err_flag, 0, sizeof(int));
    return fail(v, "a bounded device-side wait expired");
  }
  return SBM_OK;
}

// time every tile shape of the single apply (2 where available), in FP64
// and FP32, on the problem itself, and keep the faster of each
int sbm_autotune(sbm_problem* prob, int* shape64, int* shape32) {
  if (!prob) return fail(SBM_ERR_ARG, "prob is NULL");
  if (!prob->on_device) return fail(SBM_ERR_STATE, "sbm_setup_face_data not called");
  if (prob->hp.desc.dg) {
    if (shape64) *shape64 = 0;
    if (shape32) *shape32 = 0;
    return SBM_OK;
  }
  const size_t n = (size_t)prob->hp.n_dofs;
  void *x = nullptr, *y = nullptr;
  cudaError_t e = cudaMalloc(&x, n * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&y, n * sizeof(double));
  if (e == cudaSuccess) e = cudaMemset(x, 0, n * sizeof(double));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  for (int prec = 0; prec < 2 && e == cudaSuccess; ++prec) {
    float best = 1e30f;
    int bestv = 0;
    bool besto = false;
    for (int vo = 0; vo < 8 && e == cudaSuccess; ++vo) {
      const int v = vo / 2;
      const bool o = vo % 2;
      if ((v == 2 && !cell_reg_available(prob->hp, prec == 1)) || (v == 3 && prob->hp.d != 3) ||
          (o && (v == 1 || v == 2 || !prob->dd.chunks[0].ordered)))
        continue;
      prob->dd.variant[prec] = v;
      prob->dd.ordered[prec] = o;
      float tot = 0.f;
      for (int rep = 0; rep < 6 && e == cudaSuccess; ++rep) {
        cudaEventRecord(e0, 0);
        e = prec == 0 ? launch_cg_apply<double>(prob->hp, prob->dd, (const double*)x, (double*)y,
                                                0, nullptr)
                      : launch_cg_apply<float>(prob->hp, prob->dd, (const float*)x, (float*)y, 0,
                                               nullptr);
        cudaEventRecord(e1, 0);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep >= 2) tot += ms;
      }
      // colour-ordered stores only when at least 2 % faster: closer timings
      // are within the run-to-run spread, and the colour buffers keep the
      // cell kernel free of the ordering waits
      if (o) tot *= 1.02f;
      if (tot < best) {
        best = tot;
        bestv = v;
        besto = o;
      }
    }
    prob->dd.variant[prec] = bestv;
    prob->dd.ordered[prec] = besto;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(x);
  cudaFree(y);
  if (e != cudaSuccess) return cuda_fail(e, "sbm_autotune");
  if (shape64) *shape64 = prob->dd.variant[0];
  if (shape32) *shape32 = prob->dd.variant[1];
  return SBM_OK;
}

int sbm_set_tile_shape(sbm_problem* prob, int shape64, int shape32) {
  if (!prob) return fail(SBM_ERR_ARG, "prob is NULL");
  if (!prob->on_device) return fail(SBM_ERR_STATE, "sbm_setup_face_data not called");
  if (shape64 < -1 || shape64 > 3 || shape32 < -1 || shape32 > 3)
    return fail(SBM_ERR_ARG, "tile shape must be -1, 0, 1, 2 or 3");
  if (prob->hp.d != 3 && (shape64 == 3 || shape32 == 3))
    return fail(SBM_ERR_UNSUPPORTED, "tile shape 3 is for 3D problems");
  if (prob->hp.desc.dg && (shape64 >= 1 || shape32 >= 1))
    return fail(SBM_ERR_UNSUPPORTED, "DG applies have one tile shape");
  if ((shape64 == 2 && !cell_reg_available(prob->hp, false)) ||
      (shape32 == 2 && !cell_reg_available(prob->hp, true)))
    return fail(SBM_ERR_UNSUPPORTED,
                "tile shape 2 needs a 3D problem with p <= 4 (FP32) or p <= 3 (FP64)");
  if (shape64 >= 0) prob->dd.variant[0] = shape64;
  if (shape32 >= 0) prob->dd.variant[1] = shape32;
  return SBM_OK;
}

int sbm_set_ordered_stores(sbm_problem* prob, int ordered64, int ordered32) {
  if (!prob) return fail(SBM_ERR_ARG, "prob is NULL");
  if (!prob->on_device) return fail(SBM_ERR_STATE, "sbm_setup_face_data not called");
  if (ordered64 < -1 || ordered64 > 1 || ordered32 < -1 || ordered32 > 1)
    return fail(SBM_ERR_ARG, "ordered must be -1, 0 or 1");
  if ((ordered64 == 1 || ordered32 == 1) && !prob->dd.chunks[0].ordered)
    return fail(SBM_ERR_UNSUPPORTED,
                "no colour-ordered stores for this problem (DG, or a chunk with more "
                "lower-colour neighbours than the dependency table holds)");
  if (ordered64 >= 0) prob->dd.ordered[0] = ordered64 == 1;
  if (ordered32 >= 0) prob->dd.ordered[1] = ordered32 == 1;
  return SBM_OK;
}

int sbm_ordered_stores(const sbm_problem* prob, int* ordered64, int* ordered32) {
  if (!prob) return fail(SBM_ERR_ARG, "prob is NULL");
  if (ordered64) *ordered64 = prob->dd.ordered[0] ? 1 : 0;
  if (ordered32) *ordered32 = prob->dd.ordered[1] ? 1 : 0;
  return SBM_OK;
}

int sbm_selftest_timeout(sbm_problem* prob, void* stream) {
  if (!prob) return fail(SBM_ERR_ARG, "prob is NULL");
  if (!prob->on_device) return fail(SBM_ERR_STATE, "sbm_setup_face_data not called");
  cudaError_t e = launch_timeout_selftest(prob->dd.err_flag, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "sbm_selftest_timeout");
  return SBM_OK;
}

int sbm_profile_enable(sbm_problem* prob, int on) {
  if (!prob) return fail(SBM_ERR_ARG, "prob is NULL");
  prob->prof.on = (on != 0);
  return SBM_OK;
}

int sbm_profile_read(sbm_problem* prob, double* phase_ms, int64_t* launches) {
  if (!prob) return fail(SBM_ERR_ARG, "prob is NULL");
  Profiler& pf = prob->prof;
  double tot[3] = {0.0, 0.0, 0.0};
  for (size_t g = 0; g + Profiler::kMarks <= pf.used; g += Profiler::kMarks) {
    cudaError_t e = cudaEventSynchronize(pf.ev[g + Profiler::kMarks - 1]);
    if (e != cudaSuccess) return cuda_fail(e, "cudaEventSynchronize");
    for (int k = 0; k < 3; ++k) {
      float ms = 0.f;
      e = cudaEventElapsedTime(&ms, pf.ev[g + k], pf.ev[g + k + 1]);
      if (e != cudaSuccess) return cuda_fail(e, "cudaEventElapsedTime");
      tot[k] += ms;
    }
  }
  if (phase_ms)
    for (int k = 0; k < 3; ++k) phase_ms[k] = tot[k];
  if (launches) *launches = pf.launches;
  pf.used = 0;
  pf.launches = 0;
  return SBM_OK;
}

}  // extern "C"
