// Internal definitions shared by the C ABI and the kernel launchers.
#pragma once

#include <cuda_runtime.h>

#include <type_traits>

#include <cstdint>
#include <string>
#include <vector>

#include "setup.hpp"

namespace sbm {

// 1D operator tables handed to kernels by value (kernel parameter space is a
// constant bank: every FMA with a table operand reads it for free).
constexpr int kMaxH = (kMaxN + 1) / 2;

// A centrosymmetric n x n matrix (A[i][j] = A[n-1-i][n-1-j]) split into its
// even and odd parts: with e_j = v_j + v_{n-1-j}, o_j = v_j - v_{n-1-j} (and
// e_mid = v_mid for odd n), s_i = sum_j E[i][j] e_j, d_i = sum_j O[i][j] o_j,
// the product is y_i = s_i + d_i, y_{n-1-i} = s_i - d_i (y_mid = s_mid), where
// E[i][j] = (A[i][j] + A[i][n-1-j]) / 2, E[i][mid] = A[i][mid] and
// O[i][j] = (A[i][j] - A[i][n-1-j]) / 2.
template <typename T>
struct Folded {
  T E[kMaxH][kMaxH];
  T O[kMaxH][kMaxH];
};

template <typename T>
struct KTab {
  T M[kMaxN][kMaxN];     // 1D mass on [0,1]
  T K[kMaxN][kMaxN];     // 1D stiffness on [0,1]
  T Mh[kMaxN][kMaxN];    // h^(d-2) * M   (last sweep of the cell operator)
  T Kh[kMaxN][kMaxN];    // h^(d-2) * K
  T S[kMaxN][kMaxN];     // S[q][j] = phi_j(g_q)
  T Dg[kMaxN][kMaxN];    // Dg[q][j] = phi_j'(g_q)
  T D0[kMaxN];           // phi_j'(0)
  T D1[kMaxN];           // phi_j'(1)
  T W[kMaxN * kMaxN];    // face weights h^(d-1) w_qa w_qb (tangential Gauss index q)
  T h_inv;
  T hface;               // h^(d-1), the face Jacobian
  T sigma;
  Folded<T> fM, fK, fMh, fKh;  // even/odd parts of M, K, Mh, Kh (GLL nodes are symmetric)
  // eigenbasis of the pencil (K, M) (M = V V^T, K = V diag(lam) V^T; even
  // modes first): fVt maps a folded nodal line to its modes, fV modes back
  // to a line; hlam = h^(d-2) lam
  Folded<T> fVt, fV;
  T hlam[kMaxN];
};

template <typename T>
KTab<T> make_ktab(const HostProblem& hp);

constexpr int kMaxSlabs = 16;   // slabs of the pipelined host-buffer apply, at most
// Their cumulative shares of the cells: small first and last slabs (the copy
// of x before the first kernel, the copy of y after the last one), large
// ones between (full launches).
constexpr double kSlabCuts[] = {0.04, 0.16, 0.40, 0.64, 0.84, 0.96};

// CG chunking: runs of up to R consecutive active cells of one x-row.
struct ChunkTable {
  int n = 0;
  int32_t* first = nullptr;      // [n + 1] first ordered cell of each chunk
  uint8_t* colour = nullptr;     // [n] colour of each chunk
  uint32_t* run_bits = nullptr;  // [n][bit_words]: bit l*S + kk of chunk ch set if element kk
  int bit_words = 0;             //   of its run l is a DoF that several colours touch
  int32_t* multi = nullptr;      // [nmulti] DoFs touched by two colours or more, grouped by
                                 //   colour count (2, 3-4, 5-8), ascending within a group
  uint8_t* multi_mask = nullptr; // [nmulti] their colour masks
  int64_t nmulti = 0;
  // colour-ordered stores (chunking of tile shape 0; ordered == false where
  // not built): chunks by ascending colour (ticket -> chunk), per chunk the
  // run bits of the DoFs a lower colour also touches (read-add-write), the
  // chunks of lower colours it shares a DoF with ([n][dep_cap], ndeps of
  // them), per-chunk completion counts and the ticket / exit counters
  bool ordered = false;
  int dep_cap = 0;
  int32_t* ord = nullptr;
  uint32_t* add_bits = nullptr;
  int32_t* deps = nullptr;
  int32_t* ndeps = nullptr;
  int32_t* done = nullptr;
  uint32_t* tickets = nullptr;   // [2]
  // slabs of the pipelined host-buffer apply: chunks [slab_chunk[s],
  // slab_chunk[s+1]), shared DoFs multi[slab_multi[s], slab_multi[s+1])
  std::vector<int> slab_chunk;
  std::vector<int64_t> slab_multi;
};

// Device-built set-up tables (setup_gpu.cu).  For one chunking: the colour set
// of every DoF (from the chunk-ordered line table `lines` on the device), the
// list of DoFs several colours share and the per-chunk run bits, into ct.
// The shared DoFs are listed slab by slab (slab s: DoFs [ycut[s], ycut[s+1]);
// ct->slab_multi receives the offsets), then by colour count.  ordered:
// also the tables of the colour-ordered stores (ct->ordered stays false if a
// chunk has more lower-colour neighbours than the dependency table holds).
cudaError_t device_chunk_tables(const int32_t* lines, int64_t nc, int L, int n, int64_t n_dofs,
                                const std::vector<int32_t>& ch_first,
                                const std::vector<uint8_t>& ch_col, int R,
                                const int32_t* first_dev, const std::vector<int64_t>& ycut,
                                ChunkTable* ct, bool ordered);

// The 1D Lagrange values at every shifted surrogate point (exact extension) or
// the shift vectors (first-order Taylor), in kernel face order (fsrc[k] = the
// face index of kernel face k), FP64 and FP32, allocated here.
cudaError_t device_face_phi(const HostProblem& hp, const std::vector<int64_t>& fsrc,
                            double** phi, float** phi32);
// 3D exact extension: the per-point products of the two non-first axes'
// values from the FP64 table phi ([F][Q][3][n]) into pp ([F][n^2][Q]),
// allocated here.
cudaError_t device_face_pp(int64_t F, int L, int n, const double* phi, double** pp);

// Device-resident set-up data of one problem.
struct DeviceData {
  // cells in kernel order: for each colour (CG) -- interior cells, then cells
  // that own surrogate faces; DG uses one "colour" with the same split.
  int ncolours = 0;
  std::vector<int> col_start;    // [ncolours + 1] offsets into the ordered cell list
  std::vector<int> col_nint;     // [ncolours] interior cells in each colour
  std::vector<int32_t> order;    // ordered position -> active-cell rank
  int32_t* lines = nullptr;      // CG [Nc * L]: global index of node (0, line) per x-line
  int32_t* cell_rank = nullptr;  // [Nc] ordered position -> active-cell rank (DG base)
  int32_t* face_start = nullptr; // [Nc + 1] per ordered cell, range into the ordered face list
  int32_t* face_kind = nullptr;  // [F] k | (s << 2)
  int32_t* face_cell = nullptr;  // [F] ordered cell position of the face's cell
  int nface = 0;
  double* face_out = nullptr;    // [F * 2L] per-face results of the face kernel (scratch)
  float* face_out32 = nullptr;
  int* err_flag = nullptr;       // device error word (SBM_ERR_TIMEOUT from bounded waits)
  ChunkTable chunks[2];          // CG: R and R/2 cells per chunk (two tile shapes)
  int variant[2] = {0, 0};       // tile shape of the single applies: [FP64, FP32]
  bool ordered[2] = {false, false};  // colour-ordered stores instead of the assembly
  // tile shape 2 (3D CG, n <= 5; cell_reg.cu): one thread per cell on the
  // chunks of shape 0 -- chunk of every ordered cell, blocks of whole
  // chunks, per-cell bits of the nodes several colours share
  int32_t* reg_cell_chunk = nullptr;
  int32_t* reg_block_first = nullptr;
  uint32_t* reg_mask = nullptr;
  int reg_nblocks = 0;
  int32_t* diag_pos = nullptr;   // CG: ordered positions grouped by cell parity (diagonal)
  std::vector<int> diag_col_start;
  double* ycol = nullptr;        // CG [ncolours * n_dofs] colour accumulation buffers (scratch)
  float* ycol32 = nullptr;
  // per surrogate-face point: exact extension: [F * Q * d * n] phi_j(xi_{q,l})
  // at the shifted point; first-order Taylor: [F * Q * d] the shift d_q
  double* face_phi = nullptr;
  float* face_phi32 = nullptr;   // the same table rounded to FP32
  // 3D exact extension (FP64 face kernel): [F][n^2][Q] the products
  // phi_j1(xi_{q,1}) phi_j2(xi_{q,2}) of the two non-first axes, index
  // j1 + n j2 (point index fastest)
  double* face_pp = nullptr;
  int32_t* nbr = nullptr;        // DG [Nc * 2d] neighbour rank per (k, s), -1 = surrogate
  double* stage_x = nullptr;     // host-apply staging buffers (allocated on first use)
  double* stage_y = nullptr;
  // CG: the pipelined host-buffer apply cuts the cells into nslab slabs of
  // whole cell layers along the last axis (the DoF numbering's slowest);
  // slab s has the faces [slab_face[s], slab_face[s+1]), needs x on the DoFs
  // [0, slab_x[s]) and makes y final on [slab_y[s], slab_y[s+1]).  Its copies
  // run on copy_in / copy_out, its face kernel on face_st (beside the
  // previous slab's cells), ordered by ev_in[s], ev_face[s], ev_done[s].
  int nslab = 0;
  std::vector<int> slab_face;
  std::vector<int64_t> slab_x, slab_y;
  cudaStream_t copy_in = nullptr, copy_out = nullptr, face_st = nullptr;
  std::vector<cudaEvent_t> ev_in, ev_face, ev_done;
  // the pipeline captured per page-locked (x, y) buffer pair and FP64 tile
  // shape (at most 4 kept), and the stream it is captured on
  struct HostGraph {
    const void* x;
    const void* y;
    int variant;
    cudaGraphExec_t exec;
  };
  std::vector<HostGraph> host_graphs;
  cudaStream_t cap_st = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
};

// Optional kernel timing: CUDA events on the apply's stream at the phase
// boundaries of every apply (start | face kernel | cell kernel | assembly),
// read back by sbm_profile_read.
struct Profiler {
  static constexpr int kMarks = 4;
  bool on = false;
  std::vector<cudaEvent_t> ev;   // groups of kMarks events
  size_t used = 0;               // events recorded since the last read
  int64_t launches = 0;          // operator kernel launches since the last read
  cudaError_t mark(cudaStream_t st);   // record the next boundary
  void count(int nlaunch) { launches += nlaunch; }
  void release();
};

struct CellLaunch {
  int d, n;
  int cpb;          // cells per block on interior tiles
  int threads;      // block size
};
CellLaunch cell_launch_shape(int d, int n);
int chunk_cells(int d, int n);    // R: cells per chunk of the CG chunk kernel

// Record an error detail for sbm_last_error_detail() and return the code.
int sbm_fail_detail(int code, const std::string& msg);
int sbm_cuda_fail_detail(cudaError_t e, const char* where);

template <typename T> inline T* ycol_of(const DeviceData& dd);
template <> inline double* ycol_of<double>(const DeviceData& dd) { return dd.ycol; }
template <> inline float* ycol_of<float>(const DeviceData& dd) { return dd.ycol32; }

template <typename T> inline T* face_out_of(const DeviceData& dd);
template <> inline double* face_out_of<double>(const DeviceData& dd) { return dd.face_out; }
template <> inline float* face_out_of<float>(const DeviceData& dd) { return dd.face_out32; }

// Launch kern<<<grid, block, smem, st>>>(args...), with programmatic
// stream serialization when pdl (the kernel may start before the previous
// kernel of the stream completes; it waits with griddepcontrol.wait before
// it reads that kernel's results).
template <typename... KArgs, typename... Args>
cudaError_t launch_maybe_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem,
                             cudaStream_t st, bool pdl, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = pdl ? at : nullptr;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kern, args...);
}

// Tile shape 2: the cell term with one thread per cell and the tile in
// registers (cell_reg.cu); available for 3D CG problems with n <= 5 (FP32)
// or n <= 4 (FP64); bitwise equal to tile shape 0.
bool cell_reg_available(const HostProblem& hp, bool fp32);
cudaError_t build_cell_reg_tables(const HostProblem& hp, const std::vector<int32_t>& ch_first,
                                  DeviceData* dd);
template <typename T>
cudaError_t launch_cell_reg(const HostProblem& hp, const DeviceData& dd, const T* x, T* y,
                            const T* fo, T* ycol, cudaStream_t st, bool pdl = false);

// The surrogate faces [fb, fe) of the kernel face order (all: 0, -1) into
// the per-face scratch (face_kernel.cu).
template <typename T>
cudaError_t launch_face_kernel(const HostProblem& hp, const DeviceData& dd, const T* x, T* out,
                               cudaStream_t st, int fb = 0, int fe = -1);
template <typename T> inline const T* face_phi_of(const DeviceData& dd);
template <> inline const double* face_phi_of<double>(const DeviceData& dd) { return dd.face_phi; }
template <> inline const float* face_phi_of<float>(const DeviceData& dd) { return dd.face_phi32; }
template <typename T> inline const T* face_pp_of(const DeviceData& dd);
template <> inline const double* face_pp_of<double>(const DeviceData& dd) { return dd.face_pp; }
template <> inline const float* face_pp_of<float>(const DeviceData&) { return nullptr; }

// Surrogate faces on the tensor cores (3D, FP32 apply): face_mode
// SBM_FACE_TF32 or SBM_FACE_BF16; same output as launch_face_kernel.
cudaError_t launch_tc_face_kernel(const HostProblem& hp, const DeviceData& dd, const float* x,
                                  float* out, int face_mode, cudaStream_t st);
// One bounded mbarrier wait that expires (diagnostic of the timeout path).
cudaError_t launch_timeout_selftest(int* err, cudaStream_t st);

// Apply, CG: face kernel, cell kernel, assembly; T = double or float
// (face_mode applies to float: SBM_FACE_FP32 / TF32 / BF16).
template <typename T>
cudaError_t launch_cg_apply(const HostProblem& hp, const DeviceData& dd, const T* x, T* y,
                            cudaStream_t st, Profiler* prof, int face_mode = 0);
// Apply, CG, with caller-provided scratch (per-face results [F][2L] and the
// colour buffers [ncolours][n_dofs]) instead of the problem's own; variant =
// cell-kernel tile shape (0 or 1).
template <typename T>
cudaError_t launch_cg_apply_scratch(const HostProblem& hp, const DeviceData& dd, const T* x, T* y,
                                    T* face_scratch, T* colour_scratch, int variant,
                                    cudaStream_t st);
// Apply, DG: one launch.
template <typename T>
cudaError_t launch_dg_apply(const HostProblem& hp, const DeviceData& dd, const T* x, T* y,
                            cudaStream_t st, Profiler* prof, int face_mode = 0);

// the face stage of an apply: CUDA-core kernel, or the tensor-core kernel for
// an FP32 apply in TF32 / BF16 face mode
template <typename T>
inline cudaError_t launch_faces(const HostProblem& hp, const DeviceData& dd, const T* x, T* out,
                                int face_mode, cudaStream_t st) {
  if constexpr (std::is_same<T, float>::value) {
    if (face_mode != 0) return launch_tc_face_kernel(hp, dd, x, out, face_mode, st);
  }
  return launch_face_kernel<T>(hp, dd, x, out, st);
}
// The slab pipeline of the host-buffer apply on the problem's streams,
// forked from and joined back to origin (api.cu).
cudaError_t enqueue_host_pipeline(const HostProblem& hp, const DeviceData& dd, const double* x_host,
                                  double* y_host, cudaStream_t origin);

// Slab s of the CG FP64 apply on the problem's own scratch (cg_apply.cu):
// stages 1 = its surrogate faces, 2 = its cells and the assembly it completes.
cudaError_t launch_cg_apply_slab(const HostProblem& hp, const DeviceData& dd, const double* x,
                                 double* y, int slab, int stages, cudaStream_t st);
// FP64 diagonal.
cudaError_t launch_diag_f64(const HostProblem& hp, const DeviceData& dd, double* diag,
                            cudaStream_t st);

}  // namespace sbm

struct sbm_problem {
  sbm::HostProblem hp;
  sbm::DeviceData dd;
  int device = 0;
  bool on_device = false;   // sbm_setup_face_data done
  sbm::Profiler prof;
};
