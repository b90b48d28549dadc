// Diagonal of the SBM operator (FP64), for Jacobi scaling.
//
// diag_i = sum over cells K containing i of A_K[i,i] + sum over surrogate faces
// F of K of A_F[i,i], with (tensor-product closed form of the cell term)
//   A_K[j,j] = h^(d-2) sum_k prod_l (l == k ? K[j_l][j_l] : M[j_l][j_l])
// and, per face point q (same integrand as the apply, Algorithm 3),
//   A_F[j,j] = sum_q W_q [ -psi_j(x~_q) dn psi_j(x~_q) - dn psi_j(x~_q) E psi_j
//                          + sigma psi_j(x~_q) E psi_j ],
// E psi_j = psi_j(x_q) (exact extension) or psi_j(x~_q) + d_q . grad psi_j(x~_q)
// (first-order Taylor).
// CG: one launch per cell colour, plain read-modify-write (no atomics).
// DG: one launch over all cells, plus the interior-face blocks' diagonals.
#include "internal.hpp"

namespace sbm {

struct DiagArgs {
  double* __restrict__ diag;
  const int32_t* __restrict__ lines;       // CG: ordered cells x L (null for DG)
  const int32_t* __restrict__ cell_rank;   // ordered cell -> active-cell rank
  const int32_t* __restrict__ face_start;
  const int32_t* __restrict__ face_kind;
  const double* __restrict__ face_phi;      // 1D values at x_q, or the shifts d_q (Taylor)
  const int32_t* __restrict__ nbr;         // DG neighbours (null for CG)
  const int32_t* __restrict__ pos;         // CG: ordered positions of this colour's cells
  int cell0, ncell, dg, taylor;
  double sigma_f;                          // DG interior penalty
};

template <int D, int N>
__global__ void diag_f64_kernel(const DiagArgs a, const __grid_constant__ KTab<double> t) {
  constexpr int L = (D == 3) ? N * N : N, ND = L * N;
  const int cell = a.pos ? a.pos[a.cell0 + blockIdx.x] : a.cell0 + blockIdx.x;
  for (int j = threadIdx.x; j < ND; j += blockDim.x) {
    int jj[3] = {j % N, (j / N) % N, (D == 3) ? j / (N * N) : 0};
    // cell term: h^(d-2) sum_k prod_l (k == l ? K : M)
    double v = 0.0;
    for (int k = 0; k < D; ++k) {
      double pr = 1.0;
      for (int l = 0; l < D; ++l) pr *= (l == k) ? t.Kh[jj[l]][jj[l]] : t.M[jj[l]][jj[l]];
      v += pr;
    }
    // surrogate faces of this cell
    const int fs = a.face_start[cell], fe = a.face_start[cell + 1];
    for (int f = fs; f < fe; ++f) {
      const int kind = a.face_kind[f], k = kind & 3, s = kind >> 2;
      const double vn = (jj[k] == (s ? N - 1 : 0)) ? 1.0 : 0.0;     // phi_{j_k}(s)
      const double dn = (s ? t.D1[jj[k]] : t.D0[jj[k]]) * (s ? 1.0 : -1.0) * t.h_inv;
      int ta = (k == 0) ? 1 : 0;
      int tb = (k == 2) ? 1 : 2;
      for (int q = 0; q < L; ++q) {
        const int qa = q % N, qb = q / N;
        double tang = t.S[qa][jj[ta]];
        if (D == 3) tang *= t.S[qb][jj[tb]];
        double shifted;
        if (a.taylor) {
          // psi_j(x~_q) + (1/h) d_q . grad_xi psi_j(x~_q)
          const double* dq = a.face_phi + ((size_t)f * L + q) * D;
          const double dnr = s ? t.D1[jj[k]] : t.D0[jj[k]];
          const double ta_v = t.S[qa][jj[ta]], ta_d = t.Dg[qa][jj[ta]];
          const double tb_v = (D == 3) ? t.S[qb][jj[tb]] : 1.0;
          const double tb_d = (D == 3) ? t.Dg[qb][jj[tb]] : 0.0;
          double g = dq[k] * dnr * ta_v * tb_v + dq[ta] * vn * ta_d * tb_v;
          if (D == 3) g += dq[tb] * vn * ta_v * tb_d;
          shifted = vn * ta_v * tb_v + t.h_inv * g;
        } else {
          const double* ph = a.face_phi + ((size_t)f * L + q) * D * N;
          shifted = 1.0;
          for (int l = 0; l < D; ++l) shifted *= ph[l * N + jj[l]];
        }
        const double vt = vn * tang, dt = dn * tang;
        v += t.W[q] * (-vt * dt - dt * shifted + t.sigma * vt * shifted);
      }
    }
    if (a.dg) {
      // SIPG interior faces (Algorithm 2), diagonal of the own-cell block:
      // sigma_F V^2 - V dn V (the average carries 1/2, the jump sign cancels)
      const int rank = a.cell_rank[cell];
      for (int k = 0; k < D; ++k)
        for (int s = 0; s < 2; ++s) {
          if (a.nbr[(size_t)rank * 2 * D + 2 * k + s] < 0) continue;
          const double vn = (jj[k] == (s ? N - 1 : 0)) ? 1.0 : 0.0;
          // outward normal of this cell on the face: (2s-1) e_k; {dn u} uses
          // the face normal n = +e_k, the jump [v] = v for the lower cell
          // (s = 1) and -v for the upper one: both give -1/2 V (n.grad V)(2s-1)
          const double dn = (s ? t.D1[jj[k]] : t.D0[jj[k]]) * t.h_inv;
          const double sg = s ? 1.0 : -1.0;
          int ta = (k == 0) ? 1 : 0;
          int tb = (k == 2) ? 1 : 2;
          for (int q = 0; q < L; ++q) {
            const int qa = q % N, qb = q / N;
            double tang = t.S[qa][jj[ta]];
            if (D == 3) tang *= t.S[qb][jj[tb]];
            const double vt = vn * tang, dt = dn * tang;
            v += t.W[q] * (a.sigma_f * vt * vt - sg * vt * dt);
          }
        }
      a.diag[(size_t)rank * ND + j] = v;
    } else {
      const int g = a.lines[(size_t)cell * L + j / N] + (j % N);
      a.diag[g] += v;
    }
  }
}

template <int D, int N>
static cudaError_t diag_t(const HostProblem& hp, const DeviceData& dd, double* diag,
                          cudaStream_t st) {
  constexpr int L = (D == 3) ? N * N : N, ND = L * N;
  const KTab<double> t = make_ktab<double>(hp);
  cudaError_t err;
  if (!hp.desc.dg) {
    err = cudaMemsetAsync(diag, 0, (size_t)hp.n_dofs * sizeof(double), st);
    if (err != cudaSuccess) return err;
  }
  const std::vector<int>& cs = hp.desc.dg ? dd.col_start : dd.diag_col_start;
  for (int c = 0; c < dd.ncolours; ++c) {
    const int n = cs[c + 1] - cs[c];
    if (n == 0) continue;
    DiagArgs a;
    a.diag = diag;
    a.lines = dd.lines;
    a.cell_rank = dd.cell_rank;
    a.face_start = dd.face_start;
    a.face_kind = dd.face_kind;
    a.face_phi = dd.face_phi;
    a.nbr = dd.nbr;
    a.cell0 = cs[c];
    a.pos = hp.desc.dg ? nullptr : dd.diag_pos;
    a.ncell = n;
    a.dg = hp.desc.dg;
    a.taylor = hp.desc.extension == SBM_EXT_TAYLOR1;
    a.sigma_f = hp.sigma_f;
    const int threads = ND < 128 ? ((ND + 31) / 32) * 32 : 128;
    diag_f64_kernel<D, N><<<n, threads, 0, st>>>(a, t);
  }
  return cudaGetLastError();
}

cudaError_t launch_diag_f64(const HostProblem& hp, const DeviceData& dd, double* diag,
                            cudaStream_t st) {
#define SBM_CASE(DD, NN) \
  if (hp.d == DD && hp.n == NN) return diag_t<DD, NN>(hp, dd, diag, st);
  SBM_CASE(2, 2) SBM_CASE(2, 3) SBM_CASE(2, 4) SBM_CASE(2, 5) SBM_CASE(2, 6) SBM_CASE(2, 7)
  SBM_CASE(3, 2) SBM_CASE(3, 3) SBM_CASE(3, 4) SBM_CASE(3, 5) SBM_CASE(3, 6) SBM_CASE(3, 7)
#undef SBM_CASE
  return cudaErrorInvalidValue;
}

}  // namespace sbm
