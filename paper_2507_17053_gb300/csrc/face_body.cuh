// Surrogate-boundary faces (Algorithm 3): the per-face device routine shared
// by the single-problem face kernel (face_kernel.cu) and the persistent
// batched apply.  See face_kernel.cu for the method.
#pragma once

#include <type_traits>

#include "sweeps.cuh"

namespace sbm {

template <typename T>
struct FaceArgs {
  const T* __restrict__ x;
  const int32_t* __restrict__ lines;       // CG gather (null for DG)
  const int32_t* __restrict__ cell_rank;   // DG gather
  const int32_t* __restrict__ face_cell;   // face -> ordered cell position
  const int32_t* __restrict__ face_kind;   // k | (s << 2)
  const T* __restrict__ face_phi;          // [F][L][D][N], or the shifts [F][L][D] (Taylor)
  const T* __restrict__ face_pp;           // 3D exact, FP64: [F][N^2][L] products of axes 1, 2
  T* __restrict__ out;                     // [F][2L]
  int face0, nface;                        // this launch: faces [face0, nface)
  int dg;
  int64_t ldx, ld_out;                     // right-hand side blockIdx.y offsets
};

// scratch arrays of L values per face: 6, or 9 with the Taylor extension
template <int EXT>
struct FaceScratch {
  static constexpr int n = EXT ? 9 : 6;
};

// shared-memory bytes of one group of FPB faces
template <typename T, int D, int N, int EXT, int FPB>
constexpr size_t face_group_smem() {
  return (size_t)(FPB * Shape<D, N>::ND + FPB * FaceScratch<EXT>::n * Shape<D, N>::L) * sizeof(T);
}

// Faces [f0, min(f0 + FPB, fend)) of right-hand side rhs, L threads per
// face (threads beyond FPB L idle but take part in the barriers).  t
// supplies the h-independent 1D tables, ts the problem's h-scaled ones (the
// face weights W, sigma, 1/h, h^(d-1)); the single-problem kernel passes its
// one table for both.
template <typename T, int D, int N, int EXT, int FPB>
__device__ __forceinline__ void face_group(const FaceArgs<T>& a, const KTab<T>& t,
                                           const KTab<T>& ts, unsigned char* smem_raw, int f0,
                                           int fend, int rhs) {
  constexpr int L = Shape<D, N>::L, ND = Shape<D, N>::ND;
  constexpr int NS = FaceScratch<EXT>::n;
  const T* __restrict__ xr = a.x + rhs * a.ldx;
  T* __restrict__ outr = a.out + rhs * a.ld_out;
  T* X = reinterpret_cast<T*>(smem_raw);
  T* SC = X + FPB * ND;            // NS L per face
  const int tid = threadIdx.x;
  const int nf = min(FPB, fend - f0);
  for (int r = tid; r < nf * ND; r += blockDim.x) {
    const int f = r / ND, loc = r - f * ND;
    const int cell = __ldg(a.face_cell + f0 + f);
    size_t g;
    if (a.dg) g = (size_t)__ldg(a.cell_rank + cell) * ND + loc;
    else g = (size_t)__ldg(a.lines + (size_t)cell * L + loc / N) + (loc % N);
    X[r] = __ldg(xr + g);
  }
  __syncthreads();
  const int fl = tid / L, tl = tid - fl * L;
  const bool act = fl < nf;
  const int f = f0 + (act ? fl : 0);
  const int kind = act ? __ldg(a.face_kind + f) : 0;
  const int k = kind & 3, s = kind >> 2;
  const T* Xf = X + fl * ND;
  T* sc = SC + fl * NS * L;
  T* Td = sc;
  T* Da = sc + L;
  T* val = sc + 2 * L;
  T* grd = sc + 3 * L;
  T* Va = sc + 4 * L;
  T* Ga = sc + 5 * L;
  T* Tv = sc + 6 * L;              // Taylor: value trace, then its two
  T* VA = sc + 7 * L;              // first-direction interpolants (value,
  T* VD = sc + 8 * L;              // derivative)
  int sk, sa, sb;
  if (D == 2) {
    sk = (k == 0) ? 1 : N;
    sa = (k == 0) ? N : 1;
    sb = 0;
  } else {
    sk = (k == 0) ? 1 : (k == 1 ? N : N * N);
    sa = (k == 0) ? N : 1;
    sb = (k == 2) ? N : N * N;
  }
  const int kend = s ? (N - 1) : 0;
  const T sg = s ? T(1) : T(-1);
  const int bt = (tl % N) * sa + (D == 3 ? (tl / N) * sb : 0);

  // 1. normal-derivative trace at the tangential nodes (with the exact
  //    extension the value trace u(x~_q) does not enter the operator: only
  //    E u at the shifted point does; the Taylor extension needs it)
  if (act) {
    T dsum = T(0);
#pragma unroll
    for (int j = 0; j < N; ++j) dsum = fma(s ? t.D1[j] : t.D0[j], Xf[j * sk + bt], dsum);
    Td[tl] = dsum;
    if (EXT) Tv[tl] = Xf[kend * sk + bt];
  }
  __syncthreads();
  T rv = T(0), rg = T(0);
  if constexpr (EXT == 0) {
    // 2. the exact extension: the normal-derivative integrand is a multiple
    //    of E u, and the normal-derivative trace enters only through
    //    (S x S)^T diag(W) (S x S) Td = h^(d-1) (M x M) Td (the face's Gauss
    //    rule is exact for it), so one transposed interpolation (of W E)
    //    and one mass product replace the interpolation of Td and two
    //    transposed interpolations
    T tm = T(0);                  // (M x M) Td at tangential node tl
    if (D == 3) {
      if (act) {
        const int ia = tl % N, jb = tl / N;
        T v = T(0);
#pragma unroll
        for (int j = 0; j < N; ++j) v = fma(t.M[ia][j], Td[j + N * jb], v);
        Da[tl] = v;
      }
      __syncthreads();
      if (act) {
        const int ia = tl % N, ib = tl / N;
#pragma unroll
        for (int j = 0; j < N; ++j) tm = fma(t.M[ib][j], Da[ia + N * j], tm);
      }
    } else if (act) {
#pragma unroll
      for (int j = 0; j < N; ++j) tm = fma(t.M[tl][j], Td[j], tm);
    }
    // 3. E u at the shifted point of Gauss point tl, weighted.  3D FP64:
    //    E u = sum_j0 phi_j0 sum_{j1,j2} P[j1 + n j2] u[j0, j1, j2] with the
    //    stored products P of the other two axes' values: n^3 + n FMAs
    //    instead of n^3 + n^2 + n (FP32: the products cost less than their
    //    loads, the 1D values are contracted axis by axis)
    if (act) {
      const T* pq = a.face_phi + ((size_t)f * L + tl) * D * N;
      T p0[N];
#pragma unroll
      for (int j = 0; j < N; ++j) p0[j] = __ldg(pq + j);
      T e = T(0);
      if (D == 3 && !std::is_same<T, double>::value) {
        T p1[N], p2[N];
#pragma unroll
        for (int j = 0; j < N; ++j) {
          p1[j] = __ldg(pq + N + j);
          p2[j] = __ldg(pq + 2 * N + j);
        }
#pragma unroll
        for (int j2 = 0; j2 < N; ++j2) {
          T s1 = T(0);
#pragma unroll
          for (int j1 = 0; j1 < N; ++j1) {
            T s0 = T(0);
#pragma unroll
            for (int j0 = 0; j0 < N; ++j0) s0 = fma(p0[j0], Xf[j0 + N * j1 + N * N * j2], s0);
            s1 = fma(p1[j1], s0, s1);
          }
          e = fma(p2[j2], s1, e);
        }
      } else if (D == 3) {
        const T* pp = a.face_pp + (size_t)f * N * N * L + tl;
        T acc[N];
#pragma unroll
        for (int j0 = 0; j0 < N; ++j0) acc[j0] = T(0);
#pragma unroll
        for (int j12 = 0; j12 < N * N; ++j12) {
          const T w = __ldg(pp + (size_t)j12 * L);
#pragma unroll
          for (int j0 = 0; j0 < N; ++j0) acc[j0] = fma(w, Xf[j0 + N * j12], acc[j0]);
        }
#pragma unroll
        for (int j0 = 0; j0 < N; ++j0) e = fma(p0[j0], acc[j0], e);
      } else {
        T p1[N];
#pragma unroll
        for (int j = 0; j < N; ++j) p1[j] = __ldg(pq + N + j);
#pragma unroll
        for (int j1 = 0; j1 < N; ++j1) {
          T s0 = T(0);
#pragma unroll
          for (int j0 = 0; j0 < N; ++j0) s0 = fma(p0[j0], Xf[j0 + N * j1], s0);
          e = fma(p1[j1], s0, e);
        }
      }
      val[tl] = ts.W[tl] * e;
    }
    __syncthreads();
    // 4. q = (S x S)^T (W E) at tangential node tl
    T q = T(0);
    if (D == 3) {
      if (act) {
        const int ja = tl % N, qb = tl / N;
        T v = T(0);
#pragma unroll
        for (int g = 0; g < N; ++g) v = fma(t.S[g][ja], val[g + N * qb], v);
        Va[tl] = v;
      }
      __syncthreads();
      if (act) {
        const int ja = tl % N, jb = tl / N;
#pragma unroll
        for (int g = 0; g < N; ++g) q = fma(t.S[g][jb], Va[ja + N * g], q);
      }
    } else if (act) {
#pragma unroll
      for (int g = 0; g < N; ++g) q = fma(t.S[g][tl], val[g], q);
    }
    // value test: sigma E - dn u (h^-1 for the physical derivative); normal-
    // derivative test: -E (with the outward sign and h^-1)
    rv = fma(ts.sigma, q, -(sg * ts.h_inv * ts.hface) * tm);
    rg = -(sg * ts.h_inv) * q;
  } else {
    // 2. first-order Taylor extension: the normal derivative, the value and
    //    its derivatives along the tangential axes ta, tb at the tangential
    //    Gauss points (axis ta is the one of stride sa, interpolated first)
    T dg = T(0), uv = T(0), da = T(0), db = T(0);
    if (D == 3) {
      if (act) {
        const int qa = tl % N, jb = tl / N;
        T dv = T(0), va = T(0), vd = T(0);
  #pragma unroll
        for (int j = 0; j < N; ++j) {
          dv = fma(t.S[qa][j], Td[j + N * jb], dv);
          if (EXT) {
            va = fma(t.S[qa][j], Tv[j + N * jb], va);
            vd = fma(t.Dg[qa][j], Tv[j + N * jb], vd);
          }
        }
        Da[tl] = dv;
        if (EXT) {
          VA[tl] = va;
          VD[tl] = vd;
        }
      }
      __syncthreads();
      if (act) {
        const int qa = tl % N, qb = tl / N;
  #pragma unroll
        for (int j = 0; j < N; ++j) {
          dg = fma(t.S[qb][j], Da[qa + N * j], dg);
          if (EXT) {
            uv = fma(t.S[qb][j], VA[qa + N * j], uv);
            da = fma(t.S[qb][j], VD[qa + N * j], da);
            db = fma(t.Dg[qb][j], VA[qa + N * j], db);
          }
        }
      }
    } else {
      if (act) {
  #pragma unroll
        for (int j = 0; j < N; ++j) {
          dg = fma(t.S[tl][j], Td[j], dg);
          if (EXT) {
            uv = fma(t.S[tl][j], Tv[j], uv);
            da = fma(t.Dg[tl][j], Tv[j], da);
          }
        }
      }
    }
    // 3. the extension at x~_q, pointwise integrands
    if (act && EXT) {
      // E u = u + d . grad u, grad = (1/h) reference gradient; reference
      // derivatives: along k dg, along ta da, along tb db
      const T* dq = a.face_phi + ((size_t)f * L + tl) * D;
      const int ta = (D == 2) ? 1 - k : (k == 0 ? 1 : 0);
      const int tb = (k == 2) ? 1 : 2;
      T g = fma(__ldg(dq + k), dg, __ldg(dq + ta) * da);
      if (D == 3) g = fma(__ldg(dq + tb), db, g);
      const T e = fma(ts.h_inv, g, uv);
      const T W = ts.W[tl];
      val[tl] = W * (ts.sigma * e - sg * ts.h_inv * dg);
      grd[tl] = -W * e * sg * ts.h_inv;
    }
    __syncthreads();
    // 4. transposed interpolation back to the tangential nodes
    if (D == 3) {
      if (act) {
        const int ja = tl % N, qb = tl / N;
        T v1 = T(0), v2 = T(0);
  #pragma unroll
        for (int q = 0; q < N; ++q) {
          v1 = fma(t.S[q][ja], val[q + N * qb], v1);
          v2 = fma(t.S[q][ja], grd[q + N * qb], v2);
        }
        Va[tl] = v1;
        Ga[tl] = v2;
      }
      __syncthreads();
      if (act) {
        const int ja = tl % N, jb = tl / N;
  #pragma unroll
        for (int q = 0; q < N; ++q) {
          rv = fma(t.S[q][jb], Va[ja + N * q], rv);
          rg = fma(t.S[q][jb], Ga[ja + N * q], rg);
        }
      }
    } else {
      if (act) {
  #pragma unroll
        for (int q = 0; q < N; ++q) {
          rv = fma(t.S[q][tl], val[q], rv);
          rg = fma(t.S[q][tl], grd[q], rg);
        }
      }
    }
  }
  if (act) {
    outr[(size_t)f * 2 * L + tl] = rv;
    outr[(size_t)f * 2 * L + L + tl] = rg;
  }
}

}  // namespace sbm
