// Adjoint (vector-Jacobian product) of the DG operator:
//   (dL/dU)^T W = -(dF/dU)^T Y,   Y = M^{-1} W   (M symmetric; no body force)
// The kernel evaluates (dF/dU)^T Y element-centrically, like the forward
// kernel: F = T^T Phi(I U) per cell and per face, so (dF/dU)^T Y = I^T Phi'^T (T Y):
// interpolate U (values, gradients) and the test quantities of Y (values and
// reference gradients of the field Y at the same points), apply the
// transposed pointwise Jacobians (dg_adjoint_point.cuh), and test back with
// the transposed interpolation.  For every face the cell evaluates both the
// transpose of its own face term (adjoint input Y of the cell) and of the
// neighbour's face term in which the cell is the exterior side (adjoint input
// Y of the neighbour), so no two CTAs write the same cell.
#pragma once
#include "dg_adjoint_point.cuh"
#include "dg_faces.cuh"
#include "dg_launchers.h"

namespace dgcns {

template <int N, int QC, int QV>
struct AdjSizes {
  static constexpr int N2 = N * N, N3 = N * N * N;
  static constexpr int PC = QC * QC * QC, PV = QV * QV * QV;
  static constexpr int CELL = (25 * PC > 40 * PV ? 25 * PC : 40 * PV);
  static constexpr int FCONV = 4 * 5 * N2 + 5 * QC * N + 4 * 5 * QC * QC;
  static constexpr int FVISC = 8 * 5 * N2 + 5 * QV * N + 16 * 5 * QV * QV;
  static constexpr int FACE = FCONV > FVISC ? FCONV : FVISC;
  static constexpr int ARENA = CELL > FACE ? CELL : FACE;
};

// PAIR: face terms come as shares from the face-centric adjoint face kernel (no neighbour states,
// cell arena only).
template <int N, int QC, int QV, bool PAIR>
constexpr int adj_cell_elems() {
  using S = AdjSizes<N, QC, QV>;
  return PAIR ? 3 * 5 * S::N3 + S::CELL : 5 * 5 * S::N3 + S::ARENA;
}

template <typename T, int N, int QC, int QV, bool PAIR>
constexpr int adj_cells_per_cta() {
  constexpr int per_cell = adj_cell_elems<N, QC, QV, PAIR>() * (int)sizeof(T) + 16;
  constexpr int cb = (112 * 1024 - table_elems<N, QC, QV>() * (int)sizeof(T)) / per_cell;
  return cb < 1 ? 1 : (cb > 4 ? 4 : cb);
}

template <typename T, int N, int QC, int QV, int CB, bool PAIR>
constexpr size_t adj_smem_bytes() {
  return (table_elems<N, QC, QV>() + (size_t)CB * adj_cell_elems<N, QC, QV, PAIR>() + CB) * sizeof(T) +
         2 * CB * sizeof(int) + 64;
}

// geometry at a cell point: J^{-1}[b][a] (index 3b+a) and |J| w
template <typename T, int GEO>
__device__ __forceinline__ void cell_geo(const KParams& kp, const void* g, int P, size_t cell, int p, T wq,
                                         T Ji[9], T& jw) {
  if (GEO == GEO_AFFINE) {
#pragma unroll
    for (int m = 0; m < 9; ++m) Ji[m] = T(0);
    const KConst<T>& kc = kconst<T>(kp);
    Ji[0] = kc.hinv[0];
    Ji[4] = kc.hinv[1];
    Ji[8] = kc.hinv[2];
    jw = wq * kc.detJ;
  } else {
    const T* gg = static_cast<const T*>(g) + cell * 10 * P + p;
#pragma unroll
    for (int m = 0; m < 9; ++m) Ji[m] = gg[m * P];
    jw = wq * gg[9 * P];
  }
}

// ---------------------------------------------------------------------------
// Cell terms of (dF/dU)^T Y, accumulated into sg.
// ---------------------------------------------------------------------------
template <typename T, int N, int QC, int QV, int CB, int GEO>
__device__ void adj_cell_terms(const T* su, const T* sy, T* sg, T* ar, const Tab<T>& tb, const KParams& kp,
                               const PhysT<T>& ph, int e0, int nb) {
  const int nbl = nb * 5;
  if (kp.conv) {
    constexpr int P = QC * QC * QC;
    T* A0 = ar;
    T* B0 = ar + CB * 5 * P;
    T* B1 = B0 + CB * 5 * P;
    T* B2 = B1 + CB * 5 * P;
    T* B3 = B2 + CB * 5 * P;
    sweep<T, 0, N, N, N, QC, 1, false>(su, B1, tb.eSc, nbl);
    __syncthreads();
    sweep<T, 1, QC, N, N, QC, 1, false>(B1, B2, tb.eSc, nbl);
    __syncthreads();
    sweep<T, 2, QC, QC, N, QC, 1, false>(B2, A0, tb.eSc, nbl);
    __syncthreads();
    sweep<T, 0, N, N, N, QC, 1, false>(sy, B1, tb.eSc, nbl);
    __syncthreads();
    sweep<T, 1, QC, N, N, QC, 1, false>(B1, B2, tb.eSc, nbl);
    __syncthreads();
    sweep<T, 2, QC, QC, N, QC, 1, false>(B2, B0, tb.eSc, nbl);
    __syncthreads();
    sweep<T, 0, QC, QC, QC, QC, -1, false>(B0, B1, tb.eDc, nbl);
    sweep<T, 1, QC, QC, QC, QC, -1, false>(B0, B2, tb.eDc, nbl);
    sweep<T, 2, QC, QC, QC, QC, -1, false>(B0, B3, tb.eDc, nbl);
    __syncthreads();
    for (int idx = threadIdx.x; idx < nb * P; idx += blockDim.x) {
      const int e = idx / P, p = idx - e * P;
      const int o = e * 5 * P + p;
      T Ji[9], jw;
      cell_geo<T, GEO>(kp, kp.gcc, P, (size_t)(e0 + e), p, tb.wc[p % QC] * tb.wc[(p / QC) % QC] * tb.wc[p / (QC * QC)],
                       Ji, jw);
      T u[5], ub[5], Fb[3][5];
#pragma unroll
      for (int c = 0; c < 5; ++c) {
        u[c] = A0[o + c * P];
        ub[c] = T(0);
        const T y0 = B1[o + c * P], y1 = B2[o + c * P], y2 = B3[o + c * P];
#pragma unroll
        for (int a = 0; a < 3; ++a) Fb[a][c] = jw * (Ji[a] * y0 + Ji[3 + a] * y1 + Ji[6 + a] * y2);
      }
      conv_flux_vjp(u, Fb, ph, ub);
#pragma unroll
      for (int c = 0; c < 5; ++c) A0[o + c * P] = -ub[c];  // -(grad V, F_c)
    }
    __syncthreads();
    sweep<T, 2, QC, QC, QC, N, 1, false>(A0, B1, tb.eScT, nbl);
    __syncthreads();
    sweep<T, 1, QC, QC, N, N, 1, false>(B1, B2, tb.eScT, nbl);
    __syncthreads();
    sweep<T, 0, QC, N, N, N, 1, true>(B2, sg, tb.eScT, nbl);
    __syncthreads();
  }
  if (kp.visc) {
    constexpr int P = QV * QV * QV;
    T* A0 = ar;
    T* A1 = A0 + CB * 5 * P;
    T* A2 = A1 + CB * 5 * P;
    T* A3 = A2 + CB * 5 * P;
    T* B0 = A3 + CB * 5 * P;
    T* B1 = B0 + CB * 5 * P;
    T* B2 = B1 + CB * 5 * P;
    T* B3 = B2 + CB * 5 * P;
    sweep<T, 0, N, N, N, QV, 1, false>(su, B1, tb.eSv, nbl);
    __syncthreads();
    sweep<T, 1, QV, N, N, QV, 1, false>(B1, B2, tb.eSv, nbl);
    __syncthreads();
    sweep<T, 2, QV, QV, N, QV, 1, false>(B2, A0, tb.eSv, nbl);
    __syncthreads();
    sweep<T, 0, N, N, N, QV, 1, false>(sy, B1, tb.eSv, nbl);
    __syncthreads();
    sweep<T, 1, QV, N, N, QV, 1, false>(B1, B2, tb.eSv, nbl);
    __syncthreads();
    sweep<T, 2, QV, QV, N, QV, 1, false>(B2, B0, tb.eSv, nbl);
    __syncthreads();
    sweep<T, 0, QV, QV, QV, QV, -1, false>(A0, A1, tb.eDv, nbl);
    sweep<T, 1, QV, QV, QV, QV, -1, false>(A0, A2, tb.eDv, nbl);
    sweep<T, 2, QV, QV, QV, QV, -1, false>(A0, A3, tb.eDv, nbl);
    sweep<T, 0, QV, QV, QV, QV, -1, false>(B0, B1, tb.eDv, nbl);
    sweep<T, 1, QV, QV, QV, QV, -1, false>(B0, B2, tb.eDv, nbl);
    sweep<T, 2, QV, QV, QV, QV, -1, false>(B0, B3, tb.eDv, nbl);
    __syncthreads();
    for (int idx = threadIdx.x; idx < nb * P; idx += blockDim.x) {
      const int e = idx / P, p = idx - e * P;
      const int o = e * 5 * P + p;
      T Ji[9], jw;
      cell_geo<T, GEO>(kp, kp.gcv, P, (size_t)(e0 + e), p, tb.wv[p % QV] * tb.wv[(p / QV) % QV] * tb.wv[p / (QV * QV)],
                       Ji, jw);
      T u[5], ub[5], G[5][3], Gb[5][3], Fb[5][3];
#pragma unroll
      for (int c = 0; c < 5; ++c) {
        u[c] = A0[o + c * P];
        ub[c] = T(0);
        const T g0 = A1[o + c * P], g1 = A2[o + c * P], g2 = A3[o + c * P];
        const T y0 = B1[o + c * P], y1 = B2[o + c * P], y2 = B3[o + c * P];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          G[c][a] = Ji[a] * g0 + Ji[3 + a] * g1 + Ji[6 + a] * g2;
          Fb[c][a] = jw * (Ji[a] * y0 + Ji[3 + a] * y1 + Ji[6 + a] * y2);
          Gb[c][a] = T(0);
        }
      }
      visc_flux_vjp(u, G, Fb, ph, ub, Gb);
#pragma unroll
      for (int c = 0; c < 5; ++c) {
        A0[o + c * P] = ub[c];
        A1[o + c * P] = Ji[0] * Gb[c][0] + Ji[1] * Gb[c][1] + Ji[2] * Gb[c][2];
        A2[o + c * P] = Ji[3] * Gb[c][0] + Ji[4] * Gb[c][1] + Ji[5] * Gb[c][2];
        A3[o + c * P] = Ji[6] * Gb[c][0] + Ji[7] * Gb[c][1] + Ji[8] * Gb[c][2];
      }
    }
    __syncthreads();
    sweep<T, 0, QV, QV, QV, QV, -1, true>(A1, A0, tb.eDvT, nbl);
    __syncthreads();
    sweep<T, 1, QV, QV, QV, QV, -1, true>(A2, A0, tb.eDvT, nbl);
    __syncthreads();
    sweep<T, 2, QV, QV, QV, QV, -1, true>(A3, A0, tb.eDvT, nbl);
    __syncthreads();
    sweep<T, 2, QV, QV, QV, N, 1, false>(A0, B0, tb.eSvT, nbl);
    __syncthreads();
    sweep<T, 1, QV, QV, N, N, 1, false>(B0, B1, tb.eSvT, nbl);
    __syncthreads();
    sweep<T, 0, QV, N, N, N, 1, true>(B1, sg, tb.eSvT, nbl);
    __syncthreads();
  }
}

// face geometry at a face point: own J^{-1}, neighbour J^{-1}, unit normal, dA w
template <typename T, int GEO, int d>
__device__ __forceinline__ void face_geo(const KParams& kp, const void* g, int P, size_t cell, size_t nbr, int f,
                                         int fo, int p, T wq, bool wall, int s, T Jm[9], T Jp[9], T n[3], T& w) {
  if (GEO == GEO_AFFINE) {
#pragma unroll
    for (int m = 0; m < 9; ++m) Jm[m] = T(0);
    const KConst<T>& kc = kconst<T>(kp);
    Jm[0] = kc.hinv[0];
    Jm[4] = kc.hinv[1];
    Jm[8] = kc.hinv[2];
#pragma unroll
    for (int m = 0; m < 9; ++m) Jp[m] = Jm[m];
    n[0] = n[1] = n[2] = T(0);
    n[d] = s ? T(1) : T(-1);
    w = wq * kc.area[d];
  } else {
    const T* gg = static_cast<const T*>(g) + (cell * 6 + f) * 13 * P + p;
#pragma unroll
    for (int m = 0; m < 9; ++m) Jm[m] = gg[m * P];
    n[0] = gg[9 * P];
    n[1] = gg[10 * P];
    n[2] = gg[11 * P];
    w = wq * gg[12 * P];
    if (!wall) {
      const T* gp = static_cast<const T*>(g) + (nbr * 6 + fo) * 13 * P + p;
#pragma unroll
      for (int m = 0; m < 9; ++m) Jp[m] = gp[m * P];
    } else {
#pragma unroll
      for (int m = 0; m < 9; ++m) Jp[m] = Jm[m];
    }
  }
}

// ---------------------------------------------------------------------------
// Face terms of (dF/dU)^T Y for face (d, s) of the CTA's cells.
// su/sy: own U (deviation) and Y; snu/sny: neighbour's; sg accumulates.
// ---------------------------------------------------------------------------
template <typename T, int N, int QC, int QV, int CB, int d, int GEO>
__device__ void adj_face_terms(const T* su, const T* sy, const T* snu, const T* sny, const int* wall, const int* nbi,
                               const T* tau_f, T* sg, T* fa, const Tab<T>& tb, const KParams& kp, const PhysT<T>& ph,
                               int e0, int nb, int s) {
  constexpr int N2 = N * N, N3 = N * N * N;
  constexpr int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
  const int f = 2 * d + s, fo = 2 * d + (1 - s);
  const int idm = s ? N - 1 : 0, idp = s ? 0 : N - 1;
  const T* dlm = s ? tb.dl1 : tb.dl0;
  const T* dlp = s ? tb.dl0 : tb.dl1;
  const int nbl = nb * 5;

  if (kp.conv) {
    constexpr int P = QC * QC;
    T* Lue = fa;
    T* Lun = Lue + CB * 5 * N2;
    T* Lye = Lun + CB * 5 * N2;
    T* Lyn = Lye + CB * 5 * N2;
    T* Tm = Lyn + CB * 5 * N2;
    T* ue = Tm + CB * 5 * QC * N;
    T* un = ue + CB * 5 * P;
    T* ye = un + CB * 5 * P;
    T* yn = ye + CB * 5 * P;
    for (int idx = threadIdx.x; idx < nbl * N2; idx += blockDim.x) {
      const int ec = idx / N2, j = idx - ec * N2, e = ec / 5;
      const int nm = face_node<N>(d, idm, j % N, j / N), np = face_node<N>(d, idp, j % N, j / N);
      Lue[idx] = su[ec * N3 + nm];
      Lye[idx] = sy[ec * N3 + nm];
      Lun[idx] = wall[e] ? T(0) : snu[ec * N3 + np];
      Lyn[idx] = wall[e] ? T(0) : sny[ec * N3 + np];
    }
    __syncthreads();
    T* L4[4] = {Lue, Lun, Lye, Lyn};
    T* P4[4] = {ue, un, ye, yn};
#pragma unroll 1
    for (int r = 0; r < 4; ++r) {
      sweep<T, 0, N, N, 1, QC, 1, false>(L4[r], Tm, tb.eSc, nbl);
      __syncthreads();
      sweep<T, 1, QC, N, 1, QC, 1, false>(Tm, P4[r], tb.eSc, nbl);
      __syncthreads();
    }
    for (int idx = threadIdx.x; idx < nb * P; idx += blockDim.x) {
      const int e = idx / P, p = idx - e * P;
      const int o = e * 5 * P + p;
      T Jm[9], Jp[9], n[3], w;
      face_geo<T, GEO, d>(kp, kp.gfc, P, (size_t)(e0 + e), wall[e] ? 0 : (size_t)nbi[e], f, fo, p,
                          tb.wc[p % QC] * tb.wc[p / QC], wall[e] != 0, s, Jm, Jp, n, w);
      T um[5], up[5], yv[5], umb[5], upb[5];
#pragma unroll
      for (int c = 0; c < 5; ++c) {
        um[c] = ue[o + c * P];
        up[c] = un[o + c * P];
        yv[c] = ye[o + c * P];
        umb[c] = T(0);
        upb[c] = T(0);
      }
      if (wall[e]) {
        wall_ghost(um, ph, up);
        llf_vjp(um, up, n, w, yv, ph, umb, upb);
        wall_ghost_vjp(um, upb, ph, umb);
      } else {
        llf_vjp(um, up, n, w, yv, ph, umb, upb);
        // the neighbour's face term, in which this cell is the exterior side
        T yn5[5], dummy[5], nn[3] = {-n[0], -n[1], -n[2]};
#pragma unroll
        for (int c = 0; c < 5; ++c) {
          yn5[c] = yn[o + c * P];
          dummy[c] = T(0);
        }
        llf_vjp(up, um, nn, w, yn5, ph, dummy, umb);
      }
#pragma unroll
      for (int c = 0; c < 5; ++c) ue[o + c * P] = umb[c];
    }
    __syncthreads();
    sweep<T, 1, QC, QC, 1, N, 1, false>(ue, Tm, tb.eScT, nbl);
    __syncthreads();
    sweep<T, 0, QC, N, 1, N, 1, false>(Tm, Lue, tb.eScT, nbl);
    __syncthreads();
    for (int idx = threadIdx.x; idx < nbl * N2; idx += blockDim.x) {
      const int ec = idx / N2, j = idx - ec * N2;
      sg[ec * N3 + face_node<N>(d, idm, j % N, j / N)] += Lue[idx];
    }
    __syncthreads();
  }

  if (kp.visc) {
    constexpr int P = QV * QV;
    T* Lay = fa;  // 8 layers [CB][5][N2]: U_e, dU_e, U_n, dU_n, Y_e, dY_e, Y_n, dY_n
    T* Tm = Lay + 8 * CB * 5 * N2;
    T* Pt = Tm + CB * 5 * QV * N;  // 16 point arrays [CB][5][P]
    auto PT = [&](int k) { return Pt + k * CB * 5 * P; };
    // point arrays: 0..3 U_e (val, t1, t2, d), 4..7 U_n, 8..11 Y_e, 12..15 Y_n
    for (int idx = threadIdx.x; idx < nbl * N2; idx += blockDim.x) {
      const int ec = idx / N2, j = idx - ec * N2, e = ec / 5;
      const int j1 = j % N, j2 = j / N;
      const T* a = su + ec * N3;
      const T* b = sy + ec * N3;
      T du = T(0), dy = T(0);
#pragma unroll
      for (int i = 0; i < N; ++i) {
        du += dlm[i] * a[face_node<N>(d, i, j1, j2)];
        dy += dlm[i] * b[face_node<N>(d, i, j1, j2)];
      }
      Lay[0 * CB * 5 * N2 + idx] = a[face_node<N>(d, idm, j1, j2)];
      Lay[1 * CB * 5 * N2 + idx] = du;
      Lay[4 * CB * 5 * N2 + idx] = b[face_node<N>(d, idm, j1, j2)];
      Lay[5 * CB * 5 * N2 + idx] = dy;
      if (wall[e]) {
        Lay[2 * CB * 5 * N2 + idx] = T(0);
        Lay[3 * CB * 5 * N2 + idx] = T(0);
        Lay[6 * CB * 5 * N2 + idx] = T(0);
        Lay[7 * CB * 5 * N2 + idx] = T(0);
      } else {
        const T* an = snu + ec * N3;
        const T* bn = sny + ec * N3;
        T dun = T(0), dyn = T(0);
#pragma unroll
        for (int i = 0; i < N; ++i) {
          dun += dlp[i] * an[face_node<N>(d, i, j1, j2)];
          dyn += dlp[i] * bn[face_node<N>(d, i, j1, j2)];
        }
        Lay[2 * CB * 5 * N2 + idx] = an[face_node<N>(d, idp, j1, j2)];
        Lay[3 * CB * 5 * N2 + idx] = dun;
        Lay[6 * CB * 5 * N2 + idx] = bn[face_node<N>(d, idp, j1, j2)];
        Lay[7 * CB * 5 * N2 + idx] = dyn;
      }
    }
    __syncthreads();
    // values (layers 0,2,4,6) -> point arrays 0,4,8,12; normal derivatives (1,3,5,7) -> 3,7,11,15
#pragma unroll 1
    for (int r = 0; r < 8; ++r) {
      const int dst = (r / 2) * 4 + ((r & 1) ? 3 : 0);
      sweep<T, 0, N, N, 1, QV, 1, false>(Lay + r * CB * 5 * N2, Tm, tb.eSv, nbl);
      __syncthreads();
      sweep<T, 1, QV, N, 1, QV, 1, false>(Tm, PT(dst), tb.eSv, nbl);
      __syncthreads();
    }
#pragma unroll 1
    for (int r = 0; r < 4; ++r) {
      sweep<T, 0, QV, QV, 1, QV, -1, false>(PT(4 * r), PT(4 * r + 1), tb.eDv, nbl);
      sweep<T, 1, QV, QV, 1, QV, -1, false>(PT(4 * r), PT(4 * r + 2), tb.eDv, nbl);
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < nb * P; idx += blockDim.x) {
      const int e = idx / P, p = idx - e * P;
      const int o = e * 5 * P + p;
      T Jm[9], Jp[9], n[3], w;
      face_geo<T, GEO, d>(kp, kp.gfv, P, (size_t)(e0 + e), wall[e] ? 0 : (size_t)nbi[e], f, fo, p,
                          tb.wv[p % QV] * tb.wv[p / QV], wall[e] != 0, s, Jm, Jp, n, w);
      const T tau = tau_f[e];
      // reference-direction index of the point arrays: t1 -> 1, t2 -> 2, d -> 3
      int slot[3];
      slot[t1] = 1;
      slot[t2] = 2;
      slot[d] = 3;
      T ue[5], un[5], Ge[5][3], Gn[5][3], yv[5], yb[3][5];
#pragma unroll
      for (int c = 0; c < 5; ++c) {
        ue[c] = PT(0)[o + c * P];
        un[c] = PT(4)[o + c * P];
        yv[c] = PT(8)[o + c * P];
        T ge[3], gn[3];
#pragma unroll
        for (int b = 0; b < 3; ++b) {
          ge[b] = PT(slot[b])[o + c * P];
          gn[b] = PT(4 + slot[b])[o + c * P];
          yb[b][c] = PT(8 + slot[b])[o + c * P];
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          Ge[c][a] = Jm[a] * ge[0] + Jm[3 + a] * ge[1] + Jm[6 + a] * ge[2];
          Gn[c][a] = Jp[a] * gn[0] + Jp[3 + a] * gn[1] + Jp[6 + a] * gn[2];
        }
      }
      T ueb[5], Geb[5][3], upb[5], Gpb[5][3];
#pragma unroll
      for (int c = 0; c < 5; ++c) {
        ueb[c] = T(0);
        upb[c] = T(0);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          Geb[c][a] = T(0);
          Gpb[c][a] = T(0);
        }
      }
      if (wall[e]) {
        wall_ghost(ue, ph, un);
        sipg_vjp(ue, Ge, un, Ge, n, Jm, w, tau, yv, yb, ph, ueb, Geb, upb, Gpb);
        wall_ghost_vjp(ue, upb, ph, ueb);
#pragma unroll
        for (int c = 0; c < 5; ++c)
#pragma unroll
          for (int a = 0; a < 3; ++a) Geb[c][a] += Gpb[c][a];
      } else {
        sipg_vjp(ue, Ge, un, Gn, n, Jm, w, tau, yv, yb, ph, ueb, Geb, upb, Gpb);
        // the neighbour's face term (this cell is its exterior side)
        T ynv[5], ynb[3][5], nn[3] = {-n[0], -n[1], -n[2]};
#pragma unroll
        for (int c = 0; c < 5; ++c) {
          ynv[c] = PT(12)[o + c * P];
#pragma unroll
          for (int b = 0; b < 3; ++b) ynb[b][c] = PT(12 + slot[b])[o + c * P];
        }
        T dm[5], dG[5][3];
#pragma unroll
        for (int c = 0; c < 5; ++c) {
          dm[c] = T(0);
#pragma unroll
          for (int a = 0; a < 3; ++a) dG[c][a] = T(0);
        }
        sipg_vjp(un, Gn, ue, Ge, nn, Jp, w, tau, ynv, ynb, ph, dm, dG, ueb, Geb);
      }
#pragma unroll
      for (int c = 0; c < 5; ++c) {
        PT(0)[o + c * P] = ueb[c];
#pragma unroll
        for (int b = 0; b < 3; ++b)
          PT(slot[b])[o + c * P] = Jm[3 * b] * Geb[c][0] + Jm[3 * b + 1] * Geb[c][1] + Jm[3 * b + 2] * Geb[c][2];
      }
    }
    __syncthreads();
    // test with V and with the tangential derivatives of V on the face grid, then the normal derivative
    sweep<T, 0, QV, QV, 1, QV, -1, true>(PT(1), PT(0), tb.eDvT, nbl);
    __syncthreads();
    sweep<T, 1, QV, QV, 1, QV, -1, true>(PT(2), PT(0), tb.eDvT, nbl);
    __syncthreads();
    sweep<T, 1, QV, QV, 1, N, 1, false>(PT(0), Tm, tb.eSvT, nbl);
    __syncthreads();
    sweep<T, 0, QV, N, 1, N, 1, false>(Tm, Lay, tb.eSvT, nbl);
    __syncthreads();
    sweep<T, 1, QV, QV, 1, N, 1, false>(PT(3), Tm, tb.eSvT, nbl);
    __syncthreads();
    sweep<T, 0, QV, N, 1, N, 1, false>(Tm, Lay + CB * 5 * N2, tb.eSvT, nbl);
    __syncthreads();
    for (int idx = threadIdx.x; idx < nbl * N2; idx += blockDim.x) {
      const int ec = idx / N2, j = idx - ec * N2;
      const int j1 = j % N, j2 = j / N;
      const T lv = Lay[idx], dv = Lay[CB * 5 * N2 + idx];
      T* r = sg + ec * N3;
#pragma unroll
      for (int i = 0; i < N; ++i) {
        T add = dlm[i] * dv;
        if (i == idm) add += lv;
        r[face_node<N>(d, i, j1, j2)] += add;
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Adjoint kernel.  Y = M^{-1} W for all cells (precomputed).  out_mode 0:
// G = -(dF/dU)^T Y; out_mode 2: lam_U += dt * (-(dF/dU)^T Y) (RK stage adjoint).
// ---------------------------------------------------------------------------
template <typename T, int N, int QC, int QV, int CB, int GEO, bool PAIR>
__global__ void __launch_bounds__(NT) dg_adj_kernel(const KParams kp, const double* __restrict__ U,
                                                    const T* __restrict__ Y, T* __restrict__ G,
                                                    double* __restrict__ lamU) {
  using S = AdjSizes<N, QC, QV>;
  constexpr int N3 = S::N3;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  T* stab = sm;
  T* su = stab + table_elems<N, QC, QV>();
  T* sy = su + CB * 5 * N3;
  T* sg = sy + CB * 5 * N3;
  T* snu = sg + CB * 5 * N3;
  T* sny = snu + (PAIR ? 0 : CB * 5 * N3);
  T* ar = sny + (PAIR ? 0 : CB * 5 * N3);
  T* tau_f = ar + CB * (PAIR ? S::CELL : S::ARENA);
  int* wall = reinterpret_cast<int*>(tau_f + CB);
  int* nbi = wall + CB;
  const int e0 = blockIdx.x * CB;
  const int nb = min(CB, kp.Nc - e0);
  if (nb <= 0) return;
  const Tab<T> tb = load_tables<T, N, QC, QV>(static_cast<const T*>(kp.tables), stab);
  const PhysT<T> ph = make_phys<T>(kp);
  const size_t base = (size_t)e0 * 5 * N3;
  const int nvals = nb * 5 * N3;
  for (int i = threadIdx.x; i < nvals; i += blockDim.x) {
    const int c = (i / N3) % 5;
    su[i] = T(U[base + i] - (c == 0 ? kp.rho_ref : (c == 4 ? kp.rhoE_ref : 0.0)));
    sy[i] = Y[base + i];
    sg[i] = T(0);
  }
  __syncthreads();
  adj_cell_terms<T, N, QC, QV, CB, GEO>(su, sy, sg, ar, tb, kp, ph, e0, nb);
  if constexpr (PAIR) {
    static_assert(S::CELL >= fbuf_per_cell<N>(), "adjoint arena too small for face shares");
    const T* F = static_cast<const T*>(kp.fbuf) + (size_t)e0 * fbuf_per_cell<N>();
    __syncthreads();
    for (int i = threadIdx.x; i < nb * fbuf_per_cell<N>(); i += blockDim.x) ar[i] = F[i];
    __syncthreads();
    gather_face_shares<T, N>(sg, ar, tb, nb, CtaGroup());
    __syncthreads();
  } else {
  for (int d = 0; d < 3; ++d) {
    for (int s = 0; s < 2; ++s) {
      if (threadIdx.x < nb) {
        const int e = e0 + threadIdx.x;
        int c[3] = {e % kp.nc[0], (e / kp.nc[0]) % kp.nc[1], e / (kp.nc[0] * kp.nc[1])};
        c[d] += s ? 1 : -1;
        int w = 0;
        if (c[d] < 0 || c[d] >= kp.nc[d]) {
          if (kp.periodic[d])
            c[d] = (c[d] + kp.nc[d]) % kp.nc[d];
          else
            w = 1;
        }
        const int en = w ? -1 : c[0] + kp.nc[0] * (c[1] + kp.nc[1] * c[2]);
        nbi[threadIdx.x] = en;
        wall[threadIdx.x] = w;
        const double te = kp.tau[e];
        tau_f[threadIdx.x] = T(w ? te : fmax(te, kp.tau[en]));
      }
      __syncthreads();
      for (int i = threadIdx.x; i < nvals; i += blockDim.x) {
        const int e = i / (5 * N3);
        if (!wall[e]) {
          const size_t src = (size_t)nbi[e] * 5 * N3 + (i - e * 5 * N3);
          const int c = (i / N3) % 5;
          snu[i] = T(U[src] - (c == 0 ? kp.rho_ref : (c == 4 ? kp.rhoE_ref : 0.0)));
          sny[i] = Y[src];
        }
      }
      __syncthreads();
      if (d == 0) adj_face_terms<T, N, QC, QV, CB, 0, GEO>(su, sy, snu, sny, wall, nbi, tau_f, sg, ar, tb, kp, ph, e0, nb, s);
      if (d == 1) adj_face_terms<T, N, QC, QV, CB, 1, GEO>(su, sy, snu, sny, wall, nbi, tau_f, sg, ar, tb, kp, ph, e0, nb, s);
      if (d == 2) adj_face_terms<T, N, QC, QV, CB, 2, GEO>(su, sy, snu, sny, wall, nbi, tau_f, sg, ar, tb, kp, ph, e0, nb, s);
    }
  }
  }
  if (kp.out_mode == 2) {
    for (int i = threadIdx.x; i < nvals; i += blockDim.x) lamU[base + i] -= kp.dt * double(sg[i]);
  } else {
    for (int i = threadIdx.x; i < nvals; i += blockDim.x) G[base + i] = -sg[i];
  }
}

// Stage adjoint preparation: W = lam_dU + B lam_U -> Wout; lam_dU <- A W.
template <typename T>
__global__ void dg_adj_prep_kernel(size_t n, double A, double B, const double* __restrict__ lamU, T* lamdU,
                                   T* __restrict__ Wout) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const double W = double(lamdU[i]) + B * lamU[i];
    Wout[i] = T(W);
    lamdU[i] = T(A * W);
  }
}

template <typename T, int N, int QC, int QV, int GEO, bool PAIR>
int adj_launch_geo(const KParams& kp, const double* U, const void* Y, void* G, double* lamU, cudaStream_t st) {
  constexpr int CB = adj_cells_per_cta<T, N, QC, QV, PAIR>();
  constexpr size_t smem = adj_smem_bytes<T, N, QC, QV, CB, PAIR>();
  if (smem > 227 * 1024) return -2;
  auto k = dg_adj_kernel<T, N, QC, QV, CB, GEO, PAIR>;
  static bool attr[kMaxDevices] = {};
  if (smem_attr_once(k, smem, attr)) return -1;
  const int grid = (kp.Nc + CB - 1) / CB;
  k<<<grid, NT, smem, st>>>(kp, U, static_cast<const T*>(Y), static_cast<T*>(G), lamU);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

template <typename T, int N, int QC, int QV>
int adj_launch(const KParams& kp, const double* U, const void* Y, void* G, double* lamU, cudaStream_t st) {
  using F = Feat<N, QC, QV>;
  if constexpr (!F::adj || (sizeof(T) == 4 && !F::fp32)) {
    return -2;
  } else {
    if (kp.fbuf != nullptr) {
      if constexpr (F::faces) {
        if (kp.gcc == nullptr) return adj_launch_geo<T, N, QC, QV, GEO_AFFINE, true>(kp, U, Y, G, lamU, st);
        if constexpr (F::geo) return adj_launch_geo<T, N, QC, QV, GEO_STORED, true>(kp, U, Y, G, lamU, st);
      }
      return -2;
    }
    if (kp.gcc == nullptr) return adj_launch_geo<T, N, QC, QV, GEO_AFFINE, false>(kp, U, Y, G, lamU, st);
    if constexpr (F::geo) return adj_launch_geo<T, N, QC, QV, GEO_STORED, false>(kp, U, Y, G, lamU, st);
    return -2;
  }
}

template <typename T>
int adj_prep_launch(size_t n, double A, double B, const double* lamU, void* lamdU, void* W, cudaStream_t st) {
  dg_adj_prep_kernel<T><<<1024, 256, 0, st>>>(n, A, B, lamU, static_cast<T*>(lamdU), static_cast<T*>(W));
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace dgcns
