// Face-centric adjoint face terms: every face once, the shares of both cells into the face buffer
// ([Nc][6][2][5][N^2], the layout of the forward face kernel), added by the adjoint cell kernel.
//
// With n the own side's outward normal and Y^-, Y^+ the adjoint inputs (Y = M^{-1} W) of the two cells:
//   LLF:  the other cell's face term is -f(U^-, U^+; n) tested with V^+, so both terms together
//         transpose f once with the adjoint input Y^- - Y^+;
//   SIPG: the value terms likewise combine into one transpose with Y^- - Y^+; the two
//         -1/2 (grad V, F_v(U^±, (U^- - U^+) (x) n)) terms share the jump tensor but differ in the
//         state and the inverse Jacobian, and are transposed per side (sipg_pair_vjp).
// Per face point this costs 2 convective and 4 viscous flux transposes, against 4 and 6 per face side
// (8 and 12 per face) in the element-centric adjoint kernel.
#pragma once
#include "dg_adjoint.cuh"
#include "dg_faces.cuh"

namespace dgcns {

// SIPG face point, both sides: adjoint of val^- (and of val^+ = -val^-) through yvd = Y^- - Y^+,
// of the own gradient term through ybm (reference derivatives of Y^- at the point) and, unless at a
// wall, of the other side's gradient term through ybp.  Accumulates umb, Gmb, upb, Gpb.
template <typename T>
__device__ __forceinline__ void sipg_pair_vjp(const T um[5], const T Gm[5][3], const T up[5], const T Gp[5][3],
                                              const T n[3], const T Jm[9], const T Jp[9], T w, T tau,
                                              const T yvd[5], const T ybm[3][5], const T ybp[3][5], bool wall,
                                              const PhysT<T>& ph, T umb[5], T Gmb[5][3], T upb[5], T Gpb[5][3]) {
  T jmpb[5], Jg[5][3], Jgb[5][3], Fb[5][3];
#pragma unroll
  for (int c = 0; c < 5; ++c) {
    const T jmp = um[c] - up[c];
    jmpb[c] = w * tau * yvd[c];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      Jg[c][a] = jmp * n[a];
      Jgb[c][a] = T(0);
      Fb[c][a] = T(-0.5) * w * (Jm[a] * ybm[0][c] + Jm[3 + a] * ybm[1][c] + Jm[6 + a] * ybm[2][c]);
    }
  }
  visc_flux_vjp(um, Jg, Fb, ph, umb, Jgb);
  if (!wall) {
#pragma unroll
    for (int c = 0; c < 5; ++c)
#pragma unroll
      for (int a = 0; a < 3; ++a)
        Fb[c][a] = T(-0.5) * w * (Jp[a] * ybp[0][c] + Jp[3 + a] * ybp[1][c] + Jp[6 + a] * ybp[2][c]);
    visc_flux_vjp(up, Jg, Fb, ph, upb, Jgb);
  }
#pragma unroll
  for (int c = 0; c < 5; ++c) {
    jmpb[c] += Jgb[c][0] * n[0] + Jgb[c][1] * n[1] + Jgb[c][2] * n[2];
#pragma unroll
    for (int a = 0; a < 3; ++a) Fb[c][a] = T(-0.5) * w * yvd[c] * n[a];
  }
  visc_flux_vjp(um, Gm, Fb, ph, umb, Gmb);
  visc_flux_vjp(up, Gp, Fb, ph, upb, Gpb);
#pragma unroll
  for (int c = 0; c < 5; ++c) {
    umb[c] += jmpb[c];
    upb[c] -= jmpb[c];
  }
}

template <int N, int QC, int QV>
struct AdjPairSizes {
  static constexpr int N2 = N * N;
  static constexpr int LAYERS = 8 * 5 * N2;  // U-, dU-, U+, dU+, Y-, dY-, Y+, dY+
  static constexpr int CONV = 3 * 5 * QC * N + 3 * 5 * QC * QC + 5 * N2;
  static constexpr int VISC = 8 * 5 * N * QV + 16 * 5 * QV * QV;
  static constexpr int ARENA = CONV > VISC ? CONV : VISC;
  static constexpr int PER_FACE = LAYERS + ARENA + 2 * 5 * N2;
};

template <typename T, int N, int QC, int QV, int CB, int d, int GEO>
__device__ void adj_face_pair_terms(const double* __restrict__ U, const T* __restrict__ Y, const int* eo,
                                    const int* en, const T* tau_f, T* lay, T* ar, T* lcm, T* lcp, const Tab<T>& tb,
                                    const KParams& kp, const PhysT<T>& ph, int nb, int s, T* __restrict__ FB) {
  constexpr int N2 = N * N, N3 = N * N * N;
  constexpr int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
  const int f = 2 * d + s, fo = 2 * d + (1 - s);
  const int idm = s ? N - 1 : 0, idp = s ? 0 : N - 1;
  const T* dlm = s ? tb.dl1 : tb.dl0;
  const T* dlp = s ? tb.dl0 : tb.dl1;
  const int nbl = nb * 5;
  constexpr int LS = CB * 5 * N2;  // one layer
  auto LAY = [&](int r) { return lay + r * LS; };

  // trace layers of both cells, read along the normal lines from global memory
  for (int idx = threadIdx.x; idx < nbl * N2; idx += blockDim.x) {
    const int ec = idx / N2, j = idx - ec * N2, e = ec / 5, c = ec - 5 * e;
    const int j1 = j % N, j2 = j / N;
    const double ref = c == 0 ? kp.rho_ref : (c == 4 ? kp.rhoE_ref : 0.0);
    const size_t om = ((size_t)eo[e] * 5 + c) * N3;
    T du = T(0), dy = T(0);
#pragma unroll
    for (int i = 0; i < N; ++i) {
      const int q = face_node<N>(d, i, j1, j2);
      du += dlm[i] * T(U[om + q] - ref);
      dy += dlm[i] * Y[om + q];
    }
    const int qm = face_node<N>(d, idm, j1, j2);
    LAY(0)[idx] = T(U[om + qm] - ref);
    LAY(1)[idx] = du;
    LAY(4)[idx] = Y[om + qm];
    LAY(5)[idx] = dy;
    if (en[e] < 0) {
      LAY(2)[idx] = LAY(3)[idx] = LAY(6)[idx] = LAY(7)[idx] = T(0);
    } else {
      const size_t op = ((size_t)en[e] * 5 + c) * N3;
      T dun = T(0), dyn = T(0);
#pragma unroll
      for (int i = 0; i < N; ++i) {
        const int q = face_node<N>(d, i, j1, j2);
        dun += dlp[i] * T(U[op + q] - ref);
        dyn += dlp[i] * Y[op + q];
      }
      const int qp = face_node<N>(d, idp, j1, j2);
      LAY(2)[idx] = T(U[op + qp] - ref);
      LAY(3)[idx] = dun;
      LAY(6)[idx] = Y[op + qp];
      LAY(7)[idx] = dyn;
    }
  }
  __syncthreads();

  if (kp.conv) {
    constexpr int P = QC * QC;
    T* Tm = ar;
    T* T1 = Tm + CB * 5 * QC * N;
    T* T2 = T1 + CB * 5 * QC * N;
    T* Pm = T2 + CB * 5 * QC * N;
    T* Pp = Pm + CB * 5 * P;
    T* Py = Pp + CB * 5 * P;
    T* Ldy = Py + CB * 5 * P;
    for (int idx = threadIdx.x; idx < nbl * N2; idx += blockDim.x) Ldy[idx] = LAY(4)[idx] - LAY(6)[idx];
    __syncthreads();
    sweep<T, 0, N, N, 1, QC, 1, false>(LAY(0), Tm, tb.eSc, nbl);
    sweep<T, 0, N, N, 1, QC, 1, false>(LAY(2), T1, tb.eSc, nbl);
    sweep<T, 0, N, N, 1, QC, 1, false>(Ldy, T2, tb.eSc, nbl);
    __syncthreads();
    sweep<T, 1, QC, N, 1, QC, 1, false>(Tm, Pm, tb.eSc, nbl);
    sweep<T, 1, QC, N, 1, QC, 1, false>(T1, Pp, tb.eSc, nbl);
    sweep<T, 1, QC, N, 1, QC, 1, false>(T2, Py, tb.eSc, nbl);
    __syncthreads();
    for (int idx = threadIdx.x; idx < nb * P; idx += blockDim.x) {
      const int e = idx / P, p = idx - e * P;
      const int o = e * 5 * P + p;
      const bool wall = en[e] < 0;
      T Jm[9], Jp[9], nv[3], w;
      face_geo<T, GEO, d>(kp, kp.gfc, P, (size_t)eo[e], wall ? 0 : (size_t)en[e], f, fo, p,
                          tb.wc[p % QC] * tb.wc[p / QC], wall, s, Jm, Jp, nv, w);
      T um[5], up[5], yd[5], umb[5], upb[5];
#pragma unroll
      for (int c = 0; c < 5; ++c) {
        um[c] = Pm[o + c * P];
        up[c] = Pp[o + c * P];
        yd[c] = Py[o + c * P];
        umb[c] = T(0);
        upb[c] = T(0);
      }
      if (wall) wall_ghost(um, ph, up);
      llf_vjp(um, up, nv, w, yd, ph, umb, upb);
      if (wall) {
        wall_ghost_vjp(um, upb, ph, umb);
#pragma unroll
        for (int c = 0; c < 5; ++c) upb[c] = T(0);
      }
#pragma unroll
      for (int c = 0; c < 5; ++c) {
        Pm[o + c * P] = umb[c];
        Pp[o + c * P] = upb[c];
      }
    }
    __syncthreads();
    sweep<T, 1, QC, QC, 1, N, 1, false>(Pm, Tm, tb.eScT, nbl);
    sweep<T, 1, QC, QC, 1, N, 1, false>(Pp, T1, tb.eScT, nbl);
    __syncthreads();
    sweep<T, 0, QC, N, 1, N, 1, false>(Tm, lcm, tb.eScT, nbl);
    sweep<T, 0, QC, N, 1, N, 1, false>(T1, lcp, tb.eScT, nbl);
    __syncthreads();
  } else {
    for (int idx = threadIdx.x; idx < nbl * N2; idx += blockDim.x) lcm[idx] = lcp[idx] = T(0);
  }

  if (kp.visc) {
    constexpr int P = QV * QV;
    constexpr int TS = CB * 5 * N * QV, PS = CB * 5 * P;
    T* Tt = ar;            // 8 temporaries
    T* Pt = Tt + 8 * TS;   // 16 point arrays: 4 r + {value, t1, t2, d}, r: U-, U+, Y-, Y+
    auto PT = [&](int k) { return Pt + k * PS; };
#pragma unroll 1
    for (int r = 0; r < 8; ++r) sweep<T, 0, N, N, 1, QV, 1, false>(LAY(r), Tt + r * TS, tb.eSv, nbl);
    __syncthreads();
    // layer r: state r/2 (U-, U+, Y-, Y+), value (even r) or normal derivative (odd r)
#pragma unroll 1
    for (int r = 0; r < 8; ++r)
      sweep<T, 1, QV, N, 1, QV, 1, false>(Tt + r * TS, PT(4 * (r / 2) + ((r & 1) ? 3 : 0)), tb.eSv, nbl);
    __syncthreads();
#pragma unroll 1
    for (int q = 0; q < 4; ++q) {
      sweep<T, 0, QV, QV, 1, QV, -1, false>(PT(4 * q), PT(4 * q + 1), tb.eDv, nbl);
      sweep<T, 1, QV, QV, 1, QV, -1, false>(PT(4 * q), PT(4 * q + 2), tb.eDv, nbl);
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < nb * P; idx += blockDim.x) {
      const int e = idx / P, p = idx - e * P;
      const int o = e * 5 * P + p;
      const bool wall = en[e] < 0;
      T Jm[9], Jp[9], nv[3], w;
      face_geo<T, GEO, d>(kp, kp.gfv, P, (size_t)eo[e], wall ? 0 : (size_t)en[e], f, fo, p,
                          tb.wv[p % QV] * tb.wv[p / QV], wall, s, Jm, Jp, nv, w);
      const T tau = tau_f[e];
      int slot[3];
      slot[t1] = 1;
      slot[t2] = 2;
      slot[d] = 3;
      T um[5], up[5], Gm[5][3], Gp[5][3], yvd[5], ybm[3][5], ybp[3][5];
#pragma unroll
      for (int c = 0; c < 5; ++c) {
        um[c] = PT(0)[o + c * P];
        up[c] = PT(4)[o + c * P];
        yvd[c] = PT(8)[o + c * P] - PT(12)[o + c * P];
        T gm[3], gp[3];
#pragma unroll
        for (int b = 0; b < 3; ++b) {
          gm[b] = PT(slot[b])[o + c * P];
          gp[b] = PT(4 + slot[b])[o + c * P];
          ybm[b][c] = PT(8 + slot[b])[o + c * P];
          ybp[b][c] = PT(12 + slot[b])[o + c * P];
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          Gm[c][a] = Jm[a] * gm[0] + Jm[3 + a] * gm[1] + Jm[6 + a] * gm[2];
          Gp[c][a] = Jp[a] * gp[0] + Jp[3 + a] * gp[1] + Jp[6 + a] * gp[2];
        }
      }
      if (wall) {
        wall_ghost(um, ph, up);
#pragma unroll
        for (int c = 0; c < 5; ++c)
#pragma unroll
          for (int a = 0; a < 3; ++a) Gp[c][a] = Gm[c][a];
      }
      T umb[5], Gmb[5][3], upb[5], Gpb[5][3];
#pragma unroll
      for (int c = 0; c < 5; ++c) {
        umb[c] = upb[c] = T(0);
#pragma unroll
        for (int a = 0; a < 3; ++a) Gmb[c][a] = Gpb[c][a] = T(0);
      }
      sipg_pair_vjp(um, Gm, up, Gp, nv, Jm, Jp, w, tau, yvd, ybm, ybp, wall, ph, umb, Gmb, upb, Gpb);
      if (wall) {
        wall_ghost_vjp(um, upb, ph, umb);
#pragma unroll
        for (int c = 0; c < 5; ++c) {
          upb[c] = T(0);
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            Gmb[c][a] += Gpb[c][a];
            Gpb[c][a] = T(0);
          }
        }
      }
#pragma unroll
      for (int c = 0; c < 5; ++c) {
        PT(0)[o + c * P] = umb[c];
        PT(4)[o + c * P] = upb[c];
#pragma unroll
        for (int b = 0; b < 3; ++b) {
          PT(slot[b])[o + c * P] = Jm[3 * b] * Gmb[c][0] + Jm[3 * b + 1] * Gmb[c][1] + Jm[3 * b + 2] * Gmb[c][2];
          PT(4 + slot[b])[o + c * P] = Jp[3 * b] * Gpb[c][0] + Jp[3 * b + 1] * Gpb[c][1] + Jp[3 * b + 2] * Gpb[c][2];
        }
      }
    }
    __syncthreads();
    // tests of both sides: value + tangential gradients, then the normal gradient
    sweep<T, 0, QV, QV, 1, QV, -1, true>(PT(1), PT(0), tb.eDvT, nbl);
    sweep<T, 0, QV, QV, 1, QV, -1, true>(PT(5), PT(4), tb.eDvT, nbl);
    __syncthreads();
    sweep<T, 1, QV, QV, 1, QV, -1, true>(PT(2), PT(0), tb.eDvT, nbl);
    sweep<T, 1, QV, QV, 1, QV, -1, true>(PT(6), PT(4), tb.eDvT, nbl);
    __syncthreads();
    sweep<T, 1, QV, QV, 1, N, 1, false>(PT(0), Tt, tb.eSvT, nbl);
    sweep<T, 1, QV, QV, 1, N, 1, false>(PT(4), Tt + TS, tb.eSvT, nbl);
    sweep<T, 1, QV, QV, 1, N, 1, false>(PT(3), Tt + 2 * TS, tb.eSvT, nbl);
    sweep<T, 1, QV, QV, 1, N, 1, false>(PT(7), Tt + 3 * TS, tb.eSvT, nbl);
    __syncthreads();
    sweep<T, 0, QV, N, 1, N, 1, false>(Tt, LAY(0), tb.eSvT, nbl);
    sweep<T, 0, QV, N, 1, N, 1, false>(Tt + TS, LAY(2), tb.eSvT, nbl);
    sweep<T, 0, QV, N, 1, N, 1, false>(Tt + 2 * TS, LAY(1), tb.eSvT, nbl);
    sweep<T, 0, QV, N, 1, N, 1, false>(Tt + 3 * TS, LAY(3), tb.eSvT, nbl);
    __syncthreads();
  }
  for (int idx = threadIdx.x; idx < nbl * N2; idx += blockDim.x) {
    const int ec = idx / N2, j = idx - ec * N2, e = ec / 5, c = ec - 5 * e;
    T* po = FB + ((size_t)eo[e] * 6 + f) * 10 * N2 + c * N2 + j;
    po[0] = lcm[idx] + (kp.visc ? LAY(0)[idx] : T(0));
    po[5 * N2] = kp.visc ? LAY(1)[idx] : T(0);
    if (en[e] >= 0) {
      T* pn = FB + ((size_t)en[e] * 6 + fo) * 10 * N2 + c * N2 + j;
      pn[0] = lcp[idx] + (kp.visc ? LAY(2)[idx] : T(0));
      pn[5 * N2] = kp.visc ? LAY(3)[idx] : T(0);
    }
  }
}

// Faces per CTA of the adjoint face kernel (<= 8, ~112 KB of shared memory).
template <typename T, int N, int QC, int QV>
constexpr int adj_faces_per_cta() {
  constexpr int per_face = AdjPairSizes<N, QC, QV>::PER_FACE * (int)sizeof(T) + 16;
  constexpr int cb = (112 * 1024 - table_elems<N, QC, QV>() * (int)sizeof(T)) / per_face;
  return cb < 1 ? 1 : (cb > 8 ? 8 : cb);
}

template <typename T, int N, int QC, int QV, int CB>
constexpr size_t adj_face_smem_bytes() {
  return ((size_t)table_elems<N, QC, QV>() + (size_t)CB * AdjPairSizes<N, QC, QV>::PER_FACE + CB) * sizeof(T) +
         2 * CB * sizeof(int) + 64;
}

// Grid as the forward face kernel: blockIdx.y = d; upper faces of every cell, then lower walls.
template <typename T, int N, int QC, int QV, int CB, int GEO>
__global__ void __launch_bounds__(NT) dg_adj_face_kernel(const KParams kp, const double* __restrict__ U,
                                                         const T* __restrict__ Y, T* __restrict__ FB) {
  using S = AdjPairSizes<N, QC, QV>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* stab = reinterpret_cast<T*>(smem_raw);
  T* lay = stab + table_elems<N, QC, QV>();
  T* ar = lay + CB * S::LAYERS;
  T* lcm = ar + CB * S::ARENA;
  T* lcp = lcm + CB * 5 * S::N2;
  T* tau_f = lcp + CB * 5 * S::N2;
  int* eo = reinterpret_cast<int*>(tau_f + CB);
  int* en = eo + CB;

  const int d = blockIdx.y;
  const int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
  const int nstd = (kp.Nc + CB - 1) / CB;
  int s, i0, nitems;
  if ((int)blockIdx.x < nstd) {
    s = 1;
    i0 = blockIdx.x * CB;
    nitems = kp.Nc;
  } else {
    if (kp.periodic[d]) return;
    s = 0;
    i0 = (blockIdx.x - nstd) * CB;
    nitems = kp.nc[t1] * kp.nc[t2];
    if (i0 >= nitems) return;
  }
  const int nb = min(CB, nitems - i0);
  const Tab<T> tb = load_tables<T, N, QC, QV>(static_cast<const T*>(kp.tables), stab);
  const PhysT<T> ph = make_phys<T>(kp);
  if ((int)threadIdx.x < nb) {
    const int i = i0 + threadIdx.x;
    int c[3];
    if (s == 1) {
      c[0] = i % kp.nc[0];
      c[1] = (i / kp.nc[0]) % kp.nc[1];
      c[2] = i / (kp.nc[0] * kp.nc[1]);
    } else {
      c[d] = 0;
      c[t1] = i % kp.nc[t1];
      c[t2] = i / kp.nc[t1];
    }
    const int e = c[0] + kp.nc[0] * (c[1] + kp.nc[1] * c[2]);
    c[d] += s ? 1 : -1;
    int w = 0;
    if (c[d] < 0 || c[d] >= kp.nc[d]) {
      if (kp.periodic[d])
        c[d] = (c[d] + kp.nc[d]) % kp.nc[d];
      else
        w = 1;
    }
    const int n = w ? -1 : c[0] + kp.nc[0] * (c[1] + kp.nc[1] * c[2]);
    eo[threadIdx.x] = e;
    en[threadIdx.x] = n;
    const double te = kp.tau[e];
    tau_f[threadIdx.x] = T(w ? te : fmax(te, kp.tau[n]));
  }
  __syncthreads();
  if (d == 0)
    adj_face_pair_terms<T, N, QC, QV, CB, 0, GEO>(U, Y, eo, en, tau_f, lay, ar, lcm, lcp, tb, kp, ph, nb, s, FB);
  else if (d == 1)
    adj_face_pair_terms<T, N, QC, QV, CB, 1, GEO>(U, Y, eo, en, tau_f, lay, ar, lcm, lcp, tb, kp, ph, nb, s, FB);
  else
    adj_face_pair_terms<T, N, QC, QV, CB, 2, GEO>(U, Y, eo, en, tau_f, lay, ar, lcm, lcp, tb, kp, ph, nb, s, FB);
}

template <typename T, int N, int QC, int QV, int GEO>
int launch_adj_faces(const KParams& kp, const double* U, const void* Y, void* FB, cudaStream_t st) {
  constexpr int CB = adj_faces_per_cta<T, N, QC, QV>();
  constexpr size_t smem = adj_face_smem_bytes<T, N, QC, QV, CB>();
  if (smem > 227 * 1024) return -2;
  auto k = dg_adj_face_kernel<T, N, QC, QV, CB, GEO>;
  static bool attr[kMaxDevices] = {};
  if (smem_attr_once(k, smem, attr)) return -1;
  int extra = 0;
  for (int d = 0; d < 3; ++d) {
    if (kp.periodic[d]) continue;
    const int plane = kp.nc[d == 0 ? 1 : 0] * kp.nc[d == 2 ? 1 : 2];
    const int nbk = (plane + CB - 1) / CB;
    if (nbk > extra) extra = nbk;
  }
  const dim3 grid((kp.Nc + CB - 1) / CB + extra, 3);
  k<<<grid, NT, smem, st>>>(kp, U, static_cast<const T*>(Y), static_cast<T*>(FB));
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

template <typename T, int N, int QC, int QV>
int adj_faces_dispatch(const KParams& kp, const double* U, const void* Y, void* FB, cudaStream_t st) {
  using F = Feat<N, QC, QV>;
  if constexpr (!F::adj || !F::faces || (sizeof(T) == 4 && !F::fp32)) {
    return -2;
  } else {
    if (kp.gcc == nullptr) return launch_adj_faces<T, N, QC, QV, GEO_AFFINE>(kp, U, Y, FB, st);
    if constexpr (F::geo) return launch_adj_faces<T, N, QC, QV, GEO_STORED>(kp, U, Y, FB, st);
    return -2;
  }
}

}  // namespace dgcns
