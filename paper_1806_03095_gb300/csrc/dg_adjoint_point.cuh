// Transposed pointwise Jacobians (vector-Jacobian products) of the flux
// routines of dg_kernels.cuh, hand-derived in reverse order of the forward
// statements.  Every function ACCUMULATES into its adjoint outputs.
#pragma once
#include "dg_kernels.cuh"

namespace dgcns {

// ub += (dF_c/du)^T Fb for the convective flux in all three directions,
// Fb[a][c] = adjoint of F_c[c][a] (deviation form: pressure deviation dp).
template <typename T>
__device__ __forceinline__ void conv_flux_vjp(const T u[5], const T Fb[3][5], const PhysT<T>& ph, T ub[5]) {
  const T rinv = T(1) / (ph.rho_r + u[0]);
  const T m[3] = {u[1], u[2], u[3]};
  const T v[3] = {m[0] * rinv, m[1] * rinv, m[2] * rinv};
  const T msq = m[0] * m[0] + m[1] * m[1] + m[2] * m[2];
  const T dp = ph.gm1 * (u[4] - T(0.5) * rinv * msq);
  T vb[3] = {T(0), T(0), T(0)}, mb[3] = {T(0), T(0), T(0)};
  T dpb = T(0), u4b = T(0), rinvb = T(0);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    mb[a] += Fb[a][0];  // F[0][a] = m_a
#pragma unroll
    for (int i = 0; i < 3; ++i) {  // F[1+i][a] = m_i v_a + dp delta_ia
      mb[i] += Fb[a][1 + i] * v[a];
      vb[a] += Fb[a][1 + i] * m[i];
    }
    dpb += Fb[a][1 + a];
    // F[4][a] = (H_r + rhoE' + dp) v_a
    u4b += Fb[a][4] * v[a];
    dpb += Fb[a][4] * v[a];
    vb[a] += Fb[a][4] * (ph.H_r + u[4] + dp);
  }
  // dp = (gamma-1)(rhoE' - |m|^2 rinv / 2)
  u4b += ph.gm1 * dpb;
#pragma unroll
  for (int i = 0; i < 3; ++i) mb[i] -= ph.gm1 * rinv * m[i] * dpb;
  rinvb -= T(0.5) * ph.gm1 * msq * dpb;
  // v = m rinv
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    mb[i] += vb[i] * rinv;
    rinvb += vb[i] * m[i];
  }
  ub[0] -= rinv * rinv * rinvb;
  ub[1] += mb[0];
  ub[2] += mb[1];
  ub[3] += mb[2];
  ub[4] += u4b;
}

// ub += (dF_v/du)^T Fb, Gb += (dF_v/dG)^T Fb for F_v(u, G) (Fb[c][a], Gb[c][a]).
template <typename T>
__device__ __forceinline__ void visc_flux_vjp(const T u[5], const T G[5][3], const T Fb[5][3], const PhysT<T>& ph,
                                              T ub[5], T Gb[5][3]) {
  const T rinv = T(1) / (ph.rho_r + u[0]);
  const T v[3] = {u[1] * rinv, u[2] * rinv, u[3] * rinv};
  const T E = (ph.rhoE_r + u[4]) * rinv;
  T gu[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) gu[i][j] = (G[1 + i][j] - v[i] * G[0][j]) * rinv;
  const T div = gu[0][0] + gu[1][1] + gu[2][2];
  const T twothird = T(2) / T(3);
  T gub[3][3] = {{T(0), T(0), T(0)}, {T(0), T(0), T(0)}, {T(0), T(0), T(0)}};
  T vb[3] = {T(0), T(0), T(0)};
  T Eb = T(0), rinvb = T(0), divb = T(0);
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const T tvb = Fb[4][j];           // F[4][j] = tv_j + lam_cv gTcv_j
    const T gTb = ph.lam_cv * Fb[4][j];
    // gTcv_j = gE_j - sum_i v_i gu_ij
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      vb[i] -= gTb * gu[i][j];
      gub[i][j] -= gTb * v[i];
    }
    // gE_j = (G[4][j] - E G[0][j]) rinv
    Gb[4][j] += gTb * rinv;
    Eb -= gTb * G[0][j] * rinv;
    Gb[0][j] -= gTb * E * rinv;
    rinvb += gTb * (G[4][j] - E * G[0][j]);
    // tv_j = sum_i tau_ij v_i ; F[1+i][j] = tau_ij
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      T tij = ph.mu * (gu[i][j] + gu[j][i]);
      if (i == j) tij -= ph.mu * twothird * div;
      const T taub = tvb * v[i] + Fb[1 + i][j];
      vb[i] += tvb * tij;
      // tau_ij = mu (gu_ij + gu_ji) - delta_ij 2/3 mu div
      gub[i][j] += ph.mu * taub;
      gub[j][i] += ph.mu * taub;
      if (i == j) divb -= ph.mu * twothird * taub;
    }
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) gub[i][i] += divb;
  // gu_ij = (G[1+i][j] - v_i G[0][j]) rinv
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      Gb[1 + i][j] += gub[i][j] * rinv;
      vb[i] -= gub[i][j] * G[0][j] * rinv;
      Gb[0][j] -= gub[i][j] * v[i] * rinv;
      rinvb += gub[i][j] * (G[1 + i][j] - v[i] * G[0][j]);
    }
  // E = (rhoE_r + rhoE') rinv
  ub[4] += Eb * rinv;
  rinvb += Eb * (ph.rhoE_r + u[4]);
  // v_i = m_i rinv
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    ub[1 + i] += vb[i] * rinv;
    rinvb += vb[i] * u[1 + i];
  }
  ub[0] -= rinv * rinv * rinvb;
}

// ub += lb d(lambda)/du, lambda = |m|/rho + sqrt(|gamma p / rho|)
template <typename T>
__device__ __forceinline__ void wave_speed_vjp(const T u[5], T lb, const PhysT<T>& ph, T ub[5]) {
  const T rinv = T(1) / (ph.rho_r + u[0]);
  const T msq = u[1] * u[1] + u[2] * u[2] + u[3] * u[3];
  const T mn = sqrt(msq);
  const T dp = ph.gm1 * (u[4] - T(0.5) * rinv * msq);
  const T P = ph.p_r + dp;
  const T s = ph.gamma * P * rinv;
  const T c = sqrt(fabs(s));
  T rinvb = lb * mn;
  if (mn > T(0)) {
#pragma unroll
    for (int i = 0; i < 3; ++i) ub[1 + i] += lb * rinv * u[1 + i] / mn;
  }
  if (c > T(0)) {
    const T sb = lb * (s >= T(0) ? T(1) : T(-1)) / (T(2) * c);
    const T Pb = sb * ph.gamma * rinv;
    rinvb += sb * ph.gamma * P;
    ub[4] += ph.gm1 * Pb;
#pragma unroll
    for (int i = 0; i < 3; ++i) ub[1 + i] -= ph.gm1 * rinv * u[1 + i] * Pb;
    rinvb -= T(0.5) * ph.gm1 * msq * Pb;
  }
  ub[0] -= rinv * rinv * rinvb;
}

template <typename T>
__device__ __forceinline__ T wave_speed(const T u[5], const PhysT<T>& ph) {
  const T rinv = T(1) / (ph.rho_r + u[0]);
  const T msq = u[1] * u[1] + u[2] * u[2] + u[3] * u[3];
  const T dp = ph.gm1 * (u[4] - T(0.5) * rinv * msq);
  return sqrt(msq) * rinv + sqrt(fabs(ph.gamma * (ph.p_r + dp) * rinv));
}

// umb += (d ghost / d um)^T upb for the wall state of wall_ghost().
template <typename T>
__device__ __forceinline__ void wall_ghost_vjp(const T um[5], const T upb[5], const PhysT<T>& ph, T umb[5]) {
  const T rinv = T(1) / (ph.rho_r + um[0]);
  const T msq = um[1] * um[1] + um[2] * um[2] + um[3] * um[3];
  // up4 = cvTw2 um0 - um4 + |m|^2 rinv
  umb[0] += upb[0] + upb[4] * (ph.cvTw2 - msq * rinv * rinv);
#pragma unroll
  for (int i = 0; i < 3; ++i) umb[1 + i] += -upb[1 + i] + upb[4] * T(2) * um[1 + i] * rinv;
  umb[4] -= upb[4];
}

// Local Lax--Friedrichs face point: flux[c] = w (1/2 sum_a (F(um)+F(up))[c][a] n_a + Lambda/2 (um-up)_c)
// with Lambda = max(lambda(um), lambda(up)).  Given fb = adjoint of flux.
template <typename T>
__device__ __forceinline__ void llf_vjp(const T um[5], const T up[5], const T n[3], T w, const T fb[5],
                                        const PhysT<T>& ph, T umb[5], T upb[5]) {
  T Fb[3][5];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int c = 0; c < 5; ++c) Fb[a][c] = T(0.5) * w * fb[c] * n[a];
  conv_flux_vjp(um, Fb, ph, umb);
  conv_flux_vjp(up, Fb, ph, upb);
  const T lm = wave_speed(um, ph), lp = wave_speed(up, ph);
  const T lam = lm > lp ? lm : lp;  // same branch as the forward flux (ties: the up side)
  T lamb = T(0);
#pragma unroll
  for (int c = 0; c < 5; ++c) {
    umb[c] += T(0.5) * w * lam * fb[c];
    upb[c] -= T(0.5) * w * lam * fb[c];
    lamb += T(0.5) * w * fb[c] * (um[c] - up[c]);
  }
  if (lm > lp)
    wave_speed_vjp(um, lamb, ph, umb);
  else
    wave_speed_vjp(up, lamb, ph, upb);
}

// Viscous face point of one side's face term (own side "m"):
//   val[c] = -w (1/2 sum_a (F_v(um,Gm) + F_v(up,Gp))[c][a] n_a - tau (um - up)_c)   tested with V
//   Ft_b[c] = -1/2 w sum_a Jm[b][a] F_v(um, (um - up) (x) n)[c][a]                 tested with d_b V
// Given yv (adjoint of val) and yb[b] (adjoint of Ft_b), accumulate umb, Gmb, upb, Gpb (physical gradients).
template <typename T>
__device__ __forceinline__ void sipg_vjp(const T um[5], const T Gm[5][3], const T up[5], const T Gp[5][3],
                                         const T n[3], const T Jm[9], T w, T tau, const T yv[5], const T yb[3][5],
                                         const PhysT<T>& ph, T umb[5], T Gmb[5][3], T upb[5], T Gpb[5][3]) {
  T jmp[5], jmpb[5];
  T Jg[5][3], Jgb[5][3], Fb[5][3];
#pragma unroll
  for (int c = 0; c < 5; ++c) {
    jmp[c] = um[c] - up[c];
    jmpb[c] = w * tau * yv[c];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      Jg[c][a] = jmp[c] * n[a];
      Jgb[c][a] = T(0);
      Fb[c][a] = T(-0.5) * w * (Jm[a] * yb[0][c] + Jm[3 + a] * yb[1][c] + Jm[6 + a] * yb[2][c]);
    }
  }
  visc_flux_vjp(um, Jg, Fb, ph, umb, Jgb);
#pragma unroll
  for (int c = 0; c < 5; ++c) {
    jmpb[c] += Jgb[c][0] * n[0] + Jgb[c][1] * n[1] + Jgb[c][2] * n[2];
#pragma unroll
    for (int a = 0; a < 3; ++a) Fb[c][a] = T(-0.5) * w * yv[c] * n[a];
  }
  visc_flux_vjp(um, Gm, Fb, ph, umb, Gmb);
  visc_flux_vjp(up, Gp, Fb, ph, upb, Gpb);
#pragma unroll
  for (int c = 0; c < 5; ++c) {
    umb[c] += jmpb[c];
    upb[c] -= jmpb[c];
  }
}

}  // namespace dgcns
