// Face-centric organisation of the face integrals (Sec. 2.2 loops over faces once): one kernel
// evaluates every face of the mesh once, for both adjacent cells, and writes each cell's share to a
// face buffer; the cell kernel then adds the 6 shares of each cell to its residual (no atomics,
// every (cell, face) slot has exactly one writer).
//
// Both sides of an interior face share the interpolated traces, the numerical fluxes and the
// tangential derivatives.  With n = n^- the own side's outward normal:
//   LLF:   (V^+, F*.n^+) = -(V^-, F*.n^-) at the same points, so the neighbour's convective share is
//          the negated own test;
//   SIPG:  Q*.n^+ = -Q*.n^-, so the value tests differ in sign only;
//   -1/2 (grad V, F_v(U, [[U]])):  [[U]] = (U^- - U^+) (x) n^- on both sides, but F_v is taken at
//          each side's own trace (U^- and U^+), so this term is evaluated per side.
// Shares, per cell and face f = 2d + s, in the face buffer [Nc][6][2][5][N^2]: L (coefficients of the
// face-layer nodes, i = 0 or N-1 along d) and D (coefficients of dV/dxi_d at the face, distributed
// along the normal lines with l_i'(face)).
#pragma once
#include "dg_kernels.cuh"

namespace dgcns {

template <int N>
constexpr int fbuf_per_cell() {
  return 6 * 2 * 5 * N * N;
}

// One face per item: own cell eo[b] (side s of its face), other cell en[b] (-1: wall, ghost state).
// lay: 4 trace layers [CB][5][N^2] (own values, own normal derivatives, other values, other normal
// derivatives), read along the normal lines from global memory (the deviation state Ud when given,
// else U - U_ref); lc: [CB][5][N^2] scratch; fa: face arena.
// Rotated-frame meshes (oc != nullptr): the other cell is read through its orientation code oc[b] as if
// it were aligned with the own cell, the face is evaluated in the own cell's frame, and the other cell's
// shares go to the face and node positions of its own frame (frame_facing), its normal-derivative share
// negated where its normal axis is reflected.
template <typename T, int N, int QC, int QV, int CB, int d, int GEO, class G = CtaGroup>
__device__ void face_pair_terms(const double* __restrict__ U, const T* __restrict__ Ud, const int* eo, const int* en,
                                const T* tau_f, T* lay, T* fa, T* lc, const Tab<T>& tb, const KParams& kp,
                                const PhysT<T>& ph, int nb, int s, T* __restrict__ FB, G grp = G(),
                                const T* sx = nullptr, const T* sxn = nullptr, T* go = nullptr,
                                const int* oc = nullptr) {
  const int f = 2 * d + s, fo = 2 * d + (1 - s);
  constexpr int N2 = N * N, N3 = N * N * N;
  constexpr int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
  const KConst<T>& kc = kconst<T>(kp);
  const T hinv[3] = {kc.hinv[0], kc.hinv[1], kc.hinv[2]};
  const T area = kc.area[d];
  const T sgn = s ? T(1) : T(-1);
  const int idm = s ? N - 1 : 0, idp = s ? 0 : N - 1;
  const T* dlm = s ? tb.dl1 : tb.dl0;
  const T* dlp = s ? tb.dl0 : tb.dl1;
  const int nbl = nb * 5;
  T* Lm = lay;  // own face values
  T* Dm = Lm + CB * 5 * N2;  // own normal derivatives
  T* Lp = Dm + CB * 5 * N2;  // other values
  T* Dp = Lp + CB * 5 * N2;  // other normal derivatives

  for (int idx = grp.rank(); idx < nbl * N2; idx += grp.size()) {
    const int ec = idx / N2, j = idx - ec * N2, e = ec / 5, c = ec - 5 * e;
    const int j1 = j % N, j2 = j / N;
    const double dref = c == 0 ? kp.rho_ref : (c == 4 ? kp.rhoE_ref : 0.0);
    const size_t om = ((size_t)eo[e] * 5 + c) * N3;
    T dn = T(0), vm = T(0);
#pragma unroll
    for (int i = 0; i < N; ++i) {
      const int q = face_node<N>(d, i, j1, j2);
      const T v = Ud ? Ud[om + q] : T(U[om + q] - dref);
      dn += dlm[i] * v;
      if (i == idm) vm = v;
    }
    Lm[idx] = vm;
    Dm[idx] = dn;
    if (en[e] < 0) {
      Lp[idx] = T(0);
      Dp[idx] = T(0);
    } else {
      const size_t op = ((size_t)en[e] * 5 + c) * N3;
      // the normal line through face node j; on rotated-frame meshes it is a line of the other cell too,
      // at a constant stride (+-1, +-N or +-N^2) from its reoriented first node
      int q0 = face_node<N>(d, 0, j1, j2), qs = face_node<N>(d, 1, j1, j2) - q0;
      if (oc) {
        const int r0 = frame_node<N>(oc[e], q0);
        qs = frame_node<N>(oc[e], q0 + qs) - r0;
        q0 = r0;
      }
      T dq = T(0), vp = T(0);
#pragma unroll
      for (int i = 0; i < N; ++i) {
        const int q = q0 + i * qs;
        const T v = Ud ? Ud[op + q] : T(U[op + q] - dref);
        dq += dlp[i] * v;
        if (i == idp) vp = v;
      }
      Lp[idx] = vp;
      Dp[idx] = dq;
    }
  }
  grp.sync();

  if (kp.conv) {
    constexpr int P = QC * QC;
    if (GEO == GEO_FLY) fill_face_geo<T, N, QC, CB, d>(sx, s, fa, tb.eSc, tb.eDc, dlm, go, nb, grp);
    T* Tm = fa;
    T* Tp = Tm + CB * 5 * QC * N;
    T* Um = Tp + CB * 5 * QC * N;
    T* Up = Um + CB * 5 * P;
    grp.sync();
    sweep<T, 0, N, N, 1, QC, 1, false>(Lm, Tm, tb.eSc, nbl, grp);
    sweep<T, 0, N, N, 1, QC, 1, false>(Lp, Tp, tb.eSc, nbl, grp);
    grp.sync();
    sweep<T, 1, QC, N, 1, QC, 1, false>(Tm, Um, tb.eSc, nbl, grp);
    sweep<T, 1, QC, N, 1, QC, 1, false>(Tp, Up, tb.eSc, nbl, grp);
    grp.sync();
    for (int idx = grp.rank(); idx < nb * P; idx += grp.size()) {
      const int e = idx / P, p = idx - e * P;
      const bool wall = en[e] < 0;
      T um[5], up[5];
#pragma unroll
      for (int c = 0; c < 5; ++c) {
        um[c] = Um[(e * 5 + c) * P + p];
        up[c] = Up[(e * 5 + c) * P + p];
      }
      if (wall) wall_ghost(um, ph, up);
      const T rm = T(1) / (ph.rho_r + um[0]), rp = T(1) / (ph.rho_r + up[0]);
      const T pm = pressure_dev(um, rm, ph.gm1), pp = pressure_dev(up, rp, ph.gm1);
      const T lm = sqrt(um[1] * um[1] + um[2] * um[2] + um[3] * um[3]) * rm + sqrt(fabs(ph.gamma * (ph.p_r + pm) * rm));
      const T lp = sqrt(up[1] * up[1] + up[2] * up[2] + up[3] * up[3]) * rp + sqrt(fabs(ph.gamma * (ph.p_r + pp) * rp));
      const T lam = lm > lp ? lm : lp;
      if (GEO == GEO_AFFINE) {
        const T w = tb.wc[p % QC] * tb.wc[p / QC] * area;
        T fm[5], fp[5];
        conv_flux_dir(um, rm, pm, ph.H_r, d, fm);
        conv_flux_dir(up, rp, pp, ph.H_r, d, fp);
#pragma unroll
        for (int c = 0; c < 5; ++c)
          Um[(e * 5 + c) * P + p] = w * (T(0.5) * sgn * (fm[c] + fp[c]) + T(0.5) * lam * (um[c] - up[c]));
      } else {
        const T* g = GEO == GEO_FLY ? go + (size_t)e * 13 * P + p
                                    : static_cast<const T*>(kp.gfc) + ((size_t)eo[e] * 6 + f) * 13 * P + p;
        const T nn[3] = {g[9 * P], g[10 * P], g[11 * P]};
        const T dw = g[12 * P] * tb.wc[p % QC] * tb.wc[p / QC];
        T fn[5];
#pragma unroll
        for (int c = 0; c < 5; ++c) fn[c] = T(0);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          T fm[5], fp[5];
          conv_flux_dir(um, rm, pm, ph.H_r, a, fm);
          conv_flux_dir(up, rp, pp, ph.H_r, a, fp);
#pragma unroll
          for (int c = 0; c < 5; ++c) fn[c] += (fm[c] + fp[c]) * nn[a];
        }
#pragma unroll
        for (int c = 0; c < 5; ++c) Um[(e * 5 + c) * P + p] = dw * (T(0.5) * fn[c] + T(0.5) * lam * (um[c] - up[c]));
      }
    }
    grp.sync();
    sweep<T, 1, QC, QC, 1, N, 1, false>(Um, Tm, tb.eScT, nbl, grp);
    grp.sync();
    sweep<T, 0, QC, N, 1, N, 1, false>(Tm, lc, tb.eScT, nbl, grp);
    grp.sync();
  } else {
    for (int idx = grp.rank(); idx < nbl * N2; idx += grp.size()) lc[idx] = T(0);
  }

  constexpr int P = QV * QV;
  if (kp.visc) {
    T* gnb = go + CB * 13 * P;  // GEO_FLY: the other side's face geometry
    if (GEO == GEO_FLY) {
      fill_face_geo<T, N, QV, CB, d>(sx, s, fa, tb.eSv, tb.eDv, dlm, go, nb, grp);
      fill_face_geo<T, N, QV, CB, d>(sxn, 1 - s, fa, tb.eSv, tb.eDv, dlp, gnb, nb, grp);
    }
    T* Um = fa;  // 8 point arrays [CB][5][P]
    T* Up = Um + CB * 5 * P;
    T* G1m = Up + CB * 5 * P;
    T* G2m = G1m + CB * 5 * P;
    T* Gdm = G2m + CB * 5 * P;
    T* G1p = Gdm + CB * 5 * P;
    T* G2p = G1p + CB * 5 * P;
    T* Gdp = G2p + CB * 5 * P;
    T* Tm = Gdp + CB * 5 * P;  // 4 temporaries [CB][5][N][QV]
    T* Tp = Tm + CB * 5 * N * QV;
    T* Tdm = Tp + CB * 5 * N * QV;
    T* Tdp = Tdm + CB * 5 * N * QV;
    grp.sync();
    // values and normal derivatives of both traces to the face Gauss points
    sweep<T, 0, N, N, 1, QV, 1, false>(Lm, Tm, tb.eSv, nbl, grp);
    sweep<T, 0, N, N, 1, QV, 1, false>(Lp, Tp, tb.eSv, nbl, grp);
    sweep<T, 0, N, N, 1, QV, 1, false>(Dm, Tdm, tb.eSv, nbl, grp);
    sweep<T, 0, N, N, 1, QV, 1, false>(Dp, Tdp, tb.eSv, nbl, grp);
    grp.sync();
    sweep<T, 1, QV, N, 1, QV, 1, false>(Tm, Um, tb.eSv, nbl, grp);
    sweep<T, 1, QV, N, 1, QV, 1, false>(Tp, Up, tb.eSv, nbl, grp);
    sweep<T, 1, QV, N, 1, QV, 1, false>(Tdm, Gdm, tb.eSv, nbl, grp);
    sweep<T, 1, QV, N, 1, QV, 1, false>(Tdp, Gdp, tb.eSv, nbl, grp);
    grp.sync();
    // tangential derivatives by collocation on the face grid
    sweep<T, 0, QV, QV, 1, QV, -1, false>(Um, G1m, tb.eDv, nbl, grp);
    sweep<T, 1, QV, QV, 1, QV, -1, false>(Um, G2m, tb.eDv, nbl, grp);
    sweep<T, 0, QV, QV, 1, QV, -1, false>(Up, G1p, tb.eDv, nbl, grp);
    sweep<T, 1, QV, QV, 1, QV, -1, false>(Up, G2p, tb.eDv, nbl, grp);
    grp.sync();
    for (int idx = grp.rank(); idx < nb * P; idx += grp.size()) {
      const int e = idx / P, p = idx - e * P;
      const bool wall = en[e] < 0;
      const int o = e * 5 * P + p;
      T um[5], up[5], Gm[5][3], Gp[5][3];
      T nrm[3] = {T(0), T(0), T(0)};
      T Jm[9], Jp[9];
      T wgt = tb.wv[p % QV] * tb.wv[p / QV] * area;
      if (GEO == GEO_AFFINE) {
        nrm[d] = sgn;
#pragma unroll
        for (int c = 0; c < 5; ++c) {
          um[c] = Um[o + c * P];
          up[c] = Up[o + c * P];
          Gm[c][t1] = G1m[o + c * P] * hinv[t1];
          Gm[c][t2] = G2m[o + c * P] * hinv[t2];
          Gm[c][d] = Gdm[o + c * P] * hinv[d];
          Gp[c][t1] = G1p[o + c * P] * hinv[t1];
          Gp[c][t2] = G2p[o + c * P] * hinv[t2];
          Gp[c][d] = Gdp[o + c * P] * hinv[d];
        }
      } else {
        const T* g = GEO == GEO_FLY ? go + (size_t)e * 13 * P + p
                                    : static_cast<const T*>(kp.gfv) + ((size_t)eo[e] * 6 + f) * 13 * P + p;
#pragma unroll
        for (int m = 0; m < 9; ++m) Jm[m] = g[m * P];
        nrm[0] = g[9 * P];
        nrm[1] = g[10 * P];
        nrm[2] = g[11 * P];
        wgt = g[12 * P] * tb.wv[p % QV] * tb.wv[p / QV];
        if (!wall && GEO == GEO_STORED && oc) {
          frame_face_jinv<T, QV>(static_cast<const T*>(kp.gfv), en[e], oc[e], d, s, p, Jp);
        } else if (!wall) {
          const T* gp = GEO == GEO_FLY ? gnb + (size_t)e * 13 * P + p
                                       : static_cast<const T*>(kp.gfv) + ((size_t)en[e] * 6 + fo) * 13 * P + p;
#pragma unroll
          for (int m = 0; m < 9; ++m) Jp[m] = gp[m * P];
        } else {
#pragma unroll
          for (int m = 0; m < 9; ++m) Jp[m] = Jm[m];
        }
#pragma unroll
        for (int c = 0; c < 5; ++c) {
          um[c] = Um[o + c * P];
          up[c] = Up[o + c * P];
          const T a1 = G1m[o + c * P], a2 = G2m[o + c * P], ad = Gdm[o + c * P];
          const T b1 = G1p[o + c * P], b2 = G2p[o + c * P], bd = Gdp[o + c * P];
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            Gm[c][a] = Jm[3 * t1 + a] * a1 + Jm[3 * t2 + a] * a2 + Jm[3 * d + a] * ad;
            Gp[c][a] = Jp[3 * t1 + a] * b1 + Jp[3 * t2 + a] * b2 + Jp[3 * d + a] * bd;
          }
        }
      }
      if (wall) {
        wall_ghost(um, ph, up);
#pragma unroll
        for (int c = 0; c < 5; ++c)
#pragma unroll
          for (int j = 0; j < 3; ++j) Gp[c][j] = Gm[c][j];
      }
      T Fm[5][3], Fp[5][3];
      visc_flux(um, Gm, ph, Fm);
      visc_flux(up, Gp, ph, Fp);
      const T tau = tau_f[e];
      T jmp[5];
#pragma unroll
      for (int c = 0; c < 5; ++c) {
        jmp[c] = um[c] - up[c];
        const T fvn = (Fm[c][0] + Fp[c][0]) * nrm[0] + (Fm[c][1] + Fp[c][1]) * nrm[1] + (Fm[c][2] + Fp[c][2]) * nrm[2];
        const T v = -wgt * (T(0.5) * fvn - tau * jmp[c]);
        Um[o + c * P] = v;   // own side:   -(V^-, Q*.n^-)
        Up[o + c * P] = -v;  // other side: -(V^+, Q*.n^+) = +(V^+, Q*.n^-)
      }
      T Jg[5][3];
#pragma unroll
      for (int c = 0; c < 5; ++c)
#pragma unroll
        for (int a = 0; a < 3; ++a) Jg[c][a] = jmp[c] * nrm[a];
      const T hw = T(-0.5) * wgt;
      visc_flux(um, Jg, ph, Fm);
      if (!wall) visc_flux(up, Jg, ph, Fp);
      if (GEO == GEO_AFFINE) {
#pragma unroll
        for (int c = 0; c < 5; ++c) {
          G1m[o + c * P] = hw * hinv[t1] * Fm[c][t1];
          G2m[o + c * P] = hw * hinv[t2] * Fm[c][t2];
          Gdm[o + c * P] = hw * hinv[d] * Fm[c][d];
          G1p[o + c * P] = hw * hinv[t1] * Fp[c][t1];
          G2p[o + c * P] = hw * hinv[t2] * Fp[c][t2];
          Gdp[o + c * P] = hw * hinv[d] * Fp[c][d];
        }
      } else {
#pragma unroll
        for (int c = 0; c < 5; ++c) {
          G1m[o + c * P] = hw * (Jm[3 * t1] * Fm[c][0] + Jm[3 * t1 + 1] * Fm[c][1] + Jm[3 * t1 + 2] * Fm[c][2]);
          G2m[o + c * P] = hw * (Jm[3 * t2] * Fm[c][0] + Jm[3 * t2 + 1] * Fm[c][1] + Jm[3 * t2 + 2] * Fm[c][2]);
          Gdm[o + c * P] = hw * (Jm[3 * d] * Fm[c][0] + Jm[3 * d + 1] * Fm[c][1] + Jm[3 * d + 2] * Fm[c][2]);
          G1p[o + c * P] = hw * (Jp[3 * t1] * Fp[c][0] + Jp[3 * t1 + 1] * Fp[c][1] + Jp[3 * t1 + 2] * Fp[c][2]);
          G2p[o + c * P] = hw * (Jp[3 * t2] * Fp[c][0] + Jp[3 * t2 + 1] * Fp[c][1] + Jp[3 * t2 + 2] * Fp[c][2]);
          Gdp[o + c * P] = hw * (Jp[3 * d] * Fp[c][0] + Jp[3 * d + 1] * Fp[c][1] + Jp[3 * d + 2] * Fp[c][2]);
        }
      }
    }
    grp.sync();
    // both sides: value test + tangential gradient tests, normal-gradient test
    sweep<T, 0, QV, QV, 1, QV, -1, true>(G1m, Um, tb.eDvT, nbl, grp);
    sweep<T, 0, QV, QV, 1, QV, -1, true>(G1p, Up, tb.eDvT, nbl, grp);
    grp.sync();
    sweep<T, 1, QV, QV, 1, QV, -1, true>(G2m, Um, tb.eDvT, nbl, grp);
    sweep<T, 1, QV, QV, 1, QV, -1, true>(G2p, Up, tb.eDvT, nbl, grp);
    grp.sync();
    sweep<T, 1, QV, QV, 1, N, 1, false>(Um, Tm, tb.eSvT, nbl, grp);
    sweep<T, 1, QV, QV, 1, N, 1, false>(Up, Tp, tb.eSvT, nbl, grp);
    sweep<T, 1, QV, QV, 1, N, 1, false>(Gdm, Tdm, tb.eSvT, nbl, grp);
    sweep<T, 1, QV, QV, 1, N, 1, false>(Gdp, Tdp, tb.eSvT, nbl, grp);
    grp.sync();
    sweep<T, 0, QV, N, 1, N, 1, false>(Tm, Lm, tb.eSvT, nbl, grp);
    sweep<T, 0, QV, N, 1, N, 1, false>(Tp, Lp, tb.eSvT, nbl, grp);
    sweep<T, 0, QV, N, 1, N, 1, false>(Tdm, Dm, tb.eSvT, nbl, grp);
    sweep<T, 0, QV, N, 1, N, 1, false>(Tdp, Dp, tb.eSvT, nbl, grp);
    grp.sync();
  }
  // shares of the own and the other cell
  for (int idx = grp.rank(); idx < nbl * N2; idx += grp.size()) {
    const int ec = idx / N2, j = idx - ec * N2, e = ec / 5, c = ec - 5 * e;
    const T lv = kp.visc ? Lm[idx] : T(0), dv = kp.visc ? Dm[idx] : T(0);
    T* po = FB + ((size_t)eo[e] * 6 + f) * 10 * N2 + c * N2 + j;
    po[0] = lc[idx] + lv;
    po[5 * N2] = dv;
    if (en[e] >= 0) {
      int fw = fo, jw = j;
      T dsg = T(1);
      if (oc) {
        // the other cell's face node of this face point, in its own frame
        int dn, refl, sn;
        frame_facing(oc[e], d, s, dn, refl, sn);
        const int r = frame_node<N>(oc[e], face_node<N>(d, s ? 0 : N - 1, j % N, j / N));
        const int r0 = r % N, r1 = (r / N) % N, r2 = r / (N * N);
        fw = 2 * dn + sn;
        jw = dn == 0 ? r1 + N * r2 : (dn == 1 ? r0 + N * r2 : r0 + N * r1);
        dsg = refl ? T(-1) : T(1);
      }
      T* pn = FB + ((size_t)en[e] * 6 + fw) * 10 * N2 + c * N2 + jw;
      pn[0] = (kp.visc ? Lp[idx] : T(0)) - lc[idx];
      pn[5 * N2] = kp.visc ? dsg * Dp[idx] : T(0);
    }
  }
}

// Shared memory of face_pair_terms per face: 4 trace layers; arena: conv 2 tmp + 2 point arrays,
// visc 8 point arrays + 4 tmp.
template <int N, int QC, int QV>
struct PairSizes {
  static constexpr int N2 = N * N;
  static constexpr int LAYERS = 4 * 5 * N2;
  static constexpr int CONV = 2 * 5 * QC * N + 2 * 5 * QC * QC;
  static constexpr int VISC = 8 * 5 * QV * QV + 4 * 5 * N * QV;
  static constexpr int ARENA = CONV > VISC ? CONV : VISC;
};

// sr += the 6 face shares of each cell, staged in fs [nb][6][2][5][N^2]
template <typename T, int N, class G>
__device__ void gather_face_shares(T* sr, const T* fs, const Tab<T>& tb, int nb, G grp) {
  constexpr int N2 = N * N, N3 = N * N * N;
  for (int idx = grp.rank(); idx < nb * 5 * N3; idx += grp.size()) {
    const int ec = idx / N3, q = idx - ec * N3, e = ec / 5, c = ec - 5 * e;
    const int ii[3] = {q % N, (q / N) % N, q / N2};
    T acc = T(0);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
      const int j = ii[t1] + N * ii[t2];
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        const T* F = fs + ((size_t)(e * 6 + 2 * d + s) * 2 * 5 + c) * N2 + j;
        acc += (s ? tb.dl1 : tb.dl0)[ii[d]] * F[5 * N2];
        if (ii[d] == (s ? N - 1 : 0)) acc += F[0];
      }
    }
    sr[idx] += acc;
  }
}

}  // namespace dgcns
