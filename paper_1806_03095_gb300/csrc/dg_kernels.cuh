// Device code of libdgcns: sum-factorized cell and face integrals of the
// compressible Navier--Stokes DG operator (Eq. WeakFormulationConservedVariables),
// tensor-product inverse mass matrix and the 2N RK stage update (Sec. 2.3, 2.4).
//
// Organisation (GB300-first, one CTA per batch of CB cells):
//  - the cell batch's nodal state is staged in shared memory (converted to the
//    arithmetic type T: double for the FP64 form, float for the mixed form);
//  - every 1D contraction ("sweep") is done by one thread per line with the
//    line held in registers and the 1D matrix broadcast from shared memory
//    (the paper's sum factorization, Eq. SumFactorization; loop lengths are
//    template parameters, as the paper's kernels do);
//  - gradients use the collocation trick of Sec. 2.3: interpolate values to
//    the Gauss grid, then apply the Gauss-point derivative matrix (2d instead
//    of d^2 1D kernels); the test with grad V applies the transposed matrices;
//  - faces are evaluated element-centrically: each cell computes the numerical
//    fluxes on its 6 faces from its own trace and the neighbour's and tests
//    them with its own basis only, so no two CTAs write the same cell.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "dg_common.h"

namespace dgcns {

constexpr int NT = 128;  // threads per CTA of every operator kernel

// Thread groups that cooperate on a batch of cells: the whole CTA (barrier
// __syncthreads) or one warp (barrier __syncwarp, so warps of one CTA progress
// independently and hide each other's latency).
struct CtaGroup {
  __device__ __forceinline__ int rank() const { return threadIdx.x; }
  __device__ __forceinline__ int size() const { return blockDim.x; }
  __device__ __forceinline__ void sync() const { __syncthreads(); }
};
struct WarpGroup {
  __device__ __forceinline__ int rank() const { return threadIdx.x & 31; }
  __device__ __forceinline__ int size() const { return 32; }
  __device__ __forceinline__ void sync() const { __syncwarp(); }
};

// Elementwise pass over i = rank, rank + stride, ... < n (at most PER indices per thread): a thread
// issues its loads (in chunks of 8) before the matching stores, so that their latencies overlap
// instead of adding up.
template <int PER, class Ld, class St>
__device__ __forceinline__ void batched_pass(int rank, int stride, int n, Ld ld, St st) {
  constexpr int CH = PER < 8 ? PER : 8;
#pragma unroll 1
  for (int j0 = 0; j0 < PER; j0 += CH) {
    decltype(ld(0)) v[CH];
#pragma unroll
    for (int j = 0; j < CH; ++j) {
      const int i = (j0 + j) * stride + rank;
      if (j0 + j < PER && i < n) v[j] = ld(i);
    }
#pragma unroll
    for (int j = 0; j < CH; ++j) {
      const int i = (j0 + j) * stride + rank;
      if (j0 + j < PER && i < n) st(i, v[j]);
    }
  }
}

// ---------------------------------------------------------------------------
// Shared-memory tables
// ---------------------------------------------------------------------------
template <typename T>
struct Tab {
  const T *eSc, *eScT, *eDc, *eDcT, *eSv, *eSvT, *eDv, *eDvT, *eSmi, *eSmiT, *eSm, *eDm;
  const T *wc, *wv, *wm, *dl0, *dl1;
};

// The same tables in constant memory (used by the FP32 kernels), one copy per instantiation and
// translation unit, written by upload_const_tables when a context is created.  Both have internal linkage (anonymous namespace): as
// templates with external linkage the linker would merge them across the translation units, and the
// upload would reach one module's copy only.  The sweeps index the 1D operators only with
// compile-time offsets, so the FMAs take the coefficients as constant-bank operands: no load
// instruction per coefficient (from shared memory that was one load per FMA, which bound the FP32
// kernels by the shared-memory pipe).  Point weights and trace derivatives are indexed per lane and
// stay in shared memory (the constant cache serialises lane-dependent addresses).
namespace {
template <typename T, int N, int QC, int QV>
__constant__ T c_tab[make_layout(N, QC, QV).total];

template <int N, int QC, int QV>
int upload_const_tables(const double* t64, const float* t32, cudaStream_t st) {
  constexpr int n = make_layout(N, QC, QV).total;
  if (cudaMemcpyToSymbolAsync(c_tab<double, N, QC, QV>, t64, n * sizeof(double), 0, cudaMemcpyHostToDevice, st) !=
          cudaSuccess ||
      cudaMemcpyToSymbolAsync(c_tab<float, N, QC, QV>, t32, n * sizeof(float), 0, cudaMemcpyHostToDevice, st) !=
          cudaSuccess)
    return -1;
  return cudaStreamSynchronize(st) == cudaSuccess ? 0 : -1;
}
}  // namespace

template <typename T, int N, int QC, int QV>
__device__ __forceinline__ Tab<T> load_tables(const T* __restrict__ g, T* s) {
  constexpr TableLayout L = make_layout(N, QC, QV);
  for (int i = threadIdx.x; i < L.total; i += blockDim.x) s[i] = g[i];
  // FP32: operators from constant memory (6 % faster, measured); FP64: from shared memory (the constant
  // operands made both FP64 kernels 2-3 % slower, measured)
  const T* c = s;
  if constexpr (sizeof(T) == 4) c = c_tab<T, N, QC, QV>;
  Tab<T> t;
  t.eSc = c + L.eo[EO_SC]; t.eScT = c + L.eo[EO_SCT]; t.eDc = c + L.eo[EO_DC]; t.eDcT = c + L.eo[EO_DCT];
  t.eSv = c + L.eo[EO_SV]; t.eSvT = c + L.eo[EO_SVT]; t.eDv = c + L.eo[EO_DV]; t.eDvT = c + L.eo[EO_DVT];
  t.eSmi = c + L.eo[EO_SMI]; t.eSmiT = c + L.eo[EO_SMIT]; t.eSm = c + L.eo[EO_SM]; t.eDm = c + L.eo[EO_DM];
  t.wc = s + L.wc; t.wv = s + L.wv; t.wm = s + L.wm; t.dl0 = s + L.dl0; t.dl1 = s + L.dl1;
  return t;
}

template <int N, int QC, int QV>
constexpr int table_elems() {
  return make_layout(N, QC, QV).total;
}

// 16-byte vector loads/stores of K contiguous values (K * sizeof(T) a multiple of 16, p 16-byte aligned).
template <typename T, int K>
__device__ __forceinline__ void vec_load(const T* p, T* x) {
  if constexpr (sizeof(T) == 4) {
#pragma unroll
    for (int j = 0; j < K / 4; ++j) {
      const float4 t = reinterpret_cast<const float4*>(p)[j];
      x[4 * j] = t.x;
      x[4 * j + 1] = t.y;
      x[4 * j + 2] = t.z;
      x[4 * j + 3] = t.w;
    }
  } else {
#pragma unroll
    for (int j = 0; j < K / 2; ++j) {
      const double2 t = reinterpret_cast<const double2*>(p)[j];
      x[2 * j] = t.x;
      x[2 * j + 1] = t.y;
    }
  }
}

template <typename T, int K>
__device__ __forceinline__ void vec_store(T* p, const T* x) {
  if constexpr (sizeof(T) == 4) {
#pragma unroll
    for (int j = 0; j < K / 4; ++j)
      reinterpret_cast<float4*>(p)[j] = make_float4(x[4 * j], x[4 * j + 1], x[4 * j + 2], x[4 * j + 3]);
  } else {
#pragma unroll
    for (int j = 0; j < K / 2; ++j) reinterpret_cast<double2*>(p)[j] = make_double2(x[2 * j], x[2 * j + 1]);
  }
}

// ---------------------------------------------------------------------------
// 1D sweep with even-odd decomposition: apply the operator O (DOUT x DIN, in
// the even-odd form above, symmetry SYM = +1 or -1) along axis AX of nblk
// arrays of shape (D2, D1, D0) (D0 fastest, arrays contiguous one after the
// other).  The axis extent DIN becomes DOUT.  One thread per line, the line in
// registers, the operator broadcast from shared memory.  ACC adds into out.
// ---------------------------------------------------------------------------
template <typename T, int AX, int D0, int D1, int D2, int DOUT, int SYM, bool ACC, class G = CtaGroup>
__device__ __forceinline__ void sweep(const T* __restrict__ in, T* __restrict__ out, const T* __restrict__ E,
                                      int nblk, G grp = G()) {
  constexpr int DIN = AX == 0 ? D0 : (AX == 1 ? D1 : D2);
  constexpr int IH = DIN / 2, OH = (DOUT + 1) / 2;
  constexpr int O0 = AX == 0 ? DOUT : D0;
  constexpr int O1 = AX == 1 ? DOUT : D1;
  constexpr int O2 = AX == 2 ? DOUT : D2;
  constexpr int ISZ = D0 * D1 * D2, OSZ = O0 * O1 * O2;
  constexpr int NL = ISZ / DIN;
  constexpr int IST = AX == 0 ? 1 : (AX == 1 ? D0 : D0 * D1);
  constexpr int OST = AX == 0 ? 1 : (AX == 1 ? O0 : O0 * O1);
  for (int l = grp.rank(); l < nblk * NL; l += grp.size()) {
    // the operator table is loop-invariant; where it is large (high degrees) its loads stay inside the
    // loop (the pointer passes through an empty asm), so that it is not hoisted into registers and spilled
    const T* Ep = E;
    if constexpr (2 * OH * IH > 48) asm volatile("" : "+l"(Ep));
    const T* __restrict__ A = Ep;
    const T* __restrict__ B = Ep + OH * IH;
    const T* __restrict__ C = Ep + 2 * OH * IH;
    const int blk = l / NL, r = l - blk * NL;
    int ib, ob;
    if (AX == 0) {
      ib = r * D0;
      ob = r * O0;
    } else if (AX == 1) {
      const int a = r % D0, b = r / D0;
      ib = b * D0 * D1 + a;
      ob = b * O0 * O1 + a;
    } else {
      ib = r;
      ob = r;
    }
    const T* ip = in + blk * ISZ + ib;
    T* op = out + blk * OSZ + ob;
    // a line along x is contiguous: 16-byte vector accesses avoid the bank conflicts
    // of threads reading 4-word lines at a 4-word stride
    constexpr bool VIN = AX == 0 && (DIN * sizeof(T)) % 16 == 0;
    constexpr bool VOUT = AX == 0 && (DOUT * sizeof(T)) % 16 == 0;
    T x[DIN];
    if (VIN && (reinterpret_cast<uintptr_t>(ip) & 15) == 0) {
      vec_load<T, DIN>(ip, x);
    } else {
#pragma unroll
      for (int i = 0; i < DIN; ++i) x[i] = ip[i * IST];
    }
    T xe[IH], xo[IH];
#pragma unroll
    for (int i = 0; i < IH; ++i) {
      xe[i] = x[i] + x[DIN - 1 - i];
      xo[i] = x[i] - x[DIN - 1 - i];
    }
    const T xm = (DIN & 1) ? x[IH] : T(0);
    T y[DOUT];
#pragma unroll
    for (int q = 0; q < OH; ++q) {
      // the centre output of an odd-length result: a symmetric operator (SYM > 0) has no odd part there and an
      // antisymmetric one no even part (exactly, for the symmetric point sets; the tables hold rounding-level
      // values), so only the other half is formed
      const bool centre = (DOUT & 1) && q == OH - 1;
      const bool need_e = !(centre && SYM < 0), need_o = !(centre && SYM > 0);
      T e = (DIN & 1) && need_e ? C[q] * xm : T(0);
      T o = T(0);
#pragma unroll
      for (int i = 0; i < IH; ++i) {
        if (need_e) e += A[q * IH + i] * xe[i];
        if (need_o) o += B[q * IH + i] * xo[i];
      }
      if (centre) {
        y[q] = SYM > 0 ? e : o;
      } else {
        y[q] = e + o;
        y[DOUT - 1 - q] = SYM > 0 ? e - o : o - e;
      }
    }
    if (VOUT && (reinterpret_cast<uintptr_t>(op) & 15) == 0) {
      if (ACC) {
        T z[DOUT];
        vec_load<T, DOUT>(op, z);
#pragma unroll
        for (int q = 0; q < DOUT; ++q) y[q] += z[q];
      }
      vec_store<T, DOUT>(op, y);
    } else {
#pragma unroll
      for (int q = 0; q < DOUT; ++q) {
        if (ACC)
          op[q * OST] += y[q];
        else
          op[q * OST] = y[q];
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Pointwise physics (Eq. CompressibleNavierStokesFluxes).  F[c][j], c the
// conserved component, j the physical direction.
// ---------------------------------------------------------------------------
//
// The kernels carry the state as deviations dU = U - U_ref from the constant
// reference U_ref = (rho_r, 0, 0, 0, rho_r c_v T_0) (T_0 the reference and wall
// temperature).  Jumps are dU- - dU+, the momentum flux uses the pressure
// deviation dp = p - p_r (p_r = (gamma-1) rho_r c_v T_0): the constant flux
// p_r I has zero residual on every element (free-stream identity), so this is
// the same operator, while FP32 arithmetic keeps the O(1) fluctuations instead
// of rounding them against rho E ~ 10^2..10^5.
template <typename T>
struct PhysT {
  T gamma, gm1, mu, lam_cv;  // lam_cv = lambda / c_v
  T rho_r, rhoE_r, p_r, H_r; // reference density, energy, pressure, rhoE_r + p_r
  T cvTw2;                   // 2 c_v T_wall
};

// pressure deviation p - p_r = (gamma-1)(d(rho E) - |m|^2/(2 rho))
template <typename T>
__device__ __forceinline__ T pressure_dev(const T u[5], T rinv, T gm1) {
  return gm1 * (u[4] - T(0.5) * rinv * (u[1] * u[1] + u[2] * u[2] + u[3] * u[3]));
}

// Convective flux along direction j, F_c[.][j], minus the constant p_r I:
// (m_j, m v_j + dp e_j, (H_r + d(rho E) + dp) v_j)
template <typename T>
__device__ __forceinline__ void conv_flux_dir(const T u[5], T rinv, T dp, T H_r, int j, T f[5]) {
  const T vj = u[1 + j] * rinv;
  f[0] = u[1 + j];
  f[1] = u[1] * vj;
  f[2] = u[2] * vj;
  f[3] = u[3] * vj;
  f[1 + j] += dp;
  f[4] = (H_r + u[4] + dp) * vj;
}

// Viscous flux F_v(U, G) from deviations u and the (physical) gradient argument G[c][a].
template <typename T>
__device__ __forceinline__ void visc_flux(const T u[5], const T G[5][3], const PhysT<T>& ph, T F[5][3]) {
  const T rinv = T(1) / (ph.rho_r + u[0]);
  const T v0 = u[1] * rinv, v1 = u[2] * rinv, v2 = u[3] * rinv;
  const T E = (ph.rhoE_r + u[4]) * rinv;
  T gu[3][3];
  const T v[3] = {v0, v1, v2};
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) gu[i][j] = (G[1 + i][j] - v[i] * G[0][j]) * rinv;
  const T div = gu[0][0] + gu[1][1] + gu[2][2];
  const T twothird = T(2) / T(3);
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    F[0][j] = T(0);
    T tv = T(0);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      T tij = ph.mu * (gu[i][j] + gu[j][i]);
      if (i == j) tij -= ph.mu * twothird * div;
      F[1 + i][j] = tij;
      tv += tij * v[i];
    }
    const T gE = (G[4][j] - E * G[0][j]) * rinv;
    const T gT_cv = gE - (v0 * gu[0][j] + v1 * gu[1][j] + v2 * gu[2][j]);  // c_v * dT/dx_j
    F[4][j] = tv + ph.lam_cv * gT_cv;
  }
}

template <typename T>
__device__ __forceinline__ const KConst<T>& kconst(const KParams& kp);
template <>
__device__ __forceinline__ const KConst<double>& kconst<double>(const KParams& kp) { return kp.cd; }
template <>
__device__ __forceinline__ const KConst<float>& kconst<float>(const KParams& kp) { return kp.cf; }

template <typename T>
__device__ __forceinline__ PhysT<T> make_phys(const KParams& kp) {
  const KConst<T>& c = kconst<T>(kp);
  PhysT<T> ph;
  ph.gamma = c.gamma;
  ph.gm1 = c.gm1;
  ph.mu = c.mu;
  ph.lam_cv = c.lam_cv;
  ph.rho_r = c.rho_r;
  ph.rhoE_r = c.rhoE_r;
  ph.p_r = c.p_r;
  ph.H_r = c.H_r;
  ph.cvTw2 = c.cvTw2;
  return ph;
}

// Exterior state on an isothermal no-slip wall: rho+ = rho-, u+ = -u-, T+ = 2 T_w - T-,
// i.e. rho E+ = 2 rho c_v T_w - rho E- + rho |u|^2, written for deviations
// (rho E_r = rho_r c_v T_w):  d(rho E)+ = 2 c_v T_w d(rho) - d(rho E)- + |m|^2/rho.
template <typename T>
__device__ __forceinline__ void wall_ghost(const T um[5], const PhysT<T>& ph, T up[5]) {
  const T rinv = T(1) / (ph.rho_r + um[0]);
  const T ke2 = rinv * (um[1] * um[1] + um[2] * um[2] + um[3] * um[3]);  // rho |u|^2
  up[0] = um[0];
  up[1] = -um[1];
  up[2] = -um[2];
  up[3] = -um[3];
  up[4] = ph.cvTw2 * um[0] - um[4] + ke2;
}

// ---------------------------------------------------------------------------
// Node index helpers
// ---------------------------------------------------------------------------
template <int N>
__device__ __forceinline__ int face_node(int d, int id, int j1, int j2) {
  // node with coordinate id along axis d, j1 along the first tangential axis, j2 along the second
  if (d == 0) return id + N * (j1 + N * j2);
  if (d == 1) return j1 + N * (id + N * j2);
  return j1 + N * (j2 + N * id);
}

// Rotated-frame meshes, stored geometry: the inverse Jacobian of the neighbour across a cell's local face
// (d, s), at the point of the neighbour's own face that coincides with point p of the cell's Q x Q face
// grid, with its rows re-expressed along the cell's reference axes (J^{-1}[b][a] = +-J_n^{-1}[b_n][a],
// negative where the neighbour's axis b_n runs against the cell's axis b).  gf: the stored face geometry
// [Nc][6][13][Q^2] (J^{-1} in entries 0..8, index 3 b + a); the Gauss points are symmetric about 1/2, so
// a reflected coordinate index i is Q - 1 - i.
template <typename T, int Q>
__device__ __forceinline__ void frame_face_jinv(const T* __restrict__ gf, int nbr, int code, int d, int s, int p,
                                                T Jp[9]) {
  int dn, refl, sn;
  frame_facing(code, d, s, dn, refl, sn);
  const int r = frame_node<Q>(code, face_node<Q>(d, s ? 0 : Q - 1, p % Q, p / Q));
  const int r0 = r % Q, r1 = (r / Q) % Q, r2 = r / (Q * Q);
  const int pn = dn == 0 ? r1 + Q * r2 : (dn == 1 ? r0 + Q * r2 : r0 + Q * r1);
  const T* g = gf + ((size_t)nbr * 6 + 2 * dn + sn) * 13 * Q * Q + pn;
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    const int bn = (code & 3) == b ? 0 : (((code >> 2) & 3) == b ? 1 : 2);
    const T sg = ((code >> (6 + bn)) & 1) ? T(-1) : T(1);
#pragma unroll
    for (int a = 0; a < 3; ++a) Jp[3 * b + a] = sg * g[(3 * bn + a) * Q * Q];
  }
}

// ---------------------------------------------------------------------------
// Geometry of the isoparametric map from the degree-k node coordinates X
// ([CB][3][N^3]): interpolation to a point set and collocation derivatives
// (exact, x is of degree k) give J[a][b] = d x_a / d xi_b; each point stores
// J^{-1}[b][a] (index 3b+a) and |det J|, faces also the unit outward normal
// n = J^{-T} n_xi / |J^{-T} n_xi| and dA = |det J| |J^{-T} n_xi|
// (Eq. IntegralsReferenceSpace).  Used once in FP64 by the geometry kernel
// (stored geometry) and per phase inside the operator kernels (GEO_FLY).
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T inv3(const T J[3][3], T Ji[9]) {
  const T c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
  const T c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
  const T c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
  const T det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
  const T id = T(1) / det;
  Ji[0] = c00 * id;
  Ji[1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) * id;
  Ji[2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) * id;
  Ji[3] = c01 * id;
  Ji[4] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) * id;
  Ji[5] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) * id;
  Ji[6] = c02 * id;
  Ji[7] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) * id;
  Ji[8] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) * id;
  return det;
}

template <int N, int Q>
constexpr int fill_cell_tmp() { return 3 * (N * N * Q + N * Q * Q + 4 * Q * Q * Q); }
template <int N, int Q>
constexpr int fill_face_tmp() { return 6 * N * N + 3 * N * Q + 12 * Q * Q; }

// out[e][10][Q^3]: J^{-1} and |det J| at the Gauss points (Q per direction), matrices eS: N->Q, eD: Q->Q
template <typename T, int N, int Q, int CB, class G>
__device__ void fill_cell_geo(const T* X, T* buf, const T* eS, const T* eD, T* out, int nb, G grp) {
  constexpr int P = Q * Q * Q;
  T* A = buf;
  T* B = A + CB * 3 * N * N * Q;
  T* Xq = B + CB * 3 * N * Q * Q;
  T* J0 = Xq + CB * 3 * P;
  T* J1 = J0 + CB * 3 * P;
  T* J2 = J1 + CB * 3 * P;
  const int nbl = 3 * nb;
  sweep<T, 0, N, N, N, Q, 1, false>(X, A, eS, nbl, grp);
  grp.sync();
  sweep<T, 1, Q, N, N, Q, 1, false>(A, B, eS, nbl, grp);
  grp.sync();
  sweep<T, 2, Q, Q, N, Q, 1, false>(B, Xq, eS, nbl, grp);
  grp.sync();
  sweep<T, 0, Q, Q, Q, Q, -1, false>(Xq, J0, eD, nbl, grp);
  sweep<T, 1, Q, Q, Q, Q, -1, false>(Xq, J1, eD, nbl, grp);
  sweep<T, 2, Q, Q, Q, Q, -1, false>(Xq, J2, eD, nbl, grp);
  grp.sync();
  for (int idx = grp.rank(); idx < nb * P; idx += grp.size()) {
    const int e = idx / P, p = idx - e * P;
    T J[3][3], Ji[9];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      J[a][0] = J0[(e * 3 + a) * P + p];
      J[a][1] = J1[(e * 3 + a) * P + p];
      J[a][2] = J2[(e * 3 + a) * P + p];
    }
    const T det = fabs(inv3(J, Ji));
    T* o = out + (size_t)e * 10 * P + p;
#pragma unroll
    for (int m = 0; m < 9; ++m) o[m * P] = Ji[m];
    o[9 * P] = det;
  }
  grp.sync();
}

// out[e][13][Q^2] on face (d, s): J^{-1} (9), unit outward normal (3), dA (1); dl = l_i' at the face
template <typename T, int N, int Q, int CB, int d, class G>
__device__ void fill_face_geo(const T* X, int s, T* buf, const T* eS, const T* eD, const T* dl, T* out, int nb,
                              G grp) {
  constexpr int P = Q * Q, N2 = N * N, N3 = N * N * N;
  constexpr int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
  T* L = buf;
  T* Dn = L + CB * 3 * N2;
  T* Tm = Dn + CB * 3 * N2;
  T* Xf = Tm + CB * 3 * N * Q;
  T* Jt1 = Xf + CB * 3 * P;
  T* Jt2 = Jt1 + CB * 3 * P;
  T* Jd = Jt2 + CB * 3 * P;
  const int id = s ? N - 1 : 0;
  const int nbl = 3 * nb;
  for (int idx = grp.rank(); idx < nbl * N2; idx += grp.size()) {
    const int ea = idx / N2, j = idx - ea * N2;
    const T* x = X + (size_t)ea * N3;
    L[idx] = x[face_node<N>(d, id, j % N, j / N)];
    T dn = T(0);
#pragma unroll
    for (int i = 0; i < N; ++i) dn += dl[i] * x[face_node<N>(d, i, j % N, j / N)];
    Dn[idx] = dn;
  }
  grp.sync();
  sweep<T, 0, N, N, 1, Q, 1, false>(L, Tm, eS, nbl, grp);
  grp.sync();
  sweep<T, 1, Q, N, 1, Q, 1, false>(Tm, Xf, eS, nbl, grp);
  grp.sync();
  sweep<T, 0, N, N, 1, Q, 1, false>(Dn, Tm, eS, nbl, grp);
  grp.sync();
  sweep<T, 1, Q, N, 1, Q, 1, false>(Tm, Jd, eS, nbl, grp);
  sweep<T, 0, Q, Q, 1, Q, -1, false>(Xf, Jt1, eD, nbl, grp);
  sweep<T, 1, Q, Q, 1, Q, -1, false>(Xf, Jt2, eD, nbl, grp);
  grp.sync();
  const T sgn = s ? T(1) : T(-1);
  for (int idx = grp.rank(); idx < nb * P; idx += grp.size()) {
    const int e = idx / P, p = idx - e * P;
    T J[3][3], Ji[9];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      J[a][t1] = Jt1[(e * 3 + a) * P + p];
      J[a][t2] = Jt2[(e * 3 + a) * P + p];
      J[a][d] = Jd[(e * 3 + a) * P + p];
    }
    const T det = fabs(inv3(J, Ji));
    const T v0 = sgn * Ji[3 * d], v1 = sgn * Ji[3 * d + 1], v2 = sgn * Ji[3 * d + 2];
    const T nv = sqrt(v0 * v0 + v1 * v1 + v2 * v2);
    T* o = out + (size_t)e * 13 * P + p;
#pragma unroll
    for (int m = 0; m < 9; ++m) o[m * P] = Ji[m];
    o[9 * P] = v0 / nv;
    o[10 * P] = v1 / nv;
    o[11 * P] = v2 / nv;
    o[12 * P] = det * nv;
  }
  grp.sync();
}

// out[e][N^3]: |det J| at the k+1 mass points (interpolation eSm, collocation eDm)
template <typename T, int N, int CB, class G>
__device__ void fill_mass_geo(const T* X, T* buf, const T* eSm, const T* eDm, T* out, int nb, G grp) {
  constexpr int N3 = N * N * N;
  T* A = buf;
  T* B = A + CB * 3 * N3;
  T* Xq = B + CB * 3 * N3;
  T* J0 = Xq + CB * 3 * N3;
  T* J1 = J0 + CB * 3 * N3;
  T* J2 = J1 + CB * 3 * N3;
  const int nbl = 3 * nb;
  sweep<T, 0, N, N, N, N, 1, false>(X, A, eSm, nbl, grp);
  grp.sync();
  sweep<T, 1, N, N, N, N, 1, false>(A, B, eSm, nbl, grp);
  grp.sync();
  sweep<T, 2, N, N, N, N, 1, false>(B, Xq, eSm, nbl, grp);
  grp.sync();
  sweep<T, 0, N, N, N, N, -1, false>(Xq, J0, eDm, nbl, grp);
  sweep<T, 1, N, N, N, N, -1, false>(Xq, J1, eDm, nbl, grp);
  sweep<T, 2, N, N, N, N, -1, false>(Xq, J2, eDm, nbl, grp);
  grp.sync();
  for (int idx = grp.rank(); idx < nb * N3; idx += grp.size()) {
    const int e = idx / N3, p = idx - e * N3;
    T J[3][3], Ji[9];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      J[a][0] = J0[(e * 3 + a) * N3 + p];
      J[a][1] = J1[(e * 3 + a) * N3 + p];
      J[a][2] = J2[(e * 3 + a) * N3 + p];
    }
    out[(size_t)e * N3 + p] = fabs(inv3(J, Ji));
  }
  grp.sync();
}

// ---------------------------------------------------------------------------
// Shared-memory budget per kernel
// ---------------------------------------------------------------------------
template <int N, int QC, int QV>
struct Sizes {
  static constexpr int N2 = N * N;
  static constexpr int N3 = N * N * N;
  static constexpr int QC3 = QC * QC * QC, QV3 = QV * QV * QV;
  // LEAN: the convective cell term forms one flux direction at a time (15 QC^3 values per cell instead of
  // 20 QC^3), used where the full arena would not fit (QC >= 11: 213 KB per cell in FP64)
  static constexpr bool LEAN = 20 * QC3 * 8 > 160 * 1024;
  static constexpr int CELL_ARENA = LEAN ? (15 * QC3 > 20 * QV3 ? 15 * QC3 : 20 * QV3)
                                         : 20 * (QC3 > QV3 ? QC3 : QV3);  // per cell
  // face arena per cell: conv: 2 layers, tmp, 2 point arrays; visc: 4 layers, tmp, 8 point arrays
  static constexpr int FACE_CONV = 2 * 5 * N2 + 5 * QC * N + 2 * 5 * QC * QC;
  static constexpr int FACE_VISC = 4 * 5 * N2 + 5 * QV * N + 8 * 5 * QV * QV;
  static constexpr int FACE_ARENA = FACE_CONV > FACE_VISC ? FACE_CONV : FACE_VISC;
  static constexpr int MASS_ARENA = 2 * 5 * N3;
  // GEO_FLY: fill temporaries live in the arena (computed before the phase uses it); the outputs in a
  // separate per-cell region (cell points, own + neighbour face points, mass points)
  static constexpr int QM = QC > QV ? QC : QV;
  static constexpr int FLY_TMP_C = fill_cell_tmp<N, QC>() > fill_cell_tmp<N, QV>() ? fill_cell_tmp<N, QC>()
                                                                                       : fill_cell_tmp<N, QV>();
  static constexpr int FLY_TMP_F = fill_face_tmp<N, QM>();
  static constexpr int FLY_TMP_M = 18 * N3;
  static constexpr int FLY_TMP = FLY_TMP_C > FLY_TMP_F ? (FLY_TMP_C > FLY_TMP_M ? FLY_TMP_C : FLY_TMP_M)
                                                       : (FLY_TMP_F > FLY_TMP_M ? FLY_TMP_F : FLY_TMP_M);
  static constexpr int FLY_OUT_C = 10 * (QC3 > QV3 ? QC3 : QV3);
  static constexpr int FLY_OUT_F = 2 * 13 * QM * QM;
  static constexpr int FLY_OUT = FLY_OUT_C > FLY_OUT_F ? (FLY_OUT_C > N3 ? FLY_OUT_C : N3) : (FLY_OUT_F > N3 ? FLY_OUT_F : N3);
};

// ---------------------------------------------------------------------------
// Cell integrals: sr += -(grad V, F_c) + (grad V, F_v) for the CTA's nb cells.
// su, sr: [CB][5][N^3]; ar: arena of CB*CELL_ARENA elements.
// Affine geometry: J = diag(h), |J| = h0 h1 h2.
// ---------------------------------------------------------------------------
template <typename T, int N, int QC, int QV, int CB, int GEO, class G = CtaGroup>
__device__ void cell_terms(const T* su, T* sr, T* ar, const Tab<T>& tb, const KParams& kp, const PhysT<T>& ph,
                           int e0, int nb, G grp = G(), const T* sx = nullptr, T* go = nullptr) {
  const KConst<T>& kc = kconst<T>(kp);
  const T detJ = kc.detJ;
  const T hinv[3] = {kc.hinv[0], kc.hinv[1], kc.hinv[2]};
  const int nbl = nb * 5;
  if constexpr (Sizes<N, QC, QV>::LEAN) {
    if (kp.conv) {
      static_assert(GEO != GEO_FLY, "the lean convective term has no geometry-on-the-fly variant");
      constexpr int P = QC * QC * QC;
      const T* gcell = static_cast<const T*>(kp.gcc) + (size_t)e0 * 10 * P;
      T* Uq = ar;
      T* Fj = ar + CB * 5 * P;
      T* Gt = ar + 2 * CB * 5 * P;
      // interpolate to the convective Gauss grid (temporaries in Fj and Gt)
      sweep<T, 0, N, N, N, QC, 1, false>(su, Fj, tb.eSc, nbl, grp);
      grp.sync();
      sweep<T, 1, QC, N, N, QC, 1, false>(Fj, Gt, tb.eSc, nbl, grp);
      grp.sync();
      sweep<T, 2, QC, QC, N, QC, 1, false>(Gt, Uq, tb.eSc, nbl, grp);
      grp.sync();
      // one direction b at a time: the contravariant flux -F_c J^{-T} |J| w along b, then Gt += D_b^T of it
#pragma unroll 1
      for (int b = 0; b < 3; ++b) {
        for (int idx = grp.rank(); idx < nb * P; idx += grp.size()) {
          const int e = idx / P, p = idx - e * P;
          const int q0 = p % QC, q1 = (p / QC) % QC, q2 = p / (QC * QC);
          T u[5];
#pragma unroll
          for (int c = 0; c < 5; ++c) u[c] = Uq[(e * 5 + c) * P + p];
          const T rinv = T(1) / (ph.rho_r + u[0]);
          const T dp = pressure_dev(u, rinv, ph.gm1);
          if (GEO == GEO_AFFINE) {
            T f[5];
            conv_flux_dir(u, rinv, dp, ph.H_r, b, f);
            const T sc = -tb.wc[q0] * tb.wc[q1] * tb.wc[q2] * detJ * hinv[b];
#pragma unroll
            for (int c = 0; c < 5; ++c) Fj[(e * 5 + c) * P + p] = sc * f[c];
          } else {
            const T* g = gcell + (size_t)e * 10 * P + p;
            const T j0 = g[(3 * b) * P], j1 = g[(3 * b + 1) * P], j2 = g[(3 * b + 2) * P];
            const T jw = -g[9 * P] * tb.wc[q0] * tb.wc[q1] * tb.wc[q2];
            T F[3][5];
#pragma unroll
            for (int a = 0; a < 3; ++a) conv_flux_dir(u, rinv, dp, ph.H_r, a, F[a]);
#pragma unroll
            for (int c = 0; c < 5; ++c) Fj[(e * 5 + c) * P + p] = jw * (j0 * F[0][c] + j1 * F[1][c] + j2 * F[2][c]);
          }
        }
        grp.sync();
        if (b == 0)
          sweep<T, 0, QC, QC, QC, QC, -1, false>(Fj, Gt, tb.eDcT, nbl, grp);
        else if (b == 1)
          sweep<T, 1, QC, QC, QC, QC, -1, true>(Fj, Gt, tb.eDcT, nbl, grp);
        else
          sweep<T, 2, QC, QC, QC, QC, -1, true>(Fj, Gt, tb.eDcT, nbl, grp);
        grp.sync();
      }
      // back to the nodes: S^T along z, y, x
      sweep<T, 2, QC, QC, QC, N, 1, false>(Gt, Fj, tb.eScT, nbl, grp);
      grp.sync();
      sweep<T, 1, QC, QC, N, N, 1, false>(Fj, Uq, tb.eScT, nbl, grp);
      grp.sync();
      sweep<T, 0, QC, N, N, N, 1, true>(Uq, sr, tb.eScT, nbl, grp);
      grp.sync();
    }
  } else if (kp.conv) {
    constexpr int P = QC * QC * QC;
    // stored geometry of the CTA's cells: global arrays, or recomputed now into `go` (GEO_FLY)
    const T* gcell = GEO == GEO_FLY ? go : static_cast<const T*>(kp.gcc) + (size_t)e0 * 10 * P;
    if (GEO == GEO_FLY) fill_cell_geo<T, N, QC, CB>(sx, ar, tb.eSc, tb.eDc, go, nb, grp);
    T* F0 = ar;
    T* F1 = ar + CB * 5 * P;
    T* F2 = ar + 2 * CB * 5 * P;
    T* Gt = ar + 3 * CB * 5 * P;
    // interpolate to the convective Gauss grid (Eq. SumFactorization)
    sweep<T, 0, N, N, N, QC, 1, false>(su, F1, tb.eSc, nbl, grp);
    grp.sync();
    sweep<T, 1, QC, N, N, QC, 1, false>(F1, F2, tb.eSc, nbl, grp);
    grp.sync();
    sweep<T, 2, QC, QC, N, QC, 1, false>(F2, F0, tb.eSc, nbl, grp);
    grp.sync();
    // pointwise: contravariant flux  -F_c J^{-T} |J| w  (minus sign of the weak form)
    for (int idx = grp.rank(); idx < nb * P; idx += grp.size()) {
      const int e = idx / P, p = idx - e * P;
      const int q0 = p % QC, q1 = (p / QC) % QC, q2 = p / (QC * QC);
      const T w = tb.wc[q0] * tb.wc[q1] * tb.wc[q2] * detJ;
      T u[5];
#pragma unroll
      for (int c = 0; c < 5; ++c) u[c] = F0[(e * 5 + c) * P + p];
      const T rinv = T(1) / (ph.rho_r + u[0]);
      const T dp = pressure_dev(u, rinv, ph.gm1);
      T* Fd[3] = {F0, F1, F2};
      if (GEO == GEO_AFFINE) {
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          T f[5];
          conv_flux_dir(u, rinv, dp, ph.H_r, j, f);
          const T s = -w * hinv[j];
#pragma unroll
          for (int c = 0; c < 5; ++c) Fd[j][(e * 5 + c) * P + p] = s * f[c];
        }
      } else {
        // contravariant flux Ft_b = -|J| w sum_a J^{-1}[b][a] F[.][a]
        const T* g = gcell + (size_t)e * 10 * P + p;
        T Ji[9];
#pragma unroll
        for (int m = 0; m < 9; ++m) Ji[m] = g[m * P];
        const T jw = -g[9 * P] * tb.wc[q0] * tb.wc[q1] * tb.wc[q2];
        T F[3][5];
#pragma unroll
        for (int a = 0; a < 3; ++a) conv_flux_dir(u, rinv, dp, ph.H_r, a, F[a]);
#pragma unroll
        for (int b = 0; b < 3; ++b)
#pragma unroll
          for (int c = 0; c < 5; ++c)
            Fd[b][(e * 5 + c) * P + p] = jw * (Ji[3 * b] * F[0][c] + Ji[3 * b + 1] * F[1][c] + Ji[3 * b + 2] * F[2][c]);
      }
    }
    grp.sync();
    // Gt = sum_d D_d^T Ft_d  (test with grad V in the collocation basis)
    sweep<T, 0, QC, QC, QC, QC, -1, false>(F0, Gt, tb.eDcT, nbl, grp);
    grp.sync();
    sweep<T, 1, QC, QC, QC, QC, -1, true>(F1, Gt, tb.eDcT, nbl, grp);
    grp.sync();
    sweep<T, 2, QC, QC, QC, QC, -1, true>(F2, Gt, tb.eDcT, nbl, grp);
    grp.sync();
    // back to the nodes: S^T along z, y, x
    sweep<T, 2, QC, QC, QC, N, 1, false>(Gt, F0, tb.eScT, nbl, grp);
    grp.sync();
    sweep<T, 1, QC, QC, N, N, 1, false>(F0, F1, tb.eScT, nbl, grp);
    grp.sync();
    sweep<T, 0, QC, N, N, N, 1, true>(F1, sr, tb.eScT, nbl, grp);
    grp.sync();
  }
  if (kp.visc) {
    constexpr int P = QV * QV * QV;
    const T* gcell = GEO == GEO_FLY ? go : static_cast<const T*>(kp.gcv) + (size_t)e0 * 10 * P;
    if (GEO == GEO_FLY) fill_cell_geo<T, N, QV, CB>(sx, ar, tb.eSv, tb.eDv, go, nb, grp);
    T* V0 = ar;
    T* V1 = ar + CB * 5 * P;
    T* V2 = ar + 2 * CB * 5 * P;
    T* V3 = ar + 3 * CB * 5 * P;
    sweep<T, 0, N, N, N, QV, 1, false>(su, V1, tb.eSv, nbl, grp);
    grp.sync();
    sweep<T, 1, QV, N, N, QV, 1, false>(V1, V2, tb.eSv, nbl, grp);
    grp.sync();
    sweep<T, 2, QV, QV, N, QV, 1, false>(V2, V0, tb.eSv, nbl, grp);
    grp.sync();
    // reference gradients by collocation
    sweep<T, 0, QV, QV, QV, QV, -1, false>(V0, V1, tb.eDv, nbl, grp);
    sweep<T, 1, QV, QV, QV, QV, -1, false>(V0, V2, tb.eDv, nbl, grp);
    sweep<T, 2, QV, QV, QV, QV, -1, false>(V0, V3, tb.eDv, nbl, grp);
    grp.sync();
    for (int idx = grp.rank(); idx < nb * P; idx += grp.size()) {
      const int e = idx / P, p = idx - e * P;
      const int q0 = p % QV, q1 = (p / QV) % QV, q2 = p / (QV * QV);
      const T w = tb.wv[q0] * tb.wv[q1] * tb.wv[q2] * detJ;
      T u[5], Gr[5][3], F[5][3];
      T* Vd[3] = {V1, V2, V3};
      if (GEO == GEO_AFFINE) {
#pragma unroll
        for (int c = 0; c < 5; ++c) {
          u[c] = V0[(e * 5 + c) * P + p];
#pragma unroll
          for (int j = 0; j < 3; ++j) Gr[c][j] = Vd[j][(e * 5 + c) * P + p] * hinv[j];
        }
        visc_flux(u, Gr, ph, F);
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          const T s = w * hinv[j];
#pragma unroll
          for (int c = 0; c < 5; ++c) Vd[j][(e * 5 + c) * P + p] = s * F[c][j];
        }
      } else {
        const T* g = gcell + (size_t)e * 10 * P + p;
        T Ji[9];
#pragma unroll
        for (int m = 0; m < 9; ++m) Ji[m] = g[m * P];
        const T jw = g[9 * P] * tb.wv[q0] * tb.wv[q1] * tb.wv[q2];
#pragma unroll
        for (int c = 0; c < 5; ++c) {
          u[c] = V0[(e * 5 + c) * P + p];
          const T g0 = Vd[0][(e * 5 + c) * P + p], g1 = Vd[1][(e * 5 + c) * P + p], g2 = Vd[2][(e * 5 + c) * P + p];
#pragma unroll
          for (int a = 0; a < 3; ++a) Gr[c][a] = Ji[a] * g0 + Ji[3 + a] * g1 + Ji[6 + a] * g2;
        }
        visc_flux(u, Gr, ph, F);
#pragma unroll
        for (int b = 0; b < 3; ++b)
#pragma unroll
          for (int c = 0; c < 5; ++c)
            Vd[b][(e * 5 + c) * P + p] = jw * (Ji[3 * b] * F[c][0] + Ji[3 * b + 1] * F[c][1] + Ji[3 * b + 2] * F[c][2]);
      }
    }
    grp.sync();
    sweep<T, 0, QV, QV, QV, QV, -1, false>(V1, V0, tb.eDvT, nbl, grp);
    grp.sync();
    sweep<T, 1, QV, QV, QV, QV, -1, true>(V2, V0, tb.eDvT, nbl, grp);
    grp.sync();
    sweep<T, 2, QV, QV, QV, QV, -1, true>(V3, V0, tb.eDvT, nbl, grp);
    grp.sync();
    sweep<T, 2, QV, QV, QV, N, 1, false>(V0, V1, tb.eSvT, nbl, grp);
    grp.sync();
    sweep<T, 1, QV, QV, N, N, 1, false>(V1, V2, tb.eSvT, nbl, grp);
    grp.sync();
    sweep<T, 0, QV, N, N, N, 1, true>(V2, sr, tb.eSvT, nbl, grp);
    grp.sync();
  }
}

// ---------------------------------------------------------------------------
// Face integrals of one face (direction d, side s) for the CTA's cells,
// element-centric: the cell's own trace (-) and the neighbour's trace (+)
// give the numerical fluxes, tested with the own basis only.
//   + (V, ({{F_c}} + Lambda/2 [[U]]) . n)                 at QC x QC points
//   - (V, ({{F_v}} - tau [[U]]) . n) - 1/2 (grad V, F_v(U-, [[U]]))   at QV x QV
// su: own nodal state, sn: neighbour nodal state (unused where wall[e]),
// tau_f[e]: face penalty, sr: accumulated residual, fa: face arena.
// ---------------------------------------------------------------------------
template <typename T, int N, int QC, int QV, int CB, int d, int GEO, class G = CtaGroup>
__device__ void face_terms(const T* su, const T* sn, const int* wall, const int* nbi, const T* tau_f, T* sr, T* fa,
                           const Tab<T>& tb, const KParams& kp, const PhysT<T>& ph, int e0, int nb, int s,
                           G grp = G(), const T* sx = nullptr, const T* sxn = nullptr, T* go = nullptr) {
  const int f = 2 * d + s, fo = 2 * d + (1 - s);  // own face, neighbour's face
  constexpr int N2 = N * N, N3 = N * N * N;
  constexpr int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
  const KConst<T>& kc = kconst<T>(kp);
  const T hinv[3] = {kc.hinv[0], kc.hinv[1], kc.hinv[2]};
  const T area = kc.area[d];
  const T sgn = s ? T(1) : T(-1);  // outward unit normal n = sgn e_d
  const int idm = s ? N - 1 : 0, idp = s ? 0 : N - 1;
  const T* dlm = s ? tb.dl1 : tb.dl0;  // l_i' at the own face
  const T* dlp = s ? tb.dl0 : tb.dl1;  // l_i' at the neighbour's face
  const int nbl = nb * 5;

  if (kp.conv) {
    constexpr int P = QC * QC;
    // own face geometry: stored [Nc][6][13][P], or recomputed now into go [CB][13][P] (GEO_FLY)
    const T* gfo = GEO == GEO_FLY ? go : static_cast<const T*>(kp.gfc) + ((size_t)e0 * 6 + f) * 13 * P;
    const size_t gfs = GEO == GEO_FLY ? (size_t)13 * P : (size_t)6 * 13 * P;
    if (GEO == GEO_FLY) fill_face_geo<T, N, QC, CB, d>(sx, s, fa, tb.eSc, tb.eDc, s ? tb.dl1 : tb.dl0, go, nb, grp);
    T* Lm = fa;                   // own face layer      [CB][5][N2]
    T* Lp = Lm + CB * 5 * N2;     // neighbour face layer
    T* Tm = Lp + CB * 5 * N2;     // tmp [CB][5][N][QC]
    T* Um = Tm + CB * 5 * QC * N; // [CB][5][P]
    T* Up = Um + CB * 5 * P;
    for (int idx = grp.rank(); idx < nbl * N2; idx += grp.size()) {
      const int ec = idx / N2, j = idx - ec * N2, e = ec / 5;
      Lm[idx] = su[ec * N3 + face_node<N>(d, idm, j % N, j / N)];
      Lp[idx] = wall[e] ? T(0) : sn[ec * N3 + face_node<N>(d, idp, j % N, j / N)];
    }
    grp.sync();
    sweep<T, 0, N, N, 1, QC, 1, false>(Lm, Tm, tb.eSc, nbl, grp);
    grp.sync();
    sweep<T, 1, QC, N, 1, QC, 1, false>(Tm, Um, tb.eSc, nbl, grp);
    grp.sync();
    sweep<T, 0, N, N, 1, QC, 1, false>(Lp, Tm, tb.eSc, nbl, grp);
    grp.sync();
    sweep<T, 1, QC, N, 1, QC, 1, false>(Tm, Up, tb.eSc, nbl, grp);
    grp.sync();
    for (int idx = grp.rank(); idx < nb * P; idx += grp.size()) {
      const int e = idx / P, p = idx - e * P;
      const T w = tb.wc[p % QC] * tb.wc[p / QC] * area;
      T um[5], up[5];
#pragma unroll
      for (int c = 0; c < 5; ++c) {
        um[c] = Um[(e * 5 + c) * P + p];
        up[c] = Up[(e * 5 + c) * P + p];
      }
      if (wall[e]) wall_ghost(um, ph, up);
      const T rm = T(1) / (ph.rho_r + um[0]), rp = T(1) / (ph.rho_r + up[0]);
      const T pm = pressure_dev(um, rm, ph.gm1), pp = pressure_dev(up, rp, ph.gm1);
      const T lm = sqrt(um[1] * um[1] + um[2] * um[2] + um[3] * um[3]) * rm + sqrt(fabs(ph.gamma * (ph.p_r + pm) * rm));
      const T lp = sqrt(up[1] * up[1] + up[2] * up[2] + up[3] * up[3]) * rp + sqrt(fabs(ph.gamma * (ph.p_r + pp) * rp));
      const T lam = lm > lp ? lm : lp;
      if (GEO == GEO_AFFINE) {
        T fm[5], fp[5];
        conv_flux_dir(um, rm, pm, ph.H_r, d, fm);
        conv_flux_dir(up, rp, pp, ph.H_r, d, fp);
#pragma unroll
        for (int c = 0; c < 5; ++c)
          Um[(e * 5 + c) * P + p] = w * (T(0.5) * sgn * (fm[c] + fp[c]) + T(0.5) * lam * (um[c] - up[c]));
      } else {
        const T* g = gfo + e * gfs + p;
        const T n0 = g[9 * P], n1 = g[10 * P], n2 = g[11 * P];
        const T dw = g[12 * P] * tb.wc[p % QC] * tb.wc[p / QC];
        T fn[5];
#pragma unroll
        for (int c = 0; c < 5; ++c) fn[c] = T(0);
        const T nn[3] = {n0, n1, n2};
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
    sweep<T, 0, QC, N, 1, N, 1, false>(Tm, Lm, tb.eScT, nbl, grp);
    grp.sync();
    for (int idx = grp.rank(); idx < nbl * N2; idx += grp.size()) {
      const int ec = idx / N2, j = idx - ec * N2;
      sr[ec * N3 + face_node<N>(d, idm, j % N, j / N)] += Lm[idx];
    }
    grp.sync();
  }

  if (kp.visc) {
    constexpr int P = QV * QV;
    const T* gfo = GEO == GEO_FLY ? go : static_cast<const T*>(kp.gfv) + ((size_t)e0 * 6 + f) * 13 * P;
    const size_t gfs = GEO == GEO_FLY ? (size_t)13 * P : (size_t)6 * 13 * P;
    T* gnb = go + CB * 13 * P;  // GEO_FLY: the neighbours' face geometry
    if (GEO == GEO_FLY) {
      fill_face_geo<T, N, QV, CB, d>(sx, s, fa, tb.eSv, tb.eDv, s ? tb.dl1 : tb.dl0, go, nb, grp);
      fill_face_geo<T, N, QV, CB, d>(sxn, 1 - s, fa, tb.eSv, tb.eDv, s ? tb.dl0 : tb.dl1, gnb, nb, grp);
    }
    T* Lm = fa;                    // face layers and normal-derivative layers [CB][5][N2]
    T* Lp = Lm + CB * 5 * N2;
    T* Dm = Lp + CB * 5 * N2;
    T* Dp = Dm + CB * 5 * N2;
    T* Tm = Dp + CB * 5 * N2;      // tmp [CB][5][N][QV]
    T* Um = Tm + CB * 5 * QV * N;  // 8 point arrays [CB][5][P]
    T* Up = Um + CB * 5 * P;
    T* G1m = Up + CB * 5 * P;
    T* G2m = G1m + CB * 5 * P;
    T* Gdm = G2m + CB * 5 * P;
    T* G1p = Gdm + CB * 5 * P;
    T* G2p = G1p + CB * 5 * P;
    T* Gdp = G2p + CB * 5 * P;
    for (int idx = grp.rank(); idx < nbl * N2; idx += grp.size()) {
      const int ec = idx / N2, j = idx - ec * N2, e = ec / 5;
      const int j1 = j % N, j2 = j / N;
      const T* um = su + ec * N3;
      Lm[idx] = um[face_node<N>(d, idm, j1, j2)];
      T dn = T(0);
#pragma unroll
      for (int i = 0; i < N; ++i) dn += dlm[i] * um[face_node<N>(d, i, j1, j2)];
      Dm[idx] = dn;
      if (wall[e]) {
        Lp[idx] = T(0);
        Dp[idx] = T(0);
      } else {
        const T* un = sn + ec * N3;
        Lp[idx] = un[face_node<N>(d, idp, j1, j2)];
        T dp = T(0);
#pragma unroll
        for (int i = 0; i < N; ++i) dp += dlp[i] * un[face_node<N>(d, i, j1, j2)];
        Dp[idx] = dp;
      }
    }
    grp.sync();
    // values and normal derivatives to the face Gauss points
    sweep<T, 0, N, N, 1, QV, 1, false>(Lm, Tm, tb.eSv, nbl, grp);
    grp.sync();
    sweep<T, 1, QV, N, 1, QV, 1, false>(Tm, Um, tb.eSv, nbl, grp);
    grp.sync();
    sweep<T, 0, N, N, 1, QV, 1, false>(Lp, Tm, tb.eSv, nbl, grp);
    grp.sync();
    sweep<T, 1, QV, N, 1, QV, 1, false>(Tm, Up, tb.eSv, nbl, grp);
    grp.sync();
    sweep<T, 0, N, N, 1, QV, 1, false>(Dm, Tm, tb.eSv, nbl, grp);
    grp.sync();
    sweep<T, 1, QV, N, 1, QV, 1, false>(Tm, Gdm, tb.eSv, nbl, grp);
    grp.sync();
    sweep<T, 0, N, N, 1, QV, 1, false>(Dp, Tm, tb.eSv, nbl, grp);
    grp.sync();
    sweep<T, 1, QV, N, 1, QV, 1, false>(Tm, Gdp, tb.eSv, nbl, grp);
    // tangential derivatives by collocation on the face grid
    sweep<T, 0, QV, QV, 1, QV, -1, false>(Um, G1m, tb.eDv, nbl, grp);
    sweep<T, 1, QV, QV, 1, QV, -1, false>(Um, G2m, tb.eDv, nbl, grp);
    sweep<T, 0, QV, QV, 1, QV, -1, false>(Up, G1p, tb.eDv, nbl, grp);
    sweep<T, 1, QV, QV, 1, QV, -1, false>(Up, G2p, tb.eDv, nbl, grp);
    grp.sync();
    for (int idx = grp.rank(); idx < nb * P; idx += grp.size()) {
      const int e = idx / P, p = idx - e * P;
      const T w = tb.wv[p % QV] * tb.wv[p / QV] * area;
      const int o = e * 5 * P + p;
      T um[5], up[5], Gm[5][3], Gp[5][3];
      T nrm[3] = {T(0), T(0), T(0)};
      T Jm[9];
      T wgt = w;
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
        // reference derivative directions: t1, t2, d  ->  physical G[c][a] = sum_b J^{-1}[b][a] g_b
        const T* g = gfo + e * gfs + p;
#pragma unroll
        for (int m = 0; m < 9; ++m) Jm[m] = g[m * P];
        nrm[0] = g[9 * P];
        nrm[1] = g[10 * P];
        nrm[2] = g[11 * P];
        wgt = g[12 * P] * tb.wv[p % QV] * tb.wv[p / QV];
        T Jp[9];
        if (!wall[e]) {
          if (GEO == GEO_STORED && kp.fnbr) {
            frame_face_jinv<T, QV>(static_cast<const T*>(kp.gfv), nbi[e], kp.fnbr[((size_t)(e0 + e) * 6 + f) * 2 + 1],
                                   d, s, p, Jp);
          } else {
            const T* gp = GEO == GEO_FLY ? gnb + (size_t)e * 13 * P + p
                                         : static_cast<const T*>(kp.gfv) + ((size_t)nbi[e] * 6 + fo) * 13 * P + p;
#pragma unroll
            for (int m = 0; m < 9; ++m) Jp[m] = gp[m * P];
          }
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
      if (wall[e]) {
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
        // -(V, Q*.n):  Q*.n = {{F_v}}.n - tau (U- - U+)
        const T fvn = (Fm[c][0] + Fp[c][0]) * nrm[0] + (Fm[c][1] + Fp[c][1]) * nrm[1] + (Fm[c][2] + Fp[c][2]) * nrm[2];
        Um[o + c * P] = -wgt * (T(0.5) * fvn - tau * jmp[c]);
      }
      // -1/2 (grad V, F_v(U-, [[U]])) with [[U]] = (U- - U+) (x) n
      T Jg[5][3];
#pragma unroll
      for (int c = 0; c < 5; ++c)
#pragma unroll
        for (int a = 0; a < 3; ++a) Jg[c][a] = jmp[c] * nrm[a];
      visc_flux(um, Jg, ph, Fm);
      const T hw = T(-0.5) * wgt;
      if (GEO == GEO_AFFINE) {
#pragma unroll
        for (int c = 0; c < 5; ++c) {
          G1m[o + c * P] = hw * hinv[t1] * Fm[c][t1];
          G2m[o + c * P] = hw * hinv[t2] * Fm[c][t2];
          Gdm[o + c * P] = hw * hinv[d] * Fm[c][d];
        }
      } else {
#pragma unroll
        for (int c = 0; c < 5; ++c) {
          G1m[o + c * P] = hw * (Jm[3 * t1] * Fm[c][0] + Jm[3 * t1 + 1] * Fm[c][1] + Jm[3 * t1 + 2] * Fm[c][2]);
          G2m[o + c * P] = hw * (Jm[3 * t2] * Fm[c][0] + Jm[3 * t2 + 1] * Fm[c][1] + Jm[3 * t2 + 2] * Fm[c][2]);
          Gdm[o + c * P] = hw * (Jm[3 * d] * Fm[c][0] + Jm[3 * d + 1] * Fm[c][1] + Jm[3 * d + 2] * Fm[c][2]);
        }
      }
    }
    grp.sync();
    // value test + tangential gradient tests on the face grid
    sweep<T, 0, QV, QV, 1, QV, -1, true>(G1m, Um, tb.eDvT, nbl, grp);
    grp.sync();
    sweep<T, 1, QV, QV, 1, QV, -1, true>(G2m, Um, tb.eDvT, nbl, grp);
    grp.sync();
    sweep<T, 1, QV, QV, 1, N, 1, false>(Um, Tm, tb.eSvT, nbl, grp);
    grp.sync();
    sweep<T, 0, QV, N, 1, N, 1, false>(Tm, Lm, tb.eSvT, nbl, grp);
    grp.sync();
    // normal gradient test
    sweep<T, 1, QV, QV, 1, N, 1, false>(Gdm, Tm, tb.eSvT, nbl, grp);
    grp.sync();
    sweep<T, 0, QV, N, 1, N, 1, false>(Tm, Dm, tb.eSvT, nbl, grp);
    grp.sync();
    for (int idx = grp.rank(); idx < nbl * N2; idx += grp.size()) {
      const int ec = idx / N2, j = idx - ec * N2;
      const int j1 = j % N, j2 = j / N;
      const T lv = Lm[idx], dv = Dm[idx];
      T* r = sr + ec * N3;
#pragma unroll
      for (int i = 0; i < N; ++i) {
        T add = dlm[i] * dv;
        if (i == idm) add += lv;
        r[face_node<N>(d, i, j1, j2)] += add;
      }
    }
    grp.sync();
  }
}

// ---------------------------------------------------------------------------
// L = M^{-1}(-R + F_rhs) in place on sr (Sec. 2.3: the LGL-to-Gauss matrix S at
// the k+1 mass points is square, so M_e^{-1} = S^{-1} diag(1/(|J| w)) S^{-T});
// with the body force integrated at the same points, M^{-1}(V, F_rhs) =
// S^{-1} F_rhs(x_q) (nodal coefficients of its Gauss-point interpolant).
// su is needed only for the body force (u at the mass points).
// ---------------------------------------------------------------------------
template <typename T, int N, int CB, int GEO, class G = CtaGroup>
__device__ void inverse_mass(const T* su, T* sr, T* ma, const Tab<T>& tb, const KParams& kp, int e0, int nb,
                             bool negate, bool add_force, G grp = G(), const T* sx = nullptr, T* go = nullptr,
                             const T* sin = nullptr) {
  // sin: optional separate input (default: sr, overwritten by the result)
  if (GEO == GEO_FLY) fill_mass_geo<T, N, CB>(sx, ma, tb.eSm, tb.eDm, go, nb, grp);
  constexpr int N3 = N * N * N;
  const int nbl = nb * 5;
  T* A = ma;
  T* B = ma + CB * 5 * N3;
  const T detJ = kconst<T>(kp).detJ;
  sweep<T, 0, N, N, N, N, 1, false>(sin ? sin : sr, A, tb.eSmiT, nbl, grp);
  grp.sync();
  sweep<T, 1, N, N, N, N, 1, false>(A, B, tb.eSmiT, nbl, grp);
  grp.sync();
  sweep<T, 2, N, N, N, N, 1, false>(B, A, tb.eSmiT, nbl, grp);
  grp.sync();
  const T sg = negate ? T(-1) : T(1);
  for (int idx = grp.rank(); idx < nbl * N3; idx += grp.size()) {
    const int p = idx % N3;
    T w;
    if (GEO == GEO_AFFINE)
      w = tb.wm[p % N] * tb.wm[(p / N) % N] * tb.wm[p / (N * N)] * detJ;
    else
      w = tb.wm[p % N] * tb.wm[(p / N) % N] * tb.wm[p / (N * N)] *
          (GEO == GEO_FLY ? go[(size_t)(idx / (5 * N3)) * N3 + p]
                          : static_cast<const T*>(kp.gm)[(size_t)(e0 + idx / (5 * N3)) * N3 + p]);
    A[idx] *= sg / w;
  }
  grp.sync();
  sweep<T, 0, N, N, N, N, 1, false>(A, B, tb.eSmi, nbl, grp);
  grp.sync();
  sweep<T, 1, N, N, N, N, 1, false>(B, A, tb.eSmi, nbl, grp);
  grp.sync();
  sweep<T, 2, N, N, N, N, 1, false>(A, sr, tb.eSmi, nbl, grp);
  grp.sync();
  if (add_force) {
    // F_rhs = (0, f, f.u): momentum rows are the constant f (S^{-1} 1 = 1), energy row S^{-1}(f . u)(x_q)
    const T f0 = kconst<T>(kp).bf[0], f1 = kconst<T>(kp).bf[1], f2 = kconst<T>(kp).bf[2];
    // interpolate rho and momenta (components 0..3) to the mass points
    for (int e = 0; e < nb; ++e) {
      sweep<T, 0, N, N, N, N, 1, false>(su + e * 5 * N3, A + e * 4 * N3, tb.eSm, 4, grp);
    }
    grp.sync();
    for (int e = 0; e < nb; ++e) sweep<T, 1, N, N, N, N, 1, false>(A + e * 4 * N3, B + e * 4 * N3, tb.eSm, 4, grp);
    grp.sync();
    for (int e = 0; e < nb; ++e) sweep<T, 2, N, N, N, N, 1, false>(B + e * 4 * N3, A + e * 4 * N3, tb.eSm, 4, grp);
    grp.sync();
    for (int idx = grp.rank(); idx < nb * N3; idx += grp.size()) {
      const int e = idx / N3, p = idx - e * N3;
      const T* a = A + e * 4 * N3;
      B[idx] = (f0 * a[N3 + p] + f1 * a[2 * N3 + p] + f2 * a[3 * N3 + p]) / (kconst<T>(kp).rho_r + a[p]);
    }
    grp.sync();
    sweep<T, 0, N, N, N, N, 1, false>(B, A, tb.eSmi, nb, grp);
    grp.sync();
    sweep<T, 1, N, N, N, N, 1, false>(A, B, tb.eSmi, nb, grp);
    grp.sync();
    sweep<T, 2, N, N, N, N, 1, false>(B, A, tb.eSmi, nb, grp);
    grp.sync();
    for (int idx = grp.rank(); idx < nb * N3; idx += grp.size()) {
      const int e = idx / N3, p = idx - e * N3;
      T* r = sr + e * 5 * N3;
      r[N3 + p] += f0;
      r[2 * N3 + p] += f1;
      r[3 * N3 + p] += f2;
      r[4 * N3 + p] += A[idx];
    }
    grp.sync();
  }
}

// 2N update of a batch: dU <- A dU + dt L (residual type), U_out <- U + B dU (FP64); the loads of U and
// dU of a thread are issued together before the stores.  With kp.devOut (mixed form inside a
// multi-step call) also float(U_out - U_ref), the deviation state the next stage reads.
template <int PER, int N3, typename T>
__device__ __forceinline__ void stage_update(const KParams& kp, const double* U, T* dU, double* Uout, const T* sr,
                                             size_t base, int nvals, int rank, int stride) {
  struct UD {
    double u;
    T d;
  };
  const T A = T(kp.A), dt = T(kp.dt);
  const double B = kp.B;
  const bool readD = kp.A != 0.0;
  T* dev = static_cast<T*>(kp.devOut);
  batched_pass<PER>(rank, stride, nvals,
                    [&](int i) { return UD{U[base + i], readD ? dU[base + i] : T(0)}; },
                    [&](int i, UD v) {
                      const T du = A * v.d + dt * sr[i];
                      dU[base + i] = du;
                      const double uo = v.u + B * double(du);
                      Uout[base + i] = uo;
                      if (dev) {
                        const int c = (i / N3) % 5;
                        dev[base + i] = T(uo - (c == 0 ? kp.rho_ref : (c == 4 ? kp.rhoE_ref : 0.0)));
                      }
                    });
}

}  // namespace dgcns
