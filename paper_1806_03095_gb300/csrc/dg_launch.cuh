// Kernels and launchers of libdgcns for one (N = k+1, QC, QV) instantiation.
// Included by the per-configuration translation units (dg_inst.cu).
#pragma once
#include <cuda_runtime.h>

#include "dg_kernels.cuh"
#include "dg_launchers.h"

namespace dgcns {

constexpr int NT = 128;  // threads per CTA

// Cells per CTA: the largest batch (<= 8) whose shared memory stays below ~112 KB,
// so that two CTAs fit on one SM (228 KB).
template <typename T, int N, int QC, int QV>
constexpr int cells_per_cta() {
  using S = Sizes<N, QC, QV>;
  constexpr int arena = S::CELL_ARENA > S::FACE_ARENA ? S::CELL_ARENA : S::FACE_ARENA;
  constexpr int per_cell = (3 * 5 * S::N3 + arena) * (int)sizeof(T) + 8;
  constexpr int cb = (112 * 1024 - table_elems<N, QC, QV>() * (int)sizeof(T)) / per_cell;
  return cb < 1 ? 1 : (cb > 8 ? 8 : cb);
}

template <typename T, int N, int QC, int QV, int CB, bool CELL, bool FACE, bool MASS>
constexpr size_t op_smem_bytes() {
  using S = Sizes<N, QC, QV>;
  size_t arena = 0;
  if (CELL) arena = (size_t)CB * S::CELL_ARENA;
  if (FACE && (size_t)CB * S::FACE_ARENA > arena) arena = (size_t)CB * S::FACE_ARENA;
  if (MASS && (size_t)CB * S::MASS_ARENA > arena) arena = (size_t)CB * S::MASS_ARENA;
  const size_t elems = table_elems<N, QC, QV>() + (size_t)CB * 5 * S::N3 * (FACE ? 3 : 2) + arena + 2 * CB;
  return elems * sizeof(T) + 2 * CB * sizeof(int) + 64;
}

// component c of the reference state U_ref = (rho_r, 0, 0, 0, rho_r c_v T_0)
__device__ __forceinline__ double ref_of(const KParams& kp, int c) {
  return c == 0 ? kp.rho_ref : (c == 4 ? kp.rhoE_ref : 0.0);
}

// ---------------------------------------------------------------------------
// Generic operator kernel.  CELL: cell integrals; FACE: the 6 face integrals of
// every cell; MASS: L = M^{-1}(-R + F_rhs).  Without CELL the partial residual
// is read from Rin.  Output (kp.out_mode): 0 write R, 1 write L, 2 RK stage
// dU <- A dU + dt L, U_out <- U + B dU.
// ---------------------------------------------------------------------------
template <typename T, int N, int QC, int QV, int CB, bool CELL, bool FACE, bool MASS>
__global__ void __launch_bounds__(NT) dg_op_kernel(const KParams kp, const double* __restrict__ U,
                                                   const T* Rin, T* Rout, T* dU, double* Uout) {
  using S = Sizes<N, QC, QV>;
  constexpr int N3 = S::N3;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  T* stab = sm;
  T* su = stab + table_elems<N, QC, QV>();
  T* sr = su + CB * 5 * N3;
  T* sn = sr + CB * 5 * N3;
  T* ar = sn + (FACE ? CB * 5 * N3 : 0);
  size_t arena = 0;
  if (CELL) arena = (size_t)CB * S::CELL_ARENA;
  if (FACE && (size_t)CB * S::FACE_ARENA > arena) arena = (size_t)CB * S::FACE_ARENA;
  if (MASS && (size_t)CB * S::MASS_ARENA > arena) arena = (size_t)CB * S::MASS_ARENA;
  T* tau_f = ar + arena;
  int* wall = reinterpret_cast<int*>(tau_f + CB);
  int* nbi = wall + CB;

  const int e0 = blockIdx.x * CB;
  const int nb = min(CB, kp.Nc - e0);
  if (nb <= 0) return;
  const Tab<T> tb = load_tables<T, N, QC, QV>(static_cast<const T*>(kp.tables), stab);
  PhysT<T> ph;
  ph.gamma = T(kp.gamma);
  ph.gm1 = T(kp.gamma - 1.0);
  ph.mu = T(kp.mu);
  ph.lam_cv = T(kp.lam / kp.cv);
  ph.rho_r = T(kp.rho_ref);
  ph.rhoE_r = T(kp.rhoE_ref);
  ph.p_r = T((kp.gamma - 1.0) * kp.rhoE_ref);
  ph.H_r = T(kp.gamma * kp.rhoE_ref);
  ph.cvTw2 = T(2.0 * kp.cv * kp.Tw);

  const size_t base = (size_t)e0 * 5 * N3;
  const int nvals = nb * 5 * N3;
  const bool need_u = CELL || FACE || (MASS && kp.has_bf);
  for (int i = threadIdx.x; i < nvals; i += blockDim.x) {
    if (need_u) su[i] = T(U[base + i] - ref_of(kp, (i / N3) % 5));
    sr[i] = CELL ? T(0) : Rin[base + i];
  }
  __syncthreads();

  if (CELL) cell_terms<T, N, QC, QV, CB>(su, sr, ar, tb, kp, ph, nb);

  if (FACE) {
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
          if (!wall[e]) sn[i] = T(U[(size_t)nbi[e] * 5 * N3 + (i - e * 5 * N3)] - ref_of(kp, (i / N3) % 5));
        }
        __syncthreads();
        if (d == 0) face_terms<T, N, QC, QV, CB, 0>(su, sn, wall, tau_f, sr, ar, tb, kp, ph, nb, s);
        if (d == 1) face_terms<T, N, QC, QV, CB, 1>(su, sn, wall, tau_f, sr, ar, tb, kp, ph, nb, s);
        if (d == 2) face_terms<T, N, QC, QV, CB, 2>(su, sn, wall, tau_f, sr, ar, tb, kp, ph, nb, s);
      }
    }
  }

  if (MASS) inverse_mass<T, N, CB>(su, sr, ar, tb, kp, nb, CELL || FACE || kp.out_mode != 0, kp.has_bf != 0);

  if (kp.out_mode == 2) {
    const double A = kp.A, B = kp.B, dt = kp.dt;
    for (int i = threadIdx.x; i < nvals; i += blockDim.x) {
      const double du_old = A != 0.0 ? double(dU[base + i]) : 0.0;
      const T du = T(A * du_old + dt * double(sr[i]));
      dU[base + i] = du;
      Uout[base + i] = U[base + i] + B * double(du);
    }
  } else {
    for (int i = threadIdx.x; i < nvals; i += blockDim.x) Rout[base + i] = sr[i];
  }
}

// ---------------------------------------------------------------------------
// Diagnostics (always FP64): per-CTA partial sums of
//   [vol, int |u|^2/2, int grad u : grad u, int u.(dm/dt - u drho/dt)/rho, int U (5), nonfinite]
// ---------------------------------------------------------------------------
constexpr int NACC = 10;

template <typename TL, int N, int QC, int QV, int CB>
__global__ void __launch_bounds__(NT) dg_diag_kernel(const KParams kp, const double* __restrict__ U,
                                                     const TL* __restrict__ LU, double* __restrict__ partial) {
  constexpr int N3 = N * N * N, P = QC * QC * QC;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* sm = reinterpret_cast<double*>(smem_raw);
  double* stab = sm;
  double* su = stab + table_elems<N, QC, QV>();
  double* sl = su + CB * 5 * N3;
  double* V0 = sl + CB * 5 * N3;   // values at the Gauss points
  double* V1 = V0 + CB * 5 * P;    // temporaries / one gradient direction
  double* V2 = V1 + CB * 5 * P;
  double* L0 = V2 + CB * 5 * P;    // L(U) at the Gauss points
  double* red = L0 + CB * 5 * P;   // [NT][NACC]
  const Tab<double> tb = load_tables<double, N, QC, QV>(static_cast<const double*>(kp.tables), stab);
  const int e0 = blockIdx.x * CB;
  const int nb = min(CB, kp.Nc - e0);
  double acc[NACC];
#pragma unroll
  for (int a = 0; a < NACC; ++a) acc[a] = 0.0;
  if (nb > 0) {
    const size_t base = (size_t)e0 * 5 * N3;
    const int nvals = nb * 5 * N3;
    for (int i = threadIdx.x; i < nvals; i += blockDim.x) {
      const double v = U[base + i];
      su[i] = v;
      if (!isfinite(v)) acc[9] += 1.0;
      sl[i] = LU ? double(LU[base + i]) : 0.0;
    }
    __syncthreads();
    const int nbl = nb * 5;
    sweep<double, 0, N, N, N, QC, 1, false>(su, V1, tb.eSc, nbl);
    __syncthreads();
    sweep<double, 1, QC, N, N, QC, 1, false>(V1, V2, tb.eSc, nbl);
    __syncthreads();
    sweep<double, 2, QC, QC, N, QC, 1, false>(V2, V0, tb.eSc, nbl);
    __syncthreads();
    if (LU) {
      sweep<double, 0, N, N, N, QC, 1, false>(sl, V1, tb.eSc, nbl);
      __syncthreads();
      sweep<double, 1, QC, N, N, QC, 1, false>(V1, V2, tb.eSc, nbl);
      __syncthreads();
      sweep<double, 2, QC, QC, N, QC, 1, false>(V2, L0, tb.eSc, nbl);
      __syncthreads();
    }
    const double detJ = kp.h[0] * kp.h[1] * kp.h[2];
    const double hinv[3] = {1.0 / kp.h[0], 1.0 / kp.h[1], 1.0 / kp.h[2]};
    for (int idx = threadIdx.x; idx < nb * P; idx += blockDim.x) {
      const int e = idx / P, p = idx - e * P;
      const double w = tb.wc[p % QC] * tb.wc[(p / QC) % QC] * tb.wc[p / (QC * QC)] * detJ;
      const int o = e * 5 * P + p;
      const double rinv = 1.0 / V0[o];
      const double u[3] = {V0[o + P] * rinv, V0[o + 2 * P] * rinv, V0[o + 3 * P] * rinv};
      acc[0] += w;
      acc[1] += 0.5 * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]) * w;
      if (LU) {
        double s = 0.0;
#pragma unroll
        for (int i = 0; i < 3; ++i) s += u[i] * (L0[o + (1 + i) * P] - u[i] * L0[o]) * rinv;
        acc[3] += s * w;
      }
    }
    // grad u : grad u, one reference direction at a time (the sum over j separates)
#pragma unroll 1
    for (int j = 0; j < 3; ++j) {
      __syncthreads();
      if (j == 0) sweep<double, 0, QC, QC, QC, QC, -1, false>(V0, V1, tb.eDc, nbl);
      if (j == 1) sweep<double, 1, QC, QC, QC, QC, -1, false>(V0, V1, tb.eDc, nbl);
      if (j == 2) sweep<double, 2, QC, QC, QC, QC, -1, false>(V0, V1, tb.eDc, nbl);
      __syncthreads();
      for (int idx = threadIdx.x; idx < nb * P; idx += blockDim.x) {
        const int e = idx / P, p = idx - e * P;
        const double w = tb.wc[p % QC] * tb.wc[(p / QC) % QC] * tb.wc[p / (QC * QC)] * detJ;
        const int o = e * 5 * P + p;
        const double rinv = 1.0 / V0[o];
        const double gr = V1[o] * hinv[j];
        double gg = 0.0;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          const double ui = V0[o + (1 + i) * P] * rinv;
          const double gui = (V1[o + (1 + i) * P] * hinv[j] - ui * gr) * rinv;
          gg += gui * gui;
        }
        acc[2] += gg * w;
      }
    }
    __syncthreads();
    // conservation totals with the k+1 point rule: int U = sum_q U(x_q) |J| w_q
    sweep<double, 0, N, N, N, N, 1, false>(su, V1, tb.eSm, nbl);
    __syncthreads();
    sweep<double, 1, N, N, N, N, 1, false>(V1, V2, tb.eSm, nbl);
    __syncthreads();
    sweep<double, 2, N, N, N, N, 1, false>(V2, V1, tb.eSm, nbl);
    __syncthreads();
    for (int idx = threadIdx.x; idx < nbl * N3; idx += blockDim.x) {
      const int c = (idx / N3) % 5, p = idx % N3;
      const double w = tb.wm[p % N] * tb.wm[(p / N) % N] * tb.wm[p / (N * N)] * detJ;
      acc[4 + c] += V1[idx] * w;
    }
  }
  // deterministic block reduction
  __syncthreads();
#pragma unroll
  for (int a = 0; a < NACC; ++a) red[threadIdx.x * NACC + a] = acc[a];
  __syncthreads();
  if (threadIdx.x < NACC) {
    double s = 0.0;
    for (int t = 0; t < blockDim.x; ++t) s += red[t * NACC + threadIdx.x];
    partial[(size_t)blockIdx.x * NACC + threadIdx.x] = s;
  }
}

template <int N, int QC, int QV, int CB>
constexpr size_t diag_smem_bytes() {
  constexpr int N3 = N * N * N, P = QC * QC * QC;
  return (table_elems<N, QC, QV>() + 2 * CB * 5 * N3 + 4 * CB * 5 * P + NT * NACC) * sizeof(double) + 64;
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
template <typename T, int N, int QC, int QV, int CB, bool CELL, bool FACE, bool MASS>
int launch_op(const KParams& kp, const double* U, const void* Rin, void* Rout, void* dU, double* Uout,
              cudaStream_t st) {
  auto k = dg_op_kernel<T, N, QC, QV, CB, CELL, FACE, MASS>;
  constexpr size_t smem = op_smem_bytes<T, N, QC, QV, CB, CELL, FACE, MASS>();
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return -1;
    attr = true;
  }
  const int grid = (kp.Nc + CB - 1) / CB;
  k<<<grid, NT, smem, st>>>(kp, U, static_cast<const T*>(Rin), static_cast<T*>(Rout), static_cast<T*>(dU), Uout);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

template <typename T, int N, int QC, int QV>
int op_dispatch(int mode, const KParams& kp, const double* U, const void* Rin, void* Rout, void* dU, double* Uout,
                cudaStream_t st) {
  constexpr int CB = cells_per_cta<T, N, QC, QV>();
  switch (mode) {
    case OP_CELL: return launch_op<T, N, QC, QV, CB, true, false, false>(kp, U, Rin, Rout, dU, Uout, st);
    case OP_FACE: return launch_op<T, N, QC, QV, CB, false, true, false>(kp, U, Rin, Rout, dU, Uout, st);
    case OP_MASS: return launch_op<T, N, QC, QV, CB, false, false, true>(kp, U, Rin, Rout, dU, Uout, st);
    case OP_CELL | OP_FACE: return launch_op<T, N, QC, QV, CB, true, true, false>(kp, U, Rin, Rout, dU, Uout, st);
    case OP_CELL | OP_FACE | OP_MASS:
      return launch_op<T, N, QC, QV, CB, true, true, true>(kp, U, Rin, Rout, dU, Uout, st);
    default: return -2;
  }
}

template <typename TL, int N, int QC, int QV>
int diag_launch(const KParams& kp, const double* U, const void* LU, double* partial, int* nblocks,
                cudaStream_t st) {
  constexpr int CB = QC * QC * QC > 300 ? 1 : 2;
  auto k = dg_diag_kernel<TL, N, QC, QV, CB>;
  constexpr size_t smem = diag_smem_bytes<N, QC, QV, CB>();
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return -1;
    attr = true;
  }
  const int grid = (kp.Nc + CB - 1) / CB;
  *nblocks = grid;
  if (partial == nullptr) return 0;
  k<<<grid, NT, smem, st>>>(kp, U, static_cast<const TL*>(LU), partial);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

template <int N, int QC, int QV>
Launchers make_launchers() {
  Launchers L;
  L.op_fp64 = op_dispatch<double, N, QC, QV>;
  L.op_fp32 = op_dispatch<float, N, QC, QV>;
  L.diag_fp64 = diag_launch<double, N, QC, QV>;
  L.diag_fp32 = diag_launch<float, N, QC, QV>;
  L.cb_fp64 = cells_per_cta<double, N, QC, QV>();
  L.cb_fp32 = cells_per_cta<float, N, QC, QV>();
  return L;
}

}  // namespace dgcns
