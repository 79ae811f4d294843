// Kernels and launchers of libdgcns for one (N = k+1, QC, QV) instantiation.
// Included by the per-configuration translation units (dg_inst.cu).
#pragma once
#include <cuda_runtime.h>

#include "dg_adjoint.cuh"
#include "dg_adjoint_faces.cuh"
#include "dg_faces.cuh"
#include "dg_cell_fp32.cuh"
#include "dg_faces_fp32.cuh"
#include "dg_kernels.cuh"
#include "dg_mass.cuh"
#include "dg_launchers.h"

namespace dgcns {


// Batch caps of the CTA-wide kernels (compile-time tuning parameters: cells per CTA of the FP64
// operator kernel, faces per CTA of the FP64 face kernel; 4 faces per CTA were 3 % slower than 8).
#ifndef DGCNS_FP64_CELL_CAP
#define DGCNS_FP64_CELL_CAP 8
#endif
#ifndef DGCNS_FP64_FACE_CAP
#define DGCNS_FP64_FACE_CAP 8
#endif
#ifndef DGCNS_FP64_FACE_THREADS
#define DGCNS_FP64_FACE_THREADS 256
#endif
// FP32 affine face terms at k = 3 by the register-resident task kernel (dg_faces_fp32.cuh); 0 keeps the
// warp-per-face kernel (for comparison)
#ifndef DGCNS_FP32_TASK_FACES
#define DGCNS_FP32_TASK_FACES 1
#endif
// FP32 affine face-centric cell + mass stage at k = 3 by the register-resident task kernel
// (dg_cell_fp32.cuh); 0 keeps the warp-per-cell kernel (for comparison)
#ifndef DGCNS_FP32_TASK_CELL
#define DGCNS_FP32_TASK_CELL 1
#endif

// Cells per CTA: the largest batch (<= 4 for FP32, <= DGCNS_FP64_CELL_CAP for FP64) whose shared
// memory stays below ~112 KB, so that two or more CTAs fit on one SM (228 KB).
template <typename T, int N, int QC, int QV, bool FACE = false>
constexpr int cells_per_cta() {
  using S = Sizes<N, QC, QV>;
  constexpr int arena = S::CELL_ARENA > S::FACE_ARENA ? S::CELL_ARENA : S::FACE_ARENA;
  constexpr int per_cell = (3 * 5 * S::N3 + arena) * (int)sizeof(T) + 8;
  constexpr int cb = (112 * 1024 - table_elems<N, QC, QV>() * (int)sizeof(T)) / per_cell;
  // FP64 at k >= 3 without element-centric faces: 2 cells per CTA (4 CTAs per SM hide more latency than
  // 4 cells in 2 CTAs: the face-centric cell + stage kernel at k = 3 is 2.5 % faster, measured; the fused
  // kernel is 9 % slower with 2 cells, so it keeps the larger batch)
  constexpr int cap = sizeof(T) == 4 ? 4
                                     : (!FACE && N >= 4 && DGCNS_FP64_CELL_CAP > 2 ? 2 : DGCNS_FP64_CELL_CAP);
  return cb < 1 ? 1 : (cb > cap ? cap : cb);
}

// Threads per CTA of the operator kernel: the FP32 form needs more warps per SM to
// hide latency (its FMA pipe is 64x wider than the FP64 one).
template <typename T>
constexpr int op_threads() {
  return sizeof(T) == 4 ? 256 : 128;
}

// Deviation state U - U_ref in the arithmetic type (elementwise pre-pass of the mixed form).
template <typename T>
__global__ void dg_dev_kernel(const KParams kp, const double* __restrict__ U, T* __restrict__ D, size_t n, int N3) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int c = (int)((i / N3) % 5);
    D[i] = T(U[i] - (c == 0 ? kp.rho_ref : (c == 4 ? kp.rhoE_ref : 0.0)));
  }
}

template <int N, int QC, int QV, int CB, bool CELL, bool FACE, bool MASS, int GEO>
constexpr size_t op_arena_elems() {
  using S = Sizes<N, QC, QV>;
  size_t arena = 0;
  if (CELL) arena = (size_t)CB * S::CELL_ARENA;
  if (FACE && (size_t)CB * S::FACE_ARENA > arena) arena = (size_t)CB * S::FACE_ARENA;
  if (MASS && (size_t)CB * S::MASS_ARENA > arena) arena = (size_t)CB * S::MASS_ARENA;
  if (GEO == GEO_FLY && (size_t)CB * S::FLY_TMP > arena) arena = (size_t)CB * S::FLY_TMP;
  return (arena + 3) & ~(size_t)3;
}

// GEO_FLY: own and neighbour node coordinates [CB][3][N^3] and the per-phase geometry outputs
template <int N, int QC, int QV, int CB, bool FACE, int GEO>
constexpr size_t op_geo_elems() {
  using S = Sizes<N, QC, QV>;
  return GEO == GEO_FLY ? (size_t)CB * (3 * S::N3 * (FACE ? 2 : 1) + S::FLY_OUT) : 0;
}

template <typename T, int N, int QC, int QV, int CB, bool CELL, bool FACE, bool MASS, int GEO>
constexpr size_t op_smem_bytes() {
  using S = Sizes<N, QC, QV>;
  const size_t elems = table_elems<N, QC, QV>() + (size_t)CB * 5 * S::N3 * (FACE ? 3 : 2) +
                       op_arena_elems<N, QC, QV, CB, CELL, FACE, MASS, GEO>() +
                       op_geo_elems<N, QC, QV, CB, FACE, GEO>() + 2 * CB;
  return elems * sizeof(T) + 2 * CB * sizeof(int) + 64;
}

// Per-CTA working set of the operator kernel (everything but the 1D tables), slices 256-byte aligned.
// Where it does not fit shared memory next to the tables (at high degrees one cell's arena alone is
// 15-20 q^3 values), it lives in the context's global workspace kp.gws instead, cached by L1 and L2.
template <typename T, int N, int QC, int QV, int CB, bool CELL, bool FACE, bool MASS, int GEO>
constexpr size_t op_work_elems() {
  using S = Sizes<N, QC, QV>;
  const size_t e = (size_t)CB * 5 * S::N3 * (FACE ? 3 : 2) + op_arena_elems<N, QC, QV, CB, CELL, FACE, MASS, GEO>() +
                   op_geo_elems<N, QC, QV, CB, FACE, GEO>() + 4 * CB + 8;
  return (e + 31) & ~(size_t)31;
}

template <typename T, int N, int QC, int QV, int CB, bool CELL, bool FACE, bool MASS, int GEO>
constexpr bool op_gws() {
  return op_smem_bytes<T, N, QC, QV, CB, CELL, FACE, MASS, GEO>() > 227 * 1024;
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
template <typename T, int N, int QC, int QV, int CB, bool CELL, bool FACE, bool MASS, int GEO>
__global__ void __launch_bounds__(op_threads<T>()) dg_op_kernel(const KParams kp, const double* __restrict__ U,
                                                   const T* Rin, T* Rout, T* dU, double* Uout) {
  using S = Sizes<N, QC, QV>;
  constexpr int N3 = S::N3;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  T* stab = sm;
  T* su = stab + table_elems<N, QC, QV>();
  if constexpr (op_gws<T, N, QC, QV, CB, CELL, FACE, MASS, GEO>())  // this CTA's slice of the global workspace
    su = static_cast<T*>(kp.gws) + (size_t)blockIdx.x * op_work_elems<T, N, QC, QV, CB, CELL, FACE, MASS, GEO>();
  T* sr = su + CB * 5 * N3;
  T* sn = sr + CB * 5 * N3;
  T* ar = sn + (FACE ? CB * 5 * N3 : 0);
  T* sx = ar + op_arena_elems<N, QC, QV, CB, CELL, FACE, MASS, GEO>();  // GEO_FLY only
  T* sxn = sx + CB * 3 * N3;
  T* go = sxn + (FACE ? CB * 3 * N3 : 0);
  T* tau_f = sx + op_geo_elems<N, QC, QV, CB, FACE, GEO>();
  int* wall = reinterpret_cast<int*>(tau_f + CB);
  int* nbi = wall + CB;

  const int e0 = kp.cell0 + blockIdx.x * CB;
  const int nb = min(CB, kp.Nc - e0);
  if (nb <= 0) return;
  const Tab<T> tb = load_tables<T, N, QC, QV>(static_cast<const T*>(kp.tables), stab);
  const PhysT<T> ph = make_phys<T>(kp);

  const size_t base = (size_t)e0 * 5 * N3;
  const int nvals = nb * 5 * N3;
  constexpr int PER = (CB * 5 * N3 + op_threads<T>() - 1) / op_threads<T>();  // values per thread
  const bool need_u = CELL || FACE || (MASS && kp.has_bf);
  const T* Ud = static_cast<const T*>(kp.Udev);
  if (need_u) {
    if (Ud)
      batched_pass<PER>(threadIdx.x, blockDim.x, nvals, [&](int i) { return Ud[base + i]; },
                        [&](int i, T v) { su[i] = v; });
    else
      batched_pass<PER>(threadIdx.x, blockDim.x, nvals, [&](int i) { return U[base + i]; },
                        [&](int i, double v) { su[i] = T(v - ref_of(kp, (i / N3) % 5)); });
  }
  if (CELL) {
    for (int i = threadIdx.x; i < nvals; i += blockDim.x) sr[i] = T(0);
  } else {
    batched_pass<PER>(threadIdx.x, blockDim.x, nvals, [&](int i) { return Rin[base + i]; },
                      [&](int i, T v) { sr[i] = v; });
  }
  if (GEO == GEO_FLY) {
    const T* X = static_cast<const T*>(kp.xyzT) + (size_t)e0 * 3 * N3;
    for (int i = threadIdx.x; i < nb * 3 * N3; i += blockDim.x) sx[i] = X[i];
  }
  __syncthreads();

  if (CELL) cell_terms<T, N, QC, QV, CB, GEO>(su, sr, ar, tb, kp, ph, e0, nb, CtaGroup(), sx, go);

  if (CELL && !FACE && kp.fbuf != nullptr) {
    // face-centric organisation: add the face shares of the batch (contiguous), staged in the arena
    const T* F = static_cast<const T*>(kp.fbuf) + (size_t)e0 * fbuf_per_cell<N>();
    __syncthreads();
    if constexpr (S::CELL_ARENA >= fbuf_per_cell<N>()) {
      constexpr int PF = (CB * fbuf_per_cell<N>() + op_threads<T>() - 1) / op_threads<T>();
      batched_pass<PF>(threadIdx.x, blockDim.x, nb * fbuf_per_cell<N>(), [&](int i) { return F[i]; },
                       [&](int i, T v) { ar[i] = v; });
      __syncthreads();
      gather_face_shares<T, N>(sr, ar, tb, nb, CtaGroup());
    } else {
      gather_face_shares<T, N>(sr, F, tb, nb, CtaGroup());
    }
    __syncthreads();
  }

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
          // rotated-frame meshes: the neighbour across the local face from the face table
          const int en = kp.fnbr ? kp.fnbr[((size_t)e * 6 + 2 * d + s) * 2]
                                 : (w ? -1 : c[0] + kp.nc[0] * (c[1] + kp.nc[1] * c[2]));
          nbi[threadIdx.x] = en;
          wall[threadIdx.x] = w;
          const double te = kp.tau[e];
          tau_f[threadIdx.x] = T(w ? te : fmax(te, kp.tau[en]));
        }
        __syncthreads();
        // the neighbour's block, on rotated-frame meshes reoriented into this cell's frame
        for (int i = threadIdx.x; i < nvals; i += blockDim.x) {
          const int e = i / (5 * N3);
          if (!wall[e]) {
            int r = i - e * 5 * N3;
            if (kp.fnbr) {
              const int cq = r / N3;
              r = cq * N3 + frame_node<N>(kp.fnbr[((size_t)(e0 + e) * 6 + 2 * d + s) * 2 + 1], r - cq * N3);
            }
            const size_t src = (size_t)nbi[e] * 5 * N3 + r;
            sn[i] = Ud ? Ud[src] : T(U[src] - ref_of(kp, (i / N3) % 5));
          }
        }
        if (GEO == GEO_FLY) {
          for (int i = threadIdx.x; i < nb * 3 * N3; i += blockDim.x) {
            const int e = i / (3 * N3);
            int r = i - e * 3 * N3;
            if (kp.fnbr) {
              const int cq = r / N3;
              r = cq * N3 + frame_node<N>(kp.fnbr[((size_t)(e0 + e) * 6 + 2 * d + s) * 2 + 1], r - cq * N3);
            }
            sxn[i] = wall[e] ? sx[i] : static_cast<const T*>(kp.xyzT)[(size_t)nbi[e] * 3 * N3 + r];
          }
        }
        __syncthreads();
        const CtaGroup cg;
        if (d == 0)
          face_terms<T, N, QC, QV, CB, 0, GEO>(su, sn, wall, nbi, tau_f, sr, ar, tb, kp, ph, e0, nb, s, cg, sx, sxn, go);
        if (d == 1)
          face_terms<T, N, QC, QV, CB, 1, GEO>(su, sn, wall, nbi, tau_f, sr, ar, tb, kp, ph, e0, nb, s, cg, sx, sxn, go);
        if (d == 2)
          face_terms<T, N, QC, QV, CB, 2, GEO>(su, sn, wall, nbi, tau_f, sr, ar, tb, kp, ph, e0, nb, s, cg, sx, sxn, go);
      }
    }
  }

  if (MASS)
    inverse_mass<T, N, CB, GEO>(su, sr, ar, tb, kp, e0, nb, CELL || FACE || kp.out_mode != 0, kp.has_bf != 0,
                                CtaGroup(), sx, go);

  if (kp.out_mode == 2) {
    // 2N update: dU in the residual type, the state accumulated in FP64
    stage_update<PER, N3>(kp, U, dU, Uout, sr, base, nvals, threadIdx.x, blockDim.x);
  } else {
    for (int i = threadIdx.x; i < nvals; i += blockDim.x) Rout[base + i] = sr[i];
  }
}

// ---------------------------------------------------------------------------
// Diagnostics (always FP64): per-CTA partial sums of
//   [vol, int |u|^2/2, int grad u : grad u, int u.(dm/dt - u drho/dt)/rho, int U (5), nonfinite]
// ---------------------------------------------------------------------------
constexpr int NACC = 10;

template <typename TL, int N, int QC, int QV, int CB, int GEO>
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
  double* GU = red + NT * NACC;    // [9][CB P] physical velocity gradient (stored geometry only)
  const double* gcc = static_cast<const double*>(kp.gcc);
  const double* gmv = static_cast<const double*>(kp.gm);
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
      const double w = tb.wc[p % QC] * tb.wc[(p / QC) % QC] * tb.wc[p / (QC * QC)] *
                       (GEO == GEO_AFFINE ? detJ : gcc[((size_t)(e0 + e) * 10 + 9) * P + p]);
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
    if (GEO == GEO_AFFINE) {
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
    } else {
      // physical velocity gradient du_i/dx_a = sum_b J^{-1}[b][a] du_i/dxi_b, accumulated direction by direction
      for (int idx = threadIdx.x; idx < 9 * nb * P; idx += blockDim.x) GU[idx] = 0.0;
#pragma unroll 1
      for (int j = 0; j < 3; ++j) {
        __syncthreads();
        if (j == 0) sweep<double, 0, QC, QC, QC, QC, -1, false>(V0, V1, tb.eDc, nbl);
        if (j == 1) sweep<double, 1, QC, QC, QC, QC, -1, false>(V0, V1, tb.eDc, nbl);
        if (j == 2) sweep<double, 2, QC, QC, QC, QC, -1, false>(V0, V1, tb.eDc, nbl);
        __syncthreads();
        for (int idx = threadIdx.x; idx < nb * P; idx += blockDim.x) {
          const int e = idx / P, p = idx - e * P;
          const int o = e * 5 * P + p;
          const double* g = gcc + (size_t)(e0 + e) * 10 * P + p;
          const double rinv = 1.0 / V0[o];
#pragma unroll
          for (int i = 0; i < 3; ++i) {
            const double ui = V0[o + (1 + i) * P] * rinv;
            const double gui = (V1[o + (1 + i) * P] - ui * V1[o]) * rinv;
#pragma unroll
            for (int a = 0; a < 3; ++a) GU[(3 * i + a) * nb * P + idx] += g[(3 * j + a) * P] * gui;
          }
        }
      }
      __syncthreads();
      for (int idx = threadIdx.x; idx < nb * P; idx += blockDim.x) {
        const int e = idx / P, p = idx - e * P;
        const double w = tb.wc[p % QC] * tb.wc[(p / QC) % QC] * tb.wc[p / (QC * QC)] *
                         gcc[((size_t)(e0 + e) * 10 + 9) * P + p];
        double gg = 0.0;
#pragma unroll
        for (int m = 0; m < 9; ++m) gg += GU[m * nb * P + idx] * GU[m * nb * P + idx];
        acc[2] += gg * w;
      }
    }
    // conservation totals with the k+1 point rule: int U = sum_q U(x_q) |J| w_q
    sweep<double, 0, N, N, N, N, 1, false>(su, V1, tb.eSm, nbl);
    __syncthreads();
    sweep<double, 1, N, N, N, N, 1, false>(V1, V2, tb.eSm, nbl);
    __syncthreads();
    sweep<double, 2, N, N, N, N, 1, false>(V2, V1, tb.eSm, nbl);
    __syncthreads();
    for (int idx = threadIdx.x; idx < nbl * N3; idx += blockDim.x) {
      const int c = (idx / N3) % 5, p = idx % N3;
      const double w = tb.wm[p % N] * tb.wm[(p / N) % N] * tb.wm[p / (N * N)] *
                       (GEO == GEO_AFFINE ? detJ : gmv[(size_t)(e0 + idx / (5 * N3)) * N3 + p]);
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

template <int N, int QC, int QV, int CB, int GEO>
constexpr size_t diag_smem_bytes() {
  constexpr int N3 = N * N * N, P = QC * QC * QC;
  return (table_elems<N, QC, QV>() + 2 * CB * 5 * N3 + 4 * CB * 5 * P + NT * NACC + (GEO ? 9 * CB * P : 0)) *
             sizeof(double) + 64;
}

// ---------------------------------------------------------------------------
// Geometry precomputation in FP64 (non-affine meshes), one CTA per cell: the
// Jacobian of the isoparametric map x(xi) = sum_i x_i phi_i(xi) at every point
// set by interpolation of the node coordinates and collocation derivatives
// (exact: x is of degree k, the point sets have >= k+1 points), its inverse
// and determinant; on faces the unit outward normal n = J^{-T} n_xi / |J^{-T} n_xi|
// and dA = |det J| |J^{-T} n_xi| (Eq. IntegralsReferenceSpace); the penalty
// tau_e = nu (k+1)^2 (A_interior / 2 + A_boundary) / V with areas and volume
// as Gauss sums at the convective points (Eq. TauIP_Element).
// ---------------------------------------------------------------------------
__device__ __forceinline__ double inv3(const double J[3][3], double Ji[9]) {
  // Ji[3b + a] = (J^{-1})[b][a], J[a][b] = d x_a / d xi_b
  const double c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
  const double c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
  const double c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
  const double det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
  const double id = 1.0 / det;
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

// Cell points of one point set (Q points per direction, matrices eS: N->Q, eD: Q->Q collocation).
template <int N, int Q>
__device__ void geom_cell(const double* X, double* buf, const double* eS, const double* eD, const double* w1,
                          double* g, double* vol) {
  constexpr int P = Q * Q * Q;
  double* A = buf;            // [3][P]
  double* B = A + 3 * P;
  double* Xq = B + 3 * P;
  double* J0 = Xq + 3 * P;
  double* J1 = J0 + 3 * P;
  double* J2 = J1 + 3 * P;
  sweep<double, 0, N, N, N, Q, 1, false>(X, A, eS, 3);
  __syncthreads();
  sweep<double, 1, Q, N, N, Q, 1, false>(A, B, eS, 3);
  __syncthreads();
  sweep<double, 2, Q, Q, N, Q, 1, false>(B, Xq, eS, 3);
  __syncthreads();
  sweep<double, 0, Q, Q, Q, Q, -1, false>(Xq, J0, eD, 3);
  sweep<double, 1, Q, Q, Q, Q, -1, false>(Xq, J1, eD, 3);
  sweep<double, 2, Q, Q, Q, Q, -1, false>(Xq, J2, eD, 3);
  __syncthreads();
  double v = 0.0;
  for (int p = threadIdx.x; p < P; p += blockDim.x) {
    double J[3][3], Ji[9];
    for (int a = 0; a < 3; ++a) {
      J[a][0] = J0[a * P + p];
      J[a][1] = J1[a * P + p];
      J[a][2] = J2[a * P + p];
    }
    const double det = fabs(inv3(J, Ji));
    for (int m = 0; m < 9; ++m) g[m * P + p] = Ji[m];
    g[9 * P + p] = det;
    v += det * w1[p % Q] * w1[(p / Q) % Q] * w1[p / (Q * Q)];
  }
  if (vol) atomicAdd(vol, v);
  __syncthreads();
}

// Face points of face (d, s) for one point set; returns the face area (Gauss sum) via *area.
template <int N, int Q, int d>
__device__ void geom_face(const double* X, double* buf, const double* eS, const double* eD, const double* w1,
                          const double* dl, int s, double* g, double* area) {
  constexpr int P = Q * Q, N2 = N * N, N3 = N * N * N;
  constexpr int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
  double* L = buf;        // [3][N2] face layer
  double* Dn = L + 3 * N2;  // [3][N2] normal derivative layer
  double* Tm = Dn + 3 * N2; // [3][N Q]
  double* Xf = Tm + 3 * N * Q;
  double* Jt1 = Xf + 3 * P;
  double* Jt2 = Jt1 + 3 * P;
  double* Jd = Jt2 + 3 * P;
  const int id = s ? N - 1 : 0;
  for (int idx = threadIdx.x; idx < 3 * N2; idx += blockDim.x) {
    const int a = idx / N2, j = idx % N2;
    const double* x = X + a * N3;
    L[idx] = x[face_node<N>(d, id, j % N, j / N)];
    double dn = 0.0;
    for (int i = 0; i < N; ++i) dn += dl[i] * x[face_node<N>(d, i, j % N, j / N)];
    Dn[idx] = dn;
  }
  __syncthreads();
  sweep<double, 0, N, N, 1, Q, 1, false>(L, Tm, eS, 3);
  __syncthreads();
  sweep<double, 1, Q, N, 1, Q, 1, false>(Tm, Xf, eS, 3);
  __syncthreads();
  sweep<double, 0, N, N, 1, Q, 1, false>(Dn, Tm, eS, 3);
  __syncthreads();
  sweep<double, 1, Q, N, 1, Q, 1, false>(Tm, Jd, eS, 3);
  sweep<double, 0, Q, Q, 1, Q, -1, false>(Xf, Jt1, eD, 3);
  sweep<double, 1, Q, Q, 1, Q, -1, false>(Xf, Jt2, eD, 3);
  __syncthreads();
  const double sgn = s ? 1.0 : -1.0;
  double ar = 0.0;
  for (int p = threadIdx.x; p < P; p += blockDim.x) {
    double J[3][3], Ji[9];
    for (int a = 0; a < 3; ++a) {
      J[a][t1] = Jt1[a * P + p];
      J[a][t2] = Jt2[a * P + p];
      J[a][d] = Jd[a * P + p];
    }
    const double det = fabs(inv3(J, Ji));
    const double v0 = sgn * Ji[3 * d], v1 = sgn * Ji[3 * d + 1], v2 = sgn * Ji[3 * d + 2];
    const double nv = sqrt(v0 * v0 + v1 * v1 + v2 * v2);
    for (int m = 0; m < 9; ++m) g[m * P + p] = Ji[m];
    g[9 * P + p] = v0 / nv;
    g[10 * P + p] = v1 / nv;
    g[11 * P + p] = v2 / nv;
    g[12 * P + p] = det * nv;
    ar += det * nv * w1[p % Q] * w1[p / Q];
  }
  if (area) atomicAdd(area, ar);
  __syncthreads();
}

template <int N, int QC, int QV>
constexpr int geom_buf_elems() {
  constexpr int Q = QC > QV ? QC : QV;
  constexpr int cell = 6 * 3 * Q * Q * Q;
  constexpr int face = 6 * N * N + 3 * N * Q + 4 * 3 * Q * Q;
  return (cell > face ? cell : face) > 6 * 3 * N * N * N ? (cell > face ? cell : face) : 6 * 3 * N * N * N;
}

template <int N, int QC, int QV>
__global__ void __launch_bounds__(NT) dg_geom_kernel(const KParams kp, const double* __restrict__ xyz,
                                                     double* gcc, double* gcv, double* gfc, double* gfv, double* gm,
                                                     double* tau, double* vol, double nu_kk) {
  constexpr int N3 = N * N * N;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* sm = reinterpret_cast<double*>(smem_raw);
  double* stab = sm;
  double* X = stab + table_elems<N, QC, QV>();
  double* buf = X + 3 * N3;
  double* red = buf + geom_buf_elems<N, QC, QV>();  // [0] volume, [1] interior area, [2] boundary area, [3] face tmp
  const Tab<double> tb = load_tables<double, N, QC, QV>(static_cast<const double*>(kp.tables), stab);
  const int e = blockIdx.x;
  for (int i = threadIdx.x; i < 3 * N3; i += blockDim.x) X[i] = xyz[(size_t)e * 3 * N3 + i];
  if (threadIdx.x < 4) red[threadIdx.x] = 0.0;
  __syncthreads();
  geom_cell<N, QC>(X, buf, tb.eSc, tb.eDc, tb.wc, gcc + (size_t)e * 10 * QC * QC * QC, red);
  geom_cell<N, QV>(X, buf, tb.eSv, tb.eDv, tb.wv, gcv + (size_t)e * 10 * QV * QV * QV, nullptr);
  {
    // |det J| at the k+1 mass points
    double* A = buf;
    double* B = A + 3 * N3;
    double* Xq = B + 3 * N3;
    double* J0 = Xq + 3 * N3;
    double* J1 = J0 + 3 * N3;
    double* J2 = J1 + 3 * N3;
    sweep<double, 0, N, N, N, N, 1, false>(X, A, tb.eSm, 3);
    __syncthreads();
    sweep<double, 1, N, N, N, N, 1, false>(A, B, tb.eSm, 3);
    __syncthreads();
    sweep<double, 2, N, N, N, N, 1, false>(B, Xq, tb.eSm, 3);
    __syncthreads();
    sweep<double, 0, N, N, N, N, -1, false>(Xq, J0, tb.eDm, 3);
    sweep<double, 1, N, N, N, N, -1, false>(Xq, J1, tb.eDm, 3);
    sweep<double, 2, N, N, N, N, -1, false>(Xq, J2, tb.eDm, 3);
    __syncthreads();
    for (int p = threadIdx.x; p < N3; p += blockDim.x) {
      double J[3][3], Ji[9];
      for (int a = 0; a < 3; ++a) {
        J[a][0] = J0[a * N3 + p];
        J[a][1] = J1[a * N3 + p];
        J[a][2] = J2[a * N3 + p];
      }
      gm[(size_t)e * N3 + p] = fabs(inv3(J, Ji));
    }
    __syncthreads();
  }
  const int cc[3] = {e % kp.nc[0], (e / kp.nc[0]) % kp.nc[1], e / (kp.nc[0] * kp.nc[1])};
  for (int d = 0; d < 3; ++d)
    for (int s = 0; s < 2; ++s) {
      const int f = 2 * d + s;
      const double* dl = s ? tb.dl1 : tb.dl0;
      double* gc = gfc + ((size_t)e * 6 + f) * 13 * QC * QC;
      double* gv = gfv + ((size_t)e * 6 + f) * 13 * QV * QV;
      if (threadIdx.x == 0) red[3] = 0.0;
      __syncthreads();
      if (d == 0) { geom_face<N, QC, 0>(X, buf, tb.eSc, tb.eDc, tb.wc, dl, s, gc, red + 3); geom_face<N, QV, 0>(X, buf, tb.eSv, tb.eDv, tb.wv, dl, s, gv, nullptr); }
      if (d == 1) { geom_face<N, QC, 1>(X, buf, tb.eSc, tb.eDc, tb.wc, dl, s, gc, red + 3); geom_face<N, QV, 1>(X, buf, tb.eSv, tb.eDv, tb.wv, dl, s, gv, nullptr); }
      if (d == 2) { geom_face<N, QC, 2>(X, buf, tb.eSc, tb.eDc, tb.wc, dl, s, gc, red + 3); geom_face<N, QV, 2>(X, buf, tb.eSv, tb.eDv, tb.wv, dl, s, gv, nullptr); }
      if (threadIdx.x == 0) {
        const bool boundary = !kp.periodic[d] && ((s == 0 && cc[d] == 0) || (s == 1 && cc[d] == kp.nc[d] - 1));
        red[boundary ? 2 : 1] += red[3];
      }
      __syncthreads();
    }
  if (threadIdx.x == 0) {
    tau[e] = nu_kk * (0.5 * red[1] + red[2]) / red[0];
    vol[e] = red[0];
  }
}

template <int N, int QC, int QV>
int geom_launch(const KParams& kp, const double* xyz, double* gcc, double* gcv, double* gfc, double* gfv, double* gm,
                double* tau, double* vol, double nu_kk, cudaStream_t st) {
  if constexpr (!Feat<N, QC, QV>::geo) {
    return -2;
  } else {
  auto k = dg_geom_kernel<N, QC, QV>;
  constexpr size_t smem = (table_elems<N, QC, QV>() + 3 * N * N * N + geom_buf_elems<N, QC, QV>() + 8) * sizeof(double);
  if (smem > 227 * 1024) return -2;
  static bool attr[kMaxDevices] = {};
  if (smem_attr_once(k, smem, attr)) return -1;
  k<<<kp.Nc, NT, smem, st>>>(kp, xyz, gcc, gcv, gfc, gfv, gm, tau, vol, nu_kk);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
  }
}

// ---------------------------------------------------------------------------
// Gradient of the kinetic energy e_k = (1/V) int |u|^2/2, u = m/rho (convective Gauss
// rule, as dg_diag_kernel) with respect to the nodal state (FP64):
//   d/d rho_j = (1/V) sum_q (-|u|^2/rho) |J| w phi_j(x_q),  d/d m_j = (1/V) sum_q (u/rho) |J| w phi_j(x_q).
// ---------------------------------------------------------------------------
template <int N, int QC, int QV, int CB, int GEO>
__global__ void __launch_bounds__(NT) dg_ekgrad_kernel(const KParams kp, const double* __restrict__ U,
                                                       double* __restrict__ G, double inv_volume) {
  constexpr int N3 = N * N * N, P = QC * QC * QC;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* sm = reinterpret_cast<double*>(smem_raw);
  double* stab = sm;
  double* su = stab + table_elems<N, QC, QV>();
  double* V0 = su + CB * 5 * N3;
  double* V1 = V0 + CB * 5 * P;
  double* V2 = V1 + CB * 5 * P;
  const Tab<double> tb = load_tables<double, N, QC, QV>(static_cast<const double*>(kp.tables), stab);
  const int e0 = blockIdx.x * CB;
  const int nb = min(CB, kp.Nc - e0);
  if (nb <= 0) return;
  const size_t base = (size_t)e0 * 5 * N3;
  const int nvals = nb * 5 * N3, nbl = nb * 5;
  for (int i = threadIdx.x; i < nvals; i += blockDim.x) su[i] = U[base + i];
  __syncthreads();
  sweep<double, 0, N, N, N, QC, 1, false>(su, V1, tb.eSc, nbl);
  __syncthreads();
  sweep<double, 1, QC, N, N, QC, 1, false>(V1, V2, tb.eSc, nbl);
  __syncthreads();
  sweep<double, 2, QC, QC, N, QC, 1, false>(V2, V0, tb.eSc, nbl);
  __syncthreads();
  const double detJ = kp.h[0] * kp.h[1] * kp.h[2];
  const double* gcc = static_cast<const double*>(kp.gcc);
  for (int idx = threadIdx.x; idx < nb * P; idx += blockDim.x) {
    const int e = idx / P, p = idx - e * P;
    const int o = e * 5 * P + p;
    const double w = tb.wc[p % QC] * tb.wc[(p / QC) % QC] * tb.wc[p / (QC * QC)] *
                     (GEO == GEO_AFFINE ? detJ : gcc[((size_t)(e0 + e) * 10 + 9) * P + p]) * inv_volume;
    // e = |u|^2 / 2 with u = m / rho:  de/drho = -|u|^2 / rho,  de/dm = u / rho
    const double rinv = 1.0 / V0[o];
    const double u0 = V0[o + P] * rinv, u1 = V0[o + 2 * P] * rinv, u2 = V0[o + 3 * P] * rinv;
    const double wr = w * rinv;
    V0[o] = -(u0 * u0 + u1 * u1 + u2 * u2) * wr;
    V0[o + P] = u0 * wr;
    V0[o + 2 * P] = u1 * wr;
    V0[o + 3 * P] = u2 * wr;
    V0[o + 4 * P] = 0.0;
  }
  __syncthreads();
  sweep<double, 2, QC, QC, QC, N, 1, false>(V0, V1, tb.eScT, nbl);
  __syncthreads();
  sweep<double, 1, QC, QC, N, N, 1, false>(V1, V2, tb.eScT, nbl);
  __syncthreads();
  sweep<double, 0, QC, N, N, N, 1, false>(V2, su, tb.eScT, nbl);
  __syncthreads();
  for (int i = threadIdx.x; i < nvals; i += blockDim.x) G[base + i] = su[i];
}

template <int N, int QC, int QV, int GEO>
int ekgrad_launch_geo(const KParams& kp, const double* U, double* G, double inv_volume, cudaStream_t st) {
  constexpr int CB = QC * QC * QC > 300 ? 1 : 2;
  constexpr size_t smem = (table_elems<N, QC, QV>() + CB * 5 * N * N * N + 3 * CB * 5 * QC * QC * QC) * sizeof(double) + 64;
  if (smem > 227 * 1024) return -2;
  auto k = dg_ekgrad_kernel<N, QC, QV, CB, GEO>;
  static bool attr[kMaxDevices] = {};
  if (smem_attr_once(k, smem, attr)) return -1;
  k<<<(kp.Nc + CB - 1) / CB, NT, smem, st>>>(kp, U, G, inv_volume);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

template <int N, int QC, int QV>
int ekgrad_launch(const KParams& kp, const double* U, double* G, double inv_volume, cudaStream_t st) {
  if (kp.gcc == nullptr) return ekgrad_launch_geo<N, QC, QV, GEO_AFFINE>(kp, U, G, inv_volume, st);
  if constexpr (Feat<N, QC, QV>::geo) return ekgrad_launch_geo<N, QC, QV, GEO_STORED>(kp, U, G, inv_volume, st);
  return -2;
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
template <typename T, int N, int QC, int QV, int CB, bool CELL, bool FACE, bool MASS, int GEO>
int launch_op(const KParams& kp, const double* U, const void* Rin, void* Rout, void* dU, double* Uout,
              cudaStream_t st) {
  auto k = dg_op_kernel<T, N, QC, QV, CB, CELL, FACE, MASS, GEO>;
  constexpr bool GWS = op_gws<T, N, QC, QV, CB, CELL, FACE, MASS, GEO>();
  constexpr size_t smem = GWS ? table_elems<N, QC, QV>() * sizeof(T) + 64
                              : op_smem_bytes<T, N, QC, QV, CB, CELL, FACE, MASS, GEO>();
  if (smem > 227 * 1024) return -2;
  static bool attr[kMaxDevices] = {};
  if (smem_attr_once(k, smem, attr)) return -1;
  const int grid = (kp.Nc + CB - 1) / CB;
  if constexpr (GWS) {
    // global workspace: chunks of as many CTAs as it holds; returns the number of launches
    constexpr size_t work = op_work_elems<T, N, QC, QV, CB, CELL, FACE, MASS, GEO>();
    const int per = (int)(kp.gws ? kp.gws_elems / work : 0);
    if (per < 1) return -2;
    int launches = 0;
    for (int b0 = 0; b0 < grid; b0 += per) {
      KParams kc = kp;
      kc.cell0 = b0 * CB;
      k<<<min(per, grid - b0), op_threads<T>(), smem, st>>>(kc, U, static_cast<const T*>(Rin), static_cast<T*>(Rout),
                                                            static_cast<T*>(dU), Uout);
      if (cudaGetLastError() != cudaSuccess) return -1;
      ++launches;
    }
    return launches;
  } else {
    k<<<grid, op_threads<T>(), smem, st>>>(kp, U, static_cast<const T*>(Rin), static_cast<T*>(Rout),
                                            static_cast<T*>(dU), Uout);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
  }
}

// Bytes per CTA of the global workspace that an (N, QC, QV) instantiation's CTA-wide operator kernels
// need (0 when every variant fits shared memory): the largest over the variants with and without
// element-centric faces.
template <typename T, int N, int QC, int QV>
constexpr size_t op_gws_bytes() {
  constexpr int CB0 = cells_per_cta<T, N, QC, QV, false>(), CB1 = cells_per_cta<T, N, QC, QV, true>();
  constexpr size_t a = op_gws<T, N, QC, QV, CB0, true, false, true, GEO_AFFINE>()
                           ? op_work_elems<T, N, QC, QV, CB0, true, false, true, GEO_AFFINE>() * sizeof(T) : 0;
  constexpr size_t b = op_gws<T, N, QC, QV, CB1, true, true, true, GEO_AFFINE>()
                           ? op_work_elems<T, N, QC, QV, CB1, true, true, true, GEO_AFFINE>() * sizeof(T) : 0;
  return a > b ? a : b;
}

// ---------------------------------------------------------------------------
// Warp-per-cell organisation of the same operator (used for the FP32 form):
// WPC warps per CTA, each warp carries one cell through all phases with
// warp-level barriers only, so the warps of an SM progress independently and
// hide each other's latency.  Shared memory: the tables (per CTA) and one
// private slice per warp.
// ---------------------------------------------------------------------------
template <typename T, int N, int QC, int QV, bool CELL, bool FACE, bool MASS, int GEO>
constexpr int warp_slice_elems() {
  using S = Sizes<N, QC, QV>;
  const int e = 5 * S::N3 * (FACE ? 3 : 2) + (int)op_arena_elems<N, QC, QV, 1, CELL, FACE, MASS, GEO>() +
                (int)op_geo_elems<N, QC, QV, 1, FACE, GEO>() + 1 + 2 * 8 / (int)sizeof(T) + 2;
  return (e + 7) & ~7;
}

template <typename T, int N, int QC, int QV, int WPC, bool CELL, bool FACE, bool MASS, int GEO>
constexpr size_t warp_smem_bytes() {
  return ((size_t)table_elems<N, QC, QV>() +
          (size_t)WPC * warp_slice_elems<T, N, QC, QV, CELL, FACE, MASS, GEO>()) * sizeof(T) + 64;
}

template <typename T, int N, int QC, int QV, int WPC, bool CELL, bool FACE, bool MASS, int GEO>
__global__ void __launch_bounds__(WPC * 32) dg_op_warp_kernel(const KParams kp, const double* __restrict__ U,
                                                              const T* Rin, T* Rout, T* dU, double* Uout) {
  using S = Sizes<N, QC, QV>;
  constexpr int N3 = S::N3;
  constexpr int SL = warp_slice_elems<T, N, QC, QV, CELL, FACE, MASS, GEO>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  T* stab = sm;
  const Tab<T> tb = load_tables<T, N, QC, QV>(static_cast<const T*>(kp.tables), stab);
  __syncthreads();
  const int w = threadIdx.x >> 5;
  const int e0 = blockIdx.x * WPC + w;
  if (e0 >= kp.Nc) return;  // only warp barriers below
  const WarpGroup grp;
  T* su = stab + table_elems<N, QC, QV>() + w * SL;
  T* sr = su + 5 * N3;
  T* sn = sr + 5 * N3;
  T* ar = sn + (FACE ? 5 * N3 : 0);
  T* sx = ar + op_arena_elems<N, QC, QV, 1, CELL, FACE, MASS, GEO>();  // GEO_FLY only
  T* sxn = sx + 3 * N3;
  T* go = sxn + (FACE ? 3 * N3 : 0);
  T* tau_f = sx + op_geo_elems<N, QC, QV, 1, FACE, GEO>();
  int* wall = reinterpret_cast<int*>(su + SL) - 2;  // two ints at the end of the slice
  int* nbi = wall + 1;
  const PhysT<T> ph = make_phys<T>(kp);
  const size_t base = (size_t)e0 * 5 * N3;
  constexpr int nvals = 5 * N3;
  constexpr int PER = (nvals + 31) / 32;  // values per lane
  const bool need_u = CELL || FACE || (MASS && kp.has_bf);
  const T* Ud = static_cast<const T*>(kp.Udev);
  if (need_u) {
    if (Ud)
      batched_pass<PER>(grp.rank(), 32, nvals, [&](int i) { return Ud[base + i]; }, [&](int i, T v) { su[i] = v; });
    else
      batched_pass<PER>(grp.rank(), 32, nvals, [&](int i) { return U[base + i]; },
                        [&](int i, double v) { su[i] = T(v - ref_of(kp, (i / N3) % 5)); });
  }
  if (CELL) {
    for (int i = grp.rank(); i < nvals; i += 32) sr[i] = T(0);
  } else {
    batched_pass<PER>(grp.rank(), 32, nvals, [&](int i) { return Rin[base + i]; }, [&](int i, T v) { sr[i] = v; });
  }
  if (GEO == GEO_FLY) {
    const T* X = static_cast<const T*>(kp.xyzT) + (size_t)e0 * 3 * N3;
    for (int i = grp.rank(); i < 3 * N3; i += 32) sx[i] = X[i];
  }
  grp.sync();
  if (CELL) cell_terms<T, N, QC, QV, 1, GEO>(su, sr, ar, tb, kp, ph, e0, 1, grp, sx, go);
  if (CELL && !FACE && kp.fbuf != nullptr) {
    const T* F = static_cast<const T*>(kp.fbuf) + (size_t)e0 * fbuf_per_cell<N>();
    grp.sync();
    if constexpr (S::CELL_ARENA >= fbuf_per_cell<N>()) {
      batched_pass<(fbuf_per_cell<N>() + 31) / 32>(grp.rank(), 32, fbuf_per_cell<N>(), [&](int i) { return F[i]; },
                                                   [&](int i, T v) { ar[i] = v; });
      grp.sync();
      gather_face_shares<T, N>(sr, ar, tb, 1, grp);
    } else {
      gather_face_shares<T, N>(sr, F, tb, 1, grp);
    }
    grp.sync();
  }
  if (FACE) {
    for (int d = 0; d < 3; ++d) {
      for (int s = 0; s < 2; ++s) {
        if (grp.rank() == 0) {
          int c[3] = {e0 % kp.nc[0], (e0 / kp.nc[0]) % kp.nc[1], e0 / (kp.nc[0] * kp.nc[1])};
          c[d] += s ? 1 : -1;
          int wl = 0;
          if (c[d] < 0 || c[d] >= kp.nc[d]) {
            if (kp.periodic[d])
              c[d] = (c[d] + kp.nc[d]) % kp.nc[d];
            else
              wl = 1;
          }
          const int en = kp.fnbr ? kp.fnbr[((size_t)e0 * 6 + 2 * d + s) * 2]
                                 : (wl ? -1 : c[0] + kp.nc[0] * (c[1] + kp.nc[1] * c[2]));
          nbi[0] = en;
          wall[0] = wl;
          const double te = kp.tau[e0];
          tau_f[0] = T(wl ? te : fmax(te, kp.tau[en]));
        }
        grp.sync();
        if (!wall[0]) {
          // the neighbour's block, on rotated-frame meshes reoriented into this cell's frame
          const size_t nb0 = (size_t)nbi[0] * 5 * N3;
          const int code = kp.fnbr ? kp.fnbr[((size_t)e0 * 6 + 2 * d + s) * 2 + 1] : 0;
          for (int i = grp.rank(); i < nvals; i += 32) {
            const int cq = i / N3;
            const int r = kp.fnbr ? cq * N3 + frame_node<N>(code, i - cq * N3) : i;
            sn[i] = Ud ? Ud[nb0 + r] : T(U[nb0 + r] - ref_of(kp, cq % 5));
          }
          if (GEO == GEO_FLY) {
            const T* Xn = static_cast<const T*>(kp.xyzT) + (size_t)nbi[0] * 3 * N3;
            for (int i = grp.rank(); i < 3 * N3; i += 32) {
              const int cq = i / N3;
              sxn[i] = Xn[kp.fnbr ? cq * N3 + frame_node<N>(code, i - cq * N3) : i];
            }
          }
        } else if (GEO == GEO_FLY) {
          for (int i = grp.rank(); i < 3 * N3; i += 32) sxn[i] = sx[i];
        }
        grp.sync();
        if (d == 0)
          face_terms<T, N, QC, QV, 1, 0, GEO>(su, sn, wall, nbi, tau_f, sr, ar, tb, kp, ph, e0, 1, s, grp, sx, sxn, go);
        if (d == 1)
          face_terms<T, N, QC, QV, 1, 1, GEO>(su, sn, wall, nbi, tau_f, sr, ar, tb, kp, ph, e0, 1, s, grp, sx, sxn, go);
        if (d == 2)
          face_terms<T, N, QC, QV, 1, 2, GEO>(su, sn, wall, nbi, tau_f, sr, ar, tb, kp, ph, e0, 1, s, grp, sx, sxn, go);
      }
    }
  }
  if (MASS)
    inverse_mass<T, N, 1, GEO>(su, sr, ar, tb, kp, e0, 1, CELL || FACE || kp.out_mode != 0, kp.has_bf != 0, grp,
                               sx, go);
  if (kp.out_mode == 2) {
    stage_update<PER, N3>(kp, U, dU, Uout, sr, base, nvals, grp.rank(), 32);
  } else {
    for (int i = grp.rank(); i < nvals; i += 32) Rout[base + i] = sr[i];
  }
}

template <typename T, int N, int QC, int QV, bool CELL, bool FACE, bool MASS, int GEO>
int launch_op_warp(const KParams& kp, const double* U, const void* Rin, void* Rout, void* dU, double* Uout,
                   cudaStream_t st) {
  constexpr int WPC = 4;
  constexpr size_t smem = warp_smem_bytes<T, N, QC, QV, WPC, CELL, FACE, MASS, GEO>();
  if (smem > 227 * 1024) return -2;
  auto k = dg_op_warp_kernel<T, N, QC, QV, WPC, CELL, FACE, MASS, GEO>;
  static bool attr[kMaxDevices] = {};
  if (smem_attr_once(k, smem, attr)) return -1;
  const int grid = (kp.Nc + WPC - 1) / WPC;
  k<<<grid, WPC * 32, smem, st>>>(kp, U, static_cast<const T*>(Rin), static_cast<T*>(Rout), static_cast<T*>(dU),
                                    Uout);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

template <typename T, int N, int QC, int QV, int GEO, bool WARP, bool CELL, bool FACE, bool MASS>
int launch_op_any(const KParams& kp, const double* U, const void* Rin, void* Rout, void* dU, double* Uout,
                  cudaStream_t st) {
  if constexpr (WARP) {
    return launch_op_warp<T, N, QC, QV, CELL, FACE, MASS, GEO>(kp, U, Rin, Rout, dU, Uout, st);
  } else {
    constexpr int CB = cells_per_cta<T, N, QC, QV, FACE>();
    return launch_op<T, N, QC, QV, CB, CELL, FACE, MASS, GEO>(kp, U, Rin, Rout, dU, Uout, st);
  }
}

template <typename T, int N, int QC, int QV, int GEO>
int op_dispatch_geo(int mode, const KParams& kp, const double* U, const void* Rin, void* Rout, void* dU,
                    double* Uout, cudaStream_t st) {
  // FP32: warp per cell (latency-bound otherwise); FP64: CTA per cell batch (FP64-pipe bound)
  // (only while a warp's slice stays small: at k = 5 a cell needs ~49 KB, which would leave 4 warps per SM)
  constexpr bool WARP =
      sizeof(T) == 4 && warp_slice_elems<T, N, QC, QV, true, true, true, GEO>() * sizeof(T) <= 20 * 1024;
  switch (mode) {
    case OP_CELL: return launch_op_any<T, N, QC, QV, GEO, WARP, true, false, false>(kp, U, Rin, Rout, dU, Uout, st);
    case OP_FACE: return launch_op_any<T, N, QC, QV, GEO, WARP, false, true, false>(kp, U, Rin, Rout, dU, Uout, st);
    case OP_MASS:
      if constexpr (sizeof(T) == 4 && GEO == GEO_AFFINE && mass_reg_ok<N, QC, QV>()) {
        // FP32 at k = 3: every block in registers (16-byte aligned arrays, no body force)
        const auto al = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; };
        if (!kp.has_bf && al(Rin) && al(Rout) && al(dU) && al(U) && al(Uout)) {
          if (kp.out_mode == 2) return launch_mass_reg<N, QC, QV, true>(kp, Rin, Rout, dU, U, Uout, st);
          return launch_mass_reg<N, QC, QV, false>(kp, Rin, Rout, dU, U, Uout, st);
        }
      }
      if constexpr (mass_tma_ok<T, N>() && GEO != GEO_FLY && mass_tma_bytes<T, N, QC, QV, true>(1) <= 227 * 1024) {
        // the TMA-pipelined kernel needs 16-byte aligned arrays and no body force (no state read)
        const auto al = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; };
        if (!kp.has_bf && kp.err != nullptr && al(Rin) && al(Rout) && al(dU) && al(U) && al(Uout)) {
          if (kp.out_mode == 2) return launch_mass_tma<T, N, QC, QV, true, GEO>(kp, Rin, Rout, dU, U, Uout, st);
          return launch_mass_tma<T, N, QC, QV, false, GEO>(kp, Rin, Rout, dU, U, Uout, st);
        }
      }
      return launch_op_any<T, N, QC, QV, GEO, WARP, false, false, true>(kp, U, Rin, Rout, dU, Uout, st);
    case OP_CELL | OP_FACE:
      return launch_op_any<T, N, QC, QV, GEO, WARP, true, true, false>(kp, U, Rin, Rout, dU, Uout, st);
    case OP_CELL | OP_MASS:
      if constexpr (sizeof(T) == 4 && GEO == GEO_AFFINE && DGCNS_FP32_TASK_CELL && task_cell_ok<N, QC, QV>()) {
        if (kp.fbuf != nullptr && kp.Udev != nullptr && !kp.has_bf && (kp.out_mode == 1 || kp.out_mode == 2))
          return launch_task_cell<N, QC, QV>(kp, U, Rout, dU, Uout, st);
      }
      if constexpr (Feat<N, QC, QV>::faces)
        return launch_op_any<T, N, QC, QV, GEO, WARP, true, false, true>(kp, U, Rin, Rout, dU, Uout, st);
      return -2;
    case OP_CELL | OP_FACE | OP_MASS:
      return launch_op_any<T, N, QC, QV, GEO, WARP, true, true, true>(kp, U, Rin, Rout, dU, Uout, st);
    default: return -2;
  }
}

template <typename T, int N, int QC, int QV>
int op_dispatch(int mode, const KParams& kp, const double* U, const void* Rin, void* Rout, void* dU, double* Uout,
                cudaStream_t st) {
  using F = Feat<N, QC, QV>;
  if constexpr (sizeof(T) == 4 && !F::fp32) {
    return -2;
  } else {
    if (kp.xyzT != nullptr) {
      if constexpr (F::fly) return op_dispatch_geo<T, N, QC, QV, GEO_FLY>(mode, kp, U, Rin, Rout, dU, Uout, st);
      return -2;
    }
    if (kp.gcc != nullptr) {
      if constexpr (F::geo) return op_dispatch_geo<T, N, QC, QV, GEO_STORED>(mode, kp, U, Rin, Rout, dU, Uout, st);
      return -2;
    }
    return op_dispatch_geo<T, N, QC, QV, GEO_AFFINE>(mode, kp, U, Rin, Rout, dU, Uout, st);
  }
}

template <typename TL, int N, int QC, int QV, int GEO>
int diag_launch_geo(const KParams& kp, const double* U, const void* LU, double* partial, int* nblocks,
                    cudaStream_t st) {
  constexpr int CB = QC * QC * QC > 300 ? 1 : 2;
  auto k = dg_diag_kernel<TL, N, QC, QV, CB, GEO>;
  constexpr size_t smem = diag_smem_bytes<N, QC, QV, CB, GEO>();
  if (smem > 227 * 1024) return -2;
  static bool attr[kMaxDevices] = {};
  if (smem_attr_once(k, smem, attr)) return -1;
  const int grid = (kp.Nc + CB - 1) / CB;
  *nblocks = grid;
  if (partial == nullptr) return 0;
  k<<<grid, NT, smem, st>>>(kp, U, static_cast<const TL*>(LU), partial);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

template <typename TL, int N, int QC, int QV>
int diag_launch(const KParams& kp, const double* U, const void* LU, double* partial, int* nblocks,
                cudaStream_t st) {
  using F = Feat<N, QC, QV>;
  if constexpr (sizeof(TL) == 4 && !F::fp32) {
    return -2;
  } else {
    if (kp.gcc == nullptr) return diag_launch_geo<TL, N, QC, QV, GEO_AFFINE>(kp, U, LU, partial, nblocks, st);
    if constexpr (F::geo) return diag_launch_geo<TL, N, QC, QV, GEO_STORED>(kp, U, LU, partial, nblocks, st);
    return -2;
  }
}

template <typename T, int N>
int dev_launch(const KParams& kp, const double* U, void* D, cudaStream_t st) {
  const size_t n = (size_t)kp.Nc * 5 * N * N * N;
  dg_dev_kernel<T><<<2 * 152 * 8, 256, 0, st>>>(kp, U, static_cast<T*>(D), n, N * N * N);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// ---------------------------------------------------------------------------
// Face-centric face kernel: blockIdx.y = direction d.  Blocks [0, ceil(Nc/CB)) take the faces
// at the upper side (s = 1) of every cell (interior faces with both shares, upper walls with
// one); on a non-periodic direction the following blocks take the lower wall faces (s = 0) of
// the cells with c_d = 0.
// ---------------------------------------------------------------------------
template <typename T, int N, int QC, int QV, int CB, int GEO>
constexpr size_t face_arena_elems() {
  using S = Sizes<N, QC, QV>;
  size_t arena = (size_t)CB * PairSizes<N, QC, QV>::ARENA;
  if (GEO == GEO_FLY && (size_t)CB * S::FLY_TMP > arena) arena = (size_t)CB * S::FLY_TMP;
  return (arena + 3) & ~(size_t)3;
}

template <typename T, int N, int QC, int QV, int CB, int GEO>
constexpr size_t face_smem_bytes() {
  using S = Sizes<N, QC, QV>;
  const size_t geo = GEO == GEO_FLY ? (size_t)CB * (2 * 3 * S::N3 + S::FLY_OUT) : 0;
  const size_t elems = table_elems<N, QC, QV>() + (size_t)CB * PairSizes<N, QC, QV>::LAYERS +
                       (size_t)CB * 5 * S::N2 + face_arena_elems<T, N, QC, QV, CB, GEO>() + geo + CB;
  return elems * sizeof(T) + 3 * CB * sizeof(int) + 64;
}

// Faces per CTA: the largest batch (<= 8) below ~112 KB of shared memory.
template <typename T, int N, int QC, int QV, int GEO>
constexpr int faces_per_cta() {
  using S = Sizes<N, QC, QV>;
  constexpr int arena = GEO == GEO_FLY && S::FLY_TMP > PairSizes<N, QC, QV>::ARENA ? S::FLY_TMP
                                                                                    : PairSizes<N, QC, QV>::ARENA;
  constexpr int geo = GEO == GEO_FLY ? 2 * 3 * S::N3 + S::FLY_OUT : 0;
  constexpr int per_face = (PairSizes<N, QC, QV>::LAYERS + 5 * S::N2 + arena + geo) * (int)sizeof(T) + 16;
  constexpr int cb = (112 * 1024 - table_elems<N, QC, QV>() * (int)sizeof(T)) / per_face;
  constexpr int cap = sizeof(T) == 4 ? 8 : DGCNS_FP64_FACE_CAP;
  return cb < 1 ? 1 : (cb > cap ? cap : cb);
}

// Threads per CTA of the CTA-wide face kernel.  FP64 affine, 8 faces per CTA at k = 3: 256 threads 8 %
// faster than 128 (160 and 192 in between), measured; the non-affine variants hold fewer faces per CTA
// and were slower with 256 (channel 32^3: -5 % stored, -30 % on the fly), so they keep 128.
template <typename T, int GEO>
constexpr int face_threads() {
  return sizeof(T) == 8 ? (GEO == GEO_AFFINE ? DGCNS_FP64_FACE_THREADS : 128) : op_threads<T>();
}

template <typename T, int N, int QC, int QV, int CB, int GEO>
__global__ void __launch_bounds__(face_threads<T, GEO>()) dg_face_kernel(const KParams kp, const double* __restrict__ U,
                                                                  T* __restrict__ FB) {
  using S = Sizes<N, QC, QV>;
  constexpr int N3 = S::N3;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* stab = reinterpret_cast<T*>(smem_raw);
  T* lay = stab + table_elems<N, QC, QV>();
  T* lc = lay + CB * PairSizes<N, QC, QV>::LAYERS;
  T* fa = lc + CB * 5 * S::N2;
  T* sx = fa + face_arena_elems<T, N, QC, QV, CB, GEO>();  // GEO_FLY only
  T* sxn = sx + CB * 3 * N3;
  T* go = sxn + CB * 3 * N3;
  T* tau_f = sx + (GEO == GEO_FLY ? CB * (2 * 3 * N3 + S::FLY_OUT) : 0);
  int* eo = reinterpret_cast<int*>(tau_f + CB);
  int* en = eo + CB;
  int* oc = en + CB;  // rotated-frame meshes: orientation code of the other cell

  const int d = blockIdx.y;
  const int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
  int s, i0, nitems;
  if (kp.flist) {  // rotated-frame meshes: the faces owned through local face (d, 1), then (d, 0)
    const int nb1 = (kp.flen[2 * d + 1] + CB - 1) / CB;
    s = (int)blockIdx.x < nb1 ? 1 : 0;
    i0 = (s ? (int)blockIdx.x : (int)blockIdx.x - nb1) * CB;
    nitems = kp.flen[2 * d + s];
    if (i0 >= nitems) return;
  } else {
    const int nstd = (kp.Nc + CB - 1) / CB;
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
  }
  const int nb = min(CB, nitems - i0);
  const Tab<T> tb = load_tables<T, N, QC, QV>(static_cast<const T*>(kp.tables), stab);
  const PhysT<T> ph = make_phys<T>(kp);
  if ((int)threadIdx.x < nb && kp.flist) {
    const int e = kp.flist[kp.foff[2 * d + s] + i0 + threadIdx.x];
    const int* t = kp.fnbr + ((size_t)e * 6 + 2 * d + s) * 2;
    eo[threadIdx.x] = e;
    en[threadIdx.x] = t[0];
    oc[threadIdx.x] = t[1];
    tau_f[threadIdx.x] = T(fmax(kp.tau[e], kp.tau[t[0]]));
  } else if ((int)threadIdx.x < nb) {
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
  const T* Ud = static_cast<const T*>(kp.Udev);
  const int* ocp = kp.flist ? oc : nullptr;
  if (GEO == GEO_FLY) {
    const T* X = static_cast<const T*>(kp.xyzT);
    for (int i = threadIdx.x; i < nb * 3 * N3; i += blockDim.x) {
      const int b = i / (3 * N3), r = i - b * 3 * N3;
      sx[i] = X[(size_t)eo[b] * 3 * N3 + r];
      // the other cell's coordinates, on rotated-frame meshes reoriented into the own cell's frame
      const int cq = r / N3;
      const int rn = ocp ? cq * N3 + frame_node<N>(ocp[b], r - cq * N3) : r;
      sxn[i] = X[(size_t)(en[b] >= 0 ? en[b] : eo[b]) * 3 * N3 + rn];
    }
  }
  __syncthreads();
  const CtaGroup cg;
  if (d == 0)
    face_pair_terms<T, N, QC, QV, CB, 0, GEO>(U, Ud, eo, en, tau_f, lay, fa, lc, tb, kp, ph, nb, s, FB, cg, sx, sxn, go,
                                              ocp);
  else if (d == 1)
    face_pair_terms<T, N, QC, QV, CB, 1, GEO>(U, Ud, eo, en, tau_f, lay, fa, lc, tb, kp, ph, nb, s, FB, cg, sx, sxn, go,
                                              ocp);
  else
    face_pair_terms<T, N, QC, QV, CB, 2, GEO>(U, Ud, eo, en, tau_f, lay, fa, lc, tb, kp, ph, nb, s, FB, cg, sx, sxn, go,
                                              ocp);
}

// Warp-per-face organisation of the same face kernel (used for the FP32 form, as the warp-per-cell
// cell kernel): WPC warps per CTA, each warp takes one face through every phase with warp barriers.
template <typename T, int N, int QC, int QV, int GEO>
constexpr int face_warp_slice_elems() {
  using S = Sizes<N, QC, QV>;
  const int geo = GEO == GEO_FLY ? 2 * 3 * S::N3 + S::FLY_OUT : 0;
  const int e = PairSizes<N, QC, QV>::LAYERS + 5 * S::N2 + (int)face_arena_elems<T, N, QC, QV, 1, GEO>() + geo + 1 +
                2 * 8 / (int)sizeof(T) + 2;
  return (e + 7) & ~7;
}

template <typename T, int N, int QC, int QV, int WPC, int GEO>
constexpr size_t face_warp_smem_bytes() {
  return ((size_t)table_elems<N, QC, QV>() + (size_t)WPC * face_warp_slice_elems<T, N, QC, QV, GEO>()) * sizeof(T) +
         64;
}

template <typename T, int N, int QC, int QV, int WPC, int GEO>
__global__ void __launch_bounds__(WPC * 32) dg_face_warp_kernel(const KParams kp, const double* __restrict__ U,
                                                                T* __restrict__ FB) {
  using S = Sizes<N, QC, QV>;
  constexpr int N3 = S::N3;
  constexpr int SL = face_warp_slice_elems<T, N, QC, QV, GEO>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* stab = reinterpret_cast<T*>(smem_raw);
  const Tab<T> tb = load_tables<T, N, QC, QV>(static_cast<const T*>(kp.tables), stab);
  __syncthreads();
  const int w = threadIdx.x >> 5;
  const int d = blockIdx.y;
  const int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
  int s, i;
  if (kp.flist) {  // rotated-frame meshes: the faces owned through local face (d, 1), then (d, 0)
    const int nb1 = (kp.flen[2 * d + 1] + WPC - 1) / WPC;
    s = (int)blockIdx.x < nb1 ? 1 : 0;
    i = (s ? (int)blockIdx.x : (int)blockIdx.x - nb1) * WPC + w;
    if (i >= kp.flen[2 * d + s]) return;  // only warp barriers below
  } else {
    const int nstd = (kp.Nc + WPC - 1) / WPC;
    if ((int)blockIdx.x < nstd) {
      s = 1;
      i = blockIdx.x * WPC + w;
      if (i >= kp.Nc) return;  // only warp barriers below
    } else {
      if (kp.periodic[d]) return;
      s = 0;
      i = (blockIdx.x - nstd) * WPC + w;
      if (i >= kp.nc[t1] * kp.nc[t2]) return;
    }
  }
  const WarpGroup grp;
  T* lay = stab + table_elems<N, QC, QV>() + w * SL;
  T* lc = lay + PairSizes<N, QC, QV>::LAYERS;
  T* fa = lc + 5 * S::N2;
  T* sx = fa + face_arena_elems<T, N, QC, QV, 1, GEO>();  // GEO_FLY only
  T* sxn = sx + 3 * N3;
  T* go = sxn + 3 * N3;
  T* tau_f = sx + (GEO == GEO_FLY ? 2 * 3 * N3 + S::FLY_OUT : 0);
  int* eo = reinterpret_cast<int*>(lay + SL) - 3;  // three ints at the end of the slice
  int* en = eo + 1;
  int* oc = eo + 2;  // rotated-frame meshes: orientation code of the other cell
  const PhysT<T> ph = make_phys<T>(kp);
  if (grp.rank() == 0 && kp.flist) {
    const int e = kp.flist[kp.foff[2 * d + s] + i];
    const int* t = kp.fnbr + ((size_t)e * 6 + 2 * d + s) * 2;
    eo[0] = e;
    en[0] = t[0];
    oc[0] = t[1];
    tau_f[0] = T(fmax(kp.tau[e], kp.tau[t[0]]));
  } else if (grp.rank() == 0) {
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
    int wl = 0;
    if (c[d] < 0 || c[d] >= kp.nc[d]) {
      if (kp.periodic[d])
        c[d] = (c[d] + kp.nc[d]) % kp.nc[d];
      else
        wl = 1;
    }
    const int n = wl ? -1 : c[0] + kp.nc[0] * (c[1] + kp.nc[1] * c[2]);
    eo[0] = e;
    en[0] = n;
    const double te = kp.tau[e];
    tau_f[0] = T(wl ? te : fmax(te, kp.tau[n]));
  }
  grp.sync();
  const T* Ud = static_cast<const T*>(kp.Udev);
  const int* ocp = kp.flist ? oc : nullptr;
  if (GEO == GEO_FLY) {
    const T* X = static_cast<const T*>(kp.xyzT);
    for (int r = grp.rank(); r < 3 * N3; r += 32) {
      sx[r] = X[(size_t)eo[0] * 3 * N3 + r];
      // the other cell's coordinates, on rotated-frame meshes reoriented into the own cell's frame
      const int cq = r / N3;
      const int rn = ocp ? cq * N3 + frame_node<N>(ocp[0], r - cq * N3) : r;
      sxn[r] = X[(size_t)(en[0] >= 0 ? en[0] : eo[0]) * 3 * N3 + rn];
    }
    grp.sync();
  }
  if (d == 0)
    face_pair_terms<T, N, QC, QV, 1, 0, GEO>(U, Ud, eo, en, tau_f, lay, fa, lc, tb, kp, ph, 1, s, FB, grp, sx, sxn, go,
                                             ocp);
  else if (d == 1)
    face_pair_terms<T, N, QC, QV, 1, 1, GEO>(U, Ud, eo, en, tau_f, lay, fa, lc, tb, kp, ph, 1, s, FB, grp, sx, sxn, go,
                                             ocp);
  else
    face_pair_terms<T, N, QC, QV, 1, 2, GEO>(U, Ud, eo, en, tau_f, lay, fa, lc, tb, kp, ph, 1, s, FB, grp, sx, sxn, go,
                                             ocp);
}

template <typename T, int N, int QC, int QV, int GEO>
int launch_faces(const KParams& kp, const double* U, void* FB, cudaStream_t st) {
  int extra_items = 0;
  for (int d = 0; d < 3; ++d) {
    if (kp.periodic[d]) continue;
    const int plane = kp.nc[d == 0 ? 1 : 0] * kp.nc[d == 2 ? 1 : 2];
    if (plane > extra_items) extra_items = plane;
  }
  if constexpr (sizeof(T) == 4 && GEO == GEO_AFFINE && DGCNS_FP32_TASK_FACES && task_faces_ok<N, QC, QV>()) {
    if (kp.Udev != nullptr && kp.flist == nullptr) return launch_task_faces<N, QC, QV>(kp, FB, st);
  }
  // rotated-frame meshes: per direction, the blocks of the (d, 1) list, then those of the (d, 0) list
  auto list_blocks = [&](int per) {
    int g = 0;
    for (int d = 0; d < 3; ++d) {
      const int b = (kp.flen[2 * d + 1] + per - 1) / per + (kp.flen[2 * d] + per - 1) / per;
      if (b > g) g = b;
    }
    return g;
  };
  if constexpr (sizeof(T) == 4) {
    constexpr int WPC = 8;
    constexpr size_t smem = face_warp_smem_bytes<T, N, QC, QV, WPC, GEO>();
    static_assert(smem <= 227 * 1024, "face kernel shared memory");
    auto k = dg_face_warp_kernel<T, N, QC, QV, WPC, GEO>;
    static bool attr[kMaxDevices] = {};
    if (smem_attr_once(k, smem, attr)) return -1;
    const dim3 grid(kp.flist ? list_blocks(WPC) : (kp.Nc + WPC - 1) / WPC + (extra_items + WPC - 1) / WPC, 3);
    k<<<grid, WPC * 32, smem, st>>>(kp, U, static_cast<T*>(FB));
  } else {
    constexpr int CB = faces_per_cta<T, N, QC, QV, GEO>();
    constexpr size_t smem = face_smem_bytes<T, N, QC, QV, CB, GEO>();
    static_assert(smem <= 227 * 1024, "face kernel shared memory");
    auto k = dg_face_kernel<T, N, QC, QV, CB, GEO>;
    static bool attr[kMaxDevices] = {};
    if (smem_attr_once(k, smem, attr)) return -1;
    const dim3 grid(kp.flist ? list_blocks(CB) : (kp.Nc + CB - 1) / CB + (extra_items + CB - 1) / CB, 3);
    k<<<grid, face_threads<T, GEO>(), smem, st>>>(kp, U, static_cast<T*>(FB));
  }
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

template <typename T, int N, int QC, int QV>
int faces_dispatch(const KParams& kp, const double* U, void* FB, cudaStream_t st) {
  using F = Feat<N, QC, QV>;
  if constexpr (!F::faces || (sizeof(T) == 4 && !F::fp32)) {
    return -2;
  } else {
    if (kp.xyzT != nullptr) {
      if constexpr (F::fly) return launch_faces<T, N, QC, QV, GEO_FLY>(kp, U, FB, st);
      return -2;
    }
    if (kp.gcc != nullptr) {
      if constexpr (F::geo) return launch_faces<T, N, QC, QV, GEO_STORED>(kp, U, FB, st);
      return -2;
    }
    return launch_faces<T, N, QC, QV, GEO_AFFINE>(kp, U, FB, st);
  }
}

// One part of the launcher table of (N, QC, QV); each part is its own translation unit so that the
// instantiations compile in parallel.
template <int N, int QC, int QV, int PART>
void fill_launchers(Launchers& L) {
  static_assert(PART >= 0 && PART < DGCNS_PARTS && DGCNS_PARTS == 7, "parts");
  L.const_tables[PART] = upload_const_tables<N, QC, QV>;
  if constexpr (PART == 0) {  // FP64 operator
    L.features = Feat<N, QC, QV>::bits;
    L.op_fp64 = op_dispatch<double, N, QC, QV>;
    L.cb_fp64 = cells_per_cta<double, N, QC, QV>();
    L.gws_fp64 = op_gws_bytes<double, N, QC, QV>();
  } else if constexpr (PART == 1) {  // FP32 operator (mixed form)
    L.op_fp32 = op_dispatch<float, N, QC, QV>;
    L.dev_fp32 = dev_launch<float, N>;
    L.cb_fp32 = cells_per_cta<float, N, QC, QV>();
  } else if constexpr (PART == 2) {  // diagnostics, geometry, kinetic-energy gradient
    L.diag_fp64 = diag_launch<double, N, QC, QV>;
    L.diag_fp32 = diag_launch<float, N, QC, QV>;
    L.geom = geom_launch<N, QC, QV>;
    L.ekgrad = ekgrad_launch<N, QC, QV>;
  } else if constexpr (PART == 3) {  // adjoint
    L.adj_fp64 = adj_launch<double, N, QC, QV>;
    L.adj_fp32 = adj_launch<float, N, QC, QV>;
    L.prep_fp64 = adj_prep_launch<double>;
    L.prep_fp32 = adj_prep_launch<float>;
  } else if constexpr (PART == 4) {  // face-centric face kernel, FP64
    L.faces_fp64 = faces_dispatch<double, N, QC, QV>;
  } else if constexpr (PART == 5) {  // face-centric face kernel, FP32
    L.faces_fp32 = faces_dispatch<float, N, QC, QV>;
  } else {  // face-centric adjoint face kernels
    L.adj_faces_fp64 = adj_faces_dispatch<double, N, QC, QV>;
    L.adj_faces_fp32 = adj_faces_dispatch<float, N, QC, QV>;
  }
}

}  // namespace dgcns
