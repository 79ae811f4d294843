// Cell kernel of the mixed form's face-centric organisation (FP32 arithmetic, affine meshes, k = 3):
// cell integrals (Sec. 2.2.2: -(grad V, F_c) + (grad V, F_v)), the cell's face shares, the inverse mass
// matrix (Sec. 2.3) and the 2N stage update (Sec. 2.4) -- the same operations as dg_op_warp_kernel with
// CELL and MASS, organised so that the 1D contractions run in registers.  A thread takes one xy-plane
// (fixed z) or one z-line of one component of one cell at a time:
//
//  1. plane tasks (cell, component, z = j): the plane's 4 x-lines come from the FP32 deviation state; S
//     along x and y for the convective points, S along x and y and the x and y collocation derivatives for
//     the viscous points, in registers;
//  2. line tasks (cell, component, x, y point): S along z finishes the interpolation (and D along z gives
//     the viscous z derivative);
//  3. point tasks: the convective flux (contravariant, times the quadrature weight) and the viscous flux;
//  4. line tasks: S^T along z of the flux's x and y parts, S^T D^T along z of its z part;
//  5. plane tasks: D^T along x and y, S^T along x and y, plus the 6 face shares of the plane's nodes (face
//     buffer), then S_m^-T along x and y of the inverse mass matrix;
//  6. line tasks: S_m^-T along z, the scaling by -1 / (|J| w), S_m^-1 along z;
//  7. plane tasks: S_m^-1 along x and y, then the stage update (or L itself) written to global memory.
//
// Each phase's results go to shared memory once; every array is laid out so that the tasks of a
// quarter-warp meet distinct banks.
#pragma once
#include "dg_faces_fp32.cuh"

namespace dgcns {

// Shared-memory layout per cell (floats).  Region X: plane results of phase 1 (convective [5][N][QC^2],
// viscous [5][N][VP] with the S_xy values and the x and y derivatives, VP = 3 QV^2 + 4), later the
// line results of phase 4 (convective [5][N][3 QC^2], viscous [5][N][VP]).  Region Y: point values and
// fluxes (convective [3][5][QC^3], the x flux in place of the values; viscous [5][4][QV^3]), later the
// inverse-mass planes of the two parts of phase 5, [2][5][N][N^2].
template <int N, int QC, int QV>
struct TaskCellSizes {
  static constexpr int PC2 = QC * QC, PV2 = QV * QV, PC3 = QC * QC * QC, PV3 = QV * QV * QV, N2 = N * N;
  static constexpr int VP = 3 * PV2 + 4;
  static constexpr int AC = 5 * N * PC2, AV = 5 * N * VP;
  static constexpr int BC = 5 * N * 3 * PC2, BV = 5 * N * VP;
  static constexpr int XR = ((AC + AV > BC + BV ? AC + AV : BC + BV) + 3) & ~3;
  static constexpr int FC = 3 * 5 * PC3, PVS = 5 * 4 * PV3, MS = 5 * N * N2;
  static constexpr int YR = ((FC + PVS > 2 * MS ? FC + PVS : 2 * MS) + 3) & ~3;
  static constexpr int RAW = XR + YR;
  static constexpr int PER_CELL = RAW + ((8 - RAW % 32) + 32) % 32;
};

template <int N, int QC, int QV, int CPB>
constexpr size_t task_cell_smem_bytes() {
  return ((size_t)table_elems<N, QC, QV>() + 4 + (size_t)CPB * TaskCellSizes<N, QC, QV>::PER_CELL) * sizeof(float) +
         64;
}

// Phase 1: plane (cell e, component c, z = j) of the deviation state -> convective S_x S_y values and
// viscous S_x S_y values with their x and y collocation derivatives.
template <int N, int QC, int QV>
__device__ __forceinline__ void cell_plane_interp(const float* __restrict__ src, const Tab<float>& tb, bool conv,
                                                  bool visc, float* ac, float* av) {
  constexpr int N2 = N * N, PC2 = QC * QC, PV2 = QV * QV;
  float X[N2];
#pragma unroll
  for (int y = 0; y < N; ++y) {
    float x[N];
    vec_load<float, N>(src + y * N, x);
#pragma unroll
    for (int a = 0; a < N; ++a) X[y * N + a] = x[a];
  }
  if (conv) {
    float Y[PC2];
    eo_2d<N, N, QC, QC, 1, 1>(tb.eSc, tb.eSc, X, Y);
#pragma unroll
    for (int p = 0; p < PC2; ++p) ac[p] = Y[p];
  }
  if (visc) {
    float V[PV2], G[PV2];
    eo_2d<N, N, QV, QV, 1, 1>(tb.eSv, tb.eSv, X, V);
    vec_store<float, PV2>(av, V);
    eo_dir0<QV, QV, QV, -1>(tb.eDv, V, G);
    vec_store<float, PV2>(av + PV2, G);
    eo_dir1<QV, QV, QV, -1>(tb.eDv, V, G);
    vec_store<float, PV2>(av + 2 * PV2, G);
  }
}


// CELL + face shares + MASS (+ stage update) of CPB consecutive cells per CTA.  kp.out_mode: 1 writes
// L(U) to Rout, 2 the stage update (dU <- A dU + dt L, U_out <- U + B dU in FP64, and with kp.devOut the
// next stage's deviation state float(U_out - U_ref)).  kp.Udev: the FP32 deviation state; kp.fbuf: the
// face shares of the face-centric face kernel.
template <int N, int QC, int QV, int CPB, int NTH>
__global__ void __launch_bounds__(NTH) dg_cell_task_kernel(const KParams kp, const double* __restrict__ U,
                                                           float* __restrict__ Rout, float* __restrict__ dU,
                                                           double* __restrict__ Uout) {
  using S = TaskCellSizes<N, QC, QV>;
  constexpr int N2 = N * N, N3 = N * N * N, PC2 = S::PC2, PV2 = S::PV2, PC3 = S::PC3, PV3 = S::PV3;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* stab = reinterpret_cast<float*>(smem_raw);
  float* scell = stab + ((table_elems<N, QC, QV>() + 3) & ~3);
  const int e0 = blockIdx.x * CPB;
  const int nb = min(CPB, kp.Nc - e0);
  if (nb <= 0) return;
  const Tab<float> tb = load_tables<float, N, QC, QV>(static_cast<const float*>(kp.tables), stab);
  const PhysT<float> ph = make_phys<float>(kp);
  const KConst<float>& kc = kconst<float>(kp);
  const float hinv[3] = {kc.hinv[0], kc.hinv[1], kc.hinv[2]};
  const float detJ = kc.detJ;
  const float* __restrict__ Ud = static_cast<const float*>(kp.Udev);
  const bool conv = kp.conv != 0, visc = kp.visc != 0;
  __syncthreads();

  // 1. plane tasks: (b, c, j, part): part 0 the convective, part 1 the viscous interpolation
  for (int t = threadIdx.x; t < nb * 10 * N; t += NTH) {
    const int b = t / (10 * N), r = t - 10 * N * b, part = r / (5 * N), r2 = r - 5 * N * part, c = r2 / N,
              j = r2 - N * c;
    float* X = scell + b * S::PER_CELL;
    cell_plane_interp<N, QC, QV>(Ud + ((size_t)(e0 + b) * 5 + c) * N3 + j * N2, tb, conv && part == 0,
                                 visc && part == 1, X + (c * N + j) * PC2, X + S::AC + (c * N + j) * S::VP);
  }
  __syncthreads();

  // 2. line tasks: convective (b, c, point (q0, q1)) and viscous (b, c, point (q0, q1)): S along z
  {
    constexpr int TC = 5 * PC2, TV = 5 * PV2;
    const int ntc = conv ? nb * TC : 0, ntv = visc ? nb * TV : 0;
    for (int t = threadIdx.x; t < ntc + ntv; t += NTH) {
      if (t < ntc) {
        const int b = t / TC, r = t - TC * b, c = r / PC2, q = r - PC2 * c;
        float* X = scell + b * S::PER_CELL;
        float* Y = X + S::XR;
        float x[N], y[QC];
#pragma unroll
        for (int j = 0; j < N; ++j) x[j] = X[(c * N + j) * PC2 + q];
        eo_apply<N, QC, 1>(tb.eSc, x, y);
#pragma unroll
        for (int k = 0; k < QC; ++k) Y[c * PC3 + k * PC2 + q] = y[k];
      } else {
        const int tt = t - ntc, b = tt / TV, r = tt - TV * b, c = r / PV2, q = r - PV2 * c;
        float* X = scell + b * S::PER_CELL;
        float* Y = X + S::XR + S::FC + c * 4 * PV3;
        const float* av = X + S::AC + c * N * S::VP + q;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          float x[N], y[QV];
#pragma unroll
          for (int j = 0; j < N; ++j) x[j] = av[j * S::VP + a * PV2];
          eo_apply<N, QV, 1>(tb.eSv, x, y);
#pragma unroll
          for (int k = 0; k < QV; ++k) Y[a * PV3 + k * PV2 + q] = y[k];
          if (a == 0) {
            float g[QV];
            eo_apply<QV, QV, -1>(tb.eDv, y, g);
#pragma unroll
            for (int k = 0; k < QV; ++k) Y[3 * PV3 + k * PV2 + q] = g[k];
          }
        }
      }
    }
  }
  __syncthreads();

  // 3. point tasks: convective fluxes -F_c J^{-T} |J| w (x part in place of the values), viscous fluxes
  //    F_v J^{-T} |J| w (in place of the three gradient arrays)
  {
    const int ntc = conv ? nb * PC3 : 0, ntv = visc ? nb * PV3 : 0;
    for (int t = threadIdx.x; t < ntc + ntv; t += NTH) {
      if (t < ntc) {
        const int b = t / PC3, p = t - PC3 * b;
        float* Y = scell + b * S::PER_CELL + S::XR;
        const int q0 = p % QC, q1 = (p / QC) % QC, q2 = p / PC2;
        const float w = tb.wc[q0] * tb.wc[q1] * tb.wc[q2] * detJ;
        float u[5];
#pragma unroll
        for (int c = 0; c < 5; ++c) u[c] = Y[c * PC3 + p];
        const float rinv = 1.f / (ph.rho_r + u[0]);
        const float dp = pressure_dev(u, rinv, ph.gm1);
#pragma unroll
        for (int jd = 0; jd < 3; ++jd) {
          float f[5];
          conv_flux_dir(u, rinv, dp, ph.H_r, jd, f);
          const float sc = -w * hinv[jd];
#pragma unroll
          for (int c = 0; c < 5; ++c) Y[(jd * 5 + c) * PC3 + p] = sc * f[c];
        }
      } else {
        const int tt = t - ntc, b = tt / PV3, p = tt - PV3 * b;
        float* Y = scell + b * S::PER_CELL + S::XR + S::FC;
        const int q0 = p % QV, q1 = (p / QV) % QV, q2 = p / PV2;
        const float w = tb.wv[q0] * tb.wv[q1] * tb.wv[q2] * detJ;
        float u[5], Gr[5][3], F[5][3];
#pragma unroll
        for (int c = 0; c < 5; ++c) {
          const float* q = Y + c * 4 * PV3 + p;
          u[c] = q[0];
          Gr[c][0] = q[PV3] * hinv[0];
          Gr[c][1] = q[2 * PV3] * hinv[1];
          Gr[c][2] = q[3 * PV3] * hinv[2];
        }
        visc_flux(u, Gr, ph, F);
#pragma unroll
        for (int c = 0; c < 5; ++c) {
          float* q = Y + c * 4 * PV3 + p;
#pragma unroll
          for (int jd = 0; jd < 3; ++jd) q[(jd + 1) * PV3] = w * hinv[jd] * F[c][jd];
        }
      }
    }
  }
  __syncthreads();

  // 4. line tasks: S^T along z of the x and y flux parts, S^T D^T along z of the z part
  {
    constexpr int TC = 5 * PC2, TV = 5 * PV2;
    const int ntc = conv ? nb * TC : 0, ntv = visc ? nb * TV : 0;
    for (int t = threadIdx.x; t < ntc + ntv; t += NTH) {
      if (t < ntc) {
        const int b = t / TC, r = t - TC * b, c = r / PC2, q = r - PC2 * c;
        float* X = scell + b * S::PER_CELL;
        const float* Y = X + S::XR;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          float x[QC], y[N];
#pragma unroll
          for (int k = 0; k < QC; ++k) x[k] = Y[(a * 5 + c) * PC3 + k * PC2 + q];
          if (a == 2) {
            float g[QC];
            eo_apply<QC, QC, -1>(tb.eDcT, x, g);
            eo_apply<QC, N, 1>(tb.eScT, g, y);
          } else {
            eo_apply<QC, N, 1>(tb.eScT, x, y);
          }
#pragma unroll
          for (int j = 0; j < N; ++j) X[((c * N + j) * 3 + a) * PC2 + q] = y[j];
        }
      } else {
        const int tt = t - ntc, b = tt / TV, r = tt - TV * b, c = r / PV2, q = r - PV2 * c;
        float* X = scell + b * S::PER_CELL;
        const float* Y = X + S::XR + S::FC + c * 4 * PV3;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          float x[QV], y[N];
#pragma unroll
          for (int k = 0; k < QV; ++k) x[k] = Y[(a + 1) * PV3 + k * PV2 + q];
          if (a == 2) {
            float g[QV];
            eo_apply<QV, QV, -1>(tb.eDvT, x, g);
            eo_apply<QV, N, 1>(tb.eSvT, g, y);
          } else {
            eo_apply<QV, N, 1>(tb.eSvT, x, y);
          }
#pragma unroll
          for (int j = 0; j < N; ++j) X[S::BC + (c * N + j) * S::VP + a * PV2 + q] = y[j];
        }
      }
    }
  }
  __syncthreads();

  // 5. plane tasks (b, c, j, part): D^T along x and y and S^T along x and y of the convective (part 0) or
  //    the viscous terms together with the face shares of the plane's nodes (part 1), then S_m^-T along x
  //    and y of that part (the inverse mass matrix is linear: the parts are summed in phase 6)
  const float* __restrict__ FBf = static_cast<const float*>(kp.fbuf);
  for (int t = threadIdx.x; t < nb * 10 * N; t += NTH) {
    const int b = t / (10 * N), r = t - 10 * N * b, part = r / (5 * N), r2 = r - 5 * N * part, c = r2 / N,
              j = r2 - N * c;
    const int cell = e0 + b;
    float* X = scell + b * S::PER_CELL;
    float R[N2];
#pragma unroll
    for (int n = 0; n < N2; ++n) R[n] = 0.f;
    if (conv && part == 0) {
      const float* B = X + (c * N + j) * 3 * PC2;
      float A0[PC2], A1[PC2], T0[PC2], Y[N2];
#pragma unroll
      for (int p = 0; p < PC2; ++p) {
        A0[p] = B[p];
        A1[p] = B[PC2 + p];
      }
      eo_dir0<QC, QC, QC, -1>(tb.eDcT, A0, T0);
      eo_dir1<QC, QC, QC, -1>(tb.eDcT, A1, A0);
#pragma unroll
      for (int p = 0; p < PC2; ++p) T0[p] += A0[p] + B[2 * PC2 + p];
      eo_2d<QC, QC, N, N, 1, 1>(tb.eScT, tb.eScT, T0, Y);
#pragma unroll
      for (int n = 0; n < N2; ++n) R[n] = Y[n];
    }
    if (visc && part == 1) {
      const float* B = X + S::BC + (c * N + j) * S::VP;
      float A0[PV2], A1[PV2], T0[PV2], Y[N2];
      vec_load<float, PV2>(B, A0);
      vec_load<float, PV2>(B + PV2, A1);
      eo_dir0<QV, QV, QV, -1>(tb.eDvT, A0, T0);
      eo_dir1<QV, QV, QV, -1>(tb.eDvT, A1, A0);
      vec_load<float, PV2>(B + 2 * PV2, A1);
#pragma unroll
      for (int p = 0; p < PV2; ++p) T0[p] += A0[p] + A1[p];
      eo_2d<QV, QV, N, N, 1, 1>(tb.eSvT, tb.eSvT, T0, Y);
#pragma unroll
      for (int n = 0; n < N2; ++n) R[n] += Y[n];
    }
    if (FBf != nullptr && part == 1) {
      // face f = 2d + s: value-layer share L (nodes on the face) and normal-derivative share D (every node
      // of the normal line, weighted by l_i'(face)); face node index: first tangent fastest
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        const float* dl = s ? tb.dl1 : tb.dl0;
        const int end = s ? N - 1 : 0;
        {  // d = 0: face node (y, z)
          const float* F = FBf + (((size_t)cell * 6 + s) * 2 * 5 + c) * N2 + N * j;
          float Lf[N], Df[N];
          vec_load<float, N>(F, Lf);
          vec_load<float, N>(F + 5 * N2, Df);
#pragma unroll
          for (int y = 0; y < N; ++y)
#pragma unroll
            for (int x = 0; x < N; ++x) R[y * N + x] = fmaf(dl[x], Df[y], R[y * N + x]) + (x == end ? Lf[y] : 0.f);
        }
        {  // d = 1: face node (x, z)
          const float* F = FBf + (((size_t)cell * 6 + 2 + s) * 2 * 5 + c) * N2 + N * j;
          float Lf[N], Df[N];
          vec_load<float, N>(F, Lf);
          vec_load<float, N>(F + 5 * N2, Df);
#pragma unroll
          for (int y = 0; y < N; ++y)
#pragma unroll
            for (int x = 0; x < N; ++x) R[y * N + x] = fmaf(dl[y], Df[x], R[y * N + x]) + (y == end ? Lf[x] : 0.f);
        }
        {  // d = 2: face node (x, y)
          const float* F = FBf + (((size_t)cell * 6 + 4 + s) * 2 * 5 + c) * N2;
          float Df[N2];
          vec_load<float, N2>(F + 5 * N2, Df);
          const float w = dl[j];
#pragma unroll
          for (int n = 0; n < N2; ++n) R[n] = fmaf(w, Df[n], R[n]);
          if (j == end) {
            float Lf[N2];
            vec_load<float, N2>(F, Lf);
#pragma unroll
            for (int n = 0; n < N2; ++n) R[n] += Lf[n];
          }
        }
      }
    }
    float M[N2];
    eo_2d<N, N, N, N, 1, 1>(tb.eSmiT, tb.eSmiT, R, M);
    vec_store<float, N2>(X + S::XR + part * S::MS + (c * N + j) * N2, M);
  }
  __syncthreads();

  // 6. line tasks (b, c, node (x, y)): S_m^-T along z, scaling by -1 / (|J| w), S_m^-1 along z
  for (int t = threadIdx.x; t < nb * 5 * N2; t += NTH) {
    const int b = t / (5 * N2), r = t - 5 * N2 * b, c = r / N2, q = r - N2 * c;
    float* Mp = scell + b * S::PER_CELL + S::XR + c * N * N2 + q;
    float x[N], y[N];
#pragma unroll
    for (int k = 0; k < N; ++k) x[k] = Mp[k * N2] + Mp[S::MS + k * N2];
    eo_apply<N, N, 1>(tb.eSmiT, x, y);
    const float wxy = tb.wm[q % N] * tb.wm[q / N] * detJ;
#pragma unroll
    for (int k = 0; k < N; ++k) y[k] *= -1.f / (wxy * tb.wm[k]);
    eo_apply<N, N, 1>(tb.eSmi, y, x);
#pragma unroll
    for (int k = 0; k < N; ++k) Mp[k * N2] = x[k];
  }
  __syncthreads();

  // 7. plane tasks (b, c, j): S_m^-1 along x and y -> L, stored for the whole batch in the cell layout
  //    ([b][c][z][y][x], in the first cell's region X, free since phase 5)
  float* Lb = scell;
  for (int t = threadIdx.x; t < nb * 5 * N; t += NTH) {
    const int b = t / (5 * N), r = t - 5 * N * b, c = r / N, j = r - N * c;
    float Mv[N2], L[N2];
    vec_load<float, N2>(scell + b * S::PER_CELL + S::XR + (c * N + j) * N2, Mv);
    eo_2d<N, N, N, N, 1, 1>(tb.eSmi, tb.eSmi, Mv, L);
    vec_store<float, N2>(Lb + (b * 5 + c) * N3 + j * N2, L);
  }
  __syncthreads();
  // 8. L or the stage update, elementwise over the batch with every thread (coalesced global accesses;
  //    the FP64 accumulation of the state spread over all warps)
  const size_t base = (size_t)e0 * 5 * N3;
  const int nvals = nb * 5 * N3;
  if (kp.out_mode == 2) {
    stage_update<(CPB * 5 * N3 + NTH - 1) / NTH, N3>(kp, U, dU, Uout, Lb, base, nvals, threadIdx.x, NTH);
  } else {
    for (int i = threadIdx.x; i < nvals; i += NTH) Rout[base + i] = Lb[i];
  }
}

// The task cell kernel serves the FP32 affine face-centric cell + mass stage at k = 3 (k+1 viscous rule).
template <int N, int QC, int QV>
constexpr bool task_cell_ok() {
  return N == 4 && QV == N && (N * N) % 4 == 0 && ((QV * QV) % 4) == 0;
}

// Cells per CTA and threads of the task cell kernel (compile-time tuning parameters; mixed TGV 64^3,
// k = 3, per stage: 1 cell and 128 threads 2.24 ms, 2 cells 2.40 ms, 3 cells 2.73 ms, 4 cells 3.81 ms,
// 1 cell and 64 threads 2.44 ms; the warp-per-cell kernel 2.28 ms; measured).
#ifndef DGCNS_FP32_CELL_CPB
#define DGCNS_FP32_CELL_CPB 1
#endif
#ifndef DGCNS_FP32_CELL_NTH
#define DGCNS_FP32_CELL_NTH 128
#endif

template <int N, int QC, int QV>
int launch_task_cell(const KParams& kp, const double* U, void* Rout, void* dU, double* Uout, cudaStream_t st) {
  constexpr int CPB = DGCNS_FP32_CELL_CPB, NTH = DGCNS_FP32_CELL_NTH;
  constexpr size_t smem = task_cell_smem_bytes<N, QC, QV, CPB>();
  static_assert(smem <= 227 * 1024, "task cell kernel shared memory");
  auto k = dg_cell_task_kernel<N, QC, QV, CPB, NTH>;
  static bool attr[kMaxDevices] = {};
  if (smem_attr_once(k, smem, attr)) return -1;
  const int grid = (kp.Nc + CPB - 1) / CPB;
  k<<<grid, NTH, smem, st>>>(kp, U, static_cast<float*>(Rout), static_cast<float*>(dU), Uout);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}
}  // namespace dgcns
