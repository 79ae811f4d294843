// Host-visible launcher table of one (N, QC, QV) instantiation.
#pragma once
#include <cuda_runtime.h>

#include "dg_common.h"

namespace dgcns {

enum { OP_CELL = 1, OP_FACE = 2, OP_MASS = 4 };

using OpFn = int (*)(int mode, const KParams&, const double* U, const void* Rin, void* Rout, void* dU, double* Uout,
                     cudaStream_t);
// partial == nullptr: only report the number of blocks (partial sums needed).
using DiagFn = int (*)(const KParams&, const double* U, const void* LU, double* partial, int* nblocks,
                       cudaStream_t);

using GeomFn = int (*)(const KParams&, const double* xyz, double* gcc, double* gcv, double* gfc, double* gfv,
                      double* gm, double* tau, double* vol, double nu_kk, cudaStream_t);

// Adjoint: G = -(dF/dU)^T Y (lamU == nullptr) or lamU += dt * that (out_mode 2 in kp).
using AdjFn = int (*)(const KParams&, const double* U, const void* Y, void* G, double* lamU, cudaStream_t);
// Face-centric adjoint face kernel: shares of (dF/dU)^T Y of every face into FB.
using AdjFaceFn = int (*)(const KParams&, const double* U, const void* Y, void* FB, cudaStream_t);
using PrepFn = int (*)(size_t n, double A, double B, const double* lamU, void* lamdU, void* W, cudaStream_t);
// Face-centric face integrals: the face shares of every cell into FB ([Nc][6][2][5][N^2]).
using FaceFn = int (*)(const KParams&, const double* U, void* FB, cudaStream_t);
// G = d e_k / dU (FP64), e_k = (1/V) int |u|^2 / 2 at the convective points.
using EkGradFn = int (*)(const KParams&, const double* U, double* G, double inv_volume, cudaStream_t);

// Feature bits of an instantiation (only what the workloads and tests use is compiled, to keep
// the build short): FP32 (mixed form), stored non-affine geometry, geometry on the fly, adjoint,
// the face-centric organisation.
enum { FEAT_FP32 = 1, FEAT_GEO = 2, FEAT_FLY = 4, FEAT_ADJ = 8, FEAT_FACES = 16 };

template <int N, int QC, int QV>
struct Feat {
  static constexpr bool rule = QC == (3 * (N - 1)) / 2 + 1 && QV == N;  // 3/2-rule convective, k+1 viscous
  static constexpr bool fp32 = rule && (N == 4 || N == 5 || N == 6);   // k = 3, 4, 5
  static constexpr bool geo = rule && (N == 3 || N == 4 || N == 6);    // k = 2, 3, 5
  static constexpr bool fly = rule && N == 4;                          // k = 3
  static constexpr bool adj = rule && (N == 3 || N == 4 || N == 5);    // k = 2, 3, 4
  static constexpr bool faces = true;
  static constexpr int bits = (fp32 ? FEAT_FP32 : 0) | (geo ? FEAT_GEO : 0) | (fly ? FEAT_FLY : 0) |
                              (adj ? FEAT_ADJ : 0) | (faces ? FEAT_FACES : 0);
};

struct Launchers {
  int features;
  OpFn op_fp64, op_fp32;
  FaceFn faces_fp64, faces_fp32;
  DiagFn diag_fp64, diag_fp32;
  GeomFn geom;
  AdjFn adj_fp64, adj_fp32;
  AdjFaceFn adj_faces_fp64, adj_faces_fp32;
  PrepFn prep_fp64, prep_fp32;
  EkGradFn ekgrad;
  int (*dev_fp32)(const KParams&, const double* U, void* D, cudaStream_t);  // D = float(U - U_ref)
  int cb_fp64, cb_fp32;
  // bytes per CTA of the global workspace of the CTA-wide operator kernels (0: everything in shared memory)
  size_t gws_fp64;
  // per part: write the 1D tables (layout of make_layout, FP64 and FP32) to the part's constant memory on
  // the current device
  int (*const_tables[7])(const double* t64, const float* t32, cudaStream_t);
};

// (N = k+1, QC, QV) triples compiled into the library.  Default rules:
// QC = floor(3k/2)+1 (3/2-rule, Sec. 2.2.3) and QV = k+1 (k = 1..8, 11, 15); plus the
// standard rule QC = QV = k+1 at k = 3, 5, the paper's own setting with the 3/2
// rule on both terms (QV = QC) at k = 2..5, and the 2k+1 rule on both terms
// (QC = QV = 2k+1) at k = 2..5 and 7 (Sec. 4.1.2, over-integration).  From k = 8 (and
// for the 2k+1 rule from k = 5) one cell's working set exceeds shared memory and the
// CTA-wide operator kernels use the global workspace.
#define DGCNS_CONFIGS(X) \
  X(2, 2, 2)             \
  X(3, 4, 3)             \
  X(4, 5, 4)             \
  X(5, 7, 5)             \
  X(6, 8, 6)             \
  X(7, 10, 7)            \
  X(8, 11, 8)            \
  X(4, 4, 4)             \
  X(6, 6, 6)             \
  X(3, 4, 4)             \
  X(4, 5, 5)             \
  X(5, 7, 7)             \
  X(6, 8, 8)             \
  X(3, 5, 5)             \
  X(4, 7, 7)             \
  X(5, 9, 9)             \
  X(6, 11, 11)           \
  X(8, 15, 15)           \
  X(9, 13, 9)            \
  X(12, 17, 12)          \
  X(16, 23, 16)

// Parts of each instantiation (separate translation units): FP64 operator, FP32 operator,
// diagnostics + geometry, adjoint, FP64 face kernel, FP32 face kernel, adjoint face kernels.
#define DGCNS_PARTS 7
#define DGCNS_DECLARE(N, QC, QV)                     \
  void launchers_##N##_##QC##_##QV##_0(Launchers&); \
  void launchers_##N##_##QC##_##QV##_1(Launchers&); \
  void launchers_##N##_##QC##_##QV##_2(Launchers&); \
  void launchers_##N##_##QC##_##QV##_3(Launchers&); \
  void launchers_##N##_##QC##_##QV##_4(Launchers&); \
  void launchers_##N##_##QC##_##QV##_5(Launchers&); \
  void launchers_##N##_##QC##_##QV##_6(Launchers&);
DGCNS_CONFIGS(DGCNS_DECLARE)
#undef DGCNS_DECLARE

}  // namespace dgcns
