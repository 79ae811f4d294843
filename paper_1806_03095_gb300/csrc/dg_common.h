// Shared host/device declarations of libdgcns (not part of the public ABI).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace dgcns {

// Offsets (in elements) of the 1D tables inside one contiguous table buffer.
// Every table is computed on the host in FP64 and stored once as double and
// once as float.  The point sets (LGL nodes, Gauss points) are symmetric about
// 1/2, so every 1D operator O (DOUT x DIN) satisfies
// O[DOUT-1-q][DIN-1-i] = s O[q][i] with s = +1 (interpolation) or -1
// (derivative); it is stored in even-odd form (Sec. 2.3, even-odd
// decomposition): for q < ceil(DOUT/2), i < floor(DIN/2)
//   a[q][i] = (O[q][i] + O[q][DIN-1-i]) / 2,  b[q][i] = (O[q][i] - O[q][DIN-1-i]) / 2,
//   c[q]    = O[q][DIN/2] (middle column, DIN odd; else 0).
enum EoOp { EO_SC, EO_SCT, EO_DC, EO_DCT, EO_SV, EO_SVT, EO_DV, EO_DVT, EO_SMI, EO_SMIT, EO_SM, EO_DM, EO_NOPS };

constexpr int eo_size(int dout, int din) { return ((dout + 1) / 2) * (din / 2) * 2 + (dout + 1) / 2; }

struct TableLayout {
  int N, QC, QV;
  int eo[EO_NOPS];  // offsets of the even-odd operators
  int wc, wv, wm;   // 1D Gauss weights on [0,1]
  int dl0, dl1;     // dl0[i] = l_i'(0), dl1[i] = l_i'(1)
  int total;
};

constexpr TableLayout make_layout(int N, int QC, int QV) {
  TableLayout L{};
  L.N = N;
  L.QC = QC;
  L.QV = QV;
  int o = 0;
  const int dims[EO_NOPS][2] = {{QC, N}, {N, QC}, {QC, QC}, {QC, QC}, {QV, N}, {N, QV},
                                {QV, QV}, {QV, QV}, {N, N},   {N, N},   {N, N},  {N, N}};
  for (int k = 0; k < EO_NOPS; ++k) {
    L.eo[k] = o;
    o += eo_size(dims[k][0], dims[k][1]);
  }
  L.wc = o; o += QC;
  L.wv = o; o += QV;
  L.wm = o; o += N;
  L.dl0 = o; o += N;
  L.dl1 = o; o += N;
  L.total = (o + 3) & ~3;
  return L;
}

// Constants precomputed on the host in the kernel's precision, so that the FP32
// kernels issue no FP64 instruction for them (GB300 has 2 FP64 units per SM).
template <typename T>
struct KConst {
  T hinv[3], detJ, area[3];  // affine geometry: 1/h_d, h0 h1 h2, face area h_t1 h_t2 per direction d
  T gamma, gm1, mu, lam_cv;  // gamma, gamma - 1, mu, lambda / c_v
  T rho_r, rhoE_r, p_r, H_r; // reference state, its pressure and rhoE_r + p_r
  T cvTw2;                   // 2 c_v T_wall
  T bf[3];                   // body force
};

// Per-launch parameters (passed by value).
struct KParams {
  int Nc;
  int nc[3];
  int periodic[3];
  int conv, visc;       // evaluate convective / viscous terms
  int out_mode;         // 0: write F(U); 1: write L(U); 2: RK stage update
  int has_bf;           // body force present
  double gamma, mu, lam, cv;
  double Tw;            // wall temperature
  double rho_ref;       // reference state (rho_ref, 0, 0, 0, rho_ref c_v T_w): the kernels carry U - U_ref
  double rhoE_ref;
  double h[3];          // affine cell extents
  double bf[3];         // body force vector
  double A, B, dt;      // 2N stage coefficients (out_mode 2)
  const double* tau;    // [Nc] penalty per cell (FP64)
  const void* tables;   // device tables of the kernel's precision
  // Stored geometry (non-affine meshes), in the kernel's precision (quadrature weights excluded):
  //   gcc [Nc][10][QC^3], gcv [Nc][10][QV^3]: J^{-1}[b][a] (index 3b+a) and |det J| at cell points;
  //   gfc [Nc][6][13][QC^2], gfv [Nc][6][13][QV^2]: J^{-1} (9), unit outward normal n (3) and the
  //   area element dA = |det J| |J^{-T} n_xi| (1), face f = 2d + s;  gm [Nc][N^3]: |det J| at
  //   the k+1 mass points.
  const void *gcc, *gcv, *gfc, *gfv, *gm;
  // Optional deviation state U - U_ref already converted to the kernel's precision (same layout as U);
  // when set, the operator kernels read own and neighbour values from it instead of converting U.
  const void* Udev;
  // Node coordinates [Nc][3][N^3] in the kernel's precision (GEO_FLY: Jacobians recomputed in the kernels).
  const void* xyzT;
  // Face shares [Nc][6][2][5][N^2] written by the face-centric face kernel; when set, the cell kernel
  // (without FACE) adds them to the residual.
  const void* fbuf;
  // Optional output (mixed form, stage update): float(U_out - U_ref), the next stage's deviation state.
  void* devOut;
  // Device error word of the context: kernels with bounded waits set it to 1 when a wait gives up.
  int* err;
  // Rotated-frame meshes (DGCNS_MAP_ROTATED): per cell and local face [Nc][6][2] the neighbour cell and the
  // orientation code of its frame relative to the cell's (frame_node); nullptr on structured meshes.
  const int* fnbr;
  // Face-centric kernels on rotated-frame meshes: every face once, by the local face 2 d + s of the cell
  // that owns it; flist + foff[2 d + s] holds flen[2 d + s] owner cells (nullptr: structured enumeration).
  const int* flist;
  int foff[6], flen[6];
  // Operator kernels whose per-cell working set does not fit shared memory (high degrees): a global
  // workspace of gws_elems values of the arithmetic type, one slice per CTA; the launcher runs the grid
  // in chunks of as many CTAs as it holds, the first cell of a chunk in cell0 (0 otherwise).
  void* gws;
  size_t gws_elems;
  int cell0;
  KConst<double> cd;
  KConst<float> cf;
};

template <typename T>
void fill_kconst(const KParams& kp, KConst<T>& c) {
  for (int d = 0; d < 3; ++d) {
    c.hinv[d] = T(1.0 / kp.h[d]);
    c.area[d] = T(kp.h[(d + 1) % 3] * kp.h[(d + 2) % 3]);
    c.bf[d] = T(kp.bf[d]);
  }
  c.detJ = T(kp.h[0] * kp.h[1] * kp.h[2]);
  c.gamma = T(kp.gamma);
  c.gm1 = T(kp.gamma - 1.0);
  c.mu = T(kp.mu);
  c.lam_cv = T(kp.lam / kp.cv);
  c.rho_r = T(kp.rho_ref);
  c.rhoE_r = T(kp.rhoE_ref);
  c.p_r = T((kp.gamma - 1.0) * kp.rhoE_ref);
  c.H_r = T(kp.gamma * kp.rhoE_ref);
  c.cvTw2 = T(2.0 * kp.cv * kp.Tw);
}

constexpr int GEO_AFFINE = 0, GEO_STORED = 1, GEO_FLY = 2;

// Node index, in its own frame, of the neighbour's node that sits at node q = (i0, i1, i2) of the
// neighbour seen in the cell's frame: j_b = i_{src_b} or N - 1 - i_{src_b} (code bits: src_b at 2b, the
// reflection of axis b at 6 + b).
template <int N>
__host__ __device__ __forceinline__ int frame_node(int code, int q) {
  const int i0 = q % N, i1 = (q / N) % N, i2 = q / (N * N);
  int j[3];
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    const int src = (code >> (2 * b)) & 3;
    const int v = src == 0 ? i0 : (src == 1 ? i1 : i2);
    j[b] = ((code >> (6 + b)) & 1) ? N - 1 - v : v;
  }
  return j[0] + N * (j[1] + N * j[2]);
}

// The face of the neighbour that faces a cell across the cell's local face (d, s), seen through the
// orientation code of frame_node: the neighbour's axis dn that the cell's axis d maps to, whether it is
// reflected (then dV/dxi_d = -dV/dxi_dn), and the neighbour's side sn of that face.
__host__ __device__ __forceinline__ void frame_facing(int code, int d, int s, int& dn, int& refl, int& sn) {
  dn = ((code & 3) == d) ? 0 : (((code >> 2) & 3) == d ? 1 : 2);
  refl = (code >> (6 + dn)) & 1;
  sn = refl ? s : 1 - s;
}

// Dynamic shared-memory attribute of a kernel: a per-device setting, made once per (kernel, device) on
// the current device.  done[] is the kernel's own flag array (a static of its launcher).
constexpr int kMaxDevices = 64;
template <class K>
inline int smem_attr_once(K kernel, size_t smem, bool* done) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return -1;
  if (dev >= 0 && dev < kMaxDevices && done[dev]) return 0;
  if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return -1;
  if (dev >= 0 && dev < kMaxDevices) done[dev] = true;
  return 0;
}

}  // namespace dgcns
