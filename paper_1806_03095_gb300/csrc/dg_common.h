// Shared host/device declarations of libdgcns (not part of the public ABI).
#pragma once
#include <cstdint>

namespace dgcns {

// Offsets (in elements) of the 1D tables inside one contiguous table buffer.
// Every table is computed on the host in FP64 and stored once as double and
// once as float.  Matrices are row-major [rows][cols].
struct TableLayout {
  int N, QC, QV;
  int Sc, Dc;   // Sc[QC][N]  l_i(x_q), convective Gauss points; Dc[QC][QC] collocation derivative
  int Sv, Dv;   // Sv[QV][N], Dv[QV][QV]  same for the viscous points
  int Sm, Smi;  // Sm[N][N] at the N = k+1 mass points; Smi = Sm^-1
  int wc, wv, wm;  // 1D Gauss weights on [0,1]
  int dl0, dl1;    // dl0[i] = l_i'(0), dl1[i] = l_i'(1)
  int total;
};

constexpr TableLayout make_layout(int N, int QC, int QV) {
  TableLayout L{};
  L.N = N; L.QC = QC; L.QV = QV;
  int o = 0;
  L.Sc = o; o += QC * N;
  L.Dc = o; o += QC * QC;
  L.Sv = o; o += QV * N;
  L.Dv = o; o += QV * QV;
  L.Sm = o; o += N * N;
  L.Smi = o; o += N * N;
  L.wc = o; o += QC;
  L.wv = o; o += QV;
  L.wm = o; o += N;
  L.dl0 = o; o += N;
  L.dl1 = o; o += N;
  L.total = (o + 3) & ~3;
  return L;
}

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
  double h[3];          // affine cell extents
  double bf[3];         // body force vector
  double A, B, dt;      // 2N stage coefficients (out_mode 2)
  const double* tau;    // [Nc] penalty per cell (FP64)
  const void* tables;   // device tables of the kernel's precision
};

}  // namespace dgcns
