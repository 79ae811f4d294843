// Host side of libdgcns: argument checks, the host plan (1D tables in FP64,
// penalty per cell, node coordinates), dispatch to the compiled (k, n_q)
// instantiations, and the C ABI of include/dgcns.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <functional>
#include <vector>

#include "dg_common.h"
#include "dg_launchers.h"
#include "dgcns.h"

using namespace dgcns;

// ---------------------------------------------------------------------------
// Low-storage RK(5,4), 2N form (Carpenter & Kennedy 1994, five stages, fourth order).
// ---------------------------------------------------------------------------
static const double RK_A[5] = {0.0, -567301805773.0 / 1357537059087.0, -2404267990393.0 / 2016746695238.0,
                               -3550918686646.0 / 2091501179385.0, -1275806237668.0 / 842570457699.0};
static const double RK_B[5] = {1432997174477.0 / 9575080441755.0, 5161836677717.0 / 13612068292357.0,
                               1720146321549.0 / 2090206949498.0, 3134564353537.0 / 4481467310338.0,
                               2277821191437.0 / 14882151754819.0};
// (The stage times C_i are not needed: the operator is autonomous, the body force constant.)

// ---------------------------------------------------------------------------
// 1D polynomial tables (FP64)
// ---------------------------------------------------------------------------
namespace {

// Legendre P_n and P_n' at x in [-1, 1] by the three-term recurrence.
void legendre(int n, double x, double* p, double* dp) {
  double p0 = 1.0, p1 = x;
  if (n == 0) {
    *p = 1.0;
    *dp = 0.0;
    return;
  }
  for (int m = 2; m <= n; ++m) {
    const double p2 = ((2 * m - 1) * x * p1 - (m - 1) * p0) / m;
    p0 = p1;
    p1 = p2;
  }
  *p = p1;
  // (1 - x^2) P_n' = n (P_{n-1} - x P_n)
  *dp = (std::fabs(1.0 - x * x) < 1e-300) ? 0.0 : n * (p0 - x * p1) / (1.0 - x * x);
}

// Gauss--Legendre points and weights on [0,1], ascending.
void gauss(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    double t = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; ++it) {
      double p, dp;
      legendre(n, t, &p, &dp);
      const double dt = p / dp;
      t -= dt;
      if (std::fabs(dt) < 1e-16) break;
    }
    double p, dp;
    legendre(n, t, &p, &dp);
    // t descends with i; store ascending on [0,1]
    x[n - 1 - i] = 0.5 * (1.0 + t);
    w[n - 1 - i] = 0.5 * 2.0 / ((1.0 - t * t) * dp * dp);
  }
}

// k+1 Legendre--Gauss--Lobatto points on [0,1]: 0, 1 and the roots of P_k'.
std::vector<double> lgl(int k) {
  std::vector<double> x(k + 1);
  x[0] = 0.0;
  x[k] = 1.0;
  for (int i = 1; i < k; ++i) {
    double t = std::cos(M_PI * i / k);
    for (int it = 0; it < 100; ++it) {
      double p, dp;
      legendre(k, t, &p, &dp);
      const double d2p = (2.0 * t * dp - k * (k + 1) * p) / (1.0 - t * t);  // Legendre ODE
      const double dt = dp / d2p;
      t -= dt;
      if (std::fabs(dt) < 1e-16) break;
    }
    x[k - i] = 0.5 * (1.0 + t);
  }
  return x;
}

// Lagrange basis on `nodes`: values V[q][i] = l_i(x_q), derivatives D[q][i] = l_i'(x_q).
void lagrange(const std::vector<double>& nodes, const std::vector<double>& x, std::vector<double>& V,
              std::vector<double>& D) {
  const int n = (int)nodes.size(), m = (int)x.size();
  V.assign((size_t)m * n, 0.0);
  D.assign((size_t)m * n, 0.0);
  for (int q = 0; q < m; ++q)
    for (int i = 0; i < n; ++i) {
      double v = 1.0;
      for (int j = 0; j < n; ++j)
        if (j != i) v *= (x[q] - nodes[j]) / (nodes[i] - nodes[j]);
      double d = 0.0;
      for (int l = 0; l < n; ++l) {
        if (l == i) continue;
        double t = 1.0 / (nodes[i] - nodes[l]);
        for (int j = 0; j < n; ++j)
          if (j != i && j != l) t *= (x[q] - nodes[j]) / (nodes[i] - nodes[j]);
        d += t;
      }
      V[(size_t)q * n + i] = v;
      D[(size_t)q * n + i] = d;
    }
}

// In-place inverse of an n x n matrix by Gauss--Jordan elimination with partial pivoting.
bool invert(std::vector<double>& A, int n) {
  std::vector<double> I((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) I[(size_t)i * n + i] = 1.0;
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(A[(size_t)r * n + c]) > std::fabs(A[(size_t)piv * n + c])) piv = r;
    if (std::fabs(A[(size_t)piv * n + c]) < 1e-300) return false;
    if (piv != c)
      for (int j = 0; j < n; ++j) {
        std::swap(A[(size_t)c * n + j], A[(size_t)piv * n + j]);
        std::swap(I[(size_t)c * n + j], I[(size_t)piv * n + j]);
      }
    const double inv = 1.0 / A[(size_t)c * n + c];
    for (int j = 0; j < n; ++j) {
      A[(size_t)c * n + j] *= inv;
      I[(size_t)c * n + j] *= inv;
    }
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      const double f = A[(size_t)r * n + c];
      if (f == 0.0) continue;
      for (int j = 0; j < n; ++j) {
        A[(size_t)r * n + j] -= f * A[(size_t)c * n + j];
        I[(size_t)r * n + j] -= f * I[(size_t)c * n + j];
      }
    }
  }
  A = I;
  return true;
}

// Make a point set exactly symmetric about 1/2 (x[n-1-i] = 1 - x[i]) so that the
// even-odd form of every 1D operator is exact.
void symmetrize(std::vector<double>& x, std::vector<double>* w = nullptr) {
  const int n = (int)x.size();
  for (int i = 0; i < n / 2; ++i) {
    const double a = 0.5 * (x[i] + (1.0 - x[n - 1 - i]));
    x[i] = a;
    x[n - 1 - i] = 1.0 - a;
    if (w) {
      const double b = 0.5 * ((*w)[i] + (*w)[n - 1 - i]);
      (*w)[i] = b;
      (*w)[n - 1 - i] = b;
    }
  }
  if (n & 1) x[n / 2] = 0.5;
}

// Even-odd form of the operator O (dout x din, row-major) at t + off.
void put_eo(std::vector<double>& t, int off, const std::vector<double>& O, int dout, int din) {
  const int oh = (dout + 1) / 2, ih = din / 2;
  for (int q = 0; q < oh; ++q) {
    for (int i = 0; i < ih; ++i) {
      const double lo = O[(size_t)q * din + i], hi = O[(size_t)q * din + din - 1 - i];
      t[off + q * ih + i] = 0.5 * (lo + hi);
      t[off + oh * ih + q * ih + i] = 0.5 * (lo - hi);
    }
    t[off + 2 * oh * ih + q] = (din & 1) ? O[(size_t)q * din + ih] : 0.0;
  }
}

std::vector<double> transpose(const std::vector<double>& O, int rows, int cols) {
  std::vector<double> T((size_t)rows * cols);
  for (int r = 0; r < rows; ++r)
    for (int c = 0; c < cols; ++c) T[(size_t)c * rows + r] = O[(size_t)r * cols + c];
  return T;
}

std::vector<double> build_tables(int k, int QC, int QV) {
  const int N = k + 1;
  const TableLayout L = make_layout(N, QC, QV);
  std::vector<double> t(L.total, 0.0);
  std::vector<double> nodes = lgl(k);
  symmetrize(nodes);
  std::vector<double> xc, wc, xv, wv, xm, wm, V, D, Vg, Dg;
  gauss(QC, xc, wc);
  gauss(QV, xv, wv);
  gauss(N, xm, wm);
  symmetrize(xc, &wc);
  symmetrize(xv, &wv);
  symmetrize(xm, &wm);
  lagrange(nodes, xc, V, D);  // S_c[q][i] = l_i(x_q)
  put_eo(t, L.eo[EO_SC], V, QC, N);
  put_eo(t, L.eo[EO_SCT], transpose(V, QC, N), N, QC);
  lagrange(xc, xc, Vg, Dg);  // collocation derivative on the convective Gauss points
  put_eo(t, L.eo[EO_DC], Dg, QC, QC);
  put_eo(t, L.eo[EO_DCT], transpose(Dg, QC, QC), QC, QC);
  lagrange(nodes, xv, V, D);
  put_eo(t, L.eo[EO_SV], V, QV, N);
  put_eo(t, L.eo[EO_SVT], transpose(V, QV, N), N, QV);
  lagrange(xv, xv, Vg, Dg);
  put_eo(t, L.eo[EO_DV], Dg, QV, QV);
  put_eo(t, L.eo[EO_DVT], transpose(Dg, QV, QV), QV, QV);
  lagrange(xm, xm, Vg, Dg);  // collocation derivative on the mass points (geometry)
  put_eo(t, L.eo[EO_DM], Dg, N, N);
  lagrange(nodes, xm, V, D);  // square LGL-to-Gauss matrix at the k+1 mass points
  put_eo(t, L.eo[EO_SM], V, N, N);
  if (!invert(V, N)) return {};
  put_eo(t, L.eo[EO_SMI], V, N, N);
  put_eo(t, L.eo[EO_SMIT], transpose(V, N, N), N, N);
  std::copy(wc.begin(), wc.end(), t.begin() + L.wc);
  std::copy(wv.begin(), wv.end(), t.begin() + L.wv);
  std::copy(wm.begin(), wm.end(), t.begin() + L.wm);
  lagrange(nodes, std::vector<double>{0.0, 1.0}, V, D);
  for (int i = 0; i < N; ++i) {
    t[L.dl0 + i] = D[i];
    t[L.dl1 + i] = D[N + i];
  }
  return t;
}

struct Registry {
  int N, QC, QV;
  void (*part[DGCNS_PARTS])(Launchers&);
};

#define DGCNS_ENTRY(N, QC, QV)                                                                           \
  {N, QC, QV,                                                                                            \
   {&launchers_##N##_##QC##_##QV##_0, &launchers_##N##_##QC##_##QV##_1, &launchers_##N##_##QC##_##QV##_2, \
    &launchers_##N##_##QC##_##QV##_3, &launchers_##N##_##QC##_##QV##_4, &launchers_##N##_##QC##_##QV##_5, \
    &launchers_##N##_##QC##_##QV##_6}},
const Registry kRegistry[] = {DGCNS_CONFIGS(DGCNS_ENTRY)};
#undef DGCNS_ENTRY

}  // namespace

// ---------------------------------------------------------------------------
// Context
// ---------------------------------------------------------------------------
struct dgcns_ctx {
  dgcns_mesh mesh;
  dgcns_params prm;
  int device = 0;  // the CUDA device current at dg_cns_create: every call runs there
  cudaStream_t stream = nullptr;
  Launchers L{};
  KParams kp{};
  int Nc = 0, N = 0, N3 = 0;
  size_t state_elems = 0;
  double mu = 0, lam = 0, cv = 0, nu = 0, Tw = 0;
  double* d_tab64 = nullptr;
  float* d_tab32 = nullptr;
  double* d_tau = nullptr;
  void* d_R = nullptr;        // residual scratch (split kernels)
  float* d_dev = nullptr;     // FP32 deviation state U - U_ref (mixed form)
  float* d_dev2 = nullptr;    // second deviation buffer: the one a stage writes inside dg_cns_rk_steps
  void* d_fb = nullptr;       // face shares [Nc][6][2][5][N^2] (face-centric organisation)
  double* g64[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};  // stored geometry, FP64 (gcc gcv gfc gfv gm)
  void* d_xyz = nullptr;  // node coordinates in the residual precision (geometry on the fly)
  float* g32[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};   // FP32 copies for the mixed form
  size_t gsize[5] = {0, 0, 0, 0, 0};
  double* d_partial = nullptr;
  int* d_err = nullptr;  // error word of the kernels with bounded waits
  int* d_fnbr = nullptr;  // rotated-frame meshes: neighbour and orientation per local face
  int* d_flist = nullptr;  // rotated-frame meshes, face-centric kernels: faces by owner's local face
  void* d_gws = nullptr;   // high degrees: global workspace of the operator kernels
  int diag_blocks = 0;
  int64_t launches = 0;
  // per-kernel timing (dg_cns_timing): event pairs awaiting readout, a pool of free events, totals
  struct TimedLaunch {
    int kind;
    cudaEvent_t a, b;
  };
  bool timing = false;
  std::vector<TimedLaunch> pending;
  std::vector<cudaEvent_t> pool;
  double kt_ms[DGCNS_KT_COUNT] = {};
  int64_t kt_n[DGCNS_KT_COUNT] = {};
  double volume = 0.0;  // domain volume (Gauss sum at the convective points)
  std::string err;
};

static thread_local std::string g_create_err = "no error";

// Every entry point runs on its context's device: it makes that device current for the call and
// gives the caller's current device back on return.
struct DeviceScope {
  int prev = -1;
  explicit DeviceScope(const dgcns_ctx* c) {
    int cur = 0;
    if (cudaGetDevice(&cur) == cudaSuccess && cur != c->device && cudaSetDevice(c->device) == cudaSuccess) prev = cur;
  }
  ~DeviceScope() {
    if (prev >= 0) cudaSetDevice(prev);
  }
  DeviceScope(const DeviceScope&) = delete;
  DeviceScope& operator=(const DeviceScope&) = delete;
};

static int fail(dgcns_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

static int cuda_fail(dgcns_ctx* c, const char* what) {
  const cudaError_t e = cudaGetLastError();
  return fail(c, DGCNS_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// A CUDA call of dg_cns_create failed: OOM when the device ran out of memory, else the CUDA error
// (no device, driver mismatch, ...).  Releases the partly built context.
static int create_fail(dgcns_ctx* c, const char* what) {
  const cudaError_t e = cudaGetLastError();
  const bool oom = e == cudaErrorMemoryAllocation;
  g_create_err = std::string(oom ? "out of device memory (" : "CUDA error (") + what + ")" +
                 (oom ? std::string() : std::string(": ") + cudaGetErrorString(e));
  dg_cns_destroy(c);
  return oom ? DGCNS_ERR_OOM : DGCNS_ERR_CUDA;
}

static size_t res_bytes(const dgcns_ctx* c) {
  return c->state_elems * (c->prm.precision == DGCNS_MIXED ? sizeof(float) : sizeof(double));
}

// Arrays given to one call must not share memory (views at an offset included): [a, a + na) and
// [b, b + nb) in bytes.
static bool overlap(const void* a, size_t na, const void* b, size_t nb) {
  const uintptr_t x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
  return x < y + nb && y < x + na;
}

static size_t state_bytes(const dgcns_ctx* c) { return c->state_elems * sizeof(double); }

// Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw, SC'11): 10 rounds, each
// multiplying words 0 and 2 by the round multipliers, mixing the high halves with words 1 and 3 and
// the key, permuting; the key advances by the Weyl increments between rounds.
__host__ __device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
  for (int r = 0; r < 10; ++r) {
    const uint64_t p0 = (uint64_t)0xD2511F53u * c[0], p1 = (uint64_t)0xCD9E8D57u * c[2];
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
}

// Uniform in [0, 1) for element i: block i / 2 (counter (i / 2, 0, 0, 0), key = seed), words (0, 1) for
// even i, (2, 3) for odd i, 53 bits as (a >> 5) 2^26 + (b >> 6).
__host__ __device__ __forceinline__ double philox_u01(uint64_t i, uint64_t seed) {
  const uint64_t j = i >> 1;
  uint32_t c[4] = {(uint32_t)j, (uint32_t)(j >> 32), 0u, 0u};
  philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
  const uint32_t a = (i & 1) ? c[2] : c[0], b = (i & 1) ? c[3] : c[1];
  const uint64_t k = ((uint64_t)(a >> 5) << 26) | (uint64_t)(b >> 6);
  return (double)k * 0x1.0p-53;
}


// Frames of DGCNS_MAP_ROTATED: g in [0, 48), permutation kFramePerm[g / 8], reflection bits g % 8; a local
// reference point xi lies at eta_a = xi_{P[a]} (bit a clear) or 1 - xi_{P[a]} (set) of the cell's box.
static const int kFramePerm[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};

static std::vector<int> cell_frames(const dgcns_mesh& m) {
  const long long Nc = (long long)m.n[0] * m.n[1] * m.n[2];
  std::vector<int> g((size_t)Nc, 0);
  if (m.mapping != DGCNS_MAP_ROTATED) return g;
  const uint64_t seed = (uint64_t)m.map_param;
  for (long long e = 0; e < Nc; ++e) {
    const int v = (int)(philox_u01((uint64_t)e, seed) * 48.0);
    g[(size_t)e] = v > 47 ? 47 : v;
  }
  return g;
}

// Local axis of frame g that lies along box axis a, and whether it is reflected.
static int frame_axis(int g, int a) { return kFramePerm[g / 8][a]; }
static bool frame_flip(int g, int a) { return ((g % 8) >> a) & 1; }

// Per cell e and local face f = 2 d + s: the neighbour cell across it and the orientation code of that
// neighbour relative to e's frame, [Nc][6][2].  The code maps the node index (i0, i1, i2) of the
// neighbour seen in e's frame to its own node index: j_b = i_{src_b}, or N - 1 - i_{src_b} when bit 6 + b
// is set, with src_b in bits 2b..2b+1 (the composition of e's frame with the inverse of n's).  Periodic
// boxes only.
static std::vector<int> frame_face_table(const dgcns_mesh& m, const std::vector<int>& frames) {
  const int nx = m.n[0], ny = m.n[1], nz = m.n[2];
  const long long Nc = (long long)nx * ny * nz;
  std::vector<int> t((size_t)Nc * 12);
  for (long long e = 0; e < Nc; ++e) {
    const int cc[3] = {(int)(e % nx), (int)((e / nx) % ny), (int)(e / ((long long)nx * ny))};
    const int ge = frames[(size_t)e];
    for (int d = 0; d < 3; ++d)
      for (int s = 0; s < 2; ++s) {
        int A = 0;
        while (frame_axis(ge, A) != d) ++A;
        const int S = frame_flip(ge, A) ? 1 - s : s;  // the face's side along box axis A
        int c2[3] = {cc[0], cc[1], cc[2]};
        c2[A] = (c2[A] + (S ? 1 : -1) + m.n[A]) % m.n[A];
        const long long n = c2[0] + (long long)nx * (c2[1] + (long long)ny * c2[2]);
        const int gn = frames[(size_t)n];
        int code = 0;
        for (int a = 0; a < 3; ++a) {
          const int b = frame_axis(gn, a), src = frame_axis(ge, a);
          code |= src << (2 * b);
          if (frame_flip(ge, a) != frame_flip(gn, a)) code |= 1 << (6 + b);
        }
        t[((size_t)e * 6 + 2 * d + s) * 2] = (int)n;
        t[((size_t)e * 6 + 2 * d + s) * 2 + 1] = code;
      }
  }
  return t;
}

// Face lists of the face-centric kernels on rotated-frame meshes: every face once, owned by the cell whose
// local upper face it is (the lower-indexed cell when it is an upper or a lower face of both), grouped by the
// owner's local face f = 2 d + s, each group in owner order; off[f] and len[f] locate group f.  (Ordering the
// groups by the box axis of the face, or interleaving the six groups block by block, did not reduce the
// DRAM re-reads of the mixed form's face kernel, and the interleaving slowed the FP64 one: measured.)
static std::vector<int> frame_face_lists(long long Nc, const std::vector<int>& t, int off[6], int len[6]) {
  std::vector<std::vector<int>> groups(6);
  for (long long e = 0; e < Nc; ++e)
    for (int f = 0; f < 6; ++f) {
      const int s = f & 1, n = t[((size_t)e * 6 + f) * 2], code = t[((size_t)e * 6 + f) * 2 + 1];
      int dn, refl, sn;
      frame_facing(code, f >> 1, s, dn, refl, sn);
      if (s == 1 ? (sn == 0 || e < n) : (sn == 0 && e < n)) groups[f].push_back((int)e);
    }
  std::vector<int> out;
  for (int f = 0; f < 6; ++f) {
    off[f] = (int)out.size();
    len[f] = (int)groups[f].size();
    out.insert(out.end(), groups[f].begin(), groups[f].end());
  }
  return out;
}

static void map_point(const dgcns_mesh& m, double* x) {
  const double L[3] = {m.hi[0] - m.lo[0], m.hi[1] - m.lo[1], m.hi[2] - m.lo[2]};
  if (m.mapping == DGCNS_MAP_CHANNEL) {
    const double C = m.map_param;
    const double eta = (x[1] - m.lo[1]) / L[1];
    x[1] = 0.5 * (m.lo[1] + m.hi[1]) + 0.5 * L[1] * std::tanh(C * (2.0 * eta - 1.0)) / std::tanh(C);
  } else if (m.mapping == DGCNS_MAP_SINE || (m.mapping == DGCNS_MAP_ROTATED && m.deform != 0.0)) {
    const double A = m.mapping == DGCNS_MAP_SINE ? m.map_param : m.deform;
    double X[3], disp[3];
    for (int b = 0; b < 3; ++b) X[b] = (x[b] - m.lo[b]) / L[b];
    for (int a = 0; a < 3; ++a) {
      double s = 1.0;
      for (int b = 0; b < 3; ++b) s *= std::sin(2.0 * M_PI * X[b] + 0.5 * a * (b + 1));
      disp[a] = A * L[a] * s;
    }
    for (int a = 0; a < 3; ++a) x[a] += disp[a];
  }
}

namespace {
__global__ void d2f_kernel(const double* __restrict__ in, float* __restrict__ out, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = (float)in[i];
}

// Node coordinates of the degree-k geometry on the host: [Nc][3][n^3].
std::vector<double> host_node_coords(const dgcns_mesh& m, int k) {
  const int N = k + 1, N3 = N * N * N;
  std::vector<double> nodes = lgl(k);
  symmetrize(nodes);
  double h[3];
  for (int d = 0; d < 3; ++d) h[d] = (m.hi[d] - m.lo[d]) / m.n[d];
  const long long Nc = (long long)m.n[0] * m.n[1] * m.n[2];
  std::vector<double> host((size_t)Nc * 3 * N3);
  const std::vector<int> frames = cell_frames(m);
  for (long long e = 0; e < Nc; ++e) {
    const int cc[3] = {(int)(e % m.n[0]), (int)((e / m.n[0]) % m.n[1]), (int)(e / ((long long)m.n[0] * m.n[1]))};
    const int g = frames[(size_t)e];
    for (int i = 0; i < N3; ++i) {
      const int ii[3] = {i % N, (i / N) % N, i / (N * N)};
      double x[3];
      for (int d = 0; d < 3; ++d) {
        // the node's position along box axis d: local axis frame_axis(g, d), reflected or not (the LGL
        // nodes are symmetric: node N-1-i sits at 1 - xi_i)
        const int li = ii[frame_axis(g, d)];
        x[d] = m.lo[d] + (cc[d] + nodes[frame_flip(g, d) ? N - 1 - li : li]) * h[d];
      }
      map_point(m, x);
      for (int d = 0; d < 3; ++d) host[((size_t)e * 3 + d) * N3 + i] = x[d];
    }
  }
  return host;
}
}  // namespace


// ---------------------------------------------------------------------------
// Initial states (dg_cns_set_initial_tgv / dg_cns_set_initial_channel)
// ---------------------------------------------------------------------------
// Channel start (Sec. 4.3.1): rho = rho0, u1 = u_max (1 - y^2) + a p1, u2 = a p2, u3 = a p3 with
// a = 5 % u_max and p in [-1, 1) from Philox (element (cell 3 + component) n^3 + node); rho E =
// rho0 (c_v T0 + |u|^2 / 2).  Every operation explicitly rounded, in a fixed order, so that the result
// does not depend on contraction into FMAs.
__global__ void init_channel_kernel(const double* __restrict__ xyz, double* __restrict__ U, int Nc, int N3,
                                    uint64_t seed, double u_max, double amp_u, double e0, double rho0) {
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < (size_t)Nc * N3;
       idx += (size_t)gridDim.x * blockDim.x) {
    const size_t e = idx / N3, q = idx - e * N3;
    const double y = xyz[(e * 3 + 1) * N3 + q];
    double p[3];
    for (int d = 0; d < 3; ++d) p[d] = __dadd_rn(-1.0, __dmul_rn(2.0, philox_u01((e * 3 + d) * N3 + q, seed)));
    const double u1 = __dadd_rn(__dmul_rn(u_max, __dsub_rn(1.0, __dmul_rn(y, y))), __dmul_rn(amp_u, p[0]));
    const double u2 = __dmul_rn(amp_u, p[1]), u3 = __dmul_rn(amp_u, p[2]);
    const double s2 = __dadd_rn(__dadd_rn(__dmul_rn(u1, u1), __dmul_rn(u2, u2)), __dmul_rn(u3, u3));
    const double E = __dadd_rn(e0, __dmul_rn(0.5, s2));
    double* o = U + e * 5 * N3 + q;
    o[0] = rho0;
    o[N3] = __dmul_rn(rho0, u1);
    o[2 * N3] = __dmul_rn(rho0, u2);
    o[3 * N3] = __dmul_rn(rho0, u3);
    o[4 * N3] = __dmul_rn(rho0, E);
  }
}

// Taylor--Green vortex (Sec. 4.2.1): u = U0 (sin x cos y cos z, -cos x sin y cos z, 0) with x = X / L,
// p = p0 + rho0 U0^2 / 16 (cos 2x + cos 2y)(cos 2z + 2), uniform T0 = (U0 / Ma)^2 / (gamma R),
// rho = p / (R T0), rho E = rho (c_v T0 + |u|^2 / 2).
__global__ void init_tgv_kernel(const double* __restrict__ xyz, double* __restrict__ U, int Nc, int N3, double U0,
                                double Linv, double p0, double q0, double RT0, double e0) {
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < (size_t)Nc * N3;
       idx += (size_t)gridDim.x * blockDim.x) {
    const size_t e = idx / N3, q = idx - e * N3;
    const double x = xyz[(e * 3) * N3 + q] * Linv, y = xyz[(e * 3 + 1) * N3 + q] * Linv,
                 z = xyz[(e * 3 + 2) * N3 + q] * Linv;
    const double u1 = U0 * sin(x) * cos(y) * cos(z), u2 = -U0 * cos(x) * sin(y) * cos(z);
    const double p = p0 + q0 * (cos(2 * x) + cos(2 * y)) * (cos(2 * z) + 2.0);
    const double rho = p / RT0;
    double* o = U + e * 5 * N3 + q;
    o[0] = rho;
    o[N3] = rho * u1;
    o[2 * N3] = rho * u2;
    o[3 * N3] = 0.0;
    o[4 * N3] = rho * (e0 + 0.5 * (u1 * u1 + u2 * u2));
  }
}

extern "C" {

int dg_cns_create(const dgcns_mesh* mesh, const dgcns_params* prm, void* stream, dgcns_ctx** out) {
  if (!out) return DGCNS_ERR_INVALID_ARG;
  *out = nullptr;
  g_create_err = "no error";
  if (!mesh || !prm) {
    g_create_err = "NULL mesh or params";
    return DGCNS_ERR_INVALID_ARG;
  }
  dgcns_ctx* c = new dgcns_ctx();
  c->mesh = *mesh;
  c->prm = *prm;
  c->stream = static_cast<cudaStream_t>(stream);
  auto bad = [&](int code, const std::string& m) {
    g_create_err = m;
    delete c;
    return code;
  };
  const int k = prm->k;
  if (k < 1 || k > 15) return bad(DGCNS_ERR_UNSUPPORTED, "k must be in 1..15");
  if (prm->nq_conv < k + 1 || prm->nq_visc < k + 1)
    return bad(DGCNS_ERR_INVALID_ARG, "nq_conv and nq_visc must be >= k+1 (collocation gradients)");
  for (int d = 0; d < 3; ++d) {
    if (mesh->n[d] < 1 || !(mesh->hi[d] > mesh->lo[d])) return bad(DGCNS_ERR_INVALID_ARG, "bad mesh extents");
  }
  if (!(prm->gamma > 1.0) || !(prm->Pr > 0) || !(prm->Re > 0) || !(prm->Ma > 0) || !(prm->R > 0) ||
      !(prm->rho0 > 0) || !(prm->U0 > 0) || !(prm->L > 0))
    return bad(DGCNS_ERR_INVALID_ARG, "physical parameters must be positive (gamma > 1)");
  if (prm->precision != DGCNS_FP64 && prm->precision != DGCNS_MIXED)
    return bad(DGCNS_ERR_INVALID_ARG, "precision must be DGCNS_FP64 or DGCNS_MIXED");
  if (prm->geometry != DGCNS_GEO_STORED && prm->geometry != DGCNS_GEO_ON_THE_FLY)
    return bad(DGCNS_ERR_INVALID_ARG, "geometry must be DGCNS_GEO_STORED or DGCNS_GEO_ON_THE_FLY");
  if (prm->kernel != DGCNS_KERNEL_SPLIT && prm->kernel != DGCNS_KERNEL_FUSED && prm->kernel != DGCNS_KERNEL_FACES)
    return bad(DGCNS_ERR_INVALID_ARG, "kernel must be DGCNS_KERNEL_SPLIT, DGCNS_KERNEL_FUSED or DGCNS_KERNEL_FACES");
  if (mesh->mapping != DGCNS_MAP_AFFINE && mesh->mapping != DGCNS_MAP_CHANNEL && mesh->mapping != DGCNS_MAP_SINE &&
      mesh->mapping != DGCNS_MAP_ROTATED)
    return bad(DGCNS_ERR_INVALID_ARG, "unknown mapping");
  if (mesh->mapping == DGCNS_MAP_ROTATED) {
    if (!mesh->periodic[0] || !mesh->periodic[1] || !mesh->periodic[2])
      return bad(DGCNS_ERR_INVALID_ARG, "rotated-frame meshes must be periodic on every axis");
    if (!(mesh->map_param >= 0.0 && mesh->map_param < 18446744073709551616.0) ||
        mesh->map_param != std::floor(mesh->map_param))
      return bad(DGCNS_ERR_INVALID_ARG, "the frame seed (map_param) must be a non-negative integer below 2^64");
  }
  if (mesh->mapping == DGCNS_MAP_ROTATED ? !std::isfinite(mesh->deform) : mesh->deform != 0.0)
    return bad(DGCNS_ERR_INVALID_ARG, "deform must be finite, and 0 unless the mapping is DGCNS_MAP_ROTATED");
  if (mesh->mapping == DGCNS_MAP_CHANNEL && !(mesh->map_param > 0.0))
    return bad(DGCNS_ERR_INVALID_ARG, "channel stretch factor must be positive");
  // checked factor by factor, so that the product cannot overflow before the comparison
  long long ncell = 1;
  for (int d = 0; d < 3; ++d) {
    ncell *= mesh->n[d];
    if (ncell > (1LL << 30)) return bad(DGCNS_ERR_INVALID_ARG, "too many cells (more than 2^30)");
  }
  const int N = k + 1;
  bool found = false;
  for (const Registry& r : kRegistry)
    if (r.N == N && r.QC == prm->nq_conv && r.QV == prm->nq_visc) {
      c->L = Launchers{};
      for (int q = 0; q < DGCNS_PARTS; ++q) r.part[q](c->L);
      found = true;
    }
  if (!found) return bad(DGCNS_ERR_UNSUPPORTED, "no instantiation for this (k, nq_conv, nq_visc)");
  if (prm->precision == DGCNS_MIXED && !(c->L.features & FEAT_FP32))
    return bad(DGCNS_ERR_UNSUPPORTED, "the mixed form is not compiled for this (k, nq_conv, nq_visc)");
  if (prm->kernel == DGCNS_KERNEL_FACES && !(c->L.features & FEAT_FACES))
    return bad(DGCNS_ERR_UNSUPPORTED, "the face-centric kernels are not compiled for this (k, nq_conv, nq_visc)");
  if (mesh->mapping != DGCNS_MAP_AFFINE && !(c->L.features & FEAT_GEO))
    return bad(DGCNS_ERR_UNSUPPORTED, "non-affine meshes are not compiled for this (k, nq_conv, nq_visc)");
  if (mesh->mapping != DGCNS_MAP_AFFINE && prm->geometry == DGCNS_GEO_ON_THE_FLY && !(c->L.features & FEAT_FLY))
    return bad(DGCNS_ERR_UNSUPPORTED, "geometry on the fly is not compiled for this (k, nq_conv, nq_visc)");

  c->Nc = (int)ncell;
  c->N = N;
  c->N3 = N * N * N;
  c->state_elems = (size_t)c->Nc * 5 * c->N3;
  // physics (Sec. 4.2.1): mu = rho0 U0 L / Re, lambda = mu c_p / Pr, T0 = c0^2/(gamma R)
  c->cv = prm->R / (prm->gamma - 1.0);
  c->mu = prm->rho0 * prm->U0 * prm->L / prm->Re;
  c->lam = c->mu * prm->gamma * c->cv / prm->Pr;
  c->nu = c->mu / prm->rho0;
  const double umach = prm->u_mach > 0 ? prm->u_mach : prm->U0;
  const double c0 = umach / prm->Ma;
  c->Tw = c0 * c0 / (prm->gamma * prm->R);

  // tables
  std::vector<double> t64 = build_tables(k, prm->nq_conv, prm->nq_visc);
  if (t64.empty()) return bad(DGCNS_ERR_INVALID_ARG, "singular mass interpolation matrix");
  std::vector<float> t32(t64.begin(), t64.end());
  // penalty per cell (Eq. TauIP_Element): nu (k+1)^2 (A_interior/2 + A_boundary)/V; affine box
  double h[3];
  for (int d = 0; d < 3; ++d) h[d] = (mesh->hi[d] - mesh->lo[d]) / mesh->n[d];
  const double vol = h[0] * h[1] * h[2];
  std::vector<double> tau(c->Nc);
  for (int e = 0; e < c->Nc; ++e) {
    const int cc[3] = {e % mesh->n[0], (e / mesh->n[0]) % mesh->n[1], e / (mesh->n[0] * mesh->n[1])};
    double a = 0.0;
    for (int d = 0; d < 3; ++d) {
      const double area = vol / h[d];
      for (int s = 0; s < 2; ++s) {
        const bool boundary = !mesh->periodic[d] && ((s == 0 && cc[d] == 0) || (s == 1 && cc[d] == mesh->n[d] - 1));
        a += boundary ? area : 0.5 * area;
      }
    }
    tau[e] = c->nu * (k + 1) * (k + 1) * a / vol;
  }

  if (cudaGetDevice(&c->device) != cudaSuccess) return create_fail(c, "cudaGetDevice");
  if (prm->precision == DGCNS_FP64 && c->L.gws_fp64 > 0) {
    // high degrees: the operator kernels' per-cell working set in a global workspace of 4 CTA slices per
    // SM (the launcher runs the grid in chunks of that many CTAs)
    int nsm = 0;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess || nsm < 1)
      return create_fail(c, "multiprocessor count");
    const size_t ctas = (size_t)4 * nsm;
    if (cudaMalloc(&c->d_gws, ctas * c->L.gws_fp64) != cudaSuccess) return create_fail(c, "operator workspace");
    c->kp.gws = c->d_gws;
    c->kp.gws_elems = ctas * c->L.gws_fp64 / sizeof(double);
  }
  if (cudaMalloc(&c->d_tab64, t64.size() * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&c->d_tab32, t32.size() * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&c->d_tau, tau.size() * sizeof(double)) != cudaSuccess)
    return create_fail(c, "tables");
  if (cudaMemcpy(c->d_tab64, t64.data(), t64.size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(c->d_tab32, t32.data(), t32.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(c->d_tau, tau.data(), tau.size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess)
    return create_fail(c, "table upload");
  // the 1D operators also go to the constant memory of every part (the same values for every context of
  // this (k, nq_conv, nq_visc), so rewriting them is harmless to contexts already running)
  for (int q = 0; q < DGCNS_PARTS; ++q)
    if (c->L.const_tables[q] && c->L.const_tables[q](t64.data(), t32.data(), c->stream) != 0)
      return create_fail(c, "constant tables");
  const size_t fb_bytes = (size_t)c->Nc * 60 * N * N * (prm->precision == DGCNS_MIXED ? sizeof(float) : sizeof(double));
  if (cudaMalloc(&c->d_R, res_bytes(c)) != cudaSuccess ||
      (prm->precision == DGCNS_MIXED && cudaMalloc(&c->d_dev, c->state_elems * sizeof(float)) != cudaSuccess) ||
      (prm->precision == DGCNS_MIXED && prm->kernel != DGCNS_KERNEL_SPLIT &&
       cudaMalloc(&c->d_dev2, c->state_elems * sizeof(float)) != cudaSuccess) ||
      (prm->kernel == DGCNS_KERNEL_FACES && cudaMalloc(&c->d_fb, fb_bytes) != cudaSuccess))
    return create_fail(c, "residual, deviation and face buffers");
  KParams& kp = c->kp;
  kp.Nc = c->Nc;
  for (int d = 0; d < 3; ++d) {
    kp.nc[d] = mesh->n[d];
    kp.periodic[d] = mesh->periodic[d] ? 1 : 0;
    kp.h[d] = h[d];
    kp.bf[d] = prm->body_force[d];
  }
  kp.has_bf = (prm->body_force[0] != 0.0 || prm->body_force[1] != 0.0 || prm->body_force[2] != 0.0) ? 1 : 0;
  kp.gamma = prm->gamma;
  kp.mu = c->mu;
  kp.lam = c->lam;
  kp.cv = c->cv;
  kp.Tw = c->Tw;
  kp.rho_ref = prm->rho0;
  kp.rhoE_ref = prm->rho0 * c->cv * c->Tw;
  fill_kconst(kp, kp.cd);
  fill_kconst(kp, kp.cf);
  kp.tau = c->d_tau;
  kp.conv = kp.visc = 1;
  c->volume = (mesh->hi[0] - mesh->lo[0]) * (mesh->hi[1] - mesh->lo[1]) * (mesh->hi[2] - mesh->lo[2]);
  kp.tables = prm->precision == DGCNS_MIXED ? (const void*)c->d_tab32 : (const void*)c->d_tab64;
  if (mesh->mapping != DGCNS_MAP_AFFINE) {
    // stored geometry: node coordinates -> Jacobians at every point set (FP64 kernel), tau per cell
    const int QC = prm->nq_conv, QV = prm->nq_visc;
    c->gsize[0] = (size_t)c->Nc * 10 * QC * QC * QC;
    c->gsize[1] = (size_t)c->Nc * 10 * QV * QV * QV;
    c->gsize[2] = (size_t)c->Nc * 6 * 13 * QC * QC;
    c->gsize[3] = (size_t)c->Nc * 6 * 13 * QV * QV;
    c->gsize[4] = (size_t)c->Nc * c->N3;
    for (int i = 0; i < 5; ++i)
      if (cudaMalloc(&c->g64[i], c->gsize[i] * sizeof(double)) != cudaSuccess) return create_fail(c, "geometry");
    std::vector<double> xyz = host_node_coords(*mesh, k);
    double* d_xyz = nullptr;
    if (cudaMalloc(&d_xyz, xyz.size() * sizeof(double)) != cudaSuccess) return create_fail(c, "coordinates");
    if (cudaMemcpy(d_xyz, xyz.data(), xyz.size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess) {
      const int r = create_fail(c, "coordinate upload");
      cudaFree(d_xyz);
      return r;
    }
    KParams kg = kp;
    kg.tables = c->d_tab64;
    double* d_vol = nullptr;
    if (cudaMalloc(&d_vol, (size_t)c->Nc * sizeof(double)) != cudaSuccess) {
      const int r = create_fail(c, "volumes");
      cudaFree(d_xyz);
      return r;
    }
    const int rg = c->L.geom(kg, d_xyz, c->g64[0], c->g64[1], c->g64[2], c->g64[3], c->g64[4], c->d_tau, d_vol,
                             c->nu * (k + 1) * (k + 1), c->stream);
    c->launches += 1;
    const cudaError_t se = cudaStreamSynchronize(c->stream);
    if (prm->geometry == DGCNS_GEO_ON_THE_FLY) {
      if (prm->precision == DGCNS_MIXED) {
        float* x32 = nullptr;
        if (cudaMalloc(&x32, xyz.size() * sizeof(float)) == cudaSuccess) {
          d2f_kernel<<<1024, 256, 0, c->stream>>>(d_xyz, x32, xyz.size());
          c->launches += 1;
          cudaStreamSynchronize(c->stream);
        }
        cudaFree(d_xyz);
        c->d_xyz = x32;
      } else {
        c->d_xyz = d_xyz;
      }
      if (!c->d_xyz) {
        cudaFree(d_vol);
        return create_fail(c, "FP32 coordinates");
      }
    } else {
      cudaFree(d_xyz);
    }
    if (rg == 0 && se == cudaSuccess) {
      std::vector<double> vol(c->Nc);
      cudaMemcpy(vol.data(), d_vol, vol.size() * sizeof(double), cudaMemcpyDeviceToHost);
      double v = 0.0;
      for (double x : vol) v += x;
      c->volume = v;
    }
    cudaFree(d_vol);
    if (rg == -2) {
      dg_cns_destroy(c);
      g_create_err = "stored geometry not available for this (k, nq) (shared memory)";
      return DGCNS_ERR_UNSUPPORTED;
    }
    if (rg != 0 || se != cudaSuccess) return create_fail(c, "geometry kernel");
    if (prm->precision == DGCNS_MIXED) {
      for (int i = 0; i < 5; ++i) {
        if (cudaMalloc(&c->g32[i], c->gsize[i] * sizeof(float)) != cudaSuccess) return create_fail(c, "FP32 geometry");
        d2f_kernel<<<1024, 256, 0, c->stream>>>(c->g64[i], c->g32[i], c->gsize[i]);
        c->launches += 1;
      }
      kp.gcc = c->g32[0];
      kp.gcv = c->g32[1];
      kp.gfc = c->g32[2];
      kp.gfv = c->g32[3];
      kp.gm = c->g32[4];
    } else {
      kp.gcc = c->g64[0];
      kp.gcv = c->g64[1];
      kp.gfc = c->g64[2];
      kp.gfv = c->g64[3];
      kp.gm = c->g64[4];
    }
  }
  kp.xyzT = c->d_xyz;  // the operator kernels recompute the Jacobians when set
  if (mesh->mapping == DGCNS_MAP_ROTATED) {
    const std::vector<int> ft = frame_face_table(*mesh, cell_frames(*mesh));
    if (cudaMalloc(&c->d_fnbr, ft.size() * sizeof(int)) != cudaSuccess) return create_fail(c, "face table");
    if (cudaMemcpy(c->d_fnbr, ft.data(), ft.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess)
      return create_fail(c, "face table upload");
    kp.fnbr = c->d_fnbr;
    if (prm->kernel == DGCNS_KERNEL_FACES) {
      const std::vector<int> fl = frame_face_lists(c->Nc, ft, kp.foff, kp.flen);
      if (cudaMalloc(&c->d_flist, fl.size() * sizeof(int)) != cudaSuccess) return create_fail(c, "face lists");
      if (cudaMemcpy(c->d_flist, fl.data(), fl.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess)
        return create_fail(c, "face list upload");
      kp.flist = c->d_flist;
    }
  }
  // diagnostics partial sums
  KParams kd = kp;
  kd.tables = c->d_tab64;
  if (c->g64[0]) {
    kd.gcc = c->g64[0];
    kd.gcv = c->g64[1];
    kd.gfc = c->g64[2];
    kd.gfv = c->g64[3];
    kd.gm = c->g64[4];
  }
  int nblk = 0;
  c->L.diag_fp64(kd, nullptr, nullptr, nullptr, &nblk, c->stream);
  c->diag_blocks = nblk;
  if (cudaMalloc(&c->d_partial, ((size_t)nblk + 1) * 10 * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&c->d_err, sizeof(int)) != cudaSuccess)
    return create_fail(c, "diagnostics scratch");
  if (cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream) != cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess)
    return create_fail(c, "set-up");
  c->kp.err = c->d_err;
  if (cudaPeekAtLastError() != cudaSuccess) return create_fail(c, "set-up launches");
  *out = c;
  return DGCNS_OK;
}

int dg_cns_destroy(dgcns_ctx* c) {
  if (!c) return DGCNS_ERR_INVALID_ARG;
  DeviceScope ds(c);
  if (c->stream) cudaStreamSynchronize(c->stream);
  cudaFree(c->d_tab64);
  cudaFree(c->d_tab32);
  cudaFree(c->d_tau);
  cudaFree(c->d_R);
  cudaFree(c->d_dev);
  cudaFree(c->d_dev2);
  cudaFree(c->d_fb);
  cudaFree(c->d_xyz);
  for (const auto& t : c->pending) {
    cudaEventDestroy(t.a);
    cudaEventDestroy(t.b);
  }
  for (cudaEvent_t e : c->pool) cudaEventDestroy(e);
  cudaFree(c->d_partial);
  cudaFree(c->d_err);
  cudaFree(c->d_fnbr);
  cudaFree(c->d_flist);
  cudaFree(c->d_gws);
  for (int i = 0; i < 5; ++i) {
    cudaFree(c->g64[i]);
    cudaFree(c->g32[i]);
  }
  delete c;
  return DGCNS_OK;
}

int dg_cns_set_stream(dgcns_ctx* c, void* stream) {
  if (!c) return DGCNS_ERR_INVALID_ARG;
  c->stream = static_cast<cudaStream_t>(stream);
  return DGCNS_OK;
}

int dg_cns_sizes(const dgcns_ctx* c, int64_t* nc, int64_t* nn, int64_t* nd) {
  if (!c) return DGCNS_ERR_INVALID_ARG;
  if (nc) *nc = c->Nc;
  if (nn) *nn = (int64_t)c->Nc * c->N3;
  if (nd) *nd = (int64_t)c->Nc * c->N3 * 5;
  return DGCNS_OK;
}

// Node coordinates in a temporary device buffer (set-up calls only), then one initial-state kernel.
static int with_device_coords(dgcns_ctx* c, const std::function<void(const double*)>& launch) {
  const std::vector<double> host = host_node_coords(c->mesh, c->prm.k);
  double* d = nullptr;
  if (cudaMalloc(&d, host.size() * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return fail(c, DGCNS_ERR_OOM, "out of device memory (node coordinates)");
  }
  int r = DGCNS_OK;
  if (cudaMemcpyAsync(d, host.data(), host.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream) !=
      cudaSuccess) {
    r = cuda_fail(c, "node coordinates copy");
  } else {
    launch(d);
    c->launches += 1;
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(c->stream) != cudaSuccess)
      r = cuda_fail(c, "initial-state kernel");
  }
  cudaFree(d);
  return r;
}

int dg_cns_set_initial_tgv(dgcns_ctx* c, double* U) {
  if (!c) return DGCNS_ERR_INVALID_ARG;
  DeviceScope ds(c);
  if (!U) return fail(c, DGCNS_ERR_INVALID_ARG, "U is NULL");
  const dgcns_params& p = c->prm;
  const double U0 = p.U0, c0 = U0 / p.Ma, T0 = c0 * c0 / (p.gamma * p.R), p0 = p.rho0 * p.R * T0;
  const double q0 = p.rho0 * U0 * U0 / 16.0, cv = p.R / (p.gamma - 1.0);
  return with_device_coords(c, [&](const double* xyz) {
    init_tgv_kernel<<<2 * 152 * 8, 256, 0, c->stream>>>(xyz, U, c->Nc, c->N3, U0, 1.0 / p.L, p0, q0, p.R * T0,
                                                         cv * T0);
  });
}

int dg_cns_set_initial_channel(dgcns_ctx* c, double* U, uint64_t seed) {
  if (!c) return DGCNS_ERR_INVALID_ARG;
  DeviceScope ds(c);
  if (!U) return fail(c, DGCNS_ERR_INVALID_ARG, "U is NULL");
  const dgcns_params& p = c->prm;
  if (!(p.u_mach > 0.0)) return fail(c, DGCNS_ERR_INVALID_ARG, "the channel start needs u_mach (u_max) > 0");
  const double u_max = p.u_mach, cs = u_max / p.Ma, T0 = cs * cs / (p.gamma * p.R), cv = p.R / (p.gamma - 1.0);
  const double amp_u = 0.05 * u_max, e0 = cv * T0;
  return with_device_coords(c, [&](const double* xyz) {
    init_channel_kernel<<<2 * 152 * 8, 256, 0, c->stream>>>(xyz, U, c->Nc, c->N3, seed, u_max, amp_u, e0, p.rho0);
  });
}

int dg_cns_node_coords(dgcns_ctx* c, double* xyz) {
  if (!c) return DGCNS_ERR_INVALID_ARG;
  DeviceScope ds(c);
  if (!xyz) return fail(c, DGCNS_ERR_INVALID_ARG, "xyz is NULL");
  const std::vector<double> host = host_node_coords(c->mesh, c->prm.k);
  if (cudaMemcpyAsync(xyz, host.data(), host.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream) !=
          cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess)
    return cuda_fail(c, "node coordinates copy");
  return DGCNS_OK;
}

// Per-kernel timing: an event before and after each launch on the context's stream (RAII scope).
static cudaEvent_t take_event(dgcns_ctx* c) {
  if (!c->pool.empty()) {
    cudaEvent_t e = c->pool.back();
    c->pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

struct TimedScope {
  dgcns_ctx* c;
  int kind;
  cudaEvent_t a = nullptr;
  TimedScope(dgcns_ctx* c_, int k) : c(c_), kind(k) {
    if (c->timing && (a = take_event(c)) != nullptr) cudaEventRecord(a, c->stream);
  }
  ~TimedScope() {
    if (!a) return;
    cudaEvent_t b = take_event(c);
    if (!b) {
      c->pool.push_back(a);
      return;
    }
    cudaEventRecord(b, c->stream);
    c->pending.push_back({kind, a, b});
  }
};

static int flush_times(dgcns_ctx* c) {
  if (c->pending.empty()) return DGCNS_OK;
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return cuda_fail(c, "timing synchronize");
  for (const auto& t : c->pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, t.a, t.b) == cudaSuccess) {
      c->kt_ms[t.kind] += ms;
      c->kt_n[t.kind] += 1;
    }
    c->pool.push_back(t.a);
    c->pool.push_back(t.b);
  }
  c->pending.clear();
  return DGCNS_OK;
}

static int op_kind(int mode) {
  switch (mode) {
    case OP_CELL: return DGCNS_KT_CELL;
    case OP_FACE: return DGCNS_KT_FACE;
    case OP_MASS: return DGCNS_KT_MASS;
    case OP_CELL | OP_MASS: return DGCNS_KT_CELL_STAGE;
    default: return DGCNS_KT_FUSED;
  }
}

static int run_op(dgcns_ctx* c, int mode, KParams kp, const double* U, const void* Rin, void* Rout, void* dU,
                  double* Uout) {
  const OpFn f = c->prm.precision == DGCNS_MIXED ? c->L.op_fp32 : c->L.op_fp64;
  TimedScope ts(c, op_kind(mode));
  const int r = f(mode, kp, U, Rin, Rout, dU, Uout, c->stream);  // >= 0: launches made (0 stands for 1)
  if (r == -2) return fail(c, DGCNS_ERR_UNSUPPORTED, "operator variant not compiled or too large for shared memory");
  if (r < 0) return cuda_fail(c, "operator kernel launch");
  c->launches += r > 0 ? r : 1;
  return DGCNS_OK;
}

// Face-centric organisation: every face once, the shares of both cells into d_fb; the cell kernel that
// follows adds them (kp.fbuf).
static int run_faces(dgcns_ctx* c, KParams& kp, const double* U) {
  const FaceFn f = c->prm.precision == DGCNS_MIXED ? c->L.faces_fp32 : c->L.faces_fp64;
  TimedScope ts(c, DGCNS_KT_FACES);
  const int r = f(kp, U, c->d_fb, c->stream);
  c->launches += 1;
  if (r == -2) return fail(c, DGCNS_ERR_UNSUPPORTED, "face kernel not compiled or too large for shared memory");
  if (r != 0) return cuda_fail(c, "face kernel launch");
  kp.fbuf = c->d_fb;
  return DGCNS_OK;
}

// L(U) into dst (mode 1) or a stage update (mode 2) with the configured kernel organisation.
// The mixed form reads own and neighbour states as FP32 deviations U - U_ref: convert U once per
// operator evaluation (an elementwise pass) so that the operator kernels do no FP64 conversions.
static int prep_dev(dgcns_ctx* c, KParams& kp, const double* U) {
  if (!c->d_dev || !U) return DGCNS_OK;
  TimedScope ts(c, DGCNS_KT_DEV);
  if (c->L.dev_fp32(kp, U, c->d_dev, c->stream) != 0) return cuda_fail(c, "deviation pre-pass");
  c->launches += 1;
  kp.Udev = c->d_dev;
  return DGCNS_OK;
}

// kp.Udev already set (multi-step calls of the mixed form): the deviation state is current.
static int eval_L(dgcns_ctx* c, KParams kp, const double* U, void* dst, void* dU, double* Uout) {
  if (kp.Udev == nullptr) {
    const int rd = prep_dev(c, kp, U);
    if (rd) return rd;
  }
  if (c->prm.kernel == DGCNS_KERNEL_FUSED) return run_op(c, OP_CELL | OP_FACE | OP_MASS, kp, U, nullptr, dst, dU, Uout);
  if (c->prm.kernel == DGCNS_KERNEL_FACES) {
    const int rf = run_faces(c, kp, U);
    if (rf) return rf;
    return run_op(c, OP_CELL | OP_MASS, kp, U, nullptr, dst, dU, Uout);
  }
  KParams k0 = kp;
  k0.out_mode = 0;
  int r = run_op(c, OP_CELL, k0, U, nullptr, c->d_R, nullptr, nullptr);
  if (r) return r;
  r = run_op(c, OP_FACE, k0, U, c->d_R, c->d_R, nullptr, nullptr);
  if (r) return r;
  return run_op(c, OP_MASS, kp, U, c->d_R, dst, dU, Uout);
}

int dg_cns_apply(dgcns_ctx* c, const double* U, void* R, int op) {
  if (!c) return DGCNS_ERR_INVALID_ARG;
  DeviceScope ds(c);
  if (!U || !R) return fail(c, DGCNS_ERR_INVALID_ARG, "NULL array");
  if (overlap(U, state_bytes(c), R, res_bytes(c))) return fail(c, DGCNS_ERR_INVALID_ARG, "R must not overlap U");
  KParams kp = c->kp;
  switch (op) {
    case DGCNS_OP_L:
      kp.out_mode = 1;
      return eval_L(c, kp, U, R, nullptr, nullptr);
    case DGCNS_OP_F:
    case DGCNS_OP_FC:
    case DGCNS_OP_FV: {
      kp.out_mode = 0;
      kp.conv = op != DGCNS_OP_FV;
      kp.visc = op != DGCNS_OP_FC;
      const int rd = prep_dev(c, kp, U);
      if (rd) return rd;
      if (c->prm.kernel == DGCNS_KERNEL_FUSED) return run_op(c, OP_CELL | OP_FACE, kp, U, nullptr, R, nullptr, nullptr);
      if (c->prm.kernel == DGCNS_KERNEL_FACES) {
        const int rf = run_faces(c, kp, U);
        if (rf) return rf;
        return run_op(c, OP_CELL, kp, U, nullptr, R, nullptr, nullptr);
      }
      int r = run_op(c, OP_CELL, kp, U, nullptr, R, nullptr, nullptr);
      if (r) return r;
      return run_op(c, OP_FACE, kp, U, R, R, nullptr, nullptr);
    }
    default:
      return fail(c, DGCNS_ERR_INVALID_ARG, "unknown op");
  }
}

int dg_cns_inverse_mass(dgcns_ctx* c, const void* in, void* out) {
  if (!c) return DGCNS_ERR_INVALID_ARG;
  DeviceScope ds(c);
  if (!in || !out) return fail(c, DGCNS_ERR_INVALID_ARG, "NULL array");
  KParams kp = c->kp;
  kp.out_mode = 0;
  kp.has_bf = 0;
  return run_op(c, OP_MASS, kp, nullptr, in, out, nullptr, nullptr);
}

// One 2N stage with coefficients (A, B): argument checks, then dU <- A dU + dt L(U_in), U_out <- U_in + B dU.
static int stage_2n(dgcns_ctx* c, double A, double B, double dt, const double* U_in, void* dU, double* U_out) {
  if (!U_in || !dU || !U_out) return fail(c, DGCNS_ERR_INVALID_ARG, "NULL array");
  if (overlap(dU, res_bytes(c), U_in, state_bytes(c)) || overlap(dU, res_bytes(c), U_out, state_bytes(c)))
    return fail(c, DGCNS_ERR_INVALID_ARG, "dU must not overlap U_in or U_out");
  if (U_in != U_out && overlap(U_in, state_bytes(c), U_out, state_bytes(c)))
    return fail(c, DGCNS_ERR_INVALID_ARG, "U_out must be U_in itself or not overlap it");
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(c, DGCNS_ERR_INVALID_ARG, "dt must be positive and finite");
  if (!std::isfinite(A) || !std::isfinite(B)) return fail(c, DGCNS_ERR_INVALID_ARG, "A and B must be finite");
  if (c->prm.kernel == DGCNS_KERNEL_FUSED && U_in == U_out)
    return fail(c, DGCNS_ERR_INVALID_ARG, "fused kernel needs U_out != U_in");
  KParams kp = c->kp;
  kp.out_mode = 2;
  kp.A = A;
  kp.B = B;
  kp.dt = dt;
  return eval_L(c, kp, U_in, nullptr, dU, U_out);
}

int dg_cns_rk_stage(dgcns_ctx* c, int stage, double dt, double t, const double* U_in, void* dU, double* U_out) {
  if (!c) return DGCNS_ERR_INVALID_ARG;
  DeviceScope ds(c);
  (void)t;  // the operator is autonomous (constant body force)
  if (stage < 0 || stage > 4) return fail(c, DGCNS_ERR_INVALID_ARG, "stage must be 0..4");
  return stage_2n(c, RK_A[stage], RK_B[stage], dt, U_in, dU, U_out);
}

int dg_cns_lsrk_stage(dgcns_ctx* c, double A, double B, double dt, const double* U_in, void* dU, double* U_out) {
  if (!c) return DGCNS_ERR_INVALID_ARG;
  DeviceScope ds(c);
  return stage_2n(c, A, B, dt, U_in, dU, U_out);
}

// nsteps steps of the 2N scheme (A, B) with `stages` stages; U holds the result.
static int steps_2n(dgcns_ctx* c, int stages, const double* A, const double* B, int nsteps, double dt, double* U,
                    double* U_tmp, void* dU) {
  if (nsteps < 0) return fail(c, DGCNS_ERR_INVALID_ARG, "nsteps < 0");
  if (!U || !U_tmp || !dU || overlap(U, state_bytes(c), U_tmp, state_bytes(c)) ||
      overlap(dU, res_bytes(c), U, state_bytes(c)) || overlap(dU, res_bytes(c), U_tmp, state_bytes(c)))
    return fail(c, DGCNS_ERR_INVALID_ARG, "U, U_tmp and dU must be non-NULL arrays that do not overlap");
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(c, DGCNS_ERR_INVALID_ARG, "dt must be positive and finite");
  for (int s = 0; s < stages; ++s)
    if (!std::isfinite(A[s]) || !std::isfinite(B[s])) return fail(c, DGCNS_ERR_INVALID_ARG, "A and B must be finite");
  double* a = U;
  double* b = U_tmp;
  // Mixed form (fused or face-centric kernels): the stage kernel also writes float(U_out - U_ref)
  // into the second deviation buffer, so only the first stage of the call needs the pre-pass.
  const bool chain = c->d_dev2 != nullptr && nsteps > 0;
  float* dcur = c->d_dev;
  float* dnxt = c->d_dev2;
  if (chain) {
    KParams kp0 = c->kp;
    const int rd = prep_dev(c, kp0, U);
    if (rd) return rd;
  }
  for (int n = 0; n < nsteps; ++n)
    for (int s = 0; s < stages; ++s) {
      int r;
      if (chain) {
        KParams kp = c->kp;
        kp.out_mode = 2;
        kp.A = A[s];
        kp.B = B[s];
        kp.dt = dt;
        kp.Udev = dcur;
        kp.devOut = dnxt;
        r = eval_L(c, kp, a, nullptr, dU, b);
        std::swap(dcur, dnxt);
      } else {
        r = stage_2n(c, A[s], B[s], dt, a, dU, b);
      }
      if (r) return r;
      std::swap(a, b);
    }
  if (a != U) {
    if (cudaMemcpyAsync(U, a, c->state_elems * sizeof(double), cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess)
      return cuda_fail(c, "state copy");
  }
  return DGCNS_OK;
}

int dg_cns_rk_steps(dgcns_ctx* c, int nsteps, double dt, double t0, double* U, double* U_tmp, void* dU) {
  if (!c) return DGCNS_ERR_INVALID_ARG;
  DeviceScope ds(c);
  (void)t0;  // the operator is autonomous (constant body force)
  return steps_2n(c, 5, RK_A, RK_B, nsteps, dt, U, U_tmp, dU);
}

int dg_cns_lsrk_steps(dgcns_ctx* c, int stages, const double* A, const double* B, int nsteps, double dt, double* U,
                      double* U_tmp, void* dU) {
  if (!c) return DGCNS_ERR_INVALID_ARG;
  DeviceScope ds(c);
  if (stages < 1 || stages > DGCNS_MAX_STAGES || !A || !B)
    return fail(c, DGCNS_ERR_INVALID_ARG, "stages must be 1..DGCNS_MAX_STAGES with host arrays A and B");
  return steps_2n(c, stages, A, B, nsteps, dt, U, U_tmp, dU);
}

// Adjoint VJP kernel(s) for Y in d_R: the face-centric organisation first writes the face shares.
static int run_adj(dgcns_ctx* c, KParams ka, const double* U, void* G, double* lam_U) {
  if (c->prm.kernel == DGCNS_KERNEL_FACES) {
    const AdjFaceFn ff = c->prm.precision == DGCNS_MIXED ? c->L.adj_faces_fp32 : c->L.adj_faces_fp64;
    TimedScope ts(c, DGCNS_KT_ADJ_FACES);
    const int rf = ff(ka, U, c->d_R, c->d_fb, c->stream);
    c->launches += 1;
    if (rf == -2) return fail(c, DGCNS_ERR_UNSUPPORTED, "adjoint face kernel not compiled for this (k, nq)");
    if (rf) return cuda_fail(c, "adjoint face kernel launch");
    ka.fbuf = c->d_fb;
  }
  const AdjFn f = c->prm.precision == DGCNS_MIXED ? c->L.adj_fp32 : c->L.adj_fp64;
  TimedScope ts(c, DGCNS_KT_ADJ);
  const int ra = f(ka, U, c->d_R, G, lam_U, c->stream);
  c->launches += 1;
  if (ra == -2) return fail(c, DGCNS_ERR_UNSUPPORTED, "adjoint kernel does not fit shared memory for this (k, nq)");
  if (ra) return cuda_fail(c, "adjoint kernel launch");
  return DGCNS_OK;
}

int dg_cns_adjoint_apply(dgcns_ctx* c, const double* U, const void* W, void* G) {
  if (!c) return DGCNS_ERR_INVALID_ARG;
  DeviceScope ds(c);
  if (!U || !W || !G) return fail(c, DGCNS_ERR_INVALID_ARG, "NULL array");
  if (c->kp.fnbr) return fail(c, DGCNS_ERR_UNSUPPORTED, "adjoint on rotated-frame meshes is not implemented");
  if (c->kp.has_bf) return fail(c, DGCNS_ERR_UNSUPPORTED, "adjoint with a body force is not implemented");
  if (!(c->L.features & FEAT_ADJ)) return fail(c, DGCNS_ERR_UNSUPPORTED, "adjoint not compiled for this (k, nq)");
  if (overlap(G, res_bytes(c), U, state_bytes(c))) return fail(c, DGCNS_ERR_INVALID_ARG, "G must not overlap U");
  KParams km = c->kp;
  km.out_mode = 0;
  km.has_bf = 0;
  int r = run_op(c, OP_MASS, km, nullptr, W, c->d_R, nullptr, nullptr);  // Y = M^-1 W
  if (r) return r;
  KParams ka = c->kp;
  ka.out_mode = 0;
  return run_adj(c, ka, U, G, nullptr);
}

int dg_cns_rk_stage_adjoint(dgcns_ctx* c, int stage, double dt, const double* U_in, double* lam_U, void* lam_dU) {
  if (!c) return DGCNS_ERR_INVALID_ARG;
  DeviceScope ds(c);
  if (stage < 0 || stage > 4) return fail(c, DGCNS_ERR_INVALID_ARG, "stage must be 0..4");
  if (!U_in || !lam_U || !lam_dU) return fail(c, DGCNS_ERR_INVALID_ARG, "NULL array");
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(c, DGCNS_ERR_INVALID_ARG, "dt must be positive and finite");
  if (c->kp.fnbr) return fail(c, DGCNS_ERR_UNSUPPORTED, "adjoint on rotated-frame meshes is not implemented");
  if (c->kp.has_bf) return fail(c, DGCNS_ERR_UNSUPPORTED, "adjoint with a body force is not implemented");
  if (!(c->L.features & FEAT_ADJ)) return fail(c, DGCNS_ERR_UNSUPPORTED, "adjoint not compiled for this (k, nq)");
  if (overlap(lam_U, state_bytes(c), U_in, state_bytes(c)) || overlap(lam_dU, res_bytes(c), U_in, state_bytes(c)) ||
      overlap(lam_dU, res_bytes(c), lam_U, state_bytes(c)))
    return fail(c, DGCNS_ERR_INVALID_ARG, "U_in, lam_U and lam_dU must not overlap");
  const PrepFn prep = c->prm.precision == DGCNS_MIXED ? c->L.prep_fp32 : c->L.prep_fp64;
  // W = lam_dU + B lam_U (scratch), lam_dU <- A W
  {
    TimedScope ts(c, DGCNS_KT_ADJ_PREP);
    if (prep(c->state_elems, RK_A[stage], RK_B[stage], lam_U, lam_dU, c->d_R, c->stream) != 0)
      return cuda_fail(c, "adjoint stage preparation");
  }
  c->launches += 1;
  KParams km = c->kp;
  km.out_mode = 0;
  km.has_bf = 0;
  int r = run_op(c, OP_MASS, km, nullptr, c->d_R, c->d_R, nullptr, nullptr);  // Y = M^-1 W in place
  if (r) return r;
  KParams ka = c->kp;
  ka.out_mode = 2;
  ka.dt = dt;
  return run_adj(c, ka, U_in, nullptr, lam_U);
}

int dg_cns_kinetic_energy_gradient(dgcns_ctx* c, const double* U, double* G) {
  if (!c) return DGCNS_ERR_INVALID_ARG;
  DeviceScope ds(c);
  if (!U || !G || overlap(U, state_bytes(c), G, state_bytes(c)))
    return fail(c, DGCNS_ERR_INVALID_ARG, "U and G must be non-NULL arrays that do not overlap");
  KParams kp = c->kp;
  kp.tables = c->d_tab64;
  if (c->g64[0]) {
    kp.gcc = c->g64[0];
    kp.gm = c->g64[4];
  }
  TimedScope ts(c, DGCNS_KT_OTHER);
  const int r = c->L.ekgrad(kp, U, G, 1.0 / c->volume, c->stream);
  c->launches += 1;
  if (r == -2) return fail(c, DGCNS_ERR_UNSUPPORTED, "kinetic-energy gradient does not fit shared memory");
  if (r) return cuda_fail(c, "kinetic-energy gradient launch");
  return DGCNS_OK;
}

static KParams diag_params(const dgcns_ctx* c) {
  KParams kp = c->kp;
  kp.tables = c->d_tab64;
  if (c->g64[0]) {
    kp.gcc = c->g64[0];
    kp.gcv = c->g64[1];
    kp.gfc = c->g64[2];
    kp.gfv = c->g64[3];
    kp.gm = c->g64[4];
  }
  return kp;
}

int dg_cns_diagnostics(dgcns_ctx* c, const double* U, const void* LU, double* out) {
  if (!c) return DGCNS_ERR_INVALID_ARG;
  DeviceScope ds(c);
  if (!U || !out) return fail(c, DGCNS_ERR_INVALID_ARG, "NULL array");
  KParams kp = diag_params(c);
  int nblk = 0;
  const DiagFn f = c->prm.precision == DGCNS_MIXED ? c->L.diag_fp32 : c->L.diag_fp64;
  {
    TimedScope ts(c, DGCNS_KT_OTHER);
    const int r = f(kp, U, LU, c->d_partial, &nblk, c->stream);
    if (r == -2) return fail(c, DGCNS_ERR_UNSUPPORTED, "diagnostics kernel does not fit shared memory for this (k, nq)");
    if (r != 0) return cuda_fail(c, "diagnostics kernel launch");
  }
  c->launches += 1;
  std::vector<double> part((size_t)nblk * 10);
  if (cudaMemcpyAsync(part.data(), c->d_partial, part.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream) !=
          cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess)
    return cuda_fail(c, "diagnostics copy");
  double acc[10] = {0};
  for (int b = 0; b < nblk; ++b)
    for (int a = 0; a < 10; ++a) acc[a] += part[(size_t)b * 10 + a];
  out[0] = acc[1] / acc[0];
  out[1] = c->nu * acc[2] / acc[0];
  out[2] = LU ? -acc[3] / acc[0] : 0.0;
  for (int a = 0; a < 5; ++a) out[3 + a] = acc[4 + a];
  out[8] = acc[9];
  return acc[9] > 0 ? fail(c, DGCNS_ERR_NONFINITE, "state has non-finite entries") : DGCNS_OK;
}

// ---------------------------------------------------------------------------
// Diagnostics without allocation: the per-block partial sums live in a static
// device array instead of the context's buffer, and the final reduction runs
// on the GPU into the caller's device output.
// ---------------------------------------------------------------------------
}  // extern "C"

namespace {
constexpr int kNoallocRows = (int)(DGCNS_NOALLOC_SCRATCH_BYTES / (10 * sizeof(double)));
static __device__ __align__(256) double g_noalloc_partials[(size_t)kNoallocRows * 10];

std::mutex g_noalloc_mu;
double* g_noalloc_ptr[256] = {nullptr};

// Device address of g_noalloc_partials on the current device (looked up once per device).
int noalloc_scratch(dgcns_ctx* c, double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return cuda_fail(c, "cudaGetDevice");
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);
    if (e != cudaSuccess || !p)
      return fail(c, DGCNS_ERR_CUDA, std::string("cudaGetSymbolAddress of the no-alloc scratch: ") +
                                         cudaGetErrorString(e));
    g_noalloc_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_noalloc_ptr[dev];
  return DGCNS_OK;
}

// Sum the partial rows and write the normalised diagnostics: warp w sums column w (lane l takes rows
// l, l + 32, ... in order, then a shuffle tree in a fixed order), so the result is deterministic and
// differs from the host's serial sum only by rounding.
__global__ void noalloc_finalize(const double* __restrict__ partial, int nrows, double nu, int has_L,
                                 double* __restrict__ out) {
  __shared__ double acc[10];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (w < 10) {
    double s = 0.0;
    for (int b = lane; b < nrows; b += 32) s += partial[(size_t)b * 10 + w];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) acc[w] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    out[0] = acc[1] / acc[0];
    out[1] = nu * acc[2] / acc[0];
    out[2] = has_L ? -acc[3] / acc[0] : 0.0;
    for (int a = 0; a < 5; ++a) out[3 + a] = acc[4 + a];
    out[8] = acc[9];
  }
}
}  // namespace

extern "C" {

int dg_cns_diagnostics_noalloc(dgcns_ctx* c, const double* U, const void* LU, double* out_dev) {
  if (!c) return DGCNS_ERR_INVALID_ARG;
  DeviceScope ds(c);
  if (!U || !out_dev) return fail(c, DGCNS_ERR_INVALID_ARG, "NULL array");
  KParams kp = diag_params(c);
  const DiagFn f = c->prm.precision == DGCNS_MIXED ? c->L.diag_fp32 : c->L.diag_fp64;
  int nblk = 0;
  if (f(kp, nullptr, nullptr, nullptr, &nblk, c->stream) != 0) return cuda_fail(c, "diagnostics set-up");
  if (nblk > kNoallocRows)
    return fail(c, DGCNS_ERR_INVALID_ARG,
                "mesh too large for the no-alloc diagnostics: it needs " + std::to_string(nblk) +
                    " partial rows, the static scratch holds " + std::to_string(kNoallocRows));
  double* scratch = nullptr;
  const int r = noalloc_scratch(c, &scratch);
  if (r) return r;
  if (f(kp, U, LU, scratch, &nblk, c->stream) != 0) return cuda_fail(c, "no-alloc diagnostics kernel launch");
  noalloc_finalize<<<1, 320, 0, c->stream>>>(scratch, nblk, c->nu, LU ? 1 : 0, out_dev);
  c->launches += 2;
  if (cudaGetLastError() != cudaSuccess) return cuda_fail(c, "no-alloc diagnostics finalize launch");
  return DGCNS_OK;
}

int dg_cns_launch_count(const dgcns_ctx* c, int64_t* count) {
  if (!c || !count) return DGCNS_ERR_INVALID_ARG;
  *count = c->launches;
  return DGCNS_OK;
}

int dg_cns_status(dgcns_ctx* c) {
  if (!c) return DGCNS_ERR_INVALID_ARG;
  DeviceScope ds(c);
  int h = 0;
  if (cudaStreamSynchronize(c->stream) != cudaSuccess ||
      cudaMemcpy(&h, c->d_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return cuda_fail(c, "status read");
  if (h) {
    if (cudaMemset(c->d_err, 0, sizeof(int)) != cudaSuccess) return cuda_fail(c, "status reset");
    return fail(c, DGCNS_ERR_TIMEOUT, "a bounded wait in a kernel gave up (its results are invalid)");
  }
  return DGCNS_OK;
}

int dg_cns_timing(dgcns_ctx* c, int enable) {
  if (!c) return DGCNS_ERR_INVALID_ARG;
  DeviceScope ds(c);
  const int r = flush_times(c);
  if (r) return r;
  if (enable) {
    for (int i = 0; i < DGCNS_KT_COUNT; ++i) {
      c->kt_ms[i] = 0.0;
      c->kt_n[i] = 0;
    }
  }
  c->timing = enable != 0;
  return DGCNS_OK;
}

int dg_cns_kernel_times(dgcns_ctx* c, double* ms, int64_t* counts, int n) {
  if (!c) return DGCNS_ERR_INVALID_ARG;
  DeviceScope ds(c);
  if (n < 0 || n > DGCNS_KT_COUNT) return fail(c, DGCNS_ERR_INVALID_ARG, "n must be 0..DGCNS_KT_COUNT");
  const int r = flush_times(c);
  if (r) return r;
  for (int i = 0; i < n; ++i) {
    if (ms) ms[i] = c->kt_ms[i];
    if (counts) counts[i] = c->kt_n[i];
  }
  return DGCNS_OK;
}

int dg_cns_face_table(const dgcns_mesh* mesh, int* table, int* frames) {
  auto bad = [](const char* m) {
    g_create_err = m;
    return DGCNS_ERR_INVALID_ARG;
  };
  if (!mesh || (!table && !frames)) return bad("null mesh, or neither output given");
  if (mesh->mapping != DGCNS_MAP_ROTATED) return bad("the mesh is not a rotated-frame mesh");
  long long ncell = 1;
  for (int d = 0; d < 3; ++d) {
    if (mesh->n[d] < 1 || !(mesh->hi[d] > mesh->lo[d])) return bad("bad mesh extents");
    if (!mesh->periodic[d]) return bad("rotated-frame meshes must be periodic on every axis");
    ncell *= mesh->n[d];
    if (ncell > (1LL << 30)) return bad("too many cells (more than 2^30)");
  }
  if (!(mesh->map_param >= 0.0 && mesh->map_param < 18446744073709551616.0) ||
      mesh->map_param != std::floor(mesh->map_param))
    return bad("the frame seed (map_param) must be a non-negative integer below 2^64");
  const std::vector<int> fr = cell_frames(*mesh);
  if (frames) std::copy(fr.begin(), fr.end(), frames);
  if (table) {
    const std::vector<int> t = frame_face_table(*mesh, fr);
    std::copy(t.begin(), t.end(), table);
  }
  return DGCNS_OK;
}

const char* dg_cns_last_error(const dgcns_ctx* c) {
  if (!c) return g_create_err.c_str();
  return c->err.c_str();
}

}  // extern "C"
