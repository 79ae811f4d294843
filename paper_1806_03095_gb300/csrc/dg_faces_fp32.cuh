// Face-centric face kernel of the mixed form (FP32 arithmetic), affine meshes: the same face terms as
// face_pair_terms (Sec. 2.2.2: LLF flux, SIPG flux and the -1/2 (grad V, F_v(U, [[U]])) term; both cells'
// shares of every face once), organised so that every 1D contraction runs in registers:
//
//  1. trace tasks, one thread per (face, side, component): the thread reads its cell's component block as
//     x-lines, forms the face-layer values L and the normal derivatives D at the face nodes, interpolates
//     L to the convective and viscous face points, differentiates along both tangents by collocation and
//     interpolates D; the 2D tensor contractions of a face are held in the thread's registers, and each
//     result goes to shared memory once;
//  2. convective points, one thread per (face, point): the LLF flux, tested with the own side's V (the
//     other side's test is its negative);
//  3. viscous points: one thread per (face, point, side) forms F_v(U, grad U) . n of its side, then one
//     thread per (face, point) forms the SIPG flux and F_v(U^-+, [[U]] (x) n) of both sides;
//  4. test tasks, one thread per (face, side, component): the transposed contractions in registers, and the
//     two shares (value layer and normal derivative) written to the face buffer.
//
// Shares, signs and the layout of the face buffer are those of face_pair_terms.  The even-odd 1D
// operators come from constant memory with compile-time offsets.
#pragma once
#include "dg_faces.cuh"

namespace dgcns {

// One 1D line through an even-odd operator (DOUT x DIN, symmetry SYM) in registers: y = O x.
template <int DIN, int DOUT, int SYM>
__device__ __forceinline__ void eo_apply(const float* __restrict__ E, const float (&x)[DIN], float (&y)[DOUT]) {
  constexpr int IH = DIN / 2, OH = (DOUT + 1) / 2;
  const float* A = E;
  const float* B = E + OH * IH;
  const float* C = E + 2 * OH * IH;
  float xe[IH > 0 ? IH : 1], xo[IH > 0 ? IH : 1];
#pragma unroll
  for (int i = 0; i < IH; ++i) {
    xe[i] = x[i] + x[DIN - 1 - i];
    xo[i] = x[i] - x[DIN - 1 - i];
  }
#pragma unroll
  for (int q = 0; q < OH; ++q) {
    float e = (DIN & 1) ? C[q] * x[IH] : 0.f;
    float o = 0.f;
#pragma unroll
    for (int i = 0; i < IH; ++i) {
      e = fmaf(A[q * IH + i], xe[i], e);
      o = fmaf(B[q * IH + i], xo[i], o);
    }
    y[q] = e + o;
    if (!((DOUT & 1) && q == OH - 1)) y[DOUT - 1 - q] = SYM > 0 ? e - o : o - e;
  }
}

// K consecutive floats between registers and memory: 16-byte vectors when K is a multiple of 4 (the
// address then 16-byte aligned), else scalars.
template <int K>
__device__ __forceinline__ void arr_load(const float* p, float (&x)[K]) {
  if constexpr (K % 4 == 0) {
    vec_load<float, K>(p, x);
  } else {
#pragma unroll
    for (int i = 0; i < K; ++i) x[i] = p[i];
  }
}

template <int K>
__device__ __forceinline__ void arr_store(float* p, const float (&x)[K]) {
  if constexpr (K % 4 == 0) {
    vec_store<float, K>(p, x);
  } else {
#pragma unroll
    for (int i = 0; i < K; ++i) p[i] = x[i];
  }
}

// 2D tensor contraction in registers: X[NI1][NI0] (index 0 fastest) -> Y[NO1][NO0] with operator E0 along
// index 0 and E1 along index 1 (either may be the identity: NI == NO and E == nullptr is not used; every
// call applies both).
template <int NI0, int NI1, int NO0, int NO1, int SYM0, int SYM1>
__device__ __forceinline__ void eo_2d(const float* __restrict__ E0, const float* __restrict__ E1,
                                      const float (&X)[NI1 * NI0], float (&Y)[NO1 * NO0]) {
  float T[NI1][NO0];
#pragma unroll
  for (int b = 0; b < NI1; ++b) {
    float x[NI0], y[NO0];
#pragma unroll
    for (int a = 0; a < NI0; ++a) x[a] = X[b * NI0 + a];
    eo_apply<NI0, NO0, SYM0>(E0, x, y);
#pragma unroll
    for (int a = 0; a < NO0; ++a) T[b][a] = y[a];
  }
#pragma unroll
  for (int a = 0; a < NO0; ++a) {
    float x[NI1], y[NO1];
#pragma unroll
    for (int b = 0; b < NI1; ++b) x[b] = T[b][a];
    eo_apply<NI1, NO1, SYM1>(E1, x, y);
#pragma unroll
    for (int b = 0; b < NO1; ++b) Y[b * NO0 + a] = y[b];
  }
}

// Contraction along index 0 only: X[NB][NI] -> Y[NB][NO].
template <int NI, int NO, int NB, int SYM>
__device__ __forceinline__ void eo_dir0(const float* __restrict__ E, const float (&X)[NB * NI], float (&Y)[NB * NO]) {
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    float x[NI], y[NO];
#pragma unroll
    for (int a = 0; a < NI; ++a) x[a] = X[b * NI + a];
    eo_apply<NI, NO, SYM>(E, x, y);
#pragma unroll
    for (int a = 0; a < NO; ++a) Y[b * NO + a] = y[a];
  }
}

// Contraction along index 1 only: X[NI][NA] -> Y[NO][NA].
template <int NI, int NO, int NA, int SYM>
__device__ __forceinline__ void eo_dir1(const float* __restrict__ E, const float (&X)[NI * NA], float (&Y)[NO * NA]) {
#pragma unroll
  for (int a = 0; a < NA; ++a) {
    float x[NI], y[NO];
#pragma unroll
    for (int b = 0; b < NI; ++b) x[b] = X[b * NA + a];
    eo_apply<NI, NO, SYM>(E, x, y);
#pragma unroll
    for (int b = 0; b < NO; ++b) Y[b * NA + a] = y[b];
  }
}

// Face-layer values L and normal derivatives D (sum_i dl_i u_i along the normal lines) at the face nodes
// (j1 along the first tangent, fastest) of one component block src [N^3] of a cell, the face at layer
// id (0 or N-1) along direction DIR; the block is read as its N^2 x-lines.
template <int N, int DIR>
__device__ __forceinline__ void face_traces(const float* __restrict__ src, const float* __restrict__ dl, int id,
                                            float (&L)[N * N], float (&D)[N * N]) {
  const bool last = id != 0;
#pragma unroll
  for (int j = 0; j < N * N; ++j) D[j] = 0.f;
#pragma unroll
  for (int zz = 0; zz < N; ++zz)
#pragma unroll
    for (int yy = 0; yy < N; ++yy) {
      float x[N];
      if constexpr ((N * sizeof(float)) % 16 == 0) {
        vec_load<float, N>(src + (zz * N + yy) * N, x);
      } else {
#pragma unroll
        for (int a = 0; a < N; ++a) x[a] = src[(zz * N + yy) * N + a];
      }
      if constexpr (DIR == 0) {  // face node (y, z), layer x
        const int j = yy + N * zz;
        float acc = 0.f;
#pragma unroll
        for (int a = 0; a < N; ++a) acc = fmaf(dl[a], x[a], acc);
        D[j] = acc;
        L[j] = last ? x[N - 1] : x[0];
      } else if constexpr (DIR == 1) {  // face node (x, z), layer y
        const float w = dl[yy];
#pragma unroll
        for (int a = 0; a < N; ++a) D[a + N * zz] = fmaf(w, x[a], D[a + N * zz]);
        if (yy == 0 && !last) {
#pragma unroll
          for (int a = 0; a < N; ++a) L[a + N * zz] = x[a];
        }
        if (yy == N - 1 && last) {
#pragma unroll
          for (int a = 0; a < N; ++a) L[a + N * zz] = x[a];
        }
      } else {  // face node (x, y), layer z
        const float w = dl[zz];
#pragma unroll
        for (int a = 0; a < N; ++a) D[a + N * yy] = fmaf(w, x[a], D[a + N * yy]);
        if (zz == 0 && !last) {
#pragma unroll
          for (int a = 0; a < N; ++a) L[a + N * yy] = x[a];
        }
        if (zz == N - 1 && last) {
#pragma unroll
          for (int a = 0; a < N; ++a) L[a + N * yy] = x[a];
        }
      }
    }
}

// Shared-memory layout of one CTA (floats): per face, conv traces [2][5][QC^2] (the own side's slots
// later hold the LLF integrand), viscous traces [2][5][VS] with VS >= 4 QV^2 (U, d/dt1, d/dt2, normal
// derivative; later the four test integrands), the viscous normal fluxes [2][5][QV^2].  Padding against
// shared-memory bank conflicts: a (side, component) task writes and reads its 4 QV^2 viscous values as
// 16-byte vectors, so VS = 4 QV^2 + 4 puts the blocks of 8 neighbouring tasks on distinct banks (a stride
// of 4 QV^2 = 64 words put them all on the same 4 banks); the per-face stride is 8 (mod 32) words, so the
// tasks of the next face in the same quarter-warp land on other banks too.
template <int N, int QC, int QV>
struct TaskFaceSizes {
  static constexpr int PC = QC * QC, PV = QV * QV;
  static constexpr int CIN = (2 * 5 * PC + 3) & ~3;
  static constexpr int VS = 4 * PV + 4;
  static constexpr int VIN = 2 * 5 * VS;
  static constexpr int FVN = 2 * 5 * PV;
  static constexpr int RAW = CIN + VIN + FVN;
  static constexpr int PER_FACE = RAW + ((8 - RAW % 32) + 32) % 32;
};

template <int N, int QC, int QV, int FPB>
constexpr size_t task_face_smem_bytes() {
  return ((size_t)table_elems<N, QC, QV>() + (size_t)FPB * TaskFaceSizes<N, QC, QV>::PER_FACE + 3 * FPB) *
             sizeof(float) + 64;
}

// Phases 1-4 of the task kernel for faces normal to direction DIR (compile-time, so that the small
// per-point arrays indexed by direction stay in registers).
template <int N, int QC, int QV, int FPB, int NTH, int DIR>
__device__ __forceinline__ void face_task_body(const KParams& kp, float* __restrict__ FB, const Tab<float>& tb,
                                               const PhysT<float>& ph, float* sface, const float* stau, const int* eo,
                                               const int* en, int nb, int s) {
  using S = TaskFaceSizes<N, QC, QV>;
  constexpr int N2 = N * N, N3 = N * N * N, PC = S::PC, PV = S::PV;
  constexpr int d = DIR, t1 = DIR == 0 ? 1 : 0, t2 = DIR == 2 ? 1 : 2;
  const KConst<float>& kc = kconst<float>(kp);
  const float hinv_d = kc.hinv[d], hinv_1 = kc.hinv[t1], hinv_2 = kc.hinv[t2];
  const float area = kc.area[d];
  const float sgn = s ? 1.f : -1.f;
  const float* __restrict__ Ud = static_cast<const float*>(kp.Udev);

  // 1. trace tasks (face b, side sd: 0 own / 1 other, component c)
  for (int task = threadIdx.x; task < nb * 10; task += NTH) {
    const int b = task / 10, r = task - 10 * b, sd = r / 5, c = r - 5 * sd;
    const int cell = sd ? en[b] : eo[b];
    if (cell < 0) continue;  // wall: the ghost state is formed at the points
    const int id = (sd ? 1 - s : s) ? N - 1 : 0;  // the face's layer index along d in this cell
    const float* dl = (sd ? 1 - s : s) ? tb.dl1 : tb.dl0;
    const float* __restrict__ src = Ud + ((size_t)cell * 5 + c) * N3;
    float L[N2], D[N2];
    face_traces<N, DIR>(src, dl, id, L, D);
    float* fb = sface + b * S::PER_FACE;
    if (kp.conv) {
      float Uc[PC];
      eo_2d<N, N, QC, QC, 1, 1>(tb.eSc, tb.eSc, L, Uc);
      float* o = fb + (sd * 5 + c) * PC;
#pragma unroll
      for (int p = 0; p < PC; ++p) o[p] = Uc[p];
    }
    if (kp.visc) {
      float Uv[PV], G[PV];
      float* o = fb + S::CIN + (sd * 5 + c) * S::VS;
      eo_2d<N, N, QV, QV, 1, 1>(tb.eSv, tb.eSv, L, Uv);
      arr_store<PV>(o, Uv);
      eo_dir0<QV, QV, QV, -1>(tb.eDv, Uv, G);
      arr_store<PV>(o + PV, G);
      eo_dir1<QV, QV, QV, -1>(tb.eDv, Uv, G);
      arr_store<PV>(o + 2 * PV, G);
      eo_2d<N, N, QV, QV, 1, 1>(tb.eSv, tb.eSv, D, G);
      arr_store<PV>(o + 3 * PV, G);
    }
  }
  __syncthreads();

  // 2. convective points: LLF integrand of the own side (the other side's is its negative)
  if (kp.conv) {
    for (int task = threadIdx.x; task < nb * PC; task += NTH) {
      const int b = task / PC, p = task - PC * b;
      float* fb = sface + b * S::PER_FACE;
      float um[5], up[5];
#pragma unroll
      for (int c = 0; c < 5; ++c) um[c] = fb[c * PC + p];
      if (en[b] < 0) {
        wall_ghost(um, ph, up);
      } else {
#pragma unroll
        for (int c = 0; c < 5; ++c) up[c] = fb[(5 + c) * PC + p];
      }
      const float rm = 1.f / (ph.rho_r + um[0]), rp = 1.f / (ph.rho_r + up[0]);
      const float pm = pressure_dev(um, rm, ph.gm1), pp = pressure_dev(up, rp, ph.gm1);
      const float lm = sqrtf(um[1] * um[1] + um[2] * um[2] + um[3] * um[3]) * rm + sqrtf(fabsf(ph.gamma * (ph.p_r + pm) * rm));
      const float lp = sqrtf(up[1] * up[1] + up[2] * up[2] + up[3] * up[3]) * rp + sqrtf(fabsf(ph.gamma * (ph.p_r + pp) * rp));
      const float lam = lm > lp ? lm : lp;
      const float w = tb.wc[p % QC] * tb.wc[p / QC] * area;
      float fm[5], fp[5];
      conv_flux_dir(um, rm, pm, ph.H_r, d, fm);
      conv_flux_dir(up, rp, pp, ph.H_r, d, fp);
#pragma unroll
      for (int c = 0; c < 5; ++c) fb[c * PC + p] = w * (0.5f * sgn * (fm[c] + fp[c]) + 0.5f * lam * (um[c] - up[c]));
    }
  }

  if (kp.visc) {
    // 3a. F_v(U, grad U) . n of each side (n = sgn e_d: the d column), from the side's own traces
    for (int task = threadIdx.x; task < nb * 2 * PV; task += NTH) {
      const int b = task / (2 * PV), r = task - 2 * PV * b, sd = r / PV, p = r - PV * sd;
      float* fb = sface + b * S::PER_FACE;
      const bool wall = en[b] < 0;
      const int src = wall ? 0 : sd;  // wall: grad U+ = grad U-, U+ the ghost state
      const float* vi = fb + S::CIN;
      float u[5], Gr[5][3], F[5][3];
#pragma unroll
      for (int c = 0; c < 5; ++c) {
        const float* q = vi + (src * 5 + c) * S::VS + p;
        u[c] = q[0];
        Gr[c][t1] = q[PV] * hinv_1;
        Gr[c][t2] = q[2 * PV] * hinv_2;
        Gr[c][d] = q[3 * PV] * hinv_d;
      }
      if (wall && sd == 1) {
        float g[5];
        wall_ghost(u, ph, g);
#pragma unroll
        for (int c = 0; c < 5; ++c) u[c] = g[c];
      }
      visc_flux(u, Gr, ph, F);
      float* o = fb + S::CIN + S::VIN + sd * 5 * PV + p;
#pragma unroll
      for (int c = 0; c < 5; ++c) o[c * PV] = F[c][d] * sgn;
    }
    __syncthreads();
    // 3b. SIPG value integrands and the -1/2 (grad V, F_v(U, [[U]] (x) n)) integrands of both sides
    for (int task = threadIdx.x; task < nb * PV; task += NTH) {
      const int b = task / PV, p = task - PV * b;
      float* fb = sface + b * S::PER_FACE;
      const bool wall = en[b] < 0;
      float* vi = fb + S::CIN;
      const float* fv = vi + S::VIN;
      float um[5], up[5];
#pragma unroll
      for (int c = 0; c < 5; ++c) um[c] = vi[c * S::VS + p];
      if (wall) {
        wall_ghost(um, ph, up);
      } else {
#pragma unroll
        for (int c = 0; c < 5; ++c) up[c] = vi[(5 + c) * S::VS + p];
      }
      const float wgt = tb.wv[p % QV] * tb.wv[p / QV] * area;
      const float tau = stau[b];
      float jmp[5];
#pragma unroll
      for (int c = 0; c < 5; ++c) {
        jmp[c] = um[c] - up[c];
        const float v = -wgt * (0.5f * (fv[c * PV + p] + fv[(5 + c) * PV + p]) - tau * jmp[c]);
        vi[c * S::VS + p] = v;
        if (!wall) vi[(5 + c) * S::VS + p] = -v;
      }
      float Jg[5][3], F[5][3];
#pragma unroll
      for (int c = 0; c < 5; ++c) {
        Jg[c][t1] = 0.f;
        Jg[c][t2] = 0.f;
        Jg[c][d] = jmp[c] * sgn;
      }
      const float hw = -0.5f * wgt;
      visc_flux(um, Jg, ph, F);
#pragma unroll
      for (int c = 0; c < 5; ++c) {
        float* q = vi + c * S::VS + p;
        q[PV] = hw * hinv_1 * F[c][t1];
        q[2 * PV] = hw * hinv_2 * F[c][t2];
        q[3 * PV] = hw * hinv_d * F[c][d];
      }
      if (!wall) {
        visc_flux(up, Jg, ph, F);
#pragma unroll
        for (int c = 0; c < 5; ++c) {
          float* q = vi + (5 + c) * S::VS + p;
          q[PV] = hw * hinv_1 * F[c][t1];
          q[2 * PV] = hw * hinv_2 * F[c][t2];
          q[3 * PV] = hw * hinv_d * F[c][d];
        }
      }
    }
  }
  __syncthreads();

  // 4. test tasks: value-layer share L and normal-derivative share D of (face b, side sd, component c)
  for (int task = threadIdx.x; task < nb * 10; task += NTH) {
    const int b = task / 10, r = task - 10 * b, sd = r / 5, c = r - 5 * sd;
    const int cell = sd ? en[b] : eo[b];
    if (cell < 0) continue;
    const float* fb = sface + b * S::PER_FACE;
    float Ls[N2], Ds[N2];
#pragma unroll
    for (int j = 0; j < N2; ++j) {
      Ls[j] = 0.f;
      Ds[j] = 0.f;
    }
    if (kp.conv) {
      float X[PC], Y[N2];
      const float sg = sd ? -1.f : 1.f;
#pragma unroll
      for (int p = 0; p < PC; ++p) X[p] = sg * fb[c * PC + p];
      eo_2d<QC, QC, N, N, 1, 1>(tb.eScT, tb.eScT, X, Y);
#pragma unroll
      for (int j = 0; j < N2; ++j) Ls[j] = Y[j];
    }
    if (kp.visc) {
      const float* vi = fb + S::CIN + (sd * 5 + c) * S::VS;
      float V[PV], G[PV], T[PV], Y[N2];
      arr_load<PV>(vi, V);
      arr_load<PV>(vi + PV, G);
      eo_dir0<QV, QV, QV, -1>(tb.eDvT, G, T);
#pragma unroll
      for (int p = 0; p < PV; ++p) V[p] += T[p];
      arr_load<PV>(vi + 2 * PV, G);
      eo_dir1<QV, QV, QV, -1>(tb.eDvT, G, T);
#pragma unroll
      for (int p = 0; p < PV; ++p) V[p] += T[p];
      eo_2d<QV, QV, N, N, 1, 1>(tb.eSvT, tb.eSvT, V, Y);
#pragma unroll
      for (int j = 0; j < N2; ++j) Ls[j] += Y[j];
      arr_load<PV>(vi + 3 * PV, G);
      eo_2d<QV, QV, N, N, 1, 1>(tb.eSvT, tb.eSvT, G, Y);
#pragma unroll
      for (int j = 0; j < N2; ++j) Ds[j] = Y[j];
    }
    const int f = 2 * d + (sd ? 1 - s : s);
    float* po = FB + (((size_t)cell * 6 + f) * 2 * 5 + c) * N2;
    arr_store<N2>(po, Ls);
    arr_store<N2>(po + 5 * N2, Ds);
  }
}

template <int N, int QC, int QV, int FPB, int NTH>
__global__ void __launch_bounds__(NTH) dg_face_task_kernel(const KParams kp, float* __restrict__ FB) {
  using S = TaskFaceSizes<N, QC, QV>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* stab = reinterpret_cast<float*>(smem_raw);
  float* sface = stab + ((table_elems<N, QC, QV>() + 3) & ~3);
  float* stau = sface + FPB * S::PER_FACE;
  int* eo = reinterpret_cast<int*>(stau + FPB);
  int* en = eo + FPB;

  const int d = blockIdx.y;
  const int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
  const int nstd = (kp.Nc + FPB - 1) / FPB;
  int s, i0, nitems;
  if ((int)blockIdx.x < nstd) {
    s = 1;
    i0 = blockIdx.x * FPB;
    nitems = kp.Nc;
  } else {
    if (kp.periodic[d]) return;
    s = 0;
    i0 = (blockIdx.x - nstd) * FPB;
    nitems = kp.nc[t1] * kp.nc[t2];
    if (i0 >= nitems) return;
  }
  const int nb = min(FPB, nitems - i0);
  const Tab<float> tb = load_tables<float, N, QC, QV>(static_cast<const float*>(kp.tables), stab);
  const PhysT<float> ph = make_phys<float>(kp);
  if ((int)threadIdx.x < nb) {
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
    stau[threadIdx.x] = float(w ? te : fmax(te, kp.tau[n]));
  }
  __syncthreads();

  if (d == 0)
    face_task_body<N, QC, QV, FPB, NTH, 0>(kp, FB, tb, ph, sface, stau, eo, en, nb, s);
  else if (d == 1)
    face_task_body<N, QC, QV, FPB, NTH, 1>(kp, FB, tb, ph, sface, stau, eo, en, nb, s);
  else
    face_task_body<N, QC, QV, FPB, NTH, 2>(kp, FB, tb, ph, sface, stau, eo, en, nb, s);
}

// The task kernel serves the FP32 affine face terms at k = 3.  It compiles without spills at k = 4 and 5
// (128 and 255 registers per thread), but there it was slower than the warp-per-face kernel (mixed TGV per
// stage: k = 4, 51^3: 2.00 against 1.68 ms; k = 5, 40^3: 1.66 against 1.30 ms; measured): fewer warps fit
// an SM.  Faces per CTA by degree, for the shared memory of larger faces.
template <int N, int QC, int QV>
constexpr bool task_faces_ok() {
  return N == 4;
}

template <int N>
constexpr int task_faces_per_cta() {
  return N == 4 ? 12 : (N == 5 ? 8 : 6);
}

template <int N, int QC, int QV>
int launch_task_faces(const KParams& kp, void* FB, cudaStream_t st) {
  constexpr int FPB = task_faces_per_cta<N>(), NTH = 128;
  constexpr size_t smem = task_face_smem_bytes<N, QC, QV, FPB>();
  static_assert(smem <= 227 * 1024, "task face kernel shared memory");
  int extra_items = 0;
  for (int d = 0; d < 3; ++d) {
    if (kp.periodic[d]) continue;
    const int plane = kp.nc[d == 0 ? 1 : 0] * kp.nc[d == 2 ? 1 : 2];
    if (plane > extra_items) extra_items = plane;
  }
  auto k = dg_face_task_kernel<N, QC, QV, FPB, NTH>;
  static bool attr[kMaxDevices] = {};
  if (smem_attr_once(k, smem, attr)) return -1;
  const dim3 grid((kp.Nc + FPB - 1) / FPB + (extra_items + FPB - 1) / FPB, 3);
  k<<<grid, NTH, smem, st>>>(kp, static_cast<float*>(FB));
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace dgcns
