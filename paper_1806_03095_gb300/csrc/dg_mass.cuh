// Inverse mass (Sec. 2.3) and, optionally, the 2N stage update as a persistent, TMA-pipelined kernel.
// The standalone M^{-1} (and the split organisation's M^{-1} + update) has little arithmetic per byte
// in FP32, so it is bound by how many bytes each SM keeps in flight: every CTA streams batches of CB
// consecutive cells (one contiguous range) into shared memory with cp.async.bulk through a ring of NS
// buffers and mbarriers, so that the copies of batches i+1 .. i+NS-1 are in flight while batch i is
// swept.  Waits are bounded: after kWaitPolls unsuccessful polls the kernel sets the context's error
// word and returns.
#pragma once
#include <cstdint>

#include "dg_faces_fp32.cuh"
#include "dg_kernels.cuh"

namespace dgcns {

constexpr long long kWaitPolls = 1LL << 26;

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}

// global -> shared bulk copy (16-byte aligned addresses, size a multiple of 16), completion on bar
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// Poll the phase with the given parity; false after kWaitPolls unsuccessful polls.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  for (long long i = 0; i < kWaitPolls; ++i) {
    uint32_t done = 0;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// Usable when every cell's block is a multiple of 16 bytes in the residual type and in FP64.
template <typename T, int N>
constexpr bool mass_tma_ok() {
  return (5 * N * N * N * sizeof(T)) % 16 == 0 && (5 * N * N * N * 8) % 16 == 0;
}

template <typename T, int N, int QC, int QV, bool STAGE>
constexpr int mass_tma_table_elems() {
  return (int)(((table_elems<N, QC, QV>() * sizeof(T) + 15) / 16) * 16 / sizeof(T));
}

// Pipeline depth: FP32 needs more bytes in flight per SM (its sweeps are short); FP64 is ALU-bound.
template <typename T>
constexpr int mass_tma_stages() {
  return sizeof(T) == 4 ? 4 : 2;
}

template <typename T, int N, int QC, int QV, bool STAGE>
constexpr size_t mass_tma_bytes(int cb) {
  constexpr int NS = mass_tma_stages<T>();
  const size_t BV = (size_t)cb * 5 * N * N * N;
  return 8 * NS + 16 + (STAGE ? NS * BV * 8 : 0) + mass_tma_table_elems<T, N, QC, QV, STAGE>() * sizeof(T) +
         (NS * BV + (STAGE ? NS * BV : 0) + BV + 2 * BV) * sizeof(T);
}

// Cells per batch: the largest CB <= 8 with the CTA's shared memory below ~75 KB (3 CTAs per SM).
template <typename T, int N, int QC, int QV, bool STAGE>
constexpr int mass_tma_cells() {
  int cb = 8;
  while (cb > 1 && mass_tma_bytes<T, N, QC, QV, STAGE>(cb) > 75 * 1024) --cb;
  return cb;
}

constexpr int kMassThreads = 256;

// One 1D line through a square even-odd operator table (the layout of the sweep tables: even part
// OH x IH, odd part OH x IH, centre column when DIN is odd), input and output in registers.
template <typename T, int DIN, int DOUT>
__device__ __forceinline__ void eo_line(const T* __restrict__ E, const T (&x)[DIN], T (&y)[DOUT]) {
  constexpr int IH = DIN / 2, OH = (DOUT + 1) / 2;
  const T* A = E;
  const T* B = E + OH * IH;
  const T* C = E + 2 * OH * IH;
  T xe[IH > 0 ? IH : 1], xo[IH > 0 ? IH : 1];
#pragma unroll
  for (int i = 0; i < IH; ++i) {
    xe[i] = x[i] + x[DIN - 1 - i];
    xo[i] = x[i] - x[DIN - 1 - i];
  }
#pragma unroll
  for (int q = 0; q < OH; ++q) {
    T e = (DIN & 1) ? C[q] * x[IH] : T(0);
    T o = T(0);
#pragma unroll
    for (int i = 0; i < IH; ++i) {
      e += A[q * IH + i] * xe[i];
      o += B[q * IH + i] * xo[i];
    }
    y[q] = e + o;
    if (!((DOUT & 1) && q == OH - 1)) y[DOUT - 1 - q] = e - o;
  }
}

// M^{-1} of a batch (Sec. 2.3, M_e^{-1} = S^{-1} diag(1/(|J| w)) S^{-T}, the three 1D factors of each
// commuting): S^{-T} along x, y; then per z-line, in registers, S^{-T} along z, the scaling and S^{-1}
// along z; then S^{-1} along y, x, the last sweep writing to `out` (global memory or shared).  Five
// passes through shared memory instead of the eight of the generic routine.
template <typename T, int N, int CB, int GEO>
__device__ void mass_apply(const T* in, T* Abuf, T* Bbuf, T* out, const Tab<T>& tb, const KParams& kp, int e0,
                           int nb, bool negate) {
  constexpr int N2 = N * N, N3 = N * N * N;
  const int nbl = nb * 5;
  sweep<T, 0, N, N, N, N, 1, false>(in, Abuf, tb.eSmiT, nbl);
  __syncthreads();
  sweep<T, 1, N, N, N, N, 1, false>(Abuf, Bbuf, tb.eSmiT, nbl);
  __syncthreads();
  const T sg = negate ? T(-1) : T(1);
  const T detJ = kconst<T>(kp).detJ;
  for (int l = threadIdx.x; l < nbl * N2; l += blockDim.x) {
    const int blk = l / N2, r = l - blk * N2;
    const T* ip = Bbuf + blk * N3 + r;
    T x[N], y[N], z[N];
#pragma unroll
    for (int i = 0; i < N; ++i) x[i] = ip[i * N2];
    eo_line<T, N, N>(tb.eSmiT, x, y);
    const T wxy = tb.wm[r % N] * tb.wm[r / N];
#pragma unroll
    for (int q = 0; q < N; ++q) {
      T w = wxy * tb.wm[q];
      if (GEO == GEO_AFFINE)
        w *= detJ;
      else
        w *= static_cast<const T*>(kp.gm)[(size_t)(e0 + blk / 5) * N3 + r + q * N2];
      y[q] *= sg / w;
    }
    eo_line<T, N, N>(tb.eSmi, y, z);
    T* op = Abuf + blk * N3 + r;
#pragma unroll
    for (int i = 0; i < N; ++i) op[i * N2] = z[i];
  }
  __syncthreads();
  sweep<T, 1, N, N, N, N, 1, false>(Abuf, Bbuf, tb.eSmi, nbl);
  __syncthreads();
  sweep<T, 0, N, N, N, N, 1, false>(Bbuf, out, tb.eSmi, nbl);
}

// out_mode 0/1: Rout = (-1 if out_mode 1) M^{-1} Rin;  STAGE (out_mode 2): dU <- A dU + dt (-M^{-1} Rin),
// U_out <- U + B dU.  Rin may alias Rout, U may alias U_out (each batch is read before it is written).
template <typename T, int N, int QC, int QV, int CB, bool STAGE, int GEO>
__global__ void __launch_bounds__(kMassThreads) dg_mass_tma_kernel(const KParams kp, const double* U, const T* Rin,
                                                                   T* Rout, T* dU, double* Uout) {
  constexpr int N3 = N * N * N, CV = 5 * N3, BV = CB * CV;
  constexpr int NS = mass_tma_stages<T>();
  constexpr int HDR = ((8 * NS + 15) / 16) * 16;  // barriers, padded to 16 bytes
  extern __shared__ __align__(16) unsigned char smem_raw[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);        // [NS]
  double* bufU = reinterpret_cast<double*>(smem_raw + HDR);     // STAGE: [NS][BV]
  T* stab = reinterpret_cast<T*>(smem_raw + HDR + (STAGE ? NS * BV * 8 : 0));
  T* bufR = stab + mass_tma_table_elems<T, N, QC, QV, STAGE>();  // [NS][BV]
  T* bufD = bufR + NS * BV;                                       // STAGE: [NS][BV]
  T* sr = bufD + (STAGE ? NS * BV : 0);                           // result [BV]
  T* ma = sr + BV;                                                // sweep arena [2 BV]
  const int nbatch = (kp.Nc + CB - 1) / CB;
  if ((int)blockIdx.x >= nbatch) return;
  const Tab<T> tb = load_tables<T, N, QC, QV>(static_cast<const T*>(kp.tables), stab);
  const bool readD = STAGE && kp.A != 0.0;
  if (threadIdx.x == 0) {
    for (int q = 0; q < NS; ++q) mbar_init(&bar[q], 1);
    mbar_fence_init();
  }
  __syncthreads();
  auto issue = [&](int b, int slot) {  // thread 0
    const int e0 = b * CB, nb = min(CB, kp.Nc - e0);
    const uint32_t bt = (uint32_t)(nb * CV * sizeof(T)), b8 = (uint32_t)(nb * CV * 8);
    mbar_expect_tx(&bar[slot], bt + (STAGE ? b8 + (readD ? bt : 0u) : 0u));
    bulk_load(bufR + slot * BV, Rin + (size_t)e0 * CV, bt, &bar[slot]);
    if (STAGE) {
      bulk_load(bufU + slot * BV, U + (size_t)e0 * CV, b8, &bar[slot]);
      if (readD) bulk_load(bufD + slot * BV, dU + (size_t)e0 * CV, bt, &bar[slot]);
    }
  };
  // prologue: the first NS-1 batches of this CTA
  if (threadIdx.x == 0)
    for (int q = 0; q < NS - 1; ++q)
      if ((int)blockIdx.x + q * (int)gridDim.x < nbatch) issue(blockIdx.x + q * gridDim.x, q);
  int it = 0;
  bool timed_out = false;
  for (int b = blockIdx.x; b < nbatch; b += gridDim.x, ++it) {
    const int slot = it % NS;
    // batch it+NS-1 goes into the slot released at the end of iteration it-1
    const int bn = b + (NS - 1) * gridDim.x;
    if (threadIdx.x == 0 && bn < nbatch) issue(bn, (it + NS - 1) % NS);
    const int e0 = b * CB, nb = min(CB, kp.Nc - e0);
    const bool ok = mbar_wait(&bar[slot], (uint32_t)((it / NS) & 1));
    if (__syncthreads_or(!ok)) {
      timed_out = true;
      break;
    }
    const size_t base = (size_t)e0 * CV;
    // without the stage update the last sweep writes the result straight to global memory
    mass_apply<T, N, CB, GEO>(bufR + slot * BV, ma, ma + BV, STAGE ? sr : Rout + base, tb, kp, e0, nb,
                              kp.out_mode != 0);
    __syncthreads();
    if (STAGE) {
      const T A = T(kp.A), dt = T(kp.dt);
      const double B = kp.B;
      const T* dold = bufD + slot * BV;
      const double* uold = bufU + slot * BV;
      for (int i = threadIdx.x; i < nb * CV; i += blockDim.x) {
        const T du = (readD ? A * dold[i] : T(0)) + dt * sr[i];
        dU[base + i] = du;
        Uout[base + i] = uold[i] + B * double(du);
      }
    }
    __syncthreads();
  }
  if (timed_out) {
    // give the copies still in flight (iterations it .. it+NS-1) a bounded chance to land before the CTA exits
    if (threadIdx.x == 0) {
      atomicExch(kp.err, 1);
      for (int q = 0; q < NS; ++q) {
        const int j = it + q;
        if ((int)blockIdx.x + j * (int)gridDim.x < nbatch) mbar_wait(&bar[j % NS], (uint32_t)((j / NS) & 1));
      }
    }
    __syncthreads();
  }
}

template <typename T, int N, int QC, int QV, bool STAGE, int GEO>
int launch_mass_tma(const KParams& kp, const void* Rin, void* Rout, void* dU, const double* U, double* Uout,
                    cudaStream_t st) {
  constexpr int CB = mass_tma_cells<T, N, QC, QV, STAGE>();
  constexpr size_t smem = mass_tma_bytes<T, N, QC, QV, STAGE>(CB);
  static_assert(smem <= 227 * 1024, "mass kernel shared memory");
  auto k = dg_mass_tma_kernel<T, N, QC, QV, CB, STAGE, GEO>;
  // persistent grid: SMs x resident CTAs of the current device (looked up once per device)
  static int grid_per_sm_dev[kMaxDevices] = {};
  static int nsm_dev[kMaxDevices] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return -1;
  int& grid_per_sm = grid_per_sm_dev[dev];
  int& nsm = nsm_dev[dev];
  if (grid_per_sm == 0) {
    int g = 0, m = 0;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
        cudaDeviceGetAttribute(&m, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g, k, kMassThreads, smem) != cudaSuccess || g < 1)
      return -1;
    nsm = m;
    grid_per_sm = g;
  }
  const int nbatch = (kp.Nc + CB - 1) / CB;
  const int grid = nbatch < nsm * grid_per_sm ? nbatch : nsm * grid_per_sm;
  k<<<grid, kMassThreads, smem, st>>>(kp, U, static_cast<const T*>(Rin), static_cast<T*>(Rout), static_cast<T*>(dU),
                                      Uout);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}


// ---------------------------------------------------------------------------
// M^{-1} of FP32 data at k = 3 (affine): one (cell, component) block of N^3 = 64 values per thread, the six
// 1D sweeps and the scaling in registers (S^-T along x, y, z; 1 / (|J| w); S^-1 along x, y, z).  A CTA
// takes 128 consecutive blocks (one contiguous range): coalesced 16-byte loads into shared memory rows
// padded to N^3 + 4 floats (so the 16-byte row reads of 8 neighbouring threads meet distinct banks),
// the per-thread sweeps, and coalesced 16-byte stores; with STAGE the 2N update (and the next deviation
// state when kp.devOut is set) runs in that store pass.  No shared-memory traffic inside the sweeps, so
// the kernel is bound by HBM.  out_mode 0: Rout = M^-1 Rin; 1: Rout = -M^-1 Rin; STAGE: L = -M^-1 Rin.
// Rin may alias Rout and U may alias Uout (a CTA reads its whole range before it writes).
// ---------------------------------------------------------------------------
constexpr int kMassRegThreads = 128;

template <int N>
__device__ __forceinline__ void mass_block_regs(float (&x)[N * N * N], const Tab<float>& tb, float sg_detJinv) {
  constexpr int N2 = N * N;
  // S^-T along x (index 0), y, z
#pragma unroll
  for (int l = 0; l < N2; ++l) {
    float a[N], b[N];
#pragma unroll
    for (int i = 0; i < N; ++i) a[i] = x[l * N + i];
    eo_apply<N, N, 1>(tb.eSmiT, a, b);
#pragma unroll
    for (int i = 0; i < N; ++i) x[l * N + i] = b[i];
  }
#pragma unroll
  for (int z = 0; z < N; ++z)
#pragma unroll
    for (int i0 = 0; i0 < N; ++i0) {
      float a[N], b[N];
#pragma unroll
      for (int i = 0; i < N; ++i) a[i] = x[z * N2 + i * N + i0];
      eo_apply<N, N, 1>(tb.eSmiT, a, b);
#pragma unroll
      for (int i = 0; i < N; ++i) x[z * N2 + i * N + i0] = b[i];
    }
  float iw[N];
#pragma unroll
  for (int i = 0; i < N; ++i) iw[i] = 1.f / tb.wm[i];
#pragma unroll
  for (int l = 0; l < N2; ++l) {
    float a[N], b[N];
#pragma unroll
    for (int i = 0; i < N; ++i) a[i] = x[i * N2 + l];
    eo_apply<N, N, 1>(tb.eSmiT, a, b);
    const float wl = iw[l % N] * iw[l / N] * sg_detJinv;
#pragma unroll
    for (int i = 0; i < N; ++i) b[i] *= wl * iw[i];
    eo_apply<N, N, 1>(tb.eSmi, b, a);
#pragma unroll
    for (int i = 0; i < N; ++i) x[i * N2 + l] = a[i];
  }
  // S^-1 along y, x
#pragma unroll
  for (int z = 0; z < N; ++z)
#pragma unroll
    for (int i0 = 0; i0 < N; ++i0) {
      float a[N], b[N];
#pragma unroll
      for (int i = 0; i < N; ++i) a[i] = x[z * N2 + i * N + i0];
      eo_apply<N, N, 1>(tb.eSmi, a, b);
#pragma unroll
      for (int i = 0; i < N; ++i) x[z * N2 + i * N + i0] = b[i];
    }
#pragma unroll
  for (int l = 0; l < N2; ++l) {
    float a[N], b[N];
#pragma unroll
    for (int i = 0; i < N; ++i) a[i] = x[l * N + i];
    eo_apply<N, N, 1>(tb.eSmi, a, b);
#pragma unroll
    for (int i = 0; i < N; ++i) x[l * N + i] = b[i];
  }
}

template <int N, int QC, int QV, bool STAGE>
__global__ void __launch_bounds__(kMassRegThreads) dg_mass_reg_kernel(const KParams kp, const double* U,
                                                                      const float* Rin, float* Rout, float* dU,
                                                                      double* Uout) {
  constexpr int N3 = N * N * N, V4 = N3 / 4, RS = N3 + 4, NB = kMassRegThreads;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* stab = reinterpret_cast<float*>(smem_raw);
  float* sb = stab + ((table_elems<N, QC, QV>() + 3) & ~3);  // [NB][RS]
  const long long nblocks = (long long)kp.Nc * 5;
  const long long b0 = (long long)blockIdx.x * NB;
  if (b0 >= nblocks) return;
  const int nb = (int)min((long long)NB, nblocks - b0);
  const Tab<float> tb = load_tables<float, N, QC, QV>(static_cast<const float*>(kp.tables), stab);
  const size_t base = (size_t)b0 * N3;
  const float4* src = reinterpret_cast<const float4*>(Rin + base);
  batched_pass<(NB * V4 + kMassRegThreads - 1) / kMassRegThreads>(
      threadIdx.x, kMassRegThreads, nb * V4, [&](int f) { return src[f]; },
      [&](int f, float4 v) { reinterpret_cast<float4*>(sb + (f / V4) * RS)[f % V4] = v; });
  __syncthreads();
  if ((int)threadIdx.x < nb) {
    float x[N3];
    float* row = sb + threadIdx.x * RS;
    vec_load<float, N3>(row, x);
    const float sg = (STAGE || kp.out_mode != 0) ? -1.f : 1.f;
    mass_block_regs<N>(x, tb, sg / kconst<float>(kp).detJ);
    vec_store<float, N3>(row, x);
  }
  __syncthreads();
  if (!STAGE) {
    float4* dst = reinterpret_cast<float4*>(Rout + base);
    for (int f = threadIdx.x; f < nb * V4; f += kMassRegThreads)
      dst[f] = reinterpret_cast<const float4*>(sb + (f / V4) * RS)[f % V4];
    return;
  }
  const float A = float(kp.A), dt = float(kp.dt);
  const double B = kp.B;
  const bool readD = kp.A != 0.0;
  float* dev = static_cast<float*>(kp.devOut);
  struct In {
    float4 d;
    double2 u0, u1;
  };
  batched_pass<(NB * V4 + kMassRegThreads - 1) / kMassRegThreads>(
      threadIdx.x, kMassRegThreads, nb * V4,
      [&](int f) {
        In v;
        v.d = readD ? reinterpret_cast<const float4*>(dU + base)[f] : make_float4(0.f, 0.f, 0.f, 0.f);
        v.u0 = reinterpret_cast<const double2*>(U + base)[2 * f];
        v.u1 = reinterpret_cast<const double2*>(U + base)[2 * f + 1];
        return v;
      },
      [&](int f, In v) {
        const float4 L = reinterpret_cast<const float4*>(sb + (f / V4) * RS)[f % V4];
        float4 d;
        d.x = A * v.d.x + dt * L.x;
        d.y = A * v.d.y + dt * L.y;
        d.z = A * v.d.z + dt * L.z;
        d.w = A * v.d.w + dt * L.w;
        reinterpret_cast<float4*>(dU + base)[f] = d;
        double2 o0, o1;
        o0.x = v.u0.x + B * double(d.x);
        o0.y = v.u0.y + B * double(d.y);
        o1.x = v.u1.x + B * double(d.z);
        o1.y = v.u1.y + B * double(d.w);
        reinterpret_cast<double2*>(Uout + base)[2 * f] = o0;
        reinterpret_cast<double2*>(Uout + base)[2 * f + 1] = o1;
        if (dev != nullptr) {
          const int c = (int)(((b0 + f / V4)) % 5);
          const double ref = c == 0 ? kp.rho_ref : (c == 4 ? kp.rhoE_ref : 0.0);
          reinterpret_cast<float4*>(dev + base)[f] =
              make_float4(float(o0.x - ref), float(o0.y - ref), float(o1.x - ref), float(o1.y - ref));
        }
      });
}

template <int N, int QC, int QV>
constexpr bool mass_reg_ok() {
  return N == 4;
}

template <int N, int QC, int QV, bool STAGE>
int launch_mass_reg(const KParams& kp, const void* Rin, void* Rout, void* dU, const double* U, double* Uout,
                    cudaStream_t st) {
  constexpr size_t smem =
      ((size_t)((table_elems<N, QC, QV>() + 3) & ~3) + (size_t)kMassRegThreads * (N * N * N + 4)) * sizeof(float) + 64;
  static_assert(smem <= 227 * 1024, "register mass kernel shared memory");
  auto k = dg_mass_reg_kernel<N, QC, QV, STAGE>;
  static bool attr[kMaxDevices] = {};
  if (smem_attr_once(k, smem, attr)) return -1;
  const long long nblocks = (long long)kp.Nc * 5;
  const int grid = (int)((nblocks + kMassRegThreads - 1) / kMassRegThreads);
  k<<<grid, kMassRegThreads, smem, st>>>(kp, U, static_cast<const float*>(Rin), static_cast<float*>(Rout),
                                         static_cast<float*>(dU), Uout);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}
}  // namespace dgcns
