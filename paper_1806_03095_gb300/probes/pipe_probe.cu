// Throughput probe of the arithmetic pipes the operator kernels can use on GB300 (not part of libdgcns):
// FP64 FMA on the CUDA cores (DFMA), FP64 tensor-core MMA (mma.sync m8n8k4 f64), both at once (half the
// warps of every CTA each), FP32 FMA (FFMA) and TF32 tensor-core MMA (mma.sync m16n8k8, FP32 accumulate).
// Every thread runs independent dependency chains; the result is stored so nothing is dead code.
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o pipe_probe pipe_probe.cu && ./pipe_probe
#include <cstdio>
#include <cuda_runtime.h>

constexpr int kChains = 8;

__device__ __forceinline__ void dfma_block(double (&a)[kChains], double b, double c) {
#pragma unroll
  for (int j = 0; j < kChains; ++j) a[j] = fma(a[j], b, c);
}

__device__ __forceinline__ void dmma_block(double (&acc)[4][2], double a, double b) {
#pragma unroll
  for (int j = 0; j < 4; ++j)
    asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};\n"
                 : "+d"(acc[j][0]), "+d"(acc[j][1])
                 : "d"(a), "d"(b));
}

// mode 0 DFMA, 1 DMMA, 2 DFMA on even warps and DMMA on odd warps, 3 FFMA, 4 TF32 MMA
__global__ void probe(int mode, int iters, double* out) {
  const int warp = threadIdx.x >> 5;
  const bool use_mma = mode == 1 || (mode == 2 && (warp & 1));
  double r = 0.0;
  if (mode <= 2) {
    if (use_mma) {
      double acc[4][2];
      for (int j = 0; j < 4; ++j) acc[j][0] = acc[j][1] = 1e-3 * (threadIdx.x + j);
      const double a = 1.0 + 1e-9 * threadIdx.x, b = 1.0 - 1e-9 * threadIdx.x;
      for (int it = 0; it < iters; ++it) dmma_block(acc, a, b);
      for (int j = 0; j < 4; ++j) r += acc[j][0] + acc[j][1];
    } else {
      double a[kChains];
      for (int j = 0; j < kChains; ++j) a[j] = 1e-3 * (threadIdx.x + j);
      const double b = 0.999999, c = 1e-7;
      // 4 DFMA blocks per iteration: the same number of FP64 flops as the MMA iteration per warp
      // (4 x 256 FMA per warp = 1024; 4 x 8 chains x 32 lanes = 1024)
      for (int it = 0; it < iters; ++it) {
        dfma_block(a, b, c);
        dfma_block(a, b, c);
        dfma_block(a, b, c);
        dfma_block(a, b, c);
      }
      for (int j = 0; j < kChains; ++j) r += a[j];
    }
  } else if (mode == 3) {
    float a[kChains];
    for (int j = 0; j < kChains; ++j) a[j] = 1e-3f * (threadIdx.x + j);
    const float b = 0.999999f, c = 1e-7f;
    for (int it = 0; it < iters; ++it)
#pragma unroll
      for (int rep = 0; rep < 16; ++rep)
#pragma unroll
        for (int j = 0; j < kChains; ++j) a[j] = fmaf(a[j], b, c);
    for (int j = 0; j < kChains; ++j) r += a[j];
  } else {
    float acc[4][4];
    for (int j = 0; j < 4; ++j)
      for (int k = 0; k < 4; ++k) acc[j][k] = 1e-3f * (threadIdx.x + j + k);
    const unsigned a0 = __float_as_uint(1.0f), a1 = __float_as_uint(0.5f), a2 = __float_as_uint(0.25f),
                   a3 = __float_as_uint(0.125f), b0 = __float_as_uint(1.0f), b1 = __float_as_uint(0.75f);
    for (int it = 0; it < iters; ++it)
#pragma unroll
      for (int j = 0; j < 4; ++j)
        asm volatile(
            "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
            "{%0, %1, %2, %3};\n"
            : "+f"(acc[j][0]), "+f"(acc[j][1]), "+f"(acc[j][2]), "+f"(acc[j][3])
            : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
    for (int j = 0; j < 4; ++j) r += acc[j][0] + acc[j][1] + acc[j][2] + acc[j][3];
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = r;
}

int main() {
  int dev = 0, nsm = 0, clk = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int threads = 256, blocks = nsm * 8;
  double* out = nullptr;
  if (cudaMalloc(&out, sizeof(double) * threads * blocks) != cudaSuccess) return 1;
  const char* names[5] = {"DFMA (FP64, CUDA cores)", "DMMA m8n8k4 (FP64 tensor)", "DFMA + DMMA (half the warps each)",
                          "FFMA (FP32, CUDA cores)", "TF32 MMA m16n8k8 (FP32 accumulate)"};
  const int iters[5] = {1 << 12, 1 << 12, 1 << 12, 1 << 13, 1 << 14};
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  printf("SMs %d, %d CTAs x %d threads\n", nsm, blocks, threads);
  for (int mode = 0; mode < 5; ++mode) {
    probe<<<blocks, threads>>>(mode, 16, out);  // warm-up
    cudaEventRecord(e0);
    probe<<<blocks, threads>>>(mode, iters[mode], out);
    cudaEventRecord(e1);
    if (cudaEventSynchronize(e1) != cudaSuccess) {
      printf("mode %d failed: %s\n", mode, cudaGetErrorString(cudaGetLastError()));
      return 1;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    const double warps = (double)blocks * threads / 32.0;
    double flop;  // 2 flops per FMA
    if (mode <= 2)
      flop = warps * iters[mode] * 1024.0 * 2.0;  // 1024 FMA per warp and iteration (both kinds)
    else if (mode == 3)
      flop = (double)blocks * threads * iters[mode] * 16.0 * kChains * 2.0;
    else
      flop = warps * iters[mode] * 4.0 * 16 * 8 * 8 * 2.0;
    printf("%-40s %9.3f ms  %9.2f TFLOP/s\n", names[mode], ms, flop / (ms * 1e-3) / 1e12);
  }
  cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, dev);
  printf("max SM clock %.0f MHz\n", clk / 1e3);
  cudaFree(out);
  return 0;
}
