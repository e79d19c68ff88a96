// Measured arithmetic rates of the CUDA-core pipes that the FP64-grade steps can use: native
// FP64 fused multiply-adds and FP32 fused multiply-adds. A float-float complex multiply-add of
// arith.cuh is 48 FP32-pipe operations, so the FP32 rate / 96 (flops / 2 per operation / 48) is
// the ALU roofline of the float-float kernels (screening, bosonic transforms).
//
// Each thread runs 8 independent dependency chains for a fixed number of steps; the result is
// written only if it is a particular value no input produces, so the compiler keeps the work
// and the output buffer is never touched in practice.
#include <cuda_runtime.h>

#include "gw_internal.h"

namespace gwi {
namespace {

constexpr int kChains = 8;
constexpr int kBlocks = 152 * 8, kThreads = 256;

__global__ void k_rate_fp64(int steps, double seed, double* sink) {
  double a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) a[c] = seed + threadIdx.x + c;
  const double m = 1.0 - 1e-9, s = 1e-9;
  for (int i = 0; i < steps; ++i)
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = fma(a[c], m, s);
  double t = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) t += a[c];
  if (t == -1.2345) sink[0] = t;
}

__global__ void k_rate_fp32(int steps, float seed, float* sink) {
  float a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) a[c] = seed + threadIdx.x + c;
  const float m = 1.0f - 1e-6f, s = 1e-6f;
  for (int i = 0; i < steps; ++i)
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = fmaf(a[c], m, s);
  float t = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) t += a[c];
  if (t == -1.2345f) sink[0] = t;
}

template <class K, class... A>
double time_ms(K kernel, cudaStream_t st, A... args) {
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  kernel<<<kBlocks, kThreads, 0, st>>>(args...);  // warm-up
  cudaEventRecord(e0, st);
  kernel<<<kBlocks, kThreads, 0, st>>>(args...);
  cudaEventRecord(e1, st);
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return ms;
}

}  // namespace
}  // namespace gwi

using namespace gwi;

extern "C" gw_status gw_measure_alu(int device, double* fp64_tflops, double* fp32_tflops) {
  if (!fp64_tflops || !fp32_tflops) return GW_EINVAL;
  if (cudaSetDevice(device) != cudaSuccess) return GW_ECUDA;
  double* sink = nullptr;
  if (cudaMalloc((void**)&sink, 64) != cudaSuccess) {
    cudaGetLastError();
    return GW_ENOMEM;
  }
  cudaStream_t st = nullptr;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
    cudaFree(sink);
    return GW_ECUDA;
  }
  const double threads = (double)kBlocks * kThreads;
  const int s64 = 2000, s32 = 40000;
  const double t64 = time_ms(k_rate_fp64, st, s64, 1.0, sink);
  const double t32 = time_ms(k_rate_fp32, st, s32, 1.0f, (float*)sink);
  const cudaError_t e = cudaGetLastError();
  cudaStreamDestroy(st);
  cudaFree(sink);
  if (e != cudaSuccess || !(t64 > 0) || !(t32 > 0)) return GW_ECUDA;
  *fp64_tflops = 2.0 * threads * kChains * s64 / (t64 * 1e-3) / 1e12;
  *fp32_tflops = 2.0 * threads * kChains * s32 / (t32 * 1e-3) / 1e12;
  return GW_OK;
}
