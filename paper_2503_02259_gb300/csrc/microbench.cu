// Pipe-rate microbenchmarks behind gp_measure_pipe_rates (include/gp.h).
//
// The on-the-fly product is bound by the SM's arithmetic pipes, not by HBM:
// the FP32 FMA pipe (the contraction, packed FP32x2 FMAs) and the MUFU unit
// (ex2 / sqrt of the kernel evaluation).  These kernels measure both rates on
// the current device so that the roofline denominators derived from unit
// counts and clocks can be checked against the hardware.  Every loop has a
// fixed trip count; nothing waits on anything.
#include <cuda_runtime.h>

#include "gp_internal.cuh"

namespace {

constexpr int kMbThreads = 256;
constexpr int kMbBlocksPerSm = 8;     // 2048 resident threads per SM
constexpr int kFmaChains = 8;         // independent FFMA2 chains per thread
constexpr int kFmaIters = 40000;      // x 4 unrolled x 8 chains FFMA2 per thread
constexpr int kMufuChains = 16;       // independent ex2 chains per thread
constexpr int kMufuIters = 2500;      // x 8 unrolled x 16 chains ex2 per thread

__device__ float g_mb_sink;           // written only if a chain hits a value it never reaches

__global__ void __launch_bounds__(kMbThreads) fma2_rate_kernel(float seed) {
  float2 acc[kFmaChains];
  const float2 mul = make_float2(0.9999999f, 0.9999998f);
  const float2 add = make_float2(seed * 1e-7f, seed * 2e-7f);
#pragma unroll
  for (int c = 0; c < kFmaChains; ++c)
    acc[c] = make_float2(static_cast<float>(threadIdx.x) * 1e-3f + c, blockIdx.x * 1e-3f);
  for (int it = 0; it < kFmaIters; ++it) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
#pragma unroll
      for (int c = 0; c < kFmaChains; ++c) acc[c] = __ffma2_rn(acc[c], mul, add);
    }
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kFmaChains; ++c) s += acc[c].x + acc[c].y;
  if (s == 1234.5f) g_mb_sink = s;   // keeps every chain live
}

__global__ void __launch_bounds__(kMbThreads) mufu_rate_kernel(float seed) {
  float x[kMufuChains];
#pragma unroll
  for (int c = 0; c < kMufuChains; ++c) x[c] = seed + 1e-3f * c + 1e-6f * threadIdx.x;
  for (int it = 0; it < kMufuIters; ++it) {
#pragma unroll
    for (int r = 0; r < 8; ++r) {
#pragma unroll
      for (int c = 0; c < kMufuChains; ++c) x[c] = gp::dev::ex2_approx(-x[c]);   // stays in (0, 1]
    }
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kMufuChains; ++c) s += x[c];
  if (s == 1234.5f) g_mb_sink = s;
}

}  // namespace

extern "C" gp_status gp_measure_pipe_rates(double* fp32_tflops, double* mufu_ex2_gops, void* stream) {
  if (fp32_tflops == nullptr || mufu_ex2_gops == nullptr) {
    gp::set_error("gp_measure_pipe_rates: NULL output");
    return GP_ERR_ARG;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  for (int i = 0; i < 4 && e == cudaSuccess; ++i) e = cudaEventCreate(&ev[i]);
  const int blocks = nsm * kMbBlocksPerSm;
  if (e == cudaSuccess) {
    // One untimed launch of each, then one timed launch of each.
    fma2_rate_kernel<<<blocks, kMbThreads, 0, st>>>(1.f);
    mufu_rate_kernel<<<blocks, kMbThreads, 0, st>>>(0.5f);
    cudaEventRecord(ev[0], st);
    fma2_rate_kernel<<<blocks, kMbThreads, 0, st>>>(1.f);
    cudaEventRecord(ev[1], st);
    cudaEventRecord(ev[2], st);
    mufu_rate_kernel<<<blocks, kMbThreads, 0, st>>>(0.5f);
    cudaEventRecord(ev[3], st);
    e = cudaGetLastError();
  }
  float ms_fma = 0.f, ms_mufu = 0.f;
  if (e == cudaSuccess) e = cudaEventSynchronize(ev[3]);
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms_fma, ev[0], ev[1]);
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms_mufu, ev[2], ev[3]);
  for (int i = 0; i < 4; ++i)
    if (ev[i]) cudaEventDestroy(ev[i]);
  if (e != cudaSuccess) {
    gp::set_error(std::string("gp_measure_pipe_rates: ") + cudaGetErrorString(e));
    return GP_ERR_CUDA;
  }
  const double threads = static_cast<double>(blocks) * kMbThreads;
  // FFMA2 = two fused multiply-adds = 4 flops.
  const double flops = threads * kFmaIters * 4.0 * kFmaChains * 4.0;
  const double ex2s = threads * kMufuIters * 8.0 * kMufuChains;
  *fp32_tflops = flops / (ms_fma * 1e-3) / 1e12;
  *mufu_ex2_gops = ex2s / (ms_mufu * 1e-3) / 1e9;
  return GP_OK;
}
