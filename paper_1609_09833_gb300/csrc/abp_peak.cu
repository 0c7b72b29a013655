// abp_peak.cu -- measurement support: the FP32 FMA throughput of the device
// (the denominator of the ALU rooflines of the coordination-number pair
// loops), measured with a kernel of independent FMA chains on every SM.
#include <cuda_runtime.h>

#include <algorithm>

#include "abp.h"
#include "abp_launch.h"

namespace abp {
namespace {

constexpr int kChains = 8;  // independent FMA chains per thread

// Every thread advances kChains chains x <- x b + c for `iters` rounds; the
// chains' sum is stored so that none of the work can be dropped.
__global__ void __launch_bounds__(256) k_fma_peak(float b, float c, int iters, float *out) {
  float x[kChains];
#pragma unroll
  for (int q = 0; q < kChains; ++q) x[q] = (float)(threadIdx.x + q);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int q = 0; q < kChains; ++q) x[q] = __fmaf_rn(x[q], b, c);
  }
  float s = 0.f;
#pragma unroll
  for (int q = 0; q < kChains; ++q) s += x[q];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace
}  // namespace abp

extern "C" abp_status abp_fp32_fma_peak(int device, void *cuda_stream, int iters, double *flops_per_s,
                                        double *seconds) {
  using namespace abp;
  if (!flops_per_s || iters < 1) return record_error(ABP_ERR_INVALID_ARG, "flops_per_s is NULL or iters < 1");
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) return record_error(ABP_ERR_CUDA, "cudaGetDevice failed");
  if (cudaSetDevice(device) != cudaSuccess) return record_error(ABP_ERR_CUDA, "cudaSetDevice failed");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  const int threads = 256, blocks = std::max(1, sms) * 8;
  float *out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  abp_status rc = ABP_OK;
  float ms = 0.f;
  if (cudaMalloc(&out, sizeof(float) * (size_t)blocks * threads) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess) {
    rc = record_error(ABP_ERR_CUDA, "allocation of the measurement buffers failed");
  } else {
    k_fma_peak<<<blocks, threads, 0, st>>>(0.999999f, 1e-6f, std::max(1, iters / 10), out);  // warm-up
    cudaEventRecord(e0, st);
    k_fma_peak<<<blocks, threads, 0, st>>>(0.999999f, 1e-6f, iters, out);
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
      rc = record_error(ABP_ERR_CUDA, "the FMA kernel failed");
    } else {
      cudaEventElapsedTime(&ms, e0, e1);
      const double flops = 2.0 * kChains * (double)iters * (double)blocks * threads;
      *flops_per_s = flops / (ms * 1e-3);
      if (seconds) *seconds = ms * 1e-3;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (out) cudaFree(out);
  cudaSetDevice(prev);
  return rc;
}
