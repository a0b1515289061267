// The FP32 FMA throughput of the device, measured: the denominator of the tick
// kernels' ALU roofline.  Every resident warp runs kChains independent FMA chains
// (enough to hide the FMA latency) for a fixed number of iterations; the flop
// count over the CUDA-event time of the launch is the device's sustained FP32
// rate at the clocks it ran at.
#include <cuda_runtime.h>

#include <string>

#include "internal.h"

namespace mpmi {

constexpr int kChains = 8;
constexpr int kPeakBlock = 256;

__global__ void __launch_bounds__(kPeakBlock) ffma_loop(int iters, float a, float b, float* sink) {
  float v[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) v[c] = (float)(threadIdx.x + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) v[c] = __fmaf_rn(v[c], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += v[c];
  // a store that never happens for the arguments the host passes, but the
  // compiler cannot know that
  if (s == 1234.5f) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace mpmi

using namespace mpmi;

extern "C" int mpmi_measure_fp32_peak(int32_t device, double seconds, double* tflops_out) {
  if (!tflops_out) return fail(MPMI_E_INVALID_ARG, "measure_fp32_peak: tflops_out is NULL");
  if (!(seconds > 0.0 && seconds <= 10.0))
    return fail(MPMI_E_INVALID_ARG, "measure_fp32_peak: seconds must be in (0, 10]");
  int prev = 0;
  if (cudaGetDevice(&prev) != cudaSuccess || cudaSetDevice(device) != cudaSuccess) {
    cudaGetLastError();
    return fail(MPMI_E_CUDA, "measure_fp32_peak: cudaSetDevice");
  }
  int rc = MPMI_OK;
  float* sink = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  do {
    int sms = 0, nb = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, ffma_loop, kPeakBlock, 0) !=
            cudaSuccess ||
        nb < 1) {
      rc = fail(MPMI_E_CUDA, "measure_fp32_peak: device attributes");
      break;
    }
    const int grid = sms * nb;
    if (cudaMalloc(&sink, sizeof(float) * (size_t)grid * kPeakBlock) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
      rc = fail(MPMI_E_OOM, "measure_fp32_peak: allocation");
      break;
    }
    // calibrate the iteration count on a short launch, then time the real one
    int iters = 1 << 12;
    float ms = 0.f;
    for (int pass = 0; pass < 2; ++pass) {
      cudaEventRecord(e0);
      ffma_loop<<<grid, kPeakBlock>>>(iters, 0.999999f, 1e-7f, sink);
      cudaEventRecord(e1);
      if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) !=
                                                         cudaSuccess) {
        rc = fail(MPMI_E_CUDA, "measure_fp32_peak: launch");
        break;
      }
      if (pass == 0) {
        const double scale = seconds * 1e3 / (ms > 0.01f ? ms : 0.01f);
        const double want = iters * scale;
        iters = want > (double)(1 << 30) ? (1 << 30) : (want < 1024.0 ? 1024 : (int)want);
      }
    }
    if (rc != MPMI_OK) break;
    const double flops = 2.0 * kChains * (double)iters * grid * kPeakBlock;
    *tflops_out = flops / (ms * 1e-3) / 1e12;
  } while (false);
  if (sink) cudaFree(sink);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaGetLastError();
  cudaSetDevice(prev);
  return rc;
}
