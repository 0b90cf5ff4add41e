// Float64 FMA throughput of the current device, measured: the denominator of
// the float64 stage kernels' arithmetic roofline (the float64 step is bound
// by the float64 pipe, not by HBM).  Each thread runs eight independent
// chains of dependent FMAs (enough in flight to fill the pipe), on a grid of
// 8 CTAs of 256 threads per SM; the launch is timed with CUDA events after
// one warm-up launch.
#include "rsst_internal.h"

namespace rsst {

__global__ void __launch_bounds__(256) fp64_fma_kernel(double* out, int iters, double a, double b) {
  double x[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) x[c] = 1e-3 * (threadIdx.x + 7 * c);
#pragma unroll 1
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int c = 0; c < 8; ++c) x[c] = fma(x[c], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < 8; ++c) s += x[c];
  if (s == 12345.6789) out[0] = s;  // keeps the chains live; never true for these inputs
}

}  // namespace rsst

extern "C" int rsst_fp64_fma_peak(int32_t iters, double* tflops, double* ms) {
  if (iters < 1 || !tflops) {
    rsst_set_error("rsst_fp64_fma_peak: need iters >= 1 and an output");
    return RSST_EINVAL;
  }
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    rsst_set_error("rsst_fp64_fma_peak: cannot query the device");
    return RSST_ECUDA;
  }
  double* out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaMalloc((void**)&out, sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    rsst_set_error("rsst_fp64_fma_peak: allocation failed");
    return RSST_ENOMEM;
  }
  int rc = RSST_OK;
  float t = 0.0f;
  const int blocks = 8 * sms, threads = 256;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = RSST_ECUDA;
  if (rc == RSST_OK) {
    rsst::fp64_fma_kernel<<<blocks, threads>>>(out, iters, 0.999999, 1e-9);  // warm-up
    cudaEventRecord(e0);
    rsst::fp64_fma_kernel<<<blocks, threads>>>(out, iters, 0.999999, 1e-9);
    cudaEventRecord(e1);
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&t, e0, e1) != cudaSuccess ||
        cudaGetLastError() != cudaSuccess)
      rc = RSST_ECUDA;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(out);
  if (rc != RSST_OK) {
    rsst_set_error("rsst_fp64_fma_peak: the probe launch failed");
    return rc;
  }
  const double flops = 2.0 * 32.0 * iters * (double)threads * blocks;
  *tflops = flops / (t * 1e-3) / 1e12;
  if (ms) *ms = t;
  return RSST_OK;
}
