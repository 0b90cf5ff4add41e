// Device self-test of the float64 helpers the kernels use instead of the
// compiler's sequences: the Newton-Raphson reciprocal against CUDA's
// correctly rounded division (largest error in ulps), the integer-pipe MC
// limiter against the direct float64 form of the same definition, and the
// c_tot square root against CUDA's sqrt (largest relative error, plus its
// zero, subnormal and negative cases).
#include <cmath>
#include <cstring>

#include "rsst_internal.h"
#include "rsst_math_fp64.cuh"

namespace rsst {

__device__ __forceinline__ double mc_direct(double a, double b) {
  const double aa = 2.0 * fabs(a), bb = 2.0 * fabs(b), cc = 0.5 * fabs(a + b);
  const double s = (aa <= bb && aa <= cc) ? 2.0 * a : ((bb <= cc) ? 2.0 * b : 0.5 * (a + b));
  return (a * b > 0.0) ? s : 0.0;
}

// SplitMix64 stream for the test inputs.
__device__ __forceinline__ unsigned long long smix(unsigned long long z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void selftest_kernel(int n, unsigned long long* max_ulp, unsigned int* mc_bad,
                                unsigned long long* sqrt_rel_bits) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const unsigned long long r1 = smix(2 * (unsigned long long)i), r2 = smix(2 * (unsigned long long)i + 1);
  const double u1 = (double)(r1 >> 11) * (1.0 / 9007199254740992.0);
  const double u2 = (double)(r2 >> 11) * (1.0 / 9007199254740992.0);
  // reciprocal over densities 1e-6 .. 1e6
  const double x = exp2(-20.0 + 40.0 * u1);
  const long long got = __double_as_longlong(rcp_nr(x)), want = __double_as_longlong(1.0 / x);
  const unsigned long long ulp = (unsigned long long)(got > want ? got - want : want - got);
  atomicMax(max_ulp, ulp);
  // MC limiter: random signs and magnitudes, exact zeros and ties
  double a = (u1 - 0.5) * exp2(-30.0 + 60.0 * u2), b = (u2 - 0.5) * exp2(-30.0 + 60.0 * u1);
  const int mode = i & 7;
  if (mode == 1) b = a;            // equal slopes
  if (mode == 2) b = 3.0 * a;      // 2|a| == |a+b|/2
  if (mode == 3) a = 3.0 * b;      // 2|b| == |a+b|/2
  if (mode == 4) a = 0.0;
  if (mode == 5) b = -a;
  if (__double_as_longlong(mc_slope(a, b)) != __double_as_longlong(mc_direct(a, b)) &&
      !(mc_slope(a, b) == 0.0 && mc_direct(a, b) == 0.0))
    atomicAdd(mc_bad, 1u);
  // c_tot square root over 1e-60 .. 1e60, exact squares and powers of two
  double xs = exp2(-200.0 + 400.0 * u2);
  if (mode == 6) xs = exp2((double)((int)(u1 * 400.0) - 200));
  if (mode == 7) xs = (1.0 + u1) * (1.0 + u1);
  const double rel = fabs(sqrt_ctot(xs) - sqrt(xs)) / sqrt(xs);
  atomicMax(sqrt_rel_bits, (unsigned long long)__double_as_longlong(rel));  // non-negative: bits order as values
  // the float-pair square root of the LLF speed, read back as s + c
  float ps, pc;
  sqrt_pair(xs, ps, pc);
  const double prel = fabs(((double)ps + (double)pc) - sqrt(xs)) / sqrt(xs);
  atomicMax(sqrt_rel_bits, (unsigned long long)__double_as_longlong(prel));
  if (i == 0) {
    float z0, z1, s0, s1, n0, n1, q0, q1;
    sqrt_pair(0.0, z0, z1);
    sqrt_pair(4.9e-324, s0, s1);
    sqrt_pair(-1.0, n0, n1);
    sqrt_pair(__longlong_as_double(0x7ff8000000000000ll), q0, q1);
    const bool specials = sqrt_ctot(0.0) == 0.0 && sqrt_ctot(4.9e-324) == 0.0 && isnan(sqrt_ctot(-1.0)) &&
                          z0 == 0.0f && z1 == 0.0f && s0 == 0.0f && s1 == 0.0f && isnan(n0) && isnan(q0) &&
                          f2d_bits(1.5f) == 1.5 && f2d_bits(-0.25f) == -0.25 && f2d_bits(0.0f) == 0.0 &&
                          f2d_bits(3.0e-39f) == 0.0 && isinf(f2d_bits(__int_as_float(0x7f800000)));
    if (!specials) atomicAdd(mc_bad, 1u << 20);
  }
}

}  // namespace rsst

extern "C" int rsst_math_selftest(int32_t n, double* rcp_max_ulp, int32_t* mc_mismatches, double* sqrt_max_rel) {
  if (n < 1 || !rcp_max_ulp || !mc_mismatches || !sqrt_max_rel) {
    rsst_set_error("rsst_math_selftest: bad arguments");
    return RSST_EINVAL;
  }
  unsigned long long* d_ulp = nullptr;  // [0] rcp ulps, [1] sqrt relative error bits
  unsigned int* d_bad = nullptr;
  if (cudaMalloc((void**)&d_ulp, 2 * sizeof(*d_ulp)) != cudaSuccess || cudaMalloc((void**)&d_bad, sizeof(*d_bad)) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(d_ulp);
    rsst_set_error("rsst_math_selftest: allocation failed");
    return RSST_ENOMEM;
  }
  if (cudaMemset(d_ulp, 0, 2 * sizeof(*d_ulp)) != cudaSuccess || cudaMemset(d_bad, 0, sizeof(*d_bad)) != cudaSuccess) {
    cudaFree(d_ulp);
    cudaFree(d_bad);
    rsst_set_error("rsst_math_selftest: memset failed");
    return RSST_ECUDA;
  }
  rsst::selftest_kernel<<<(n + 255) / 256, 256>>>(n, d_ulp, d_bad, d_ulp + 1);
  unsigned long long ulp[2] = {0, 0};
  unsigned int bad = 0;
  const cudaError_t e1 = cudaMemcpy(ulp, d_ulp, sizeof ulp, cudaMemcpyDeviceToHost);
  const cudaError_t e2 = cudaMemcpy(&bad, d_bad, sizeof bad, cudaMemcpyDeviceToHost);
  cudaFree(d_ulp);
  cudaFree(d_bad);
  if (e1 != cudaSuccess || e2 != cudaSuccess) {
    rsst_set_error("rsst_math_selftest: %s", cudaGetErrorString(e1 != cudaSuccess ? e1 : e2));
    return RSST_ECUDA;
  }
  *rcp_max_ulp = (double)ulp[0];
  *mc_mismatches = (int32_t)bad;
  double rel;
  memcpy(&rel, &ulp[1], sizeof rel);
  *sqrt_max_rel = rel;
  return RSST_OK;
}
