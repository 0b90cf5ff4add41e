// Device helpers shared by the float64 and float32 kernels.
#pragma once

#include "rsst_internal.h"

namespace rsst {

// Padded-layout offset of interior cell (i, j, k) (ghosts at -2, -1, n, n+1).
__device__ __forceinline__ int64_t pidx(const Geom& g, int i, int j, int k) {
  return (int64_t)(k + g.gz) * g.plane + (int64_t)(j + g.gy) * g.pitch + (i + g.xoff);
}

__device__ __forceinline__ double warp_max(double x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_xor_sync(0xffffffffu, x, o));
  return x;
}

// Block-wide maximum of non-negative values, then one atomicMax on the bit
// pattern (monotone for non-negative doubles).  All threads must call it.
template <int NT>
__device__ __forceinline__ void block_max_to(double x, double* dst, double* sred) {
  x = warp_max(x);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sred[wid] = x;
  __syncthreads();
  if (wid == 0) {
    double y = lane < NT / 32 ? sred[lane] : 0.0;
    y = warp_max(y);
    if (lane == 0 && y > 0.0)
      atomicMax(reinterpret_cast<unsigned long long*>(dst), (unsigned long long)__double_as_longlong(y));
  }
}

// Store a perturbation-state cell and the edge ghost cells that wrap it or
// mirror it (normal momentum negated).  The perturbation about a background
// is mirrored without a background term: U1(ghost) = mirror(U1(image)).
template <typename T, int NV>
__device__ __forceinline__ void store_mirror_ghosts(T* __restrict__ out, const Geom& g, const Phys& p, int i, int j,
                                                    int k, const T (&u)[NV]) {
  constexpr int ND = NV - 2;
  const int64_t fs = g.fstride;
  const int64_t o = pidx(g, i, j, k);
#pragma unroll
  for (int v = 0; v < NV; ++v) out[v * fs + o] = u[v];
  const int c[3] = {i, j, k};
#pragma unroll
  for (int d = 0; d < ND; ++d) {
    const int n = g.n[d], cd = c[d];
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      const bool hit = side == 0 ? (cd < RSST_G) : (cd >= n - RSST_G);
      if (!hit) continue;
      const bool per = p.bc[d] == RSST_BC_PERIODIC;
      const int gp = per ? (side == 0 ? cd + n : cd - n) : (side == 0 ? -1 - cd : 2 * n - 1 - cd);
      const int ii = d == 0 ? gp : i, jj = d == 1 ? gp : j, kk = d == 2 ? gp : k;
      const int64_t og = pidx(g, ii, jj, kk);
#pragma unroll
      for (int v = 0; v < NV; ++v) out[v * fs + og] = (!per && v == 1 + d) ? -u[v] : u[v];
    }
  }
}

}  // namespace rsst
