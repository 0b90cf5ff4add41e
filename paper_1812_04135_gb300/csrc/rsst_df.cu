// Double-float kernels (precision RSST_FP64_DF): the state is stored as
// float32 pairs (hi, lo) in the padded layout (8 bytes per value, like
// float64) and the fused stage kernel computes in double-float on the
// float32 pipe.  Tile structure as in the float64 kernel (rsst_fp64.cu).
#include "rsst_common.cuh"
#include "rsst_internal.h"
#include "rsst_attr.h"
#include "rsst_math_df.cuh"

namespace rsst {

__device__ __forceinline__ df ld_df(const float2* p, int64_t i) {
  const float2 v = p[i];
  return {v.x, v.y};
}
__device__ __forceinline__ void st_df(float2* p, int64_t i, df v) { p[i] = make_float2(v.hi, v.lo); }

// Store a cell and the edge ghosts it is the image of (wrap, or mirror with
// the normal momentum negated and the background difference added).
template <int NV>
__device__ __forceinline__ void store_ghosts_df(float2* __restrict__ out, const Geom& g, const Phys& p,
                                                const double* __restrict__ bg, int bg_len, int i, int j, int k,
                                                const df (&u)[NV]) {
  constexpr int ND = NV - 2;
  const int64_t fs = g.fstride;
  const int64_t o = pidx(g, i, j, k);
#pragma unroll
  for (int v = 0; v < NV; ++v) st_df(out, v * fs + o, u[v]);
  const int c[3] = {i, j, k};
#pragma unroll
  for (int d = 0; d < ND; ++d) {
    const int n = g.n[d], cd = c[d];
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      const bool hit = side == 0 ? (cd < RSST_G) : (cd >= n - RSST_G);
      if (!hit) continue;
      df w[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) w[v] = u[v];
      int gp;
      if (p.bc[d] == RSST_BC_PERIODIC) {
        gp = side == 0 ? cd + n : cd - n;
      } else {
        gp = side == 0 ? -1 - cd : 2 * n - 1 - cd;
        w[1 + d] = -w[1 + d];
        if (bg != nullptr && d == p.vertical) {
          w[0] = w[0] + df_from(bg[gp + RSST_G] - bg[cd + RSST_G]);
          w[NV - 1] = w[NV - 1] + df_from(bg[bg_len + gp + RSST_G] - bg[bg_len + cd + RSST_G]);
        }
      }
      const int ii = d == 0 ? gp : i, jj = d == 1 ? gp : j, kk = d == 2 ? gp : k;
      const int64_t og = pidx(g, ii, jj, kk);
#pragma unroll
      for (int v = 0; v < NV; ++v) st_df(out, v * fs + og, w[v]);
    }
  }
}

__device__ __forceinline__ df warp_max_df(df x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const df y = {__shfl_xor_sync(0xffffffffu, x.hi, o), __shfl_xor_sync(0xffffffffu, x.lo, o)};
    if (df_lt(x, y)) x = y;
  }
  return x;
}

// Block maximum of non-negative double-floats, one float64 atomicMax.
template <int NT>
__device__ __forceinline__ void block_max_df(df x, double* dst, df* sred) {
  x = warp_max_df(x);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sred[wid] = x;
  __syncthreads();
  if (wid == 0) {
    df y = lane < NT / 32 ? sred[lane] : df_make(0.0f);
    y = warp_max_df(y);
    if (lane == 0 && df_pos(y))
      atomicMax(reinterpret_cast<unsigned long long*>(dst), (unsigned long long)__double_as_longlong(df_to(y)));
  }
}

template <int NDIM, int BX, int BY, int BZ, int NT>
struct TileCfgDF {
  static constexpr int NV = NDIM + 2;
  static constexpr int HX = 2, HY = NDIM >= 2 ? 2 : 0, HZ = NDIM >= 3 ? 2 : 0;
  static constexpr int SX = BX + 2 * HX, SY = BY + 2 * HY, SZ = BZ + 2 * HZ;
  static constexpr int SCELLS = SX * SY * SZ;
  static constexpr int NCELL = BX * BY * BZ;
  static constexpr int CPT = (NCELL + NT - 1) / NT;
  static constexpr int FX = (BX + 1) * BY * BZ;
  static constexpr int FY = NDIM >= 2 ? BX * (BY + 1) * BZ : 0;
  static constexpr int FZ = NDIM >= 3 ? BX * BY * (BZ + 1) : 0;
  static constexpr int FMAX = FX > FY ? (FX > FZ ? FX : FZ) : (FY > FZ ? FY : FZ);
  // each cell's MC slope along the current axis, once per cell (cells -1 .. B
  // along that axis), when it fits beside the tile with room for several CTAs
  static constexpr int EX0 = (BX + 2) * BY * BZ, EX1 = NDIM >= 2 ? BX * (BY + 2) * BZ : 0;
  static constexpr int EX2 = NDIM >= 3 ? BX * BY * (BZ + 2) : 0;
  static constexpr int EXM = EX0 > EX1 ? (EX0 > EX2 ? EX0 : EX2) : (EX1 > EX2 ? EX1 : EX2);
  static constexpr bool SLOPES = NDIM <= 2 || sizeof(df) * (size_t)NV * (SCELLS + FMAX + EXM) <= (size_t)76 * 1024;
  static constexpr int SEMAX = SLOPES ? EXM : 0;
  static constexpr size_t SMEM = sizeof(df) * ((size_t)NV * (SCELLS + FMAX + SEMAX) + 64);
};

template <int NDIM, int BX, int BY, int BZ, int NT, int D>
__device__ __forceinline__ void face_pass_df(const df* __restrict__ su, df* __restrict__ sf, df* __restrict__ ss,
                                             const PhysDF& p, const Geom& g, int i0, int j0, int k0,
                                             df (&dU)[TileCfgDF<NDIM, BX, BY, BZ, NT>::CPT][NDIM + 2]) {
  using C = TileCfgDF<NDIM, BX, BY, BZ, NT>;
  constexpr int NV = C::NV;
  constexpr int EX = BX + (D == 0), EY = BY + (D == 1), EZ = BZ + (D == 2);
  constexpr int NF = EX * EY * EZ;
  constexpr int STRIDE = D == 0 ? 1 : (D == 1 ? C::SX : C::SX * C::SY);
  constexpr int XX = BX + 2 * (D == 0), YY = BY + 2 * (D == 1), ZZ = BZ + 2 * (D == 2);
  constexpr int NE = XX * YY * ZZ;
  const int baseD = D == 0 ? i0 : (D == 1 ? j0 : k0);
  if constexpr (C::SLOPES) {
    for (int e = threadIdx.x; e < NE; e += NT) {
      const int ex = e % XX;
      const int t = e / XX;
      const int ey = t % YY;
      const int ez = t / YY;
      const int s0 = (ez - (D == 2) + C::HZ) * C::SX * C::SY + (ey - (D == 1) + C::HY) * C::SX + (ex - (D == 0) + C::HX);
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const df* sv = su + v * C::SCELLS + s0;
        ss[v * C::SEMAX + e] = mc_df(sv[0] - sv[-STRIDE], sv[STRIDE] - sv[0]);
      }
    }
    __syncthreads();
  }
  for (int fid = threadIdx.x; fid < NF; fid += NT) {
    const int fx = fid % EX;
    const int t = fid / EX;
    const int fy = t % EY;
    const int fz = t / EY;
    const int fD = D == 0 ? fx : (D == 1 ? fy : fz);
    const bool valid = (i0 + fx <= g.n[0] - (D == 0 ? 0 : 1)) && (NDIM < 2 || j0 + fy <= g.n[1] - (D == 1 ? 0 : 1)) &&
                       (NDIM < 3 || k0 + fz <= g.n[2] - (D == 2 ? 0 : 1)) && (baseD + fD <= g.n[D]);
    if (!valid) continue;
    const int s0 = (fz + C::HZ) * C::SX * C::SY + (fy + C::HY) * C::SX + (fx + C::HX);
    df qL[NV], qR[NV];
    if constexpr (C::SLOPES) {
      constexpr int STRIDE_E = D == 0 ? 1 : (D == 1 ? XX : XX * YY);
      const int er = ((fz + (D == 2)) * YY + (fy + (D == 1))) * XX + (fx + (D == 0));
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const df* sv = su + v * C::SCELLS + s0;
        qL[v] = sv[-STRIDE] + scale(ss[v * C::SEMAX + er - STRIDE_E], 0.5f);
        qR[v] = sv[0] - scale(ss[v * C::SEMAX + er], 0.5f);
      }
    } else {
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const df* sv = su + v * C::SCELLS + s0;
        const df um2 = sv[-2 * STRIDE], um1 = sv[-STRIDE], u0 = sv[0], up1 = sv[STRIDE];
        const df dm = um1 - um2, d0 = u0 - um1, dp = up1 - u0;
        qL[v] = um1 + scale(mc_df(dm, d0), 0.5f);
        qR[v] = u0 - scale(mc_df(d0, dp), 0.5f);
      }
    }
    df F[NV];
    llf_flux_df<NV, D>(qL, qR, p, F);
#pragma unroll
    for (int v = 0; v < NV; ++v) sf[v * C::FMAX + fid] = F[v];
  }
  __syncthreads();
  const df idx = p.inv_dx[D];
#pragma unroll
  for (int c = 0; c < C::CPT; ++c) {
    const int cell = threadIdx.x + c * NT;
    if (cell >= C::NCELL) break;
    const int cx = cell % BX;
    const int t = cell / BX;
    const int cy = t % BY;
    const int cz = t / BY;
    const int flo = (cz * EY + cy) * EX + cx;
    const int fhi = flo + (D == 0 ? 1 : (D == 1 ? EX : EX * EY));
#pragma unroll
    for (int v = 0; v < NV; ++v) dU[c][v] = dU[c][v] - (sf[v * C::FMAX + fhi] - sf[v * C::FMAX + flo]) * idx;
  }
  __syncthreads();
}

struct DFArgs {
  const float2* in;
  const float2* base;
  float2* out;
  Geom g;
  Phys p;
  PhysDF q;
  const double* bg;
  int bg_len;
  double* scal;
  unsigned int* flag;
  int slot, stage;
  double dt_fixed;
};

template <int NDIM, int BX, int BY, int BZ, int NT>
__global__ void __launch_bounds__(NT) stage_df_kernel(const DFArgs a) {
  using C = TileCfgDF<NDIM, BX, BY, BZ, NT>;
  constexpr int NV = C::NV;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  df* su = reinterpret_cast<df*>(smem_raw);
  df* sf = su + NV * C::SCELLS;
  df* ss = sf + NV * C::FMAX;  // slopes, when they fit
  df* sred = ss + NV * C::SEMAX;
  double* sdt = reinterpret_cast<double*>(sred + 32);
  const Geom& g = a.g;
  const PhysDF& p = a.q;
  const int i0 = blockIdx.x * BX, j0 = blockIdx.y * BY, k0 = blockIdx.z * BZ;
  if (threadIdx.x == 0) {
    const double dt = a.dt_fixed > 0.0 ? a.dt_fixed : a.p.cfl / a.scal[a.slot];
    *sdt = dt;
    if (a.stage == 1 && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0) {
      a.scal[a.slot ^ 1] = 0.0;
      a.scal[2] = dt;
      a.scal[3] += dt;
    }
  }
  for (int id = threadIdx.x; id < NV * C::SCELLS; id += NT) {
    const int v = id / C::SCELLS;
    const int r = id - v * C::SCELLS;
    const int lx = r % C::SX;
    const int t = r / C::SX;
    const int ly = t % C::SY;
    const int lz = t / C::SY;
    const int gi = i0 + lx - C::HX, gj = j0 + ly - C::HY, gk = k0 + lz - C::HZ;
    df val = {0.0f, 0.0f};
    if (gi <= g.n[0] + 1 && (NDIM < 2 || gj <= g.n[1] + 1) && (NDIM < 3 || gk <= g.n[2] + 1))
      val = ld_df(a.in, v * g.fstride + pidx(g, gi, gj, gk));
    su[id] = val;
  }
  __syncthreads();
  const df dt = df_from(*sdt);

  df dU[C::CPT][NV];
#pragma unroll
  for (int c = 0; c < C::CPT; ++c)
#pragma unroll
    for (int v = 0; v < NV; ++v) dU[c][v] = {0.0f, 0.0f};
  face_pass_df<NDIM, BX, BY, BZ, NT, 0>(su, sf, ss, p, g, i0, j0, k0, dU);
  if constexpr (NDIM >= 2) face_pass_df<NDIM, BX, BY, BZ, NT, 1>(su, sf, ss, p, g, i0, j0, k0, dU);
  if constexpr (NDIM >= 3) face_pass_df<NDIM, BX, BY, BZ, NT, 2>(su, sf, ss, p, g, i0, j0, k0, dU);

  df rmax = {0.0f, 0.0f};
  bool ok_all = true;
#pragma unroll
  for (int c = 0; c < C::CPT; ++c) {
    const int cell = threadIdx.x + c * NT;
    if (cell >= C::NCELL) break;
    const int cx = cell % BX;
    const int t = cell / BX;
    const int cy = t % BY;
    const int cz = t / BY;
    const int i = i0 + cx, j = j0 + cy, k = k0 + cz;
    if (i >= g.n[0] || (NDIM >= 2 && j >= g.n[1]) || (NDIM >= 3 && k >= g.n[2])) continue;
    const int s0 = (cz + C::HZ) * C::SX * C::SY + (cy + C::HY) * C::SX + (cx + C::HX);
    df q[NV], L[NV], u[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      q[v] = su[v * C::SCELLS + s0];
      L[v] = dU[c][v];
    }
    rsst_rhs_df<NV>(q, L, p);
    if (a.stage == 1) {
#pragma unroll
      for (int v = 0; v < NV; ++v) u[v] = q[v] + dt * L[v];
    } else {
      const int64_t o = pidx(g, i, j, k);
#pragma unroll
      for (int v = 0; v < NV; ++v) u[v] = scale(ld_df(a.base, v * g.fstride + o) + (q[v] + dt * L[v]), 0.5f);
      bool ok;
      const df r = cfl_rate_df<NV>(u, p, ok);
      if (ok && df_lt(rmax, r)) rmax = r;
      ok_all = ok_all && ok;
    }
    store_ghosts_df<NV>(a.out, g, a.p, a.bg, a.bg_len, i, j, k, u);
  }
  if (a.stage == 2) {
    if (!ok_all) atomicOr(a.flag, RSST_FLAG_NONPHYSICAL);
    block_max_df<NT>(rmax, a.scal + (a.slot ^ 1), sred);
  }
}

// ---------------------------------------------------------------------------
// Packing, CFL maximum, sums (double-float storage)
// ---------------------------------------------------------------------------

__global__ void pack_df_kernel(const double* __restrict__ src, float2* __restrict__ dst, Geom g, Phys p,
                               const double* __restrict__ bg, int bg_len) {
  const int nv = g.ndim + 2;
  const int ex = g.n[0] + 2 * RSST_G;
  const int ey = g.ndim >= 2 ? g.n[1] + 2 * RSST_G : 1;
  const int ez = g.ndim >= 3 ? g.n[2] + 2 * RSST_G : 1;
  const int64_t total = (int64_t)ex * ey * ez;
  for (int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; id < total; id += (int64_t)gridDim.x * blockDim.x) {
    const int c[3] = {(int)(id % ex) - RSST_G, g.ndim >= 2 ? (int)((id / ex) % ey) - RSST_G : 0,
                      g.ndim >= 3 ? (int)(id / ((int64_t)ex * ey)) - RSST_G : 0};
    int s[3] = {c[0], c[1], c[2]};
    double sign[3] = {1.0, 1.0, 1.0};
    int vimg = 0, vgh = 0;
    bool vmirror = false;
    for (int d = 0; d < g.ndim; ++d) {
      const int n = g.n[d];
      if (s[d] >= 0 && s[d] < n) continue;
      if (p.bc[d] == RSST_BC_PERIODIC) {
        s[d] = (s[d] + n) % n;
      } else {
        const int img = s[d] < 0 ? -1 - s[d] : 2 * n - 1 - s[d];
        if (d == p.vertical) { vgh = s[d]; vimg = img; vmirror = true; }
        s[d] = img;
        sign[d] = -1.0;
      }
    }
    const int64_t si = ((int64_t)s[2] * g.n[1] + s[1]) * g.n[0] + s[0];
    const int64_t di = pidx(g, c[0], c[1], c[2]);
    for (int v = 0; v < nv; ++v) {
      double w = src[v * g.ncells + si];
      if (v >= 1 && v <= g.ndim) w *= sign[v - 1];
      if (bg != nullptr && vmirror && (v == 0 || v == nv - 1)) {
        const double* row = bg + (v == 0 ? 0 : bg_len);
        w += row[vgh + RSST_G] - row[vimg + RSST_G];
      }
      st_df(dst, v * g.fstride + di, df_from(w));
    }
  }
}

__global__ void unpack_df_kernel(const float2* __restrict__ src, double* __restrict__ dst, Geom g) {
  const int nv = g.ndim + 2;
  for (int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; id < g.ncells; id += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(id % g.n[0]);
    const int j = (int)((id / g.n[0]) % g.n[1]);
    const int k = (int)(id / ((int64_t)g.n[0] * g.n[1]));
    const int64_t o = pidx(g, i, j, k);
    for (int v = 0; v < nv; ++v) dst[v * g.ncells + id] = df_to(ld_df(src, v * g.fstride + o));
  }
}

template <int NV>
__global__ void __launch_bounds__(256) cfl_df_kernel(const float2* __restrict__ U, Geom g, PhysDF p, double* dst,
                                                     unsigned int* flag) {
  __shared__ df sred[32];
  df rmax = {0.0f, 0.0f};
  bool ok_all = true;
  for (int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; id < g.ncells; id += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(id % g.n[0]);
    const int j = (int)((id / g.n[0]) % g.n[1]);
    const int k = (int)(id / ((int64_t)g.n[0] * g.n[1]));
    const int64_t o = pidx(g, i, j, k);
    df q[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) q[v] = ld_df(U, v * g.fstride + o);
    bool ok;
    const df r = cfl_rate_df<NV>(q, p, ok);
    if (ok && df_lt(rmax, r)) rmax = r;
    ok_all = ok_all && ok;
  }
  if (!ok_all) atomicOr(flag, RSST_FLAG_NONPHYSICAL);
  block_max_df<256>(rmax, dst, sred);
}

constexpr int SUM_BLOCKS_DF = 1024;
constexpr int SUM_THREADS_DF = 256;

__global__ void __launch_bounds__(SUM_THREADS_DF) sums_partial_df_kernel(const float2* __restrict__ U, Geom g,
                                                                         double* __restrict__ partial) {
  __shared__ double sh[SUM_THREADS_DF];
  const int nv = g.ndim + 2;
  const int64_t chunk = (g.ncells + SUM_BLOCKS_DF - 1) / SUM_BLOCKS_DF;
  const int64_t lo = blockIdx.x * chunk;
  const int64_t hi = min(g.ncells, lo + chunk);
  for (int v = 0; v < nv; ++v) {
    double acc = 0.0;
    for (int64_t id = lo + threadIdx.x; id < hi; id += SUM_THREADS_DF) {
      const int i = (int)(id % g.n[0]);
      const int j = (int)((id / g.n[0]) % g.n[1]);
      const int k = (int)(id / ((int64_t)g.n[0] * g.n[1]));
      acc += df_to(ld_df(U, v * g.fstride + pidx(g, i, j, k)));
    }
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int s = SUM_THREADS_DF / 2; s > 0; s >>= 1) {
      if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
      __syncthreads();
    }
    if (threadIdx.x == 0) partial[v * SUM_BLOCKS_DF + blockIdx.x] = sh[0];
    __syncthreads();
  }
}

__global__ void __launch_bounds__(SUM_THREADS_DF) sums_final_df_kernel(const double* __restrict__ partial, int nv,
                                                                       double scale_, double* __restrict__ out) {
  __shared__ double sh[SUM_THREADS_DF];
  for (int v = 0; v < nv; ++v) {
    double acc = 0.0;
    for (int b = threadIdx.x; b < SUM_BLOCKS_DF; b += SUM_THREADS_DF) acc += partial[v * SUM_BLOCKS_DF + b];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int s = SUM_THREADS_DF / 2; s > 0; s >>= 1) {
      if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
      __syncthreads();
    }
    if (threadIdx.x == 0) out[v] = sh[0] * scale_;
    __syncthreads();
  }
}

static df split_host(double x) {
  const float h = (float)x;
  return {h, (float)(x - (double)h)};
}

static PhysDF make_physdf(const Phys& p) {
  PhysDF q;
  q.gamma = split_host(p.gamma);
  q.gm1 = split_host(p.gm1);
  q.hgm1 = split_host(p.hgm1);
  q.inv_gm1 = split_host(p.inv_gm1);
  q.inv_xi = split_host(p.inv_xi);
  q.f = split_host(p.f);
  q.inv_cmax4 = split_host(p.inv_cmax4);
  for (int d = 0; d < 3; ++d) {
    q.grav[d] = split_host(p.grav[d]);
    q.inv_dx[d] = split_host(p.inv_dx[d]);
  }
  q.sum_inv_dx = split_host(p.sum_inv_dx);
  q.variant = p.variant;
  q.use_cmax = p.use_cmax;
  q.has_grav = p.has_grav;
  return q;
}

template <int NDIM, int BX, int BY, int BZ, int NT>
static int launch_df(const DFArgs& a, cudaStream_t s) {
  using C = TileCfgDF<NDIM, BX, BY, BZ, NT>;
  auto kern = stage_df_kernel<NDIM, BX, BY, BZ, NT>;
  const size_t smem = C::SMEM + 64;
  static std::atomic<unsigned long long> attr{0};
  if (set_smem_limit_once(kern, smem, attr) != cudaSuccess) {
    rsst_set_error("cudaFuncSetAttribute failed for the double-float stage kernel");
    return RSST_ECUDA;
  }
  dim3 grid((a.g.n[0] + BX - 1) / BX, NDIM >= 2 ? (a.g.n[1] + BY - 1) / BY : 1, NDIM >= 3 ? (a.g.n[2] + BZ - 1) / BZ : 1);
  kern<<<grid, NT, smem, s>>>(a);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    rsst_set_error("double-float stage kernel launch: %s", cudaGetErrorString(e));
    return RSST_ECUDA;
  }
  return RSST_OK;
}

}  // namespace rsst

using namespace rsst;

int rsst_launch_stage_df(const StageArgs<float2>& sa, cudaStream_t s) {
  DFArgs a;
  a.in = sa.in;
  a.base = sa.base;
  a.out = sa.out;
  a.g = sa.g;
  a.p = sa.p;
  a.q = make_physdf(sa.p);
  a.bg = sa.bg;
  a.bg_len = sa.bg_len;
  a.scal = sa.scal;
  a.flag = sa.flag;
  a.slot = sa.slot;
  a.stage = sa.stage;
  a.dt_fixed = sa.dt_fixed;
  switch (a.g.ndim) {
    case 1:
      if (a.g.n[0] <= RSST_SMALL_1D) return launch_df<1, 16, 1, 1, 32>(a, s);
      return launch_df<1, 256, 1, 1, 256>(a, s);
    case 2: return launch_df<2, 32, 8, 1, 288>(a, s);  // 9 warps: each face pass in one round
    case 3: return launch_df<3, 8, 8, 4, 320>(a, s);  // 10 warps: each face pass in one round
  }
  rsst_set_error("ndim must be 1, 2 or 3");
  return RSST_EINVAL;
}

static int grid_df(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b > 152 * 16) b = 152 * 16;
  return (int)(b < 1 ? 1 : b);
}

static int err_df(const char* what) {
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    rsst_set_error("%s launch: %s", what, cudaGetErrorString(e));
    return RSST_ECUDA;
  }
  return RSST_OK;
}

int rsst_launch_pack_df(const double* src, float2* dst, const Geom& g, const Phys& p, const double* bg, int bg_len,
                        cudaStream_t s) {
  const int64_t total = (int64_t)(g.n[0] + 4) * (g.ndim >= 2 ? g.n[1] + 4 : 1) * (g.ndim >= 3 ? g.n[2] + 4 : 1);
  pack_df_kernel<<<grid_df(total), 256, 0, s>>>(src, dst, g, p, bg, bg_len);
  return err_df("pack (double-float)");
}

int rsst_launch_unpack_df(const float2* src, double* dst, const Geom& g, cudaStream_t s) {
  unpack_df_kernel<<<grid_df(g.ncells), 256, 0, s>>>(src, dst, g);
  return err_df("unpack (double-float)");
}

int rsst_launch_cfl_df(const float2* U, const Geom& g, const Phys& p, double* slot_ptr, unsigned int* flag,
                       cudaStream_t s) {
  const PhysDF q = make_physdf(p);
  const int gb = grid_df(g.ncells);
  switch (g.ndim) {
    case 1: cfl_df_kernel<3><<<gb, 256, 0, s>>>(U, g, q, slot_ptr, flag); break;
    case 2: cfl_df_kernel<4><<<gb, 256, 0, s>>>(U, g, q, slot_ptr, flag); break;
    default: cfl_df_kernel<5><<<gb, 256, 0, s>>>(U, g, q, slot_ptr, flag); break;
  }
  return err_df("cfl (double-float)");
}

int rsst_launch_sums_df(const float2* U, const Geom& g, double* partial, double* out, double scale_, cudaStream_t s) {
  sums_partial_df_kernel<<<SUM_BLOCKS_DF, SUM_THREADS_DF, 0, s>>>(U, g, partial);
  const int rc = err_df("sums (double-float)");
  if (rc) return rc;
  sums_final_df_kernel<<<1, SUM_THREADS_DF, 0, s>>>(partial, g.ndim + 2, scale_, out);
  return err_df("sums final (double-float)");
}
