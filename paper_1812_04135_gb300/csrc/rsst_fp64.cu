// Float64 kernels of the RSST step: one fused kernel per SSP-RK2 stage
// (Sec. 4.2 steps 2-8 of arXiv:1812.04135), plus state packing, the
// standalone CFL maximum (step 1) and deterministic conservation sums.
//
// Fused stage kernel, one CTA per tile of BX x BY x BZ cells:
//   1. the tile plus two halo layers on every active axis (all fields) is
//      copied from the padded state into shared memory: in 2D and 3D by one
//      cp.async.bulk.tensor of the whole box (x origin on a 16-byte
//      boundary, rows and planes beyond the padded state zero-filled, a
//      bounded mbarrier wait), in 1D (tiles wider than a TMA box) with
//      coalesced loads;
//   2. per axis D, the MC slope of every cell along D is computed once into
//      shared memory (1D/2D tiles and small 3D tiles; larger 3D tiles take
//      the two slopes per face), then every face of the tile gets twice its
//      LLF flux, F(qL) + F(qR) - alpha (qR - qL), from the face states of
//      the two cells beside it; a face shared by two tiles is computed the
//      same way in both, so both get bit-identical values (discrete
//      conservation);
//   3. each cell accumulates -(2F_{+} - 2F_{-}) / (2 dx_D) in registers;
//   4. epilogue per cell: RSST correction, force, RK combine, store, the
//      edge ghost cells the cell is the image of, and in stage 2 the CFL
//      maximum for the next step and the physical-state flag.
#include <cstdio>

#include "rsst_common.cuh"
#include "rsst_internal.h"
#include "rsst_attr.h"
#include "rsst_math_fp64.cuh"
#include "rsst_tma.cuh"

namespace rsst {

// Store a cell and the edge ghost cells that mirror or wrap it.
template <int NV>
__device__ __forceinline__ void store_with_ghosts(double* __restrict__ out, const Geom& g,
                                                  const Phys& p, const double* __restrict__ bg,
                                                  int bg_len, int i, int j, int k,
                                                  const double (&u)[NV]) {
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
      int gp;
      double w[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) w[v] = u[v];
      if (p.bc[d] == RSST_BC_PERIODIC) {
        gp = side == 0 ? cd + n : cd - n;
      } else {
        gp = side == 0 ? -1 - cd : 2 * n - 1 - cd;
        w[1 + d] = -w[1 + d];
        if (bg != nullptr && d == p.vertical) {
          const double* rho0 = bg;
          const double* e0 = bg + bg_len;
          w[0] += rho0[gp + RSST_G] - rho0[cd + RSST_G];
          w[NV - 1] += e0[gp + RSST_G] - e0[cd + RSST_G];
        }
      }
      const int ii = d == 0 ? gp : i, jj = d == 1 ? gp : j, kk = d == 2 ? gp : k;
      const int64_t og = pidx(g, ii, jj, kk);
#pragma unroll
      for (int v = 0; v < NV; ++v) out[v * fs + og] = w[v];
    }
  }
}

template <int NDIM, int BX, int BY, int BZ, int NT>
struct TileCfg {
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
  // Tiles keep each cell's MC slope along the current axis in shared memory
  // (cells -1 .. B along that axis), computed once per cell instead of once
  // per face side, when the slope array still leaves room for several CTAs
  // per SM; larger 3D tiles recompute them per face.
  static constexpr int EX0 = (BX + 2) * BY * BZ, EX1 = NDIM >= 2 ? BX * (BY + 2) * BZ : 0;
  static constexpr int EX2 = NDIM >= 3 ? BX * BY * (BZ + 2) : 0;
  static constexpr int EXM = EX0 > EX1 ? (EX0 > EX2 ? EX0 : EX2) : (EX1 > EX2 ? EX1 : EX2);
  static constexpr bool SLOPES =
      NDIM <= 2 || sizeof(double) * (size_t)NV * (SCELLS + FMAX + EXM) <= (size_t)76 * 1024;
  static constexpr int SEMAX = SLOPES ? EXM : 0;
  // halo tile, faces, slopes, the block reduction's 64 doubles, and two
  // mbarriers (the tile copy; the failure-detection test wait)
  static constexpr size_t SMEM = sizeof(double) * (size_t)NV * (SCELLS + FMAX + SEMAX) + 64 * sizeof(double) + 16;
  static constexpr uint32_t TILE_BYTES = (uint32_t)(sizeof(double) * NV * SCELLS);
  static_assert(NDIM == 1 || (SX <= 256 && SY <= 256 && SZ <= 256), "TMA box dimensions are at most 256");
  static_assert((SX * sizeof(double)) % 16 == 0 && (HX * sizeof(double)) % 16 == 0,
                "the box's row bytes and the x origin (interior x0 - HX) stay on 16-byte boundaries");
};

// Faces along axis D of the tile: index space (BX + [D==0]) x (BY + [D==1]) x (BZ + [D==2]).
template <int NDIM, int BX, int BY, int BZ, int NT, int D, bool CV>
__device__ __forceinline__ void face_pass(const double* __restrict__ su, double* __restrict__ sf,
                                          double* __restrict__ ss, const Phys& p, const Geom& g, int i0, int j0,
                                          int k0, double (&dU)[TileCfg<NDIM, BX, BY, BZ, NT>::CPT][NDIM + 2]) {
  using C = TileCfg<NDIM, BX, BY, BZ, NT>;
  constexpr int NV = C::NV;
  constexpr int EX = BX + (D == 0), EY = BY + (D == 1), EZ = BZ + (D == 2);
  constexpr int NF = EX * EY * EZ;
  constexpr int STRIDE = D == 0 ? 1 : (D == 1 ? C::SX : C::SX * C::SY);
  // slope cells: tile coordinates -1 .. B along D, 0 .. B-1 across
  constexpr int XX = BX + 2 * (D == 0), YY = BY + 2 * (D == 1), ZZ = BZ + 2 * (D == 2);
  constexpr int NE = XX * YY * ZZ;
  const int nD = g.n[D];
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
        const double* sv = su + v * C::SCELLS + s0;
        const double um = sv[-STRIDE], u0 = sv[0], up = sv[STRIDE];
        ss[v * C::SEMAX + e] = mc_slope(u0 - um, up - u0);
      }
    }
    __syncthreads();
  }
  for (int fid = threadIdx.x; fid < NF; fid += NT) {
    const int fx = fid % EX;
    const int t = fid / EX;
    const int fy = t % EY;
    const int fz = t / EY;
    // face fD - 1/2 of tile cell (fx, fy, fz); valid if its cells exist
    const int fD = D == 0 ? fx : (D == 1 ? fy : fz);
    const bool valid = (i0 + fx <= g.n[0] - (D == 0 ? 0 : 1)) && (NDIM < 2 || j0 + fy <= g.n[1] - (D == 1 ? 0 : 1)) &&
                       (NDIM < 3 || k0 + fz <= g.n[2] - (D == 2 ? 0 : 1)) && (baseD + fD <= nD);
    if (!valid) continue;
    // shared-memory index of the cell right of the face
    const int s0 = (fz + C::HZ) * C::SX * C::SY + (fy + C::HY) * C::SX + (fx + C::HX);
    double qL[NV], qR[NV];
    if constexpr (C::SLOPES) {
      // slope index of the cell right of the face; the left one is STRIDE_E before
      constexpr int STRIDE_E = D == 0 ? 1 : (D == 1 ? XX : XX * YY);
      const int er = ((fz + (D == 2)) * YY + (fy + (D == 1))) * XX + (fx + (D == 0));
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const double* sv = su + v * C::SCELLS + s0;
        qL[v] = fma(0.5, ss[v * C::SEMAX + er - STRIDE_E], sv[-STRIDE]);
        qR[v] = fma(-0.5, ss[v * C::SEMAX + er], sv[0]);
      }
    } else {
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const double* sv = su + v * C::SCELLS + s0;
        const double um2 = sv[-2 * STRIDE], um1 = sv[-STRIDE], u0 = sv[0], up1 = sv[STRIDE];
        const double sl = mc_slope(um1 - um2, u0 - um1);
        const double sr = mc_slope(u0 - um1, up1 - u0);
        qL[v] = um1 + 0.5 * sl;
        qR[v] = u0 - 0.5 * sr;
      }
    }
    double F[NV];  // twice the face flux
    llf_flux_x2<NV, D, CV>(qL, qR, p, F);
#pragma unroll
    for (int v = 0; v < NV; ++v) sf[v * C::FMAX + fid] = F[v];
  }
  __syncthreads();
  const double idx = 0.5 * p.inv_dx[D];  // the faces hold 2 F
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
    for (int v = 0; v < NV; ++v) dU[c][v] -= (sf[v * C::FMAX + fhi] - sf[v * C::FMAX + flo]) * idx;
  }
  __syncthreads();
}

template <int NDIM, int BX, int BY, int BZ, int NT, bool TMA, bool CV>
__global__ void __launch_bounds__(NT, NDIM == 3 ? 3 : 0)
    stage_fp64_kernel(const __grid_constant__ CUtensorMap tin, const StageArgs<double> a) {
  using C = TileCfg<NDIM, BX, BY, BZ, NT>;
  constexpr int NV = C::NV;
  extern __shared__ __align__(128) double smem[];
  double* su = smem;
  double* sf = smem + NV * C::SCELLS;
  double* ss = sf + NV * C::FMAX;  // slopes (1D/2D tiles)
  double* sred = ss + NV * C::SEMAX;
  const Geom& g = a.g;
  const Phys& p = a.p;
  const int i0 = blockIdx.x * BX, j0 = blockIdx.y * BY, k0 = blockIdx.z * BZ;

  // 1. halo tile -> shared memory
  if constexpr (TMA) {
    // The box of the padded state [nvar][pz][py][pitch] whose first cell is
    // interior (i0 - HX, j0 - HY, k0 - HZ): padded x i0 + xoff - HX, padded
    // y j0 (HY = gy), padded z k0 (HZ = gz).
    uint64_t* bar = reinterpret_cast<uint64_t*>(sred + 64);
    uint64_t* test_bar = bar + 1;
    const bool stall = a.stall_ns > 0;
    if (threadIdx.x == 0) {
      mbar_init(bar, 1);
      if (stall) mbar_init(test_bar, 1);
      fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      fence_proxy_async_smem();
      mbar_expect_tx(bar, C::TILE_BYTES);
      if constexpr (NDIM == 2) tma_load_3d(su, &tin, bar, i0 + g.xoff - C::HX, j0, 0);
      else tma_load_4d(su, &tin, bar, i0 + g.xoff - C::HX, j0, k0, 0);
      // failure-detection test: a barrier that expects 16 bytes no copy
      // delivers, waited on while the tile copy is still in flight
      if (stall) mbar_expect_tx(test_bar, 16);
    }
    const bool landed = stall ? mbar_wait_bounded(test_bar, 0u, (uint64_t)a.stall_ns) : mbar_wait_bounded(bar, 0u);
    // Giving up is decided by the whole block: flag the run and, before
    // leaving, wait (bounded) for the tile copy, so that it cannot land in
    // shared memory the next CTA on this SM may own.
    if (__syncthreads_or(!landed)) {
      if (threadIdx.x == 0) {
        atomicOr(a.flag, RSST_FLAG_TIMEOUT);
        mbar_wait_bounded(bar, 0u);
      }
      return;
    }
  } else {
  for (int id = threadIdx.x; id < NV * C::SCELLS; id += NT) {
    const int v = id / C::SCELLS;
    const int r = id - v * C::SCELLS;
    const int lx = r % C::SX;
    const int t = r / C::SX;
    const int ly = t % C::SY;
    const int lz = t / C::SY;
    const int gi = i0 + lx - C::HX, gj = j0 + ly - C::HY, gk = k0 + lz - C::HZ;
    double val = 0.0;
    if (gi <= g.n[0] + 1 && (NDIM < 2 || gj <= g.n[1] + 1) && (NDIM < 3 || gk <= g.n[2] + 1))
      val = a.in[v * g.fstride + pidx(g, gi, gj, gk)];
    su[id] = val;
  }
  __syncthreads();
  }

  // 2-3. face fluxes and divergence, axis by axis
  double dU[C::CPT][NV];
#pragma unroll
  for (int c = 0; c < C::CPT; ++c)
#pragma unroll
    for (int v = 0; v < NV; ++v) dU[c][v] = 0.0;
  face_pass<NDIM, BX, BY, BZ, NT, 0, CV>(su, sf, ss, p, g, i0, j0, k0, dU);
  if constexpr (NDIM >= 2) face_pass<NDIM, BX, BY, BZ, NT, 1, CV>(su, sf, ss, p, g, i0, j0, k0, dU);
  if constexpr (NDIM >= 3) face_pass<NDIM, BX, BY, BZ, NT, 2, CV>(su, sf, ss, p, g, i0, j0, k0, dU);

  // 4. epilogue
  const double dt = a.dt_fixed > 0.0 ? a.dt_fixed : p.cfl / a.scal[a.slot];
  if (a.stage == 1 && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && threadIdx.x == 0) {
    a.scal[a.slot ^ 1] = 0.0;
    a.scal[2] = dt;
    a.scal[3] += dt;
  }
  double rmax = 0.0;
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
    double q[NV], L[NV], u[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      q[v] = su[v * C::SCELLS + s0];
      L[v] = dU[c][v];
    }
    if (a.dU_out) {
      const int64_t o = pidx(g, i, j, k);
#pragma unroll
      for (int v = 0; v < NV; ++v) a.dU_out[v * g.fstride + o] = L[v];
    }
    rsst_rhs<NV, CV>(q, L, p);
    if (a.stage == 1) {
#pragma unroll
      for (int v = 0; v < NV; ++v) u[v] = q[v] + dt * L[v];
    } else {
      const int64_t o = pidx(g, i, j, k);
#pragma unroll
      for (int v = 0; v < NV; ++v) u[v] = 0.5 * a.base[v * g.fstride + o] + 0.5 * (q[v] + dt * L[v]);
      bool ok;
      const double r = cfl_rate<NV, CV>(u, p, ok);
      if (ok) rmax = fmax(rmax, r);
      ok_all = ok_all && ok;
    }
    store_with_ghosts<NV>(a.out, g, p, a.bg, a.bg_len, i, j, k, u);
  }
  if (a.stage == 2) {
    if (!ok_all) atomicOr(a.flag, RSST_FLAG_NONPHYSICAL);
    block_max_to<NT>(rmax, a.scal + (a.slot ^ 1), sred);
  }
}

// ---------------------------------------------------------------------------
// Packing, CFL maximum, sums
// ---------------------------------------------------------------------------

// Caller layout [nvar][nz][ny][nx] -> padded layout, ghost cells included.
// Each padded cell maps every out-of-range coordinate to its source by the
// boundary rule (periodic wrap, or mirror with the normal momentum negated and
// the background difference added); corner ghosts are filled too (unused).
__global__ void pack_fp64_kernel(const double* __restrict__ src, double* __restrict__ dst, Geom g, Phys p,
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
      dst[v * g.fstride + di] = w;
    }
  }
}

__global__ void unpack_fp64_kernel(const double* __restrict__ src, double* __restrict__ dst, Geom g) {
  const int nv = g.ndim + 2;
  for (int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; id < g.ncells; id += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(id % g.n[0]);
    const int j = (int)((id / g.n[0]) % g.n[1]);
    const int k = (int)(id / ((int64_t)g.n[0] * g.n[1]));
    const int64_t o = pidx(g, i, j, k);
    for (int v = 0; v < nv; ++v) dst[v * g.ncells + id] = src[v * g.fstride + o];
  }
}

template <int NV, bool CV>
__global__ void __launch_bounds__(256) cfl_fp64_kernel(const double* __restrict__ U, Geom g, Phys p, double* dst,
                                                       unsigned int* flag) {
  __shared__ double sred[8];
  double rmax = 0.0;
  bool ok_all = true;
  for (int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; id < g.ncells; id += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(id % g.n[0]);
    const int j = (int)((id / g.n[0]) % g.n[1]);
    const int k = (int)(id / ((int64_t)g.n[0] * g.n[1]));
    const int64_t o = pidx(g, i, j, k);
    double q[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) q[v] = U[v * g.fstride + o];
    bool ok;
    const double r = cfl_rate<NV, CV>(q, p, ok);
    if (ok) rmax = fmax(rmax, r);
    ok_all = ok_all && ok;
  }
  if (!ok_all) atomicOr(flag, RSST_FLAG_NONPHYSICAL);
  block_max_to<256>(rmax, dst, sred);
}

// Deterministic sums: block b reduces a fixed contiguous chunk of cells with a
// fixed thread striding and shared-memory tree; a single block then reduces
// the per-block partials in index order.
constexpr int SUM_BLOCKS = 1024;
constexpr int SUM_THREADS = 256;

__global__ void __launch_bounds__(SUM_THREADS) sums_partial_fp64_kernel(const double* __restrict__ U, Geom g,
                                                                        double* __restrict__ partial) {
  __shared__ double sh[SUM_THREADS];
  const int nv = g.ndim + 2;
  const int64_t chunk = (g.ncells + SUM_BLOCKS - 1) / SUM_BLOCKS;
  const int64_t lo = blockIdx.x * chunk;
  const int64_t hi = min(g.ncells, lo + chunk);
  for (int v = 0; v < nv; ++v) {
    double acc = 0.0;
    for (int64_t id = lo + threadIdx.x; id < hi; id += SUM_THREADS) {
      const int i = (int)(id % g.n[0]);
      const int j = (int)((id / g.n[0]) % g.n[1]);
      const int k = (int)(id / ((int64_t)g.n[0] * g.n[1]));
      acc += U[v * g.fstride + pidx(g, i, j, k)];
    }
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int s = SUM_THREADS / 2; s > 0; s >>= 1) {
      if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
      __syncthreads();
    }
    if (threadIdx.x == 0) partial[v * SUM_BLOCKS + blockIdx.x] = sh[0];
    __syncthreads();
  }
}

__global__ void __launch_bounds__(SUM_THREADS) sums_final_kernel(const double* __restrict__ partial, int nv,
                                                                 double scale, double* __restrict__ out) {
  __shared__ double sh[SUM_THREADS];
  for (int v = 0; v < nv; ++v) {
    double acc = 0.0;
    for (int b = threadIdx.x; b < SUM_BLOCKS; b += SUM_THREADS) acc += partial[v * SUM_BLOCKS + b];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int s = SUM_THREADS / 2; s > 0; s >>= 1) {
      if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
      __syncthreads();
    }
    if (threadIdx.x == 0) out[v] = sh[0] * scale;
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------

template <int NDIM, int BX, int BY, int BZ, int NT, bool TMA, bool CV>
static int launch_stage_eos(const CUtensorMap* tin, const StageArgs<double>& a, cudaStream_t s) {
  using C = TileCfg<NDIM, BX, BY, BZ, NT>;
  auto kern = stage_fp64_kernel<NDIM, BX, BY, BZ, NT, TMA, CV>;
  static std::atomic<unsigned long long> attr{0};
  if (set_smem_limit_once(kern, C::SMEM, attr) != cudaSuccess) {
    rsst_set_error("cudaFuncSetAttribute failed for the float64 stage kernel");
    return RSST_ECUDA;
  }
  static const CUtensorMap none = {};
  dim3 grid((a.g.n[0] + BX - 1) / BX, NDIM >= 2 ? (a.g.n[1] + BY - 1) / BY : 1, NDIM >= 3 ? (a.g.n[2] + BZ - 1) / BZ : 1);
  kern<<<grid, NT, C::SMEM, s>>>(TMA ? *tin : none, a);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    rsst_set_error("float64 stage kernel launch: %s", cudaGetErrorString(e));
    return RSST_ECUDA;
  }
  return RSST_OK;
}

// The gas law is a compile-time choice (no covolume arithmetic in ideal-gas runs).
template <int NDIM, int BX, int BY, int BZ, int NT, bool TMA>
static int launch_stage(const CUtensorMap* tin, const StageArgs<double>& a, cudaStream_t s) {
  if (a.p.covol != 0.0) return launch_stage_eos<NDIM, BX, BY, BZ, NT, TMA, true>(tin, a, s);
  return launch_stage_eos<NDIM, BX, BY, BZ, NT, TMA, false>(tin, a, s);
}

}  // namespace rsst

using namespace rsst;

// Tiles: 1D short lines take 16-cell tiles (17 faces, one per thread of a
// warp) to spread the float64 work over SMs, longer ones 256 cells; 2D 16 x 16
// with 9 warps (every face and slope pass in one round; 0.7 % ahead of 32 x 8
// with the halo by TMA, from fewer halo slopes and faces); 3D 8 x 8 x 4 with
// slopes in shared memory and 10 warps (each face pass in one round).
using Tile2 = TileCfg<2, 16, 16, 1, 288>;
using Tile3 = TileCfg<3, 8, 8, 4, 320>;

void rsst_stage_fp64_box(int ndim, int* sx, int* sy, int* sz) {
  *sx = ndim == 3 ? Tile3::SX : Tile2::SX;
  *sy = ndim == 3 ? Tile3::SY : Tile2::SY;
  *sz = ndim == 3 ? Tile3::SZ : 1;
}

int rsst_launch_stage_fp64(const CUtensorMap* tin, const StageArgs<double>& a, cudaStream_t s) {
  switch (a.g.ndim) {
    case 1:
      if (a.g.n[0] <= RSST_SMALL_1D) return launch_stage<1, 16, 1, 1, 32, false>(nullptr, a, s);
      return launch_stage<1, 256, 1, 1, 256, false>(nullptr, a, s);
    case 2:
      return tin ? launch_stage<2, 16, 16, 1, 288, true>(tin, a, s) : launch_stage<2, 16, 16, 1, 288, false>(nullptr, a, s);
    case 3:
      return tin ? launch_stage<3, 8, 8, 4, 320, true>(tin, a, s) : launch_stage<3, 8, 8, 4, 320, false>(nullptr, a, s);
  }
  rsst_set_error("ndim must be 1, 2 or 3");
  return RSST_EINVAL;
}

static int grid_for(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b > 152 * 16) b = 152 * 16;
  return (int)(b < 1 ? 1 : b);
}

static int check_launch(const char* what) {
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    rsst_set_error("%s launch: %s", what, cudaGetErrorString(e));
    return RSST_ECUDA;
  }
  return RSST_OK;
}

int rsst_launch_pack_fp64(const double* src, double* dst, const Geom& g, const Phys& p, const double* bg, int bg_len,
                          cudaStream_t s) {
  const int64_t total = (int64_t)(g.n[0] + 4) * (g.ndim >= 2 ? g.n[1] + 4 : 1) * (g.ndim >= 3 ? g.n[2] + 4 : 1);
  pack_fp64_kernel<<<grid_for(total), 256, 0, s>>>(src, dst, g, p, bg, bg_len);
  return check_launch("pack");
}

int rsst_launch_unpack_fp64(const double* src, double* dst, const Geom& g, cudaStream_t s) {
  unpack_fp64_kernel<<<grid_for(g.ncells), 256, 0, s>>>(src, dst, g);
  return check_launch("unpack");
}

int rsst_launch_cfl_fp64(const double* U, const Geom& g, const Phys& p, double* slot_ptr, unsigned int* flag,
                         cudaStream_t s) {
  const int gb = grid_for(g.ncells);
  switch (g.ndim) {
    case 1:
      if (p.covol != 0.0) cfl_fp64_kernel<3, true><<<gb, 256, 0, s>>>(U, g, p, slot_ptr, flag);
      else cfl_fp64_kernel<3, false><<<gb, 256, 0, s>>>(U, g, p, slot_ptr, flag);
      break;
    case 2:
      if (p.covol != 0.0) cfl_fp64_kernel<4, true><<<gb, 256, 0, s>>>(U, g, p, slot_ptr, flag);
      else cfl_fp64_kernel<4, false><<<gb, 256, 0, s>>>(U, g, p, slot_ptr, flag);
      break;
    default:
      if (p.covol != 0.0) cfl_fp64_kernel<5, true><<<gb, 256, 0, s>>>(U, g, p, slot_ptr, flag);
      else cfl_fp64_kernel<5, false><<<gb, 256, 0, s>>>(U, g, p, slot_ptr, flag);
      break;
  }
  return check_launch("cfl");
}

int rsst_launch_sums_fp64(const double* U, const Geom& g, double* partial, double* out, double scale, cudaStream_t s) {
  sums_partial_fp64_kernel<<<SUM_BLOCKS, SUM_THREADS, 0, s>>>(U, g, partial);
  int rc = check_launch("sums");
  if (rc) return rc;
  sums_final_kernel<<<1, SUM_THREADS, 0, s>>>(partial, g.ndim + 2, scale, out);
  return check_launch("sums final");
}
