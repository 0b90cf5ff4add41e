// 2D float32 perturbation tile routine (see rsst_fp32_2d.cu for the layout).
#pragma once

#include "rsst_common.cuh"
#include "rsst_internal.h"
#include "rsst_math_fp32.cuh"
#include "rsst_tma.cuh"

namespace rsst {

// Tile geometry: BX_ x BY_ cells, each thread owning one column of SEG_
// cells (BX_ * BY_ / SEG_ threads).  Shared memory: the TMA box (halo tile,
// all fields), the x fluxes, the background rows, a barrier, dt, reduction.
template <int BX_, int BY_, int SEG_>
struct T2Cfg {
  static constexpr int NV = 4, BX = BX_, BY = BY_, SEG = SEG_;
  static constexpr int NT = BX * (BY / SEG);
  static constexpr int SXP = BX + 8;   // TMA box width: 4 columns each side (2 used), 16-byte aligned origin
  static constexpr int SYP = BY + 4;   // halo rows
  static constexpr int XO = 4;         // smem column of tile x = 0
  static constexpr int FXW = BX + 1;   // x faces per row
  static constexpr int U_FLOATS = NV * SYP * SXP;
  static constexpr int FX_FLOATS = NV * BY * FXW;
  static constexpr int TAB_FLOATS = TB_COUNT * SYP;
  static constexpr size_t SCRATCH = (size_t)(U_FLOATS + FX_FLOATS + TAB_FLOATS) * 4;
  static constexpr uint32_t BOX_BYTES = U_FLOATS * 4;
  static constexpr size_t smem_bytes() { return SCRATCH + 16 + 8 * 8 + 512 + 128; }
  static_assert(BY % SEG == 0, "column segments must tile BY");
  static_assert(SCRATCH % 8 == 0, "the barriers after the scratch area need 8-byte alignment");
  static_assert(SXP <= 256 && SYP <= 256, "TMA box dimensions are at most 256");
};

using T2 = T2Cfg<128, 8, 8>;  // single-run default (best of a 13-shape sweep on GB300: 5 CTAs of 4 warps per SM)

template <class C>
__device__ __forceinline__ uint64_t* t2_barrier(unsigned char* smem) {
  return reinterpret_cast<uint64_t*>(smem + C::SCRATCH);
}
template <class C>
__device__ __forceinline__ double* t2_sred(unsigned char* smem) {
  return reinterpret_cast<double*>(smem + C::SCRATCH + 16);
}
// free shared memory after the reduction slots (used by the batched kernel)
template <class C>
__device__ __forceinline__ unsigned char* t2_extra(unsigned char* smem) {
  return smem + C::SCRATCH + 16 + 8 * 8;
}
// barrier of the failure-detection test wait (after the batched kernel's 512 bytes)
template <class C>
__device__ __forceinline__ uint64_t* t2_stall_barrier(unsigned char* smem) {
  return reinterpret_cast<uint64_t*>(smem + C::SCRATCH + 16 + 8 * 8 + 512);
}

// Everything one tile needs about its run.
struct TileRun {
  Geom g;
  Phys p;
  PhysF pf;
  const float* base;
  float* out;
  const float* tab;
  int tab_len;
  unsigned int* flag;
  int stage;
  int64_t stall_ns;  // > 0 only in failure-detection tests (see tile2d_f)
};

// LLF flux of the x face between tile cells with smem columns c-1 | c (row sr).
template <class T2, int VERT>
__device__ __forceinline__ void t2_xflux(const float* __restrict__ sU, const float* __restrict__ st, int sr, int c,
                                         const PhysF& pf, float (&F)[4]) {
  constexpr int NV = 4;
  float qL[NV], qR[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const float* row = sU + (v * T2::SYP + sr) * T2::SXP + c;
    const float um2 = row[-2], um1 = row[-1], u0 = row[0], up1 = row[1];
    qL[v] = um1 + 0.5f * mc_slope_f(um1 - um2, u0 - um1);
    qR[v] = u0 - 0.5f * mc_slope_f(u0 - um1, up1 - u0);
  }
  float FL[NV], FR[NV], cL, cR, dum;
  if constexpr (VERT < 0) {
    euler_flux_f<NV, 0>(qL, pf, FL, cL);
    euler_flux_f<NV, 0>(qR, pf, FR, cR);
  } else {
    const float rho0 = st[TB_RHO0 * T2::SYP + sr], P0 = st[TB_P0 * T2::SYP + sr], H0 = st[TB_H0 * T2::SYP + sr];
    pert_flux_f<NV, 0, false>(qL, rho0, P0, H0, 0.0f, pf, FL, cL, dum);
    pert_flux_f<NV, 0, false>(qR, rho0, P0, H0, 0.0f, pf, FR, cR, dum);
  }
  const float alpha = cL >= cR ? cL : cR;
#pragma unroll
  for (int v = 0; v < NV; ++v) F[v] = 0.5f * (FL[v] + FR[v]) - 0.5f * alpha * (qR[v] - qL[v]);
}

// MC slope along y of the cell at smem row r from its neighbours' values.
template <class T2, int VERT>
__device__ __forceinline__ void t2_yslope(const float (&um)[4], const float (&u0)[4], const float (&up)[4],
                                          const float* __restrict__ st, int r, float (&s)[4]) {
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    const float da = u0[v] - um[v], db = up[v] - u0[v];
    if (VERT == 1 && (v == 0 || v == 3))
      s[v] = bg_slope_f(st + (TB_S + 6 * (v == 0 ? 0 : 1)) * T2::SYP, T2::SYP, r, da, db);
    else
      s[v] = mc_slope_f(da, db);
  }
}

// y-face flux between cells (u0, s0) below and (u1, s1) above; face table at smem row rf.
template <class T2, int VERT>
__device__ __forceinline__ void t2_yflux(const float (&u0)[4], const float (&s0)[4], const float (&u1)[4],
                                         const float (&s1)[4], const float* __restrict__ st, int rf, const PhysF& pf,
                                         float (&F)[4]) {
  constexpr int NV = 4;
  float qL[NV], qR[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    qL[v] = u0[v] + 0.5f * s0[v];
    qR[v] = u1[v] - 0.5f * s1[v];
  }
  float FL[NV], FR[NV], cL, cR;
  if constexpr (VERT < 0) {
    euler_flux_f<NV, 1>(qL, pf, FL, cL);
    euler_flux_f<NV, 1>(qR, pf, FR, cR);
    const float alpha = cL >= cR ? cL : cR;
#pragma unroll
    for (int v = 0; v < NV; ++v) F[v] = 0.5f * (FL[v] + FR[v]) - 0.5f * alpha * (qR[v] - qL[v]);
  } else {
    float dcL, dcR;
    const float gdiff = st[TB_FG * T2::SYP + rf], al0 = st[TB_FALPHA * T2::SYP + rf];
    const float c0L = gdiff >= 0.0f ? al0 : al0 + gdiff, c0R = gdiff >= 0.0f ? al0 - gdiff : al0;
    pert_flux_f<NV, 1, true>(qL, st[TB_FRHOL * T2::SYP + rf], st[TB_FPL * T2::SYP + rf], st[TB_FHL * T2::SYP + rf],
                             st[TB_FAL * T2::SYP + rf], pf, FL, cL, dcL, c0L);
    pert_flux_f<NV, 1, true>(qR, st[TB_FRHOR * T2::SYP + rf], st[TB_FPR * T2::SYP + rf], st[TB_FHR * T2::SYP + rf],
                             st[TB_FAR * T2::SYP + rf], pf, FR, cR, dcR, c0R);
    const float dalpha = gdiff >= 0.0f ? fmaxf(dcL, dcR - gdiff) : fmaxf(dcL + gdiff, dcR);
    const float alpha = st[TB_FALPHA * T2::SYP + rf] + dalpha;
    const float jr = st[TB_FDRHO * T2::SYP + rf], je = st[TB_FDE * T2::SYP + rf];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const float j0v = v == 0 ? jr : (v == NV - 1 ? je : 0.0f);
      F[v] = 0.5f * (FL[v] + FR[v]) - 0.5f * (alpha * (qR[v] - qL[v]) + dalpha * j0v);
    }
  }
}

// Process tile (tx, ty) of run r: returns false if the TMA wait timed out
// (flag set).  Accumulates the stage-2 CFL rate maximum and physical check.
// The caller initialised the barrier; `phase` is its current parity.
template <class T2, int VERT>
__device__ __forceinline__ bool tile2d_f(const CUtensorMap* tin, const TileRun& r, float dt, int tx, int ty,
                                         unsigned char* smem, uint32_t& phase, float& rmax, bool& ok_all) {
  constexpr int NV = 4;
  float* sU = reinterpret_cast<float*>(smem);
  float* sFx = sU + T2::U_FLOATS;
  float* st = sFx + T2::FX_FLOATS;
  uint64_t* bar = t2_barrier<T2>(smem);
  const Geom& g = r.g;
  const PhysF& pf = r.pf;
  const int i0 = tx * T2::BX, j0 = ty * T2::BY;
  const int tid = threadIdx.x;

  __syncthreads();  // previous tile's shared-memory reads are done
  if (tid == 0) {
    fence_proxy_async_smem();
    mbar_expect_tx(bar, T2::BOX_BYTES);
    tma_load_3d(sU, tin, bar, i0 + g.xoff - T2::XO, j0, 0);
  }
  if constexpr (VERT >= 0) {
    for (int id = tid; id < T2::TAB_FLOATS; id += T2::NT) {
      const int f = id / T2::SYP, rr = id - f * T2::SYP;
      const int kp = j0 + rr;
      st[id] = kp < r.tab_len ? r.tab[(size_t)f * r.tab_len + kp] : 0.0f;
    }
  }
  // the give-up decision is taken by the whole block (no thread may leave
  // while others wait at a barrier); a late copy gets one more bounded wait
  if (__syncthreads_or(!mbar_wait_bounded(bar, phase))) {
    if (tid == 0) atomicOr(r.flag, RSST_FLAG_TIMEOUT);
    mbar_wait_bounded(bar, phase);
    return false;
  }
  phase ^= 1u;
  if (r.stall_ns > 0) {
    // Failure-detection test: with the tile's copy landed (nothing in
    // flight), wait on a barrier that expects 16 bytes no copy delivers, so
    // the bounded wait runs out and the give-up path above is taken.
    uint64_t* sb = t2_stall_barrier<T2>(smem);
    if (tid == 0) {
      mbar_init(sb, 1);
      fence_mbar_init();
      mbar_expect_tx(sb, 16);
    }
    __syncthreads();
    if (__syncthreads_or(!mbar_wait_bounded(sb, 0u, (uint64_t)r.stall_ns))) {
      if (tid == 0) atomicOr(r.flag, RSST_FLAG_TIMEOUT);
      return false;
    }
  }

  // x faces
  const int nx = g.n[0], ny = g.n[1];
  for (int fid = tid; fid < T2::BY * T2::FXW; fid += T2::NT) {
    const int row = fid / T2::FXW;
    const int fx = fid - row * T2::FXW;
    if (i0 + fx > nx || j0 + row >= ny) continue;
    float F[NV];
    t2_xflux<T2, VERT>(sU, st, row + 2, fx + T2::XO, pf, F);
#pragma unroll
    for (int v = 0; v < NV; ++v) sFx[(v * T2::BY + row) * T2::FXW + fx] = F[v];
  }
  __syncthreads();

  // column march with the fused epilogue
  const int col = tid % T2::BX;
  const int seg = tid / T2::BX;
  const int x = i0 + col;
  const int jb = seg * T2::SEG;  // first tile row of this thread
  if (x < nx && j0 + jb < ny) {
    const int sc = col + T2::XO;
    auto ld = [&](int srow, float (&u)[4]) {
#pragma unroll
      for (int v = 0; v < NV; ++v) u[v] = sU[(v * T2::SYP + srow) * T2::SXP + sc];
    };
    float um[4], u0[4], u1[4], u2[4], s0[4], s1[4], sm[4], Fm[4], Fp[4];
    // cells jb-2 .. jb+1 live at smem rows jb .. jb+3
    ld(jb, u2);   // u2 used as scratch for cell jb-2
    ld(jb + 1, um);
    ld(jb + 2, u0);
    ld(jb + 3, u1);
    t2_yslope<T2, VERT>(u2, um, u0, st, jb + 1, sm);   // slope of cell jb-1
    t2_yslope<T2, VERT>(um, u0, u1, st, jb + 2, s0);   // slope of cell jb
    t2_yflux<T2, VERT>(um, sm, u0, s0, st, jb + 2, pf, Fm);
    const float idx = pf.inv_dx[0], idy = pf.inv_dx[1];
    const int64_t fs = g.fstride;
#pragma unroll 1
    for (int jj = 0; jj < T2::SEG; ++jj) {
      const int j = jb + jj;       // tile row of the cell
      if (j0 + j >= ny) break;
      ld(j + 4, u2);               // cell j+2
      t2_yslope<T2, VERT>(u0, u1, u2, st, j + 3, s1);   // slope of cell j+1
      t2_yflux<T2, VERT>(u0, s0, u1, s1, st, j + 3, pf, Fp);
      float L[4], Dl[4];
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const float* fr = sFx + (v * T2::BY + j) * T2::FXW + col;
        L[v] = -(Fp[v] - Fm[v]) * idy - (fr[1] - fr[0]) * idx;
        Dl[v] = L[v];
      }
      float rho0 = 0.0f, P0 = 0.0f;
      const int srow = j + 2;
      if constexpr (VERT >= 0) {
        rho0 = st[TB_RHO0 * T2::SYP + srow];
        P0 = st[TB_P0 * T2::SYP + srow];
        Dl[0] += st[TB_D0RHO * T2::SYP + srow];
        Dl[2] += st[TB_D0MV * T2::SYP + srow];
        Dl[3] += st[TB_D0E * T2::SYP + srow];
#pragma unroll
        for (int v = 0; v < NV; ++v) L[v] += st[(TB_R0 + v) * T2::SYP + srow];
      }
      const int y = j0 + j;
      const int64_t o = pidx(g, x, y, 0);
      float bv[4];
      if (r.stage == 2) {
#pragma unroll
        for (int v = 0; v < NV; ++v) bv[v] = r.base[v * fs + o];
      }
      float u[4], rate;
      bool ok;
      cell_update_f<4>(u0, L, Dl, rho0, P0, pf, r.p.variant, r.p.has_grav != 0, r.stage, dt, bv, u, rate, ok);
      if (r.stage == 2) {
        rmax = fmaxf(rmax, rate);
        ok_all = ok_all && ok;
      }
      store_mirror_ghosts<float, 4>(r.out, g, r.p, x, y, 0, u);
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        u0[v] = u1[v];
        u1[v] = u2[v];
        s0[v] = s1[v];
        Fm[v] = Fp[v];
      }
    }
  }
  return true;
}

}  // namespace rsst
