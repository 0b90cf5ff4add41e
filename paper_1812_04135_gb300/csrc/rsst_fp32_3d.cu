// Float32 perturbation stage kernel for 3D grids: TMA-streamed z-march.
//
// A CTA owns a 16 x 8 block of (x, y) columns and a chunk of CZ = 16
// z-planes (the best of a nine-shape sweep on GB300: five CTAs per SM).
// Planes (with two-cell x/y halos, all five fields; x origin rounded down to
// a 16-byte boundary) stream through a six-slot shared-memory ring, one
// cp.async.bulk.tensor per plane issued three planes ahead, each slot with
// its own mbarrier (bounded waits).  For the current plane k: the x and y
// faces of the plane are computed in parallel into shared memory; then each
// thread (one column) takes one new MC slope and one z-face flux from a
// register window, adds the plane's x and y flux differences, and applies the
// reduced tendency, force, RK combine, store and edge ghosts (and in stage 2
// the CFL rate), all fused.  The vertical axis (background) is z or absent.
#include "rsst_common.cuh"
#include "rsst_internal.h"
#include "rsst_math_fp32.cuh"
#include "rsst_tma.cuh"
#include "rsst_attr.h"

namespace rsst {

struct T3 {
  static constexpr int NV = 5, BX = 16, BY = 8, NT = BX * BY, CZ = 16, NS = 6;
  static constexpr int SXP = BX + 8, SYP = BY + 4, XO = 4, YO = 2;
  static constexpr int PLANE = NV * SYP * SXP;  // floats per plane slot
  static constexpr int FXW = BX + 1, FYH = BY + 1;
  static constexpr int FX_FLOATS = NV * BY * FXW, FY_FLOATS = NV * FYH * BX;
  static constexpr int TROWS = CZ + 4;
  static constexpr int TAB_FLOATS = TB_COUNT * TROWS;
  static constexpr size_t RING = (size_t)NS * PLANE * 4;
  static constexpr size_t SCRATCH = RING + (size_t)(FX_FLOATS + FY_FLOATS + TAB_FLOATS) * 4;
  static constexpr size_t SMEM = SCRATCH + NS * 8 + 16 + 8 * 8 + 128;
  static constexpr uint32_t BOX_BYTES = PLANE * 4;
};

template <int VERT>
__device__ __forceinline__ void t3_xyflux(const float* __restrict__ P, int D, int r, int c, float rho0, float P0,
                                          float H0, const PhysF& pf, float (&F)[5]) {
  constexpr int NV = 5;
  const int stride = D == 0 ? 1 : T3::SXP;
  float qL[NV], qR[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const float* s = P + (v * T3::SYP + r) * T3::SXP + c;
    const float um2 = s[-2 * stride], um1 = s[-stride], u0 = s[0], up1 = s[stride];
    qL[v] = um1 + 0.5f * mc_slope_f(um1 - um2, u0 - um1);
    qR[v] = u0 - 0.5f * mc_slope_f(u0 - um1, up1 - u0);
  }
  float FL[NV], FR[NV], cL, cR, dum;
  if (D == 0) {
    if constexpr (VERT < 0) {
      euler_flux_f<NV, 0>(qL, pf, FL, cL);
      euler_flux_f<NV, 0>(qR, pf, FR, cR);
    } else {
      pert_flux_f<NV, 0, false>(qL, rho0, P0, H0, 0.0f, pf, FL, cL, dum);
      pert_flux_f<NV, 0, false>(qR, rho0, P0, H0, 0.0f, pf, FR, cR, dum);
    }
  } else {
    if constexpr (VERT < 0) {
      euler_flux_f<NV, 1>(qL, pf, FL, cL);
      euler_flux_f<NV, 1>(qR, pf, FR, cR);
    } else {
      pert_flux_f<NV, 1, false>(qL, rho0, P0, H0, 0.0f, pf, FL, cL, dum);
      pert_flux_f<NV, 1, false>(qR, rho0, P0, H0, 0.0f, pf, FR, cR, dum);
    }
  }
  const float alpha = cL >= cR ? cL : cR;
#pragma unroll
  for (int v = 0; v < NV; ++v) F[v] = 0.5f * (FL[v] + FR[v]) - 0.5f * alpha * (qR[v] - qL[v]);
}

template <int VERT>
__device__ __forceinline__ void t3_zslope(const float (&um)[5], const float (&u0)[5], const float (&up)[5],
                                          const float* __restrict__ st, int r, float (&s)[5]) {
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    const float da = u0[v] - um[v], db = up[v] - u0[v];
    if (VERT == 2 && (v == 0 || v == 4))
      s[v] = bg_slope_f(st + (TB_S + 6 * (v == 0 ? 0 : 1)) * T3::TROWS, T3::TROWS, r, da, db);
    else
      s[v] = mc_slope_f(da, db);
  }
}

template <int VERT>
__device__ __forceinline__ void t3_zflux(const float (&u0)[5], const float (&s0)[5], const float (&u1)[5],
                                         const float (&s1)[5], const float* __restrict__ st, int rf, const PhysF& pf,
                                         float (&F)[5]) {
  constexpr int NV = 5;
  float qL[NV], qR[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    qL[v] = u0[v] + 0.5f * s0[v];
    qR[v] = u1[v] - 0.5f * s1[v];
  }
  float FL[NV], FR[NV], cL, cR;
  if constexpr (VERT < 0) {
    euler_flux_f<NV, 2>(qL, pf, FL, cL);
    euler_flux_f<NV, 2>(qR, pf, FR, cR);
    const float alpha = cL >= cR ? cL : cR;
#pragma unroll
    for (int v = 0; v < NV; ++v) F[v] = 0.5f * (FL[v] + FR[v]) - 0.5f * alpha * (qR[v] - qL[v]);
  } else {
    constexpr int R = T3::TROWS;
    float dcL, dcR;
    const float gdiff = st[TB_FG * R + rf], al0 = st[TB_FALPHA * R + rf];
    const float c0L = gdiff >= 0.0f ? al0 : al0 + gdiff, c0R = gdiff >= 0.0f ? al0 - gdiff : al0;
    pert_flux_f<NV, 2, true>(qL, st[TB_FRHOL * R + rf], st[TB_FPL * R + rf], st[TB_FHL * R + rf], st[TB_FAL * R + rf],
                             pf, FL, cL, dcL, c0L);
    pert_flux_f<NV, 2, true>(qR, st[TB_FRHOR * R + rf], st[TB_FPR * R + rf], st[TB_FHR * R + rf], st[TB_FAR * R + rf],
                             pf, FR, cR, dcR, c0R);
    const float dalpha = gdiff >= 0.0f ? fmaxf(dcL, dcR - gdiff) : fmaxf(dcL + gdiff, dcR);
    const float alpha = st[TB_FALPHA * R + rf] + dalpha;
    const float jr = st[TB_FDRHO * R + rf], je = st[TB_FDE * R + rf];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const float j0v = v == 0 ? jr : (v == NV - 1 ? je : 0.0f);
      F[v] = 0.5f * (FL[v] + FR[v]) - 0.5f * (alpha * (qR[v] - qL[v]) + dalpha * j0v);
    }
  }
}

template <int VERT>
__global__ void __launch_bounds__(T3::NT, 2) stage3d_tma_kernel(const __grid_constant__ CUtensorMap tin,
                                                                 const StageArgs<float> a) {
  constexpr int NV = 5;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float* ring = reinterpret_cast<float*>(smem_raw);
  float* sFx = ring + T3::NS * T3::PLANE;
  float* sFy = sFx + T3::FX_FLOATS;
  float* st = sFy + T3::FY_FLOATS;
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + T3::SCRATCH);
  float* sdt = reinterpret_cast<float*>(bar + T3::NS);
  double* sred = reinterpret_cast<double*>(smem_raw + T3::SCRATCH + T3::NS * 8 + 16);
  const Geom& g = a.g;
  const Phys& p = a.p;
  const PhysF& pf = a.pf;
  const int tid = threadIdx.x;
  const int i0 = blockIdx.x * T3::BX, j0 = blockIdx.y * T3::BY;
  const int k0 = blockIdx.z * T3::CZ;
  const int nz = g.n[2];
  const int k1 = min(k0 + T3::CZ, nz);
  const int pfirst = k0 - 2, plast = k1 + 1;  // planes needed by this chunk

  if (tid == 0) {
    const double dtd = a.dt_fixed > 0.0 ? a.dt_fixed : p.cfl / a.scal[a.slot];
    *sdt = (float)dtd;
    if (a.stage == 1 && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0) {
      a.scal[a.slot ^ 1] = 0.0;
      a.scal[2] = dtd;
      a.scal[3] += dtd;
    }
    for (int s = 0; s < T3::NS; ++s) mbar_init(&bar[s], 1);
    fence_mbar_init();
  }
  __syncthreads();
  auto slot_of = [&](int pl) { return (pl - pfirst) % T3::NS; };
  auto phase_of = [&](int pl) { return (uint32_t)(((pl - pfirst) / T3::NS) & 1); };
  auto issue = [&](int pl) {
    const int s = slot_of(pl);
    mbar_expect_tx(&bar[s], T3::BOX_BYTES);
    tma_load_4d(ring + s * T3::PLANE, &tin, &bar[s], i0 + g.xoff - T3::XO, j0, pl + RSST_G, 0);
  };
  int issued = min(pfirst + 4, plast);  // last plane whose copy has been issued
  if (tid == 0) {
    fence_proxy_async_smem();
    for (int pl = pfirst; pl <= issued; ++pl) issue(pl);
  }
  if constexpr (VERT >= 0) {
    for (int id = tid; id < T3::TAB_FLOATS; id += T3::NT) {
      const int f = id / T3::TROWS, rr = id - f * T3::TROWS;
      const int kp = k0 + rr;  // padded z index of table row rr (interior k0 - 2 + rr)
      st[id] = kp < a.tab_len ? a.tab[(size_t)f * a.tab_len + kp] : 0.0f;
    }
  }
  const float dt = *sdt;
  int waited = pfirst - 1;  // planes up to this one are resident
  auto wait_upto = [&](int pl) -> bool {
    for (int q = waited + 1; q <= pl; ++q) {
      if (!mbar_wait_bounded(&bar[slot_of(q)], phase_of(q))) return false;
    }
    if (pl > waited) waited = pl;
    return true;
  };
  // Giving up: flag the run, and before the CTA leaves, wait (bounded) for
  // every plane copy still in flight, so that none lands in shared memory
  // the next CTA on this SM may own.
  auto give_up = [&]() {
    if (tid == 0) {
      atomicOr(a.flag, RSST_FLAG_TIMEOUT);
      for (int q = waited + 1; q <= issued; ++q) mbar_wait_bounded(&bar[slot_of(q)], phase_of(q));
    }
  };
  // the give-up decision is taken by the whole block (no thread may leave
  // while others wait at a barrier)
  if (__syncthreads_or(!wait_upto(pfirst + 3))) {
    give_up();
    return;
  }

  const int cx = tid % T3::BX, cy = tid / T3::BX;
  const int x = i0 + cx, y = j0 + cy;
  const bool mine = x < g.n[0] && y < g.n[1];
  const int sxy = (cy + T3::YO) * T3::SXP + (cx + T3::XO);  // smem offset of my column in a plane
  auto ld = [&](int pl, float (&u)[5]) {
    const float* P = ring + slot_of(pl) * T3::PLANE;
#pragma unroll
    for (int v = 0; v < NV; ++v) u[v] = P[v * T3::SYP * T3::SXP + sxy];
  };
  // z window: rows of the table are indexed by padded z - k0 (interior z - k0 + 2)
  float u0[5], u1[5], u2[5], s0[5], s1[5], Fm[5], Fp[5];
  {
    float um[5], umm[5], sm[5];
    ld(k0 - 2, umm);
    ld(k0 - 1, um);
    ld(k0, u0);
    ld(k0 + 1, u1);
    t3_zslope<VERT>(umm, um, u0, st, 1, sm);
    t3_zslope<VERT>(um, u0, u1, st, 2, s0);
    t3_zflux<VERT>(um, sm, u0, s0, st, 2, pf, Fm);
  }
  float rmax = 0.0f;
  bool ok_all = true;
  const float idx = pf.inv_dx[0], idy = pf.inv_dx[1], idz = pf.inv_dx[2];
  const int64_t fs = g.fstride;
#pragma unroll 1
  for (int k = k0; k < k1; ++k) {
    // everyone sees plane k+2 and the slot of plane k-3 is free
    if (__syncthreads_or(!wait_upto(k + 2))) {
      give_up();
      return;
    }
    if (k + 3 <= plast) {
      if (tid == 0) {
        fence_proxy_async_smem();
        issue(k + 3);
      }
      issued = k + 3;
    }
    const int rz = k - k0 + 2;  // table row of plane k
    float rho0 = 0.0f, P0 = 0.0f, H0 = 0.0f;
    if constexpr (VERT >= 0) {
      rho0 = st[TB_RHO0 * T3::TROWS + rz];
      P0 = st[TB_P0 * T3::TROWS + rz];
      H0 = st[TB_H0 * T3::TROWS + rz];
    }
    const float* P = ring + slot_of(k) * T3::PLANE;
    // x faces (33 x 8) and y faces (32 x 9) of plane k
    for (int f = tid; f < T3::BY * T3::FXW + T3::FYH * T3::BX; f += T3::NT) {
      float F[5];
      if (f < T3::BY * T3::FXW) {
        const int r = f / T3::FXW, c = f - r * T3::FXW;
        if (i0 + c > g.n[0] || j0 + r >= g.n[1]) continue;
        t3_xyflux<VERT>(P, 0, r + T3::YO, c + T3::XO, rho0, P0, H0, pf, F);
#pragma unroll
        for (int v = 0; v < NV; ++v) sFx[(v * T3::BY + r) * T3::FXW + c] = F[v];
      } else {
        const int ff = f - T3::BY * T3::FXW;
        const int r = ff / T3::BX, c = ff - r * T3::BX;
        if (i0 + c >= g.n[0] || j0 + r > g.n[1]) continue;
        t3_xyflux<VERT>(P, 1, r + T3::YO, c + T3::XO, rho0, P0, H0, pf, F);
#pragma unroll
        for (int v = 0; v < NV; ++v) sFy[(v * T3::FYH + r) * T3::BX + c] = F[v];
      }
    }
    __syncthreads();
    if (mine) {
      ld(k + 2, u2);
      t3_zslope<VERT>(u0, u1, u2, st, rz + 1, s1);
      t3_zflux<VERT>(u0, s0, u1, s1, st, rz + 1, pf, Fp);
      float L[5], Dl[5];
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const float* fx = sFx + (v * T3::BY + cy) * T3::FXW + cx;
        const float* fy = sFy + (v * T3::FYH + cy) * T3::BX + cx;
        L[v] = -(Fp[v] - Fm[v]) * idz - (fx[1] - fx[0]) * idx - (fy[T3::BX] - fy[0]) * idy;
        Dl[v] = L[v];
      }
      if constexpr (VERT >= 0) {
        Dl[0] += st[TB_D0RHO * T3::TROWS + rz];
        Dl[3] += st[TB_D0MV * T3::TROWS + rz];
        Dl[4] += st[TB_D0E * T3::TROWS + rz];
#pragma unroll
        for (int v = 0; v < NV; ++v) L[v] += st[(TB_R0 + v) * T3::TROWS + rz];
      }
      const int64_t o = pidx(g, x, y, k);
      float bv[5];
      if (a.stage == 2) {
#pragma unroll
        for (int v = 0; v < NV; ++v) bv[v] = a.base[v * fs + o];
      }
      float u[5], rate;
      bool ok;
      cell_update_f<5>(u0, L, Dl, rho0, P0, pf, p.variant, p.has_grav != 0, a.stage, dt, bv, u, rate, ok);
      if (a.stage == 2) {
        rmax = fmaxf(rmax, rate);
        ok_all = ok_all && ok;
      }
      store_mirror_ghosts<float, 5>(a.out, g, p, x, y, k, u);
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        u0[v] = u1[v];
        u1[v] = u2[v];
        s0[v] = s1[v];
        Fm[v] = Fp[v];
      }
    }
  }
  if (a.stage == 2) {
    if (!ok_all) atomicOr(a.flag, RSST_FLAG_NONPHYSICAL);
    block_max_to<T3::NT>((double)rmax, a.scal + (a.slot ^ 1), sred);
  }
}

}  // namespace rsst

using namespace rsst;

// TMA box of one plane of the 3D tile (halo included), for the tensor maps.
void rsst_stage3d_box(int* box_x, int* box_y) {
  *box_x = T3::SXP;
  *box_y = T3::SYP;
}

int rsst_launch_stage3d_tma(const CUtensorMap* tin, const StageArgs<float>& a, cudaStream_t s) {
  const int vert = a.tab ? a.p.vertical : -1;
  dim3 grid((a.g.n[0] + T3::BX - 1) / T3::BX, (a.g.n[1] + T3::BY - 1) / T3::BY, (a.g.n[2] + T3::CZ - 1) / T3::CZ);
  if (vert == 2) {
    static std::atomic<unsigned long long> attr{0};
    if (set_smem_limit_once(stage3d_tma_kernel<2>, T3::SMEM, attr) != cudaSuccess) {
      rsst_set_error("cudaFuncSetAttribute failed for the 3D float32 TMA stage kernel");
      return RSST_ECUDA;
    }
    stage3d_tma_kernel<2><<<grid, T3::NT, T3::SMEM, s>>>(*tin, a);
  } else if (vert < 0) {
    static std::atomic<unsigned long long> attr{0};
    if (set_smem_limit_once(stage3d_tma_kernel<-1>, T3::SMEM, attr) != cudaSuccess) {
      rsst_set_error("cudaFuncSetAttribute failed for the 3D float32 TMA stage kernel");
      return RSST_ECUDA;
    }
    stage3d_tma_kernel<-1><<<grid, T3::NT, T3::SMEM, s>>>(*tin, a);
  } else {
    rsst_set_error("3D TMA kernel supports a vertical axis of z or none");
    return RSST_EUNSUPPORTED;
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    rsst_set_error("3D float32 TMA stage launch: %s", cudaGetErrorString(e));
    return RSST_ECUDA;
  }
  return RSST_OK;
}
