// Float32 perturbation stage kernel for 3D grids: TMA-streamed z-march.
//
// A CTA owns a BX x BY = 32 x 4 block of (x, y) columns (one warp per row of
// the block) and a chunk of CZ = 12 z-planes (the best of 8, 11, 12 and 16
// planes, and of 32 x 8 blocks, on the 256 x 128 x 128 workload).  Planes (two-cell x/y halos,
// all five fields; x origin rounded down to a 16-byte boundary) stream
// through an NS = 5 slot shared-memory ring, one cp.async.bulk.tensor per
// plane issued three planes ahead, each slot with its own mbarrier (bounded
// waits).  Per plane k, with two block barriers:
//   A. every thread takes the y half slope of its cell, writes the cell's
//      upper y face state U + h to shared memory and keeps the lower one;
//      the first and last warps also take the halo rows -1 and BY (done at
//      the end of step C of the previous plane, so the barrier that opens
//      the plane also publishes these states);
//   B. every thread forms twice the LLF flux of the y face below its cell
//      from the state written by the cell below (the last warp also the
//      face above the block), and the warps walk the x faces of the plane in
//      chunks of 64 slope cells, two per lane (as in the 2D kernel: a lane
//      forms the face between its cells and, with the state passed one lane
//      up, the face on its left; no lane runs alone);
//   C. each thread advances its column: one new z half slope and z-face flux
//      from a register window, the divergence (its x and y faces from shared
//      memory), the reduced tendency, force, RK combine, store and edge
//      ghosts (and in stage 2 the CFL rate), all fused.
// The vertical axis (background) is z or absent.  The arithmetic is that of
// rsst_fp32_lean.cuh.
#pragma once

#include "rsst_common.cuh"
#include "rsst_internal.h"
#include "rsst_fp32_lean.cuh"
#include "rsst_math_fp32.cuh"
#include "rsst_tma.cuh"
#include "rsst_attr.h"

namespace rsst {

struct T3 {
  static constexpr int NV = 5, BX = 32, BY = 4, NT = BX * BY, CZ = 12, NS = 5;
  static constexpr int SXP = BX + 8, SYP = BY + 4, XO = 4, YO = 2;
  static constexpr int PF = SYP * SXP;     // floats per field in a plane slot
  static constexpr int PLANE = NV * PF;    // floats per plane slot
  static constexpr int FXW = BX + 1;       // x faces per row
  static constexpr int FX_FLOATS = NV * BY * FXW;
  static constexpr int FY_FLOATS = NV * (BY + 1) * BX;
  static constexpr int QROWS = BY + 1;     // upper y face states of rows -1 .. BY-1
  static constexpr int Q_FLOATS = NV * QROWS * BX;
  static constexpr int TROWS = CZ + 4;
  static constexpr int TAB_FLOATS = TR_W * TROWS;
  static constexpr int CW2 = BX + 4;       // x slope cells per row (-1 .. BX, padded to an even count)
  static constexpr int NCHUNK2 = (BY * CW2 - 2 + 61) / 62;  // chunks of 64 cells, one every 62
  static constexpr size_t RING = (size_t)NS * PLANE * 4;
  static constexpr size_t SCRATCH = RING + (size_t)(FX_FLOATS + FY_FLOATS + Q_FLOATS + TAB_FLOATS) * 4;
  static constexpr size_t SMEM = SCRATCH + NS * 8 + 16 + 8 * 8 + 8 + 128;  // ring barriers, dt, reduction, test barrier
  static constexpr uint32_t BOX_BYTES = PLANE * 4;
  static_assert(BX == 32, "one warp per row of the column block");
  static_assert(RING % 16 == 0 && (FX_FLOATS + FY_FLOATS + Q_FLOATS) % 4 == 0, "table rows on a 16-byte boundary");
  static_assert(SCRATCH % 8 == 0, "barriers after the scratch area need 8-byte alignment");
};

template <int VERT, int FORM, int CM, int ST>
__global__ void __launch_bounds__(T3::NT, 5) stage3d_tma_kernel(const __grid_constant__ CUtensorMap tin,
                                                                 const StageArgs<float> a) {
  constexpr int NV = 5;
  constexpr bool BG = VERT >= 0;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float* ring = reinterpret_cast<float*>(smem_raw);
  float* sFx = ring + T3::NS * T3::PLANE;
  float* sFy = sFx + T3::FX_FLOATS;
  float* sQ = sFy + T3::FY_FLOATS;  // [NV][QROWS][BX]: U + h of rows -1 .. BY-1
  float* st = sQ + T3::Q_FLOATS;    // table rows of padded z k0 .. k0 + TROWS - 1
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + T3::SCRATCH);
  float* sdt = reinterpret_cast<float*>(bar + T3::NS);
  double* sred = reinterpret_cast<double*>(smem_raw + T3::SCRATCH + T3::NS * 8 + 16);
  const Geom& g = a.g;
  const Phys& p = a.p;
  const PhysF& pf = a.pf;
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int i0 = blockIdx.x * T3::BX, j0 = blockIdx.y * T3::BY;
  const int k0 = blockIdx.z * T3::CZ;
  const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
  const int k1 = min(k0 + T3::CZ, nz);
  const int pfirst = k0 - 2, plast = k1 + 1;  // planes needed by this chunk

  if (tid == 0) {
    const double dtd = a.dt_fixed > 0.0 ? a.dt_fixed : p.cfl / a.scal[a.slot];
    *sdt = (float)dtd;
    if (ST == 1 && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0) {
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
  int issued = min(pfirst + T3::NS - 1, plast);  // last plane whose copy has been issued
  if (tid == 0) {
    fence_proxy_async_smem();
    for (int pl = pfirst; pl <= issued; ++pl) issue(pl);
  }
  if constexpr (BG) {
    const float4* src = reinterpret_cast<const float4*>(a.tabr);
    float4* dst = reinterpret_cast<float4*>(st);
    constexpr int N4 = T3::TAB_FLOATS / 4;
    const int first4 = k0 * (TR_W / 4), last4 = a.tab_len * (TR_W / 4);
    for (int id = tid; id < N4; id += T3::NT)
      dst[id] = first4 + id < last4 ? src[first4 + id] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
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
  if (a.stall_ns > 0) {
    // Failure-detection test: wait on a barrier that expects 16 bytes no copy
    // delivers; the wait runs out with the next plane's copy possibly still
    // in flight, so the give-up path (flag, drain, return) runs in full.
    uint64_t* sb = reinterpret_cast<uint64_t*>(smem_raw + T3::SCRATCH + T3::NS * 8 + 16 + 8 * 8);
    if (tid == 0) {
      mbar_init(sb, 1);
      fence_mbar_init();
      mbar_expect_tx(sb, 16);
    }
    __syncthreads();
    if (__syncthreads_or(!mbar_wait_bounded(sb, 0u, (uint64_t)a.stall_ns))) {
      give_up();
      return;
    }
  }

  const int cx = lane, cy = tid >> 5;
  const int x = i0 + cx, y = j0 + cy;
  const bool colok = x < nx && y < ny;
  const int sxy = (cy + T3::YO) * T3::SXP + (cx + T3::XO);  // smem offset of my column in a plane
  auto ld = [&](int pl, int off, float (&u)[NV]) {
    const float* P = ring + slot_of(pl) * T3::PLANE + sxy + off;
#pragma unroll
    for (int v = 0; v < NV; ++v) u[v] = P[v * T3::PF];
  };
  // z window; table rows are indexed by padded z - k0 (interior z - k0 + 2)
  float u0[NV], u1[NV], h0[NV], Fm[NV];
  {
    float um[NV], umm[NV], hm[NV], qL[NV], qR[NV];
    ld(k0 - 2, 0, umm);
    ld(k0 - 1, 0, um);
    ld(k0, 0, u0);
    ld(k0 + 1, 0, u1);
    vslope_f<NV, BG>(umm, um, u0, st + 1 * TR_W, hm);
    vslope_f<NV, BG>(um, u0, u1, st + 2 * TR_W, h0);
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      qL[v] = um[v] + hm[v];
      qR[v] = u0[v] - h0[v];
    }
    face_vert_cm<NV, 2, BG, CM>(qL, qR, st + 2 * TR_W, pf, Fm);
  }
  float rmax = 0.0f;
  bool ok_all = true;
  const float idx = 0.5f * pf.inv_dx[0], idy = 0.5f * pf.inv_dx[1], idz = 0.5f * pf.inv_dx[2];  // faces hold 2F
  const int64_t fs = g.fstride;
  const bool xyghost = x < RSST_G || x >= nx - RSST_G || y < RSST_G || y >= ny - RSST_G;
  const int64_t o0 = pidx(g, x, y, k0);
  float bnext[NV] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
  if (ST == 2 && colok) {
#pragma unroll
    for (int v = 0; v < NV; ++v) bnext[v] = a.base[v * fs + o0];
  }
  // A. y half slope of my cell in plane pl (value u): its upper face state
  // to shared memory, its lower one kept in qBot; the first warp also writes
  // row -1's upper state, the last warp keeps row BY's lower state in qBotN.
  // Done for plane k at the end of step C of plane k-1 (the exchange array is
  // free once step B has read it), so a plane takes two block barriers.
  float qBot[NV], qBotN[NV];
  auto ystates = [&](int pl, const float (&u)[NV]) {
    const float* Pc = ring + slot_of(pl) * T3::PLANE + sxy;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const float um = Pc[v * T3::PF - T3::SXP], up = Pc[v * T3::PF + T3::SXP];
      const float h = half_mc_f(u[v] - um, up - u[v]);
      sQ[(v * T3::QROWS + cy + 1) * T3::BX + cx] = u[v] + h;
      qBot[v] = u[v] - h;
    }
    if (cy == 0) {
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const float* c = Pc + v * T3::PF - T3::SXP;  // row -1
        const float um = c[-T3::SXP], uu = c[0], up = c[T3::SXP];
        sQ[(v * T3::QROWS + 0) * T3::BX + cx] = uu + half_mc_f(uu - um, up - uu);
      }
    }
    if (cy == T3::BY - 1) {
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const float* c = Pc + v * T3::PF + T3::SXP;  // row BY
        const float um = c[-T3::SXP], uu = c[0], up = c[T3::SXP];
        qBotN[v] = uu - half_mc_f(uu - um, up - uu);
      }
    }
  };
  ystates(k0, u0);

#pragma unroll 1
  for (int k = k0; k < k1; ++k) {
    // everyone sees plane k+2 and the slot of plane k-2 is free
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
    const float* P = ring + slot_of(k) * T3::PLANE;
    float4 cb = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    if constexpr (BG) cb = *reinterpret_cast<const float4*>(st + rz * TR_W + TR_RHO0);
    // B. y faces, then the x faces of the plane
    {
      float qL[NV], G[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) qL[v] = sQ[(v * T3::QROWS + cy) * T3::BX + cx];  // row cy-1, upper state
      face_flat_cm<NV, 1, BG, CM>(qL, qBot, cb, pf, G);
#pragma unroll
      for (int v = 0; v < NV; ++v) sFy[(v * (T3::BY + 1) + cy) * T3::BX + cx] = G[v];
      if (cy == T3::BY - 1) {  // the face above the block
#pragma unroll
        for (int v = 0; v < NV; ++v) qL[v] = sQ[(v * T3::QROWS + T3::BY) * T3::BX + cx];
        face_flat_cm<NV, 1, BG, CM>(qL, qBotN, cb, pf, G);
#pragma unroll
        for (int v = 0; v < NV; ++v) sFy[(v * (T3::BY + 1) + T3::BY) * T3::BX + cx] = G[v];
      }
      for (int c = cy; c < T3::NCHUNK2; c += T3::NT / 32) {
        int A = 62 * c + 2 * lane;  // my two cells A, A + 1 (same row)
        const bool inb = A < T3::BY * T3::CW2;
        A = inb ? A : T3::BY * T3::CW2 - 2;  // keeps the loads inside the box
        const int row = A / T3::CW2;
        const int ca = A - row * T3::CW2 - 1;  // tile column of A: -1 .. BX + 1
        const float* ur = P + (row + T3::YO) * T3::SXP + T3::XO + ca;
        float qRl[NV], qLl[NV], qLi[NV], qRi[NV], G[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          const float* uv = ur + v * T3::PF;
          const float am = uv[-1], ua = uv[0], ub = uv[1], bp = uv[2];
          const float d1 = ua - am, d2 = ub - ua, d3 = bp - ub;
          const float ha = half_mc_f(d1, d2), hb = half_mc_f(d2, d3);
          qRl[v] = ua - ha;
          qLi[v] = ua + ha;
          qRi[v] = ub - hb;
          qLl[v] = __shfl_up_sync(0xffffffffu, ub + hb, 1);
        }
        face_flat_cm<NV, 0, BG, CM>(qLi, qRi, cb, pf, G);  // face between A and A + 1: index ca + 1
        if (inb && ca + 1 <= T3::BX) {
#pragma unroll
          for (int v = 0; v < NV; ++v) sFx[(v * T3::BY + row) * T3::FXW + ca + 1] = G[v];
        }
        face_flat_cm<NV, 0, BG, CM>(qLl, qRl, cb, pf, G);  // face between A - 1 and A: index ca
        if (inb && lane > 0 && ca >= 0 && ca <= T3::BX) {
#pragma unroll
          for (int v = 0; v < NV; ++v) sFx[(v * T3::BY + row) * T3::FXW + ca] = G[v];
        }
      }
    }
    __syncthreads();
    // C. advance my column
    float u2[NV], h1[NV], Fp[NV];
    ld(k + 2, 0, u2);
    vslope_f<NV, BG>(u0, u1, u2, st + (rz + 1) * TR_W, h1);
    {
      float qL[NV], qR[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        qL[v] = u0[v] + h0[v];
        qR[v] = u1[v] - h1[v];
      }
      face_vert_cm<NV, 2, BG, CM>(qL, qR, st + (rz + 1) * TR_W, pf, Fp);
    }
    float bv[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) bv[v] = bnext[v];
    if (ST == 2 && colok && k + 1 < k1) {
      const int64_t on = o0 + (int64_t)(k + 1 - k0) * g.plane;
#pragma unroll
      for (int v = 0; v < NV; ++v) bnext[v] = a.base[v * fs + on];
    }
    float L[NV], Dl[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const float* fx = sFx + (v * T3::BY + cy) * T3::FXW + cx;
      const float* fy = sFy + (v * (T3::BY + 1) + cy) * T3::BX + cx;
      L[v] = fmaf(-(Fp[v] - Fm[v]), idz, fmaf(-(fx[1] - fx[0]), idx, -(fy[T3::BX] - fy[0]) * idy));
    }
    float rho0 = 0.0f, P0 = 0.0f;
    if constexpr (BG) {
      const float* tr = st + rz * TR_W;
      const float4 r0 = *reinterpret_cast<const float4*>(tr + TR_R0);
      const float4 d0 = *reinterpret_cast<const float4*>(tr + TR_R0 + 4);  // R0[4], D0 rho, mv, E
      rho0 = cb.x;
      P0 = cb.y;
      Dl[0] = L[0] + d0.y;
      Dl[1] = L[1];
      Dl[2] = L[2];
      Dl[3] = L[3] + d0.z;
      Dl[4] = L[4] + d0.w;
      L[0] += r0.x;
      L[1] += r0.y;
      L[2] += r0.z;
      L[3] += r0.w;
      L[4] += d0.x;
    } else {
#pragma unroll
      for (int v = 0; v < NV; ++v) Dl[v] = L[v];
    }
    float u[NV], rate;
    bool ok;
    cell_lean<NV, FORM, CM, ST>(u0, L, Dl, rho0, P0, pf, p.variant, p.has_grav != 0, ST, dt, bv, u, rate, ok);
    if (colok) {
      if (ST == 2) {
        rmax = fmaxf(rmax, rate);
        ok_all = ok_all && ok;
      }
      const int64_t o = o0 + (int64_t)(k - k0) * g.plane;
#pragma unroll
      for (int v = 0; v < NV; ++v) a.out[v * fs + o] = u[v];
      if (xyghost || k < RSST_G || k >= nz - RSST_G) store_mirror_ghosts<float, 5>(a.out, g, p, x, y, k, u);
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      u0[v] = u1[v];
      u1[v] = u2[v];
      h0[v] = h1[v];
      Fm[v] = Fp[v];
    }
    if (k + 1 < k1) ystates(k + 1, u0);  // step A of the next plane (resident: plane k+2 was waited for)
  }
  if (ST == 2) {
    if (!ok_all) atomicOr(a.flag, RSST_FLAG_NONPHYSICAL);
    block_max_to<T3::NT>((double)rmax, a.scal + (a.slot ^ 1), sred);
  }
}

template <int VERT, int FORM, int CM, int ST>
static int launch3d(const CUtensorMap* tin, const StageArgs<float>& a, cudaStream_t s) {
  static std::atomic<unsigned long long> attr{0};
  if (set_smem_limit_once(stage3d_tma_kernel<VERT, FORM, CM, ST>, T3::SMEM, attr) != cudaSuccess) {
    rsst_set_error("cudaFuncSetAttribute failed for the 3D float32 TMA stage kernel");
    return RSST_ECUDA;
  }
  dim3 grid((a.g.n[0] + T3::BX - 1) / T3::BX, (a.g.n[1] + T3::BY - 1) / T3::BY, (a.g.n[2] + T3::CZ - 1) / T3::CZ);
  stage3d_tma_kernel<VERT, FORM, CM, ST><<<grid, T3::NT, T3::SMEM, s>>>(*tin, a);
  return RSST_OK;
}

template <int VERT, int FORM>
static int launch3d_form(const CUtensorMap* tin, const StageArgs<float>& a, cudaStream_t s) {
  const bool cm = a.pf.use_cmax != 0;
  if (a.stage == 1) return cm ? launch3d<VERT, FORM, 1, 1>(tin, a, s) : launch3d<VERT, FORM, 0, 1>(tin, a, s);
  return cm ? launch3d<VERT, FORM, 1, 2>(tin, a, s) : launch3d<VERT, FORM, 0, 2>(tin, a, s);
}

// Every form of one background case (VERT = 2: background along z; -1: none).
template <int VERT>
static int launch3d_vert(const CUtensorMap* tin, const StageArgs<float>& a, cudaStream_t s) {
  switch (a.p.variant) {
    case RSST_EULER: return launch3d_form<VERT, RSST_EULER>(tin, a, s);
    case RSST_DVS: return launch3d_form<VERT, RSST_DVS>(tin, a, s);
    case RSST_PVS: return launch3d_form<VERT, RSST_PVS>(tin, a, s);
    case RSST_DMS: return launch3d_form<VERT, RSST_DMS>(tin, a, s);
    case RSST_PMS: return launch3d_form<VERT, RSST_PMS>(tin, a, s);
    default: return launch3d_form<VERT, RSST_PD>(tin, a, s);
  }
}

}  // namespace rsst
