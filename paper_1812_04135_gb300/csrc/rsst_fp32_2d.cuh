// 2D float32 perturbation tile routine (see rsst_fp32_2d.cu for the layout).
//
// The state is U = U0 + U1, U0 = (rho0, 0, 0, E0) a float64 background that
// varies along y only (or is absent), U1 the stored float32 perturbation.
// Every term that feeds an update is formed from perturbation-sized
// quantities (see rsst_math_fp32.cuh for the splitting), with the arithmetic
// arranged for few instructions per cell:
//  - each cell's MC slope is computed once per axis, as a half slope h
//    (face states U +- h); along x a lane hands its cell's right face state
//    to the next lane by a warp shuffle, along y the column march carries it;
//  - faces hold twice the LLF flux, 2F = F(qL) + F(qR) - alpha (qR - qL),
//    and the exact 1/2 folds into 1/dx;
//  - the background enters through one row-major table row per vertical
//    index, read as float4 (broadcast: all lanes of a warp share the row).
#pragma once

#include "rsst_common.cuh"
#include "rsst_internal.h"
#include "rsst_fp32_lean.cuh"
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
  static constexpr int TAB_FLOATS = TR_W * SYP;
  static constexpr size_t SCRATCH = (size_t)(U_FLOATS + FX_FLOATS + TAB_FLOATS) * 4;
  // x-face pass: the slope cells -1 .. BX of every row, in one flat list
  // walked by warps in chunks of 32 cells that overlap by one
  // x-face pass: the slope cells -1 .. BX of every row (padded to CW2, an
  // even count, with two cells beyond BX) form one flat list; a lane takes
  // two neighbouring cells, a warp chunk 64 cells, chunks start every 62
  static constexpr int CW2 = BX + 4;
  static constexpr int NCHUNK2 = (BY * CW2 - 2 + 61) / 62;
  static constexpr uint32_t BOX_BYTES = U_FLOATS * 4;
  static constexpr size_t smem_bytes() { return SCRATCH + 16 + 8 * 8 + 512 + 128; }
  static_assert(BY % SEG == 0, "column segments must tile BY");
  static_assert(BX % 32 == 0, "a warp of the column march covers 32 columns of one segment");
  static_assert((U_FLOATS + FX_FLOATS) % 4 == 0, "the table rows start on a 16-byte boundary");
  static_assert(NT % 32 == 0, "whole warps");
  static_assert(SCRATCH % 8 == 0, "the barriers after the scratch area need 8-byte alignment");
  static_assert(SXP <= 256 && SYP <= 256, "TMA box dimensions are at most 256");
};

using T2 = T2Cfg<128, 8, 8>;  // single-run default

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
  const float* tabr;  // row-major background table, or null (no background)
  int tab_len;
  unsigned int* flag;
  int stage;
  int64_t stall_ns;  // > 0 only in failure-detection tests (see tile2d_f)
};

// Process tile (tx, ty) of run r: returns false if a bounded wait gave up
// (flag set, nothing left in flight).  Accumulates the stage-2 CFL rate
// maximum and physical check.  The caller initialised the barrier; `phase` is
// its current parity.  FORM, CM and ST fix the form, the C_max law and the
// stage at compile time (-1, -1, 0: read from the run).
template <class T2, int VERT, int FORM, int CM, int ST>
__device__ __forceinline__ bool tile2d_f(const CUtensorMap* tin, const TileRun& r, float dt, int tx, int ty,
                                         unsigned char* smem, uint32_t& phase, float& rmax, bool& ok_all) {
  constexpr int NV = 4;
  constexpr bool BG = VERT >= 0;
  constexpr int PL = T2::SYP * T2::SXP;  // floats per field in the box
  float* sU = reinterpret_cast<float*>(smem);
  float* sFx = sU + T2::U_FLOATS;
  float* st = sFx + T2::FX_FLOATS;  // table rows of padded y j0 .. j0 + SYP - 1
  uint64_t* bar = t2_barrier<T2>(smem);
  const Geom& g = r.g;
  const PhysF& pf = r.pf;
  const int stage = ST > 0 ? ST : r.stage;
  const int i0 = tx * T2::BX, j0 = ty * T2::BY;
  const int tid = threadIdx.x;

  __syncthreads();  // previous tile's shared-memory reads are done
  if (tid == 0) {
    fence_proxy_async_smem();
    mbar_expect_tx(bar, T2::BOX_BYTES);
    tma_load_3d(sU, tin, bar, i0 + g.xoff - T2::XO, j0, 0);
  }
  if constexpr (BG) {
    // SYP consecutive table rows (16-byte aligned) as float4
    const float4* src = reinterpret_cast<const float4*>(r.tabr);
    float4* dst = reinterpret_cast<float4*>(st);
    constexpr int N4 = T2::TAB_FLOATS / 4;
    const int first4 = j0 * (TR_W / 4), last4 = r.tab_len * (TR_W / 4);
    for (int id = tid; id < N4; id += T2::NT)
      dst[id] = first4 + id < last4 ? src[first4 + id] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
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
    // the bounded wait runs out and the give-up path is taken.
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

  const int nx = g.n[0], ny = g.n[1];
  const int lane = tid & 31;
  // ---- x faces.  The slope cells of every row form one flat list; chunk k
  // holds cells 62k .. 62k + 63, lane l the pair A = 62k + 2l, A + 1 (a pair
  // never straddles two rows: the rows hold an even number of cells).  The
  // lane takes both cells' half slopes (four loads and three differences per
  // field), forms the face between its two cells, and the face on A's left
  // from its own state A - h_A and the state B + h_B passed one lane up.  So
  // every face of the tile is formed (the two cells shared by consecutive
  // chunks give one face twice, with equal values), no slope is recomputed
  // within a chunk and no lane runs alone; lane 0's left face and faces
  // across rows are left out.
  {
    const int nwarp = T2::NT / 32;
    for (int k = tid >> 5; k < T2::NCHUNK2; k += nwarp) {
      int A = 62 * k + 2 * lane;  // my two cells A, A + 1 (same row: rows hold an even CW2 cells)
      const bool inb = A < T2::BY * T2::CW2;
      A = inb ? A : T2::BY * T2::CW2 - 2;  // keeps the loads inside the box
      const int row = A / T2::CW2;
      const int ca = A - row * T2::CW2 - 1;  // tile column of A: -1 .. BX + 1
      const int sr = row + 2;
      const float* ur = sU + sr * T2::SXP + T2::XO + ca;
      float qRl[NV], qLl[NV], qLi[NV], qRi[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const float* uv = ur + v * PL;
        const float am = uv[-1], a = uv[0], b = uv[1], bp = uv[2];
        const float d1 = a - am, d2 = b - a, d3 = bp - b;
        const float ha = half_mc_f(d1, d2), hb = half_mc_f(d2, d3);
        qRl[v] = a - ha;
        qLi[v] = a + ha;
        qRi[v] = b - hb;
        qLl[v] = __shfl_up_sync(0xffffffffu, b + hb, 1);
      }
      float4 cb = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      if constexpr (BG) cb = *reinterpret_cast<const float4*>(st + sr * TR_W + TR_RHO0);
      const bool rowok = inb && j0 + row < ny;
      float G[NV];
      face_flat_cm<NV, 0, BG, CM>(qLi, qRi, cb, pf, G);  // face between A and A + 1: face index ca + 1
      if (rowok && ca + 1 <= T2::BX && i0 + ca + 1 <= nx) {
#pragma unroll
        for (int v = 0; v < NV; ++v) sFx[(v * T2::BY + row) * T2::FXW + ca + 1] = G[v];
      }
      face_flat_cm<NV, 0, BG, CM>(qLl, qRl, cb, pf, G);  // face between A - 1 and A: face index ca
      if (rowok && lane > 0 && ca >= 0 && ca <= T2::BX && i0 + ca <= nx) {
#pragma unroll
        for (int v = 0; v < NV; ++v) sFx[(v * T2::BY + row) * T2::FXW + ca] = G[v];
      }
    }
  }
  __syncthreads();

  // ---- column march with the fused epilogue: each thread owns tile column
  // col, rows jb .. jb + SEG - 1; a register window carries the cell states,
  // the y half slope and the lower face's flux.
  const int col = tid % T2::BX;
  const int jb = (tid / T2::BX) * T2::SEG;
  const int x = i0 + col;
  if (x < nx && j0 + jb < ny) {
    const float* uc = sU + T2::XO + col;
    auto ld = [&](int srow, float (&u)[NV]) {
#pragma unroll
      for (int v = 0; v < NV; ++v) u[v] = uc[v * PL + srow * T2::SXP];
    };
    float u0[NV], u1[NV], h0[NV], Fm[NV];
    {
      float umm[NV], um[NV], hm[NV];
      // cells jb-2 .. jb+1 live at smem rows jb .. jb+3
      ld(jb, umm);
      ld(jb + 1, um);
      ld(jb + 2, u0);
      ld(jb + 3, u1);
      vslope_f<NV, BG>(umm, um, u0, st + (jb + 1) * TR_W, hm);  // cell jb-1
      vslope_f<NV, BG>(um, u0, u1, st + (jb + 2) * TR_W, h0);   // cell jb
      float qL[NV], qR[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        qL[v] = um[v] + hm[v];
        qR[v] = u0[v] - h0[v];
      }
      face_vert_cm<NV, 1, BG, CM>(qL, qR, st + (jb + 2) * TR_W, pf, Fm);
    }
    const float idx = 0.5f * pf.inv_dx[0], idy = 0.5f * pf.inv_dx[1];  // the faces hold 2F
    const int64_t fs = g.fstride;
    const bool xghost = x < RSST_G || x >= nx - RSST_G;
    const int64_t o0 = pidx(g, x, j0 + jb, 0);
    // stage 2: U^n of the next row's cell is loaded one row ahead, so its
    // global-memory latency overlaps a row of arithmetic
    float bnext[NV] = {0.0f, 0.0f, 0.0f, 0.0f};
    if (stage == 2) {
#pragma unroll
      for (int v = 0; v < NV; ++v) bnext[v] = r.base[v * fs + o0];
    }
#pragma unroll 1
    for (int jj = 0; jj < T2::SEG; ++jj) {
      const int j = jb + jj;  // tile row of the cell
      if (j0 + j >= ny) break;
      float bv[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) bv[v] = bnext[v];
      if (stage == 2 && jj + 1 < T2::SEG && j0 + j + 1 < ny) {
        const int64_t on = o0 + (int64_t)(jj + 1) * g.pitch;
#pragma unroll
        for (int v = 0; v < NV; ++v) bnext[v] = r.base[v * fs + on];
      }
      const int sr = j + 2;  // its smem row
      float u2[NV], h1[NV], Fp[NV];
      ld(j + 4, u2);                                          // cell j+2
      vslope_f<NV, BG>(u0, u1, u2, st + (j + 3) * TR_W, h1);  // cell j+1
      {
        float qL[NV], qR[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          qL[v] = u0[v] + h0[v];
          qR[v] = u1[v] - h1[v];
        }
        face_vert_cm<NV, 1, BG, CM>(qL, qR, st + (j + 3) * TR_W, pf, Fp);
      }
      float L[NV], Dl[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const float* fr = sFx + (v * T2::BY + j) * T2::FXW + col;
        L[v] = fmaf(-(Fp[v] - Fm[v]), idy, -(fr[1] - fr[0]) * idx);
      }
      float rho0 = 0.0f, P0 = 0.0f;
      if constexpr (BG) {
        const float* tr = st + sr * TR_W;
        const float4 cb = *reinterpret_cast<const float4*>(tr + TR_RHO0);
        const float4 r0 = *reinterpret_cast<const float4*>(tr + TR_R0);
        const float4 d0 = *reinterpret_cast<const float4*>(tr + TR_R0 + 4);  // R0[4] (unused in 2D), D0 rho, mv, E
        rho0 = cb.x;
        P0 = cb.y;
        Dl[0] = L[0] + d0.y;
        Dl[1] = L[1];
        Dl[2] = L[2] + d0.z;
        Dl[3] = L[3] + d0.w;
        L[0] += r0.x;
        L[1] += r0.y;
        L[2] += r0.z;
        L[3] += r0.w;
      } else {
#pragma unroll
        for (int v = 0; v < NV; ++v) Dl[v] = L[v];
      }
      const int y = j0 + j;
      const int64_t o = o0 + (int64_t)jj * g.pitch;
      float u[NV], rate;
      bool ok;
      cell_lean<NV, FORM, CM, ST>(u0, L, Dl, rho0, P0, pf, r.p.variant, r.p.has_grav != 0, stage, dt, bv, u, rate,
                                  ok);
      if (stage == 2) {
        rmax = fmaxf(rmax, rate);
        ok_all = ok_all && ok;
      }
#pragma unroll
      for (int v = 0; v < NV; ++v) r.out[v * fs + o] = u[v];
      if (xghost || y < RSST_G || y >= ny - RSST_G) store_mirror_ghosts<float, 4>(r.out, g, r.p, x, y, 0, u);
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        u0[v] = u1[v];
        u1[v] = u2[v];
        h0[v] = h1[v];
        Fm[v] = Fp[v];
      }
    }
  }
  return true;
}

}  // namespace rsst
