// Float32 perturbation arithmetic of the TMA stage kernels (2D and 3D),
// arranged for few instructions per cell.
//
// The state is U = U0 + U1, U0 = (rho0, 0, E0) a float64 background that
// depends only on the vertical index (or is absent) and U1 the stored
// float32 perturbation; every term that feeds an update is formed from
// perturbation-sized quantities (see rsst_math_fp32.cuh for the splitting).
// Compared with the generic float32 kernel:
//  - slopes are half slopes h (face states U +- h) computed once per cell
//    and axis;
//  - faces carry twice the LLF flux, 2F = F(qL) + F(qR) - alpha (qR - qL),
//    the exact 1/2 folding into 1/dx;
//  - the background comes from one row-major table row per vertical index
//    (read as float4; all lanes of a warp share it);
//  - the form, the C_max law and the stage can be compile-time constants
//    (template arguments; -1 or 0 reads them at run time), so a launch
//    carries no per-cell branches on them.
#pragma once

#include "rsst_internal.h"
#include "rsst_math_fp32.cuh"

namespace rsst {

// Half the monotonized-central slope (Sec. 4.2): 0 unless a and b have the
// same sign, else the smallest in magnitude of a, b, (a+b)/4 with the sign
// of a.  Branch-free in six instructions: with sa the sign bit of a,
// m = max(0, min(|a|, sa*b, |a+b|/4)) is that magnitude when the signs agree
// (sa*b = |b|) and 0 when they differ (sa*b < 0); a zero a or b gives 0
// either way.  The result is m with a's sign.
__device__ __forceinline__ float half_mc_f(float a, float b) {
  const unsigned sa = __float_as_uint(a) & 0x80000000u;
  const float bs = __uint_as_float(__float_as_uint(b) ^ sa);
  const float t = 0.25f * fabsf(a + b);
  float m;
  asm("min.f32 %0, %1, %2, %3;" : "=f"(m) : "f"(fabsf(a)), "f"(bs), "f"(t));
  m = fmaxf(m, 0.0f);
  return __uint_as_float(__float_as_uint(m) | sa);
}

// Half the perturbation slope of a component whose background varies along
// the axis: [lin_B(d1) + lin_B(d0) - MC(d0)] / 2, B the branch MC takes on
// the full differences d0 + d1 (ties in the order 2a, 2b, (a+b)/2, as the
// oracle's limiter).  t points at the component's six table entries: d0L,
// d0R and the four halved background terms.
__device__ __forceinline__ float half_bg_slope_f(const float* t, float da, float db) {
  const float A = t[0] + da, B = t[1] + db;
  const float aa = fabsf(A), bb = fabsf(B), cc = 0.25f * fabsf(A + B);
  const bool same = A * B > 0.0f;
  const bool p1 = aa <= bb && aa <= cc;
  const bool p2 = !p1 && bb <= cc;
  const float lin = p1 ? da : (p2 ? db : 0.25f * (da + db));
  const float del = p1 ? t[3] : (p2 ? t[4] : t[5]);
  return same ? lin + del : t[2];
}

// a/xi from gx P/rho: (a/xi)^2 for a constant xi, a^2 under the C_max law
// (xi = [1 + (a/C_max)^4]^(1/4), Eq. cx: a/xi = sqrt(a^2 / sqrt(w)),
// w = 1 + a^4/C_max^4).
template <bool CMAX>
__device__ __forceinline__ float sound_x(float a2x, const PhysF& pf) {
  if constexpr (CMAX) return sqrt_f(a2x * rcp_f(sqrt_f(fmaf(a2x * a2x, pf.inv_cmax4, 1.0f))));
  return sqrt_f(a2x);
}

// F(U0 + q) - F(U0) along D of a face state q (perturbation) about a
// background state (rho0, P0, gx P0, H0 = E0 + P0), with the full
// c_tot = |V| + a/xi; WANT_DC also gives dc = c_tot - c0 from
// perturbation-sized terms: (a/xi)^2 - (a0/xi)^2 = gx (P1 rho0 - P0 rho1) /
// (rho rho0), divided by a/xi + a0/xi (constant xi; under the C_max law
// dc = |V| + a/xi(a) - c0).  Without a background every background argument
// is 0 and this is the Euler flux of the full state.
template <int NV, int D, bool WANT_DC, bool CMAX>
__device__ __forceinline__ void flux_lean(const float (&q)[NV], float rho0, float P0, float gxP0, float H0, float a0x,
                                          float gxr0, float c0, const PhysF& pf, float (&F)[NV], float& c, float& dc) {
  constexpr int ND = NV - 2;
  const float rho = rho0 + q[0];
  const float ir = rcp_f(rho);
  float v[ND];
#pragma unroll
  for (int e = 0; e < ND; ++e) v[e] = q[1 + e] * ir;
  float v2 = v[0] * v[0];
#pragma unroll
  for (int e = 1; e < ND; ++e) v2 = fmaf(v[e], v[e], v2);
  const float P1 = fmaf(-pf.hgm1, rho * v2, pf.gm1 * q[NV - 1]);
  const float a2x = fmaf(pf.gx, P1, gxP0) * ir;
  const float vm = sqrt_f(v2);
  const float ax = sound_x<CMAX>(a2x, pf);
  c = vm + ax;
  if constexpr (WANT_DC) {
    if constexpr (CMAX) {
      dc = vm + (ax - c0);
    } else {
      const float da2x = fmaf(P1, rho0, -P0 * q[0]) * ir * gxr0;
      dc = fmaf(da2x, rcp_f(ax + a0x), vm);
    }
  }
  F[0] = q[1 + D];
#pragma unroll
  for (int e = 0; e < ND; ++e) F[1 + e] = e == D ? fmaf(q[1 + e], v[D], P1) : q[1 + e] * v[D];
  F[NV - 1] = (H0 + q[NV - 1] + P1) * v[D];
}

// Twice the LLF flux of a face across which the background is constant
// (cb = rho0, P0, gx P0, H0 of the row; zero without a background).
template <int NV, int D, bool BG, bool CMAX>
__device__ __forceinline__ void face_flat(const float (&qL)[NV], const float (&qR)[NV], const float4 cb,
                                          const PhysF& pf, float (&G)[NV]) {
  float FL[NV], FR[NV], cL, cR, dum;
  if constexpr (BG) {
    flux_lean<NV, D, false, CMAX>(qL, cb.x, cb.y, cb.z, cb.w, 0.0f, 0.0f, 0.0f, pf, FL, cL, dum);
    flux_lean<NV, D, false, CMAX>(qR, cb.x, cb.y, cb.z, cb.w, 0.0f, 0.0f, 0.0f, pf, FR, cR, dum);
  } else {
    flux_lean<NV, D, false, CMAX>(qL, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, pf, FL, cL, dum);
    flux_lean<NV, D, false, CMAX>(qR, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, pf, FR, cR, dum);
  }
  const float alpha = fmaxf(cL, cR);
#pragma unroll
  for (int v = 0; v < NV; ++v) G[v] = fmaf(-alpha, qR[v] - qL[v], FL[v] + FR[v]);
}

// Twice the LLF flux of a face across the vertical axis D; trow = the face's
// table row.  The background's face jump U0R - U0L also enters:
// -(alpha - alpha0)(U0R - U0L), with alpha - alpha0 from the per-side dc and
// the float64 difference g = c0L - c0R.
template <int NV, int D, bool CMAX>
__device__ __forceinline__ void face_vertical(const float (&qL)[NV], const float (&qR)[NV],
                                              const float* __restrict__ trow, const PhysF& pf, float (&G)[NV]) {
  const float4 fl = *reinterpret_cast<const float4*>(trow + TR_FL);
  const float4 fr = *reinterpret_cast<const float4*>(trow + TR_FR);
  const float4 fa = *reinterpret_cast<const float4*>(trow + TR_FA0X);
  const float4 fg = *reinterpret_cast<const float4*>(trow + TR_FG);  // g, alpha0, jump rho, jump E
  const float g = fg.x;
  const float c0L = g >= 0.0f ? fg.y : fg.y + g, c0R = g >= 0.0f ? fg.y - g : fg.y;
  float FL[NV], FR[NV], cL, cR, dcL, dcR;
  flux_lean<NV, D, true, CMAX>(qL, fl.x, fl.y, fl.z, fl.w, fa.x, fa.z, c0L, pf, FL, cL, dcL);
  flux_lean<NV, D, true, CMAX>(qR, fr.x, fr.y, fr.z, fr.w, fa.y, fa.w, c0R, pf, FR, cR, dcR);
  const float dalpha = g >= 0.0f ? fmaxf(dcL, dcR - g) : fmaxf(dcL + g, dcR);
  const float alpha = fg.y + dalpha;
#pragma unroll
  for (int v = 0; v < NV; ++v) G[v] = fmaf(-alpha, qR[v] - qL[v], FL[v] + FR[v]);
  G[0] = fmaf(-dalpha, fg.z, G[0]);
  G[NV - 1] = fmaf(-dalpha, fg.w, G[NV - 1]);
}

// C_max law fixed at compile time (CM = 0 or 1) or read at run time (CM < 0).
template <int NV, int D, bool BG, int CM>
__device__ __forceinline__ void face_flat_cm(const float (&qL)[NV], const float (&qR)[NV], const float4 cb,
                                             const PhysF& pf, float (&G)[NV]) {
  if constexpr (CM >= 0) {
    face_flat<NV, D, BG, CM != 0>(qL, qR, cb, pf, G);
  } else {
    if (pf.use_cmax) face_flat<NV, D, BG, true>(qL, qR, cb, pf, G);
    else face_flat<NV, D, BG, false>(qL, qR, cb, pf, G);
  }
}
template <int NV, int D, bool BG, int CM>
__device__ __forceinline__ void face_vert_cm(const float (&qL)[NV], const float (&qR)[NV],
                                             const float* __restrict__ trow, const PhysF& pf, float (&G)[NV]) {
  if constexpr (!BG) {
    face_flat_cm<NV, D, false, CM>(qL, qR, make_float4(0.0f, 0.0f, 0.0f, 0.0f), pf, G);
  } else if constexpr (CM >= 0) {
    face_vertical<NV, D, CM != 0>(qL, qR, trow, pf, G);
  } else {
    if (pf.use_cmax) face_vertical<NV, D, true>(qL, qR, trow, pf, G);
    else face_vertical<NV, D, false>(qL, qR, trow, pf, G);
  }
}

// Half slopes across the vertical axis of the cell u0 between um and up;
// srow = the cell's table row (its background slope entries).
template <int NV, bool BG>
__device__ __forceinline__ void vslope_f(const float (&um)[NV], const float (&u0)[NV], const float (&up)[NV],
                                         const float* __restrict__ srow, float (&h)[NV]) {
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const float da = u0[v] - um[v], db = up[v] - u0[v];
    if (BG && (v == 0 || v == NV - 1))
      h[v] = half_bg_slope_f(srow + (v == 0 ? TR_SRHO : TR_SE), da, db);
    else
      h[v] = half_mc_f(da, db);
  }
}

// Reduced tendency, force and RK combine of one cell (Sec. 4.2 steps 6-8)
// from the stage state q (perturbation), the tendency L (divergence of the
// perturbation fluxes plus the background residual) and Dl (the full Euler
// tendency, for s); in stage 2 also the CFL rate and the physical check of
// the new state.  FORM < 0, CM < 0 and ST = 0 read the form, the C_max law
// and the stage at run time.
template <int NV, int FORM, int CM, int ST>
__device__ __forceinline__ void cell_lean(const float (&q)[NV], float (&L)[NV], const float (&Dl)[NV], float rho0,
                                          float P0, const PhysF& pf, int form_rt, bool has_grav, int stage_rt,
                                          float dt, const float (&b)[NV], float (&u)[NV], float& rate, bool& ok) {
  constexpr int ND = NV - 2;
  const int form = FORM >= 0 ? FORM : form_rt;
  const int stage = ST > 0 ? ST : stage_rt;
  const bool cmax = CM >= 0 ? CM != 0 : pf.use_cmax != 0;
  const float rho = rho0 + q[0];
  const float ir = rcp_f(rho);
  float v[ND];
#pragma unroll
  for (int e = 0; e < ND; ++e) v[e] = q[1 + e] * ir;
  float v2 = v[0] * v[0];
#pragma unroll
  for (int e = 1; e < ND; ++e) v2 = fmaf(v[e], v[e], v2);
  const float kin = 0.5f * rho * v2;
  const float P = fmaf(pf.gm1, q[NV - 1] - kin, P0);
  if (form != RSST_EULER) {
    const float fcell = cmax ? f_of_f(pf.gamma * P * ir, pf) : pf.f;
    const float hP = pf.gam_gm1 * P;  // e + P
    if (form == RSST_PVS || form == RSST_PMS || form == RSST_PD) {
      float vdm = v[0] * Dl[1];
#pragma unroll
      for (int e = 1; e < ND; ++e) vdm = fmaf(v[e], Dl[1 + e], vdm);
      const float fs = fcell * pf.gm1 * (fmaf(0.5f * v2, Dl[0], Dl[NV - 1]) - vdm);  // f dP
      if (form == RSST_PD) {
        L[NV - 1] = fmaf(-fs, pf.inv_gm1, L[NV - 1]);
      } else {
        const float igp = rcp_f(pf.gamma * P);  // 1/(rho a^2)
        const float w = fs * rho * igp;         // f dP / a^2
        L[0] -= w;
        if (form == RSST_PVS) {
#pragma unroll
          for (int e = 0; e < ND; ++e) L[1 + e] = fmaf(-w, v[e], L[1 + e]);
        }
        L[NV - 1] = fmaf(-fs * igp, form == RSST_PVS ? hP + kin : hP - kin, L[NV - 1]);
      }
    } else {  // DVS, DMS: s = drho
      const float fs = fcell * Dl[0];
      L[0] -= fs;
      if (form == RSST_DVS) {
#pragma unroll
        for (int e = 0; e < ND; ++e) L[1 + e] = fmaf(-fs, v[e], L[1 + e]);
      }
      L[NV - 1] = fmaf(-fs * ir, form == RSST_DVS ? hP + kin : hP - kin, L[NV - 1]);
    }
  }
  if (has_grav) {  // perturbation force: rho1 F and m.F (rho0 F is in the background residual)
    float mg = q[1] * pf.grav[0];
#pragma unroll
    for (int e = 0; e < ND; ++e) {
      L[1 + e] = fmaf(q[0], pf.grav[e], L[1 + e]);
      if (e > 0) mg = fmaf(q[1 + e], pf.grav[e], mg);
    }
    L[NV - 1] += mg;
  }
  rate = 0.0f;
  ok = true;
  if (stage == 1) {
#pragma unroll
    for (int k = 0; k < NV; ++k) u[k] = fmaf(dt, L[k], q[k]);
  } else {
#pragma unroll
    for (int k = 0; k < NV; ++k) u[k] = 0.5f * (b[k] + fmaf(dt, L[k], q[k]));
    const float rn = rho0 + u[0];
    const float irn = rcp_f(rn);
    float w[ND];
#pragma unroll
    for (int e = 0; e < ND; ++e) w[e] = u[1 + e] * irn;
    float w2 = w[0] * w[0];
#pragma unroll
    for (int e = 1; e < ND; ++e) w2 = fmaf(w[e], w[e], w2);
    const float Pn = fmaf(pf.gm1, fmaf(-0.5f * rn, w2, u[NV - 1]), P0);
    // rho and P positive and finite (a NaN or infinite component reaches one of them)
    ok = (__float_as_uint(rn) - 1u < 0x7f7fffffu) && (__float_as_uint(Pn) - 1u < 0x7f7fffffu);
    if (ok) {
      const float a2x = pf.gx * Pn * irn;
      const float ax = cmax ? sound_x<true>(a2x, pf) : sound_x<false>(a2x, pf);
      rate = (sqrt_f(w2) + ax) * pf.sum_inv_dx;
    }
  }
}

}  // namespace rsst
