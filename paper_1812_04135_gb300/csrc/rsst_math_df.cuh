// Double-float arithmetic and the RSST step in it.
//
// A double-float is the unevaluated sum hi + lo of two float32 values with
// |lo| <= ulp(hi)/2: a 48-bit significand (relative rounding ~2^-48) in the
// float32 exponent range, computed entirely on the float32 pipe.  The
// operations are the classical error-free transformations with a fused
// multiply-add (Dekker 1971; Knuth, TAOCP vol. 2, Sec. 4.2.2; Shewchuk 1997):
//   two_sum(a, b):  s = a + b exactly as s + e,
//   two_prod(a, b): a * b exactly as p + e with e = fma(a, b, -p),
// followed by renormalisation.  Reciprocal and square root take the float32
// hardware value and one Newton step carried in double-float.
//
// The step functions mirror the float64 ones (rsst_math_fp64.cuh) term for
// term, with the same readings of Sec. 4.2 (MC limiter, LLF with
// c_tot = |V| + a/xi, ties to the left state) and the same corrections
// (Sec. 3.2, App. A) and force (App. B).
#pragma once

#include "rsst_internal.h"

namespace rsst {

struct df {
  float hi, lo;
};

__device__ __forceinline__ df df_make(float h, float l = 0.0f) { return {h, l}; }

__device__ __forceinline__ df fast_two_sum(float a, float b) {  // |a| >= |b|
  const float s = a + b;
  return {s, b - (s - a)};
}
__device__ __forceinline__ df two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return {s, (a - (s - bb)) + (b - bb)};
}

__device__ __forceinline__ df operator+(df x, df y) {
  const df s = two_sum(x.hi, y.hi);
  return fast_two_sum(s.hi, s.lo + (x.lo + y.lo));
}
__device__ __forceinline__ df operator-(df x) { return {-x.hi, -x.lo}; }
__device__ __forceinline__ df operator-(df x, df y) { return x + (-y); }
__device__ __forceinline__ df operator*(df x, df y) {
  const float p = x.hi * y.hi;
  float e = fmaf(x.hi, y.hi, -p);
  e = fmaf(x.hi, y.lo, e);
  e = fmaf(x.lo, y.hi, e);
  return fast_two_sum(p, e);
}
// exact scaling by a power of two
__device__ __forceinline__ df scale(df x, float p2) { return {x.hi * p2, x.lo * p2}; }

// 1/y: float32 reciprocal r0, then r0 + r0 (1 - y r0) with 1 - y r0 formed
// from the exact product y.hi * r0 = p + pe.
__device__ __forceinline__ df rcp(df y) {
  const float r0 = 1.0f / y.hi;
  const float p = y.hi * r0;
  const float pe = fmaf(y.hi, r0, -p);
  const float e = ((1.0f - p) - pe) - y.lo * r0;
  return fast_two_sum(r0, r0 * e);
}

// sqrt(x), 0 for x <= 0: s0 = sqrt(x.hi), then s0 + (x - s0^2)/(2 s0).
__device__ __forceinline__ df dsqrt(df x) {
  if (!(x.hi > 0.0f)) return {0.0f, 0.0f};
  const float s0 = sqrtf(x.hi);
  const float p = s0 * s0;
  const float pe = fmaf(s0, s0, -p);
  const float d = ((x.hi - p) - pe) + x.lo;
  return fast_two_sum(s0, d * (0.5f / s0));
}

__device__ __forceinline__ bool df_lt(df a, df b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
__device__ __forceinline__ bool df_le(df a, df b) { return a.hi < b.hi || (a.hi == b.hi && a.lo <= b.lo); }
__device__ __forceinline__ df df_abs(df a) { return a.hi < 0.0f ? -a : a; }
__device__ __forceinline__ bool df_pos(df a) { return a.hi > 0.0f || (a.hi == 0.0f && a.lo > 0.0f); }

__device__ __forceinline__ df df_from(double d) {
  const float h = __double2float_rn(d);
  return {h, __double2float_rn(d - (double)h)};
}
__device__ __forceinline__ double df_to(df x) { return (double)x.hi + (double)x.lo; }

// Constants of the step in double-float (split once on the host).
struct PhysDF {
  df gamma, gm1, hgm1, inv_gm1, inv_xi, f, inv_cmax4;
  df grav[3], inv_dx[3], sum_inv_dx;
  int variant, use_cmax, has_grav;
};

// MC limited slope (Sec. 4.2): 0 unless a, b are nonzero with one sign; else
// 2a if |a| <= |b| and 4|a| <= |a+b|, 2b if 4|b| <= |a+b|, else (a+b)/2.
__device__ __forceinline__ df mc_df(df a, df b) {
  const bool same = (a.hi > 0.0f && b.hi > 0.0f) || (a.hi < 0.0f && b.hi < 0.0f);
  if (!same) return {0.0f, 0.0f};
  const df s = a + b;
  const df aa = df_abs(a), bb = df_abs(b), ss = df_abs(s);
  if (df_le(aa, bb) && df_le(scale(aa, 4.0f), ss)) return scale(a, 2.0f);
  if (df_le(scale(bb, 4.0f), ss)) return scale(b, 2.0f);
  return scale(s, 0.5f);
}

__device__ __forceinline__ df sound_over_xi_df(df a2, const PhysDF& p) {
  if (p.use_cmax) return dsqrt(a2 * rcp(dsqrt(df_make(1.0f) + (a2 * a2) * p.inv_cmax4)));
  return dsqrt(a2) * p.inv_xi;
}
__device__ __forceinline__ df f_of_df(df a2, const PhysDF& p) {
  if (p.use_cmax) return df_make(1.0f) - rcp(dsqrt(df_make(1.0f) + (a2 * a2) * p.inv_cmax4));
  return p.f;
}

// Half the Euler flux along D and c_tot of one state.
template <int NV, int D>
__device__ __forceinline__ void euler_flux_df(const df (&q)[NV], const PhysDF& p, df (&F)[NV], df& c) {
  constexpr int ND = NV - 2;
  const df rho = q[0];
  const df ir = rcp(rho);
  df v[ND];
  df v2 = {0.0f, 0.0f};
#pragma unroll
  for (int e = 0; e < ND; ++e) {
    v[e] = q[1 + e] * ir;
    v2 = v2 + v[e] * v[e];
  }
  const df P = p.gm1 * q[NV - 1] - p.hgm1 * (rho * v2);
  c = dsqrt(v2) + sound_over_xi_df(p.gamma * P * ir, p);
  const df hv = scale(v[D], 0.5f);
  F[0] = scale(q[1 + D], 0.5f);
#pragma unroll
  for (int e = 0; e < ND; ++e) F[1 + e] = (e == D) ? q[1 + e] * hv + scale(P, 0.5f) : q[1 + e] * hv;
  F[NV - 1] = (q[NV - 1] + P) * hv;
}

template <int NV, int D>
__device__ __forceinline__ void llf_flux_df(const df (&qL)[NV], const df (&qR)[NV], const PhysDF& p, df (&F)[NV]) {
  df FL[NV], FR[NV], cL, cR;
  euler_flux_df<NV, D>(qL, p, FL, cL);
  euler_flux_df<NV, D>(qR, p, FR, cR);
  const df halpha = scale(df_le(cR, cL) ? cL : cR, 0.5f);
#pragma unroll
  for (int k = 0; k < NV; ++k) F[k] = (FL[k] + FR[k]) - halpha * (qR[k] - qL[k]);
}

// Reduced tendency and force (Sec. 3.2 Eqs. pvs_dt / pvs_dt_dpr, App. A, App. B).
template <int NV>
__device__ __forceinline__ void rsst_rhs_df(const df (&q)[NV], df (&dU)[NV], const PhysDF& p) {
  constexpr int ND = NV - 2;
  const df rho = q[0];
  if (p.variant != RSST_EULER) {
    const df ir = rcp(rho);
    df v[ND];
    df v2 = {0.0f, 0.0f}, vdm = {0.0f, 0.0f};
#pragma unroll
    for (int e = 0; e < ND; ++e) {
      v[e] = q[1 + e] * ir;
      v2 = v2 + v[e] * v[e];
      vdm = vdm + v[e] * dU[1 + e];
    }
    const df P = p.gm1 * q[NV - 1] - p.hgm1 * (rho * v2);
    const df e_int = P * p.inv_gm1;
    const df kin = scale(rho * v2, 0.5f);
    const int var = p.variant;
    df s, r0, rv, rE;
    if (var == RSST_PVS || var == RSST_PMS || var == RSST_PD) {
      s = p.gm1 * (scale(v2 * dU[0], 0.5f) - vdm + dU[NV - 1]);
      if (var == RSST_PD) {
        r0 = {0.0f, 0.0f};
        rv = {0.0f, 0.0f};
        rE = p.inv_gm1;
      } else {
        const df ia2 = rho * rcp(p.gamma * P);
        r0 = ia2;
        rv = var == RSST_PVS ? ia2 : df_make(0.0f);
        rE = (var == RSST_PVS ? (e_int + P + kin) : (e_int + P - kin)) * ia2 * ir;
      }
    } else {
      s = dU[0];
      r0 = df_make(1.0f);
      rv = var == RSST_DVS ? df_make(1.0f) : df_make(0.0f);
      rE = (var == RSST_DVS ? (e_int + P + kin) : (e_int + P - kin)) * ir;
    }
    const df fs = f_of_df(p.gamma * P * ir, p) * s;
    dU[0] = dU[0] - fs * r0;
#pragma unroll
    for (int e = 0; e < ND; ++e) dU[1 + e] = dU[1 + e] - fs * (rv * v[e]);
    dU[NV - 1] = dU[NV - 1] - fs * rE;
  }
  if (p.has_grav) {
    df mg = {0.0f, 0.0f};
#pragma unroll
    for (int e = 0; e < ND; ++e) {
      dU[1 + e] = dU[1 + e] + rho * p.grav[e];
      mg = mg + q[1 + e] * p.grav[e];
    }
    dU[NV - 1] = dU[NV - 1] + mg;
  }
}

// CFL rate sum_d c_tot/dx_d of a cell and its physical check.
template <int NV>
__device__ __forceinline__ df cfl_rate_df(const df (&q)[NV], const PhysDF& p, bool& ok) {
  constexpr int ND = NV - 2;
  const df rho = q[0];
  const df ir = rcp(rho);
  df v2 = {0.0f, 0.0f};
  bool fin = isfinite(q[0].hi) && isfinite(q[NV - 1].hi);
#pragma unroll
  for (int e = 0; e < ND; ++e) {
    const df ve = q[1 + e] * ir;
    v2 = v2 + ve * ve;
    fin = fin && isfinite(q[1 + e].hi);
  }
  const df P = p.gm1 * q[NV - 1] - p.hgm1 * (rho * v2);
  ok = fin && df_pos(rho) && df_pos(P);
  return (dsqrt(v2) + sound_over_xi_df(p.gamma * P * ir, p)) * p.sum_inv_dx;
}

}  // namespace rsst
