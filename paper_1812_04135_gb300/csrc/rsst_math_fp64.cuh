// Float64 device arithmetic of the RSST step (arXiv:1812.04135).
//
// Each function states the passage of the paper it computes.  Variables:
// q = conservative state (rho, m_1..m_ND, E), ND = NV - 2 dimensions.
#pragma once

#include "rsst_internal.h"

namespace rsst {

// Equation of state (Sec. 3.2: the reduced equations hold for a general
// EOS; the pressure tendency needs (de/dP)_rho and (de/drho)_P, Eqs.
// pvs_cons_dpr / pvs_cons_therm).  The float64 step reads its
// thermodynamics only through these members.  Two gases, chosen at compile
// time (CV) so that the ideal-gas kernels carry no covolume arithmetic: the
// ideal gas (covolume b = 0, the only EOS the paper specifies),
// e = P/(gamma-1), and the covolume (Noble-Abel) gas,
// P = (gamma-1) e / (1 - b rho), a^2 = gamma P / (rho (1 - b rho)),
// (de/dP)_rho = (1 - b rho)/(gamma-1), (de/drho)_P = -b P/(gamma-1).  The
// launchers take CV = (b != 0) for a run.
__device__ __forceinline__ double rcp_nr(double x);

template <bool CV>
struct Eos {
  // 1 - b rho
  __device__ static __forceinline__ double omb(const Phys& p, double rho) { return fma(-p.covol, rho, 1.0); }
  // P from the total energy E and rho |V|^2
  __device__ static __forceinline__ double pressure(const Phys& p, double rho, double E, double rhov2) {
    const double Pi = p.gm1 * E - p.hgm1 * rhov2;
    if constexpr (CV) return Pi * rcp_nr(omb(p, rho));
    return Pi;
  }
  __device__ static __forceinline__ double sound2(const Phys& p, double rho, double P, double inv_rho) {
    if constexpr (CV) return p.gamma * P * inv_rho * rcp_nr(omb(p, rho));
    return p.gamma * P * inv_rho;
  }
  // (a/xi)^2 for a constant xi, with gamma/xi^2 folded into one constant
  __device__ static __forceinline__ double sound2_over_xi2(const Phys& p, double rho, double P, double inv_rho) {
    if constexpr (CV) return p.gamma_xi2 * (P * inv_rho) * rcp_nr(omb(p, rho));
    return p.gamma_xi2 * (P * inv_rho);
  }
  __device__ static __forceinline__ double internal_energy(const Phys& p, double rho, double P) {
    if constexpr (CV) return P * p.inv_gm1 * omb(p, rho);
    return P * p.inv_gm1;
  }
  __device__ static __forceinline__ double de_dP(const Phys& p, double rho, double P) {
    if constexpr (CV) return p.inv_gm1 * omb(p, rho);
    return p.inv_gm1;
  }
  __device__ static __forceinline__ double inv_de_dP(const Phys& p, double rho, double P) {
    if constexpr (CV) return p.gm1 * rcp_nr(omb(p, rho));
    return p.gm1;
  }
  // (0.5 |V|^2 - (de/drho)_P) of the pressure tendency
  __device__ static __forceinline__ double half_v2_minus_de_drho(const Phys& p, double v2, double P) {
    if constexpr (CV) return fma(p.covol * p.inv_gm1, P, 0.5 * v2);
    return 0.5 * v2;
  }
  // a state the EOS admits: 1 - b rho > 0 (always true for the ideal gas)
  __device__ static __forceinline__ bool admissible(const Phys& p, double rho) {
    if constexpr (CV) return omb(p, rho) > 0.0;
    return true;
  }
};

// 1/x to full float64 accuracy with three float64-pipe instructions: the
// hardware reciprocal approximation y, then one third-order step of the
// series 1/x = y / (1 - e) = y (1 + e + e^2 + ...), e = 1 - x y formed
// exactly by an FMA: y <- y + y (e + e^2), which cubes the seed's relative
// error (two Newton-Raphson steps square it twice at four FMAs).  Within an
// ulp of the correctly rounded quotient for the normal, positive densities
// it is used on (checked against CUDA's division by rsst_math_selftest).
__device__ __forceinline__ double rcp_nr(double x) {
  double y;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  const double e = fma(-x, y, 1.0);
  return fma(y, fma(e, e, e), y);
}

// sqrt(x) for the wave-speed estimate c_tot with three float64-pipe
// operations.  Seed: the float32 hardware reciprocal square root of
// m 2^odd, where x = m 2^e (m in [1, 2) holding x's leading 23 mantissa
// bits) and odd = e mod 2, so the argument lies in [1, 4); the result is
// rescaled by 2^(-(e - odd)/2) in the exponent field, all on the integer
// pipe.  One Newton step in Markstein's form, s = s0 + (y0/2)(x - s0^2) with
// s0 = x y0 and the residual x - s0^2 formed exactly by an FMA, squares the
// seed's relative error (about 2^-21) to below 2^-40.  Zero and subnormal x
// give 0, negative x NaN.  c_tot only sets the LLF dissipation speed and the
// CFL step, where this error is far below the 1e-10 the float64 path is
// held to; every other square root is the compiler's.
__device__ __forceinline__ double sqrt_ctot(double x) {
  const long long ix = __double_as_longlong(x);
  const int be = (int)(ix >> 52);  // biased exponent for x >= 0
  const int e = be - 1023;
  const int odd = e & 1;
  const float f = __int_as_float(((127 + odd) << 23) | (int)((ix >> 29) & 0x7fffff));
  const int ir = __float_as_int(rsqrtf(f));  // in (1/2, 1]
  const int k = (e - odd) >> 1;              // 1/sqrt(x) = rsqrt(f) 2^(-k)
  const long long yb = ((long long)(((ir >> 23) & 0xff) - 127 + 1023 - k) << 52) | ((long long)(ir & 0x7fffff) << 29);
  const double y0 = __longlong_as_double(yb);
  const double h0 = __longlong_as_double(yb - (1ll << 52));  // y0 / 2
  const double s0 = x * y0;
  const double s = fma(h0, fma(-s0, s0, x), s0);
  return be > 0 ? s : (ix >= 0 ? 0.0 : __longlong_as_double(0x7ff8000000000000ll));
}

// sqrt(x) as an unevaluated pair of floats s + c (relative error below
// 2^-42), for the LLF speed, on the integer and float32 pipes only: x =
// 2^(2k) y with y in [1, 4) read from the bit pattern, y = h + l with h its
// leading 24 significant bits and l the other 29 (rounded to a float);
// s = h rsqrt(h) and one Newton step c = (y - s^2) / (2 s) with s^2 split
// exactly by an FMA (h - s^2 is exact: Sterbenz), then both scaled by 2^k.
// Zero and subnormal x give 0, negative x and NaN give NaN, like sqrt_ctot;
// 2^k is kept to the float range (x in [2^-252, 2^256), far outside any
// physical speed^2).
__device__ __forceinline__ void sqrt_pair(double x, float& s, float& c) {
  const long long ix = __double_as_longlong(x);
  const int be = (int)(ix >> 52);  // biased exponent for x >= 0, negative for x < 0
  const int e = be - 1023;
  const int odd = e & 1;
  const float h = __int_as_float(((127 + odd) << 23) | (int)((ix >> 29) & 0x7fffff));
  const float l = __uint2float_rn((unsigned)(ix & 0x1fffffff)) * __int_as_float((75 + odd) << 23);  // * 2^(odd-52)
  const float r = rsqrtf(h);
  const float s0 = h * r;
  const float p = s0 * s0;
  const float d = ((h - p) - fmaf(s0, s0, -p)) + l;
  const float c0 = d * (0.5f * r);
  const int k = (e - odd) >> 1;
  const float sc = k < -126 ? 0.0f : (k > 127 ? __int_as_float(0x7f800000) : __int_as_float((127 + k) << 23));
  const bool fin = be > 0 && be < 2047;
  const float special = (ix >= 0 && be == 0) ? 0.0f : __int_as_float(0x7fc00000);
  s = fin ? s0 * sc : special;
  c = fin ? c0 * sc : special;
}

// A float as a double, on the integer pipe (subnormal floats read as 0).
__device__ __forceinline__ double f2d_bits(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned E = (b >> 23) & 0xffu;
  const unsigned long long sign = (unsigned long long)(b >> 31) << 63;
  const unsigned long long ex = E == 0u ? 0ull : (E == 255u ? 0x7ffull : (unsigned long long)(E + 896u)) << 52;
  const unsigned long long mant = E == 0u ? 0ull : (unsigned long long)(b & 0x7fffffu) << 29;
  return __longlong_as_double((long long)(sign | ex | mant));
}

// c_tot = |V| + a/xi from |V|^2 and (a/xi)^2 as a normalised float pair
// (h + l, |l| <= ulp(h)/2): both square roots by sqrt_pair, summed exactly
// in the leading parts (two-sum), relative error below 2^-41.
__device__ __forceinline__ void ctot_pair(double v2, double a2x, float& h, float& l) {
  float sv, cv, sa, ca;
  sqrt_pair(v2, sv, cv);
  sqrt_pair(a2x, sa, ca);
  const float t = sv + sa;
  const float bv = t - sv;
  const float lo = ((sv - (t - bv)) + (sa - bv)) + (cv + ca);
  h = t + lo;
  l = lo - (h - t);
}

// Effective sound speed a/xi from a^2 and the factor f = 1 - 1/xi^2: constant
// xi, or the C_max law xi = [1 + (a/C_max)^4]^(1/4) (Eq. cx, Sec. 4.3), for
// which a/xi = sqrt(a^2 / sqrt(w)) and f = 1 - 1/sqrt(w), w = 1 + a^4/C_max^4.
__device__ __forceinline__ double sound_over_xi(double a2, const Phys& p) {
  if (p.use_cmax) return sqrt(a2 / sqrt(fma(a2 * a2, p.inv_cmax4, 1.0)));
  return sqrt_ctot(a2) * p.inv_xi;
}
__device__ __forceinline__ double f_of(double a2, const Phys& p) {
  if (p.use_cmax) return 1.0 - 1.0 / sqrt(fma(a2 * a2, p.inv_cmax4, 1.0));
  return p.f;
}

// a/xi of a state for c_tot: constant xi as sqrt((a/xi)^2), or the C_max law.
template <bool CV>
__device__ __forceinline__ double ctot_sound(const Phys& p, double rho, double P, double ir) {
  if (p.use_cmax) return sound_over_xi(Eos<CV>::sound2(p, rho, P, ir), p);
  return sqrt_ctot(Eos<CV>::sound2_over_xi2(p, rho, P, ir));
}

// The Euler flux along dimension D, F, and the approximate RSST
// characteristic speed c_tot = |V| + a/xi of one state (Eq. pvs_dt0; Sec. 4.2)
// as a float pair ch + cl: for a constant xi from ctot_pair on the float32
// pipe, under the C_max law from the float64 form.
template <int NV, int D, bool CV = false>
__device__ __forceinline__ void euler_flux(const double (&q)[NV], const Phys& p,
                                           double (&F)[NV], float& ch, float& cl) {
  constexpr int ND = NV - 2;
  const double rho = q[0];
  const double ir = rcp_nr(rho);
  double v[ND];
  double v2 = 0.0;
#pragma unroll
  for (int e = 0; e < ND; ++e) {
    v[e] = q[1 + e] * ir;
    v2 += v[e] * v[e];
  }
  const double P = Eos<CV>::pressure(p, rho, q[NV - 1], rho * v2);
  if (p.use_cmax) {
    const double c = sqrt_ctot(v2) + ctot_sound<CV>(p, rho, P, ir);
    ch = __double2float_rn(c);
    cl = __double2float_rn(c - (double)ch);
  } else {
    ctot_pair(v2, Eos<CV>::sound2_over_xi2(p, rho, P, ir), ch, cl);
  }
  F[0] = q[1 + D];
#pragma unroll
  for (int e = 0; e < ND; ++e) F[1 + e] = (e == D) ? fma(q[1 + e], v[D], P) : q[1 + e] * v[D];
  F[NV - 1] = (q[NV - 1] + P) * v[D];
}

// Twice the local Lax-Friedrichs flux, 2 F = F(qL) + F(qR) - alpha (qR - qL)
// with alpha = max(c_tot(qL), c_tot(qR)), ties to the left state (Sec. 4.2,
// step 4).  The factor 1/2 is exact and left to the caller (it folds into
// the divergence's 1/dx), which saves the halvings inside the fluxes.
template <int NV, int D, bool CV = false>
__device__ __forceinline__ void llf_flux_x2(const double (&qL)[NV], const double (&qR)[NV],
                                            const Phys& p, double (&G)[NV]) {
  double FL[NV], FR[NV];
  float hL, lL, hR, lR;
  euler_flux<NV, D, CV>(qL, p, FL, hL, lL);
  euler_flux<NV, D, CV>(qR, p, FR, hR, lR);
  const bool left = hL > hR || (hL == hR && lL >= lR);  // normalised pairs order like their values
  const double alpha = f2d_bits(left ? hL : hR) + f2d_bits(left ? lL : lR);
#pragma unroll
  for (int k = 0; k < NV; ++k) G[k] = fma(-alpha, qR[k] - qL[k], FL[k] + FR[k]);
}

// Monotonized-central limited slope (named in Sec. 4.2): 0 if ab <= 0, else
// the smallest in magnitude of 2a, 2b, (a+b)/2, ties in that order.
// Only a + b uses the float64 pipe.  A double's bit pattern shifted left by
// one (sign dropped) orders like its magnitude as an unsigned integer, so the
// magnitude comparisons run on the integer pipe (the shift, unlike a mask of
// the sign bit, is not turned back into float64 absolute values by the
// compiler), and scaling a normal double by 2, 4 or 1/2 is an exact change
// of its exponent field (2|a| <= |a+b|/2 is |a| * 4 <= |a+b|).  Same
// decisions and values as the direct form for normal operands; differences
// of physical states are exactly zero or far above the subnormal range.
__device__ __forceinline__ double mc_slope(double a, double b) {
  const long long one = 1ll << 52;                // +1 in the exponent field
  const unsigned long long four = 1ull << 54;     // +2 in the shifted exponent field: x4
  const long long ia = __double_as_longlong(a), ib = __double_as_longlong(b);
  const unsigned long long ua = (unsigned long long)ia << 1, ub = (unsigned long long)ib << 1;
  const bool same = ((ia ^ ib) >= 0) && ua != 0 && ub != 0;
  const long long is = __double_as_longlong(a + b);
  const unsigned long long us = (unsigned long long)is << 1;
  const long long pick = (ua <= ub && ua + four <= us) ? ia + one : ((ub + four <= us) ? ib + one : is - one);
  return same ? __longlong_as_double(pick) : 0.0;
}

// Reduced tendency: dU <- dU - (1 - 1/xi^2) s r, then the external force.
//   PVS: s = dP,   r = (1/a^2, V/a^2, (e+P+rho V^2/2)/(rho a^2))   Sec. 3.2, Eqs. pvs_dt, pvs_cons_rhs
//   DVS: s = drho, r = (1, V, (e+P+rho V^2/2)/rho)                  App. A.1
//   PMS: s = dP,   r = (1/a^2, 0, (e+P-rho V^2/2)/(rho a^2))        App. A.2
//   DMS: s = drho, r = (1, 0, (e+P-rho V^2/2)/rho)                  App. A.3
//   PD : s = dP,   r = (0, 0, 1/(gamma-1))                          App. A.4
// with dP = (gamma-1)(V^2/2 drho - V.dm + dE) (Eq. pvs_dt_dpr, ideal gas),
// evaluated at the cell centre of the stage state; force terms
// (0, rho F, m.F) of App. B are added after (dP excludes them).
template <int NV, bool CV = false>
__device__ __forceinline__ void rsst_rhs(const double (&q)[NV], double (&dU)[NV], const Phys& p) {
  constexpr int ND = NV - 2;
  const double rho = q[0];
  if (p.variant != RSST_EULER) {
    const double ir = rcp_nr(rho);
    double v[ND];
    double v2 = 0.0, vdm = 0.0;
#pragma unroll
    for (int e = 0; e < ND; ++e) {
      v[e] = q[1 + e] * ir;
      v2 += v[e] * v[e];
      vdm += v[e] * dU[1 + e];
    }
    const double P = Eos<CV>::pressure(p, rho, q[NV - 1], rho * v2);
    const double e_int = Eos<CV>::internal_energy(p, rho, P);
    const double kin = 0.5 * rho * v2;
    double s, r0, rv, rE;  // r = (r0, rv * V, rE); rv in {0, 1/a^2, 1}
    const int var = p.variant;
    if (var == RSST_PVS || var == RSST_PMS || var == RSST_PD) {
      s = Eos<CV>::inv_de_dP(p, rho, P) * (Eos<CV>::half_v2_minus_de_drho(p, v2, P) * dU[0] - vdm + dU[NV - 1]);
      if (var == RSST_PD) {
        r0 = 0.0; rv = 0.0; rE = Eos<CV>::de_dP(p, rho, P);
      } else {
        const double ia2 = rcp_nr(Eos<CV>::sound2(p, rho, P, ir));  // 1/a^2
        r0 = ia2;
        rv = (var == RSST_PVS) ? ia2 : 0.0;
        rE = (var == RSST_PVS ? (e_int + P + kin) : (e_int + P - kin)) * ia2 * ir;
      }
    } else {  // DVS, DMS
      s = dU[0];
      r0 = 1.0;
      rv = (var == RSST_DVS) ? 1.0 : 0.0;
      rE = (var == RSST_DVS ? (e_int + P + kin) : (e_int + P - kin)) * ir;
    }
    const double fs = f_of(Eos<CV>::sound2(p, rho, P, ir), p) * s;
    dU[0] -= fs * r0;
#pragma unroll
    for (int e = 0; e < ND; ++e) dU[1 + e] -= fs * (rv * v[e]);
    dU[NV - 1] -= fs * rE;
  }
  if (p.has_grav) {
    double mg = 0.0;
#pragma unroll
    for (int e = 0; e < ND; ++e) {
      dU[1 + e] += rho * p.grav[e];
      mg += q[1 + e] * p.grav[e];
    }
    dU[NV - 1] += mg;
  }
}

// CFL rate sum_d c_tot/dx_d of a cell and its physical-state check.
template <int NV, bool CV = false>
__device__ __forceinline__ double cfl_rate(const double (&q)[NV], const Phys& p, bool& ok) {
  constexpr int ND = NV - 2;
  const double rho = q[0];
  const double ir = rcp_nr(rho);
  double v2 = 0.0;
  bool fin = isfinite(q[0]) && isfinite(q[NV - 1]);
#pragma unroll
  for (int e = 0; e < ND; ++e) {
    const double ve = q[1 + e] * ir;
    v2 += ve * ve;
    fin = fin && isfinite(q[1 + e]);
  }
  const double P = Eos<CV>::pressure(p, rho, q[NV - 1], rho * v2);
  ok = fin && rho > 0.0 && P > 0.0 && Eos<CV>::admissible(p, rho);
  if (p.use_cmax) return (sqrt_ctot(v2) + ctot_sound<CV>(p, rho, P, ir)) * p.sum_inv_dx;
  // c_tot as the float pair of the LLF speed (relative error below 2^-41,
  // tighter than the float64-pipe square root's 2^-40), on the float32 and
  // integer pipes
  float ch, cl;
  ctot_pair(v2, Eos<CV>::sound2_over_xi2(p, rho, P, ir), ch, cl);
  return (f2d_bits(ch) + f2d_bits(cl)) * p.sum_inv_dx;
}

}  // namespace rsst
