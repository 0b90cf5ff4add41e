// Float32 perturbation arithmetic of the RSST step.
//
// The state is U = U0 + U1 with U0 = (rho0, 0, E0) a float64 background that
// depends only on the vertical index and U1 the float32 perturbation.  Every
// quantity that feeds an update is formed from perturbation-sized terms, so
// the low-Mach pressure and density perturbations are not lost to
// cancellation against the background:
//   P1 = P - P0 = (gamma-1)(E1 - |m|^2/(2 rho))                 (m0 = 0)
//   F(U) - F(U0) = (m_D, m v_D + P1 e_D, (E0 + P0 + E1 + P1) v_D)
//   a^2 - a0^2 = gamma (P1 rho0 - P0 rho1) / (rho rho0)
// Faces across the vertical axis also carry the background's own face jump
// U0R - U0L and its LLF speed alpha0; their contribution is split as
//   alpha (U1R - U1L) + (alpha - alpha0)(U0R - U0L)
// with alpha - alpha0 formed from c - c0 on each side and the float64
// background difference g = c0L - c0R.  The MC slope of a component whose
// background varies is lin_B(d1) + [lin_B(d0) - MC(d0)], where B is the
// branch MC takes on the full differences d = d0 + d1 and the bracket is a
// float64 table entry per branch.
#pragma once

#include "rsst_internal.h"

namespace rsst {

// Hardware reciprocal and square root approximations (a few ulp), with
// subnormal inputs and results flushed to zero: the float32 kernels never
// form subnormal densities, pressures or speeds, and without the flush the
// compiler wraps each approximation in a rescaling sequence.
__device__ __forceinline__ float rcp_f(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float sqrt_f(float x) {
  float y;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Monotonized-central slope (Sec. 4.2), float32, branch-free: the magnitude
// min(2|a|, 2|b|, |a+b|/2) with the sign of a, zero unless ab > 0.  Equal to
// the branch-wise form (equal magnitudes of same-sign candidates are equal
// values, so the tie rule does not change the result).
__device__ __forceinline__ float mc_slope_f(float a, float b) {
  const float m = fminf(2.0f * fminf(fabsf(a), fabsf(b)), 0.5f * fabsf(a + b));
  return (a * b > 0.0f) ? copysignf(m, a) : 0.0f;
}

// Branch of the MC slope: 0 -> 0, 1 -> 2a, 2 -> 2b, 3 -> (a+b)/2.
__device__ __forceinline__ int mc_branch_f(float a, float b) {
  if (!(a * b > 0.0f)) return 0;
  const float aa = 2.0f * fabsf(a), bb = 2.0f * fabsf(b), cc = 0.5f * fabsf(a + b);
  return (aa <= bb && aa <= cc) ? 1 : ((bb <= cc) ? 2 : 3);
}

__device__ __forceinline__ float mc_linear_f(int br, float a, float b) {
  return br == 0 ? 0.0f : (br == 1 ? 2.0f * a : (br == 2 ? 2.0f * b : 0.5f * (a + b)));
}

// a/xi and f = 1 - 1/xi^2 from a^2 (constant xi, or the C_max law, Eq. cx).
__device__ __forceinline__ float sound_over_xi_f(float a2, const PhysF& p) {
  if (p.use_cmax) return sqrtf(a2 / sqrtf(fmaf(a2 * a2, p.inv_cmax4, 1.0f)));
  return sqrtf(a2) * p.inv_xi;
}
__device__ __forceinline__ float f_of_f(float a2, const PhysF& p) {
  if (p.use_cmax) return 1.0f - 1.0f / sqrtf(fmaf(a2 * a2, p.inv_cmax4, 1.0f));
  return p.f;
}

// Full-state Euler flux and c_tot along D in float32 (no background).
template <int NV, int D>
__device__ __forceinline__ void euler_flux_f(const float (&q)[NV], const PhysF& p, float (&F)[NV], float& c) {
  constexpr int ND = NV - 2;
  const float rho = q[0];
  const float ir = 1.0f / rho;
  float v[ND];
  float v2 = 0.0f;
#pragma unroll
  for (int e = 0; e < ND; ++e) {
    v[e] = q[1 + e] * ir;
    v2 += v[e] * v[e];
  }
  const float P = p.gm1 * (q[NV - 1] - 0.5f * rho * v2);
  c = sqrtf(v2) + sound_over_xi_f(p.gamma * P * ir, p);
  F[0] = q[1 + D];
#pragma unroll
  for (int e = 0; e < ND; ++e) F[1 + e] = q[1 + e] * v[D] + (e == D ? P : 0.0f);
  F[NV - 1] = (q[NV - 1] + P) * v[D];
}

// Perturbation flux F(U0 + q1) - F(U0) along D, the full c_tot, and c - c0.
// Background face values: rho0, E0, P0 = (gamma-1) E0, H0 = E0 + P0, its
// sound speed a0 and speed c0 = a0/xi(a0) (c0 used with the C_max law).
template <int NV, int D, bool WANT_DC>
__device__ __forceinline__ void pert_flux_f(const float (&q1)[NV], float rho0, float P0, float H0, float a0,
                                            const PhysF& p, float (&F)[NV], float& c, float& dc, float c0 = 0.0f) {
  constexpr int ND = NV - 2;
  const float rho = rho0 + q1[0];
  const float ir = 1.0f / rho;
  float v[ND];
  float v2 = 0.0f, mv = 0.0f;
#pragma unroll
  for (int e = 0; e < ND; ++e) {
    v[e] = q1[1 + e] * ir;
    v2 += v[e] * v[e];
    mv += q1[1 + e] * v[e];
  }
  const float P1 = p.gm1 * (q1[NV - 1] - 0.5f * mv);
  const float a2 = p.gamma * (P0 + P1) * ir;
  const float vm = sqrtf(v2);
  if (p.use_cmax) {
    const float g = sound_over_xi_f(a2, p);
    c = vm + g;
    if (WANT_DC) dc = vm + (g - c0);  // multiplies only the background face jump
  } else {
    const float a = sqrtf(a2);
    c = vm + a * p.inv_xi;
    if (WANT_DC) {
      const float da2 = p.gamma * (P1 * rho0 - P0 * q1[0]) * ir / rho0;
      dc = vm + (da2 / (a + a0)) * p.inv_xi;
    }
  }
  F[0] = q1[1 + D];
#pragma unroll
  for (int e = 0; e < ND; ++e) F[1 + e] = q1[1 + e] * v[D] + (e == D ? P1 : 0.0f);
  F[NV - 1] = (H0 + q1[NV - 1] + P1) * v[D];
}

}  // namespace rsst

namespace rsst {

// Perturbation slope of a component whose background varies along the axis:
// lin_B(d1) + [lin_B(d0) - MC(d0)], B the branch of MC on d0 + d1.
// row points at the component's six slope rows (d0L, d0R, four deltas), stride sv.
__device__ __forceinline__ float bg_slope_f(const float* row, int sv, int r, float da, float db) {
  const int b = mc_branch_f(row[r] + da, row[sv + r] + db);
  return mc_linear_f(b, da, db) + row[(2 + b) * sv + r];
}

// Cell update of the float32 perturbation state (Sec. 4.2 steps 6-8):
// L = R0 + div-part, reduced by -f s r from the full-state primitives, plus
// the perturbation force (rho1 F, m.F); then the RK combine.  Dl is the Euler
// tendency including the background's (for s).  Returns the new state in u,
// and in stage 2 the CFL rate and the physical check of the new state.
template <int NV>
__device__ __forceinline__ void cell_update_f(const float (&q)[NV], float (&L)[NV], const float (&Dl)[NV], float rho0,
                                              float P0, const PhysF& pf, int variant, bool has_grav, int stage,
                                              float dt, const float* base_vals, float (&u)[NV], float& rate,
                                              bool& ok) {
  constexpr int ND = NV - 2;
  const float rho = rho0 + q[0];
  const float ir = 1.0f / rho;
  float vel[ND];
  float v2 = 0.0f, mv = 0.0f, vdm = 0.0f;
#pragma unroll
  for (int e = 0; e < ND; ++e) {
    vel[e] = q[1 + e] * ir;
    v2 += vel[e] * vel[e];
    mv += q[1 + e] * vel[e];
    vdm += vel[e] * Dl[1 + e];
  }
  const float P = P0 + pf.gm1 * (q[NV - 1] - 0.5f * mv);
  if (variant != RSST_EULER) {
    const float fcell = f_of_f(pf.gamma * P * ir, pf);
    const float e_int = P * pf.inv_gm1;
    const float kin = 0.5f * mv;
    float s, r0, rv, rE;
    if (variant == RSST_PVS || variant == RSST_PMS || variant == RSST_PD) {
      s = pf.gm1 * (0.5f * v2 * Dl[0] - vdm + Dl[NV - 1]);
      if (variant == RSST_PD) {
        r0 = 0.0f; rv = 0.0f; rE = pf.inv_gm1;
      } else {
        const float ia2 = rho / (pf.gamma * P);
        r0 = ia2;
        rv = variant == RSST_PVS ? ia2 : 0.0f;
        rE = (variant == RSST_PVS ? (e_int + P + kin) : (e_int + P - kin)) * ia2 * ir;
      }
    } else {
      s = Dl[0];
      r0 = 1.0f;
      rv = variant == RSST_DVS ? 1.0f : 0.0f;
      rE = (variant == RSST_DVS ? (e_int + P + kin) : (e_int + P - kin)) * ir;
    }
    const float fs = fcell * s;
    L[0] -= fs * r0;
#pragma unroll
    for (int e = 0; e < ND; ++e) L[1 + e] -= fs * (rv * vel[e]);
    L[NV - 1] -= fs * rE;
  }
  if (has_grav) {
    float mg = 0.0f;
#pragma unroll
    for (int e = 0; e < ND; ++e) {
      L[1 + e] += q[0] * pf.grav[e];
      mg += q[1 + e] * pf.grav[e];
    }
    L[NV - 1] += mg;
  }
  rate = 0.0f;
  ok = true;
  if (stage == 1) {
#pragma unroll
    for (int v = 0; v < NV; ++v) u[v] = q[v] + dt * L[v];
  } else {
#pragma unroll
    for (int v = 0; v < NV; ++v) u[v] = 0.5f * base_vals[v] + 0.5f * (q[v] + dt * L[v]);
    const float rn = rho0 + u[0];
    const float irn = 1.0f / rn;
    float w2 = 0.0f, mw = 0.0f;
    bool fin = isfinite(u[0]) && isfinite(u[NV - 1]);
#pragma unroll
    for (int e = 0; e < ND; ++e) {
      const float ve = u[1 + e] * irn;
      w2 += ve * ve;
      mw += u[1 + e] * ve;
      fin = fin && isfinite(u[1 + e]);
    }
    const float Pn = P0 + pf.gm1 * (u[NV - 1] - 0.5f * mw);
    ok = fin && rn > 0.0f && Pn > 0.0f;
    if (ok) rate = (sqrtf(w2) + sound_over_xi_f(pf.gamma * Pn * irn, pf)) * pf.sum_inv_dx;
  }
}

}  // namespace rsst
