// Float32 perturbation kernels of the RSST step (arXiv:1812.04135, Sec. 4.2
// scheme with the Sec. 3.2 / App. A reduced tendencies and App. B force).
//
// Storage: U1 = U - U0 in float32, U0 = (rho0, 0, P0/(gamma-1)) the float64
// background along the vertical axis (none: U1 is the full state).  The
// background's own discrete tendency R0 = L(U0) (force included) and its
// face states are computed once in float64 (bgtab_kernel); the stage
// kernels then advance U1 with dU1/dt = R0 + [L(U0+U1) - L(U0)], every term
// of the bracket formed from perturbation-sized quantities (see
// rsst_math_fp32.cuh).  Tile structure is that of the float64 kernel.
#include "rsst_common.cuh"
#include "rsst_internal.h"
#include "rsst_attr.h"
#include "rsst_math_fp32.cuh"
#include "rsst_math_fp64.cuh"

namespace rsst {

// ---------------------------------------------------------------------------
// Background tables (float64 arithmetic, one thread per padded vertical index)
// ---------------------------------------------------------------------------

template <int NV, int V>
__global__ void bgtab_kernel(const double* __restrict__ bg, int L, Phys p, float* __restrict__ tab,
                             float* __restrict__ tabr) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= L) return;
  const double* r0 = bg;
  const double* e0 = bg + L;
  auto U0 = [&](int kk, int c) -> double { return c == 0 ? r0[kk] : e0[kk]; };
  auto put = [&](int f, double v) { tab[(size_t)f * L + k] = (float)v; };
  auto putr = [&](int f, double v) {
    if (tabr) tabr[(size_t)k * TR_W + f] = (float)v;
  };
  for (int f = 0; f < TB_COUNT; ++f) put(f, 0.0);
  for (int f = 0; f < TR_W; ++f) putr(f, 0.0);
  // gx P/rho is (a/xi)^2 for a constant xi and a^2 under the C_max law
  const double gx = p.use_cmax ? p.gamma : p.gamma_xi2;
  const double P0 = p.gm1 * e0[k];
  put(TB_RHO0, r0[k]);
  put(TB_E0, e0[k]);
  put(TB_P0, P0);
  put(TB_H0, e0[k] + P0);
  putr(TR_RHO0, r0[k]);
  putr(TR_P0, P0);
  putr(TR_GXP0, gx * P0);
  putr(TR_H0, e0[k] + P0);
  auto slope = [&](int kk, int c) { return mc_slope(U0(kk, c) - U0(kk - 1, c), U0(kk + 1, c) - U0(kk, c)); };
  if (k >= 1 && k <= L - 2) {
    for (int c = 0; c < 2; ++c) {
      const double dL = U0(k, c) - U0(k - 1, c), dR = U0(k + 1, c) - U0(k, c);
      const double s0 = mc_slope(dL, dR);
      put(TB_S + 6 * c + 0, dL);
      put(TB_S + 6 * c + 1, dR);
      put(TB_S + 6 * c + 2, 0.0 - s0);
      put(TB_S + 6 * c + 3, 2.0 * dL - s0);
      put(TB_S + 6 * c + 4, 2.0 * dR - s0);
      put(TB_S + 6 * c + 5, 0.5 * (dL + dR) - s0);
      const int b = c == 0 ? TR_SRHO : TR_SE;  // half slopes: the face states are U +- slope/2
      putr(b + 0, dL);
      putr(b + 1, dR);
      putr(b + 2, 0.5 * (0.0 - s0));
      putr(b + 3, 0.5 * (2.0 * dL - s0));
      putr(b + 4, 0.5 * (2.0 * dR - s0));
      putr(b + 5, 0.5 * (0.5 * (dL + dR) - s0));
    }
  }
  // background face state of the face between padded cells kk-1 and kk
  auto face = [&](int kk, double (&qL)[NV], double (&qR)[NV]) {
    for (int v = 0; v < NV; ++v) qL[v] = qR[v] = 0.0;
    qL[0] = U0(kk - 1, 0) + 0.5 * slope(kk - 1, 0);
    qL[NV - 1] = U0(kk - 1, 1) + 0.5 * slope(kk - 1, 1);
    qR[0] = U0(kk, 0) - 0.5 * slope(kk, 0);
    qR[NV - 1] = U0(kk, 1) - 0.5 * slope(kk, 1);
  };
  if (k >= 2 && k <= L - 2) {
    double qL[NV], qR[NV];
    face(k, qL, qR);
    const double PL = p.gm1 * qL[NV - 1], PR = p.gm1 * qR[NV - 1];
    const double aL = sqrt(p.gamma * PL / qL[0]), aR = sqrt(p.gamma * PR / qR[0]);
    const double cL = sound_over_xi(p.gamma * PL / qL[0], p), cR = sound_over_xi(p.gamma * PR / qR[0], p);
    put(TB_FRHOL, qL[0]);
    put(TB_FRHOR, qR[0]);
    put(TB_FEL, qL[NV - 1]);
    put(TB_FER, qR[NV - 1]);
    put(TB_FPL, PL);
    put(TB_FPR, PR);
    put(TB_FHL, qL[NV - 1] + PL);
    put(TB_FHR, qR[NV - 1] + PR);
    put(TB_FAL, aL);
    put(TB_FAR, aR);
    put(TB_FG, cL - cR);
    put(TB_FALPHA, cL >= cR ? cL : cR);
    put(TB_FDRHO, qR[0] - qL[0]);
    put(TB_FDE, qR[NV - 1] - qL[NV - 1]);
    putr(TR_FL + 0, qL[0]);
    putr(TR_FL + 1, PL);
    putr(TR_FL + 2, gx * PL);
    putr(TR_FL + 3, qL[NV - 1] + PL);
    putr(TR_FR + 0, qR[0]);
    putr(TR_FR + 1, PR);
    putr(TR_FR + 2, gx * PR);
    putr(TR_FR + 3, qR[NV - 1] + PR);
    putr(TR_FA0X + 0, aL * p.inv_xi);
    putr(TR_FA0X + 1, aR * p.inv_xi);
    putr(TR_FA0X + 2, gx / qL[0]);
    putr(TR_FA0X + 3, gx / qR[0]);
    putr(TR_FG, cL - cR);
    putr(TR_FALPHA, cL >= cR ? cL : cR);
    putr(TR_FJRHO, qR[0] - qL[0]);
    putr(TR_FJE, qR[NV - 1] - qL[NV - 1]);
  }
  if (k >= 2 && k <= L - 3) {
    double qL[NV], qR[NV], Fm[NV], Fp[NV];
    face(k, qL, qR);
    llf_flux_x2<NV, V>(qL, qR, p, Fm);
    face(k + 1, qL, qR);
    llf_flux_x2<NV, V>(qL, qR, p, Fp);
    double D0[NV];
    for (int v = 0; v < NV; ++v) D0[v] = -(Fp[v] - Fm[v]) * (0.5 * p.inv_dx[V]);
    put(TB_D0RHO, D0[0]);
    put(TB_D0MV, D0[1 + V]);
    put(TB_D0E, D0[NV - 1]);
    putr(TR_D0RHO, D0[0]);
    putr(TR_D0MV, D0[1 + V]);
    putr(TR_D0E, D0[NV - 1]);
    for (int v = 0; v < NV; ++v) {
      double R = D0[v];
      if (v >= 1 && v <= NV - 2) R += r0[k] * p.grav[v - 1];
      put(TB_R0 + v, R);
      putr(TR_R0 + v, R);
    }
  }
}

// ---------------------------------------------------------------------------
// Stage kernel
// ---------------------------------------------------------------------------

template <int NDIM, int VERT, int BX, int BY, int BZ, int NT>
struct TileCfgF {
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
  static constexpr int SV = VERT < 0 ? 0 : (VERT == 0 ? SX : (VERT == 1 ? SY : SZ));
  static constexpr int TROWS = VERT < 0 ? 0 : TB_COUNT;
  static constexpr size_t SMEM = sizeof(float) * ((size_t)NV * (SCELLS + FMAX) + (size_t)TROWS * SV) + 64 * sizeof(double);
};

template <int NDIM, int VERT, int BX, int BY, int BZ, int NT, int D>
__device__ __forceinline__ void face_pass_f(const float* __restrict__ su, float* __restrict__ sf,
                                            const float* __restrict__ st, const PhysF& pf, const Geom& g, int i0,
                                            int j0, int k0,
                                            float (&dU)[TileCfgF<NDIM, VERT, BX, BY, BZ, NT>::CPT][NDIM + 2]) {
  using C = TileCfgF<NDIM, VERT, BX, BY, BZ, NT>;
  constexpr int NV = C::NV;
  constexpr int EX = BX + (D == 0), EY = BY + (D == 1), EZ = BZ + (D == 2);
  constexpr int NF = EX * EY * EZ;
  constexpr int STRIDE = D == 0 ? 1 : (D == 1 ? C::SX : C::SX * C::SY);
  constexpr int HV = VERT == 0 ? C::HX : (VERT == 1 ? C::HY : C::HZ);
  const int baseD = D == 0 ? i0 : (D == 1 ? j0 : k0);
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
    float um2[NV], um1[NV], u0[NV], up1[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const float* sv = su + v * C::SCELLS + s0;
      um2[v] = sv[-2 * STRIDE];
      um1[v] = sv[-STRIDE];
      u0[v] = sv[0];
      up1[v] = sv[STRIDE];
    }
    float qL[NV], qR[NV], F[NV];
    if constexpr (VERT < 0) {
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        qL[v] = um1[v] + 0.5f * mc_slope_f(um1[v] - um2[v], u0[v] - um1[v]);
        qR[v] = u0[v] - 0.5f * mc_slope_f(u0[v] - um1[v], up1[v] - u0[v]);
      }
      float FL[NV], FR[NV], cL, cR;
      euler_flux_f<NV, D>(qL, pf, FL, cL);
      euler_flux_f<NV, D>(qR, pf, FR, cR);
      const float alpha = cL >= cR ? cL : cR;
#pragma unroll
      for (int v = 0; v < NV; ++v) F[v] = 0.5f * (FL[v] + FR[v]) - 0.5f * alpha * (qR[v] - qL[v]);
    } else if constexpr (D != VERT) {
      // background constant along D: exact perturbation flux, no background jump
      const int row = (VERT == 0 ? fx : (VERT == 1 ? fy : fz)) + HV;
      const float rho0 = st[TB_RHO0 * C::SV + row], P0 = st[TB_P0 * C::SV + row], H0 = st[TB_H0 * C::SV + row];
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        qL[v] = um1[v] + 0.5f * mc_slope_f(um1[v] - um2[v], u0[v] - um1[v]);
        qR[v] = u0[v] - 0.5f * mc_slope_f(u0[v] - um1[v], up1[v] - u0[v]);
      }
      float FL[NV], FR[NV], cL, cR, dum;
      pert_flux_f<NV, D, false>(qL, rho0, P0, H0, 0.0f, pf, FL, cL, dum);
      pert_flux_f<NV, D, false>(qR, rho0, P0, H0, 0.0f, pf, FR, cR, dum);
      const float alpha = cL >= cR ? cL : cR;
#pragma unroll
      for (int v = 0; v < NV; ++v) F[v] = 0.5f * (FL[v] + FR[v]) - 0.5f * alpha * (qR[v] - qL[v]);
    } else {
      // face across the vertical axis between rows rR-1 and rR
      const int rR = fD + HV, rL = rR - 1;
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const float da = um1[v] - um2[v], db = u0[v] - um1[v], dc = up1[v] - u0[v];
        float sl, sr;
        if (v == 0 || v == NV - 1) {
          const int c = v == 0 ? 0 : 1;
          const float* sL = st + (TB_S + 6 * c) * C::SV;
          const int bl = mc_branch_f(sL[rL] + da, sL[C::SV + rL] + db);
          sl = mc_linear_f(bl, da, db) + sL[(2 + bl) * C::SV + rL];
          const int br = mc_branch_f(sL[rR] + db, sL[C::SV + rR] + dc);
          sr = mc_linear_f(br, db, dc) + sL[(2 + br) * C::SV + rR];
        } else {
          sl = mc_slope_f(da, db);
          sr = mc_slope_f(db, dc);
        }
        qL[v] = um1[v] + 0.5f * sl;
        qR[v] = u0[v] - 0.5f * sr;
      }
      float FL[NV], FR[NV], cL, cR, dcL, dcR;
      const float gdiff = st[TB_FG * C::SV + rR], al0 = st[TB_FALPHA * C::SV + rR];
      const float c0L = gdiff >= 0.0f ? al0 : al0 + gdiff, c0R = gdiff >= 0.0f ? al0 - gdiff : al0;
      pert_flux_f<NV, D, true>(qL, st[TB_FRHOL * C::SV + rR], st[TB_FPL * C::SV + rR], st[TB_FHL * C::SV + rR],
                               st[TB_FAL * C::SV + rR], pf, FL, cL, dcL, c0L);
      pert_flux_f<NV, D, true>(qR, st[TB_FRHOR * C::SV + rR], st[TB_FPR * C::SV + rR], st[TB_FHR * C::SV + rR],
                               st[TB_FAR * C::SV + rR], pf, FR, cR, dcR, c0R);
      const float dalpha = gdiff >= 0.0f ? fmaxf(dcL, dcR - gdiff) : fmaxf(dcL + gdiff, dcR);
      const float alpha = st[TB_FALPHA * C::SV + rR] + dalpha;
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const float j0v = v == 0 ? st[TB_FDRHO * C::SV + rR] : (v == NV - 1 ? st[TB_FDE * C::SV + rR] : 0.0f);
        F[v] = 0.5f * (FL[v] + FR[v]) - 0.5f * (alpha * (qR[v] - qL[v]) + dalpha * j0v);
      }
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) sf[v * C::FMAX + fid] = F[v];
  }
  __syncthreads();
  const float idx = pf.inv_dx[D];
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

template <int NDIM, int VERT, int BX, int BY, int BZ, int NT>
__global__ void __launch_bounds__(NT) stage_fp32_kernel(const StageArgs<float> a) {
  using C = TileCfgF<NDIM, VERT, BX, BY, BZ, NT>;
  constexpr int NV = C::NV;
  constexpr int ND = NDIM;
  extern __shared__ double smem_d[];
  float* su = reinterpret_cast<float*>(smem_d);
  float* sf = su + NV * C::SCELLS;
  float* st = sf + NV * C::FMAX;
  constexpr int NFLOAT = NV * (C::SCELLS + C::FMAX) + C::TROWS * C::SV;
  double* sred = reinterpret_cast<double*>(su + ((NFLOAT + 1) & ~1));
  const Geom& g = a.g;
  const Phys& p = a.p;
  const PhysF& pf = a.pf;
  const int i0 = blockIdx.x * BX, j0 = blockIdx.y * BY, k0 = blockIdx.z * BZ;

  for (int id = threadIdx.x; id < NV * C::SCELLS; id += NT) {
    const int v = id / C::SCELLS;
    const int r = id - v * C::SCELLS;
    const int lx = r % C::SX;
    const int t = r / C::SX;
    const int ly = t % C::SY;
    const int lz = t / C::SY;
    const int gi = i0 + lx - C::HX, gj = j0 + ly - C::HY, gk = k0 + lz - C::HZ;
    float val = 0.0f;
    if (gi <= g.n[0] + 1 && (NDIM < 2 || gj <= g.n[1] + 1) && (NDIM < 3 || gk <= g.n[2] + 1))
      val = a.in[v * g.fstride + pidx(g, gi, gj, gk)];
    su[id] = val;
  }
  if constexpr (VERT >= 0) {
    const int baseV = VERT == 0 ? i0 : (VERT == 1 ? j0 : k0);  // padded index of tile row 0 (interior - 2)
    for (int id = threadIdx.x; id < C::TROWS * C::SV; id += NT) {
      const int f = id / C::SV, r = id - f * C::SV;
      const int kp = baseV + r;
      st[id] = kp < a.tab_len ? a.tab[(size_t)f * a.tab_len + kp] : 0.0f;
    }
  }
  __syncthreads();

  float dU[C::CPT][NV];
#pragma unroll
  for (int c = 0; c < C::CPT; ++c)
#pragma unroll
    for (int v = 0; v < NV; ++v) dU[c][v] = 0.0f;
  face_pass_f<NDIM, VERT, BX, BY, BZ, NT, 0>(su, sf, st, pf, g, i0, j0, k0, dU);
  if constexpr (NDIM >= 2) face_pass_f<NDIM, VERT, BX, BY, BZ, NT, 1>(su, sf, st, pf, g, i0, j0, k0, dU);
  if constexpr (NDIM >= 3) face_pass_f<NDIM, VERT, BX, BY, BZ, NT, 2>(su, sf, st, pf, g, i0, j0, k0, dU);

  const double dtd = a.dt_fixed > 0.0 ? a.dt_fixed : p.cfl / a.scal[a.slot];
  const float dt = (float)dtd;
  if (a.stage == 1 && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && threadIdx.x == 0) {
    a.scal[a.slot ^ 1] = 0.0;
    a.scal[2] = dtd;
    a.scal[3] += dtd;
  }
  float rmax = 0.0f;
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
    float q[NV], L[NV], Dl[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      q[v] = su[v * C::SCELLS + s0];
      L[v] = dU[c][v];
      Dl[v] = dU[c][v];
    }
    float rho0 = 0.0f, P0 = 0.0f;
    if constexpr (VERT >= 0) {
      const int row = (VERT == 0 ? cx : (VERT == 1 ? cy : cz)) + (VERT == 0 ? C::HX : (VERT == 1 ? C::HY : C::HZ));
      rho0 = st[TB_RHO0 * C::SV + row];
      P0 = st[TB_P0 * C::SV + row];
      Dl[0] += st[TB_D0RHO * C::SV + row];
      Dl[1 + VERT] += st[TB_D0MV * C::SV + row];
      Dl[NV - 1] += st[TB_D0E * C::SV + row];
#pragma unroll
      for (int v = 0; v < NV; ++v) L[v] += st[(TB_R0 + v) * C::SV + row];
    }
    // full-state primitives from perturbation-sized terms
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
    const float P1 = pf.gm1 * (q[NV - 1] - 0.5f * mv);
    const float P = P0 + P1;
    if (p.variant != RSST_EULER) {
      const int var = p.variant;
      const float e_int = P * pf.inv_gm1;
      const float kin = 0.5f * mv;
      float s, r0, rv, rE;
      if (var == RSST_PVS || var == RSST_PMS || var == RSST_PD) {
        s = pf.gm1 * (0.5f * v2 * Dl[0] - vdm + Dl[NV - 1]);
        if (var == RSST_PD) {
          r0 = 0.0f; rv = 0.0f; rE = pf.inv_gm1;
        } else {
          const float ia2 = rho / (pf.gamma * P);
          r0 = ia2;
          rv = var == RSST_PVS ? ia2 : 0.0f;
          rE = (var == RSST_PVS ? (e_int + P + kin) : (e_int + P - kin)) * ia2 * ir;
        }
      } else {
        s = Dl[0];
        r0 = 1.0f;
        rv = var == RSST_DVS ? 1.0f : 0.0f;
        rE = (var == RSST_DVS ? (e_int + P + kin) : (e_int + P - kin)) * ir;
      }
      const float fs = f_of_f(pf.gamma * P * ir, pf) * s;
      L[0] -= fs * r0;
#pragma unroll
      for (int e = 0; e < ND; ++e) L[1 + e] -= fs * (rv * vel[e]);
      L[NV - 1] -= fs * rE;
    }
    if (p.has_grav) {
      float mg = 0.0f;
#pragma unroll
      for (int e = 0; e < ND; ++e) {
        L[1 + e] += q[0] * pf.grav[e];  // rho0 * g is part of R0
        mg += q[1 + e] * pf.grav[e];
      }
      L[NV - 1] += mg;
    }
    float u[NV];
    if (a.stage == 1) {
#pragma unroll
      for (int v = 0; v < NV; ++v) u[v] = q[v] + dt * L[v];
    } else {
      const int64_t o = pidx(g, i, j, k);
#pragma unroll
      for (int v = 0; v < NV; ++v) u[v] = 0.5f * a.base[v * g.fstride + o] + 0.5f * (q[v] + dt * L[v]);
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
      const bool ok = fin && rn > 0.0f && Pn > 0.0f;
      if (ok) rmax = fmaxf(rmax, (sqrtf(w2) + sound_over_xi_f(pf.gamma * Pn * irn, pf)) * pf.sum_inv_dx);
      ok_all = ok_all && ok;
    }
    store_mirror_ghosts<float, NV>(a.out, g, p, i, j, k, u);
  }
  if (a.stage == 2) {
    if (!ok_all) atomicOr(a.flag, RSST_FLAG_NONPHYSICAL);
    block_max_to<NT>((double)rmax, a.scal + (a.slot ^ 1), sred);
  }
}

// ---------------------------------------------------------------------------
// Packing, CFL maximum, sums (float32 storage)
// ---------------------------------------------------------------------------

__device__ __forceinline__ void bg_at(const double* bg, int bg_len, int kpad, double& r0, double& e0) {
  if (bg) {
    r0 = bg[kpad];
    e0 = bg[bg_len + kpad];
  } else {
    r0 = 0.0;
    e0 = 0.0;
  }
}

// U1 = U - U0 at interior cells; ghosts: wrap, or mirror of U1 (normal momentum negated).
__global__ void pack_fp32_kernel(const double* __restrict__ src, float* __restrict__ dst, Geom g, Phys p,
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
    for (int d = 0; d < g.ndim; ++d) {
      const int n = g.n[d];
      if (s[d] >= 0 && s[d] < n) continue;
      if (p.bc[d] == RSST_BC_PERIODIC) {
        s[d] = (s[d] + n) % n;
      } else {
        s[d] = s[d] < 0 ? -1 - s[d] : 2 * n - 1 - s[d];
        sign[d] = -1.0;
      }
    }
    double r0 = 0.0, e0 = 0.0;
    if (p.vertical >= 0) bg_at(bg, bg_len, s[p.vertical] + RSST_G, r0, e0);
    const int64_t si = ((int64_t)s[2] * g.n[1] + s[1]) * g.n[0] + s[0];
    const int64_t di = pidx(g, c[0], c[1], c[2]);
    for (int v = 0; v < nv; ++v) {
      double w = src[v * g.ncells + si];
      if (v == 0) w -= r0;
      if (v == nv - 1) w -= e0;
      if (v >= 1 && v <= g.ndim) w *= sign[v - 1];
      dst[v * g.fstride + di] = (float)w;
    }
  }
}

__global__ void unpack_fp32_kernel(const float* __restrict__ src, double* __restrict__ dst, Geom g, Phys p,
                                   const double* __restrict__ bg, int bg_len) {
  const int nv = g.ndim + 2;
  for (int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; id < g.ncells; id += (int64_t)gridDim.x * blockDim.x) {
    const int c[3] = {(int)(id % g.n[0]), (int)((id / g.n[0]) % g.n[1]), (int)(id / ((int64_t)g.n[0] * g.n[1]))};
    const int64_t o = pidx(g, c[0], c[1], c[2]);
    double r0 = 0.0, e0 = 0.0;
    if (p.vertical >= 0) bg_at(bg, bg_len, c[p.vertical] + RSST_G, r0, e0);
    for (int v = 0; v < nv; ++v) {
      double w = (double)src[v * g.fstride + o];
      if (v == 0) w += r0;
      if (v == nv - 1) w += e0;
      dst[v * g.ncells + id] = w;
    }
  }
}

template <int NV>
__global__ void __launch_bounds__(256) cfl_fp32_kernel(const float* __restrict__ U, Geom g, Phys p, PhysF pf,
                                                       const float* __restrict__ tab, int tab_len, double* dst,
                                                       unsigned int* flag) {
  constexpr int ND = NV - 2;
  __shared__ double sred[8];
  float rmax = 0.0f;
  bool ok_all = true;
  for (int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; id < g.ncells; id += (int64_t)gridDim.x * blockDim.x) {
    const int c[3] = {(int)(id % g.n[0]), (int)((id / g.n[0]) % g.n[1]), (int)(id / ((int64_t)g.n[0] * g.n[1]))};
    const int64_t o = pidx(g, c[0], c[1], c[2]);
    float rho0 = 0.0f, P0 = 0.0f;
    if (tab) {
      const int kp = c[p.vertical] + RSST_G;
      rho0 = tab[TB_RHO0 * tab_len + kp];
      P0 = tab[TB_P0 * tab_len + kp];
    }
    float u[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) u[v] = U[v * g.fstride + o];
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
    const bool ok = fin && rn > 0.0f && Pn > 0.0f;
    if (ok) rmax = fmaxf(rmax, (sqrtf(w2) + sound_over_xi_f(pf.gamma * Pn * irn, pf)) * pf.sum_inv_dx);
    ok_all = ok_all && ok;
  }
  if (!ok_all) atomicOr(flag, RSST_FLAG_NONPHYSICAL);
  block_max_to<256>((double)rmax, dst, sred);
}

constexpr int SUM_BLOCKS32 = 1024;
constexpr int SUM_THREADS32 = 256;

__global__ void __launch_bounds__(SUM_THREADS32) sums_partial_fp32_kernel(const float* __restrict__ U, Geom g, Phys p,
                                                                          const double* __restrict__ bg, int bg_len,
                                                                          double* __restrict__ partial) {
  __shared__ double sh[SUM_THREADS32];
  const int nv = g.ndim + 2;
  const int64_t chunk = (g.ncells + SUM_BLOCKS32 - 1) / SUM_BLOCKS32;
  const int64_t lo = blockIdx.x * chunk;
  const int64_t hi = min(g.ncells, lo + chunk);
  for (int v = 0; v < nv; ++v) {
    double acc = 0.0;
    for (int64_t id = lo + threadIdx.x; id < hi; id += SUM_THREADS32) {
      const int c[3] = {(int)(id % g.n[0]), (int)((id / g.n[0]) % g.n[1]), (int)(id / ((int64_t)g.n[0] * g.n[1]))};
      double w = (double)U[v * g.fstride + pidx(g, c[0], c[1], c[2])];
      if (p.vertical >= 0 && (v == 0 || v == nv - 1)) {
        double r0, e0;
        bg_at(bg, bg_len, c[p.vertical] + RSST_G, r0, e0);
        w += v == 0 ? r0 : e0;
      }
      acc += w;
    }
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int s = SUM_THREADS32 / 2; s > 0; s >>= 1) {
      if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
      __syncthreads();
    }
    if (threadIdx.x == 0) partial[v * SUM_BLOCKS32 + blockIdx.x] = sh[0];
    __syncthreads();
  }
}

__global__ void __launch_bounds__(SUM_THREADS32) sums_final32_kernel(const double* __restrict__ partial, int nv,
                                                                     double scale, double* __restrict__ out) {
  __shared__ double sh[SUM_THREADS32];
  for (int v = 0; v < nv; ++v) {
    double acc = 0.0;
    for (int b = threadIdx.x; b < SUM_BLOCKS32; b += SUM_THREADS32) acc += partial[v * SUM_BLOCKS32 + b];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int s = SUM_THREADS32 / 2; s > 0; s >>= 1) {
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

static int check_launch32(const char* what) {
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    rsst_set_error("%s launch: %s", what, cudaGetErrorString(e));
    return RSST_ECUDA;
  }
  return RSST_OK;
}

template <int NDIM, int VERT, int BX, int BY, int BZ, int NT>
static int launch_stage32(const StageArgs<float>& a, cudaStream_t s) {
  using C = TileCfgF<NDIM, VERT, BX, BY, BZ, NT>;
  auto kern = stage_fp32_kernel<NDIM, VERT, BX, BY, BZ, NT>;
  static std::atomic<unsigned long long> attr{0};
  if (set_smem_limit_once(kern, C::SMEM, attr) != cudaSuccess) {
    rsst_set_error("cudaFuncSetAttribute failed for the float32 stage kernel");
    return RSST_ECUDA;
  }
  dim3 grid((a.g.n[0] + BX - 1) / BX, NDIM >= 2 ? (a.g.n[1] + BY - 1) / BY : 1, NDIM >= 3 ? (a.g.n[2] + BZ - 1) / BZ : 1);
  kern<<<grid, NT, C::SMEM, s>>>(a);
  return check_launch32("float32 stage kernel");
}

template <int NDIM, int VERT>
static int launch_stage32_dim(const StageArgs<float>& a, cudaStream_t s) {
  if constexpr (NDIM == 1) {
    if (a.g.n[0] <= RSST_SMALL_1D) return launch_stage32<1, VERT, 16, 1, 1, 32>(a, s);
    return launch_stage32<1, VERT, 256, 1, 1, 256>(a, s);
  }
  if constexpr (NDIM == 2) return launch_stage32<2, VERT, 64, 16, 1, 256>(a, s);
  if constexpr (NDIM == 3) return launch_stage32<3, VERT, 32, 8, 4, 256>(a, s);
  return RSST_EINVAL;
}

}  // namespace rsst

using namespace rsst;

int rsst_launch_stage_fp32(const StageArgs<float>& a, cudaStream_t s) {
  const int v = a.tab ? a.p.vertical : -1;
  switch (a.g.ndim) {
    case 1:
      return v < 0 ? launch_stage32_dim<1, -1>(a, s) : launch_stage32_dim<1, 0>(a, s);
    case 2:
      return v < 0 ? launch_stage32_dim<2, -1>(a, s) : (v == 0 ? launch_stage32_dim<2, 0>(a, s) : launch_stage32_dim<2, 1>(a, s));
    case 3:
      if (v < 0) return launch_stage32_dim<3, -1>(a, s);
      if (v == 0) return launch_stage32_dim<3, 0>(a, s);
      if (v == 1) return launch_stage32_dim<3, 1>(a, s);
      return launch_stage32_dim<3, 2>(a, s);
  }
  rsst_set_error("ndim must be 1, 2 or 3");
  return RSST_EINVAL;
}

int rsst_launch_bgtab(const double* bg, int bg_len, const Geom& g, const Phys& p, float* tab, float* tabr,
                      cudaStream_t s) {
  const int blocks = (bg_len + 127) / 128;
  const int nv = g.ndim + 2, V = p.vertical;
#define BG(NVv, Vv) bgtab_kernel<NVv, Vv><<<blocks, 128, 0, s>>>(bg, bg_len, p, tab, tabr)
  if (nv == 3) BG(3, 0);
  else if (nv == 4) { if (V == 0) BG(4, 0); else BG(4, 1); }
  else { if (V == 0) BG(5, 0); else if (V == 1) BG(5, 1); else BG(5, 2); }
#undef BG
  return check_launch32("background table");
}

static int grid_for32(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b > 152 * 16) b = 152 * 16;
  return (int)(b < 1 ? 1 : b);
}

int rsst_launch_pack_fp32(const double* src, float* dst, const Geom& g, const Phys& p, const double* bg, int bg_len,
                          cudaStream_t s) {
  const int64_t total = (int64_t)(g.n[0] + 4) * (g.ndim >= 2 ? g.n[1] + 4 : 1) * (g.ndim >= 3 ? g.n[2] + 4 : 1);
  pack_fp32_kernel<<<grid_for32(total), 256, 0, s>>>(src, dst, g, p, bg, bg_len);
  return check_launch32("pack (float32)");
}

int rsst_launch_unpack_fp32(const float* src, double* dst, const Geom& g, const Phys& p, const double* bg, int bg_len,
                            cudaStream_t s) {
  unpack_fp32_kernel<<<grid_for32(g.ncells), 256, 0, s>>>(src, dst, g, p, bg, bg_len);
  return check_launch32("unpack (float32)");
}

int rsst_launch_cfl_fp32(const float* U, const Geom& g, const Phys& p, const PhysF& pf, const float* tab, int tab_len,
                         double* slot_ptr, unsigned int* flag, cudaStream_t s) {
  const int gb = grid_for32(g.ncells);
  switch (g.ndim) {
    case 1: cfl_fp32_kernel<3><<<gb, 256, 0, s>>>(U, g, p, pf, tab, tab_len, slot_ptr, flag); break;
    case 2: cfl_fp32_kernel<4><<<gb, 256, 0, s>>>(U, g, p, pf, tab, tab_len, slot_ptr, flag); break;
    default: cfl_fp32_kernel<5><<<gb, 256, 0, s>>>(U, g, p, pf, tab, tab_len, slot_ptr, flag); break;
  }
  return check_launch32("cfl (float32)");
}

int rsst_launch_sums_fp32(const float* U, const Geom& g, const Phys& p, const double* bg, int bg_len, double* partial,
                          double* out, double scale, cudaStream_t s) {
  sums_partial_fp32_kernel<<<SUM_BLOCKS32, SUM_THREADS32, 0, s>>>(U, g, p, bg, bg_len, partial);
  int rc = check_launch32("sums (float32)");
  if (rc) return rc;
  sums_final32_kernel<<<1, SUM_THREADS32, 0, s>>>(partial, g.ndim + 2, scale, out);
  return check_launch32("sums final (float32)");
}
