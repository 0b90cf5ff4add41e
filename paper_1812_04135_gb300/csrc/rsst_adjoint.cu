// Discrete adjoint of the float64 SSP-RK2 step (the transpose of the
// Jacobian of the discrete map U^n -> U^{n+1}, dt held fixed), with
// checkpoint-and-recompute.  The paper has no adjoint; the conventions
// (fixed dt, forward branch of every non-smooth operation: MC branch, LLF
// max with ties to the left state, zero subgradient of |V| at V = 0) are
// this library's and match the oracle's reverse-mode derivative.
//
// One stage is out = a * base + b * (in + dt L(in)).  Its adjoint needs the
// vector-Jacobian product mu^T dL/d(in) (mu = b dt lambda_out) and
// mu^T dL/dxi:
//   adj_cell: per interior cell, with the Euler tendency dU that the forward
//     kernel wrote while the segment was recomputed, nu = mu^T dC/d(dU) and
//     the pointwise part mu^T d(C + force)/dq (C = reduced tendency, Sec. 3.2 /
//     App. A; force of App. B) plus the identity part b lambda_out, and the
//     xi partial;
//   adj_face: per face, phi = (nu_right - nu_left)/dx, then phi^T dF/dU_k for
//     the four stencil cells k of the face (MC slopes, face states, LLF flux
//     of Sec. 4.2) and the xi partial;
//   adj_gather: each padded cell (interior and edge ghosts) sums the
//     contributions of the faces whose stencil holds it;
//   adj_fold: ghost-cell adjoints go back to the cells they were copied from
//     (wrap, or mirror with the normal momentum negated).
// The derivatives are hand-derived reverse mode: each VJP recomputes its
// forward values (holding the branches the forward pass took) and then runs
// the chain rule backwards once, so a face costs about three flux
// evaluations whatever the size of its stencil.  Divisions go through the
// forward kernels' Newton-Raphson reciprocal and the square roots of c_tot
// through their c_tot square root (float64 pipe economy; same readings).
#include <cstring>
#include <vector>

#include "rsst_common.cuh"
#include "rsst_internal.h"
#include "rsst_check.h"
#include "rsst_math_fp64.cuh"

namespace rsst {

// |V| with a zero subgradient at V = 0.
__device__ __forceinline__ double speed_of(double v2) { return v2 > 0.0 ? sqrt_ctot(v2) : 0.0; }

// MC branch (Sec. 4.2): 0 -> 0, 1 -> 2a, 2 -> 2b, 3 -> (a+b)/2; the
// decisions of the oracle's comparisons (2|a| <= 2|b| and 2|a| <= |a+b|/2,
// then 2|b| <= |a+b|/2), taken on the integer pipe as in mc_slope.
__device__ __forceinline__ int mc_branch(double a, double b) {
  const unsigned long long four = 1ull << 54;  // x4 in the shifted exponent field
  const long long ia = __double_as_longlong(a), ib = __double_as_longlong(b);
  const unsigned long long ua = (unsigned long long)ia << 1, ub = (unsigned long long)ib << 1;
  if (!(((ia ^ ib) >= 0) && ua != 0 && ub != 0)) return 0;
  const unsigned long long us = (unsigned long long)__double_as_longlong(a + b) << 1;
  if (ua <= ub && ua + four <= us) return 1;
  return ub + four <= us ? 2 : 3;
}
__device__ __forceinline__ double mc_value(int br, double a, double b) {
  return br == 0 ? 0.0 : (br == 1 ? 2.0 * a : (br == 2 ? 2.0 * b : 0.5 * (a + b)));
}
// d(slope)/da and d(slope)/db of the taken branch, times the slope's adjoint ds.
__device__ __forceinline__ void mc_reverse(int br, double ds, double& da, double& db) {
  da = br == 1 ? 2.0 * ds : (br == 3 ? 0.5 * ds : 0.0);
  db = br == 2 ? 2.0 * ds : (br == 3 ? 0.5 * ds : 0.0);
}

// a/xi of a state (constant xi, or the C_max law, Eq. cx).
__device__ __forceinline__ double sound_term(double a2, const Phys& p) {
  if (p.use_cmax) return sqrt(a2 * rcp_nr(sqrt(1.0 + (a2 * a2) * p.inv_cmax4)));
  return sqrt_ctot(a2) * p.inv_xi;
}

// The forward values of one face state that the reverse of its flux reuses:
// 1/rho, V, |V|^2, P, a^2, |V| and (constant xi) a.
template <int NV>
struct StateFwd {
  double ir, v[NV - 2], v2, P, a2, sv, sa;
};

// c_tot = |V| + a/xi of one face state (Sec. 4.2; the LLF speed), keeping the
// values its flux's reverse needs.  (The flux itself enters the VJP only
// through its derivatives.)
template <int NV>
__device__ __forceinline__ double state_fwd(const double (&q)[NV], const Phys& p, StateFwd<NV>& w) {
  constexpr int ND = NV - 2;
  const double rho = q[0];
  w.ir = rcp_nr(rho);
  w.v2 = 0.0;
  for (int e = 0; e < ND; ++e) {
    w.v[e] = q[1 + e] * w.ir;
    w.v2 += w.v[e] * w.v[e];
  }
  w.P = p.gm1 * (q[NV - 1] - 0.5 * (rho * w.v2));
  w.a2 = p.gamma * w.P * w.ir;
  w.sv = speed_of(w.v2);
  if (p.use_cmax) {
    w.sa = 0.0;
    return w.sv + sound_term(w.a2, p);
  }
  w.sa = sqrt_ctot(w.a2);
  return w.sv + w.sa * p.inv_xi;
}

// Face states of the face between u0 | u1 from the stencil (um, u0 | u1, up):
// MUSCL-MC reconstruction, with the branches taken.
template <int NV>
__device__ __forceinline__ void face_states(const double (&s)[4][NV], double (&qL)[NV], double (&qR)[NV],
                                            int (&bL)[NV], int (&bR)[NV]) {
  for (int v = 0; v < NV; ++v) {
    const double aL = s[1][v] - s[0][v], dL = s[2][v] - s[1][v];
    const double aR = s[2][v] - s[1][v], dR = s[3][v] - s[2][v];
    bL[v] = mc_branch(aL, dL);
    bR[v] = mc_branch(aR, dR);
    qL[v] = s[1][v] + 0.5 * mc_value(bL[v], aL, dL);
    qR[v] = s[2][v] - 0.5 * mc_value(bR[v], aR, dR);
  }
}

// Reverse of the Euler flux along D (F_D = (m_D, m V_D + P e_D, (E + P) V_D))
// and of c_tot at q, with w = state_fwd's values at q: adds dF^T dF/dq +
// dc dc/dq to dq and returns dF^T dF/d(1/xi) + dc dc/d(1/xi).  Hand-derived
// chain rule through v = m/rho, P = (gamma-1)(E - rho|v|^2/2), a^2 = gamma P/rho.
template <int NV, int D>
__device__ __forceinline__ double flux_vjp(const double (&q)[NV], const Phys& p, const StateFwd<NV>& w,
                                           const double (&dF)[NV], double dc, double (&dq)[NV]) {
  constexpr int ND = NV - 2;
  const double rho = q[0], E = q[NV - 1];
  const double ir = w.ir, v2 = w.v2, P = w.P, a2 = w.a2;
  const double(&v)[ND] = w.v;
  double dv[ND];
  for (int e = 0; e < ND; ++e) dv[e] = 0.0;
  double dP = dF[1 + D] + dF[NV - 1] * v[D], dv2 = 0.0, drho = 0.0, dE = dF[NV - 1] * v[D], dinv_xi = 0.0;
  dq[1 + D] += dF[0];
  for (int e = 0; e < ND; ++e) {
    dq[1 + e] += dF[1 + e] * v[D];
    dv[D] += dF[1 + e] * q[1 + e];
  }
  dv[D] += dF[NV - 1] * (E + P);
  if (v2 > 0.0) dv2 += dc * 0.5 * rcp_nr(w.sv);
  double da2 = 0.0;
  if (p.use_cmax) {  // g = sqrt(u), u = a2 / t, t = sqrt(w), w = 1 + a2^2 / C^4
    const double w = 1.0 + (a2 * a2) * p.inv_cmax4, t = sqrt(w), it = rcp_nr(t), u = a2 * it;
    if (u > 0.0) {
      const double du = dc * 0.5 * rcp_nr(sqrt(u));
      const double dt = -du * u * it;
      da2 += du * it + dt * it * a2 * p.inv_cmax4;
    }
  } else {
    const double s = w.sa;
    dinv_xi += dc * s;
    if (a2 > 0.0) da2 += dc * p.inv_xi * 0.5 * rcp_nr(s);
  }
  dP += da2 * p.gamma * ir;
  drho -= da2 * a2 * ir;
  dE += dP * p.gm1;
  drho -= dP * p.gm1 * 0.5 * v2;
  dv2 -= dP * p.gm1 * 0.5 * rho;
  for (int e = 0; e < ND; ++e) {
    dv[e] += 2.0 * v[e] * dv2;
    dq[1 + e] += dv[e] * ir;
    drho -= dv[e] * v[e] * ir;
  }
  dq[0] += drho;
  dq[NV - 1] += dE;
  return dinv_xi;
}

// Reverse of the face's LLF flux (Sec. 4.2, steps 2-4, through its MUSCL-MC
// states): G[k] = phi^T dF/d(stencil cell k), and the return
// value phi^T dF/d(1/xi).  The forward branches (MC branch, LLF side) are
// recomputed and held.
template <int NV, int D>
__device__ __forceinline__ double face_vjp(const double (&s)[4][NV], const double (&phi)[NV], const Phys& p,
                                           double (&G)[4][NV]) {
  double qL[NV], qR[NV];
  int bL[NV], bR[NV];
  face_states<NV>(s, qL, qR, bL, bR);
  StateFwd<NV> wL, wR;
  const double cL = state_fwd<NV>(qL, p, wL);
  const double cR = state_fwd<NV>(qR, p, wR);
  const bool left = cL >= cR;
  const double alpha = left ? cL : cR;
  double dF[NV], dqL[NV], dqR[NV], dalpha = 0.0;
  for (int v = 0; v < NV; ++v) {
    dF[v] = 0.5 * phi[v];
    dqL[v] = 0.5 * alpha * phi[v];
    dqR[v] = -0.5 * alpha * phi[v];
    dalpha -= 0.5 * phi[v] * (qR[v] - qL[v]);
  }
  double dinv_xi = flux_vjp<NV, D>(qL, p, wL, dF, left ? dalpha : 0.0, dqL);
  dinv_xi += flux_vjp<NV, D>(qR, p, wR, dF, left ? 0.0 : dalpha, dqR);
  for (int v = 0; v < NV; ++v) {
    double da, db;
    // qL = u0 + MC(u0 - um, u1 - u0)/2
    mc_reverse(bL[v], 0.5 * dqL[v], da, db);
    G[0][v] = -da;
    G[1][v] = dqL[v] + da - db;
    G[2][v] = db;
    // qR = u1 - MC(u1 - u0, up - u1)/2
    mc_reverse(bR[v], -0.5 * dqR[v], da, db);
    G[1][v] -= da;
    G[2][v] += dqR[v] + da - db;
    G[3][v] = db;
  }
  return dinv_xi;
}

// Reverse of the reduced tendency plus force at one cell,
//   L = dU - f s r + (0, rho F, m.F)   (Sec. 3.2, App. A, App. B),
// for the cotangent mu: nu = mu^T dL/d(dU), dq = mu^T dL/dq, and the return
// value mu^T dL/df (zero under the C_max law, where f comes from the state).
// With w = mu . r the correction contributes -f s w, so ds = -f w, dw = -f s.
template <int NV>
__device__ __forceinline__ double rhs_vjp(const double (&q)[NV], const double (&dU)[NV], const double (&mu)[NV],
                                          const Phys& p, double (&nu)[NV], double (&dq)[NV]) {
  constexpr int ND = NV - 2;
  const double rho = q[0];
  double dfc_total = 0.0;
  for (int v = 0; v < NV; ++v) {
    nu[v] = mu[v];
    dq[v] = 0.0;
  }
  const int var = p.variant;
  if (var != RSST_EULER) {
    const double ir = rcp_nr(rho);
    double v[ND], dv[ND];
    double v2 = 0.0, vdm = 0.0, mv = 0.0;
    for (int e = 0; e < ND; ++e) {
      v[e] = q[1 + e] * ir;
      v2 += v[e] * v[e];
      vdm += v[e] * dU[1 + e];
      mv += mu[1 + e] * v[e];
      dv[e] = 0.0;
    }
    const double E = q[NV - 1];
    const double P = p.gm1 * (E - 0.5 * (rho * v2));
    const double kin = 0.5 * (rho * v2);
    const bool pform = var == RSST_PVS || var == RSST_PMS || var == RSST_PD;
    const double sgn = (var == RSST_PVS || var == RSST_DVS) ? 1.0 : -1.0;
    const double H = P * p.inv_gm1 + P + sgn * kin;  // e + P +- rho|V|^2/2
    double s, r0, rv, rE, ia2 = 0.0, igP = 0.0;  // igP = 1/(gamma P)
    if (pform) {
      s = p.gm1 * (0.5 * (v2 * dU[0]) - vdm + dU[NV - 1]);
      if (var == RSST_PD) {
        r0 = 0.0; rv = 0.0; rE = p.inv_gm1;
      } else {
        igP = rcp_nr(p.gamma * P);
        ia2 = rho * igP;
        r0 = ia2;
        rv = var == RSST_PVS ? ia2 : 0.0;
        rE = H * ia2 * ir;
      }
    } else {
      s = dU[0];
      r0 = 1.0;
      rv = var == RSST_DVS ? 1.0 : 0.0;
      rE = H * ir;
    }
    double a2 = 0.0, wc = 0.0, fc = p.f;
    if (p.use_cmax) {
      a2 = p.gamma * P * ir;
      wc = 1.0 + (a2 * a2) * p.inv_cmax4;
      fc = 1.0 - rcp_nr(sqrt(wc));
    }
    const double w = mu[0] * r0 + rv * mv + mu[NV - 1] * rE;
    const double ds = -fc * w, dw = -fc * s, dfc = -s * w;
    double dv2 = 0.0, drho = 0.0, dP = 0.0, dH = 0.0;
    if (pform) {
      nu[0] += ds * p.gm1 * 0.5 * v2;
      for (int e = 0; e < ND; ++e) {
        nu[1 + e] -= ds * p.gm1 * v[e];
        dv[e] -= ds * p.gm1 * dU[1 + e];
      }
      nu[NV - 1] += ds * p.gm1;
      dv2 += ds * p.gm1 * 0.5 * dU[0];
    } else {
      nu[0] += ds;
    }
    for (int e = 0; e < ND; ++e) dv[e] += dw * rv * mu[1 + e];
    if (var == RSST_PVS || var == RSST_PMS) {
      double dia2 = dw * mu[0] + (var == RSST_PVS ? dw * mv : 0.0);
      const double drE = dw * mu[NV - 1];
      dH = drE * ia2 * ir;
      dia2 += drE * H * ir;
      drho -= drE * rE * ir;
      drho += dia2 * igP;
      dP -= dia2 * ia2 * (p.gamma * igP);  // ia2 / P
    } else if (var == RSST_DVS || var == RSST_DMS) {
      dH = dw * mu[NV - 1] * ir;
      drho -= dw * mu[NV - 1] * rE * ir;
    }
    dP += dH * (p.inv_gm1 + 1.0);
    const double dkin = sgn * dH;
    if (p.use_cmax) {
      const double da2 = dfc * p.inv_cmax4 * a2 * rcp_nr(wc * sqrt(wc));
      dP += da2 * p.gamma * ir;
      drho -= da2 * a2 * ir;
    } else {
      dfc_total = dfc;
    }
    drho += dkin * 0.5 * v2;
    dv2 += dkin * 0.5 * rho;
    dq[NV - 1] += dP * p.gm1;
    drho -= dP * p.gm1 * 0.5 * v2;
    dv2 -= dP * p.gm1 * 0.5 * rho;
    for (int e = 0; e < ND; ++e) {
      dv[e] += 2.0 * v[e] * dv2;
      dq[1 + e] += dv[e] * ir;
      drho -= dv[e] * v[e] * ir;
    }
    dq[0] += drho;
  }
  if (p.has_grav) {
    for (int e = 0; e < ND; ++e) {
      dq[0] += mu[1 + e] * p.grav[e];
      dq[1 + e] += mu[NV - 1] * p.grav[e];
    }
  }
  return dfc_total;
}

struct AdjArgs {
  const double* U;   // stage input, padded
  const double* dU;  // its Euler tendency, padded (written by the forward kernel on recompute)
  const double* lam_out;  // lambda of the stage output, padded (interior used)
  double mu_scale;        // mu = mu_scale * lambda_out = b dt lambda_out
  double id_scale;        // the stage's identity part adds id_scale * lambda_out = b lambda_out
  double* nu;        // padded, interior written (ghosts stay zero)
  double* lam;       // padded output: pointwise part written to the interior
  double* faceG;     // per axis: [face][4][NV]
  double* part;      // per-block xi partials
  Geom g;
  Phys p;
  int64_t face_off[3];  // offset of each axis' block in faceG (in faces)
};

__device__ __forceinline__ int64_t pidx_c(const Geom& g, const int (&c)[3]) { return pidx(g, c[0], c[1], c[2]); }

__device__ __forceinline__ void block_sum_to(double x, double* dst, double* sh) {
  sh[threadIdx.x] = x;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) *dst = sh[0];
}

template <int NV, int D>
__device__ __forceinline__ void load_stencil(const AdjArgs& a, const int (&c)[3], double (&s)[4][NV]) {
  // cells c - 2 .. c + 1 along D (the face c - 1/2)
  for (int k = 0; k < 4; ++k) {
    int cc[3] = {c[0], c[1], c[2]};
    cc[D] += k - 2;
    const int64_t o = pidx_c(a.g, cc);
    for (int v = 0; v < NV; ++v) s[k][v] = a.U[v * a.g.fstride + o];
  }
}

template <int NV>
__global__ void __launch_bounds__(128) adj_cell_kernel(AdjArgs a) {
  __shared__ double sh[128];
  const Geom& g = a.g;
  const Phys& p = a.p;
  double dxi = 0.0;
  const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (id < g.ncells) {
    const int c[3] = {(int)(id % g.n[0]), (int)((id / g.n[0]) % g.n[1]), (int)(id / ((int64_t)g.n[0] * g.n[1]))};
    const int64_t o = pidx_c(g, c);
    double q[NV], dU[NV], mu[NV];
    for (int v = 0; v < NV; ++v) {
      q[v] = a.U[v * g.fstride + o];
      mu[v] = a.mu_scale * a.lam_out[v * g.fstride + o];
      dU[v] = a.dU[v * g.fstride + o];
    }
    // nu = mu^T dL/d(dU), pointwise mu^T dL/dq, xi partial (f = 1 - 1/xi^2)
    double nu[NV], dq[NV];
    const double df = rhs_vjp<NV>(q, dU, mu, p, nu, dq);
    for (int v = 0; v < NV; ++v) {
      a.nu[v * g.fstride + o] = nu[v];
      a.lam[v * g.fstride + o] = fma(a.id_scale, a.lam_out[v * g.fstride + o], dq[v]);
    }
    const double xi = p.xi;
    dxi = df * 2.0 / (xi * xi * xi);
  }
  block_sum_to(dxi, a.part + blockIdx.x, sh);
}

// Faces along D: index (f, other coords) with f in [0, n_D] (face f - 1/2).
template <int NV, int D>
__global__ void __launch_bounds__(128) adj_face_kernel(AdjArgs a, int part_off) {
  __shared__ double sh[128];
  const Geom& g = a.g;
  const Phys& p = a.p;
  int ext[3] = {g.n[0], g.n[1], g.n[2]};
  ext[D] += 1;
  const int64_t nf = (int64_t)ext[0] * ext[1] * ext[2];
  const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double dxi = 0.0;
  if (id < nf) {
    const int c[3] = {(int)(id % ext[0]), (int)((id / ext[0]) % ext[1]), (int)(id / ((int64_t)ext[0] * ext[1]))};
    const int f = c[D];
    double s[4][NV];
    load_stencil<NV, D>(a, c, s);
    // phi = (nu_right - nu_left) / dx, nu = 0 outside the interior
    double phi[NV];
    {
      int cr[3] = {c[0], c[1], c[2]}, cl[3] = {c[0], c[1], c[2]};
      cl[D] -= 1;
      const bool has_r = f < g.n[D], has_l = f > 0;
      const int64_t orr = pidx_c(g, cr), ol = pidx_c(g, cl);
      for (int v = 0; v < NV; ++v) {
        const double nr = has_r ? a.nu[v * g.fstride + orr] : 0.0;
        const double nl = has_l ? a.nu[v * g.fstride + ol] : 0.0;
        phi[v] = (nr - nl) * p.inv_dx[D];
      }
    }
    double G[4][NV];
    const double dinv_xi = face_vjp<NV, D>(s, phi, p, G);
    double* dst = a.faceG + (a.face_off[D] + id) * (4 * NV);
    for (int k = 0; k < 4; ++k)
      for (int v = 0; v < NV; ++v) dst[k * NV + v] = G[k][v];
    const double xi = p.xi;
    dxi = -dinv_xi / (xi * xi);  // 1/xi -> xi
  }
  block_sum_to(dxi, a.part + part_off + blockIdx.x, sh);
}

// Padded cell (interior, or an edge ghost along one axis) gathers the face
// contributions of the faces f - 1/2, f in [c-1, c+2], along each axis.
template <int NV>
__global__ void __launch_bounds__(128) adj_gather_kernel(AdjArgs a) {
  constexpr int ND = NV - 2;
  const Geom& g = a.g;
  const int ex = g.n[0] + 4, ey = ND >= 2 ? g.n[1] + 4 : 1, ez = ND >= 3 ? g.n[2] + 4 : 1;
  const int64_t total = (int64_t)ex * ey * ez;
  const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (id >= total) return;
  const int c[3] = {(int)(id % ex) - 2, ND >= 2 ? (int)((id / ex) % ey) - 2 : 0,
                    ND >= 3 ? (int)(id / ((int64_t)ex * ey)) - 2 : 0};
  int outside = 0, oaxis = -1;
  for (int d = 0; d < ND; ++d)
    if (c[d] < 0 || c[d] >= g.n[d]) { ++outside; oaxis = d; }
  if (outside > 1) return;  // corner ghosts take part in nothing
  double acc[NV];
  for (int v = 0; v < NV; ++v) acc[v] = 0.0;
  for (int d = 0; d < ND; ++d) {
    if (outside == 1 && oaxis != d) continue;  // a ghost along another axis is in no face of this axis
    int ext[3] = {g.n[0], g.n[1], g.n[2]};
    ext[d] += 1;
    for (int f = c[d] - 1; f <= c[d] + 2; ++f) {
      if (f < 0 || f > g.n[d]) continue;
      int cf[3] = {c[0], c[1], c[2]};
      cf[d] = f;
      const int64_t fid = ((int64_t)cf[2] * ext[1] + cf[1]) * ext[0] + cf[0];
      const int k = c[d] - f + 2;
      const double* G = a.faceG + (a.face_off[d] + fid) * (4 * NV) + k * NV;
      for (int v = 0; v < NV; ++v) acc[v] += G[v];
    }
  }
  const int64_t o = pidx_c(g, c);
  if (outside == 0) {
    for (int v = 0; v < NV; ++v) a.lam[v * g.fstride + o] += acc[v];
  } else {
    for (int v = 0; v < NV; ++v) a.lam[v * g.fstride + o] = acc[v];
  }
}

// Ghost adjoints back to their images: interior cell c within two cells of a
// boundary adds every ghost that was copied from it.
template <int NV>
__global__ void __launch_bounds__(128) adj_fold_kernel(double* lam, Geom g, Phys p) {
  constexpr int ND = NV - 2;
  const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (id >= g.ncells) return;
  const int c[3] = {(int)(id % g.n[0]), (int)((id / g.n[0]) % g.n[1]), (int)(id / ((int64_t)g.n[0] * g.n[1]))};
  const int64_t o = pidx_c(g, c);
  double add[NV];
  for (int v = 0; v < NV; ++v) add[v] = 0.0;
  for (int d = 0; d < ND; ++d) {
    const int n = g.n[d], cd = c[d];
    for (int side = 0; side < 2; ++side) {
      if (side == 0 ? !(cd < 2) : !(cd >= n - 2)) continue;
      const bool per = p.bc[d] == RSST_BC_PERIODIC;
      const int gp = per ? (side == 0 ? cd + n : cd - n) : (side == 0 ? -1 - cd : 2 * n - 1 - cd);
      int cg[3] = {c[0], c[1], c[2]};
      cg[d] = gp;
      const int64_t og = pidx_c(g, cg);
      for (int v = 0; v < NV; ++v) {
        const double x = lam[v * g.fstride + og];
        add[v] += (!per && v == 1 + d) ? -x : x;
      }
    }
  }
  for (int v = 0; v < NV; ++v) lam[v * g.fstride + o] += add[v];
}

// out = alpha * x + beta * y over interior cells (padded arrays); ghosts of out set to 0.
__global__ void axpby_kernel(double* out, const double* x, double alpha, const double* y, double beta, Geom g, int nv) {
  const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (id >= g.ncells) return;
  const int c[3] = {(int)(id % g.n[0]), (int)((id / g.n[0]) % g.n[1]), (int)(id / ((int64_t)g.n[0] * g.n[1]))};
  const int64_t o = pidx_c(g, c);
  for (int v = 0; v < nv; ++v) {
    const double xv = x ? x[v * g.fstride + o] : 0.0;
    const double yv = y ? y[v * g.fstride + o] : 0.0;
    out[v * g.fstride + o] = alpha * xv + beta * yv;
  }
}

// caller layout <-> padded interior
__global__ void to_padded_kernel(const double* src, double* dst, Geom g, int nv) {
  const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (id >= g.ncells) return;
  const int c[3] = {(int)(id % g.n[0]), (int)((id / g.n[0]) % g.n[1]), (int)(id / ((int64_t)g.n[0] * g.n[1]))};
  const int64_t o = pidx_c(g, c);
  for (int v = 0; v < nv; ++v) dst[v * g.fstride + o] = src[v * g.ncells + id];
}
__global__ void from_padded_kernel(const double* src, double* dst, Geom g, int nv) {
  const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (id >= g.ncells) return;
  const int c[3] = {(int)(id % g.n[0]), (int)((id / g.n[0]) % g.n[1]), (int)(id / ((int64_t)g.n[0] * g.n[1]))};
  const int64_t o = pidx_c(g, c);
  for (int v = 0; v < nv; ++v) dst[v * g.ncells + id] = src[v * g.fstride + o];
}

// Kinetic energy J = sum |m|^2/(2 rho) dV and dJ/dU = (-|V|^2/2, V, 0) dV.
template <int NV>
__global__ void __launch_bounds__(128) ke_kernel(const double* U, Geom g, double vol, double* part, double* grad) {
  constexpr int ND = NV - 2;
  __shared__ double sh[128];
  const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double J = 0.0;
  if (id < g.ncells) {
    const int c[3] = {(int)(id % g.n[0]), (int)((id / g.n[0]) % g.n[1]), (int)(id / ((int64_t)g.n[0] * g.n[1]))};
    const int64_t o = pidx_c(g, c);
    const double rho = U[o];
    double m2 = 0.0, v2 = 0.0;
    for (int e = 0; e < ND; ++e) {
      const double m = U[(1 + e) * g.fstride + o];
      m2 += m * m;
      v2 += (m / rho) * (m / rho);
      if (grad) grad[(1 + e) * g.ncells + id] = m / rho * vol;
    }
    J = 0.5 * m2 / rho * vol;
    if (grad) {
      grad[id] = -0.5 * v2 * vol;
      grad[(NV - 1) * g.ncells + id] = 0.0;
    }
  }
  block_sum_to(J, part + blockIdx.x, sh);
}

__global__ void sum_parts_kernel(const double* part, int n, double* out, int accumulate) {
  __shared__ double sh[256];
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += 256) acc += part[i];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = accumulate ? *out + sh[0] : sh[0];
}

}  // namespace rsst

using namespace rsst;

// ---------------------------------------------------------------------------
// Host orchestration
// ---------------------------------------------------------------------------

struct AdjState {
  double dt = 0.0;
  int nsteps = 0, every = 0, nseg = 0;
  std::vector<double*> ckpt;   // padded states at steps 0, every, 2 every, ...
  double* stages = nullptr;    // recompute storage: 2 * every padded states
  double* dUs = nullptr;       // their Euler tendencies (same layout)
  double* save = nullptr;      // the live state while a segment is recomputed
  double* lamA = nullptr;      // padded work arrays
  double* lamB = nullptr;
  double* lamC = nullptr;
  double* nu = nullptr;
  double* faceG = nullptr;
  double* part = nullptr;
  double* dxi = nullptr;       // device accumulator
  int64_t face_off[4] = {0, 0, 0, 0};
  int part_len = 0;
};

static AdjState* adj_of(rsst_handle* h) { return reinterpret_cast<AdjState*>(h->adj); }

void rsst_adjoint_free(rsst_handle* h) {
  AdjState* s = adj_of(h);
  if (!s) return;
  for (double* c : s->ckpt) cudaFree(c);
  cudaFree(s->stages);
  cudaFree(s->dUs);
  cudaFree(s->save);
  cudaFree(s->lamA);
  cudaFree(s->lamB);
  cudaFree(s->lamC);
  cudaFree(s->nu);
  cudaFree(s->faceG);
  cudaFree(s->part);
  cudaFree(s->dxi);
  delete s;
  h->adj = nullptr;
}

static size_t state_bytes(const rsst_handle* h) { return (size_t)(h->g.ndim + 2) * h->g.fstride * sizeof(double); }

static int blocks_for(int64_t n) { return (int)((n + 127) / 128); }

static int launch_err(const char* what) {
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    rsst_set_error("%s: %s", what, cudaGetErrorString(e));
    return RSST_ECUDA;
  }
  return RSST_OK;
}

extern "C" int rsst_adjoint_record(rsst_handle* h, double dt, int nsteps, int every) {
  if (!h || !(dt > 0.0) || !std::isfinite(dt) || nsteps < 1 || every < 1) {
    rsst_set_error("rsst_adjoint_record: need a handle, finite dt > 0, nsteps >= 1, every >= 1");
    return RSST_EINVAL;
  }
  if (h->cfg.precision != RSST_FP64) {
    rsst_set_error("rsst_adjoint_record: the adjoint is float64 only");
    return RSST_EUNSUPPORTED;
  }
  if (h->cfg.covolume != 0.0) {
    rsst_set_error("rsst_adjoint_record: the adjoint is derived for the ideal gas only");
    return RSST_EUNSUPPORTED;
  }
  rsst_adjoint_free(h);
  AdjState* s = new AdjState();
  h->adj = s;
  s->dt = dt;
  s->nsteps = nsteps;
  s->every = every;
  s->nseg = (nsteps + every - 1) / every;
  const size_t sb = state_bytes(h);
  const Geom& g = h->g;
  int64_t faces = 0;
  for (int d = 0; d < g.ndim; ++d) {
    s->face_off[d] = faces;
    faces += g.ncells / g.n[d] * (g.n[d] + 1);
  }
  s->part_len = blocks_for(g.ncells) + 3 * blocks_for(faces) + 8;
  const int nv = g.ndim + 2;
  bool ok = cudaMalloc((void**)&s->stages, 2 * (size_t)every * sb) == cudaSuccess &&
            cudaMalloc((void**)&s->dUs, 2 * (size_t)every * sb) == cudaSuccess &&
            cudaMalloc((void**)&s->save, sb) == cudaSuccess &&
            cudaMalloc((void**)&s->lamA, sb) == cudaSuccess && cudaMalloc((void**)&s->lamB, sb) == cudaSuccess &&
            cudaMalloc((void**)&s->lamC, sb) == cudaSuccess &&
            cudaMalloc((void**)&s->nu, sb) == cudaSuccess &&
            cudaMalloc((void**)&s->faceG, (size_t)faces * 4 * nv * sizeof(double)) == cudaSuccess &&
            cudaMalloc((void**)&s->part, (size_t)s->part_len * sizeof(double)) == cudaSuccess &&
            cudaMalloc((void**)&s->dxi, sizeof(double)) == cudaSuccess;
  for (int k = 0; ok && k < s->nseg; ++k) {
    double* c = nullptr;
    ok = cudaMalloc((void**)&c, sb) == cudaSuccess;
    s->ckpt.push_back(c);
  }
  if (!ok) {
    cudaGetLastError();
    rsst_adjoint_free(h);
    rsst_set_error("rsst_adjoint_record: device allocation failed");
    return RSST_ENOMEM;
  }
  for (int step = 0; step < nsteps; ++step) {
    if (step % every == 0) {
      if (cudaMemcpyAsync(s->ckpt[step / every], h->buf[0], sb, cudaMemcpyDeviceToDevice, h->stream) != cudaSuccess) {
        rsst_set_error("rsst_adjoint_record: checkpoint copy failed");
        return RSST_ECUDA;
      }
    }
    const int rc = rsst_handle_steps(h, dt, 1);
    if (rc != RSST_OK) return rc;
  }
  return RSST_OK;
}

extern "C" int rsst_adjoint_segments(rsst_handle* h, int32_t* nseg) {
  if (!h || !nseg || !adj_of(h)) { rsst_set_error("rsst_adjoint_segments: no recorded run"); return RSST_EINVAL; }
  *nseg = adj_of(h)->nseg;
  return RSST_OK;
}

// lam_out (padded, interior) -> its contribution through one stage.
// in: the stage input state; b: coefficient of (in + dt L(in)).
// Writes lam_in = b lam_out + (b dt lam_out)^T dL/d(in) into `res` (padded,
// interior, ghosts folded) and adds the xi partials to s->dxi.
static int stage_vjp(rsst_handle* h, AdjState* s, const double* in, const double* dU, const double* lam_out, double b,
                     double* res) {
  // No clearing is needed: the cell kernel writes nu and res at every
  // interior cell, the face kernels read nu at interior cells only, and the
  // gather writes every edge ghost of res that the fold reads.
  const Geom& g = h->g;
  const int nv = g.ndim + 2;
  cudaStream_t st = h->stream;
  AdjArgs a;
  memset(&a, 0, sizeof a);
  a.U = in;
  a.dU = dU;
  a.lam_out = lam_out;
  a.mu_scale = b * s->dt;
  a.id_scale = b;
  a.nu = s->nu;
  a.lam = res;
  a.faceG = s->faceG;
  a.part = s->part;
  a.g = g;
  a.p = h->p;
  for (int d = 0; d < 3; ++d) a.face_off[d] = s->face_off[d];
  const int cb = blocks_for(g.ncells);
  switch (nv) {
    case 3: adj_cell_kernel<3><<<cb, 128, 0, st>>>(a); break;
    case 4: adj_cell_kernel<4><<<cb, 128, 0, st>>>(a); break;
    default: adj_cell_kernel<5><<<cb, 128, 0, st>>>(a); break;
  }
  int rc = launch_err("adjoint cell kernel");
  if (rc) return rc;
  int off = cb;
  for (int d = 0; d < g.ndim; ++d) {
    const int64_t nf = g.ncells / g.n[d] * (g.n[d] + 1);
    const int fb = blocks_for(nf);
#define FK(NVv, Dd) adj_face_kernel<NVv, Dd><<<fb, 128, 0, st>>>(a, off)
    if (nv == 3) FK(3, 0);
    else if (nv == 4) { if (d == 0) FK(4, 0); else FK(4, 1); }
    else { if (d == 0) FK(5, 0); else if (d == 1) FK(5, 1); else FK(5, 2); }
#undef FK
    rc = launch_err("adjoint face kernel");
    if (rc) return rc;
    off += fb;
  }
  sum_parts_kernel<<<1, 256, 0, st>>>(s->part, off, s->dxi, 1);
  const int64_t padded = (int64_t)(g.n[0] + 4) * (g.ndim >= 2 ? g.n[1] + 4 : 1) * (g.ndim >= 3 ? g.n[2] + 4 : 1);
  switch (nv) {
    case 3: adj_gather_kernel<3><<<blocks_for(padded), 128, 0, st>>>(a); adj_fold_kernel<3><<<cb, 128, 0, st>>>(res, g, h->p); break;
    case 4: adj_gather_kernel<4><<<blocks_for(padded), 128, 0, st>>>(a); adj_fold_kernel<4><<<cb, 128, 0, st>>>(res, g, h->p); break;
    default: adj_gather_kernel<5><<<blocks_for(padded), 128, 0, st>>>(a); adj_fold_kernel<5><<<cb, 128, 0, st>>>(res, g, h->p); break;
  }
  h->launches += 4 + g.ndim;
  return launch_err("adjoint gather/fold");
}

extern "C" int rsst_adjoint_step(rsst_handle* h, int32_t seg, double* lam, double* dJ_dxi) {
  AdjState* s = h ? adj_of(h) : nullptr;
  if (!s || !lam || !dJ_dxi || seg < 0 || seg >= s->nseg) {
    rsst_set_error("rsst_adjoint_step: bad arguments or no recorded run");
    return RSST_EINVAL;
  }
  if (rsst_check_buffer(lam, 0, "rsst_adjoint_step (lam)") != RSST_OK) return RSST_EINVAL;
  const Geom& g = h->g;
  const int nv = g.ndim + 2;
  const size_t sb = state_bytes(h);
  cudaStream_t st = h->stream;
  const int s0 = seg * s->every;
  const int k = (s0 + s->every <= s->nsteps) ? s->every : s->nsteps - s0;
  const int64_t fe = g.fstride * (int64_t)nv;
  // recompute the segment: stages[2i] = U^{s0+i}, stages[2i+1] = U*; the
  // live state and scalars are saved and put back afterwards
  cudaError_t ce = cudaSuccess;
  auto chk = [&](cudaError_t e) { if (ce == cudaSuccess && e != cudaSuccess) ce = e; };
  int rc = RSST_OK;
  const int slot0 = h->slot;
  double save_scal[16];
  chk(cudaMemcpyAsync(h->h_small, h->d_scal, 16 * sizeof(double), cudaMemcpyDeviceToHost, st));
  chk(cudaStreamSynchronize(st));
  memcpy(save_scal, h->h_small, sizeof save_scal);
  chk(cudaMemcpyAsync(s->save, h->buf[0], sb, cudaMemcpyDeviceToDevice, st));
  chk(cudaMemcpyAsync(h->buf[0], s->ckpt[seg], sb, cudaMemcpyDeviceToDevice, st));
  for (int i = 0; i < k && rc == RSST_OK && ce == cudaSuccess; ++i) {
    chk(cudaMemcpyAsync(s->stages + (2 * i) * fe, h->buf[0], sb, cudaMemcpyDeviceToDevice, st));
    h->rec_dU[0] = s->dUs + (2 * i) * fe;      // the forward kernels also write each stage's Euler tendency
    h->rec_dU[1] = s->dUs + (2 * i + 1) * fe;
    rc = rsst_handle_steps(h, s->dt, 1);
    h->rec_dU[0] = h->rec_dU[1] = nullptr;
    // buf[1] still holds U* of this step
    chk(cudaMemcpyAsync(s->stages + (2 * i + 1) * fe, h->buf[1], sb, cudaMemcpyDeviceToDevice, st));
  }
  chk(cudaMemcpyAsync(h->buf[0], s->save, sb, cudaMemcpyDeviceToDevice, st));
  memcpy(h->h_small, save_scal, sizeof save_scal);
  chk(cudaMemcpyAsync(h->d_scal, h->h_small, 16 * sizeof(double), cudaMemcpyHostToDevice, st));
  chk(cudaStreamSynchronize(st));
  if (rc == RSST_OK && ce != cudaSuccess) {
    rsst_set_error("rsst_adjoint_step: segment recompute: %s", cudaGetErrorString(ce));
    rc = RSST_ECUDA;
  }
  h->slot = slot0;
  if (rc == RSST_OK) {
    if (cudaMemsetAsync(s->dxi, 0, sizeof(double), st) != cudaSuccess ||
        cudaMemsetAsync(s->lamA, 0, sb, st) != cudaSuccess) {
      rsst_set_error("rsst_adjoint_step: clearing the work arrays failed");
      return RSST_ECUDA;
    }
    to_padded_kernel<<<blocks_for(g.ncells), 128, 0, st>>>(lam, s->lamA, g, nv);
    for (int i = k - 1; i >= 0 && rc == RSST_OK; --i) {
      const double* Un = s->stages + (2 * i) * fe;
      const double* Us = s->stages + (2 * i + 1) * fe;
      // stage 2: U^{n+1} = 1/2 U^n + 1/2 (U* + dt L(U*)):  lamB = lambda_*
      rc = stage_vjp(h, s, Us, s->dUs + (2 * i + 1) * fe, s->lamA, 0.5, s->lamB);
      if (rc) break;
      // stage 1: U* = U^n + dt L(U^n):  lamC = lambda_* dU*/dU^n
      rc = stage_vjp(h, s, Un, s->dUs + (2 * i) * fe, s->lamB, 1.0, s->lamC);
      if (rc) break;
      // lambda^n = 1/2 lambda^{n+1} + lamC
      axpby_kernel<<<blocks_for(g.ncells), 128, 0, st>>>(s->lamA, s->lamA, 0.5, s->lamC, 1.0, g, nv);
    }
    from_padded_kernel<<<blocks_for(g.ncells), 128, 0, st>>>(s->lamA, lam, g, nv);
    rc = rc ? rc : launch_err("adjoint transfer");
  }
  double dx = 0.0;
  if (rc == RSST_OK) {
    if (cudaMemcpyAsync(h->h_small, s->dxi, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      rsst_set_error("rsst_adjoint_step: read-back failed");
      rc = RSST_ECUDA;
    } else {
      dx = h->h_small[0];
    }
  } else {
    cudaStreamSynchronize(st);
  }
  if (rc == RSST_OK) *dJ_dxi += dx;
  return rc;
}

extern "C" int rsst_kinetic_energy(rsst_handle* h, double* J, double* grad) {
  if (!h || !J) { rsst_set_error("rsst_kinetic_energy: NULL argument"); return RSST_EINVAL; }
  if (grad && rsst_check_buffer(grad, 0, "rsst_kinetic_energy (grad)") != RSST_OK) return RSST_EINVAL;
  if (h->cfg.precision != RSST_FP64) { rsst_set_error("rsst_kinetic_energy: float64 runs only"); return RSST_EUNSUPPORTED; }
  const Geom& g = h->g;
  const int nb = blocks_for(g.ncells);
  if (nb > 1024 * 64) { rsst_set_error("rsst_kinetic_energy: grid too large"); return RSST_EINVAL; }
  double* part = nullptr;
  if (cudaMalloc((void**)&part, (nb + 1) * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    rsst_set_error("rsst_kinetic_energy: allocation failed");
    return RSST_ENOMEM;
  }
  double vol = 1.0;
  for (int d = 0; d < g.ndim; ++d) vol *= h->cfg.dx[d];
  switch (g.ndim + 2) {
    case 3: ke_kernel<3><<<nb, 128, 0, h->stream>>>((const double*)h->buf[0], g, vol, part, grad); break;
    case 4: ke_kernel<4><<<nb, 128, 0, h->stream>>>((const double*)h->buf[0], g, vol, part, grad); break;
    default: ke_kernel<5><<<nb, 128, 0, h->stream>>>((const double*)h->buf[0], g, vol, part, grad); break;
  }
  sum_parts_kernel<<<1, 256, 0, h->stream>>>(part, nb, part + nb, 0);
  int rc = launch_err("kinetic energy");
  if (rc == RSST_OK) {
    if (cudaMemcpyAsync(h->h_small, part + nb, sizeof(double), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
        cudaStreamSynchronize(h->stream) != cudaSuccess) {
      rsst_set_error("rsst_kinetic_energy: read-back failed");
      rc = RSST_ECUDA;
    } else {
      *J = h->h_small[0];
    }
  }
  cudaFree(part);
  h->launches += 2;
  return rc;
}

namespace rsst {

// dJ/drho at fixed V and P from dJ/dU (ideal gas, (de/drho)_P = 0):
// lam_rho + V . lam_m + |V|^2/2 lam_E, cell by cell; caller layout, planes of
// `cells` values.
template <int NV>
__global__ void rho_fixed_vp_kernel(const double* __restrict__ U, const double* __restrict__ lam,
                                    double* __restrict__ out, int64_t cells) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < cells; i += (int64_t)gridDim.x * blockDim.x) {
    const double rho = U[i];
    double acc = lam[i], v2 = 0.0;
#pragma unroll
    for (int d = 0; d < NV - 2; ++d) {
      const double v = U[(1 + d) * cells + i] / rho;
      acc = fma(v, lam[(1 + d) * cells + i], acc);
      v2 = fma(v, v, v2);
    }
    out[i] = fma(0.5 * v2, lam[(NV - 1) * cells + i], acc);
  }
}

}  // namespace rsst

extern "C" int rsst_adjoint_rho_fixed_vp(const double* U, const double* lam, double* out, int32_t ndim,
                                         const int32_t* n, void* stream) {
  if (!U || !lam || !out || !n || ndim < 1 || ndim > 3) {
    rsst_set_error("rsst_adjoint_rho_fixed_vp: NULL pointer or ndim outside 1..3");
    return RSST_EINVAL;
  }
  int64_t cells = 1;
  for (int d = 0; d < ndim; ++d) {
    if (n[d] < 1) { rsst_set_error("rsst_adjoint_rho_fixed_vp: n[%d] < 1", d); return RSST_EINVAL; }
    cells *= n[d];
  }
  if (cells > (int64_t)1 << 31) { rsst_set_error("rsst_adjoint_rho_fixed_vp: grid too large"); return RSST_EINVAL; }
  if (rsst_check_buffer(U, 0, "rsst_adjoint_rho_fixed_vp (U)") != RSST_OK ||
      rsst_check_buffer(lam, 0, "rsst_adjoint_rho_fixed_vp (lam)") != RSST_OK ||
      rsst_check_buffer(out, 0, "rsst_adjoint_rho_fixed_vp (out)") != RSST_OK)
    return RSST_EINVAL;
  const int64_t want = (cells + 255) / 256;
  const int grid = (int)(want < 152 * 8 ? want : 152 * 8);
  cudaStream_t st = (cudaStream_t)stream;
  switch (ndim) {
    case 1: rsst::rho_fixed_vp_kernel<3><<<grid, 256, 0, st>>>(U, lam, out, cells); break;
    case 2: rsst::rho_fixed_vp_kernel<4><<<grid, 256, 0, st>>>(U, lam, out, cells); break;
    default: rsst::rho_fixed_vp_kernel<5><<<grid, 256, 0, st>>>(U, lam, out, cells); break;
  }
  return launch_err("rsst_adjoint_rho_fixed_vp");
}
