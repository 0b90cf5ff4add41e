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
//   adj_cell: per interior cell, recompute the Euler tendency dU from the
//     2 * ndim face fluxes around it, then nu = mu^T dC/d(dU) and the
//     pointwise part mu^T d(C + force)/dq (C = reduced tendency, Sec. 3.2 /
//     App. A; force of App. B), and the xi partial;
//   adj_face: per face, phi = (nu_right - nu_left)/dx, then phi^T dF/dU_k for
//     the four stencil cells k of the face (MC slopes, face states, LLF flux
//     of Sec. 4.2) and the xi partial;
//   adj_gather: each padded cell (interior and edge ghosts) sums the
//     contributions of the faces whose stencil holds it;
//   adj_fold: ghost-cell adjoints go back to the cells they were copied from
//     (wrap, or mirror with the normal momentum negated).
// The derivatives are taken with a forward-mode dual number run once per
// input component over templated copies of the step's arithmetic.
#include <cstring>
#include <vector>

#include "rsst_common.cuh"
#include "rsst_internal.h"

namespace rsst {

struct Dual {
  double v, d;
};
__device__ __forceinline__ Dual mk(double v, double d = 0.0) { return {v, d}; }
__device__ __forceinline__ Dual operator+(Dual a, Dual b) { return {a.v + b.v, a.d + b.d}; }
__device__ __forceinline__ Dual operator-(Dual a, Dual b) { return {a.v - b.v, a.d - b.d}; }
__device__ __forceinline__ Dual operator-(Dual a) { return {-a.v, -a.d}; }
__device__ __forceinline__ Dual operator+(Dual a, double b) { return {a.v + b, a.d}; }
__device__ __forceinline__ Dual operator+(double a, Dual b) { return {a + b.v, b.d}; }
__device__ __forceinline__ Dual operator-(Dual a, double b) { return {a.v - b, a.d}; }
__device__ __forceinline__ Dual operator-(double a, Dual b) { return {a - b.v, -b.d}; }
__device__ __forceinline__ Dual operator*(Dual a, Dual b) { return {a.v * b.v, a.d * b.v + a.v * b.d}; }
__device__ __forceinline__ Dual operator*(double a, Dual b) { return {a * b.v, a * b.d}; }
__device__ __forceinline__ Dual operator*(Dual a, double b) { return {a.v * b, a.d * b}; }
__device__ __forceinline__ Dual operator/(Dual a, Dual b) {
  const double q = a.v / b.v;
  return {q, (a.d - q * b.d) / b.v};
}
__device__ __forceinline__ Dual operator/(double a, Dual b) {
  const double q = a / b.v;
  return {q, -q * b.d / b.v};
}
__device__ __forceinline__ Dual dsqrt(Dual a) {
  const double s = sqrt(a.v);
  return {s, a.v > 0.0 ? a.d / (2.0 * s) : 0.0};
}
__device__ __forceinline__ double val(double a) { return a; }
__device__ __forceinline__ double val(Dual a) { return a.v; }
__device__ __forceinline__ double dsqrt(double a) { return sqrt(a); }

// |V| with a zero subgradient at V = 0.
template <class T>
__device__ __forceinline__ T speed_T(T v2) {
  if (val(v2) > 0.0) return dsqrt(v2);
  return v2 * 0.0;
}

template <class T>
__device__ __forceinline__ T mc_T(T a, T b) {
  const double av = val(a), bv = val(b);
  if (!(av * bv > 0.0)) return a * 0.0;
  const double aa = 2.0 * fabs(av), bb = 2.0 * fabs(bv), cc = 0.5 * fabs(av + bv);
  if (aa <= bb && aa <= cc) return 2.0 * a;
  if (bb <= cc) return 2.0 * b;
  return 0.5 * (a + b);
}

template <class T, int NV, int D>
__device__ __forceinline__ void euler_flux_T(const T (&q)[NV], const Phys& p, T inv_xi, T (&F)[NV], T& c) {
  constexpr int ND = NV - 2;
  const T rho = q[0];
  T v[ND];
  T v2 = q[0] * 0.0;
  for (int e = 0; e < ND; ++e) {
    v[e] = q[1 + e] / rho;
    v2 = v2 + v[e] * v[e];
  }
  const T P = p.gm1 * (q[NV - 1] - 0.5 * (rho * v2));
  const T a2 = p.gamma * P / rho;
  if (p.use_cmax)  // C_max law (Eq. cx): a/xi = sqrt(a^2 / sqrt(1 + a^4/C^4))
    c = speed_T(v2) + dsqrt(a2 / dsqrt(1.0 + (a2 * a2) * p.inv_cmax4));
  else
    c = speed_T(v2) + dsqrt(a2) * inv_xi;
  F[0] = q[1 + D];
  for (int e = 0; e < ND; ++e) F[1 + e] = (e == D) ? q[1 + e] * v[D] + P : q[1 + e] * v[D];
  F[NV - 1] = (q[NV - 1] + P) * v[D];
}

// LLF flux of the face between cells u0 | u1 from the stencil (um, u0 | u1, up).
template <class T, int NV, int D>
__device__ __forceinline__ void face_T(const T (&um)[NV], const T (&u0)[NV], const T (&u1)[NV], const T (&up)[NV],
                                       const Phys& p, T inv_xi, T (&F)[NV]) {
  T qL[NV], qR[NV], FL[NV], FR[NV], cL, cR;
  for (int v = 0; v < NV; ++v) {
    qL[v] = u0[v] + 0.5 * mc_T(u0[v] - um[v], u1[v] - u0[v]);
    qR[v] = u1[v] - 0.5 * mc_T(u1[v] - u0[v], up[v] - u1[v]);
  }
  euler_flux_T<T, NV, D>(qL, p, inv_xi, FL, cL);
  euler_flux_T<T, NV, D>(qR, p, inv_xi, FR, cR);
  const T alpha = val(cL) >= val(cR) ? cL : cR;
  for (int v = 0; v < NV; ++v) F[v] = 0.5 * (FL[v] + FR[v]) - 0.5 * (alpha * (qR[v] - qL[v]));
}

// Reduced tendency plus force at one cell: L = dU - f s r + (0, rho F, m.F).
template <class T, int NV>
__device__ __forceinline__ void rhs_T(const T (&q)[NV], const T (&dU)[NV], T f, const Phys& p, T (&L)[NV]) {
  constexpr int ND = NV - 2;
  for (int v = 0; v < NV; ++v) L[v] = dU[v];
  const T rho = q[0];
  if (p.variant != RSST_EULER) {
    T v[ND];
    T v2 = q[0] * 0.0, vdm = q[0] * 0.0;
    for (int e = 0; e < ND; ++e) {
      v[e] = q[1 + e] / rho;
      v2 = v2 + v[e] * v[e];
      vdm = vdm + v[e] * dU[1 + e];
    }
    const T P = p.gm1 * (q[NV - 1] - 0.5 * (rho * v2));
    const T e_int = P * p.inv_gm1;
    const T kin = 0.5 * (rho * v2);
    const int var = p.variant;
    T s, r0, rE;
    T rv = q[0] * 0.0;
    bool has_rv = false;
    if (var == RSST_PVS || var == RSST_PMS || var == RSST_PD) {
      s = p.gm1 * (0.5 * (v2 * dU[0]) - vdm + dU[NV - 1]);
      if (var == RSST_PD) {
        r0 = q[0] * 0.0;
        rE = q[0] * 0.0 + p.inv_gm1;
      } else {
        const T ia2 = rho / (p.gamma * P);
        r0 = ia2;
        if (var == RSST_PVS) { rv = ia2; has_rv = true; }
        rE = (var == RSST_PVS ? (e_int + P + kin) : (e_int + P - kin)) * ia2 / rho;
      }
    } else {
      s = dU[0];
      r0 = q[0] * 0.0 + 1.0;
      if (var == RSST_DVS) { rv = q[0] * 0.0 + 1.0; has_rv = true; }
      rE = (var == RSST_DVS ? (e_int + P + kin) : (e_int + P - kin)) / rho;
    }
    // f = 1 - 1/xi^2: constant, or from the cell's a^2 under the C_max law
    const T fc = p.use_cmax ? 1.0 - 1.0 / dsqrt(1.0 + ((p.gamma * P / rho) * (p.gamma * P / rho)) * p.inv_cmax4) : f;
    const T fs = fc * s;
    L[0] = L[0] - fs * r0;
    if (has_rv)
      for (int e = 0; e < ND; ++e) L[1 + e] = L[1 + e] - fs * (rv * v[e]);
    L[NV - 1] = L[NV - 1] - fs * rE;
  }
  if (p.has_grav) {
    T mg = q[0] * 0.0;
    for (int e = 0; e < ND; ++e) {
      L[1 + e] = L[1 + e] + rho * p.grav[e];
      mg = mg + q[1 + e] * p.grav[e];
    }
    L[NV - 1] = L[NV - 1] + mg;
  }
}

struct AdjArgs {
  const double* U;   // stage input, padded
  const double* mu;  // b dt lambda_out, padded (interior used)
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
  constexpr int ND = NV - 2;
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
      mu[v] = a.mu[v * g.fstride + o];
      dU[v] = 0.0;
    }
    // Euler tendency from the 2 * ndim faces
    for (int d = 0; d < ND; ++d) {
      for (int side = 0; side < 2; ++side) {
        int cf[3] = {c[0], c[1], c[2]};
        cf[d] += side;  // face cf[d] - 1/2
        double s[4][NV], F[NV];
        if (d == 0) { load_stencil<NV, 0>(a, cf, s); face_T<double, NV, 0>(s[0], s[1], s[2], s[3], p, p.inv_xi, F); }
        if (d == 1) { if constexpr (ND >= 2) { load_stencil<NV, 1>(a, cf, s); face_T<double, NV, 1>(s[0], s[1], s[2], s[3], p, p.inv_xi, F); } }
        if (d == 2) { if constexpr (ND >= 3) { load_stencil<NV, 2>(a, cf, s); face_T<double, NV, 2>(s[0], s[1], s[2], s[3], p, p.inv_xi, F); } }
        const double sg = side == 0 ? 1.0 : -1.0;
        for (int v = 0; v < NV; ++v) dU[v] += sg * F[v] * p.inv_dx[d];
      }
    }
    // nu = mu^T dL/d(dU), pointwise mu^T dL/dq, xi partial
    Dual qd[NV], dd[NV], L[NV];
    const Dual f0 = mk(p.f);
    for (int j = 0; j < NV; ++j) {
      for (int v = 0; v < NV; ++v) {
        qd[v] = mk(q[v]);
        dd[v] = mk(dU[v], v == j ? 1.0 : 0.0);
      }
      rhs_T<Dual, NV>(qd, dd, f0, p, L);
      double acc = 0.0;
      for (int v = 0; v < NV; ++v) acc += mu[v] * L[v].d;
      a.nu[j * g.fstride + o] = acc;
    }
    for (int j = 0; j < NV; ++j) {
      for (int v = 0; v < NV; ++v) {
        qd[v] = mk(q[v], v == j ? 1.0 : 0.0);
        dd[v] = mk(dU[v]);
      }
      rhs_T<Dual, NV>(qd, dd, f0, p, L);
      double acc = 0.0;
      for (int v = 0; v < NV; ++v) acc += mu[v] * L[v].d;
      a.lam[j * g.fstride + o] = acc;
    }
    for (int v = 0; v < NV; ++v) {
      qd[v] = mk(q[v]);
      dd[v] = mk(dU[v]);
    }
    const double xi = p.xi;
    rhs_T<Dual, NV>(qd, dd, mk(p.f, 2.0 / (xi * xi * xi)), p, L);  // f = 1 - 1/xi^2
    for (int v = 0; v < NV; ++v) dxi += mu[v] * L[v].d;
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
    double* G = a.faceG + (a.face_off[D] + id) * (4 * NV);
    Dual sd[4][NV], F[NV];
    const Dual ix = mk(p.inv_xi);
    for (int k = 0; k < 4; ++k) {
      for (int j = 0; j < NV; ++j) {
        for (int kk = 0; kk < 4; ++kk)
          for (int v = 0; v < NV; ++v) sd[kk][v] = mk(s[kk][v], (kk == k && v == j) ? 1.0 : 0.0);
        face_T<Dual, NV, D>(sd[0], sd[1], sd[2], sd[3], p, ix, F);
        double acc = 0.0;
        for (int v = 0; v < NV; ++v) acc += phi[v] * F[v].d;
        G[k * NV + j] = acc;
      }
    }
    for (int kk = 0; kk < 4; ++kk)
      for (int v = 0; v < NV; ++v) sd[kk][v] = mk(s[kk][v]);
    const double xi = p.xi;
    face_T<Dual, NV, D>(sd[0], sd[1], sd[2], sd[3], p, mk(p.inv_xi, -1.0 / (xi * xi)), F);
    for (int v = 0; v < NV; ++v) dxi += phi[v] * F[v].d;
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
  double* lamA = nullptr;      // padded work arrays
  double* lamB = nullptr;
  double* lamC = nullptr;
  double* mu = nullptr;
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
  cudaFree(s->lamA);
  cudaFree(s->lamB);
  cudaFree(s->lamC);
  cudaFree(s->mu);
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
  if (!h || !(dt > 0.0) || nsteps < 1 || every < 1) {
    rsst_set_error("rsst_adjoint_record: need a handle, dt > 0, nsteps >= 1, every >= 1");
    return RSST_EINVAL;
  }
  if (h->cfg.precision != RSST_FP64) {
    rsst_set_error("rsst_adjoint_record: the adjoint is float64 only");
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
            cudaMalloc((void**)&s->lamA, sb) == cudaSuccess && cudaMalloc((void**)&s->lamB, sb) == cudaSuccess &&
            cudaMalloc((void**)&s->lamC, sb) == cudaSuccess &&
            cudaMalloc((void**)&s->mu, sb) == cudaSuccess && cudaMalloc((void**)&s->nu, sb) == cudaSuccess &&
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
static int stage_vjp(rsst_handle* h, AdjState* s, const double* in, const double* lam_out, double b, double* res) {
  const Geom& g = h->g;
  const int nv = g.ndim + 2;
  cudaStream_t st = h->stream;
  const size_t sb = state_bytes(h);
  if (cudaMemsetAsync(s->nu, 0, sb, st) != cudaSuccess || cudaMemsetAsync(res, 0, sb, st) != cudaSuccess) {
    rsst_set_error("adjoint memset failed");
    return RSST_ECUDA;
  }
  axpby_kernel<<<blocks_for(g.ncells), 128, 0, st>>>(s->mu, lam_out, b * s->dt, nullptr, 0.0, g, nv);
  AdjArgs a;
  memset(&a, 0, sizeof a);
  a.U = in;
  a.mu = s->mu;
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
  rc = launch_err("adjoint gather/fold");
  if (rc) return rc;
  // res += b * lam_out (identity part of the stage)
  axpby_kernel<<<cb, 128, 0, st>>>(res, res, 1.0, lam_out, b, g, nv);
  h->launches += 6 + g.ndim;
  return launch_err("adjoint combine");
}

extern "C" int rsst_adjoint_step(rsst_handle* h, int32_t seg, double* lam, double* dJ_dxi) {
  AdjState* s = h ? adj_of(h) : nullptr;
  if (!s || !lam || !dJ_dxi || seg < 0 || seg >= s->nseg) {
    rsst_set_error("rsst_adjoint_step: bad arguments or no recorded run");
    return RSST_EINVAL;
  }
  const Geom& g = h->g;
  const int nv = g.ndim + 2;
  const size_t sb = state_bytes(h);
  cudaStream_t st = h->stream;
  const int s0 = seg * s->every;
  const int k = (s0 + s->every <= s->nsteps) ? s->every : s->nsteps - s0;
  const int64_t fe = g.fstride * (int64_t)nv;
  // recompute the segment: stages[2i] = U^{s0+i}, stages[2i+1] = U*
  double* save_state = nullptr;
  if (cudaMalloc((void**)&save_state, sb) != cudaSuccess) {
    cudaGetLastError();
    rsst_set_error("rsst_adjoint_step: allocation failed");
    return RSST_ENOMEM;
  }
  int rc = RSST_OK;
  const int slot0 = h->slot;
  double save_scal[16];
  cudaMemcpyAsync(h->h_small, h->d_scal, 16 * sizeof(double), cudaMemcpyDeviceToHost, st);
  cudaStreamSynchronize(st);
  memcpy(save_scal, h->h_small, sizeof save_scal);
  cudaMemcpyAsync(save_state, h->buf[0], sb, cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(h->buf[0], s->ckpt[seg], sb, cudaMemcpyDeviceToDevice, st);
  for (int i = 0; i < k && rc == RSST_OK; ++i) {
    cudaMemcpyAsync(s->stages + (2 * i) * fe, h->buf[0], sb, cudaMemcpyDeviceToDevice, st);
    rc = rsst_handle_steps(h, s->dt, 1);
    // buf[1] still holds U* of this step
    cudaMemcpyAsync(s->stages + (2 * i + 1) * fe, h->buf[1], sb, cudaMemcpyDeviceToDevice, st);
  }
  cudaMemcpyAsync(h->buf[0], save_state, sb, cudaMemcpyDeviceToDevice, st);
  memcpy(h->h_small, save_scal, sizeof save_scal);
  cudaMemcpyAsync(h->d_scal, h->h_small, 16 * sizeof(double), cudaMemcpyHostToDevice, st);
  cudaStreamSynchronize(st);
  h->slot = slot0;
  if (rc == RSST_OK) {
    cudaMemsetAsync(s->dxi, 0, sizeof(double), st);
    cudaMemsetAsync(s->lamA, 0, sb, st);
    to_padded_kernel<<<blocks_for(g.ncells), 128, 0, st>>>(lam, s->lamA, g, nv);
    for (int i = k - 1; i >= 0 && rc == RSST_OK; --i) {
      const double* Un = s->stages + (2 * i) * fe;
      const double* Us = s->stages + (2 * i + 1) * fe;
      // stage 2: U^{n+1} = 1/2 U^n + 1/2 (U* + dt L(U*)):  lamB = lambda_*
      rc = stage_vjp(h, s, Us, s->lamA, 0.5, s->lamB);
      if (rc) break;
      // stage 1: U* = U^n + dt L(U^n):  lamC = lambda_* dU*/dU^n
      rc = stage_vjp(h, s, Un, s->lamB, 1.0, s->lamC);
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
  cudaFree(save_state);
  if (rc == RSST_OK) *dJ_dxi += dx;
  return rc;
}

extern "C" int rsst_kinetic_energy(rsst_handle* h, double* J, double* grad) {
  if (!h || !J) { rsst_set_error("rsst_kinetic_energy: NULL argument"); return RSST_EINVAL; }
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
