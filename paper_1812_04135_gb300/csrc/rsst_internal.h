// Internal types shared by the librsst translation units (host and device).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "rsst.h"

#define RSST_G 2  // ghost layers per end of an active axis (MUSCL needs i-2..i+2)
#define RSST_DEFAULT_GRAPH_STEPS 16  // steps per replayed CUDA graph (even)
// 1D lines up to this length use 16-cell tiles (one warp each, one face per
// thread), so that a short line runs on many SMs instead of one CTA on one SM
#define RSST_SMALL_1D (32 * 152 * 4)

// Bits of a run's device flag (sticky until the next rsst_set_state).
#define RSST_FLAG_NONPHYSICAL 1u  // a stage produced rho <= 0, P <= 0 or a non-finite value
#define RSST_FLAG_TIMEOUT 2u      // a bounded wait on a TMA copy or barrier gave up

// Padded device layout of one run's state, per field:
//   interior cell (i, j, k) lives at  (k + gz) * plane + (j + gy) * pitch + (i + xoff)
// with two ghost cells before and after the interior on every active axis.
// xoff puts interior x = 0 on a 32-byte boundary.  Fields are fstride
// elements apart.
struct Geom {
  int ndim;
  int n[3];          // interior cells (1 on inactive axes)
  int gy, gz;        // ghost offset on y / z (2 if active, else 0)
  int xoff;          // padded x index of interior x = 0
  int py, pz;        // padded rows per plane, planes
  int64_t pitch;     // elements per padded row
  int64_t plane;     // elements per padded plane
  int64_t fstride;   // elements per field
  int64_t ncells;    // interior cells
};

// Physics and scheme constants, precomputed on the host.
struct Phys {
  double gamma, gm1, inv_gm1, hgm1;  // hgm1 = (gamma - 1)/2
  double xi, inv_xi, f;  // f = 1 - 1/xi^2
  double gamma_xi2;      // gamma / xi^2: (a/xi)^2 = gamma_xi2 P / rho for the ideal gas
  double inv_cmax4;      // 1/C_max^4 (state-dependent xi, Eq. cx), used if use_cmax
  int use_cmax;
  double cfl;
  double covol;          // covolume b of the gas (0: ideal gas)
  double grav[3];
  double inv_dx[3];
  double sum_inv_dx;     // sum_d 1/dx_d: CFL rate = c_tot * sum_inv_dx
  int variant;
  int vertical;          // background axis or -1
  int bc[3];
  int has_grav;
};

// Float32 copies of the constants used by the float32 kernels.
struct PhysF {
  float gamma, gm1, inv_gm1, inv_xi, f;
  float inv_cmax4;
  int use_cmax;
  float grav[3];
  float inv_dx[3];
  float sum_inv_dx;
  float hgm1;     // (gamma - 1)/2
  float gam_gm1;  // gamma/(gamma - 1): (e + P)/P of the ideal gas
  float gx;       // gamma/xi^2 (constant xi: gx P/rho = (a/xi)^2), gamma under the C_max law
};

// Background tables of the float32 perturbation mode: float32 rows of
// length tab_len (= padded vertical index k = interior index + 2), computed
// in float64 on the device at set-up.  Face entries at index k describe the
// face between padded cells k-1 and k.
enum BgTab {
  TB_RHO0 = 0, TB_E0, TB_P0, TB_H0,                 // cell background, H0 = E0 + P0
  TB_R0,                                             // 5 rows: background residual L(U0) incl. force
  TB_D0RHO = TB_R0 + 5, TB_D0MV, TB_D0E,             // background Euler tendency (rho, m_vert, E)
  TB_S = TB_D0E + 1,                                 // slope rows, 2 components (rho, E) x 6:
                                                     //   d0L, d0R, then lin_B(d0) - MC(d0) for B = 0, 2a, 2b, c
  TB_F = TB_S + 12,                                  // face rows:
  TB_FRHOL = TB_F, TB_FRHOR, TB_FEL, TB_FER, TB_FPL, TB_FPR, TB_FHL, TB_FHR,
  TB_FAL, TB_FAR,                                    // background sound speeds a0 left / right
  TB_FG,                                             // c0L - c0R
  TB_FALPHA,                                         // alpha0 = max(c0L, c0R)
  TB_FDRHO, TB_FDE,                                  // U0R - U0L (rho, E)
  TB_COUNT
};

// Row-major background table of the TMA float32 kernels: TR_W floats per
// padded vertical index k (16-byte aligned rows, read as float4).  Cell
// entries describe padded cell k, face entries the face between padded
// cells k-1 and k.  Values are computed in float64 and rounded once.
enum BgRow {
  TR_RHO0 = 0, TR_P0, TR_GXP0, TR_H0,   // cell: rho0, P0, gx P0, H0 = E0 + P0
  TR_R0 = 4,                            // cell: background residual L(U0) incl. force, NV entries (5 slots)
  TR_D0RHO = 9, TR_D0MV, TR_D0E,        // cell: background Euler tendency (rho, m_vertical, E)
  TR_SRHO = 12,                         // cell: slope rows of rho: d0L, d0R, then half of lin_B(d0) - MC(d0), B = 0..3
  TR_SE = 18,                           // cell: the same for E
  TR_FL = 24,                           // face, left state: rho0, P0, gx P0, H0
  TR_FR = 28,                           // face, right state: rho0, P0, gx P0, H0
  TR_FA0X = 32,                         // face: a0/xi left, right; gx/rho0 left, right
  TR_FG = 36, TR_FALPHA, TR_FJRHO, TR_FJE,  // face: c0L - c0R, alpha0, rho0R - rho0L, E0R - E0L
  TR_W = 40
};

// Arguments of one fused RK stage launch (single run).
template <typename T>
struct StageArgs {
  const T* in;      // stage input, padded (U^n in stage 1, U* in stage 2)
  const T* base;    // U^n (stage 2 only; may alias out)
  T* out;           // stage output, padded (interior and edge ghosts written)
  Geom g;
  Phys p;
  const double* bg; // background [2][pz_v]: rho0, E0 at padded vertical index, or null
  int bg_len;       // entries per background row
  double* scal;     // [0..1] CFL maximum slots, [2] dt of the current step
  unsigned int* flag;
  int slot;         // CFL slot read this step (stage 2 writes slot ^ 1)
  int stage;        // 1 or 2
  double dt_fixed;  // > 0: fixed step
  PhysF pf;         // float32 constants (float32 kernels)
  const float* tab; // background tables [TB_COUNT][tab_len] (float32 mode), or null
  int tab_len;
  const float* tabr; // row-major background table [tab_len][TR_W] (TMA float32 kernels), or null
  double* dU_out;   // float64 kernels: if set, the Euler tendency of each interior cell
                    // (padded layout) is written here too (adjoint recompute)
  int64_t stall_ns; // > 0 (failure-detection tests only): each tile of a TMA-staged kernel
                    // also waits this long on a barrier that nothing completes
};

// Host-side launchers (defined in the .cu files).
// tin: tensor map of a.in (2D/3D: the halo tile comes in by TMA), or null
// (plain loads; always for 1D).
int rsst_launch_stage_fp64(const CUtensorMap* tin, const StageArgs<double>& a, cudaStream_t s);
// Box (cells along x, y, z) of the float64 stage kernel's halo tile in 2D/3D.
void rsst_stage_fp64_box(int ndim, int* sx, int* sy, int* sz);
int rsst_launch_pack_fp64(const double* src, double* dst, const Geom& g, const Phys& p,
                          const double* bg, int bg_len, cudaStream_t s);
int rsst_launch_unpack_fp64(const double* src, double* dst, const Geom& g, cudaStream_t s);
int rsst_launch_cfl_fp64(const double* U, const Geom& g, const Phys& p, double* slot_ptr,
                         unsigned int* flag, cudaStream_t s);
int rsst_launch_sums_fp64(const double* U, const Geom& g, double* partial, double* out,
                          double scale, cudaStream_t s);

int rsst_launch_stage_fp32(const StageArgs<float>& a, cudaStream_t s);
int rsst_launch_stage_df(const StageArgs<float2>& a, cudaStream_t s);
int rsst_launch_pack_df(const double* src, float2* dst, const Geom& g, const Phys& p, const double* bg, int bg_len,
                        cudaStream_t s);
int rsst_launch_unpack_df(const float2* src, double* dst, const Geom& g, cudaStream_t s);
int rsst_launch_cfl_df(const float2* U, const Geom& g, const Phys& p, double* slot_ptr, unsigned int* flag,
                       cudaStream_t s);
int rsst_launch_sums_df(const float2* U, const Geom& g, double* partial, double* out, double scale_, cudaStream_t s);
int rsst_launch_stage2d_tma(const CUtensorMap* tin, const StageArgs<float>& a, cudaStream_t s);
int rsst_launch_stage3d_tma(const CUtensorMap* tin, const StageArgs<float>& a, cudaStream_t s);
int rsst_launch_bgtab(const double* bg, int bg_len, const Geom& g, const Phys& p, float* tab, float* tabr,
                      cudaStream_t s);
int rsst_launch_pack_fp32(const double* src, float* dst, const Geom& g, const Phys& p, const double* bg,
                          int bg_len, cudaStream_t s);
int rsst_launch_unpack_fp32(const float* src, double* dst, const Geom& g, const Phys& p, const double* bg,
                            int bg_len, cudaStream_t s);
int rsst_launch_cfl_fp32(const float* U, const Geom& g, const Phys& p, const PhysF& pf, const float* tab,
                         int tab_len, double* slot_ptr, unsigned int* flag, cudaStream_t s);
int rsst_launch_sums_fp32(const float* U, const Geom& g, const Phys& p, const double* bg, int bg_len,
                          double* partial, double* out, double scale, cudaStream_t s);

void rsst_set_error(const char* fmt, ...);

// One run: configuration, padded state buffers, background, scalars.
struct rsst_handle {
  rsst_config cfg;
  Geom g;
  Phys p;
  cudaStream_t stream;
  size_t elem;          // bytes per stored scalar
  void* buf[2];         // padded state: buf[0] = U^n, buf[1] = U*
  double* d_bg;         // [2][bg_len] rho0, E0 (float64), or null
  int bg_len;
  double* d_scal;       // [0..1] CFL slots, [2] dt, [8..15] sums
  unsigned int* d_flag;
  double* d_partial;    // sums partials
  double* d_stage;      // caller-layout staging for host transfers
  double* h_small;      // pinned host scratch for small read-backs
  float* d_tab;         // background tables (float32 mode), or null
  float* d_tabr;        // row-major background table (float32 mode), or null
  PhysF pf;
  int use_tma2d;        // 2D float32 runs use the TMA-staged kernel
  int use_tma3d;        // 3D float32 runs use the TMA z-march kernel
  int use_tma_fp64;     // 2D/3D float64 runs stage their halo tiles by TMA
  CUtensorMap tmap[2];  // tensor maps of buf[0], buf[1] (TMA kernels)
  void* adj;            // adjoint checkpoints and work arrays, or null
  int slot;
  int64_t launches;
  // CUDA-graph replay of blocks of graph_steps steps (0: plain launches).
  // One executable graph per CFL-slot parity; graph_steps is even, so a
  // block leaves the parity unchanged.  Captured on cap_stream.
  int graph_steps;
  int graph_warm;           // a plain step ran (one-time kernel attributes set)
  cudaStream_t cap_stream;
  cudaGraphExec_t gexec[2];
  int gvalid[2];
  double gdt[2];            // the dt each graph was captured with
  double* rec_dU[2];        // float64 plain steps: Euler tendency of stage 1 / 2 written here if set
  int64_t stall_ns;         // rsst_debug_stall_wait (0: normal steps)
};

void rsst_adjoint_free(rsst_handle* h);

// Step a single run (used by rsst_step and by the batch's looped mode).
int rsst_handle_steps(rsst_handle* h, double dt, int nsteps);
// Wait for the run's queued work and read its device flag (RSST_FLAG_* bits).
int rsst_read_flag(rsst_handle* h, unsigned int* flag);
