// Internal types shared by the librsst translation units (host and device).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "rsst.h"

#define RSST_G 2  // ghost layers per end of an active axis (MUSCL needs i-2..i+2)

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
  double gamma, gm1, inv_gm1;
  double xi, inv_xi, f;  // f = 1 - 1/xi^2
  double cfl;
  double grav[3];
  double inv_dx[3];
  double sum_inv_dx;     // sum_d 1/dx_d: CFL rate = c_tot * sum_inv_dx
  int variant;
  int vertical;          // background axis or -1
  int bc[3];
  int has_grav;
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
};

// Host-side launchers (defined in the .cu files).
int rsst_launch_stage_fp64(const StageArgs<double>& a, cudaStream_t s);
int rsst_launch_pack_fp64(const double* src, double* dst, const Geom& g, const Phys& p,
                          const double* bg, int bg_len, cudaStream_t s);
int rsst_launch_unpack_fp64(const double* src, double* dst, const Geom& g, cudaStream_t s);
int rsst_launch_cfl_fp64(const double* U, const Geom& g, const Phys& p, double* slot_ptr,
                         unsigned int* flag, cudaStream_t s);
int rsst_launch_sums_fp64(const double* U, const Geom& g, double* partial, double* out,
                          double scale, cudaStream_t s);

void rsst_set_error(const char* fmt, ...);
