// Float32 perturbation stage kernel for 2D grids, TMA-staged.
//
// One tile = 128 x 8 cells, 128 threads.
//   1. One thread issues a single cp.async.bulk.tensor load of the tile with
//      its halo for all four fields (box 136 x 12 x 4 of the padded state, the
//      x origin rounded down to a 16-byte boundary, out-of-range parts zero
//      filled); the others copy the tile's rows of the row-major background
//      table (float4).
//   2. x faces, row by row, lanes along x (conflict-free): each lane's cell
//      slope gives its face's right state and, by a warp shuffle, the next
//      face's left state; twice the LLF flux into shared memory.
//   3. Each thread owns one column of 8 cells and marches up it: one new
//      half slope and one y-face flux per cell from a register window, then
//      the cell's divergence (its two x fluxes from shared memory), the
//      reduced tendency, force, RK combine, store and edge ghosts, and in
//      stage 2 the CFL rate and physical check, all fused.
// The same tile routine serves the single-run grid and the batched
// persistent kernel (rsst_batch.cu).
#include "rsst_common.cuh"
#include "rsst_fp32_2d.cuh"
#include "rsst_attr.h"

namespace rsst {

// One launch per stage; FORM, CM (C_max law) and ST (stage) are compile-time.
template <int VERT, int FORM, int CM, int ST>
__global__ void __launch_bounds__(T2::NT, 5) stage2d_tma_kernel(const __grid_constant__ CUtensorMap tin,
                                                                 const StageArgs<float> a) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  TileRun r;
  r.g = a.g;
  r.p = a.p;
  r.pf = a.pf;
  r.base = a.base;
  r.out = a.out;
  r.tabr = a.tabr;
  r.tab_len = a.tab_len;
  r.flag = a.flag;
  r.stage = ST;
  r.stall_ns = a.stall_ns;
  uint64_t* bar = t2_barrier<T2>(smem_raw);
  float* sdt = reinterpret_cast<float*>(bar + 1);
  if (threadIdx.x == 0) {
    // the float64 division is done once per CTA, not per thread
    const double dtd = a.dt_fixed > 0.0 ? a.dt_fixed : a.p.cfl / a.scal[a.slot];
    *sdt = (float)dtd;
    if (ST == 1 && blockIdx.x == 0 && blockIdx.y == 0) {
      a.scal[a.slot ^ 1] = 0.0;
      a.scal[2] = dtd;
      a.scal[3] += dtd;
    }
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  const float dtf = *sdt;
  uint32_t phase = 0;
  float rmax = 0.0f;
  bool ok = true;
  const bool fine = tile2d_f<T2, VERT, FORM, CM, ST>(&tin, r, dtf, blockIdx.x, blockIdx.y, smem_raw, phase, rmax, ok);
  if (!fine) return;
  if (ST == 2) {
    if (!ok) atomicOr(a.flag, RSST_FLAG_NONPHYSICAL);
    block_max_to<T2::NT>((double)rmax, a.scal + (a.slot ^ 1), t2_sred<T2>(smem_raw));
  }
}

template <int VERT, int FORM, int CM, int ST>
static int launch2d(const CUtensorMap* tin, const StageArgs<float>& a, cudaStream_t s) {
  static std::atomic<unsigned long long> attr{0};
  const size_t smem = T2::smem_bytes();
  if (set_smem_limit_once(stage2d_tma_kernel<VERT, FORM, CM, ST>, smem, attr) != cudaSuccess) {
    rsst_set_error("cudaFuncSetAttribute failed for the 2D float32 TMA stage kernel");
    return RSST_ECUDA;
  }
  dim3 grid((a.g.n[0] + T2::BX - 1) / T2::BX, (a.g.n[1] + T2::BY - 1) / T2::BY, 1);
  stage2d_tma_kernel<VERT, FORM, CM, ST><<<grid, T2::NT, smem, s>>>(*tin, a);
  return RSST_OK;
}

template <int VERT, int FORM>
static int launch2d_form(const CUtensorMap* tin, const StageArgs<float>& a, cudaStream_t s) {
  const bool cm = a.pf.use_cmax != 0;
  if (a.stage == 1) return cm ? launch2d<VERT, FORM, 1, 1>(tin, a, s) : launch2d<VERT, FORM, 0, 1>(tin, a, s);
  return cm ? launch2d<VERT, FORM, 1, 2>(tin, a, s) : launch2d<VERT, FORM, 0, 2>(tin, a, s);
}

template <int VERT>
static int launch2d_vert(const CUtensorMap* tin, const StageArgs<float>& a, cudaStream_t s) {
  switch (a.p.variant) {
    case RSST_EULER: return launch2d_form<VERT, RSST_EULER>(tin, a, s);
    case RSST_DVS: return launch2d_form<VERT, RSST_DVS>(tin, a, s);
    case RSST_PVS: return launch2d_form<VERT, RSST_PVS>(tin, a, s);
    case RSST_DMS: return launch2d_form<VERT, RSST_DMS>(tin, a, s);
    case RSST_PMS: return launch2d_form<VERT, RSST_PMS>(tin, a, s);
    default: return launch2d_form<VERT, RSST_PD>(tin, a, s);
  }
}

}  // namespace rsst

using namespace rsst;

// TMA box of the single-run tile (halo included), for the tensor maps.
void rsst_stage2d_box(int* box_x, int* box_y) {
  *box_x = T2::SXP;
  *box_y = T2::SYP;
}

int rsst_launch_stage2d_tma(const CUtensorMap* tin, const StageArgs<float>& a, cudaStream_t s) {
  const int vert = a.tab ? a.p.vertical : -1;
  int rc;
  if (vert == 1) {
    rc = launch2d_vert<1>(tin, a, s);
  } else if (vert < 0) {
    rc = launch2d_vert<-1>(tin, a, s);
  } else {
    rsst_set_error("2D TMA kernel supports a vertical axis of y or none");
    return RSST_EUNSUPPORTED;
  }
  if (rc != RSST_OK) return rc;
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    rsst_set_error("2D float32 TMA stage launch: %s", cudaGetErrorString(e));
    return RSST_ECUDA;
  }
  return RSST_OK;
}
