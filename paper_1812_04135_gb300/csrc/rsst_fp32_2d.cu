// Float32 perturbation stage kernel for 2D grids, TMA-staged.
//
// One tile = 128 x 8 cells, 128 threads (five CTAs per SM).
//   1. One thread issues a single cp.async.bulk.tensor load of the tile with
//      its halo for all four fields (box 136 x 12 x 4 of the padded state, the
//      x origin rounded down to a 16-byte boundary, out-of-range parts zero
//      filled); the others stage the background table rows of the tile.
//   2. x faces, one per thread in turn (lanes along x, conflict-free), LLF
//      flux of the MC-reconstructed states into shared memory.
//   3. Each thread owns one column of 8 cells and marches up it: one new MC
//      slope and one y-face flux per cell from a register window, then the
//      cell's divergence (its two x fluxes from shared memory), the reduced
//      tendency, force, RK combine, store and edge ghosts, and in stage 2 the
//      CFL rate and physical check, all fused.
// The same tile routine serves the single-run grid and the batched
// persistent kernel (rsst_batch.cu).
#include "rsst_common.cuh"
#include "rsst_fp32_2d.cuh"
#include "rsst_attr.h"

namespace rsst {

template <int VERT>
__global__ void __launch_bounds__(T2::NT, 5) stage2d_tma_kernel(const __grid_constant__ CUtensorMap tin,
                                                                 const StageArgs<float> a) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  TileRun r;
  r.g = a.g;
  r.p = a.p;
  r.pf = a.pf;
  r.base = a.base;
  r.out = a.out;
  r.tab = a.tab;
  r.tab_len = a.tab_len;
  r.flag = a.flag;
  r.stage = a.stage;
  r.stall_ns = a.stall_ns;
  uint64_t* bar = t2_barrier<T2>(smem_raw);
  float* sdt = reinterpret_cast<float*>(bar + 1);
  if (threadIdx.x == 0) {
    // the float64 division is done once per CTA, not per thread
    const double dtd = a.dt_fixed > 0.0 ? a.dt_fixed : a.p.cfl / a.scal[a.slot];
    *sdt = (float)dtd;
    if (a.stage == 1 && blockIdx.x == 0 && blockIdx.y == 0) {
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
  const bool fine = tile2d_f<T2, VERT>(&tin, r, dtf, blockIdx.x, blockIdx.y, smem_raw, phase, rmax, ok);
  if (!fine) return;
  if (a.stage == 2) {
    if (!ok) atomicOr(a.flag, RSST_FLAG_NONPHYSICAL);
    block_max_to<T2::NT>((double)rmax, a.scal + (a.slot ^ 1), t2_sred<T2>(smem_raw));
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
  dim3 grid((a.g.n[0] + T2::BX - 1) / T2::BX, (a.g.n[1] + T2::BY - 1) / T2::BY, 1);
  const size_t smem = T2::smem_bytes();
  if (vert == 1) {
    static std::atomic<unsigned long long> attr{0};
    if (set_smem_limit_once(stage2d_tma_kernel<1>, smem, attr) != cudaSuccess) {
      rsst_set_error("cudaFuncSetAttribute failed for the 2D float32 TMA stage kernel");
      return RSST_ECUDA;
    }
    stage2d_tma_kernel<1><<<grid, T2::NT, smem, s>>>(*tin, a);
  } else if (vert < 0) {
    static std::atomic<unsigned long long> attr{0};
    if (set_smem_limit_once(stage2d_tma_kernel<-1>, smem, attr) != cudaSuccess) {
      rsst_set_error("cudaFuncSetAttribute failed for the 2D float32 TMA stage kernel");
      return RSST_ECUDA;
    }
    stage2d_tma_kernel<-1><<<grid, T2::NT, smem, s>>>(*tin, a);
  } else {
    rsst_set_error("2D TMA kernel supports a vertical axis of y or none");
    return RSST_EUNSUPPORTED;
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    rsst_set_error("2D float32 TMA stage launch: %s", cudaGetErrorString(e));
    return RSST_ECUDA;
  }
  return RSST_OK;
}
