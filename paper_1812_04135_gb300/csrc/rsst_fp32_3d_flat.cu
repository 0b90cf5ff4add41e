// Float32 stage kernel for 3D grids without a background (rsst_fp32_3d.cuh),
// compiled apart from the background case so the two build in parallel.
#include "rsst_fp32_3d.cuh"

int rsst_launch_stage3d_flat(const CUtensorMap* tin, const StageArgs<float>& a, cudaStream_t s) {
  return rsst::launch3d_vert<-1>(tin, a, s);
}
