// Float32 perturbation stage kernel for 3D grids (rsst_fp32_3d.cuh): the
// launches with a background along z, and the entry used by the C ABI.
// The kernels without a background are compiled in rsst_fp32_3d_flat.cu.
#include "rsst_fp32_3d.cuh"

int rsst_launch_stage3d_flat(const CUtensorMap* tin, const StageArgs<float>& a, cudaStream_t s);

using namespace rsst;

// TMA box of one plane of the 3D tile (halo included), for the tensor maps.
void rsst_stage3d_box(int* box_x, int* box_y) {
  *box_x = T3::SXP;
  *box_y = T3::SYP;
}

int rsst_launch_stage3d_tma(const CUtensorMap* tin, const StageArgs<float>& a, cudaStream_t s) {
  const int vert = a.tab ? a.p.vertical : -1;
  int rc;
  if (vert == 2) {
    rc = launch3d_vert<2>(tin, a, s);
  } else if (vert < 0) {
    rc = rsst_launch_stage3d_flat(tin, a, s);
  } else {
    rsst_set_error("3D TMA kernel supports a vertical axis of z or none");
    return RSST_EUNSUPPORTED;
  }
  if (rc != RSST_OK) return rc;
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    rsst_set_error("3D float32 TMA stage launch: %s", cudaGetErrorString(e));
    return RSST_ECUDA;
  }
  return RSST_OK;
}
