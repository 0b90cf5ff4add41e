// C ABI of librsst (declared in include/rsst.h): handle management, state
// transfer, step orchestration on the caller's stream, diagnostics.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include <cudaTypedefs.h>

#include <type_traits>

#include "rsst_internal.h"
#include "rsst_check.h"

static thread_local char g_err[512] = "";

void rsst_set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof g_err, fmt, ap);
  va_end(ap);
}

extern "C" const char* rsst_last_error(void) { return g_err; }

int rsst_check_buffer(const void* p, int on_host, const char* where) {
  if (!p) {
    rsst_set_error("%s: NULL buffer", where);
    return RSST_EINVAL;
  }
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    rsst_set_error("%s: cannot query the buffer's memory type", where);
    return RSST_EINVAL;
  }
  const bool dev = a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
  if (!on_host && !dev) {
    rsst_set_error("%s: on_host = 0 but the buffer is host memory", where);
    return RSST_EINVAL;
  }
  if (on_host && a.type == cudaMemoryTypeDevice) {
    rsst_set_error("%s: on_host = 1 but the buffer is device memory", where);
    return RSST_EINVAL;
  }
  return RSST_OK;
}

#define CUDA_TRY(call)                                                              \
  do {                                                                              \
    const cudaError_t e_ = (call);                                                  \
    if (e_ != cudaSuccess) {                                                        \
      rsst_set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
      return RSST_ECUDA;                                                            \
    }                                                                               \
  } while (0)

#define RC_TRY(call)          \
  do {                        \
    const int rc_ = (call);   \
    if (rc_ != RSST_OK) return rc_; \
  } while (0)



void rsst_stage2d_box(int* box_x, int* box_y);  // rsst_fp32_2d.cu
void rsst_stage3d_box(int* box_x, int* box_y);  // rsst_fp32_3d.cu

static int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

// cuTensorMapEncodeTiled from the CUDA driver, looked up once (no link-time libcuda).
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)ptr;
  }
  return fn;
}

// Tiled float32 map of a padded 2D state [nvar][py][pitch], box of one tile
// plus halo for every field (x: 4 columns each side so the origin stays on a
// 16-byte boundary; y: 2 rows each side).
// Tiled float32 map of a padded 3D state [nvar][pz][py][pitch]: one z-plane
// of a tile with its x/y halo for every field.
static int make_tmap_3d(CUtensorMap* m, void* base, const Geom& g, int nv, int box_x, int box_y) {
  auto enc = tensor_map_encoder();
  if (!enc) { rsst_set_error("cuTensorMapEncodeTiled unavailable from the CUDA driver"); return RSST_ECUDA; }
  const cuuint64_t dims[4] = {(cuuint64_t)g.pitch, (cuuint64_t)g.py, (cuuint64_t)g.pz, (cuuint64_t)nv};
  const cuuint64_t strides[3] = {(cuuint64_t)g.pitch * 4, (cuuint64_t)g.plane * 4, (cuuint64_t)g.fstride * 4};
  const cuuint32_t box[4] = {(cuuint32_t)box_x, (cuuint32_t)box_y, 1, (cuuint32_t)nv};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  const CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, base, dims, strides, box, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) { rsst_set_error("cuTensorMapEncodeTiled (3D) failed (%d)", (int)r); return RSST_ECUDA; }
  return RSST_OK;
}

static int make_tmap_2d(CUtensorMap* m, void* base, const Geom& g, int nv, int box_x, int box_y) {
  auto enc = tensor_map_encoder();
  if (!enc) { rsst_set_error("cuTensorMapEncodeTiled unavailable from the CUDA driver"); return RSST_ECUDA; }
  const cuuint64_t dims[3] = {(cuuint64_t)g.pitch, (cuuint64_t)g.py, (cuuint64_t)nv};
  const cuuint64_t strides[2] = {(cuuint64_t)g.pitch * 4, (cuuint64_t)g.fstride * 4};
  const cuuint32_t box[3] = {(cuuint32_t)box_x, (cuuint32_t)box_y, (cuuint32_t)nv};
  const cuuint32_t estr[3] = {1, 1, 1};
  const CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, strides, box, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) { rsst_set_error("cuTensorMapEncodeTiled failed (%d)", (int)r); return RSST_ECUDA; }
  return RSST_OK;
}

// Tiled float64 map of a padded 2D/3D state [nvar][pz][py][pitch]: the
// float64 stage kernel's halo tile (box sx x sy [x sz]) of every field.
static int make_tmap_f64(CUtensorMap* m, void* base, const Geom& g, int nv) {
  auto enc = tensor_map_encoder();
  if (!enc) { rsst_set_error("cuTensorMapEncodeTiled unavailable from the CUDA driver"); return RSST_ECUDA; }
  int sx, sy, sz;
  rsst_stage_fp64_box(g.ndim, &sx, &sy, &sz);
  const bool d3 = g.ndim == 3;
  const cuuint32_t rank = d3 ? 4 : 3;
  const cuuint64_t dims[4] = {(cuuint64_t)g.pitch, (cuuint64_t)g.py, d3 ? (cuuint64_t)g.pz : (cuuint64_t)nv,
                              (cuuint64_t)nv};
  const cuuint64_t strides[3] = {(cuuint64_t)g.pitch * 8, d3 ? (cuuint64_t)g.plane * 8 : (cuuint64_t)g.fstride * 8,
                                 (cuuint64_t)g.fstride * 8};
  const cuuint32_t box[4] = {(cuuint32_t)sx, (cuuint32_t)sy, d3 ? (cuuint32_t)sz : (cuuint32_t)nv, (cuuint32_t)nv};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  const CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, rank, base, dims, strides, box, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) { rsst_set_error("cuTensorMapEncodeTiled (float64) failed (%d)", (int)r); return RSST_ECUDA; }
  return RSST_OK;
}

static int validate(const rsst_config* c) {
  if (!c) { rsst_set_error("config is NULL"); return RSST_EINVAL; }
  if (c->covolume != 0.0 && c->precision != RSST_FP64) {
    rsst_set_error("a covolume gas is implemented in the RSST_FP64 precision only");
    return RSST_EUNSUPPORTED;
  }
  if (c->ndim < 1 || c->ndim > 3) { rsst_set_error("ndim must be 1, 2 or 3 (got %d)", c->ndim); return RSST_EINVAL; }
  for (int d = 0; d < c->ndim; ++d) {
    if (c->n[d] < 2) { rsst_set_error("n[%d] must be >= 2 (got %d)", d, c->n[d]); return RSST_EINVAL; }
    if (!(c->dx[d] > 0.0) || !std::isfinite(c->dx[d])) { rsst_set_error("dx[%d] must be > 0", d); return RSST_EINVAL; }
    if (c->bc[d] != RSST_BC_PERIODIC && c->bc[d] != RSST_BC_REFLECT) { rsst_set_error("bc[%d] invalid", d); return RSST_EINVAL; }
  }
  if (c->variant < RSST_EULER || c->variant > RSST_PD) { rsst_set_error("variant %d invalid", c->variant); return RSST_EINVAL; }
  if (c->precision != RSST_FP64 && c->precision != RSST_FP32_PERT && c->precision != RSST_FP64_DF) { rsst_set_error("precision %d invalid", c->precision); return RSST_EINVAL; }
  if (!(c->xi >= 1.0) || !std::isfinite(c->xi)) { rsst_set_error("xi must be finite and >= 1 (got %g)", c->xi); return RSST_EINVAL; }
  if (!(c->gamma > 1.0) || !std::isfinite(c->gamma)) { rsst_set_error("gamma must be finite and > 1"); return RSST_EINVAL; }
  if (!(c->cfl > 0.0) || !std::isfinite(c->cfl)) { rsst_set_error("cfl must be finite and > 0"); return RSST_EINVAL; }
  if (c->cfl_rule != 0 && c->cfl_rule != 1) { rsst_set_error("cfl_rule must be 0 or 1 (got %d)", c->cfl_rule); return RSST_EINVAL; }
  for (int d = 0; d < c->ndim; ++d)
    if (!std::isfinite(c->grav[d])) { rsst_set_error("grav[%d] must be finite", d); return RSST_EINVAL; }
  if (!(c->cmax >= 0.0) || !std::isfinite(c->cmax)) { rsst_set_error("cmax must be >= 0 (0: constant xi)"); return RSST_EINVAL; }
  if (!(c->covolume >= 0.0) || !std::isfinite(c->covolume)) {
    rsst_set_error("covolume must be finite and >= 0 (0: ideal gas)");
    return RSST_EINVAL;
  }
  if (c->vertical < -1 || c->vertical >= c->ndim) { rsst_set_error("vertical axis %d invalid", c->vertical); return RSST_EINVAL; }
  if (c->vertical >= 0 && (!c->bg_rho || !c->bg_p)) { rsst_set_error("background profiles required when vertical >= 0"); return RSST_EINVAL; }
  if (c->vertical >= 0) {
    // The entries rsst_init reads: all n + 4 on a wall axis, the interior on a periodic one.
    const int nvert = c->n[c->vertical];
    const bool wrap = c->bc[c->vertical] == RSST_BC_PERIODIC;
    for (int k = wrap ? RSST_G : 0; k < (wrap ? nvert + RSST_G : nvert + 2 * RSST_G); ++k)
      if (!(c->bg_rho[k] > 0.0) || !(c->bg_p[k] > 0.0) || !std::isfinite(c->bg_rho[k]) || !std::isfinite(c->bg_p[k]) ||
          !(c->covolume * c->bg_rho[k] < 1.0)) {
        rsst_set_error("background entry %d must be finite with rho > 0, P > 0 and covolume * rho < 1", k);
        return RSST_EINVAL;
      }
  }
  int64_t cells = 1;
  for (int d = 0; d < c->ndim; ++d) cells *= c->n[d];
  if (cells > (int64_t)1 << 31) { rsst_set_error("grid too large (%lld cells)", (long long)cells); return RSST_EINVAL; }
  return RSST_OK;
}

static void make_geom(const rsst_config* c, size_t elem, Geom* g) {
  memset(g, 0, sizeof *g);
  g->ndim = c->ndim;
  for (int d = 0; d < 3; ++d) g->n[d] = d < c->ndim ? c->n[d] : 1;
  g->gy = c->ndim >= 2 ? RSST_G : 0;
  g->gz = c->ndim >= 3 ? RSST_G : 0;
  g->xoff = (int)(32 / elem);
  g->py = c->ndim >= 2 ? g->n[1] + 2 * RSST_G : 1;
  g->pz = c->ndim >= 3 ? g->n[2] + 2 * RSST_G : 1;
  g->pitch = round_up(g->xoff + g->n[0] + RSST_G, 32);
  g->plane = g->pitch * g->py;
  g->fstride = round_up(g->plane * g->pz, 32);
  g->ncells = (int64_t)g->n[0] * g->n[1] * g->n[2];
}

static void make_physf(const Phys* p, PhysF* f) {
  memset(f, 0, sizeof *f);
  f->gamma = (float)p->gamma;
  f->gm1 = (float)p->gm1;
  f->inv_gm1 = (float)p->inv_gm1;
  f->inv_xi = (float)p->inv_xi;
  f->f = (float)p->f;
  f->inv_cmax4 = (float)p->inv_cmax4;
  f->use_cmax = p->use_cmax;
  for (int d = 0; d < 3; ++d) {
    f->grav[d] = (float)p->grav[d];
    f->inv_dx[d] = (float)p->inv_dx[d];
  }
  f->sum_inv_dx = (float)p->sum_inv_dx;
  f->hgm1 = (float)p->hgm1;
  f->gam_gm1 = (float)(p->gamma / p->gm1);
  f->gx = (float)(p->use_cmax ? p->gamma : p->gamma_xi2);
}

static void make_phys(const rsst_config* c, Phys* p) {
  memset(p, 0, sizeof *p);
  p->gamma = c->gamma;
  p->gm1 = c->gamma - 1.0;
  p->inv_gm1 = 1.0 / (c->gamma - 1.0);
  p->hgm1 = 0.5 * (c->gamma - 1.0);
  p->xi = c->xi;
  p->inv_xi = 1.0 / c->xi;
  p->f = 1.0 - 1.0 / (c->xi * c->xi);
  p->gamma_xi2 = c->gamma / (c->xi * c->xi);
  p->use_cmax = c->cmax > 0.0;
  p->inv_cmax4 = p->use_cmax ? 1.0 / (c->cmax * c->cmax * c->cmax * c->cmax) : 0.0;
  p->cfl = c->cfl;
  p->covol = c->covolume;
  p->variant = c->variant;
  p->vertical = c->vertical;
  p->sum_inv_dx = 0.0;
  for (int d = 0; d < 3; ++d) {
    const bool act = d < c->ndim;
    p->grav[d] = act ? c->grav[d] : 0.0;
    p->inv_dx[d] = act ? 1.0 / c->dx[d] : 0.0;
    p->bc[d] = act ? c->bc[d] : RSST_BC_PERIODIC;
    if (act) p->sum_inv_dx += 1.0 / c->dx[d];
    if (act && c->grav[d] != 0.0) p->has_grav = 1;
  }
  // Every kernel forms the CFL rate as c_tot * sum_inv_dx; the rule
  // dt = cfl min_d dx_d / max c_tot is the same with 1 / min_d dx_d.
  if (c->cfl_rule == 1) {
    double m = 0.0;
    for (int d = 0; d < c->ndim; ++d) m = std::fmax(m, 1.0 / c->dx[d]);
    p->sum_inv_dx = m;
  }
}

static void drop_graphs(rsst_handle* h) {
  for (int p = 0; p < 2; ++p) {
    if (h->gvalid[p]) cudaGraphExecDestroy(h->gexec[p]);
    h->gvalid[p] = 0;
  }
}

extern "C" void rsst_destroy(rsst_handle* h) {
  if (!h) return;
  rsst_adjoint_free(h);
  drop_graphs(h);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  cudaFree(h->buf[0]);
  cudaFree(h->buf[1]);
  cudaFree(h->d_bg);
  cudaFree(h->d_scal);
  cudaFree(h->d_flag);
  cudaFree(h->d_partial);
  cudaFree(h->d_stage);
  cudaFree(h->d_tab);
  cudaFree(h->d_tabr);
  cudaFreeHost(h->h_small);
  delete h;
}

extern "C" int rsst_init(rsst_handle** out, const rsst_config* cfg, void* stream) {
  if (!out) { rsst_set_error("handle pointer is NULL"); return RSST_EINVAL; }
  *out = nullptr;
  RC_TRY(validate(cfg));
  rsst_handle* h = new rsst_handle();
  memset(h, 0, sizeof *h);
  h->cfg = *cfg;
  h->cfg.bg_rho = nullptr;
  h->cfg.bg_p = nullptr;
  h->stream = (cudaStream_t)stream;
  h->graph_steps = RSST_DEFAULT_GRAPH_STEPS;
  h->elem = cfg->precision == RSST_FP32_PERT ? sizeof(float) : sizeof(double);  // a double-float is 8 bytes
  make_geom(cfg, h->elem, &h->g);
  make_phys(cfg, &h->p);
  make_physf(&h->p, &h->pf);
  const int nv = cfg->ndim + 2;
  const size_t sbytes = (size_t)nv * h->g.fstride * h->elem;
  int rc = RSST_OK;
#define ALLOC(ptr, bytes)                                                          \
  if (cudaMalloc((void**)&(ptr), (bytes)) != cudaSuccess) {                        \
    cudaGetLastError();                                                            \
    rsst_set_error("cudaMalloc of %zu bytes failed", (size_t)(bytes));             \
    rc = RSST_ENOMEM;                                                              \
    goto fail;                                                                     \
  }
  ALLOC(h->buf[0], sbytes);
  ALLOC(h->buf[1], sbytes);
  ALLOC(h->d_scal, 16 * sizeof(double));
  ALLOC(h->d_flag, sizeof(unsigned int));
  ALLOC(h->d_partial, (size_t)nv * 1024 * sizeof(double));
  ALLOC(h->d_stage, (size_t)nv * h->g.ncells * sizeof(double));
  if (cudaMallocHost((void**)&h->h_small, 64 * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    rsst_set_error("cudaMallocHost failed");
    rc = RSST_ENOMEM;
    goto fail;
  }
  if (cfg->vertical >= 0) {
    const int nvert = h->g.n[cfg->vertical];
    h->bg_len = nvert + 2 * RSST_G;
    double* tmp = (double*)malloc(2 * h->bg_len * sizeof(double));
    if (!tmp) { rsst_set_error("host allocation of the background failed"); rc = RSST_ENOMEM; goto fail; }
    for (int k = 0; k < h->bg_len; ++k) {
      int src = k;
      if (cfg->bc[cfg->vertical] == RSST_BC_PERIODIC) src = ((k - RSST_G) % nvert + nvert) % nvert + RSST_G;
      tmp[k] = cfg->bg_rho[src];
      // E0 = e(rho0, P0): P0/(gamma-1), times (1 - b rho0) for a covolume gas
      tmp[h->bg_len + k] = cfg->covolume == 0.0 ? cfg->bg_p[src] / (cfg->gamma - 1.0)
                                                : cfg->bg_p[src] * (1.0 - cfg->covolume * cfg->bg_rho[src]) /
                                                      (cfg->gamma - 1.0);
    }
    ALLOC(h->d_bg, 2 * h->bg_len * sizeof(double));
    const cudaError_t e = cudaMemcpy(h->d_bg, tmp, 2 * h->bg_len * sizeof(double), cudaMemcpyHostToDevice);
    free(tmp);
    if (e != cudaSuccess) { rsst_set_error("background upload: %s", cudaGetErrorString(e)); rc = RSST_ECUDA; goto fail; }
    if (cfg->precision == RSST_FP32_PERT) {
      ALLOC(h->d_tab, (size_t)TB_COUNT * h->bg_len * sizeof(float));
      ALLOC(h->d_tabr, (size_t)TR_W * h->bg_len * sizeof(float));
      rc = rsst_launch_bgtab(h->d_bg, h->bg_len, h->g, h->p, h->d_tab, h->d_tabr, 0);
      if (rc != RSST_OK) goto fail;
      if (cudaDeviceSynchronize() != cudaSuccess) { rsst_set_error("background table kernel failed"); rc = RSST_ECUDA; goto fail; }
    }
  }
  if (cudaMemset(h->buf[0], 0, sbytes) != cudaSuccess || cudaMemset(h->buf[1], 0, sbytes) != cudaSuccess ||
      cudaMemset(h->d_scal, 0, 16 * sizeof(double)) != cudaSuccess || cudaMemset(h->d_flag, 0, sizeof(unsigned)) != cudaSuccess) {
    rsst_set_error("initial memset failed");
    rc = RSST_ECUDA;
    goto fail;
  }
#undef ALLOC
  if (cfg->precision == RSST_FP32_PERT && cfg->ndim == 2 && (cfg->vertical == -1 || cfg->vertical == 1)) {
    h->use_tma2d = 1;
    for (int b = 0; b < 2; ++b) {
      int bx, by;
      rsst_stage2d_box(&bx, &by);
      rc = make_tmap_2d(&h->tmap[b], h->buf[b], h->g, nv, bx, by);
      if (rc != RSST_OK) goto fail;
    }
  }
  if (cfg->precision == RSST_FP64 && cfg->ndim >= 2) {
    h->use_tma_fp64 = 1;
    for (int b = 0; b < 2; ++b) {
      rc = make_tmap_f64(&h->tmap[b], h->buf[b], h->g, nv);
      if (rc != RSST_OK) goto fail;
    }
  }
  if (cfg->precision == RSST_FP32_PERT && cfg->ndim == 3 && (cfg->vertical == -1 || cfg->vertical == 2)) {
    h->use_tma3d = 1;
    for (int b = 0; b < 2; ++b) {
      int bx, by;
      rsst_stage3d_box(&bx, &by);
      rc = make_tmap_3d(&h->tmap[b], h->buf[b], h->g, nv, bx, by);
      if (rc != RSST_OK) goto fail;
    }
  }
  *out = h;
  return RSST_OK;
fail:
  rsst_destroy(h);
  return rc;
}

int rsst_read_flag(rsst_handle* h, unsigned int* flag) {
  CUDA_TRY(cudaMemcpyAsync(h->h_small, h->d_flag, sizeof(unsigned int), cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  memcpy(flag, h->h_small, sizeof *flag);
  return RSST_OK;
}

// A timeout is reported first: a stage that gave up left part of its output
// unwritten, which may also look non-physical.
static int check_flag(rsst_handle* h) {
  unsigned int f = 0;
  RC_TRY(rsst_read_flag(h, &f));
  if (f & RSST_FLAG_TIMEOUT) {
    rsst_set_error("a bounded device wait (TMA copy or barrier) gave up: the step's output is incomplete");
    return RSST_ETIMEOUT;
  }
  if (f & RSST_FLAG_NONPHYSICAL) {
    rsst_set_error("non-physical state (rho <= 0, P <= 0 or NaN) produced");
    return RSST_ENONPHYSICAL;
  }
  return RSST_OK;
}

extern "C" int rsst_set_state(rsst_handle* h, const double* U, int on_host) {
  if (!h || !U) { rsst_set_error("NULL argument"); return RSST_EINVAL; }
  RC_TRY(rsst_check_buffer(U, on_host, "rsst_set_state"));
  const int nv = h->g.ndim + 2;
  const size_t bytes = (size_t)nv * h->g.ncells * sizeof(double);
  const double* src = U;
  if (on_host) {
    CUDA_TRY(cudaMemcpyAsync(h->d_stage, U, bytes, cudaMemcpyHostToDevice, h->stream));
    src = h->d_stage;
  }
  const bool f32 = h->cfg.precision == RSST_FP32_PERT;
  const bool dfp = h->cfg.precision == RSST_FP64_DF;
  if (f32)
    RC_TRY(rsst_launch_pack_fp32(src, (float*)h->buf[0], h->g, h->p, h->d_bg, h->bg_len, h->stream));
  else if (dfp)
    RC_TRY(rsst_launch_pack_df(src, (float2*)h->buf[0], h->g, h->p, h->d_bg, h->bg_len, h->stream));
  else
    RC_TRY(rsst_launch_pack_fp64(src, (double*)h->buf[0], h->g, h->p, h->d_bg, h->bg_len, h->stream));
  CUDA_TRY(cudaMemsetAsync(h->d_flag, 0, sizeof(unsigned int), h->stream));
  CUDA_TRY(cudaMemsetAsync(h->d_scal + h->slot, 0, sizeof(double), h->stream));
  CUDA_TRY(cudaMemsetAsync(h->d_scal + 3, 0, sizeof(double), h->stream));  // simulated time
  if (dfp)
    RC_TRY(rsst_launch_cfl_df((const float2*)h->buf[0], h->g, h->p, h->d_scal + h->slot, h->d_flag, h->stream));
  else if (f32)
    RC_TRY(rsst_launch_cfl_fp32((const float*)h->buf[0], h->g, h->p, h->pf, h->d_tab, h->bg_len, h->d_scal + h->slot,
                                h->d_flag, h->stream));
  else
    RC_TRY(rsst_launch_cfl_fp64((const double*)h->buf[0], h->g, h->p, h->d_scal + h->slot, h->d_flag, h->stream));
  h->launches += 2;
  return RSST_OK;
}

extern "C" int rsst_get_state(rsst_handle* h, double* U, int on_host) {
  if (!h || !U) { rsst_set_error("NULL argument"); return RSST_EINVAL; }
  RC_TRY(rsst_check_buffer(U, on_host, "rsst_get_state"));
  const int nv = h->g.ndim + 2;
  const size_t bytes = (size_t)nv * h->g.ncells * sizeof(double);
  double* dst = on_host ? h->d_stage : U;
  if (h->cfg.precision == RSST_FP32_PERT)
    RC_TRY(rsst_launch_unpack_fp32((const float*)h->buf[0], dst, h->g, h->p, h->d_bg, h->bg_len, h->stream));
  else if (h->cfg.precision == RSST_FP64_DF)
    RC_TRY(rsst_launch_unpack_df((const float2*)h->buf[0], dst, h->g, h->stream));
  else
    RC_TRY(rsst_launch_unpack_fp64((const double*)h->buf[0], dst, h->g, h->stream));
  h->launches += 1;
  if (on_host) CUDA_TRY(cudaMemcpyAsync(U, h->d_stage, bytes, cudaMemcpyDeviceToHost, h->stream));
  return check_flag(h);
}

template <typename T>
static int plain_steps(rsst_handle* h, double dt, int nsteps, cudaStream_t st) {
  StageArgs<T> a;
  memset(&a, 0, sizeof a);
  a.g = h->g;
  a.p = h->p;
  a.pf = h->pf;
  a.bg = h->d_bg;
  a.bg_len = h->bg_len;
  a.tab = h->d_tab;
  a.tabr = h->d_tabr;
  a.tab_len = h->bg_len;
  a.scal = h->d_scal;
  a.flag = h->d_flag;
  a.dt_fixed = dt > 0.0 ? dt : 0.0;
  a.stall_ns = h->stall_ns;
  T* U = (T*)h->buf[0];
  T* Us = (T*)h->buf[1];
  for (int s = 0; s < nsteps; ++s) {
    a.slot = h->slot;
    a.stage = 1;
    a.in = U;
    a.base = nullptr;
    a.out = Us;
    a.dU_out = h->rec_dU[0];
    if constexpr (std::is_same<T, double>::value) RC_TRY(rsst_launch_stage_fp64(h->use_tma_fp64 ? &h->tmap[0] : nullptr, a, st));
    else if constexpr (std::is_same<T, float2>::value) RC_TRY(rsst_launch_stage_df(a, st));
    else if (h->use_tma2d) RC_TRY(rsst_launch_stage2d_tma(&h->tmap[0], a, st));
    else if (h->use_tma3d) RC_TRY(rsst_launch_stage3d_tma(&h->tmap[0], a, st));
    else RC_TRY(rsst_launch_stage_fp32(a, st));
    a.stage = 2;
    a.in = Us;
    a.base = U;
    a.out = U;
    a.dU_out = h->rec_dU[1];
    if constexpr (std::is_same<T, double>::value) RC_TRY(rsst_launch_stage_fp64(h->use_tma_fp64 ? &h->tmap[1] : nullptr, a, st));
    else if constexpr (std::is_same<T, float2>::value) RC_TRY(rsst_launch_stage_df(a, st));
    else if (h->use_tma2d) RC_TRY(rsst_launch_stage2d_tma(&h->tmap[1], a, st));
    else if (h->use_tma3d) RC_TRY(rsst_launch_stage3d_tma(&h->tmap[1], a, st));
    else RC_TRY(rsst_launch_stage_fp32(a, st));
    h->launches += 2;
    h->slot ^= 1;
  }
  return RSST_OK;
}

// Capture graph_steps steps starting at the current slot parity on the
// private capture stream (nothing runs during capture) and instantiate them.
template <typename T>
static int build_graph(rsst_handle* h, double dt) {
  const int p = h->slot;
  if (h->gvalid[p]) {
    cudaGraphExecDestroy(h->gexec[p]);
    h->gvalid[p] = 0;
  }
  if (!h->cap_stream && cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    h->cap_stream = nullptr;
    rsst_set_error("could not create the graph capture stream");
    return RSST_ECUDA;
  }
  if (cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    rsst_set_error("cudaStreamBeginCapture failed");
    return RSST_ECUDA;
  }
  const int64_t launches = h->launches;
  const int rc = plain_steps<T>(h, dt, h->graph_steps, h->cap_stream);
  h->launches = launches;
  h->slot = p;  // an even number of steps: the parity is unchanged
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(h->cap_stream, &g);
  if (rc != RSST_OK || e != cudaSuccess || cudaGraphInstantiate(&h->gexec[p], g, 0) != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    if (rc == RSST_OK) rsst_set_error("graph capture of the step failed");
    return rc != RSST_OK ? rc : RSST_ECUDA;
  }
  cudaGraphDestroy(g);
  h->gvalid[p] = 1;
  h->gdt[p] = dt;
  return RSST_OK;
}

// nsteps SSP-RK2 steps: whole blocks of graph_steps steps replay a captured
// graph on the caller's stream, the rest are plain launches.
template <typename T>
static int run_steps(rsst_handle* h, double dt, int nsteps) {
  const int K = h->graph_steps;
  if (K > 0 && nsteps >= K && !h->rec_dU[0] && !h->rec_dU[1]) {
    if (!h->graph_warm) {  // first launch sets the kernels' attributes outside any capture
      RC_TRY(plain_steps<T>(h, dt, 1, h->stream));
      h->graph_warm = 1;
      --nsteps;
    }
    while (nsteps >= K) {
      const int p = h->slot;
      if (!h->gvalid[p] || h->gdt[p] != dt) RC_TRY(build_graph<T>(h, dt));
      if (cudaGraphLaunch(h->gexec[p], h->stream) != cudaSuccess) {
        rsst_set_error("graph launch failed: %s", cudaGetErrorString(cudaGetLastError()));
        return RSST_ECUDA;
      }
      h->launches += 2 * (int64_t)K;
      nsteps -= K;
    }
  }
  return plain_steps<T>(h, dt, nsteps, h->stream);
}

int rsst_handle_steps(rsst_handle* h, double dt, int nsteps) {
  if (h->cfg.precision == RSST_FP32_PERT) return run_steps<float>(h, dt, nsteps);
  if (h->cfg.precision == RSST_FP64_DF) return run_steps<float2>(h, dt, nsteps);
  return run_steps<double>(h, dt, nsteps);
}

extern "C" int rsst_set_graph_steps(rsst_handle* h, int32_t k) {
  if (!h || k < 0 || (k & 1)) {
    rsst_set_error("rsst_set_graph_steps: need a handle and an even k >= 0");
    return RSST_EINVAL;
  }
  if (k != h->graph_steps) drop_graphs(h);
  h->graph_steps = k;
  return RSST_OK;
}

extern "C" int rsst_debug_stall_wait(rsst_handle* h, int64_t limit_ns) {
  if (!h || limit_ns < 0 || limit_ns > 1000000000LL) {
    rsst_set_error("rsst_debug_stall_wait: need a handle and 0 <= limit_ns <= 1e9");
    return RSST_EINVAL;
  }
  if (!h->use_tma2d && !h->use_tma3d && !h->use_tma_fp64) {
    rsst_set_error("rsst_debug_stall_wait: only runs on the TMA-staged kernels (float32 perturbation 2D/3D, float64 2D/3D) have the test wait");
    return RSST_EUNSUPPORTED;
  }
  if (limit_ns != h->stall_ns) drop_graphs(h);  // graphs hold the stage arguments by value
  h->stall_ns = limit_ns;
  return RSST_OK;
}

extern "C" int rsst_step(rsst_handle* h, double dt, int nsteps) {
  if (!h) { rsst_set_error("NULL handle"); return RSST_EINVAL; }
  if (nsteps < 0) { rsst_set_error("nsteps must be >= 0"); return RSST_EINVAL; }
  if (!std::isfinite(dt)) { rsst_set_error("dt must be finite"); return RSST_EINVAL; }
  return rsst_handle_steps(h, dt, nsteps);
}

extern "C" int rsst_dt(rsst_handle* h, double* dt_out) {
  if (!h || !dt_out) { rsst_set_error("NULL argument"); return RSST_EINVAL; }
  CUDA_TRY(cudaMemcpyAsync(h->h_small, h->d_scal + h->slot, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  const double cmax = h->h_small[0];
  *dt_out = h->p.cfl / cmax;
  return check_flag(h);
}

extern "C" int rsst_time(rsst_handle* h, double* t) {
  if (!h || !t) { rsst_set_error("NULL argument"); return RSST_EINVAL; }
  CUDA_TRY(cudaMemcpyAsync(h->h_small, h->d_scal + 3, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  *t = h->h_small[0];
  return check_flag(h);
}

extern "C" int rsst_sync(rsst_handle* h) {
  if (!h) { rsst_set_error("NULL handle"); return RSST_EINVAL; }
  return check_flag(h);
}

extern "C" int rsst_conserved_sums(rsst_handle* h, double* sums) {
  if (!h || !sums) { rsst_set_error("NULL argument"); return RSST_EINVAL; }
  const int nv = h->g.ndim + 2;
  double vol = 1.0;
  for (int d = 0; d < h->g.ndim; ++d) vol *= h->cfg.dx[d];
  if (h->cfg.precision == RSST_FP32_PERT)
    RC_TRY(rsst_launch_sums_fp32((const float*)h->buf[0], h->g, h->p, h->d_bg, h->bg_len, h->d_partial, h->d_scal + 8,
                                 vol, h->stream));
  else if (h->cfg.precision == RSST_FP64_DF)
    RC_TRY(rsst_launch_sums_df((const float2*)h->buf[0], h->g, h->d_partial, h->d_scal + 8, vol, h->stream));
  else
    RC_TRY(rsst_launch_sums_fp64((const double*)h->buf[0], h->g, h->d_partial, h->d_scal + 8, vol, h->stream));
  h->launches += 2;
  CUDA_TRY(cudaMemcpyAsync(h->h_small, h->d_scal + 8, nv * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  memcpy(sums, h->h_small, nv * sizeof(double));
  return check_flag(h);
}

extern "C" int64_t rsst_kernel_launches(const rsst_handle* h) { return h ? h->launches : 0; }

extern "C" size_t rsst_config_size(void) { return sizeof(rsst_config); }
