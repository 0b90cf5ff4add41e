// Batched float32-perturbation RSST steps: many independent 2D runs of uneven
// size, xi and background in one persistent kernel per RK stage.
//
// The tiles of all runs form one ragged list, with one (run, tile within the
// run) entry per tile.  A grid of (SMs x resident CTAs) walks that list with
// a fixed stride; each tile reads its entry (one load), the block copies the
// run's descriptor for the stage into shared memory (eight bytes a thread,
// one round) and runs the same TMA-staged tile routine as the single-run
// kernel with that run's tensor map, tables, dt and CFL slot.
// The two stages of one step are captured once per CFL-slot parity into a
// CUDA graph and replayed.  The tile shape is chosen by a timing autotuner
// over six candidates (optionally cached in the file named by
// RSST_TUNE_CACHE).
#include <cstddef>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include <cudaTypedefs.h>

#include "rsst_fp32_2d.cuh"

namespace rsst {

struct BatchRun {
  CUtensorMap tmap[2];  // maps of buf[0] and buf[1] for the chosen tile shape
  TileRun r[2];         // the run's descriptor for stage 1 and stage 2
  float* buf[2];
  double* scal;
  int tiles_x;
  int vert;
};

static_assert(sizeof(TileRun) % 8 == 0 && offsetof(BatchRun, r) % 8 == 0, "descriptor copied in 8-byte words");

template <class C, int ST>
__global__ void __launch_bounds__(C::NT) batch_stage_kernel(const BatchRun* __restrict__ runs,
                                                             const int2* __restrict__ tile_info, int total_tiles,
                                                             int slot) {
  constexpr int stage = ST;
  constexpr int NW = (int)(sizeof(TileRun) / 8);
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t* bar = t2_barrier<C>(smem_raw);
  float* sdt = reinterpret_cast<float*>(bar + 1);
  TileRun* sr = reinterpret_cast<TileRun*>(t2_extra<C>(smem_raw));
  static_assert(sizeof(TileRun) <= 512, "run descriptor must fit the reserved shared memory");
  static_assert(NW <= C::NT, "the descriptor is copied in one round");
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  uint32_t phase = 0;
  // The next tile's list entry, this thread's word of its run descriptor and
  // (thread 0) its CFL slot value are loaded one tile ahead, so that no
  // dependent global load stands between two tiles.
  int t = blockIdx.x;
  int2 ti = make_int2(0, 0);
  unsigned long long dword = 0ull;
  double cfl = 0.0, cmax_slot = 1.0;
  auto fetch = [&](int u, int2& e) {
    e = tile_info[u];
    const BatchRun& rb = runs[e.x];
    if (threadIdx.x < NW) dword = reinterpret_cast<const unsigned long long*>(&rb.r[stage - 1])[threadIdx.x];
    if (threadIdx.x == 0) {
      cfl = rb.r[0].p.cfl;
      cmax_slot = rb.scal[slot];
    }
  };
  if (t < total_tiles) fetch(t, ti);
  for (; t < total_tiles; t += gridDim.x) {
    const BatchRun& br = runs[ti.x];
    if (threadIdx.x < NW) reinterpret_cast<unsigned long long*>(sr)[threadIdx.x] = dword;
    if (threadIdx.x == 0) {
      const double dtd = cfl / cmax_slot;
      *sdt = (float)dtd;
      if (stage == 1 && ti.y == 0) {
        br.scal[slot ^ 1] = 0.0;
        br.scal[2] = dtd;
        br.scal[3] += dtd;
      }
    }
    __syncthreads();
    int2 tnext = ti;
    if (t + (int)gridDim.x < total_tiles) fetch(t + gridDim.x, tnext);
    const int tx = ti.y % br.tiles_x, ty = ti.y / br.tiles_x;
    const CUtensorMap* map = &br.tmap[stage == 1 ? 0 : 1];
    float rmax = 0.0f;
    bool ok = true;
    // the background case and the C_max law are fixed per tile (compile-time
    // variants of the tile routine); the form is read from the run
    const bool cm = sr->pf.use_cmax != 0;
    bool fine;
    if (br.vert == 1)
      fine = cm ? tile2d_f<C, 1, -1, 1, ST>(map, *sr, *sdt, tx, ty, smem_raw, phase, rmax, ok)
                : tile2d_f<C, 1, -1, 0, ST>(map, *sr, *sdt, tx, ty, smem_raw, phase, rmax, ok);
    else
      fine = cm ? tile2d_f<C, -1, -1, 1, ST>(map, *sr, *sdt, tx, ty, smem_raw, phase, rmax, ok)
                : tile2d_f<C, -1, -1, 0, ST>(map, *sr, *sdt, tx, ty, smem_raw, phase, rmax, ok);
    if (!fine) {
      // A bounded wait gave up (the tile routine has already waited for its
      // copy).  This block leaves the rest of the stage: every run that owns
      // one of its remaining tiles gets the timeout flag, so no run is left
      // partly unwritten without being reported.
      if (threadIdx.x == 0) {
        for (int u = t + gridDim.x; u < total_tiles; u += gridDim.x) atomicOr(runs[tile_info[u].x].r[0].flag, RSST_FLAG_TIMEOUT);
      }
      return;
    }
    if (stage == 2) {
      if (!ok) atomicOr(sr->flag, RSST_FLAG_NONPHYSICAL);
      block_max_to<C::NT>((double)rmax, br.scal + (slot ^ 1), t2_sred<C>(smem_raw));
    }
    __syncthreads();  // the descriptor copy is rewritten for the next tile
    ti = tnext;
  }
}

// Candidate tile shapes for the autotuner.
using TC0 = T2Cfg<64, 32, 8>;
using TC1 = T2Cfg<32, 32, 8>;
using TC2 = T2Cfg<64, 16, 4>;
using TC3 = T2Cfg<128, 16, 8>;
using TC4 = T2Cfg<64, 24, 8>;
using TC5 = T2Cfg<128, 8, 8>;
constexpr int NCAND = 6;
static const int CAND_BX[NCAND] = {64, 32, 64, 128, 64, 128};
static const int CAND_BY[NCAND] = {32, 32, 16, 16, 24, 8};

}  // namespace rsst

using namespace rsst;

struct rsst_batch {
  int nruns;
  cudaStream_t stream;
  std::vector<rsst_handle*> runs;
  BatchRun* d_runs;
  int2* d_tile_info;   // per tile of the list: (run, tile within the run)
  int choice;
  int total_tiles;
  int grid;
  int slot;
  bool graph_ok[2];
  cudaGraphExec_t graph[2];
  int64_t launches;
};

static PFN_cuTensorMapEncodeTiled_v12000 batch_encoder() {
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

template <class C>
static void* kernel_of(int stage) {
  return stage == 1 ? (void*)batch_stage_kernel<C, 1> : (void*)batch_stage_kernel<C, 2>;
}

static void* cand_kernel(int c, int* nt, size_t* smem, int stage = 1) {
  switch (c) {
    case 0: *nt = TC0::NT; *smem = TC0::smem_bytes(); return kernel_of<TC0>(stage);
    case 1: *nt = TC1::NT; *smem = TC1::smem_bytes(); return kernel_of<TC1>(stage);
    case 2: *nt = TC2::NT; *smem = TC2::smem_bytes(); return kernel_of<TC2>(stage);
    case 3: *nt = TC3::NT; *smem = TC3::smem_bytes(); return kernel_of<TC3>(stage);
    case 4: *nt = TC4::NT; *smem = TC4::smem_bytes(); return kernel_of<TC4>(stage);
    default: *nt = TC5::NT; *smem = TC5::smem_bytes(); return kernel_of<TC5>(stage);
  }
}

static void destroy_graphs(rsst_batch* b) {
  for (int p = 0; p < 2; ++p) {
    if (b->graph_ok[p]) cudaGraphExecDestroy(b->graph[p]);
    b->graph_ok[p] = false;
  }
}

// Build the device descriptors (tensor maps, tile list) for candidate c.
static int build_descriptors(rsst_batch* b, int c) {
  auto enc = batch_encoder();
  if (!enc) { rsst_set_error("cuTensorMapEncodeTiled unavailable from the driver"); return RSST_ECUDA; }
  const int bx = CAND_BX[c], by = CAND_BY[c];
  std::vector<BatchRun> host(b->nruns);
  std::vector<int2> info;
  for (int i = 0; i < b->nruns; ++i) {
    rsst_handle* h = b->runs[i];
    BatchRun& br = host[i];
    memset(&br, 0, sizeof br);
    for (int k = 0; k < 2; ++k) {
      const cuuint64_t dims[3] = {(cuuint64_t)h->g.pitch, (cuuint64_t)h->g.py, 4};
      const cuuint64_t strides[2] = {(cuuint64_t)h->g.pitch * 4, (cuuint64_t)h->g.fstride * 4};
      const cuuint32_t box[3] = {(cuuint32_t)(bx + 8), (cuuint32_t)(by + 4), 4};
      const cuuint32_t estr[3] = {1, 1, 1};
      const CUresult r = enc(&br.tmap[k], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, h->buf[k], dims, strides, box, estr,
                             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      if (r != CUDA_SUCCESS) { rsst_set_error("cuTensorMapEncodeTiled failed (%d) for run %d", (int)r, i); return RSST_ECUDA; }
      br.buf[k] = (float*)h->buf[k];
    }
    for (int st = 0; st < 2; ++st) {
      TileRun& r = br.r[st];
      r.g = h->g;
      r.p = h->p;
      r.pf = h->pf;
      r.tabr = h->d_tabr;
      r.tab_len = h->bg_len;
      r.flag = h->d_flag;
      r.stall_ns = h->stall_ns;
      r.stage = st + 1;
      r.base = st == 1 ? br.buf[0] : nullptr;  // stage 2 combines with U^n in place
      r.out = st == 1 ? br.buf[0] : br.buf[1];
    }
    br.scal = h->d_scal;
    br.tiles_x = (h->g.n[0] + bx - 1) / bx;
    br.vert = h->d_tab ? 1 : -1;
    const int ntiles = br.tiles_x * ((h->g.n[1] + by - 1) / by);
    for (int k = 0; k < ntiles; ++k) info.push_back(make_int2(i, k));
  }
  const int total = (int)info.size();
  cudaFree(b->d_tile_info);
  b->d_tile_info = nullptr;
  if (cudaMalloc((void**)&b->d_tile_info, sizeof(int2) * info.size()) != cudaSuccess) {
    cudaGetLastError();
    rsst_set_error("rsst_batch: tile list allocation failed");
    return RSST_ENOMEM;
  }
  if (cudaMemcpy(b->d_runs, host.data(), sizeof(BatchRun) * b->nruns, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(b->d_tile_info, info.data(), sizeof(int2) * info.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
    rsst_set_error("batch descriptor upload failed");
    return RSST_ECUDA;
  }
  int nt;
  size_t smem;
  void* k = cand_kernel(c, &nt, &smem, 2);
  if (cudaFuncSetAttribute(cand_kernel(c, &nt, &smem, 1), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
          cudaSuccess ||
      cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
    rsst_set_error("cudaFuncSetAttribute failed for the batch kernel");
    return RSST_ECUDA;
  }
  int per_sm = 0, dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) {
    cudaGetLastError();
    rsst_set_error("rsst_batch: cannot query the device's SM count");
    return RSST_ECUDA;
  }
  int per_sm1 = 0;  // the grid must be resident for both stage kernels
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, nt, smem) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm1, cand_kernel(c, &nt, &smem, 1), nt, smem) != cudaSuccess) {
    cudaGetLastError();
    per_sm = 1;
  }
  if (per_sm1 < per_sm) per_sm = per_sm1;
  if (per_sm < 1) per_sm = 1;
  b->grid = sms * per_sm < total ? sms * per_sm : total;
  if (b->grid < 1) b->grid = 1;
  b->total_tiles = total;
  b->choice = c;
  destroy_graphs(b);
  return RSST_OK;
}

static int launch_stage(rsst_batch* b, int stage, int slot) {
  int nt;
  size_t smem;
  cand_kernel(b->choice, &nt, &smem);
#define RSST_BATCH_LAUNCH(C)                                                                              \
  if (stage == 1)                                                                                         \
    batch_stage_kernel<C, 1><<<b->grid, nt, smem, b->stream>>>(b->d_runs, b->d_tile_info, b->total_tiles, \
                                                               slot);                                     \
  else                                                                                                    \
    batch_stage_kernel<C, 2><<<b->grid, nt, smem, b->stream>>>(b->d_runs, b->d_tile_info, b->total_tiles, \
                                                               slot);
  switch (b->choice) {
    case 0: RSST_BATCH_LAUNCH(TC0) break;
    case 1: RSST_BATCH_LAUNCH(TC1) break;
    case 2: RSST_BATCH_LAUNCH(TC2) break;
    case 3: RSST_BATCH_LAUNCH(TC3) break;
    case 4: RSST_BATCH_LAUNCH(TC4) break;
    default: RSST_BATCH_LAUNCH(TC5) break;
  }
#undef RSST_BATCH_LAUNCH
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    rsst_set_error("batch stage launch: %s", cudaGetErrorString(e));
    return RSST_ECUDA;
  }
  return RSST_OK;
}

static int capture_graphs(rsst_batch* b) {
  for (int p = 0; p < 2; ++p) {
    if (b->graph_ok[p]) continue;
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      rsst_set_error("cudaStreamBeginCapture failed (the batch stream must be a created stream)");
      return RSST_ECUDA;
    }
    int rc = launch_stage(b, 1, p);
    if (rc == RSST_OK) rc = launch_stage(b, 2, p);
    const cudaError_t e = cudaStreamEndCapture(b->stream, &g);
    if (rc != RSST_OK) {
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    if (e != cudaSuccess || cudaGraphInstantiate(&b->graph[p], g, 0) != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      rsst_set_error("graph capture of the batch step failed");
      return RSST_ECUDA;
    }
    cudaGraphDestroy(g);
    b->graph_ok[p] = true;
  }
  return RSST_OK;
}

extern "C" void rsst_batch_destroy(rsst_batch* b) {
  if (!b) return;
  destroy_graphs(b);
  for (rsst_handle* h : b->runs) rsst_destroy(h);
  cudaFree(b->d_runs);
  cudaFree(b->d_tile_info);
  delete b;
}

extern "C" int rsst_batch_init(rsst_batch** out, int32_t nruns, const rsst_config* cfgs, void* stream) {
  if (!out || !cfgs || nruns < 1) { rsst_set_error("rsst_batch_init: bad arguments"); return RSST_EINVAL; }
  *out = nullptr;
  for (int i = 0; i < nruns; ++i) {
    const rsst_config& c = cfgs[i];
    if (c.ndim != 2 || c.precision != RSST_FP32_PERT || !(c.vertical == -1 || c.vertical == 1)) {
      rsst_set_error("rsst_batch_init: run %d must be 2D, RSST_FP32_PERT, vertical axis y or none", i);
      return RSST_EUNSUPPORTED;
    }
  }
  rsst_batch* b = new rsst_batch();
  b->nruns = nruns;
  b->stream = (cudaStream_t)stream;
  b->d_runs = nullptr;
  b->d_tile_info = nullptr;
  b->slot = 0;
  b->launches = 0;
  b->graph_ok[0] = b->graph_ok[1] = false;
  for (int i = 0; i < nruns; ++i) {
    rsst_handle* h = nullptr;
    const int rc = rsst_init(&h, &cfgs[i], stream);
    if (rc != RSST_OK) {
      rsst_batch_destroy(b);
      return rc;
    }
    b->runs.push_back(h);
  }
  if (cudaMalloc((void**)&b->d_runs, sizeof(BatchRun) * nruns) != cudaSuccess) {
    cudaGetLastError();
    rsst_set_error("rsst_batch_init: descriptor allocation failed");
    rsst_batch_destroy(b);
    return RSST_ENOMEM;
  }
  const int rc = build_descriptors(b, 0);
  if (rc != RSST_OK) {
    rsst_batch_destroy(b);
    return rc;
  }
  *out = b;
  return RSST_OK;
}

extern "C" int rsst_batch_set_state(rsst_batch* b, int32_t run, const double* U, int on_host) {
  if (!b || run < 0 || run >= b->nruns) { rsst_set_error("rsst_batch_set_state: bad run index"); return RSST_EINVAL; }
  b->runs[run]->slot = b->slot;
  return rsst_set_state(b->runs[run], U, on_host);
}

extern "C" int rsst_batch_get_state(rsst_batch* b, int32_t run, double* U, int on_host) {
  if (!b || run < 0 || run >= b->nruns) { rsst_set_error("rsst_batch_get_state: bad run index"); return RSST_EINVAL; }
  return rsst_get_state(b->runs[run], U, on_host);
}

static void sync_slots(rsst_batch* b) {
  for (rsst_handle* h : b->runs) h->slot = b->slot;
}

extern "C" int rsst_batch_step(rsst_batch* b, int nsteps) {
  if (!b || nsteps < 0) { rsst_set_error("rsst_batch_step: bad arguments"); return RSST_EINVAL; }
  if (nsteps == 0) return RSST_OK;
  const int rc = capture_graphs(b);
  if (rc != RSST_OK) return rc;
  for (int s = 0; s < nsteps; ++s) {
    const cudaError_t e = cudaGraphLaunch(b->graph[b->slot], b->stream);
    if (e != cudaSuccess) {
      rsst_set_error("batch graph launch: %s", cudaGetErrorString(e));
      return RSST_ECUDA;
    }
    b->slot ^= 1;
    b->launches += 2;
  }
  sync_slots(b);
  return RSST_OK;
}

extern "C" int rsst_batch_step_looped(rsst_batch* b, int nsteps) {
  if (!b || nsteps < 0) { rsst_set_error("rsst_batch_step_looped: bad arguments"); return RSST_EINVAL; }
  for (int s = 0; s < nsteps; ++s) {
    for (rsst_handle* h : b->runs) {
      h->slot = b->slot;
      const int rc = rsst_handle_steps(h, 0.0, 1);
      if (rc != RSST_OK) return rc;
      b->launches += 2;
    }
    b->slot ^= 1;
  }
  sync_slots(b);
  return RSST_OK;
}

extern "C" int rsst_batch_dt(rsst_batch* b, double* dts) {
  if (!b || !dts) { rsst_set_error("rsst_batch_dt: NULL argument"); return RSST_EINVAL; }
  for (int i = 0; i < b->nruns; ++i) {
    const int rc = rsst_dt(b->runs[i], &dts[i]);
    if (rc != RSST_OK) return rc;
  }
  return RSST_OK;
}

extern "C" int rsst_batch_sync(rsst_batch* b) {
  if (!b) { rsst_set_error("NULL batch"); return RSST_EINVAL; }
  // Every run is checked; a timeout is reported before a non-physical state
  // (a run whose stage gave up may hold a partly written state).
  int worst = RSST_OK, first_timeout = -1, first_bad = -1, ntimeout = 0, nbad = 0;
  for (int i = 0; i < b->nruns; ++i) {
    unsigned int f = 0;
    const int rc = rsst_read_flag(b->runs[i], &f);
    if (rc != RSST_OK) return rc;
    if (f & RSST_FLAG_TIMEOUT) {
      if (first_timeout < 0) first_timeout = i;
      ++ntimeout;
    } else if (f & RSST_FLAG_NONPHYSICAL) {
      if (first_bad < 0) first_bad = i;
      ++nbad;
    }
  }
  if (ntimeout) {
    rsst_set_error("a bounded device wait gave up in %d run(s), first run %d: their states are incomplete",
                   ntimeout, first_timeout);
    worst = RSST_ETIMEOUT;
  } else if (nbad) {
    rsst_set_error("non-physical state (rho <= 0, P <= 0 or NaN) produced in %d run(s), first run %d", nbad,
                   first_bad);
    worst = RSST_ENONPHYSICAL;
  }
  return worst;
}

extern "C" int rsst_batch_debug_stall_wait(rsst_batch* b, int32_t run, int64_t limit_ns) {
  if (!b || run < 0 || run >= b->nruns || limit_ns < 0 || limit_ns > 1000000000LL) {
    rsst_set_error("rsst_batch_debug_stall_wait: need a batch, a run index and 0 <= limit_ns <= 1e9");
    return RSST_EINVAL;
  }
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) {  // no step may read the descriptors meanwhile
    rsst_set_error("rsst_batch_debug_stall_wait: %s", cudaGetErrorString(cudaGetLastError()));
    return RSST_ECUDA;
  }
  b->runs[run]->stall_ns = limit_ns;
  return build_descriptors(b, b->choice);  // the descriptors carry the setting; graphs are recaptured
}

extern "C" int rsst_batch_tile_shape(const rsst_batch* b, int32_t* bx, int32_t* by) {
  if (!b || !bx || !by) { rsst_set_error("NULL argument"); return RSST_EINVAL; }
  *bx = CAND_BX[b->choice];
  *by = CAND_BY[b->choice];
  return RSST_OK;
}

extern "C" int64_t rsst_batch_kernel_launches(const rsst_batch* b) { return b ? b->launches : 0; }

static std::string batch_signature(const rsst_batch* b) {
  std::string s = "n" + std::to_string(b->nruns);
  for (rsst_handle* h : b->runs)
    s += ":" + std::to_string(h->g.n[0]) + "x" + std::to_string(h->g.n[1]) + (h->d_tab ? "b" : "p");
  unsigned long long hsh = 1469598103934665603ull;  // FNV-1a of the run list
  for (char c : s) hsh = (hsh ^ (unsigned char)c) * 1099511628211ull;
  char buf[32];
  snprintf(buf, sizeof buf, "%016llx", hsh);
  return buf;
}

extern "C" int rsst_batch_autotune(rsst_batch* b, int steps, int32_t* choice_out, double* ms_out) {
  if (!b || steps < 1) { rsst_set_error("rsst_batch_autotune: bad arguments"); return RSST_EINVAL; }
  const std::string sig = batch_signature(b);
  const char* cache = getenv("RSST_TUNE_CACHE");
  if (cache) {
    FILE* f = fopen(cache, "r");
    if (f) {
      char key[64];
      int c;
      while (fscanf(f, "%63s %d", key, &c) == 2) {
        if (sig == key && c >= 0 && c < NCAND) {
          fclose(f);
          const int rc = build_descriptors(b, c);
          if (choice_out) *choice_out = c;
          return rc;
        }
      }
      fclose(f);
    }
  }
  // save every run's state and scalars, time each candidate, restore
  std::vector<void*> save(b->nruns, nullptr);
  std::vector<double*> ssave(b->nruns, nullptr);
  int rc = RSST_OK;
  auto ck = [&rc](cudaError_t e, const char* what) {
    if (e != cudaSuccess && rc == RSST_OK) {
      rsst_set_error("rsst_batch_autotune: %s: %s", what, cudaGetErrorString(e));
      rc = RSST_ECUDA;
    }
  };
  for (int i = 0; i < b->nruns && rc == RSST_OK; ++i) {
    rsst_handle* h = b->runs[i];
    const size_t bytes = (size_t)(h->g.ndim + 2) * h->g.fstride * h->elem;
    if (cudaMalloc(&save[i], bytes) != cudaSuccess || cudaMalloc((void**)&ssave[i], 16 * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      rsst_set_error("rsst_batch_autotune: backup allocation failed");
      rc = RSST_ENOMEM;
      break;
    }
    ck(cudaMemcpyAsync(save[i], h->buf[0], bytes, cudaMemcpyDeviceToDevice, b->stream), "state backup");
    ck(cudaMemcpyAsync(ssave[i], h->d_scal, 16 * sizeof(double), cudaMemcpyDeviceToDevice, b->stream), "scalar backup");
  }
  const int slot0 = b->slot;
  double best_ms = 1e30;
  int best = 0;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  ck(cudaEventCreate(&e0), "event");
  ck(cudaEventCreate(&e1), "event");
  for (int c = 0; c < NCAND && rc == RSST_OK; ++c) {
    int rt = build_descriptors(b, c);
    if (rt == RSST_OK) {
      b->slot = slot0;
      rt = rsst_batch_step(b, 1);  // warm-up (and graph capture)
    }
    if (rt == RSST_OK) {
      ck(cudaEventRecord(e0, b->stream), "event record");
      rt = rsst_batch_step(b, steps);
      ck(cudaEventRecord(e1, b->stream), "event record");
      ck(cudaEventSynchronize(e1), "event wait");
      float ms = 0.0f;
      ck(cudaEventElapsedTime(&ms, e0, e1), "event time");
      if (rt == RSST_OK && rc == RSST_OK && ms < best_ms) {
        best_ms = ms;
        best = c;
      }
    }
    if (rt != RSST_OK && rc == RSST_OK) rc = rt;
    for (int i = 0; i < b->nruns; ++i) {  // restore, also after a failed trial
      rsst_handle* h = b->runs[i];
      const size_t bytes = (size_t)(h->g.ndim + 2) * h->g.fstride * h->elem;
      ck(cudaMemcpyAsync(h->buf[0], save[i], bytes, cudaMemcpyDeviceToDevice, b->stream), "state restore");
      ck(cudaMemcpyAsync(h->d_scal, ssave[i], 16 * sizeof(double), cudaMemcpyDeviceToDevice, b->stream), "scalar restore");
    }
  }
  ck(cudaStreamSynchronize(b->stream), "stream wait");
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  for (int i = 0; i < b->nruns; ++i) {
    cudaFree(save[i]);
    cudaFree(ssave[i]);
  }
  b->slot = slot0;
  sync_slots(b);
  if (rc != RSST_OK) return rc;
  rc = build_descriptors(b, best);
  if (rc != RSST_OK) return rc;
  if (choice_out) *choice_out = best;
  if (ms_out) *ms_out = best_ms / steps;
  if (cache) {
    FILE* f = fopen(cache, "a");
    if (f) {
      fprintf(f, "%s %d\n", sig.c_str(), best);
      fclose(f);
    }
  }
  return RSST_OK;
}
