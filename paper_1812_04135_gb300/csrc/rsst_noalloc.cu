// Conservation sums that allocate nothing.
//
// rsst_conserved_sums works on a handle whose scratch (the per-block partial
// sums) was allocated by rsst_init.  Some callers cannot allocate device
// memory at the point where they need the sums: plug-ins living inside
// another framework that owns the whole device-memory budget through its own
// caching allocator, and latency-critical loops that cannot afford
// cudaMalloc's implicit device synchronisation.  This entry
// point serves them: the caller passes the state and the output, and the only
// scratch is the file-scope array below, which every GPU that loads the
// library holds until the process exits.
//
// The reduction is the same fixed-shape tree as rsst_conserved_sums (1024
// contiguous chunks, fixed thread striding, shared-memory tree, then one
// block over the partials in index order), so for the same state both give
// the same result.
#include <mutex>

#include "rsst_internal.h"
#include "rsst_check.h"

#define NOALLOC_BLOCKS 1024
#define NOALLOC_THREADS 256
#define NOALLOC_MAX_FIELDS 5  // nvar of a 3D run
#define NOALLOC_MAX_DEVICES 64

// Scratch: one partial sum per (field, block); 5 x 1024 doubles = 40 KiB.
// Every block overwrites its own entry, so nothing has to start at zero.
static __device__ __align__(256) double g_noalloc_partial[NOALLOC_MAX_FIELDS * NOALLOC_BLOCKS];

static __global__ void __launch_bounds__(NOALLOC_THREADS)
    noalloc_partial_kernel(const double* __restrict__ U, int nv, int64_t ncells, double* __restrict__ partial) {
  __shared__ double sh[NOALLOC_THREADS];
  const int64_t chunk = (ncells + NOALLOC_BLOCKS - 1) / NOALLOC_BLOCKS;
  const int64_t lo = blockIdx.x * chunk;
  const int64_t hi = lo + chunk < ncells ? lo + chunk : ncells;
  for (int v = 0; v < nv; ++v) {
    double acc = 0.0;
    for (int64_t id = lo + threadIdx.x; id < hi; id += NOALLOC_THREADS) acc += U[v * ncells + id];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int s = NOALLOC_THREADS / 2; s > 0; s >>= 1) {
      if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
      __syncthreads();
    }
    if (threadIdx.x == 0) partial[v * NOALLOC_BLOCKS + blockIdx.x] = sh[0];
    __syncthreads();
  }
}

static __global__ void __launch_bounds__(NOALLOC_THREADS)
    noalloc_final_kernel(const double* __restrict__ partial, int nv, double scale, double* __restrict__ out) {
  __shared__ double sh[NOALLOC_THREADS];
  for (int v = 0; v < nv; ++v) {
    double acc = 0.0;
    for (int b = threadIdx.x; b < NOALLOC_BLOCKS; b += NOALLOC_THREADS) acc += partial[v * NOALLOC_BLOCKS + b];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int s = NOALLOC_THREADS / 2; s > 0; s >>= 1) {
      if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
      __syncthreads();
    }
    if (threadIdx.x == 0) out[v] = sh[0] * scale;
    __syncthreads();
  }
}

// Device address of the scratch array on the current device.  In host code
// the name g_noalloc_partial is only a host-side stand-in, so the address is
// looked up once per device (with that device current) and cached.
static int scratch_for_current_device(double** out) {
  static std::mutex mu;
  static double* ptr[NOALLOC_MAX_DEVICES] = {nullptr};
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    rsst_set_error("rsst_conserved_sums_noalloc: cudaGetDevice: %s", cudaGetErrorString(e));
    return RSST_ECUDA;
  }
  if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) {
    rsst_set_error("rsst_conserved_sums_noalloc: device %d beyond the %d supported", dev, NOALLOC_MAX_DEVICES);
    return RSST_EUNSUPPORTED;
  }
  std::lock_guard<std::mutex> lock(mu);
  if (!ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_partial);
    if (e != cudaSuccess || p == nullptr) {
      rsst_set_error("rsst_conserved_sums_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
      return RSST_ECUDA;
    }
    ptr[dev] = static_cast<double*>(p);
  }
  *out = ptr[dev];
  return RSST_OK;
}

extern "C" int rsst_conserved_sums_noalloc(const double* U, int32_t ndim, const int32_t* n, const double* dx,
                                           double* sums, void* stream) {
  if (!U || !n || !dx || !sums) {
    rsst_set_error("rsst_conserved_sums_noalloc: NULL argument");
    return RSST_EINVAL;
  }
  if (rsst_check_buffer(U, 0, "rsst_conserved_sums_noalloc (U)") != RSST_OK ||
      rsst_check_buffer(sums, 0, "rsst_conserved_sums_noalloc (sums)") != RSST_OK)
    return RSST_EINVAL;
  if (ndim < 1 || ndim > 3) {
    rsst_set_error("rsst_conserved_sums_noalloc: ndim must be 1, 2 or 3 (got %d); the scratch holds at most %d fields",
                   ndim, NOALLOC_MAX_FIELDS);
    return RSST_EINVAL;
  }
  int64_t cells = 1;
  double vol = 1.0;
  for (int d = 0; d < ndim; ++d) {
    if (n[d] < 1) {
      rsst_set_error("rsst_conserved_sums_noalloc: n[%d] must be >= 1", d);
      return RSST_EINVAL;
    }
    cells *= n[d];
    vol *= dx[d];
  }
  if (cells > ((int64_t)1 << 31)) {
    rsst_set_error("rsst_conserved_sums_noalloc: %lld cells exceed the maximum of 2^31", (long long)cells);
    return RSST_EINVAL;
  }
  double* scratch = nullptr;
  const int rc = scratch_for_current_device(&scratch);
  if (rc != RSST_OK) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  const int nv = ndim + 2;
  noalloc_partial_kernel<<<NOALLOC_BLOCKS, NOALLOC_THREADS, 0, s>>>(U, nv, cells, scratch);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) {
    noalloc_final_kernel<<<1, NOALLOC_THREADS, 0, s>>>(scratch, nv, vol, sums);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    rsst_set_error("rsst_conserved_sums_noalloc launch: %s", cudaGetErrorString(e));
    return RSST_ECUDA;
  }
  return RSST_OK;
}
