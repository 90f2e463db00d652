// Allocation-free variant of sofa_lower_bounds.
//
// sofa_lower_bounds keeps its per-call work space (the canonical query series
// and their projected Fourier values) in device buffers that it allocates and
// grows on demand.  Some callers cannot let a library call cudaMalloc at that
// point: a process already at the edge of its device-memory budget, a host
// thread that must not take the driver's allocation locks, a service whose
// memory is handed out by its own pool, or a latency-critical loop that cannot
// absorb the implicit synchronisation an allocation may cause.  This entry
// point serves them: its work space is a fixed array in the library's own
// device image, so the call allocates nothing.
#include <mutex>

#include "sofa_internal.cuh"

namespace sofa {

// Work space of the allocation-free entry point: room for Q x (n + NB) floats
// (query series and projected values), 4 Mi floats = 16 MiB.  It is part of the
// library's device image: every GPU that loads the library holds it until the
// process exits.
constexpr int64_t NOALLOC_FLOATS = (int64_t)1 << 22;
static __device__ __align__(256) float g_noalloc_scratch[NOALLOC_FLOATS];

constexpr int NOALLOC_MAX_DEVICES = 64;
static float* g_noalloc_ptr[NOALLOC_MAX_DEVICES];
static std::mutex g_noalloc_mutex;

// Device address of the work space on device `dev`, which must be the current
// device.  The name of the array is only a host-side stand-in; the address must
// come from the runtime, once per device, with that device current.
static int noalloc_scratch(int dev, float** out) {
  if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return fail(SOFA_ERR_INVALID_ARG, "device index out of range");
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return fail(SOFA_ERR_CUDA, std::string("cudaGetSymbolAddress of the work space failed: ") +
                                     cudaGetErrorString(e));
    g_noalloc_ptr[dev] = static_cast<float*>(p);
  }
  *out = g_noalloc_ptr[dev];
  return 0;
}

}  // namespace sofa

using namespace sofa;

extern "C" int sofa_lower_bounds_noalloc(sofa_handle h, const float* queries, int64_t Q, float* out,
                                         sofa_stream stream) {
  if (!h || !queries || !out) return fail(SOFA_ERR_INVALID_ARG, "null argument");
  if (Q < 0) return fail(SOFA_ERR_INVALID_ARG, "Q must be >= 0");
  if (Q == 0) return 0;
  const int64_t per_query = (int64_t)h->n + h->NB;
  if (Q > NOALLOC_FLOATS / per_query)
    return fail(SOFA_ERR_INVALID_ARG, "Q = " + std::to_string(Q) + " exceeds the allocation-free work space: at most " +
                                          std::to_string(NOALLOC_FLOATS / per_query) + " queries of length " +
                                          std::to_string(h->n) + " per call");
  if (!is_device_ptr(queries)) return fail(SOFA_ERR_INVALID_ARG, "queries must be device memory");
  if (!is_device_ptr(out)) return fail(SOFA_ERR_INVALID_ARG, "out must be device memory");
  // the work space is looked up for the current device, and the index's
  // buffers live on the device it was built on: the two must agree, or the
  // kernels would mix addresses of two GPUs
  if (int rc = check_device(h)) return rc;
  float* ws = nullptr;
  if (int rc = noalloc_scratch(h->device, &ws)) return rc;
  // Every entry the kernels read is written first in this call (series, then
  // values), so nothing needs clearing between calls.
  float* zq = ws;
  float* qv = ws + Q * h->n;
  cudaStream_t st = (cudaStream_t)stream;
  if (int rc = launch_qprep(h, queries, Q, zq, qv, st)) return rc;
  return launch_lower_bounds(h, qv, Q, out, st);
}
