// lsq_apply_normal_noalloc: the fused A^T (A z) pass for callers that must
// not allocate device memory.
//
// Who needs it: code that runs where cudaMalloc is off limits -- a host
// framework that owns all device memory through its own pool and forbids
// raw allocations, a latency-critical loop where cudaMalloc's implicit
// device synchronisation (or a possible out-of-memory failure) cannot be
// tolerated, or a library called from such code.  The plan-based entry
// points allocate their workspace in lsq_plan_create; this one needs no
// plan.
//
// How: the per-CTA partial sums of the pass live in a file-scope device
// array of fixed size (kNoAllocScratchBytes).  Every GPU that loads the
// library holds this array until the process exits.  Host code cannot use
// the array's name as a device address, so the first call on each device
// looks the address up with cudaGetSymbolAddress (with that device
// current) and caches it; make that first call before any stream capture.
// All calls on a device share the array: calls that overlap on the GPU (for
// example on two streams) race on it.  Each call overwrites every slot it
// reads, so nothing has to be cleared between calls.
#include <mutex>
#include <string>

#include "lsq_common.cuh"

namespace lsq {

namespace {

constexpr size_t kNoAllocScratchBytes = 2u << 20;  // 2 MiB per device
constexpr size_t kNoAllocScratchDoubles = kNoAllocScratchBytes / sizeof(double);
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchDoubles];

std::mutex g_noalloc_mu;
double *g_noalloc_ptr[kMaxDevices] = {};

lsq_status noalloc_fail(lsq_status st, const std::string &msg) {
  set_last_error(msg.c_str());
  return st;
}

}  // namespace

}  // namespace lsq

using namespace lsq;

extern "C" lsq_status lsq_apply_normal_noalloc(const double *dA, int64_t m, int64_t n, int64_t lda,
                                               const double *dz, double *dh, void *cuda_stream) {
  if (!dA || !dz || !dh) return noalloc_fail(LSQ_ERR_INVALID, "NULL argument");
  if (n < 1 || m < 1) return noalloc_fail(LSQ_ERR_INVALID, "need m >= 1 and n >= 1");
  if (lda == 0) lda = n;
  if (lda < n) return noalloc_fail(LSQ_ERR_INVALID, "lda < n");
  if (n > LSQ_MAX_N)
    return noalloc_fail(LSQ_ERR_INVALID, "n exceeds LSQ_MAX_N (1024) for the no-allocation pass");
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return noalloc_fail(LSQ_ERR_CUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return noalloc_fail(LSQ_ERR_INVALID, "device index out of range");
  double *scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
      void *p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess)
        return noalloc_fail(LSQ_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      g_noalloc_ptr[dev] = static_cast<double *>(p);
    }
    scratch = g_noalloc_ptr[dev];
  }
  const int npad = pass_npad((int)n);
  // one partial n-vector per CTA; as many CTAs as the scratch holds, at most 2 per SM
  int grid = nsm * kPassCtasPerSm;
  const int cap = (int)(kNoAllocScratchDoubles / (size_t)npad);
  if (grid > cap) grid = cap;
  if (grid < 1) return noalloc_fail(LSQ_ERR_INVALID, "scratch too small for n");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  e = launch_pass_atax(dA, lda, m, (int)n, dz, scratch, grid, npad, nullptr, s);
  if (e == cudaSuccess)
    e = launch_reduce(scratch, grid, npad, (int)n, nullptr, dh, nullptr, nullptr, nullptr, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return noalloc_fail(LSQ_ERR_CUDA, cudaGetErrorString(e));
  return LSQ_OK;
}
