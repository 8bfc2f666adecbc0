// sgwls_noalloc.cu -- sgwls_filter_pass_noalloc: one SG-WLS pass whose
// scratch lives in a fixed device array owned by this library.
//
// Some callers cannot allocate device memory at the point where they filter:
// code running inside a memory-budgeted host that forbids further
// allocations once it has started, or code that must not call the allocator
// from a latency-critical path.  This entry point lets them run a pass with
// only their input and output buffers.  The scratch (the pass's group
// 2-ports, separator values and merge factors) is a file-scope device array
// of kNoAllocScratchBytes; every GPU that loads the library holds it until
// the process exits.
#include <mutex>

#include "../../include/sgwls.h"
#include "sgwls_common.cuh"

namespace sgwls {
sgwls_status check_pass_params(int H, int W, int C, const sgwls_params* p);
sgwls_status run_pass(const void* in, int in_dt, void* out, int out_dt, const void* g, int H, int W, int C,
                      float lambda, const sgwls_params* p, int dir, void* ws, cudaStream_t st, bool zero_counters);
}

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(16) << 20;   // 16 MiB per device
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_pass_scratch[kNoAllocScratchBytes];

std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of g_pass_scratch on the current device.  The array's name
// in host code is only a host-side stand-in, so the address is looked up
// once per device with that device current.
sgwls_status scratch_for_current_device(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return SGWLS_E_CUDA;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_pass_scratch) != cudaSuccess || !ptr) return SGWLS_E_CUDA;
    g_scratch_ptr[dev] = ptr;
  }
  *out = g_scratch_ptr[dev];
  return SGWLS_OK;
}

}  // namespace

extern "C" sgwls_status sgwls_filter_pass_noalloc(const void* f, const void* g, void* u, int H, int W, int C,
                                                   float lambda, const sgwls_params* p, int direction,
                                                   void* stream) {
  // the caller's parameters are checked exactly as sgwls_filter_pass checks
  // them, so both entry points return the same code for the same mistake
  sgwls_status s = sgwls::check_pass_params(H, W, C, p);
  if (s != SGWLS_OK) return s;
  // kept chunk factors (needed by a sliding step > 1, the refinement and a
  // vector guidance) do not fit this scratch
  if (p->step != 1 || p->refine || p->guide_channels > 1 || p->factor_cache == 1) return SGWLS_E_UNSUPPORTED;
  // u is written while other blocks of the same kernel still read f and g
  if (!f || !g || !u || f == u || g == u) return SGWLS_E_INVALID;
  if (direction != 0 && direction != 1) return SGWLS_E_INVALID;
  if (!(lambda >= 0.f) || !isfinite(lambda)) return SGWLS_E_INVALID;
  // a pass needs no intermediate image: size the scratch as for iters == 0,
  // with the chunk factors recomputed rather than kept
  sgwls_params q = *p;
  q.iters = 0;
  q.factor_cache = 2;
  const size_t need = sgwls_workspace_bytes(H, W, C, &q);
  if (need == 0) return SGWLS_E_INVALID;
  if (need > kNoAllocScratchBytes) return SGWLS_E_WORKSPACE;
  void* ws = nullptr;
  s = scratch_for_current_device(&ws);
  if (s != SGWLS_OK) return s;
  return sgwls::run_pass(f, q.storage, u, q.storage, g, H, W, C, lambda, &q, direction, ws,
                         static_cast<cudaStream_t>(stream), true);
}
