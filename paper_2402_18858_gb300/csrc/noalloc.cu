// chem_step_di_noalloc: chem_step_di for callers that cannot allocate device memory.
//
// Some callers have no way to hand this library a workspace: a flow solver written in
// Fortran or C that links the C ABI directly and has already given all free HBM to its own
// memory pool, or a time-step loop that must not call cudaMalloc/cudaFree because those calls
// synchronise the device and would stall its other streams.  This entry point takes the same
// inputs and outputs as chem_step_di but keeps its scratch (the cell work-queue counter) in a
// fixed file-scope device array, so it allocates nothing.
//
// The array is part of this library's device image: every GPU that loads the library holds it
// until the process exits.  Host code only knows a stand-in for the array's name, so the
// device address is looked up once per device with cudaGetSymbolAddress (the first call on
// each device does this set-up, with that device current) and passed to the kernel.
#include <cuda_runtime.h>

#include <mutex>

#include "internal.h"

namespace chem {

// Scratch capacity: one 256-byte line, enough for the work-queue counter of any call.
constexpr size_t kNoallocScratchBytes = 256;
static __device__ __align__(256) unsigned int g_noalloc_scratch[kNoallocScratchBytes / sizeof(unsigned int)];

constexpr int kMaxDevices = 64;
static std::mutex g_noalloc_mu;
static void* g_noalloc_addr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device (looked up once per device).
static int noalloc_scratch(void** out) {
  int dev = -1;
  int rc = cuda_check(cudaGetDevice(&dev), "chem_step_di_noalloc: cudaGetDevice");
  if (rc) return rc;
  if (dev < 0 || dev >= kMaxDevices) return set_error(CHEM_E_ARG, "chem_step_di_noalloc: device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    rc = cuda_check(cudaGetSymbolAddress(&p, g_noalloc_scratch), "chem_step_di_noalloc: cudaGetSymbolAddress");
    if (rc) return rc;
    g_noalloc_addr[dev] = p;
  }
  *out = g_noalloc_addr[dev];
  return CHEM_OK;
}

}  // namespace chem

using namespace chem;

extern "C" int chem_step_di_noalloc(chem_mech m, int64_t n, int64_t ld, double dt, double* T,
                                    const double* p, double* Y, const int32_t* idx,
                                    const chem_di_opts* opts, int32_t* status, int32_t* stats,
                                    chem_stream stream) {
  if (n < 0 || ld < n) return set_error(CHEM_E_ARG, "chem_step_di_noalloc: need 0 <= n <= ld");
  const size_t need = chem_workspace_bytes(m, n);
  if (need > kNoallocScratchBytes || n > (int64_t)0x7fffffff)
    return set_error(CHEM_E_ARG, "chem_step_di_noalloc: the call needs more scratch than the fixed "
                                 "256-byte device array holds (at most 2^31-1 cells per call)");
  void* scratch = nullptr;
  int rc = noalloc_scratch(&scratch);
  if (rc) return rc;
  // chem_step_di clears the queue counter on `stream` before its launch, so every call
  // starts from zero even though the array keeps the previous call's contents.
  return chem_step_di(m, n, ld, dt, T, p, Y, idx, opts, status, stats, scratch, kNoallocScratchBytes, stream);
}
