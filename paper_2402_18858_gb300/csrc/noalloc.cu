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
// until the process exits.  Host code only knows a stand-in for the array's name, so every
// call looks up the array's device address in the CUDA context current on the calling thread
// (cudaGetSymbolAddress allocates nothing) and passes it to the kernel.  Looking it up per
// call, rather than caching it per device ordinal, keeps the address right when the caller
// resets the device or makes another context current on it: the module is then loaded again
// and the array may sit at a different address.
#include <cuda_runtime.h>

#include "internal.h"

namespace chem {

// Scratch capacity: one 256-byte line.  The call's only scratch is the 4-byte work-queue
// counter, so the array always suffices; the guard below only protects against a future
// growth of chem_step_di's workspace.
constexpr size_t kNoallocScratchBytes = 256;
static __device__ __align__(256) unsigned int g_noalloc_scratch[kNoallocScratchBytes / sizeof(unsigned int)];

// Device address of the scratch array in the current context.
static int noalloc_scratch(void** out) {
  void* p = nullptr;
  const int rc = cuda_check(cudaGetSymbolAddress(&p, g_noalloc_scratch), "chem_step_di_noalloc: cudaGetSymbolAddress");
  if (rc) return rc;
  *out = p;
  return CHEM_OK;
}

}  // namespace chem

using namespace chem;

extern "C" int chem_step_di_noalloc(chem_mech m, int64_t n, int64_t ld, double dt, double* T,
                                    const double* p, double* Y, const int32_t* idx,
                                    const chem_di_opts* opts, int32_t* status, int32_t* stats,
                                    chem_stream stream) {
  if (n < 0 || ld < n) return set_error(CHEM_E_ARG, "chem_step_di_noalloc: need 0 <= n <= ld");
  // The work-queue counter is 32-bit: at most 2^31 - 1 cells per call (chem_step_di has the
  // same limit).
  if (n > (int64_t)0x7fffffff)
    return set_error(CHEM_E_ARG, "chem_step_di_noalloc: at most 2^31 - 1 cells per call (32-bit work-queue counter)");
  if (chem_workspace_bytes(m, n) > kNoallocScratchBytes)
    return set_error(CHEM_E_ARG, "chem_step_di_noalloc: the call needs more scratch than the fixed 256-byte device array");
  void* scratch = nullptr;
  int rc = noalloc_scratch(&scratch);
  if (rc) return rc;
  // chem_step_di clears the queue counter on `stream` before its launch, so every call
  // starts from zero even though the array keeps the previous call's contents.
  return chem_step_di(m, n, ld, dt, T, p, Y, idx, opts, status, stats, scratch, kNoallocScratchBytes, stream);
}
