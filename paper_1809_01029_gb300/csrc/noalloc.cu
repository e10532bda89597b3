// Allocation-free sparse Jacobian entry point.
//
// The regular entry points take their scratch (the per-state working arrays
// of large mechanisms) from a caller-provided workspace.  Some callers cannot
// provide one: code that may not call cudaMalloc or any allocating routine
// (for instance a solver inside a region whose device memory is owned and
// fixed by a host application, or host code that is not allowed to touch the
// CUDA allocator at that point).  For them this file keeps the scratch in a
// file-scope device array of fixed size that every GPU loading the library
// holds until the process exits, and exposes one entry point that allocates
// nothing.
#include <cuda_runtime.h>

#include <string>

#include "launch.h"
#include "pj_internal.h"


namespace {

constexpr size_t kScratchBytes = size_t(64) << 20;  // 64 MiB per device

__device__ __align__(256) double g_noalloc_scratch[kScratchBytes / sizeof(double)];

// Device address of the scratch array in the current device's context.  The
// host-side symbol is only a stand-in and must never be passed to a kernel.
// Looked up on every call (the lookup does not allocate): a cached address
// would go stale if the context were reset and the module loaded again.
int scratch_address(double** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess) return pj::check_cuda(e, "cudaGetSymbolAddress(noalloc scratch)");
  *out = static_cast<double*>(p);
  return PJ_OK;
}

}  // namespace

using namespace pj;

extern "C" int pj_eval_jacobian_sparse_noalloc(const pj_mech* m, int mode, int fmt, int64_t n, const double* param,
                                               const double* phi, int64_t ld, double* vals, double* dphi,
                                               int* status, void* stream) {
  const char* fn = "pj_eval_jacobian_sparse_noalloc";
  if (fmt != PJ_CSR && fmt != PJ_CSC) return fail(PJ_ERR_ARG, std::string(fn) + ": fmt must be PJ_CSR or PJ_CSC");
  int rc = check_common(fn, m, mode, n, ld, param, phi, vals);
  if (rc) return rc;
  if (n > 0 && !dphi) return fail(PJ_ERR_ARG, std::string(fn) + ": d_dphi is required");
  if (n == 0) return PJ_OK;
  const size_t per_thread = (size_t)jacobian_arrays() * m->ns * sizeof(double);
  const int64_t threads = (int64_t)(kScratchBytes / per_thread) / 128 * 128;
  if (threads < 128)
    return fail(PJ_ERR_UNSUPPORTED, std::string(fn) + ": mechanism too large for the fixed scratch (" +
                                        std::to_string(per_thread * 128) + " bytes needed per 128 states, " +
                                        std::to_string(kScratchBytes) + " bytes available)");
  double* scratch = nullptr;
  if ((rc = scratch_address(&scratch))) return rc;
  return launch_jacobian_on_scratch(m->dm, mode, fmt, n, param, phi, ld, vals, dphi, status, scratch, threads,
                                    (cudaStream_t)stream);
}
