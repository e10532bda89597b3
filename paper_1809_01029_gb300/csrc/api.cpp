// C-ABI evaluation entry points: argument validation and dispatch to the
// kernels in kinetics.cu.  No host synchronisation, no allocation.
#include <cuda_runtime.h>

#include <cstring>
#include <string>

#include "launch.h"
#include "pj_internal.h"

namespace pj {

int check_common(const char* fn, const pj_mech* m, int mode, int64_t n, int64_t ld, const void* param,
                 const void* phi, const void* out) {
  const std::string f(fn);
  if (!m) return fail(PJ_ERR_ARG, f + ": null mechanism");
  if (mode != PJ_CONP && mode != PJ_CONV) return fail(PJ_ERR_ARG, f + ": mode must be PJ_CONP or PJ_CONV");
  if (n < 0) return fail(PJ_ERR_ARG, f + ": n < 0");
  if (ld < n || ld < 1) return fail(PJ_ERR_ARG, f + ": ld must be >= max(n, 1)");
  if (n > 0 && (!param || !phi || !out)) return fail(PJ_ERR_ARG, f + ": null buffer");
  if (m->device < 0) return fail(PJ_ERR_CUDA, f + ": mechanism has no device copy (no CUDA device at creation)");
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return check_cuda(e, "cudaGetDevice");
  if (dev != m->device)
    return fail(PJ_ERR_ARG, f + ": current device " + std::to_string(dev) + " differs from the mechanism's device " +
                                std::to_string(m->device));
  return PJ_OK;
}
}  // namespace pj

using namespace pj;

extern "C" int pj_workspace_size(const pj_mech* m, int op, int64_t n, size_t* bytes) {
  if (!m || !bytes) return fail(PJ_ERR_ARG, "pj_workspace_size: null argument");
  if (n < 0) return fail(PJ_ERR_ARG, "pj_workspace_size: n < 0");
  switch (op) {
    case PJ_OP_SOURCE: *bytes = workspace_bytes(source_arrays(), m->ns, n); return PJ_OK;
    case PJ_OP_JACOBIAN:
    case PJ_OP_NEWTON: *bytes = workspace_bytes(jacobian_arrays(), m->ns, n); return PJ_OK;
    case PJ_OP_VJP:
    case PJ_OP_Y: *bytes = form_workspace_bytes(op, m->dm, n); return PJ_OK;
    case PJ_OP_FD: *bytes = fd_workspace_bytes(m->ns, n); return PJ_OK;
    case PJ_OP_LU: *bytes = lu_workspace_bytes(m->ns + 1, PJ_F64, n); return PJ_OK;
    default: return fail(PJ_ERR_ARG, "pj_workspace_size: unknown op");
  }
}

extern "C" int pj_debug_word(const pj_mech* m, uint32_t* h_word, int clear) {
  if (!m || !h_word) return fail(PJ_ERR_ARG, "pj_debug_word: null argument");
  if (m->device < 0 || !m->dm.dbg) return fail(PJ_ERR_CUDA, "pj_debug_word: mechanism has no device copy");
  int rc;
  if ((rc = check_cuda(cudaMemcpy(h_word, m->dm.dbg, sizeof(uint32_t), cudaMemcpyDeviceToHost),
                       "cudaMemcpy(debug word)")))
    return rc;
  if (clear) return check_cuda(cudaMemset(m->dm.dbg, 0, sizeof(uint32_t)), "cudaMemset(debug word)");
  return PJ_OK;
}

extern "C" int pj_debug_build(int32_t* on) {
  if (!on) return fail(PJ_ERR_ARG, "pj_debug_build: null argument");
#ifdef PJ_DEBUG_BOUNDS
  *on = 1;
#else
  *on = 0;
#endif
  return PJ_OK;
}

extern "C" int pj_debug_set_target(const pj_mech* m, int fmt, int32_t index, int32_t value) {
#ifdef PJ_DEBUG_BOUNDS
  if (!m) return fail(PJ_ERR_ARG, "pj_debug_set_target: null mechanism");
  if (fmt != PJ_CSR && fmt != PJ_CSC) return fail(PJ_ERR_ARG, "pj_debug_set_target: fmt must be PJ_CSR or PJ_CSC");
  if (m->device < 0) return fail(PJ_ERR_CUDA, "pj_debug_set_target: mechanism has no device copy");
  if (index < 0 || index >= m->dm.n_tgt) return fail(PJ_ERR_ARG, "pj_debug_set_target: index out of range");
  int32_t* p = const_cast<int32_t*>(fmt == PJ_CSR ? m->dm.tgt_csr : m->dm.tgt_csc) + index;
  return check_cuda(cudaMemcpy(p, &value, sizeof value, cudaMemcpyHostToDevice), "cudaMemcpy(target entry)");
#else
  (void)m;
  (void)fmt;
  (void)index;
  (void)value;
  return fail(PJ_ERR_UNSUPPORTED, "pj_debug_set_target: only in the bounds-checked build (PJ_DEBUG_BOUNDS)");
#endif
}

extern "C" int pj_jacobian_layout(const pj_mech* m, int fmt, int prec, int64_t n, int32_t* layout) {
  if (!m || !layout) return fail(PJ_ERR_ARG, "pj_jacobian_layout: null argument");
  if (n < 0) return fail(PJ_ERR_ARG, "pj_jacobian_layout: n < 0");
  if (fmt != PJ_CSR && fmt != PJ_CSC && fmt != PJ_DENSE)
    return fail(PJ_ERR_ARG, "pj_jacobian_layout: fmt must be PJ_CSR, PJ_CSC or PJ_DENSE");
  if (prec != PJ_F64 && prec != PJ_F32) return fail(PJ_ERR_ARG, "pj_jacobian_layout: prec must be PJ_F64 or PJ_F32");
  if (m->device < 0) return fail(PJ_ERR_CUDA, "pj_jacobian_layout: mechanism has no device copy");
  *layout = jacobian_layout(m->dm, fmt, prec == PJ_F32, n);
  return PJ_OK;
}

extern "C" int pj_eval_source_terms(const pj_mech* m, int mode, int64_t n, const double* param, const double* phi,
                                    int64_t ld, double* dphi, int* status, void* work, size_t work_bytes,
                                    void* stream) {
  int rc = check_common("pj_eval_source_terms", m, mode, n, ld, param, phi, dphi);
  if (rc) return rc;
  if (n == 0) return PJ_OK;
  return launch_source(m->dm, mode, n, param, phi, ld, dphi, status, work, work_bytes, (cudaStream_t)stream);
}

extern "C" int pj_eval_jacobian_sparse(const pj_mech* m, int mode, int fmt, int64_t n, const double* param,
                                       const double* phi, int64_t ld, double* vals, double* dphi, int* status,
                                       void* work, size_t work_bytes, void* stream) {
  if (fmt != PJ_CSR && fmt != PJ_CSC) return fail(PJ_ERR_ARG, "pj_eval_jacobian_sparse: fmt must be PJ_CSR or PJ_CSC");
  int rc = check_common("pj_eval_jacobian_sparse", m, mode, n, ld, param, phi, vals);
  if (rc) return rc;
  if (n > 0 && !dphi) return fail(PJ_ERR_ARG, "pj_eval_jacobian_sparse: d_dphi is required");
  if (n == 0) return PJ_OK;
  return launch_jacobian(m->dm, mode, fmt, n, param, phi, ld, vals, dphi, status, work, work_bytes,
                         (cudaStream_t)stream);
}

extern "C" int pj_eval_jacobian_fd(const pj_mech* m, int mode, int fmt, int64_t n, const double* param,
                                   const double* phi, int64_t ld, double* vals, double* dphi, int* status,
                                   void* work, size_t work_bytes, void* stream) {
  if (fmt != PJ_CSR && fmt != PJ_CSC && fmt != PJ_DENSE)
    return fail(PJ_ERR_ARG, "pj_eval_jacobian_fd: fmt must be PJ_CSR, PJ_CSC or PJ_DENSE");
  int rc = check_common("pj_eval_jacobian_fd", m, mode, n, ld, param, phi, vals);
  if (rc) return rc;
  if (n > 0 && !dphi) return fail(PJ_ERR_ARG, "pj_eval_jacobian_fd: d_dphi is required");
  if (n == 0) return PJ_OK;
  return launch_fd_jacobian(m->dm, mode, fmt, n, param, phi, ld, vals, dphi, status, work, work_bytes,
                            (cudaStream_t)stream);
}

extern "C" int pj_eval_jacobian_dense(const pj_mech* m, int mode, int64_t n, const double* param, const double* phi,
                                      int64_t ld, double* jac, double* dphi, int* status, void* work,
                                      size_t work_bytes, void* stream) {
  int rc = check_common("pj_eval_jacobian_dense", m, mode, n, ld, param, phi, jac);
  if (rc) return rc;
  if (n > 0 && !dphi) return fail(PJ_ERR_ARG, "pj_eval_jacobian_dense: d_dphi is required");
  if (n == 0) return PJ_OK;
  return launch_jacobian(m->dm, mode, PJ_DENSE, n, param, phi, ld, jac, dphi, status, work, work_bytes,
                         (cudaStream_t)stream);
}

extern "C" int pj_newton_matrix_f32(const pj_mech* m, int mode, int fmt, int64_t n, const double* param,
                                    const double* phi, int64_t ld, const double* h, double gamma, float* M,
                                    double* dphi, int* status, void* work, size_t work_bytes, void* stream) {
  if (fmt != PJ_CSR && fmt != PJ_CSC && fmt != PJ_DENSE)
    return fail(PJ_ERR_ARG, "pj_newton_matrix_f32: fmt must be PJ_CSR, PJ_CSC or PJ_DENSE");
  int rc = check_common("pj_newton_matrix_f32", m, mode, n, ld, param, phi, M);
  if (rc) return rc;
  if (n > 0 && (!dphi || !h)) return fail(PJ_ERR_ARG, "pj_newton_matrix_f32: d_h and d_dphi are required");
  if (!(gamma == gamma)) return fail(PJ_ERR_ARG, "pj_newton_matrix_f32: gamma is NaN");
  if (n == 0) return PJ_OK;
  return launch_newton_f32(m->dm, mode, fmt, n, param, phi, ld, h, gamma, M, dphi, status, work, work_bytes,
                           (cudaStream_t)stream);
}

extern "C" int pj_eval_y(const pj_mech* m, int mode, int64_t n, const double* param, const double* phi, int64_t ld,
                         double* y, int* status, void* work, size_t work_bytes, void* stream) {
  int rc = check_common("pj_eval_y", m, mode, n, ld, param, phi, y);
  if (rc) return rc;
  if (n == 0) return PJ_OK;
  return launch_eval_y(m->dm, mode, n, param, phi, ld, y, status, work, work_bytes, (cudaStream_t)stream);
}

extern "C" int pj_vjp(const pj_mech* m, int mode, int64_t n, const double* param, const double* phi, int64_t ld,
                      const double* u_wdot, const double* u_T, double* y, double* g_phi, double* g_theta,
                      int* status, void* work, size_t work_bytes, void* stream) {
  int rc = check_common("pj_vjp", m, mode, n, ld, param, phi, g_phi);
  if (rc) return rc;
  if (n > 0 && (!u_wdot || !u_T || !y)) return fail(PJ_ERR_ARG, "pj_vjp: d_u_wdot, d_u_T and d_y are required");
  if (!g_theta) return fail(PJ_ERR_ARG, "pj_vjp: d_g_theta is required");
  if (n == 0) return cudaMemsetAsync(g_theta, 0, sizeof(double) * 3 * (size_t)m->nr, (cudaStream_t)stream) == cudaSuccess
                         ? PJ_OK : fail(PJ_ERR_CUDA, "pj_vjp: cudaMemsetAsync failed");
  return launch_vjp(m->dm, mode, n, param, phi, ld, u_wdot, u_T, y, g_phi, g_theta, status, work, work_bytes,
                    (cudaStream_t)stream);
}

extern "C" int pj_diag_exp(const pj_mech* m, int64_t n, const double* x, double* y_ours, double* y_lib,
                           void* stream) {
  int rc = check_common("pj_diag_exp", m, PJ_CONP, n, n > 0 ? n : 1, x, x, y_ours);
  if (rc) return rc;
  if (n > 0 && !y_lib) return fail(PJ_ERR_ARG, "pj_diag_exp: null buffer");
  if (n == 0) return PJ_OK;
  return launch_diag_exp(m->dm, n, x, y_ours, y_lib, (cudaStream_t)stream);
}

extern "C" int pj_lu_info(const pj_mech* m, int32_t* lu_nnz, int32_t* perm) {
  if (!m || !lu_nnz) return fail(PJ_ERR_ARG, "pj_lu_info: null argument");
  *lu_nnz = (int32_t)m->lu_rows.size();
  if (perm) std::memcpy(perm, m->lu_perm.data(), m->lu_perm.size() * sizeof(int32_t));
  return PJ_OK;
}

extern "C" int pj_lu_pattern(const pj_mech* m, int32_t* rows, int32_t* cols) {
  if (!m || !rows || !cols) return fail(PJ_ERR_ARG, "pj_lu_pattern: null argument");
  std::memcpy(rows, m->lu_rows.data(), m->lu_rows.size() * sizeof(int32_t));
  std::memcpy(cols, m->lu_cols.data(), m->lu_cols.size() * sizeof(int32_t));
  return PJ_OK;
}

extern "C" int pj_lu_factor(const pj_mech* m, int prec, int64_t n, const void* vals, int64_t ld, const double* h,
                            double gamma, void* lu, int* status, void* work, size_t work_bytes, void* stream) {
  if (prec != PJ_F64 && prec != PJ_F32) return fail(PJ_ERR_ARG, "pj_lu_factor: prec must be PJ_F64 or PJ_F32");
  int rc = check_common("pj_lu_factor", m, PJ_CONP, n, ld, vals, vals, lu);
  if (rc) return rc;
  if (n == 0) return PJ_OK;
  return launch_lu_factor(m->lu, prec, n, vals, ld, h, gamma, lu, status, work, work_bytes, (cudaStream_t)stream);
}

extern "C" int pj_lu_solve(const pj_mech* m, int prec, int64_t n, const void* lu, int64_t ld, const void* b,
                           void* x, void* stream) {
  if (prec != PJ_F64 && prec != PJ_F32) return fail(PJ_ERR_ARG, "pj_lu_solve: prec must be PJ_F64 or PJ_F32");
  int rc = check_common("pj_lu_solve", m, PJ_CONP, n, ld, lu, b, x);
  if (rc) return rc;
  if (n == 0) return PJ_OK;
  return launch_lu_solve(m->lu, prec, n, lu, ld, b, x, (cudaStream_t)stream);
}
