// Host-buffer entry point: source terms and the sparse Jacobian of states in
// host memory, with the transfers inside the call.  The batch is cut into
// chunks that flow through K device staging slots on three streams -- upload
// (states), compute (the Jacobian kernel), download (values and source
// terms) -- so that the transfers of one chunk overlap the kernel of
// another.  No kernels of its own: the compute step is launch_jacobian.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>
#include <vector>

#include "launch.h"
#include "pj_internal.h"

namespace pj {
namespace {

constexpr int kSlots = 3;                              // chunks in flight
constexpr size_t kSlotBudget = size_t(4) << 30;        // device bytes per slot (default chunk)

// Everything the call allocates, released on every path out.
struct HostRun {
  cudaStream_t s_in = nullptr, s_comp = nullptr, s_out = nullptr;
  cudaEvent_t ev_start = nullptr;
  cudaEvent_t ev_in[kSlots] = {}, ev_comp[kSlots] = {}, ev_out[kSlots] = {};
  bool used[kSlots] = {};
  void* mem = nullptr;  // all slots, the workspace and the status word
  ~HostRun() {
    // drain before freeing: an error path may leave copies queued
    if (s_in) cudaStreamSynchronize(s_in);
    if (s_comp) cudaStreamSynchronize(s_comp);
    if (s_out) cudaStreamSynchronize(s_out);
    if (ev_start) cudaEventDestroy(ev_start);
    for (int k = 0; k < kSlots; k++) {
      if (ev_in[k]) cudaEventDestroy(ev_in[k]);
      if (ev_comp[k]) cudaEventDestroy(ev_comp[k]);
      if (ev_out[k]) cudaEventDestroy(ev_out[k]);
    }
    if (s_in) cudaStreamDestroy(s_in);
    if (s_comp) cudaStreamDestroy(s_comp);
    if (s_out) cudaStreamDestroy(s_out);
    if (mem) cudaFree(mem);
  }
  int create() {
    cudaError_t e = cudaStreamCreateWithFlags(&s_in, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s_comp, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s_out, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev_start, cudaEventDisableTiming);
    for (int k = 0; k < kSlots && e == cudaSuccess; k++) {
      e = cudaEventCreateWithFlags(&ev_in[k], cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev_comp[k], cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev_out[k], cudaEventDisableTiming);
    }
    return check_cuda(e, "pj_eval_jacobian_sparse_host: streams and events");
  }
};

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace
}  // namespace pj

using namespace pj;

extern "C" int pj_eval_jacobian_sparse_host(const pj_mech* m, int mode, int fmt, int64_t n, const double* h_param,
                                            const double* h_phi, double* h_vals, double* h_dphi, int* h_status,
                                            int64_t chunk, void* stream) {
  const std::string fn = "pj_eval_jacobian_sparse_host";
  if (fmt != PJ_CSR && fmt != PJ_CSC) return fail(PJ_ERR_ARG, fn + ": fmt must be PJ_CSR or PJ_CSC");
  if (chunk < 0) return fail(PJ_ERR_ARG, fn + ": chunk < 0");
  if (n > 0 && !h_dphi) return fail(PJ_ERR_ARG, fn + ": h_dphi is required");
  int rc = check_common(fn.c_str(), m, mode, n, n > 0 ? n : 1, h_param, h_phi, h_vals);
  if (rc) return rc;
  if (h_status) *h_status = 0;
  if (n == 0) return PJ_OK;
  int dev = 0, max_pitch = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&max_pitch, cudaDevAttrMaxPitch, dev);
  if (e != cudaSuccess) return check_cuda(e, "cudaDeviceGetAttribute(max pitch)");
  if ((double)n * sizeof(double) > (double)max_pitch)
    return fail(PJ_ERR_UNSUPPORTED, fn + ": n too large for one strided copy (host row of " +
                                        std::to_string(n * sizeof(double)) + " bytes)");

  const int64_t N1 = m->ns + 1, nnz = m->nnz;
  const size_t per_state = (size_t)(2 * N1 + 1 + nnz) * sizeof(double);
  int64_t c = chunk > 0 ? chunk : std::max<int64_t>(128, (int64_t)(kSlotBudget / per_state) / 128 * 128);
  c = std::min(c, n);
  const int K = n > c ? kSlots : 1;
  // one slot, ld = c: param [c], phi [N1][c], vals [nnz][c], dphi [N1][c]
  const size_t b_param = align256((size_t)c * 8), b_phi = align256((size_t)(N1 * c) * 8);
  const size_t b_vals = align256((size_t)(nnz * c) * 8), b_dphi = b_phi;
  const size_t slot_bytes = b_param + b_phi + b_vals + b_dphi;
  const size_t ws = workspace_bytes(jacobian_arrays(), m->ns, c);
  const size_t total = (size_t)K * slot_bytes + align256(ws) + 256;

  HostRun R;
  if ((rc = R.create())) return rc;
  e = cudaMalloc(&R.mem, total);
  if (e != cudaSuccess) {
    cudaGetLastError();
    R.mem = nullptr;
    return fail(PJ_ERR_NOMEM, fn + ": device staging of " + std::to_string(total) + " bytes (pass a smaller chunk)");
  }
  char* base = static_cast<char*>(R.mem);
  void* d_ws = ws ? base + (size_t)K * slot_bytes : nullptr;
  int* d_status = reinterpret_cast<int*>(base + (size_t)K * slot_bytes + align256(ws));
  auto ok = [&](cudaError_t err, const char* what) { return err == cudaSuccess ? PJ_OK : check_cuda(err, what); };

  // after the work already queued on the caller's stream
  if ((rc = ok(cudaEventRecord(R.ev_start, (cudaStream_t)stream), "cudaEventRecord"))) return rc;
  if ((rc = ok(cudaStreamWaitEvent(R.s_in, R.ev_start, 0), "cudaStreamWaitEvent"))) return rc;
  if ((rc = ok(cudaMemsetAsync(d_status, 0, sizeof(int), R.s_comp), "cudaMemsetAsync(status)"))) return rc;
  int64_t i = 0;
  for (int64_t s0 = 0; s0 < n; s0 += c, i++) {
    const int k = (int)(i % K);
    const int64_t ci = std::min(c, n - s0);
    char* sb = base + (size_t)k * slot_bytes;
    double* d_param = reinterpret_cast<double*>(sb);
    double* d_phi = reinterpret_cast<double*>(sb + b_param);
    double* d_vals = reinterpret_cast<double*>(sb + b_param + b_phi);
    double* d_dphi = reinterpret_cast<double*>(sb + b_param + b_phi + b_vals);
    const size_t w = (size_t)ci * sizeof(double), dp = (size_t)c * sizeof(double), hp = (size_t)n * sizeof(double);
    // the slot is free once its previous chunk has been downloaded
    if (R.used[k] && (rc = ok(cudaStreamWaitEvent(R.s_in, R.ev_out[k], 0), "cudaStreamWaitEvent"))) return rc;
    if ((rc = ok(cudaMemcpyAsync(d_param, h_param + s0, w, cudaMemcpyHostToDevice, R.s_in), "upload param"))) return rc;
    if ((rc = ok(cudaMemcpy2DAsync(d_phi, dp, h_phi + s0, hp, w, (size_t)N1, cudaMemcpyHostToDevice, R.s_in),
                 "upload phi")))
      return rc;
    if ((rc = ok(cudaEventRecord(R.ev_in[k], R.s_in), "cudaEventRecord"))) return rc;
    if ((rc = ok(cudaStreamWaitEvent(R.s_comp, R.ev_in[k], 0), "cudaStreamWaitEvent"))) return rc;
    if ((rc = launch_jacobian(m->dm, mode, fmt, ci, d_param, d_phi, c, d_vals, d_dphi, d_status, d_ws, ws, R.s_comp)))
      return rc;
    if ((rc = ok(cudaEventRecord(R.ev_comp[k], R.s_comp), "cudaEventRecord"))) return rc;
    if ((rc = ok(cudaStreamWaitEvent(R.s_out, R.ev_comp[k], 0), "cudaStreamWaitEvent"))) return rc;
    if ((rc = ok(cudaMemcpy2DAsync(h_vals + s0, hp, d_vals, dp, w, (size_t)nnz, cudaMemcpyDeviceToHost, R.s_out),
                 "download values")))
      return rc;
    if ((rc = ok(cudaMemcpy2DAsync(h_dphi + s0, hp, d_dphi, dp, w, (size_t)N1, cudaMemcpyDeviceToHost, R.s_out),
                 "download source terms")))
      return rc;
    if ((rc = ok(cudaEventRecord(R.ev_out[k], R.s_out), "cudaEventRecord"))) return rc;
    R.used[k] = true;
  }
  int hs = 0;
  if ((rc = ok(cudaMemcpyAsync(&hs, d_status, sizeof(int), cudaMemcpyDeviceToHost, R.s_comp), "download status")))
    return rc;
  if ((rc = ok(cudaStreamSynchronize(R.s_comp), "cudaStreamSynchronize"))) return rc;
  if ((rc = ok(cudaStreamSynchronize(R.s_out), "cudaStreamSynchronize"))) return rc;
  if (h_status) *h_status = hs;
  return PJ_OK;
}
