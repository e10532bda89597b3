// First-order forward finite-difference Jacobian: the comparator against
// which Sec. 3.5.2 measures the analytical Jacobian's speedup.  One state per
// thread: the source terms at Phi and at Phi + h_j e_j for every column j,
// with delta_j = 2^-26 max(|Phi_j|, 2^-26 n_tot), n_tot = P V / (R T), and the
// realised step h_j = (Phi_j + delta_j) - Phi_j (the paper gives no step
// rule; 2^-26 is about the square root of the unit roundoff, and a power of
// two keeps the scaling exact).  Column j is (f(Phi + h_j e_j) - f(Phi)) / h_j,
// stored in the handle's pattern (sparse) or in full (dense).  Every
// evaluation is the source-term path of source_state, so the cost is N + 1
// source-term evaluations per state.
#include <cuda_runtime.h>

#include <algorithm>

#include "kinetics_state.cuh"
#include "launch.h"

namespace pj {

constexpr double kFdScale = 0x1p-26;

// Per-thread rows of the workspace (stride ws_stride): C_k and g_k/RT when
// they do not sit in shared memory, then the perturbed state x (N rows) and
// its source terms f1 (N rows).
template <int MODE, int FMT>
__global__ void __launch_bounds__(128) k_fd_jacobian(DevMech m, int64_t n, const double* __restrict__ param,
                                                     const double* __restrict__ phi, int64_t ld,
                                                     double* __restrict__ J, double* __restrict__ dphi,
                                                     int* status, double* __restrict__ ws, int64_t ws_stride,
                                                     int arrays_in_ws) {
  PJ_DYN_SMEM;
  load_exp_table(m.exp_tab);
  const int ns = m.ns, N = m.N;
  const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double* own = ws + gtid;
  StateArrays A;
  A.ns = ns;
  if (arrays_in_ws) {
    A.base = own;
    A.stride = ws_stride;
    own += (int64_t)2 * ns * ws_stride;
  } else {
    A.base = smem + threadIdx.x;
    A.stride = blockDim.x;
  }
  double* x = own;
  double* f1 = own + (int64_t)N * ws_stride;
  for (int64_t s = gtid; s < n; s += (int64_t)gridDim.x * blockDim.x) {
    source_state<MODE>(m, A, param, phi, ld, s, dphi, status);
    const double T = phi[s], S = phi[ld + s], par = param[s];
    const double V = MODE == PJ_CONP ? S : par, P = MODE == PJ_CONP ? par : S;
    const double ntot = (P * V) / (RU * T);
    const double lo = kFdScale * ntot;
    for (int v = 0; v < N; v++) x[(int64_t)v * ws_stride] = phi[(int64_t)v * ld + s];
    for (int j = 0; j < N; j++) {
      const double xj = x[(int64_t)j * ws_stride];
      const double d = kFdScale * fmax(fabs(xj), lo);
      const double xp = xj + d;
      const double h = xp - xj;
      x[(int64_t)j * ws_stride] = xp;
      source_state<MODE>(m, A, param + s, x, ws_stride, 0, f1, nullptr);
      x[(int64_t)j * ws_stride] = xj;
      for (int i = 0; i < N; i++) {
        const int64_t e = jpos<FMT>(m, i, j);
        if (e >= 0) J[e * ld + s] = (__ldcg(f1 + (int64_t)i * ws_stride) - __ldcg(dphi + (int64_t)i * ld + s)) / h;
      }
    }
  }
}

// C_k and g_k/RT in shared memory when 128 threads' arrays fit; the grid is
// at most four blocks of 128 per SM (and no more than are resident), which
// bounds the workspace.
static bool fd_arrays_in_smem(int ns) { return (size_t)2 * ns * sizeof(double) * 128 <= kSmemCap; }

static size_t fd_per_thread(int ns) {
  const size_t N = (size_t)ns + 1;
  return (2 * N + (fd_arrays_in_smem(ns) ? 0 : (size_t)2 * ns)) * sizeof(double);
}

size_t fd_workspace_bytes(int ns, int64_t n) {
  const int64_t blocks = (n + 127) / 128;
  const int64_t cap = (int64_t)sm_count() * 4;
  const int64_t grid = std::max<int64_t>(1, std::min(blocks, cap));
  return fd_per_thread(ns) * (size_t)grid * 128;
}

template <int MODE, int FMT>
static int launch_fd_t(const DevMech& m, int64_t n, const double* param, const double* phi, int64_t ld, double* J,
                       double* dphi, int* status, double* ws, cudaStream_t st) {
  auto kern = k_fd_jacobian<MODE, FMT>;
  const bool in_smem = fd_arrays_in_smem(m.ns);
  const size_t smem = in_smem ? (size_t)2 * m.ns * sizeof(double) * 128 : 0;
  int rc;
  if ((rc = set_smem(kern, smem))) return rc;
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, 128, smem) != cudaSuccess || occ < 1) occ = 1;
  const int64_t blocks = (n + 127) / 128;
  const int64_t cap = (int64_t)sm_count() * std::min(occ, 4);
  const int64_t grid = std::max<int64_t>(1, std::min(blocks, cap));
  kern<<<(unsigned)grid, 128, smem, st>>>(m, n, param, phi, ld, J, dphi, status, ws, grid * 128, in_smem ? 0 : 1);
  return check_cuda(cudaGetLastError(), "k_fd_jacobian launch");
}

int launch_fd_jacobian(const DevMech& m, int mode, int fmt, int64_t n, const double* param, const double* phi,
                       int64_t ld, double* J, double* dphi, int* status, void* work, size_t work_bytes,
                       cudaStream_t st) {
  const size_t need = fd_workspace_bytes(m.ns, n);
  if (!work || work_bytes < need)
    return fail(PJ_ERR_NOMEM, "workspace too small for the finite-difference Jacobian (see pj_workspace_size)");
  double* ws = static_cast<double*>(work);
  if (mode == PJ_CONP) {
    if (fmt == PJ_CSR) return launch_fd_t<PJ_CONP, PJ_CSR>(m, n, param, phi, ld, J, dphi, status, ws, st);
    if (fmt == PJ_CSC) return launch_fd_t<PJ_CONP, PJ_CSC>(m, n, param, phi, ld, J, dphi, status, ws, st);
    return launch_fd_t<PJ_CONP, PJ_DENSE>(m, n, param, phi, ld, J, dphi, status, ws, st);
  }
  if (fmt == PJ_CSR) return launch_fd_t<PJ_CONV, PJ_CSR>(m, n, param, phi, ld, J, dphi, status, ws, st);
  if (fmt == PJ_CSC) return launch_fd_t<PJ_CONV, PJ_CSC>(m, n, param, phi, ld, J, dphi, status, ws, st);
  return launch_fd_t<PJ_CONV, PJ_DENSE>(m, n, param, phi, ld, J, dphi, status, ws, st);
}

}  // namespace pj
