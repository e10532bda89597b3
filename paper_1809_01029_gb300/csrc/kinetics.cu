// Source terms and the analytical Jacobian of the molar, explicitly
// mass-conserving formulation (Sec. 2.2), one thermochemical state per
// thread ("shallow" vectorisation, Sec. 2.1) over a structure-of-arrays
// batch.
//
// GB300 design notes (see the design doc for the measurements behind them):
//  * The path is bound by the FP64 pipe (about 0.4 lane-FMA per clock per SM
//    sub-partition on this part), not by HBM, so the kernels minimise FP64
//    instructions: one exp per forward rate, one per reverse rate (from
//    ln kf - ln Kc), the T-only pieces once per reaction, ln T and 1/T once
//    per state.
//  * One warp per SM sub-partition already saturates that pipe, so a block of
//    128 threads per SM is enough and every thread can keep its state's
//    concentrations, Gibbs energies and production-rate accumulators in
//    shared memory (or, for large mechanisms, in a global workspace).
//  * Reaction constants are read warp-uniformly (every thread of a warp works
//    on the same reaction), so there is no divergence except the NASA range.
//  * Jacobian entries are accumulated with fire-and-forget FP64 reductions
//    into the zero-initialised output at L2 (no read-modify-write latency on
//    the SM and no FP64 add on the SM); each entry is owned by one thread,
//    whose reductions apply in program order, so results are deterministic.
//    Targets come from a static full -> sparse index map built at mechanism
//    load (the mapping Sec. 3.3 proposes instead of a per-entry search).
#include <cuda_runtime.h>

#include <algorithm>

#include "kinetics_state.cuh"

namespace pj {

// ---------------------------------------------------------------------------
// source terms
// ---------------------------------------------------------------------------
// Shared memory holds C_k and g_k/RT per state; production rates are summed
// by L2 reductions into the output rows (the bath gas in a register).
template <int MODE>
__global__ void __launch_bounds__(128) k_source_terms(DevMech m, int64_t n, const double* __restrict__ param,
                                                      const double* __restrict__ phi, int64_t ld,
                                                      double* __restrict__ out, int* status, double* ws,
                                                      int64_t ws_stride) {
  PJ_DYN_SMEM;
  load_exp_table(m.exp_tab);
  const int ns = m.ns;
  const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  StateArrays A;
  A.ns = ns;
  if (ws) {
    A.base = ws + gtid;
    A.stride = ws_stride;
  } else {
    A.base = smem + threadIdx.x;
    A.stride = blockDim.x;
  }
  for (int64_t s = gtid; s < n; s += (int64_t)gridDim.x * blockDim.x)
    source_state<MODE>(m, A, param, phi, ld, s, out, status);
}

template <int MODE, int FMT, typename DT, bool NEWTON>
__global__ void __launch_bounds__(128) k_jacobian(DevMech m, int64_t n, const double* __restrict__ param,
                                                  const double* __restrict__ phi, int64_t ld,
                                                  DT* __restrict__ J, double* __restrict__ dphi,
                                                  int* status, double* ws, int64_t ws_stride,
                                                  const double* __restrict__ hstep, double gamma) {
  PJ_DYN_SMEM;
  load_exp_table(m.exp_tab);
  const int ns = m.ns;
  const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  StateArrays A;
  A.ns = ns;
  if (ws) {
    A.base = ws + gtid;
    A.stride = ws_stride;
  } else {
    A.base = smem + threadIdx.x;
    A.stride = blockDim.x;
  }
  for (int64_t s = gtid; s < n; s += (int64_t)gridDim.x * blockDim.x)
    jacobian_state<MODE, FMT, DT, NEWTON>(m, A, param, phi, ld, s, J, dphi, status, hstep, gamma);
}

// Jacobian with h_k/RT in tensor memory (C_k and g_k/RT in shared memory):
// blocks of 128 threads (one warp per TMEM lane quadrant) allocate `ncols`
// columns, walk the batch warp-uniformly so that the warp-collective TMEM
// accesses stay convergent, and free the columns before exiting.
template <int MODE, int FMT, typename DT, bool NEWTON>
__global__ void __launch_bounds__(128) k_jacobian_tm(DevMech m, int64_t n, const double* __restrict__ param,
                                                     const double* __restrict__ phi, int64_t ld,
                                                     DT* __restrict__ J, double* __restrict__ dphi, int* status,
                                                     const double* __restrict__ hstep, double gamma,
                                                     uint32_t ncols) {
  PJ_DYN_SMEM;
  __shared__ uint32_t tm_base;
  load_exp_table(m.exp_tab);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp == 0) {
    tmem_alloc(&tm_base, ncols);
    tmem_relinquish();
  }
  tmem_fence_before();
  __syncthreads();
  tmem_fence_after();
  const uint32_t tm_row = tm_base + ((uint32_t)(32 * (warp & 3)) << 16);
  StateArrays A;
  A.ns = m.ns;
  A.base = smem + threadIdx.x;
  A.stride = blockDim.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x + warp * 32; base < n; base += stride) {
    const int64_t s = base + lane;
    jacobian_state<MODE, FMT, DT, NEWTON, true>(m, A, param, phi, ld, s, J, dphi, status, hstep, gamma, tm_row,
                                                s < n);
  }
  tmem_fence_before();
  __syncthreads();
  tmem_fence_after();
  if (warp == 0) tmem_dealloc(tm_base, ncols);
}

// pj_exp next to the library exp, for verification (pj_diag_exp).
__global__ void k_diag_exp(const double* __restrict__ tab, int64_t n, const double* __restrict__ x,
                           double* __restrict__ y_ours, double* __restrict__ y_lib) {
  load_exp_table(tab);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    y_ours[i] = pj_exp(x[i]);
    y_lib[i] = exp(x[i]);
  }
}

#ifndef PJ_NO_LAUNCHERS
int launch_diag_exp(const DevMech& m, int64_t n, const double* x, double* y_ours, double* y_lib, cudaStream_t st) {
  int64_t blocks = (n + 255) / 256;
  if (blocks > 65535) blocks = 65535;
  if (blocks < 1) blocks = 1;
  k_diag_exp<<<(unsigned)blocks, 256, 0, st>>>(m.exp_tab, n, x, y_ours, y_lib);
  return check_cuda(cudaGetLastError(), "k_diag_exp launch");
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
struct LaunchPlan {
  int tpb;
  int grid;
  size_t smem;
  bool global_ws;
  int64_t ws_stride;
  size_t ws_bytes;
};

static int g_num_sms = 0;

static int num_sms() {
  if (g_num_sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_num_sms <= 0) g_num_sms = 1;
  }
  return g_num_sms;
}

int sm_count() { return num_sms(); }

// Per-state arrays: in shared memory when 128 threads fit, else in a global
// workspace with a fixed grid-stride grid.
LaunchPlan plan_for(int arrays, int ns, int64_t n) {
  LaunchPlan p{};
  const size_t per_thread = (size_t)arrays * ns * sizeof(double);
  const size_t smem_cap = 225 * 1024;  // 227 KB opt-in per block, less the 2 KB exp table
  // threads per SM that fit the per-state arrays in shared memory, as whole
  // warps; blocks of up to 128 threads so several can share an SM
  const int fit = (int)((smem_cap / per_thread) / 32 * 32);
  if (fit >= 128) {
    p.global_ws = false;
    p.tpb = fit >= 256 ? 128 : (fit % 64 == 0 ? 64 : 32);
    p.smem = per_thread * p.tpb;
    const int64_t blocks = (n + p.tpb - 1) / p.tpb;
    p.grid = (int)(blocks < 1 ? 1 : blocks);
    p.ws_bytes = 0;
    p.ws_stride = 0;
  } else {
    p.global_ws = true;
    p.tpb = 128;
    p.smem = 0;
    const int64_t cap = (int64_t)num_sms() * 4;
    const int64_t blocks = (n + p.tpb - 1) / p.tpb;
    p.grid = (int)(blocks < cap ? (blocks < 1 ? 1 : blocks) : cap);
    p.ws_stride = (int64_t)p.grid * p.tpb;
    p.ws_bytes = per_thread * (size_t)p.ws_stride;
  }
  return p;
}

int source_arrays() { return 2; }
int jacobian_arrays() { return 3; }

template <typename K>
static int set_smem(K kern, size_t smem) {
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return check_cuda(e, "cudaFuncSetAttribute");
  }
  return PJ_OK;
}

int launch_source(const DevMech& m, int mode, int64_t n, const double* param, const double* phi, int64_t ld,
                  double* out, int* status, void* work, size_t work_bytes, cudaStream_t st) {
  LaunchPlan p = plan_for(source_arrays(), m.ns, n);
  if (p.global_ws && (!work || work_bytes < p.ws_bytes))
    return fail(PJ_ERR_NOMEM, "workspace too small for the source-term kernel (see pj_workspace_size)");
  double* ws = p.global_ws ? static_cast<double*>(work) : nullptr;
  int rc;
  if (mode == PJ_CONP) {
    if ((rc = set_smem(k_source_terms<PJ_CONP>, p.smem))) return rc;
    k_source_terms<PJ_CONP><<<p.grid, p.tpb, p.smem, st>>>(m, n, param, phi, ld, out, status, ws, p.ws_stride);
  } else {
    if ((rc = set_smem(k_source_terms<PJ_CONV>, p.smem))) return rc;
    k_source_terms<PJ_CONV><<<p.grid, p.tpb, p.smem, st>>>(m, n, param, phi, ld, out, status, ws, p.ws_stride);
  }
  return check_cuda(cudaGetLastError(), "k_source_terms launch");
}

// TMEM mode for the Jacobian: C and g/RT in shared memory for blocks of 128,
// h/RT in TMEM.  Used when it allows more resident threads than keeping all
// three arrays in shared memory (both capped by 168 registers x 3 blocks).
struct TmPlan {
  bool use;
  uint32_t ncols;
  size_t smem;
};

static TmPlan tm_plan(int ns) {
  TmPlan t{false, 0, 0};
  const size_t cap = 225 * 1024;
  uint32_t nc = 32;
  while (nc < 2u * (uint32_t)ns) nc <<= 1;
  if (nc > 512) return t;
  const size_t smem2 = (size_t)2 * ns * sizeof(double) * 128;
  if (smem2 > cap) return t;
  const int reg_threads = 384;
  int blocks = (int)(cap / (smem2 + 2048));
  if (blocks > (int)(512 / nc)) blocks = (int)(512 / nc);
  const int tm_threads = std::min(blocks * 128, reg_threads);
  const size_t per3 = (size_t)3 * ns * sizeof(double);
  const int cur_threads = std::min((int)((cap / per3) / 32 * 32), reg_threads);
  if (tm_threads > cur_threads) {
    t.use = true;
    t.ncols = nc;
    t.smem = smem2;
  }
  return t;
}

template <int MODE, int FMT, typename DT, bool NEWTON>
static int launch_jac_tm(const DevMech& m, const TmPlan& t, int64_t n, const double* param, const double* phi,
                         int64_t ld, DT* J, double* dphi, int* status, cudaStream_t st, const double* hstep,
                         double gamma) {
  int rc;
  if ((rc = set_smem(k_jacobian_tm<MODE, FMT, DT, NEWTON>, t.smem))) return rc;
  const int64_t blocks = (n + 127) / 128;
  k_jacobian_tm<MODE, FMT, DT, NEWTON><<<(unsigned)(blocks < 1 ? 1 : blocks), 128, t.smem, st>>>(
      m, n, param, phi, ld, J, dphi, status, hstep, gamma, t.ncols);
  return check_cuda(cudaGetLastError(), "k_jacobian_tm launch");
}

template <int MODE, int FMT, typename DT = double, bool NEWTON = false>
static int launch_jac_t(const DevMech& m, const LaunchPlan& p, int64_t n, const double* param, const double* phi,
                        int64_t ld, DT* J, double* dphi, int* status, double* ws, cudaStream_t st,
                        const double* hstep = nullptr, double gamma = 0.0) {
  int rc;
  if ((rc = set_smem(k_jacobian<MODE, FMT, DT, NEWTON>, p.smem))) return rc;
  k_jacobian<MODE, FMT, DT, NEWTON><<<p.grid, p.tpb, p.smem, st>>>(m, n, param, phi, ld, J, dphi, status, ws,
                                                                     p.ws_stride, hstep, gamma);
  return check_cuda(cudaGetLastError(), "k_jacobian launch");
}

int launch_jacobian(const DevMech& m, int mode, int fmt, int64_t n, const double* param, const double* phi,
                    int64_t ld, double* J, double* dphi, int* status, void* work, size_t work_bytes,
                    cudaStream_t st) {
  const TmPlan t = tm_plan(m.ns);
  if (t.use) {
    if (mode == PJ_CONP) {
      if (fmt == PJ_CSR) return launch_jac_tm<PJ_CONP, PJ_CSR, double, false>(m, t, n, param, phi, ld, J, dphi, status, st, nullptr, 0.0);
      if (fmt == PJ_CSC) return launch_jac_tm<PJ_CONP, PJ_CSC, double, false>(m, t, n, param, phi, ld, J, dphi, status, st, nullptr, 0.0);
      return launch_jac_tm<PJ_CONP, PJ_DENSE, double, false>(m, t, n, param, phi, ld, J, dphi, status, st, nullptr, 0.0);
    }
    if (fmt == PJ_CSR) return launch_jac_tm<PJ_CONV, PJ_CSR, double, false>(m, t, n, param, phi, ld, J, dphi, status, st, nullptr, 0.0);
    if (fmt == PJ_CSC) return launch_jac_tm<PJ_CONV, PJ_CSC, double, false>(m, t, n, param, phi, ld, J, dphi, status, st, nullptr, 0.0);
    return launch_jac_tm<PJ_CONV, PJ_DENSE, double, false>(m, t, n, param, phi, ld, J, dphi, status, st, nullptr, 0.0);
  }
  LaunchPlan p = plan_for(jacobian_arrays(), m.ns, n);
  if (p.global_ws && (!work || work_bytes < p.ws_bytes))
    return fail(PJ_ERR_NOMEM, "workspace too small for the Jacobian kernel (see pj_workspace_size)");
  double* ws = p.global_ws ? static_cast<double*>(work) : nullptr;
  if (mode == PJ_CONP) {
    if (fmt == PJ_CSR) return launch_jac_t<PJ_CONP, PJ_CSR>(m, p, n, param, phi, ld, J, dphi, status, ws, st);
    if (fmt == PJ_CSC) return launch_jac_t<PJ_CONP, PJ_CSC>(m, p, n, param, phi, ld, J, dphi, status, ws, st);
    return launch_jac_t<PJ_CONP, PJ_DENSE>(m, p, n, param, phi, ld, J, dphi, status, ws, st);
  }
  if (fmt == PJ_CSR) return launch_jac_t<PJ_CONV, PJ_CSR>(m, p, n, param, phi, ld, J, dphi, status, ws, st);
  if (fmt == PJ_CSC) return launch_jac_t<PJ_CONV, PJ_CSC>(m, p, n, param, phi, ld, J, dphi, status, ws, st);
  return launch_jac_t<PJ_CONV, PJ_DENSE>(m, p, n, param, phi, ld, J, dphi, status, ws, st);
}

size_t workspace_bytes(int arrays, int ns, int64_t n) {
  if (arrays == jacobian_arrays() && tm_plan(ns).use) return 0;
  return plan_for(arrays, ns, n).ws_bytes;
}

// Newton-iteration matrix M = I - h*gamma*J in FP32 (derivative arithmetic
// in FP32, rates and source terms in FP64).
int launch_newton_f32(const DevMech& m, int mode, int fmt, int64_t n, const double* param, const double* phi,
                      int64_t ld, const double* hstep, double gamma, float* M, double* dphi, int* status,
                      void* work, size_t work_bytes, cudaStream_t st) {
  const TmPlan t = tm_plan(m.ns);
  if (t.use) {
    if (mode == PJ_CONP) {
      if (fmt == PJ_CSR) return launch_jac_tm<PJ_CONP, PJ_CSR, float, true>(m, t, n, param, phi, ld, M, dphi, status, st, hstep, gamma);
      if (fmt == PJ_CSC) return launch_jac_tm<PJ_CONP, PJ_CSC, float, true>(m, t, n, param, phi, ld, M, dphi, status, st, hstep, gamma);
      return launch_jac_tm<PJ_CONP, PJ_DENSE, float, true>(m, t, n, param, phi, ld, M, dphi, status, st, hstep, gamma);
    }
    if (fmt == PJ_CSR) return launch_jac_tm<PJ_CONV, PJ_CSR, float, true>(m, t, n, param, phi, ld, M, dphi, status, st, hstep, gamma);
    if (fmt == PJ_CSC) return launch_jac_tm<PJ_CONV, PJ_CSC, float, true>(m, t, n, param, phi, ld, M, dphi, status, st, hstep, gamma);
    return launch_jac_tm<PJ_CONV, PJ_DENSE, float, true>(m, t, n, param, phi, ld, M, dphi, status, st, hstep, gamma);
  }
  LaunchPlan p = plan_for(jacobian_arrays(), m.ns, n);
  if (p.global_ws && (!work || work_bytes < p.ws_bytes))
    return fail(PJ_ERR_NOMEM, "workspace too small for the Newton-matrix kernel (see pj_workspace_size)");
  double* ws = p.global_ws ? static_cast<double*>(work) : nullptr;
  if (mode == PJ_CONP) {
    if (fmt == PJ_CSR) return launch_jac_t<PJ_CONP, PJ_CSR, float, true>(m, p, n, param, phi, ld, M, dphi, status, ws, st, hstep, gamma);
    if (fmt == PJ_CSC) return launch_jac_t<PJ_CONP, PJ_CSC, float, true>(m, p, n, param, phi, ld, M, dphi, status, ws, st, hstep, gamma);
    return launch_jac_t<PJ_CONP, PJ_DENSE, float, true>(m, p, n, param, phi, ld, M, dphi, status, ws, st, hstep, gamma);
  }
  if (fmt == PJ_CSR) return launch_jac_t<PJ_CONV, PJ_CSR, float, true>(m, p, n, param, phi, ld, M, dphi, status, ws, st, hstep, gamma);
  if (fmt == PJ_CSC) return launch_jac_t<PJ_CONV, PJ_CSC, float, true>(m, p, n, param, phi, ld, M, dphi, status, ws, st, hstep, gamma);
  return launch_jac_t<PJ_CONV, PJ_DENSE, float, true>(m, p, n, param, phi, ld, M, dphi, status, ws, st, hstep, gamma);
}

// Run k_jacobian with its per-state arrays in a scratch region that holds
// `scratch_threads` threads' arrays (grid-stride over the states).  Used by
// the allocation-free entry point (noalloc.cu).
int launch_jacobian_on_scratch(const DevMech& m, int mode, int fmt, int64_t n, const double* param,
                               const double* phi, int64_t ld, double* J, double* dphi, int* status,
                               double* scratch, int64_t scratch_threads, cudaStream_t st) {
  LaunchPlan p{};
  p.tpb = 128;
  p.global_ws = true;
  p.smem = 0;
  const int64_t blocks = (n + p.tpb - 1) / p.tpb;
  int64_t cap = scratch_threads / p.tpb;
  const int64_t sm_cap = (int64_t)num_sms() * 4;
  if (cap > sm_cap) cap = sm_cap;
  p.grid = (int)(blocks < cap ? (blocks < 1 ? 1 : blocks) : cap);
  p.ws_stride = (int64_t)p.grid * p.tpb;
  p.ws_bytes = (size_t)jacobian_arrays() * m.ns * sizeof(double) * (size_t)p.ws_stride;
  if (mode == PJ_CONP) {
    if (fmt == PJ_CSR) return launch_jac_t<PJ_CONP, PJ_CSR>(m, p, n, param, phi, ld, J, dphi, status, scratch, st);
    return launch_jac_t<PJ_CONP, PJ_CSC>(m, p, n, param, phi, ld, J, dphi, status, scratch, st);
  }
  if (fmt == PJ_CSR) return launch_jac_t<PJ_CONV, PJ_CSR>(m, p, n, param, phi, ld, J, dphi, status, scratch, st);
  return launch_jac_t<PJ_CONV, PJ_CSC>(m, p, n, param, phi, ld, J, dphi, status, scratch, st);
}
#endif  // PJ_NO_LAUNCHERS

}  // namespace pj
