// The analytical Jacobian kernels (Sec. 2.2, assembled as in Sec. 3.4):
// k_jacobian keeps each state's C_k, g_k/RT and h_k/RT in shared memory or a
// global workspace; k_jacobian_tm keeps h_k/RT in tensor memory.  Both call
// jacobian_state for one state per thread.  Included by jacobian_inst.cu,
// which instantiates one (layout, precision) pair per translation unit.
#pragma once

#include <cuda_runtime.h>

#include "kinetics_state.cuh"
#ifndef PJ_NO_LAUNCHERS
#include "launch.h"
#endif

namespace pj {

template <int MODE, int FMT, typename DT, bool NEWTON, bool SPECIAL>
__global__ void __launch_bounds__(128, kJacRegCtas) k_jacobian(DevMech m, int64_t n, const double* __restrict__ param,
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
    jacobian_state<MODE, FMT, DT, NEWTON, false, SPECIAL>(m, A, param, phi, ld, s, J, dphi, status, hstep, gamma);
}

// Jacobian with h_k/RT in tensor memory: blocks of 128 threads (one warp per
// TMEM lane quadrant) allocate `ncols` columns, walk the batch warp-uniformly
// so that the warp-collective TMEM accesses stay convergent, and free the
// columns before exiting.  C_k and g_k/RT are the state arrays 0 and 1: the
// first SPLIT of them sit in shared memory, the rest in a global workspace
// of ws_stride threads (the grid then covers exactly ws_stride threads).
template <int MODE, int FMT, typename DT, bool NEWTON, int SPLIT, bool SPECIAL>
__global__ void __launch_bounds__(128, kJacRegCtas) k_jacobian_tm(DevMech m, int64_t n, const double* __restrict__ param,
                                                     const double* __restrict__ phi, int64_t ld,
                                                     DT* __restrict__ J, double* __restrict__ dphi, int* status,
                                                     const double* __restrict__ hstep, double gamma,
                                                     uint32_t ncols, double* __restrict__ ws, int64_t ws_stride) {
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
  StateArraysT<SPLIT> A;
  A.ns = m.ns;
  A.base = smem + threadIdx.x;
  A.stride = blockDim.x;
  A.base2 = ws + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  A.stride2 = ws_stride;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x + warp * 32; base < n; base += stride) {
    const int64_t s = base + lane;
    jacobian_state<MODE, FMT, DT, NEWTON, true, SPECIAL>(m, A, param, phi, ld, s, J, dphi, status, hstep, gamma, tm_row,
                                                s < n);
  }
  tmem_fence_before();
  __syncthreads();
  tmem_fence_after();
  if (warp == 0) tmem_dealloc(tm_base, ncols);
}

#ifndef PJ_NO_LAUNCHERS
// Shared memory to request so that no more than `ctas` blocks of `kern` are
// resident per SM (a block beyond the TMEM budget would wait in
// tcgen05.alloc for a whole resident block's lifetime).
template <typename K>
static size_t tm_smem_cap_ctas(K kern, size_t dyn, int ctas) {
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, 128, dyn) != cudaSuccess) return dyn;
  if (occ <= ctas) return dyn;
  const size_t pad = kSmemPerSm / (size_t)(ctas + 1) - kBlockOverhead + 256;
  return pad > dyn ? pad : dyn;
}

template <int MODE, int FMT, typename DT, bool NEWTON, int SPLIT, bool SPECIAL>
static int launch_jac_tm_s(const DevMech& m, const TmPlan& t, int64_t n, const JacArgs& a, double* ws,
                           cudaStream_t st) {
  auto kern = k_jacobian_tm<MODE, FMT, DT, NEWTON, SPLIT, SPECIAL>;
  int rc;
  if ((rc = set_smem(kern, t.smem))) return rc;
  const size_t smem = tm_smem_cap_ctas(kern, t.smem, t.ctas);
  if (smem != t.smem && (rc = set_smem(kern, smem))) return rc;
  const int64_t blocks = (n + 127) / 128;
  int64_t grid = blocks < 1 ? 1 : blocks;
  int64_t ws_stride = 0;
  if (t.grid > 0) {
    grid = t.grid;
    ws_stride = (int64_t)t.grid * 128;
  }
  kern<<<(unsigned)grid, 128, smem, st>>>(m, n, a.param, a.phi, a.ld, static_cast<DT*>(a.J), a.dphi, a.status,
                                          a.hstep, a.gamma, t.ncols, ws, ws_stride);
  return check_cuda(cudaGetLastError(), "k_jacobian_tm launch");
}

template <int MODE, int FMT, typename DT, bool NEWTON, bool SPECIAL>
static int launch_jac_t(const DevMech& m, const LaunchPlan& p, int64_t n, const JacArgs& a, double* ws,
                        cudaStream_t st) {
  auto kern = k_jacobian<MODE, FMT, DT, NEWTON, SPECIAL>;
  int rc;
  if ((rc = set_smem(kern, p.smem))) return rc;
  const LaunchPlan q = resident_grid(kern, p);
  kern<<<q.grid, q.tpb, q.smem, st>>>(m, n, a.param, a.phi, a.ld, static_cast<DT*>(a.J), a.dphi, a.status, ws,
                                      q.ws_stride, a.hstep, a.gamma);
  return check_cuda(cudaGetLastError(), "k_jacobian launch");
}
#endif  // PJ_NO_LAUNCHERS

}  // namespace pj
