// Source terms and the analytical Jacobian of the molar, explicitly
// mass-conserving formulation (Sec. 2.2), one thermochemical state per
// thread ("shallow" vectorisation, Sec. 2.1) over a structure-of-arrays
// batch.
//
// GB300 design notes:
//  * The path is bound by the FP64 pipe (2 FP64 FMA per clock per SM on this
//    part, a 64th of the FP32 rate), not by HBM, so the kernels minimise
//    FP64 instructions: one exp per forward rate, one per reverse rate (from
//    ln kf - ln Kc), the T-only pieces once per reaction, ln T and 1/T once
//    per state.
//  * One warp per SM sub-partition already saturates that pipe when it has
//    independent work, so blocks of 128 threads keep each state's
//    concentrations, Gibbs energies and enthalpies on chip (shared memory and
//    TMEM) or, for large mechanisms, in a global workspace.
//  * Reaction constants are read warp-uniformly (every thread of a warp works
//    on the same reaction), so there is no divergence except the NASA range.
//  * Jacobian entries are accumulated with fire-and-forget FP64 reductions
//    into the zero-initialised output at L2 (no read-modify-write latency on
//    the SM and no FP64 add on the SM).  One state per thread, each entry is
//    owned by one thread, whose reductions apply in program order, so results
//    are deterministic; the cooperative layout sums one entry from several
//    warps, in an order that can change between runs.
//    Targets come from a static full -> sparse index map built at mechanism
//    load (the mapping Sec. 3.4 proposes instead of a per-entry search).
//  * This file holds the source-term kernel and the launch planning; the
//    Jacobian kernels are in jacobian_kernels.cuh (instantiated by
//    jacobian_inst.cu).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>

#include "jacobian_kernels.cuh"  // k_jacobian_coop's tile and shared-memory size (the kernels: jacobian_inst.cu)
#include "kinetics_state.cuh"
#ifndef PJ_NO_LAUNCHERS
#include "launch.h"
#endif

namespace pj {

// ---------------------------------------------------------------------------
// source terms
// ---------------------------------------------------------------------------
// Shared memory holds C_k and g_k/RT per state; production rates are summed
// by L2 reductions into the output rows (the bath gas in a register).
template <int MODE, bool SPECIAL>
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
    source_state<MODE, SPECIAL>(m, A, param, phi, ld, s, out, status);
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
static int g_num_sms[64] = {};

int sm_count() {
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  if (g_num_sms[dev] == 0) {
    int c = 0;
    cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, dev);
    g_num_sms[dev] = c > 0 ? c : 1;
  }
  return g_num_sms[dev];
}

// Per-state arrays: in shared memory when 128 threads fit, else in a global
// workspace with a grid-stride grid (trimmed to the resident blocks at
// launch, see resident_grid).  The source terms always take the L1-cached
// workspace, at up to eight blocks of 128 per SM: at 53 species shared
// memory allowed two, and the workspace layout measured 1.18x faster.
LaunchPlan plan_for(int arrays, int ns, int64_t n) {
  LaunchPlan p{};
  const size_t per_thread = (size_t)arrays * ns * sizeof(double);
  // threads per SM that fit the per-state arrays in shared memory, as whole
  // warps; blocks of up to 128 threads so several can share an SM
  const int fit = (int)((kSmemCap / per_thread) / 32 * 32);
  const bool source = arrays == source_arrays();
  if (fit >= 128 && !source) {
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
    const int64_t cap = (int64_t)sm_count() * (source ? 8 : 4);
    const int64_t blocks = (n + p.tpb - 1) / p.tpb;
    p.grid = (int)(blocks < cap ? (blocks < 1 ? 1 : blocks) : cap);
    p.ws_stride = (int64_t)p.grid * p.tpb;
    p.ws_bytes = per_thread * (size_t)p.ws_stride;
  }
  return p;
}

int source_arrays() { return 2; }
int jacobian_arrays() { return 3; }

int launch_source(const DevMech& m, int mode, int64_t n, const double* param, const double* phi, int64_t ld,
                  double* out, int* status, void* work, size_t work_bytes, cudaStream_t st) {
  LaunchPlan p = plan_for(source_arrays(), m.ns, n);
  if (p.global_ws && (!work || work_bytes < p.ws_bytes))
    return fail(PJ_ERR_NOMEM, "workspace too small for the source-term kernel (see pj_workspace_size)");
  double* ws = p.global_ws ? static_cast<double*>(work) : nullptr;
  int rc;
  const bool special = m.nr_plain < m.nr;
  auto kern = mode == PJ_CONP ? (special ? k_source_terms<PJ_CONP, true> : k_source_terms<PJ_CONP, false>)
                              : (special ? k_source_terms<PJ_CONV, true> : k_source_terms<PJ_CONV, false>);
  if ((rc = set_smem(kern, p.smem))) return rc;
  const LaunchPlan q = resident_grid(kern, p);
  kern<<<q.grid, q.tpb, q.smem, st>>>(m, n, param, phi, ld, out, status, ws, q.ws_stride);
  return check_cuda(cudaGetLastError(), "k_source_terms launch");
}

// TMEM mode for the Jacobian.  Chosen when it keeps at least as many
// threads resident as the plain kernel (arrays in shared memory when 128
// threads fit, else in a workspace at the register-limited occupancy); of the
// splits of C_k, g_k/RT between shared memory and the workspace, the one with
// the most resident blocks, on ties the one with the fewest arrays in shared
// memory (L1-cached workspace loads measured faster than shared-memory loads
// at equal occupancy on the 53-species workload).
TmPlan tm_plan(int ns) {
  TmPlan t{false, 0, 2, 0, 0, 0, 0};
  uint32_t nc = 32;
  while (nc < 2u * (uint32_t)ns) nc <<= 1;
  if (nc > 512) return t;
  const int tm_ctas = (int)(512 / nc);
  int best_ctas = 0, best_split = 2;
  size_t best_smem = 0;
  for (int split = 0; split <= 2; split++) {
    const size_t dyn = (size_t)split * ns * sizeof(double) * 128;
    if (dyn > kSmemCap) continue;
    const int smem_ctas = (int)(kSmemPerSm / (dyn + kBlockOverhead));
    const int ctas = std::min(std::min(smem_ctas, tm_ctas), kJacRegCtas);
    if (ctas > best_ctas) {
      best_ctas = ctas;
      best_split = split;
      best_smem = dyn;
    }
  }
  if (best_ctas == 0) return t;
  const size_t per3 = (size_t)3 * ns * sizeof(double);
  const int fit = (int)((kSmemCap / per3) / 32 * 32);
  const int plain_threads = fit >= 128 ? std::min(fit, kJacRegCtas * 128) : kJacRegCtas * 128;
  if (best_ctas * 128 < plain_threads || (best_ctas * 128 == plain_threads && fit >= 128)) return t;
  t.use = true;
  t.ncols = nc;
  t.split = best_split;
  t.ctas = best_ctas;
  t.smem = best_smem;
  if (best_split < 2) {
    t.grid = sm_count() * best_ctas;
    t.ws_bytes = (size_t)(2 - best_split) * ns * sizeof(double) * (size_t)t.grid * 128;
  }
  return t;
}

// Which Jacobian layout runs, chosen by measurement on GB300 (1 Mi states
// unless stated; states/s, one state per thread against the cooperative
// shapes, warps x blocks per SM):
//  * at most one 32-state tile per SM: cooperative, 16 warps on each tile
//    (13 species, 4096 states: 64 M against 13 M);
//  * the FP64 Jacobian of TMEM-size mechanisms (53 species) and of
//    mechanisms whose one-state-per-thread arrays need a global workspace
//    (111 species), and any batch below SMs x 512 states: cooperative, 8
//    warps x 2 blocks (53 species CSR 11.47 M against 11.17 M in TMEM, CSC
//    11.46 / 11.06, CONV 11.93 / 11.73, all reaction types 9.84 / 9.75;
//    111 species 4.69 M against 4.16 M; 53 species, 64 ki states 11.0 M
//    against 9.8 M), 16 warps x 1 above 200 species (the 874-species
//    arrays are 671 KB a tile);
//  * the dense FP64 Jacobian of TMEM-size mechanisms: one state per thread
//    in TMEM (11.49 M against 11.35 M);
//  * the FP32 Newton matrix of those mechanisms: cooperative, 4 warps x 4
//    blocks, the arrays in the workspace (53 species 14.64 M against 13.22
//    M; 111 species 5.84 M against 4.85 M);
//  * otherwise (13 species, large batches): one state per thread, arrays
//    in shared memory (117 M against 114 M at 4 x 4).
// Each cooperative block keeps only its 32 states' Jacobians live in L2, a
// fraction of the one-state-per-thread kernels' live set (DRAM traffic per
// state at 53 species: 154 KB in TMEM, 34 KB at 16 x 1, 65 KB at 8 x 2), so
// 16 x 1 is the shape to force where the Jacobian shares the GPU with other
// memory-heavy work.
// The cooperative kernel keeps a tile's per-state arrays in shared memory
// where they fit, else in a workspace of 3 Ns x 32 doubles per block, which
// stays in L2 (874 species at one block per SM: 102 MB).
// PYJAC_GB_JAC_LAYOUT=coop|percore forces one family (coop only where its
// shared memory fits); PYJAC_GB_COOP_WARPS sets the warps per block (4, 8
// or 16), PYJAC_GB_COOP_CTAS the blocks per SM (at most 16 / warps) and
// PYJAC_GB_COOP_ARRAYS=global puts the arrays in the workspace; 8 warps in
// one block per SM run the instance compiled for 255 registers.
static int env_int(const char* name, int dflt) {
  const char* v = getenv(name);
  return v && *v ? atoi(v) : dflt;
}

bool coop_shape(const DevMech& m, int warps, int ctas, bool arrays_smem, int64_t tiles, CoopPlan& c) {
  c = CoopPlan{false, warps, ctas, coop_smem_bytes(m.ns, warps, arrays_smem), sm_count() * ctas,
               warps == 8 && ctas == 1, 0};
  if (warps != 4 && warps != 8 && warps != 16) return false;
  if (ctas < 1 || ctas * warps > 16) return false;
  if (c.smem + kBlockOverhead > kSmemPerSm / (size_t)ctas || c.smem > kSmemCap) return false;
  if (!arrays_smem) {
    const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>(tiles, c.grid));
    c.ws_bytes = coop_arrays_bytes(m.ns) * (size_t)blocks;
  }
  c.use = true;
  return true;
}

// per-state arrays in shared memory where they fit, else in the workspace
static bool coop_fit(const DevMech& m, int warps, int ctas, int64_t n, CoopPlan& c) {
  const int64_t tiles = (n + kCoopTile - 1) / kCoopTile;
  return coop_shape(m, warps, ctas, true, tiles, c) || coop_shape(m, warps, ctas, false, tiles, c);
}

CoopPlan coop_plan(const DevMech& m, int fmt, int dt_bytes, int64_t n) {
  CoopPlan c{false, 16, 1, 0, 0, false, 0};
  const char* lay = getenv("PYJAC_GB_JAC_LAYOUT");
  if (lay && strcmp(lay, "percore") == 0) return c;
  if (lay && strcmp(lay, "coop") == 0) {
    const int warps = env_int("PYJAC_GB_COOP_WARPS", 16), ctas = env_int("PYJAC_GB_COOP_CTAS", 16 / std::max(warps, 1));
    const char* ar = getenv("PYJAC_GB_COOP_ARRAYS");
    if (ar && strcmp(ar, "global") == 0) coop_shape(m, warps, ctas, false, (n + kCoopTile - 1) / kCoopTile, c);
    else coop_fit(m, warps, ctas, n, c);
    return c;
  }
  const TmPlan t = tm_plan(m.ns);
  const int sms = sm_count();
  const int64_t tiles = (n + kCoopTile - 1) / kCoopTile;
  const bool percore_global = !t.use && plan_for(jacobian_arrays(), m.ns, n).global_ws;
  if (tiles <= sms) {  // one tile per SM at most: all 16 warps on it
    coop_fit(m, 16, 1, n, c);
    return c;
  }
  if (n < (int64_t)sms * 512 || t.use || percore_global) {
    if (t.use && fmt == PJ_DENSE && dt_bytes == 8 && n >= (int64_t)sms * 512) {
      c.use = false;  // the dense FP64 Jacobian: tensor memory, one state per thread
      return c;
    }
    if (dt_bytes == 4 && (t.use || percore_global)) coop_fit(m, 4, 4, n, c);
    else if (m.ns > 200) coop_fit(m, 16, 1, n, c);
    else coop_fit(m, 8, 2, n, c);
    return c;
  }
  c.use = false;
  return c;
}

size_t workspace_bytes(int arrays, int ns, int64_t n) {
  if (arrays == jacobian_arrays()) {
    // the most any layout can need: the one-state-per-thread plans, or the
    // cooperative one with its arrays in the workspace
    const TmPlan t = tm_plan(ns);
    const size_t pc = t.use ? t.ws_bytes : plan_for(arrays, ns, n).ws_bytes;
    // (any shape that may not fit its arrays in shared memory: at most 4
    // blocks per SM, since a block has 4 warps or more)
    const int64_t tiles =
        std::max<int64_t>(1, std::min<int64_t>((n + kCoopTile - 1) / kCoopTile, (int64_t)sm_count() * 4));
    const char* ar = getenv("PYJAC_GB_COOP_ARRAYS");
    const bool global = 4 * (coop_smem_bytes(ns, 4) + kBlockOverhead) > kSmemPerSm ||
                        coop_smem_bytes(ns, kCoopWarpsMax) > kSmemCap || (ar && strcmp(ar, "global") == 0);
    const size_t co = global ? coop_arrays_bytes(ns) * (size_t)tiles : 0;
    return std::max(pc, co);
  }
  return plan_for(arrays, ns, n).ws_bytes;
}

// Shared by the FP64 Jacobian and the FP32 Newton matrix: pick the layout,
// check the workspace, call the launcher of that layout and precision.
static int launch_jac_any(const DevMech& m, int mode, int fmt, int64_t n, const JacArgs& a, bool f32, void* work,
                          size_t work_bytes, cudaStream_t st) {
  const CoopPlan c = coop_plan(m, fmt, f32 ? 4 : 8, n);
  if (c.use) {
    if (c.ws_bytes && (!work || work_bytes < c.ws_bytes))
      return fail(PJ_ERR_NOMEM, "workspace too small for the Jacobian kernel (see pj_workspace_size)");
    return (f32 ? launch_jac_coop_f32 : launch_jac_coop_f64)(m, c, mode, fmt, n, a, static_cast<double*>(work),
                                                            st);
  }
  const TmPlan t = tm_plan(m.ns);
  if (t.use) {
    if (t.ws_bytes && (!work || work_bytes < t.ws_bytes))
      return fail(PJ_ERR_NOMEM, "workspace too small for the Jacobian kernel (see pj_workspace_size)");
    double* ws = static_cast<double*>(work);
    if (t.split == 2) return (f32 ? launch_jac_tm2_f32 : launch_jac_tm2_f64)(m, t, mode, fmt, n, a, ws, st);
    if (t.split == 1) return (f32 ? launch_jac_tm1_f32 : launch_jac_tm1_f64)(m, t, mode, fmt, n, a, ws, st);
    return (f32 ? launch_jac_tm0_f32 : launch_jac_tm0_f64)(m, t, mode, fmt, n, a, ws, st);
  }
  LaunchPlan p = plan_for(jacobian_arrays(), m.ns, n);
  if (p.global_ws && (!work || work_bytes < p.ws_bytes))
    return fail(PJ_ERR_NOMEM, "workspace too small for the Jacobian kernel (see pj_workspace_size)");
  double* ws = p.global_ws ? static_cast<double*>(work) : nullptr;
  return (f32 ? launch_jac_plain_f32 : launch_jac_plain_f64)(m, p, mode, fmt, n, a, ws, st);
}

int jacobian_layout(const DevMech& m, int fmt, bool f32, int64_t n) {
  if (coop_plan(m, fmt, f32 ? 4 : 8, n).use) return PJ_LAYOUT_COOP;
  return tm_plan(m.ns).use ? PJ_LAYOUT_TMEM : PJ_LAYOUT_PERCORE;
}

int launch_jacobian(const DevMech& m, int mode, int fmt, int64_t n, const double* param, const double* phi,
                    int64_t ld, double* J, double* dphi, int* status, void* work, size_t work_bytes,
                    cudaStream_t st) {
  const JacArgs a{param, phi, ld, J, dphi, status, nullptr, 0.0};
  return launch_jac_any(m, mode, fmt, n, a, false, work, work_bytes, st);
}

// Newton-iteration matrix M = I - h*gamma*J in FP32 (derivative arithmetic
// in FP32, rates and source terms in FP64).
int launch_newton_f32(const DevMech& m, int mode, int fmt, int64_t n, const double* param, const double* phi,
                      int64_t ld, const double* hstep, double gamma, float* M, double* dphi, int* status,
                      void* work, size_t work_bytes, cudaStream_t st) {
  const JacArgs a{param, phi, ld, M, dphi, status, hstep, gamma};
  return launch_jac_any(m, mode, fmt, n, a, true, work, work_bytes, st);
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
  const int64_t sm_cap = (int64_t)sm_count() * 4;
  if (cap > sm_cap) cap = sm_cap;
  p.grid = (int)(blocks < cap ? (blocks < 1 ? 1 : blocks) : cap);
  p.ws_stride = (int64_t)p.grid * p.tpb;
  p.ws_bytes = (size_t)jacobian_arrays() * m.ns * sizeof(double) * (size_t)p.ws_stride;
  const JacArgs a{param, phi, ld, J, dphi, status, nullptr, 0.0};
  return launch_jac_plain_f64(m, p, mode, fmt, n, a, scratch, st);
}
#endif  // PJ_NO_LAUNCHERS

}  // namespace pj
