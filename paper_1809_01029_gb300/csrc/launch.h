// Host-side launch planning shared by the translation units that launch
// kernels: where each state's working arrays live (shared memory, TMEM or a
// global workspace), how many blocks are resident, and the launcher entry
// points behind the C ABI.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "pj_internal.h"

namespace pj {

// Per-state arrays in shared memory (blocks of tpb threads) or, when 128
// threads' arrays do not fit, in a global workspace of ws_stride threads
// walked grid-stride.
struct LaunchPlan {
  int tpb;
  int grid;
  size_t smem;
  bool global_ws;
  int64_t ws_stride;
  size_t ws_bytes;
};

// TMEM layout of the Jacobian kernel: h_k/RT in TMEM (2 columns per species),
// C_k and g_k/RT split between shared memory and a global workspace.
struct TmPlan {
  bool use;
  uint32_t ncols;   // TMEM columns per block
  int split;        // state arrays in shared memory (2: C and G; 1: C; 0: none)
  int ctas;         // resident blocks per SM
  size_t smem;      // dynamic shared memory per block
  size_t ws_bytes;  // global workspace (0 when split == 2)
  int grid;         // 0: one block per 128 states; else the persistent grid
};

// Cooperative Jacobian layout (k_jacobian_coop): `warps` warps per block
// share a tile of 32 states, `ctas` blocks per SM, a persistent grid of
// `grid` blocks walking the tiles.
struct CoopPlan {
  bool use;
  int warps;
  int ctas;
  size_t smem;
  int grid;
  bool wide_regs;   // 8 warps, one block per SM, up to 255 registers a thread
  size_t ws_bytes;  // per-state arrays in a global workspace (grid x 3 Ns x 32
                    // doubles); 0: in shared memory
};

// Tiles of several batches handed out by a block counter (the batched
// plans), instead of consecutive tiles of the one batch a launch is given.
struct CoopBatch {
  const double* param;
  const double* phi;
  double* out;
  double* dphi;
  int64_t n, ld;
};
struct CoopSrc {
  const CoopBatch* batches;     // null: the launch's own batch
  const int64_t* tile_start;    // [nb + 1] first tile of each batch
  int nb;
  unsigned long long* counter;  // zeroed before the launch
};

// Shape the cooperative layout: `warps` (4, 8, 16) warps per block, `ctas`
// blocks per SM, per-state arrays in shared memory (arrays_smem) or in a
// global workspace; false when it does not fit.  tiles bounds the grid.
bool coop_shape(const DevMech& m, int warps, int ctas, bool arrays_smem, int64_t tiles, CoopPlan& c);

constexpr size_t kSmemPerSm = 228 * 1024;                    // shared memory per SM
constexpr size_t kSmemCap = 225 * 1024;                      // per block, less the 2 KB exp table
constexpr size_t kBlockOverhead = 1024 + 2048 + 64;          // driver reserve, exp table, TMEM base
// resident blocks of 128 threads the Jacobian kernels are compiled for
// (their launch bound: at most 128 registers a thread); measured 8-14 %
// faster than the compiler's own choice of 168 registers and three blocks
constexpr int kJacRegCtas = 4;

int sm_count();
int source_arrays();
int jacobian_arrays();
LaunchPlan plan_for(int arrays, int ns, int64_t n);
TmPlan tm_plan(int ns);
CoopPlan coop_plan(const DevMech& m, int fmt, int dt_bytes, int64_t n);
int jacobian_layout(const DevMech& m, int fmt, bool f32, int64_t n);   // PJ_LAYOUT_*
size_t workspace_bytes(int arrays, int ns, int64_t n);
size_t form_workspace_bytes(int op, const DevMech& m, int64_t n);

int check_common(const char* fn, const pj_mech* m, int mode, int64_t n, int64_t ld, const void* param,
                 const void* phi, const void* out);

int launch_source(const DevMech& m, int mode, int64_t n, const double* param, const double* phi, int64_t ld,
                  double* out, int* status, void* work, size_t work_bytes, cudaStream_t st);
int launch_jacobian(const DevMech& m, int mode, int fmt, int64_t n, const double* param, const double* phi,
                    int64_t ld, double* J, double* dphi, int* status, void* work, size_t work_bytes,
                    cudaStream_t st);
int launch_newton_f32(const DevMech& m, int mode, int fmt, int64_t n, const double* param, const double* phi,
                      int64_t ld, const double* hstep, double gamma, float* M, double* dphi, int* status,
                      void* work, size_t work_bytes, cudaStream_t st);
int launch_jacobian_on_scratch(const DevMech& m, int mode, int fmt, int64_t n, const double* param,
                               const double* phi, int64_t ld, double* J, double* dphi, int* status,
                               double* scratch, int64_t scratch_threads, cudaStream_t st);
int launch_fd_jacobian(const DevMech& m, int mode, int fmt, int64_t n, const double* param, const double* phi,
                       int64_t ld, double* J, double* dphi, int* status, void* work, size_t work_bytes,
                       cudaStream_t st);
size_t fd_workspace_bytes(int ns, int64_t n);
int launch_lu_factor(const DevLu& L, int prec, int64_t n, const void* vals, int64_t ld, const double* hstep,
                     double gamma, void* lu, int* status, void* work, size_t work_bytes, cudaStream_t st);
int launch_lu_solve(const DevLu& L, int prec, int64_t n, const void* lu, int64_t ld, const void* b, void* x,
                    cudaStream_t st);
size_t lu_workspace_bytes(int N, int prec, int64_t n);
int launch_diag_exp(const DevMech& m, int64_t n, const double* x, double* y_ours, double* y_lib, cudaStream_t st);
int launch_eval_y(const DevMech& m, int mode, int64_t n, const double* param, const double* phi, int64_t ld,
                  double* y, int* status, void* work, size_t work_bytes, cudaStream_t st);
int launch_vjp(const DevMech& m, int mode, int64_t n, const double* param, const double* phi, int64_t ld,
               const double* u_wdot, const double* u_T, double* y, double* g_phi, double* g_theta, int* status,
               void* work, size_t work_bytes, cudaStream_t st);

// Arguments of one Jacobian launch; J is double* (FP64 Jacobian) or float*
// (FP32 Newton matrix, with hstep and gamma).
struct JacArgs {
  const double* param;
  const double* phi;
  int64_t ld;
  void* J;
  double* dphi;
  int* status;
  const double* hstep;
  double gamma;
  CoopSrc src;  // cooperative layout only; zero: tiles of this batch
};

// Jacobian launchers, one translation unit each (jacobian_inst.cu built once
// per layout and precision).
int launch_jac_plain_f64(const DevMech& m, const LaunchPlan& p, int mode, int fmt, int64_t n, const JacArgs& a,
                         double* ws, cudaStream_t st);
int launch_jac_plain_f32(const DevMech& m, const LaunchPlan& p, int mode, int fmt, int64_t n, const JacArgs& a,
                         double* ws, cudaStream_t st);
int launch_jac_tm0_f64(const DevMech& m, const TmPlan& p, int mode, int fmt, int64_t n, const JacArgs& a,
                       double* ws, cudaStream_t st);
int launch_jac_tm1_f64(const DevMech& m, const TmPlan& p, int mode, int fmt, int64_t n, const JacArgs& a,
                       double* ws, cudaStream_t st);
int launch_jac_tm2_f64(const DevMech& m, const TmPlan& p, int mode, int fmt, int64_t n, const JacArgs& a,
                       double* ws, cudaStream_t st);
int launch_jac_tm0_f32(const DevMech& m, const TmPlan& p, int mode, int fmt, int64_t n, const JacArgs& a,
                       double* ws, cudaStream_t st);
int launch_jac_tm1_f32(const DevMech& m, const TmPlan& p, int mode, int fmt, int64_t n, const JacArgs& a,
                       double* ws, cudaStream_t st);
int launch_jac_tm2_f32(const DevMech& m, const TmPlan& p, int mode, int fmt, int64_t n, const JacArgs& a,
                       double* ws, cudaStream_t st);
int launch_jac_coop_f64(const DevMech& m, const CoopPlan& p, int mode, int fmt, int64_t n, const JacArgs& a,
                        double* ws, cudaStream_t st);
int launch_jac_coop_f32(const DevMech& m, const CoopPlan& p, int mode, int fmt, int64_t n, const JacArgs& a,
                        double* ws, cudaStream_t st);

// Raise a kernel's dynamic shared-memory limit when it asks for more than
// the default 48 KB.
template <typename K>
inline int set_smem(K kern, size_t smem) {
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) {
      cudaGetLastError();  // not sticky: clear it so the next launch check does not report it
      return check_cuda(e, "cudaFuncSetAttribute");
    }
  }
  return PJ_OK;
}

// A grid-stride plan over a global workspace launches only as many blocks
// as can be resident at once (a multiple of the SM count), so that no block
// runs as a second, nearly empty wave.
template <typename K>
inline LaunchPlan resident_grid(K kern, const LaunchPlan& p) {
  if (!p.global_ws) return p;
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, p.tpb, p.smem) != cudaSuccess || occ < 1) return p;
  LaunchPlan q = p;
  const int64_t cap = (int64_t)sm_count() * occ;
  if (q.grid > cap) {
    q.grid = (int)cap;
    q.ws_stride = (int64_t)q.grid * q.tpb;
  }
  return q;
}

}  // namespace pj
