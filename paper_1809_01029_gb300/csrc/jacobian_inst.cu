// Instantiates the Jacobian kernels for one (layout, precision) pair.  The
// build compiles this file once per pair, with
//   PJ_INST_TM   -1: k_jacobian (arrays in shared memory or a workspace);
//                0, 1, 2: k_jacobian_tm with that many of C_k, g_k/RT in
//                shared memory; 3: k_jacobian_coop (32-state tiles);
//   PJ_INST_F32  0: FP64 Jacobian; 1: FP32 Newton matrix M = I - h gamma J;
//   PJ_INST_NAME the launcher this unit defines (declared in launch.h),
// so that the instantiations compile in parallel.
#include "jacobian_kernels.cuh"

#if !defined(PJ_INST_TM) || !defined(PJ_INST_F32) || !defined(PJ_INST_NAME)
#error "compile with -DPJ_INST_TM=<-1|0|1|2|3> -DPJ_INST_F32=<0|1> -DPJ_INST_NAME=<launcher>"
#endif

namespace pj {

#if PJ_INST_F32
using InstDT = float;
constexpr bool kInstNewton = true;
#else
using InstDT = double;
constexpr bool kInstNewton = false;
#endif

#if PJ_INST_TM == 3
using InstPlan = CoopPlan;
template <int MODE, int FMT>
static int inst_launch(const DevMech& m, const InstPlan& p, int64_t n, const JacArgs& a, double* ws,
                       cudaStream_t st) {
  if (m.nr_plain < m.nr) return launch_jac_coop_s<MODE, FMT, InstDT, kInstNewton, true>(m, p, n, a, ws, st);
  return launch_jac_coop_s<MODE, FMT, InstDT, kInstNewton, false>(m, p, n, a, ws, st);
}
#elif PJ_INST_TM < 0
using InstPlan = LaunchPlan;
template <int MODE, int FMT>
static int inst_launch(const DevMech& m, const InstPlan& p, int64_t n, const JacArgs& a, double* ws,
                       cudaStream_t st) {
  if (m.nr_plain < m.nr) return launch_jac_t<MODE, FMT, InstDT, kInstNewton, true>(m, p, n, a, ws, st);
  return launch_jac_t<MODE, FMT, InstDT, kInstNewton, false>(m, p, n, a, ws, st);
}
#else
using InstPlan = TmPlan;
template <int MODE, int FMT>
static int inst_launch(const DevMech& m, const InstPlan& p, int64_t n, const JacArgs& a, double* ws,
                       cudaStream_t st) {
  if (m.nr_plain < m.nr) return launch_jac_tm_s<MODE, FMT, InstDT, kInstNewton, PJ_INST_TM, true>(m, p, n, a, ws, st);
  return launch_jac_tm_s<MODE, FMT, InstDT, kInstNewton, PJ_INST_TM, false>(m, p, n, a, ws, st);
}
#endif

int PJ_INST_NAME(const DevMech& m, const InstPlan& p, int mode, int fmt, int64_t n, const JacArgs& a, double* ws,
                 cudaStream_t st) {
  if (mode == PJ_CONP) {
    if (fmt == PJ_CSR) return inst_launch<PJ_CONP, PJ_CSR>(m, p, n, a, ws, st);
    if (fmt == PJ_CSC) return inst_launch<PJ_CONP, PJ_CSC>(m, p, n, a, ws, st);
    return inst_launch<PJ_CONP, PJ_DENSE>(m, p, n, a, ws, st);
  }
  if (fmt == PJ_CSR) return inst_launch<PJ_CONV, PJ_CSR>(m, p, n, a, ws, st);
  if (fmt == PJ_CSC) return inst_launch<PJ_CONV, PJ_CSC>(m, p, n, a, ws, st);
  return inst_launch<PJ_CONV, PJ_DENSE>(m, p, n, a, ws, st);
}

}  // namespace pj
