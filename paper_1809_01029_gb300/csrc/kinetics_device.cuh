// Device helpers shared by the source-term, Jacobian and derived-form kernels.
#pragma once

#include <cuda_runtime.h>

#include "pj_internal.h"

namespace pj {

// Per-state working arrays: element (a, k) of the calling thread's state sits
// at base[(a*ns + k) * stride].  base/stride point either into shared memory
// (stride = blockDim.x) or into a global workspace (stride = total threads).
struct StateArrays {
  double* base;
  int64_t stride;
  int ns;
  __device__ __forceinline__ double& at(int a, int k) const { return base[(int64_t)(a * ns + k) * stride]; }
};

// NASA-7 block of species k for temperature T (low range iff T < T_mid).
__device__ __forceinline__ const double* nasa_block(const DevMech& m, int k, double T) {
  const double* b = m.nasa + (size_t)k * NASA_STRIDE;
  const double tmid = __ldg(b + 14);
  return T < tmid ? b : b + 16;
}

// cp/R, h/RT, s/R (NASA 7-coefficient polynomials).
__device__ __forceinline__ void nasa_eval(const double* __restrict__ c, double T, double invT, double lnT,
                                          double& cp, double& h, double& s) {
  const double a0 = __ldg(c + 0), a1 = __ldg(c + 1), a2 = __ldg(c + 2), a3 = __ldg(c + 3), a4 = __ldg(c + 4);
  cp = fma(fma(fma(fma(a4, T, a3), T, a2), T, a1), T, a0);
  h = fma(fma(fma(fma(__ldg(c + 10), T, __ldg(c + 9)), T, __ldg(c + 8)), T, __ldg(c + 7)), T, a0) + __ldg(c + 5) * invT;
  s = fma(a0, lnT, fma(fma(fma(fma(__ldg(c + 13), T, __ldg(c + 12)), T, __ldg(c + 11)), T, a1), T, __ldg(c + 6)));
}

// cp/R and d(cp/R)/dT
__device__ __forceinline__ void nasa_cp(const double* __restrict__ c, double T, double& cp, double& dcp) {
  const double a1 = __ldg(c + 1), a2 = __ldg(c + 2), a3 = __ldg(c + 3), a4 = __ldg(c + 4);
  cp = fma(fma(fma(fma(a4, T, a3), T, a2), T, a1), T, __ldg(c + 0));
  dcp = fma(fma(fma(4.0 * a4, T, 3.0 * a3), T, 2.0 * a2), T, a1);
}

// x^n for a small non-negative integer n (stoichiometric coefficients)
__device__ __forceinline__ double powi(double x, int n) {
  double r = 1.0;
  for (int i = 0; i < n; i++) r *= x;
  return r;
}

__device__ __forceinline__ void write_nan_state(double* out, int64_t ld, int64_t s, int rows) {
  const double qnan = __longlong_as_double(0x7ff8000000000000ULL);
  if (out)
    for (int v = 0; v < rows; v++) out[(int64_t)v * ld + s] = qnan;
}

}  // namespace pj
