// Device helpers shared by the source-term, Jacobian and derived-form kernels.
#pragma once

#include <cuda_runtime.h>

#include "pj_internal.h"

namespace pj {

// Bounds-checked build (compiled with -DPJ_DEBUG_BOUNDS): every lookup in an
// index table derived at mechanism load -- the per-reaction target lists,
// the full -> sparse position maps, the species-row and efficiency lists,
// the LU scatter / gather maps -- is checked before use.  A bad index sets a
// bit of the mechanism's device error word (pj_debug_word) and is replaced
// by a harmless one (the access is skipped), so a corrupted table shows as a
// nonzero word, never as an out-of-range access or a trap.  Without the
// macro the checks compile to nothing.
enum : uint32_t { PJ_DBG_TARGET = 1, PJ_DBG_POSMAP = 2, PJ_DBG_ROWS = 4, PJ_DBG_EFF = 8, PJ_DBG_LU = 16 };
#ifdef PJ_DEBUG_BOUNDS
__device__ __forceinline__ bool pj_dbg_ok(uint32_t* word, bool ok, uint32_t bit) {
  if (!ok && word) atomicOr(word, bit);
  return ok;
}
#define PJ_DBG_OK(word, cond, bit) pj_dbg_ok((word), (cond), (bit))
#else
#define PJ_DBG_OK(word, cond, bit) true
#endif

// Per-state working arrays: element (a, k) of the calling thread's state sits
// at base[(a*ns + k) * stride].  base/stride point either into shared memory
// (stride = blockDim.x) or into a global workspace (stride = total threads).
// Per-state arrays of one thread (C_k, g_k/RT, h_k/RT, ...): array a of
// species k sits at base[(a*ns + k)*stride] for a < SPLIT and at
// base2[((a - SPLIT)*ns + k)*stride2] otherwise, so a kernel can keep the
// first arrays in shared memory and the rest in a global workspace.  Array
// indices are compile-time constants at every use, so the choice folds away.
template <int SPLIT>
struct StateArraysT {
  double* base;
  int64_t stride;
  int ns;
  double* base2;
  int64_t stride2;
  __device__ __forceinline__ double& at(int a, int k) const {
    return a < SPLIT ? base[(int64_t)(a * ns + k) * stride] : base2[(int64_t)((a - SPLIT) * ns + k) * stride2];
  }
};
using StateArrays = StateArraysT<8>;

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

// ---------------------------------------------------------------------------
// FP64 exponential after P. T. P. Tang, "Table-driven implementation of the
// exponential function in IEEE floating-point arithmetic", ACM TOMS 15 (1989):
//   x = (256 m + j) ln2/256 + r,  |r| <= ln2/512,
//   exp(x) = 2^m * 2^(j/256) * (1 + p(r)),  p(r) = r + r^2/2 + r^3/6 + r^4/24,
// with a two-part (Cody-Waite) reduction constant so that k * LN2_256_HI is
// exact, the 256-entry table in shared memory, and the power of two applied by
// adding m to the exponent field.  About 9 FP64 operations instead of the
// library's ~16 issue slots; outside |x| < 704 (overflow, underflow,
// subnormal results, NaN) it defers to the library exp.  Error <= 1 ulp,
// checked against CUDA's exp by the diagnostic entry point pj_diag_exp.
// Every kernel that calls pj_exp fills the table first (load_exp_table).
// ---------------------------------------------------------------------------
#ifndef PJ_EXP_TABLE_DECL
__shared__ double pj_exp_tab[256];
#define PJ_EXP_TABLE_DECL
#endif

__device__ __forceinline__ void load_exp_table(const double* __restrict__ g) {
#ifdef PJ_EXP_TABLE_LOAD_ALL
  for (int i = 0; i < 256; i++) pj_exp_tab[i] = g[i];
#else
  for (int i = threadIdx.x; i < 256; i += blockDim.x) pj_exp_tab[i] = __ldg(g + i);
  __syncthreads();
#endif
}

__device__ __forceinline__ double pj_exp(double x) {
  const double SHIFT = 6755399441055744.0;            // 1.5 * 2^52: rounds to an integer in the low bits
  const double INV_LN2_256 = 0x1.71547652b82fep+8;    // 256 / ln 2
  const double LN2_256_HI = 0x1.62e42fefc0000p-9;     // ln 2 / 256, 35 significant bits
  const double LN2_256_LO = -0x1.c610ca86c3899p-45;   // ln 2 / 256 - LN2_256_HI
  if ((__double2hiint(x) & 0x7fffffff) >= 0x40860000) return exp(x);  // |x| >= 704 or NaN
  const double t = fma(x, INV_LN2_256, SHIFT);
  const int k = __double2loint(t);
  const double kd = t - SHIFT;
  double r = fma(-kd, LN2_256_HI, x);
  r = fma(-kd, LN2_256_LO, r);
  const double poly = fma(fma(r, 1.0 / 24.0, 1.0 / 6.0), r, 0.5);
  const double p = fma(r * r, poly, r);
  const double T = pj_exp_tab[k & 255];
  const double res = fma(T, p, T);
  return __longlong_as_double(__double_as_longlong(res) + ((long long)(k >> 8) << 52));
}

// ---------------------------------------------------------------------------
// Tensor memory (TMEM) as per-thread storage.  A CTA of 128 threads allocates
// `ncols` 32-bit columns across the SM's 128 TMEM lanes; thread t of warp w
// owns lane 32*(w%4) + (t%32), so element c of its row is at
// base + ((32*(w%4)) << 16) + c.  Warps read and write their 32 lanes with
// warp-collective tcgen05.ld / tcgen05.st of one (warp-uniform) column pair,
// the access pattern of per-state arrays indexed by a reaction's species.
// ---------------------------------------------------------------------------
#ifndef PJ_TMEM_EMU
__device__ __forceinline__ void tmem_alloc(uint32_t* dst_smem, uint32_t ncols) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(dst_smem);
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(a), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tmem_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tmem_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tmem_st_f64(uint32_t taddr, double v) {
  const uint32_t lo = (uint32_t)__double2loint(v), hi = (uint32_t)__double2hiint(v);
  asm volatile("tcgen05.st.sync.aligned.32x32b.x2.b32 [%0], {%1, %2};" ::"r"(taddr), "r"(lo), "r"(hi) : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
// load one double and wait for it (the wait names the registers so that no
// use can be scheduled before it)
__device__ __forceinline__ double tmem_ld_f64(uint32_t taddr) {
  uint32_t lo, hi;
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0, %1}, [%2];" : "=r"(lo), "=r"(hi) : "r"(taddr) : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" : "+r"(lo), "+r"(hi)::"memory");
  return __hiloint2double((int)hi, (int)lo);
}
#endif

}  // namespace pj
