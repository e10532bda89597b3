// Batched LU factorisation and solve of the Newton matrix M = I - h gamma J
// in the Jacobian's fixed pattern: the linear algebra an implicit
// integrator runs on the Jacobian (named as the missing piece in Sec. 5,
// which notes that library routines target one large matrix rather than many
// small ones).  The ordering, fill pattern and storage order are fixed per
// mechanism by lu_symbolic.cpp; no pivoting (M is the identity plus a small
// multiple of J for the step sizes of an implicit integrator).  A state
// whose factors are not all finite (a zero or non-finite pivot, or overflow,
// which FP32's range allows on stiff states) is counted in *status.
//
//  * Factorisation: S states per block (S = 2 or 4 when S dense matrices
//    still leave two blocks per SM, else 1).  M is scattered into a dense
//    N x N array (pivot order) in shared memory -- interleaved over the
//    block's states, so that one vector access moves an entry of all S -- or,
//    when N^2 does not fit, one state per block in a per-block slice of a
//    global workspace, and eliminated pivot by pivot with the per-pivot lists
//    of column rows and row columns: the block's threads tile the
//    |rows| x |cols| update, each pair (i, j) for all S states at once (the
//    index work and the loop are shared by the S states, whose fused
//    multiply-adds are independent).  The factors are gathered into the
//    storage order.
//  * Solve: one state per thread, streaming the factors in storage order
//    (coalesced across the warp), forward substitution then backward; the
//    solution sits in shared memory when N values per thread fit.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>

#include "kinetics_device.cuh"
#include "launch.h"
#include "pj_internal.h"

namespace pj {

template <typename T>
__device__ __forceinline__ T fma_t(T a, T b, T c) { return fma(a, b, c); }
template <>
__device__ __forceinline__ float fma_t<float>(float a, float b, float c) { return fmaf(a, b, c); }

// finiteness and zero tests on the bit pattern (integer instructions; the
// FP64 pipe is the bound of the factorisation)
__device__ __forceinline__ bool nonfinite_bits(double v) {
  return (__double_as_longlong(v) & 0x7ff0000000000000LL) == 0x7ff0000000000000LL;
}
__device__ __forceinline__ bool nonfinite_bits(float v) { return (__float_as_uint(v) & 0x7f800000u) == 0x7f800000u; }
__device__ __forceinline__ bool zero_bits(double v) { return (__double_as_longlong(v) << 1) == 0; }
__device__ __forceinline__ bool zero_bits(float v) { return (__float_as_uint(v) << 1) == 0u; }

template <typename T>
__device__ __forceinline__ bool bad_pivot(T p) { return zero_bits(p) || nonfinite_bits(p); }

// S values of one entry, one per state of the block, moved as one vector
template <typename T, int S>
struct LuVec;
template <typename T>
struct LuVec<T, 1> {
  using V = T;
};
template <>
struct LuVec<double, 2> {
  using V = double2;
};
template <>
struct LuVec<float, 2> {
  using V = float2;
};
template <>
struct LuVec<float, 4> {
  using V = float4;
};

template <typename V>
__device__ __forceinline__ V v_fms(V l, V u, V v);  // v - l u per component
template <>
__device__ __forceinline__ double v_fms(double l, double u, double v) {
  return fma(-l, u, v);
}
template <>
__device__ __forceinline__ float v_fms(float l, float u, float v) {
  return fmaf(-l, u, v);
}
template <>
__device__ __forceinline__ double2 v_fms(double2 l, double2 u, double2 v) {
  return make_double2(fma(-l.x, u.x, v.x), fma(-l.y, u.y, v.y));
}
template <>
__device__ __forceinline__ float2 v_fms(float2 l, float2 u, float2 v) {
  return make_float2(fmaf(-l.x, u.x, v.x), fmaf(-l.y, u.y, v.y));
}
template <>
__device__ __forceinline__ float4 v_fms(float4 l, float4 u, float4 v) {
  return make_float4(fmaf(-l.x, u.x, v.x), fmaf(-l.y, u.y, v.y), fmaf(-l.z, u.z, v.z), fmaf(-l.w, u.w, v.w));
}
template <typename V>
__device__ __forceinline__ V v_mul(V a, V b);
template <>
__device__ __forceinline__ double v_mul(double a, double b) {
  return a * b;
}
template <>
__device__ __forceinline__ float v_mul(float a, float b) {
  return a * b;
}
template <>
__device__ __forceinline__ double2 v_mul(double2 a, double2 b) {
  return make_double2(a.x * b.x, a.y * b.y);
}
template <>
__device__ __forceinline__ float2 v_mul(float2 a, float2 b) {
  return make_float2(a.x * b.x, a.y * b.y);
}
template <>
__device__ __forceinline__ float4 v_mul(float4 a, float4 b) {
  return make_float4(a.x * b.x, a.y * b.y, a.z * b.z, a.w * b.w);
}

// vals: CSR values of M (FROM_J = false) or of J (FROM_J: M = I - h gamma J
// formed on the way in, h per state).
template <typename T, bool FROM_J>
__global__ void __launch_bounds__(256) k_lu_factor(DevLu L, int64_t n, const T* __restrict__ vals, int64_t ld,
                                                   const double* __restrict__ hstep, double gamma,
                                                   T* __restrict__ lu, int* status, T* gws) {
  extern __shared__ __align__(16) unsigned char lu_smem[];
  const int N = L.N, NP = L.NP, tid = threadIdx.x, nt = blockDim.x;
  const int NN = N * NP;
  T* A = gws ? gws + (int64_t)blockIdx.x * NN : reinterpret_cast<T*>(lu_smem);
  __shared__ int bad;
  __shared__ T s_inv;
  for (int64_t s = blockIdx.x; s < n; s += gridDim.x) {
    if (tid == 0) bad = 0;
    for (int p = tid; p < NN; p += nt) A[p] = T(0);
    __syncthreads();
    const T hg = FROM_J ? T(-hstep[s] * gamma) : T(0);
    for (int e = tid; e < L.nnz; e += nt) {
      const T v = vals[(int64_t)e * ld + s];
      const int pos = __ldg(L.m2d + e);
      if (!PJ_DBG_OK(L.dbg, pos >= 0 && pos < NN, PJ_DBG_LU)) continue;
      A[pos] = FROM_J ? hg * v : v;
    }
    __syncthreads();
    if (FROM_J)
      for (int k = tid; k < N; k += nt) A[k * NP + k] += T(1);
    __syncthreads();
    // one thread forms each pivot's reciprocal ahead of its step (the FP64
    // pipe charges whole warps, so a division in every thread would cost as
    // much as a large part of the elimination)
    if (tid == 0) {
      const T piv = A[0];
      if (bad_pivot(piv)) bad = 1;
      s_inv = T(1) / piv;
    }
    __syncthreads();
    for (int k = 0; k < N; k++) {
      const T inv = s_inv;
      const int r0 = __ldg(L.rptr + k), nr = __ldg(L.rptr + k + 1) - r0;
      const int c0 = __ldg(L.cptr + k), nc = __ldg(L.cptr + k + 1) - c0;
      for (int a = tid; a < nr; a += nt) {
        const int i = __ldg(L.ridx + r0 + a);
        A[i * NP + k] *= inv;
      }
      __syncthreads();
      // the nr x nc update.  FP64: flattened over every thread so that warps
      // stay full (the FP64 pipe is the bound and charges idle lanes); pair
      // p = a * nc + c, walked with stride nt four pairs at a time (distinct
      // pairs touch distinct entries, so loads go out first).  FP32 (issue
      // bound): threads over columns, U_kj in a register, rows four at a time.
      const int tot = nr * nc;
      if (sizeof(T) == 4 && tot > 0) {
        const int per = nc >= nt ? 1 : nt / nc;
        const int a0 = nc >= nt ? 0 : tid / nc;
        for (int cj = nc >= nt ? tid : tid % nc; cj < nc && a0 < per; cj += nc >= nt ? nt : nc) {
          const int j = __ldg(L.cidx + c0 + cj);
          const T u = A[k * NP + j];
          int a = a0;
          for (; a + 3 * per < nr; a += 4 * per) {
            const int i0 = __ldg(L.ridx + r0 + a), i1 = __ldg(L.ridx + r0 + a + per);
            const int i2 = __ldg(L.ridx + r0 + a + 2 * per), i3 = __ldg(L.ridx + r0 + a + 3 * per);
            const T l0 = A[i0 * NP + k], l1 = A[i1 * NP + k], l2 = A[i2 * NP + k], l3 = A[i3 * NP + k];
            const T v0 = A[i0 * NP + j], v1 = A[i1 * NP + j], v2 = A[i2 * NP + j], v3 = A[i3 * NP + j];
            A[i0 * NP + j] = fma_t(-l0, u, v0);
            A[i1 * NP + j] = fma_t(-l1, u, v1);
            A[i2 * NP + j] = fma_t(-l2, u, v2);
            A[i3 * NP + j] = fma_t(-l3, u, v3);
          }
          for (; a < nr; a += per) {
            const int i = __ldg(L.ridx + r0 + a);
            A[i * NP + j] = fma_t(-A[i * NP + k], u, A[i * NP + j]);
          }
          if (nc < nt) break;  // one column per thread in that case
        }
      } else if (tid < tot) {
        const int di = nt / nc, dj = nt - di * nc;
        int ia = tid / nc, jc = tid - ia * nc;
        auto step = [&]() {
          ia += di;
          jc += dj;
          if (jc >= nc) {
            jc -= nc;
            ia++;
          }
        };
        int p = tid;
        for (; p + 3 * nt < tot; p += 4 * nt) {
          const int i0 = __ldg(L.ridx + r0 + ia), j0 = __ldg(L.cidx + c0 + jc);
          step();
          const int i1 = __ldg(L.ridx + r0 + ia), j1 = __ldg(L.cidx + c0 + jc);
          step();
          const int i2 = __ldg(L.ridx + r0 + ia), j2 = __ldg(L.cidx + c0 + jc);
          step();
          const int i3 = __ldg(L.ridx + r0 + ia), j3 = __ldg(L.cidx + c0 + jc);
          step();
          const T l0 = A[i0 * NP + k], l1 = A[i1 * NP + k], l2 = A[i2 * NP + k], l3 = A[i3 * NP + k];
          const T u0 = A[k * NP + j0], u1 = A[k * NP + j1], u2 = A[k * NP + j2], u3 = A[k * NP + j3];
          const T v0 = A[i0 * NP + j0], v1 = A[i1 * NP + j1], v2 = A[i2 * NP + j2], v3 = A[i3 * NP + j3];
          A[i0 * NP + j0] = fma_t(-l0, u0, v0);
          A[i1 * NP + j1] = fma_t(-l1, u1, v1);
          A[i2 * NP + j2] = fma_t(-l2, u2, v2);
          A[i3 * NP + j3] = fma_t(-l3, u3, v3);
        }
        for (; p < tot; p += nt) {
          const int i = __ldg(L.ridx + r0 + ia), j = __ldg(L.cidx + c0 + jc);
          A[i * NP + j] = fma_t(-A[i * NP + k], A[k * NP + j], A[i * NP + j]);
          step();
        }
      }
      __syncthreads();
      if (tid == 0) {
        A[k * NP + k] = inv;  // the diagonal slot stores 1 / U_kk
        if (k + 1 < N) {
          const T piv = A[(k + 1) * NP + k + 1];
          if (bad_pivot(piv)) bad = 1;
          s_inv = T(1) / piv;
        }
      }
      __syncthreads();
    }
    for (int e = tid; e < L.lu_nnz; e += nt) {
      const int pos = __ldg(L.l2d + e);
      if (!PJ_DBG_OK(L.dbg, pos >= 0 && pos < NN, PJ_DBG_LU)) continue;
      const T v = A[pos];
      if (nonfinite_bits(v)) bad = 1;  // overflow anywhere (FP32 range) marks the state
      lu[(int64_t)e * ld + s] = v;
    }
    __syncthreads();
    if (tid == 0 && bad && status) atomicAdd(status, 1);
    __syncthreads();
  }
}

// S states per block, the dense matrices interleaved in shared memory:
// A[p] holds entry p (pivot-order dense position, row stride NP) of the
// block's S states.  The elimination is that of k_lu_factor, value for value,
// for each state; a group's padding states (n not a multiple of S) factor
// the identity and are neither written nor counted.
//
// One barrier per pivot: when pivot k's update starts, column k already
// holds its multipliers L_ik = A_ik / U_kk and A_kk holds 1 / U_kk.  Warp 0
// takes column k+1 (the only column the next pivot scales): it applies pivot
// k's update to it, forms 1 / U_(k+1)(k+1), and scales the column -- the fill
// pattern is closed under elimination, so rows(k+1) holds every row of
// rows(k) but k+1 and no entry of the column changes after pivot k -- while
// the other warps update the pairs of every other column.
template <typename T, int S, bool FROM_J>
__global__ void __launch_bounds__(256) k_lu_factor_v(DevLu L, int64_t n, const T* __restrict__ vals, int64_t ld,
                                                     const double* __restrict__ hstep, double gamma,
                                                     T* __restrict__ lu, int* status) {
  using V = typename LuVec<T, S>::V;
  extern __shared__ __align__(16) unsigned char lu_smem[];
  V* A = reinterpret_cast<V*>(lu_smem);
  const int N = L.N, NP = L.NP, tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, warp = __shfl_sync(0xffffffffu, tid >> 5, 0);
  const int NN = N * NP;
  __shared__ int bad[S];
  __shared__ V s_inv;
  __shared__ T s_hg[S];
  auto at = [&](int p, int q) -> T& { return reinterpret_cast<T*>(A + p)[q]; };
  // warp 0: 1 / pivot c, lane q for state q (one warp instruction stream for
  // all S states), stored in the diagonal slot and broadcast; then column
  // c's entries below the pivot scaled by it
  auto finish_column = [&](int c) {
    if (lane < S) {
      const T piv = at(c * NP + c, lane);
      if (bad_pivot(piv)) bad[lane] = 1;
      const T r = T(1) / piv;
      reinterpret_cast<T*>(&s_inv)[lane] = r;
      at(c * NP + c, lane) = r;
    }
    __syncwarp();
    const V inv = s_inv;
    const int r0 = __ldg(L.rptr + c), nr = __ldg(L.rptr + c + 1) - r0;
    for (int a = lane; a < nr; a += 32) {
      const int i = __ldg(L.ridx + r0 + a);
      A[i * NP + c] = v_mul(A[i * NP + c], inv);
    }
  };
  const int64_t groups = (n + S - 1) / S;
  for (int64_t g = blockIdx.x; g < groups; g += gridDim.x) {
    const int64_t s0 = g * S;
    const int live = (int)(n - s0 < S ? n - s0 : S);
    if (tid < S) {
      bad[tid] = 0;
      s_hg[tid] = FROM_J && tid < live ? T(-hstep[s0 + tid] * gamma) : T(0);
    }
    for (int p = tid; p < NN * S; p += nt) reinterpret_cast<T*>(A)[p] = T(0);
    __syncthreads();
    // consecutive threads take the S states of one entry (adjacent in vals)
    for (int t = tid; t < L.nnz * S; t += nt) {
      const int e = t / S, q = t - e * S;
      const int pos = __ldg(L.m2d + e);
      if (q < live && PJ_DBG_OK(L.dbg, pos >= 0 && pos < NN, PJ_DBG_LU)) {
        const T v = vals[(int64_t)e * ld + s0 + q];
        at(pos, q) = FROM_J ? s_hg[q] * v : v;
      }
    }
    __syncthreads();
    for (int t = tid; t < N * S; t += nt) {
      const int k = t / S, q = t - k * S;
      if (FROM_J || q >= live) at(k * NP + k, q) += T(1);
    }
    __syncthreads();
    if (warp == 0) finish_column(0);
    __syncthreads();
    for (int k = 0; k < N - 1; k++) {
      const int r0 = __ldg(L.rptr + k), nr = __ldg(L.rptr + k + 1) - r0;
      const int c0 = __ldg(L.cptr + k), nc = __ldg(L.cptr + k + 1) - c0;
      // column k+1 is cols(k)[0] when pivot k changes it (columns ascend)
      const int j0 = nc > 0 && __ldg(L.cidx + c0) == k + 1 ? 1 : 0;
      if (warp == 0) {
        if (j0) {
          const V u = A[k * NP + k + 1];
          for (int a = lane; a < nr; a += 32) {
            const int i = __ldg(L.ridx + r0 + a);
            A[i * NP + k + 1] = v_fms(A[i * NP + k], u, A[i * NP + k + 1]);
          }
          __syncwarp();
        }
        finish_column(k + 1);
      } else {
        // the nr x (nc - j0) update of the other columns, flattened over the
        // other warps: pair p = a * ncw + c, four pairs at a time (distinct
        // pairs touch distinct entries, so their loads go out first)
        const int ncw = nc - j0, tot = nr * ncw, ntw = nt - 32;
        int p = tid - 32;
        if (p < tot) {
          const int di = ntw / ncw, dj = ntw - di * ncw;
          int ia = p / ncw, jc = p - ia * ncw;
          auto step = [&]() {
            ia += di;
            jc += dj;
            if (jc >= ncw) {
              jc -= ncw;
              ia++;
            }
          };
          const int* __restrict__ ci = L.cidx + c0 + j0;
          for (; p + 3 * ntw < tot; p += 4 * ntw) {
            const int i0 = __ldg(L.ridx + r0 + ia), jj0 = __ldg(ci + jc);
            step();
            const int i1 = __ldg(L.ridx + r0 + ia), jj1 = __ldg(ci + jc);
            step();
            const int i2 = __ldg(L.ridx + r0 + ia), jj2 = __ldg(ci + jc);
            step();
            const int i3 = __ldg(L.ridx + r0 + ia), jj3 = __ldg(ci + jc);
            step();
            const V l0 = A[i0 * NP + k], l1 = A[i1 * NP + k], l2 = A[i2 * NP + k], l3 = A[i3 * NP + k];
            const V u0 = A[k * NP + jj0], u1 = A[k * NP + jj1], u2 = A[k * NP + jj2], u3 = A[k * NP + jj3];
            const V v0 = A[i0 * NP + jj0], v1 = A[i1 * NP + jj1], v2 = A[i2 * NP + jj2], v3 = A[i3 * NP + jj3];
            A[i0 * NP + jj0] = v_fms(l0, u0, v0);
            A[i1 * NP + jj1] = v_fms(l1, u1, v1);
            A[i2 * NP + jj2] = v_fms(l2, u2, v2);
            A[i3 * NP + jj3] = v_fms(l3, u3, v3);
          }
          for (; p < tot; p += ntw) {
            const int i = __ldg(L.ridx + r0 + ia), j = __ldg(ci + jc);
            A[i * NP + j] = v_fms(A[i * NP + k], A[k * NP + j], A[i * NP + j]);
            step();
          }
        }
      }
      __syncthreads();
    }
    for (int t = tid; t < L.lu_nnz * S; t += nt) {
      const int e = t / S, q = t - e * S;
      const int pos = __ldg(L.l2d + e);
      if (q < live && PJ_DBG_OK(L.dbg, pos >= 0 && pos < NN, PJ_DBG_LU)) {
        const T v = at(pos, q);
        if (nonfinite_bits(v)) bad[q] = 1;
        lu[(int64_t)e * ld + s0 + q] = v;
      }
    }
    __syncthreads();
    if (tid < live && bad[tid] && status) atomicAdd(status, 1);
    __syncthreads();
  }
}

// x may alias b.  X: the solution of this thread's state, in shared memory
// (stride blockDim.x) or in x itself (stride ld).
template <typename T, bool SMEM_X>
__global__ void __launch_bounds__(128) k_lu_solve(DevLu L, int64_t n, const T* __restrict__ lu, int64_t ld,
                                                  const T* b, T* x) {
  extern __shared__ __align__(16) unsigned char lu_smem[];
  const int N = L.N;
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
    T* X = SMEM_X ? reinterpret_cast<T*>(lu_smem) + threadIdx.x : x + s;
    const int64_t xs = SMEM_X ? blockDim.x : ld;
    // sum over storage entries [e, e1) of value * X[column], four independent
    // partial sums so that the factor loads stream; FP32 takes eight entries
    // a step (eight loads in flight: 17 % faster at 111 species; FP64 was
    // slower that way)
    auto dot = [&](int e, int e1) -> T {
      T p0 = T(0), p1 = T(0), p2 = T(0), p3 = T(0);
      for (; sizeof(T) == 4 && e + 7 < e1; e += 8) {
        const int c0 = __ldg(L.xcol + e), c1 = __ldg(L.xcol + e + 1);
        const int c2 = __ldg(L.xcol + e + 2), c3 = __ldg(L.xcol + e + 3);
        const int c4 = __ldg(L.xcol + e + 4), c5 = __ldg(L.xcol + e + 5);
        const int c6 = __ldg(L.xcol + e + 6), c7 = __ldg(L.xcol + e + 7);
        const T v0 = lu[(int64_t)e * ld + s], v1 = lu[(int64_t)(e + 1) * ld + s];
        const T v2 = lu[(int64_t)(e + 2) * ld + s], v3 = lu[(int64_t)(e + 3) * ld + s];
        const T v4 = lu[(int64_t)(e + 4) * ld + s], v5 = lu[(int64_t)(e + 5) * ld + s];
        const T v6 = lu[(int64_t)(e + 6) * ld + s], v7 = lu[(int64_t)(e + 7) * ld + s];
        p0 = fma_t(v0, X[(int64_t)c0 * xs], p0);
        p1 = fma_t(v1, X[(int64_t)c1 * xs], p1);
        p2 = fma_t(v2, X[(int64_t)c2 * xs], p2);
        p3 = fma_t(v3, X[(int64_t)c3 * xs], p3);
        p0 = fma_t(v4, X[(int64_t)c4 * xs], p0);
        p1 = fma_t(v5, X[(int64_t)c5 * xs], p1);
        p2 = fma_t(v6, X[(int64_t)c6 * xs], p2);
        p3 = fma_t(v7, X[(int64_t)c7 * xs], p3);
      }
      for (; e + 3 < e1; e += 4) {
        const int c0 = __ldg(L.xcol + e), c1 = __ldg(L.xcol + e + 1);
        const int c2 = __ldg(L.xcol + e + 2), c3 = __ldg(L.xcol + e + 3);
        p0 = fma_t(lu[(int64_t)e * ld + s], X[(int64_t)c0 * xs], p0);
        p1 = fma_t(lu[(int64_t)(e + 1) * ld + s], X[(int64_t)c1 * xs], p1);
        p2 = fma_t(lu[(int64_t)(e + 2) * ld + s], X[(int64_t)c2 * xs], p2);
        p3 = fma_t(lu[(int64_t)(e + 3) * ld + s], X[(int64_t)c3 * xs], p3);
      }
      for (; e < e1; e++) p0 = fma_t(lu[(int64_t)e * ld + s], X[(int64_t)__ldg(L.xcol + e) * xs], p0);
      return (p0 + p1) + (p2 + p3);
    };
    // forward: y_k = b_perm[k] - sum_{j<k} L_kj y_j, y kept at X[perm[k]]
    for (int k = 0; k < N; k++) {
      const int pk = __ldg(L.perm + k);
      const T bk = b[(int64_t)pk * ld + s];
      X[(int64_t)pk * xs] = bk - dot(__ldg(L.lptr + k), __ldg(L.lptr + k + 1));
    }
    // backward: z_k = (y_k - sum_{j>k} U_kj z_j) / U_kk
    for (int q = 0; q < N; q++) {
      const int e0 = __ldg(L.uptr + q), e1 = __ldg(L.uptr + q + 1);
      const int pk = __ldg(L.perm + (N - 1 - q));
      const T yk = X[(int64_t)pk * xs];
      X[(int64_t)pk * xs] = (yk - dot(e0 + 1, e1)) * lu[(int64_t)e0 * ld + s];
    }
    if (SMEM_X)
      for (int v = 0; v < N; v++) x[(int64_t)v * ld + s] = X[(int64_t)v * xs];
  }
}

// ---------------------------------------------------------------------------
// launch planning
// ---------------------------------------------------------------------------
struct LuPlan {
  bool smem;        // dense matrix in shared memory
  int S;            // states per block (1, 2 or 4; shared-memory plans only)
  int threads;      // per block
  int grid;         // persistent blocks
  size_t dyn;       // shared memory per block
  size_t ws_bytes;  // global workspace when !smem
};

static LuPlan lu_plan(int N, size_t esize, int64_t n) {
  LuPlan p{};
  const size_t dense = (size_t)N * (size_t)(N | 1) * esize;
  const int64_t states = std::max<int64_t>(n, 1);
  if (dense <= kSmemCap) {
    p.smem = true;
    // the most states per block (16-byte vectors: 2 FP64, 4 FP32) that still
    // leave two blocks per SM
    p.S = 1;
    for (int S : {4, 2}) {
      if (S * esize > 16) continue;
      if (2 * (S * dense + 1024 + 256) <= kSmemPerSm && S * dense <= kSmemCap) {
        p.S = S;
        break;
      }
    }
    p.dyn = dense * p.S;
    const int ctas = std::max(1, std::min(16, (int)(kSmemPerSm / (p.dyn + 1024 + 256))));
    int warps = (32 + ctas - 1) / ctas;  // 32 warps per SM where blocks of 256 allow (53 species: 11 % over 16)
    warps = std::max(2, std::min(8, warps));  // warp 0 finishes columns, the others update
    p.threads = 32 * warps;
    p.grid = (int)std::min<int64_t>((states + p.S - 1) / p.S, (int64_t)sm_count() * ctas);
    p.ws_bytes = 0;
  } else {
    p.smem = false;
    p.S = 1;
    p.dyn = 0;
    p.threads = 256;
    p.grid = (int)std::min<int64_t>(states, (int64_t)sm_count() * 2);
    p.ws_bytes = dense * (size_t)((int64_t)sm_count() * 2);
  }
  return p;
}

size_t lu_workspace_bytes(int N, int prec, int64_t n) {
  return lu_plan(N, prec == PJ_F32 ? sizeof(float) : sizeof(double), n).ws_bytes;
}

template <typename T>
static int launch_factor_t(const DevLu& L, int64_t n, const void* vals, int64_t ld, const double* hstep,
                           double gamma, void* lu, int* status, void* work, size_t work_bytes, cudaStream_t st) {
  const LuPlan p = lu_plan(L.N, sizeof(T), n);
  if (!p.smem && (!work || work_bytes < p.ws_bytes))
    return fail(PJ_ERR_NOMEM, "workspace too small for the LU factorisation (see pj_workspace_size)");
  T* gws = p.smem ? nullptr : static_cast<T*>(work);
  int rc;
  if (p.smem) {
    auto pick = [&](auto kern) -> int {
      int r;
      if ((r = set_smem(kern, p.dyn))) return r;
      kern<<<p.grid, p.threads, p.dyn, st>>>(L, n, static_cast<const T*>(vals), ld, hstep, gamma,
                                             static_cast<T*>(lu), status);
      return check_cuda(cudaGetLastError(), "k_lu_factor_v launch");
    };
    if constexpr (sizeof(T) == 4) {
      if (p.S == 4) return hstep ? pick(k_lu_factor_v<T, 4, true>) : pick(k_lu_factor_v<T, 4, false>);
    }
    if (p.S == 2) return hstep ? pick(k_lu_factor_v<T, 2, true>) : pick(k_lu_factor_v<T, 2, false>);
    return hstep ? pick(k_lu_factor_v<T, 1, true>) : pick(k_lu_factor_v<T, 1, false>);
  }
  if (hstep) {
    auto kern = k_lu_factor<T, true>;
    if ((rc = set_smem(kern, p.dyn))) return rc;
    kern<<<p.grid, p.threads, p.dyn, st>>>(L, n, static_cast<const T*>(vals), ld, hstep, gamma,
                                           static_cast<T*>(lu), status, gws);
  } else {
    auto kern = k_lu_factor<T, false>;
    if ((rc = set_smem(kern, p.dyn))) return rc;
    kern<<<p.grid, p.threads, p.dyn, st>>>(L, n, static_cast<const T*>(vals), ld, hstep, gamma,
                                           static_cast<T*>(lu), status, gws);
  }
  return check_cuda(cudaGetLastError(), "k_lu_factor launch");
}

int launch_lu_factor(const DevLu& L, int prec, int64_t n, const void* vals, int64_t ld, const double* hstep,
                     double gamma, void* lu, int* status, void* work, size_t work_bytes, cudaStream_t st) {
  if (prec == PJ_F32) return launch_factor_t<float>(L, n, vals, ld, hstep, gamma, lu, status, work, work_bytes, st);
  return launch_factor_t<double>(L, n, vals, ld, hstep, gamma, lu, status, work, work_bytes, st);
}

template <typename T>
static int launch_solve_t(const DevLu& L, int64_t n, const void* lu, int64_t ld, const void* b, void* x,
                          cudaStream_t st) {
  const size_t xs_bytes = (size_t)L.N * sizeof(T) * 128;
  const bool smem_x = xs_bytes <= 200 * 1024;
  const int64_t blocks = (n + 127) / 128;
  int rc;
  if (smem_x) {
    auto kern = k_lu_solve<T, true>;
    if ((rc = set_smem(kern, xs_bytes))) return rc;
    int occ = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, 128, xs_bytes) != cudaSuccess || occ < 1) occ = 1;
    const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(blocks, (int64_t)sm_count() * occ));
    kern<<<(unsigned)grid, 128, xs_bytes, st>>>(L, n, static_cast<const T*>(lu), ld, static_cast<const T*>(b),
                                                static_cast<T*>(x));
  } else {
    auto kern = k_lu_solve<T, false>;
    const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(blocks, (int64_t)sm_count() * 16));
    kern<<<(unsigned)grid, 128, 0, st>>>(L, n, static_cast<const T*>(lu), ld, static_cast<const T*>(b),
                                         static_cast<T*>(x));
  }
  return check_cuda(cudaGetLastError(), "k_lu_solve launch");
}

int launch_lu_solve(const DevLu& L, int prec, int64_t n, const void* lu, int64_t ld, const void* b, void* x,
                    cudaStream_t st) {
  if (prec == PJ_F32) return launch_solve_t<float>(L, n, lu, ld, b, x, st);
  return launch_solve_t<double>(L, n, lu, ld, b, x, st);
}

}  // namespace pj
