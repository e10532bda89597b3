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
//  * Factorisation: one state per block.  M is scattered into a dense N x N
//    array (pivot order) in shared memory -- or, when N^2 does not fit, in a
//    per-block slice of a global workspace -- and eliminated pivot by pivot
//    with the per-pivot lists of column rows and row columns: the block's
//    threads tile the |rows| x |cols| update (threads over columns, keeping
//    U_kj in a register, and over rows).  The factors are gathered into the
//    storage order.
//  * Solve: one state per thread, streaming the factors in storage order
//    (coalesced across the warp), forward substitution then backward; the
//    solution sits in shared memory when N values per thread fit.
#include <cuda_runtime.h>

#include <algorithm>

#include "launch.h"
#include "pj_internal.h"

namespace pj {

template <typename T>
__device__ __forceinline__ T fma_t(T a, T b, T c) { return fma(a, b, c); }
template <>
__device__ __forceinline__ float fma_t<float>(float a, float b, float c) { return fmaf(a, b, c); }

template <typename T>
__device__ __forceinline__ bool bad_pivot(T p) { return !(p != T(0)) || !isfinite(p); }

// vals: CSR values of M (FROM_J = false) or of J (FROM_J: M = I - h gamma J
// formed on the way in, h per state).
template <typename T, bool FROM_J>
__global__ void __launch_bounds__(256) k_lu_factor(DevLu L, int64_t n, const T* __restrict__ vals, int64_t ld,
                                                   const double* __restrict__ hstep, double gamma,
                                                   T* __restrict__ lu, int* status, T* gws) {
  extern __shared__ __align__(16) unsigned char lu_smem[];
  const int N = L.N, tid = threadIdx.x, nt = blockDim.x;
  const int NN = N * N;
  T* A = gws ? gws + (int64_t)blockIdx.x * NN : reinterpret_cast<T*>(lu_smem);
  __shared__ int bad;
  for (int64_t s = blockIdx.x; s < n; s += gridDim.x) {
    if (tid == 0) bad = 0;
    for (int p = tid; p < NN; p += nt) A[p] = T(0);
    __syncthreads();
    const T hg = FROM_J ? T(-hstep[s] * gamma) : T(0);
    for (int e = tid; e < L.nnz; e += nt) {
      const T v = vals[(int64_t)e * ld + s];
      A[__ldg(L.m2d + e)] = FROM_J ? hg * v : v;
    }
    __syncthreads();
    if (FROM_J)
      for (int k = tid; k < N; k += nt) A[k * N + k] += T(1);
    __syncthreads();
    for (int k = 0; k < N; k++) {
      const T piv = A[k * N + k];
      const T inv = T(1) / piv;
      const int r0 = __ldg(L.rptr + k), nr = __ldg(L.rptr + k + 1) - r0;
      const int c0 = __ldg(L.cptr + k), nc = __ldg(L.cptr + k + 1) - c0;
      for (int a = tid; a < nr; a += nt) {
        const int i = __ldg(L.ridx + r0 + a);
        A[i * N + k] *= inv;
      }
      __syncthreads();
      if (nr > 0 && nc > 0) {
        if (nc >= nt) {
          for (int cj = tid; cj < nc; cj += nt) {
            const int j = __ldg(L.cidx + c0 + cj);
            const T u = A[k * N + j];
            for (int a = 0; a < nr; a++) {
              const int i = __ldg(L.ridx + r0 + a);
              A[i * N + j] = fma_t(-A[i * N + k], u, A[i * N + j]);
            }
          }
        } else {
          const int per = nt / nc;
          const int cj = tid % nc, a0 = tid / nc;
          if (a0 < per) {
            const int j = __ldg(L.cidx + c0 + cj);
            const T u = A[k * N + j];
            for (int a = a0; a < nr; a += per) {
              const int i = __ldg(L.ridx + r0 + a);
              A[i * N + j] = fma_t(-A[i * N + k], u, A[i * N + j]);
            }
          }
        }
      }
      __syncthreads();
      if (tid == 0) {
        if (bad_pivot(piv)) bad = 1;
        A[k * N + k] = inv;  // the diagonal slot stores 1 / U_kk
      }
      __syncthreads();
    }
    for (int e = tid; e < L.lu_nnz; e += nt) {
      const T v = A[__ldg(L.l2d + e)];
      if (!isfinite(v)) bad = 1;  // overflow anywhere (FP32 range) marks the state
      lu[(int64_t)e * ld + s] = v;
    }
    __syncthreads();
    if (tid == 0 && bad && status) atomicAdd(status, 1);
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
    // forward: y_k = b_perm[k] - sum_{j<k} L_kj y_j, y kept at X[perm[k]]
    for (int k = 0; k < N; k++) {
      const int pk = __ldg(L.perm + k);
      T acc = b[(int64_t)pk * ld + s];
      for (int e = __ldg(L.lptr + k), e1 = __ldg(L.lptr + k + 1); e < e1; e++)
        acc = fma_t(-lu[(int64_t)e * ld + s], X[(int64_t)__ldg(L.xcol + e) * xs], acc);
      X[(int64_t)pk * xs] = acc;
    }
    // backward: z_k = (y_k - sum_{j>k} U_kj z_j) / U_kk
    for (int q = 0; q < N; q++) {
      const int e0 = __ldg(L.uptr + q), e1 = __ldg(L.uptr + q + 1);
      const int pk = __ldg(L.perm + (N - 1 - q));
      T acc = X[(int64_t)pk * xs];
      for (int e = e0 + 1; e < e1; e++)
        acc = fma_t(-lu[(int64_t)e * ld + s], X[(int64_t)__ldg(L.xcol + e) * xs], acc);
      X[(int64_t)pk * xs] = acc * lu[(int64_t)e0 * ld + s];
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
  int threads;      // per block
  int grid;         // persistent blocks
  size_t dyn;       // shared memory per block
  size_t ws_bytes;  // global workspace when !smem
};

static LuPlan lu_plan(int N, size_t esize, int64_t n) {
  LuPlan p{};
  const size_t dense = (size_t)N * N * esize;
  const int64_t states = std::max<int64_t>(n, 1);
  if (dense <= kSmemCap) {
    p.smem = true;
    p.dyn = dense;
    const int ctas = std::max(1, std::min(16, (int)(kSmemPerSm / (dense + 1024 + 256))));
    int warps = (8 + ctas - 1) / ctas;  // at least 8 warps per SM
    warps = std::max(1, std::min(8, warps));
    p.threads = 32 * warps;
    p.grid = (int)std::min<int64_t>(states, (int64_t)sm_count() * ctas);
    p.ws_bytes = 0;
  } else {
    p.smem = false;
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
