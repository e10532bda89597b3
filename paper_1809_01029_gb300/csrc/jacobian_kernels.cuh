// The analytical Jacobian kernels (Sec. 2.2, assembled as in Sec. 3.4):
// k_jacobian keeps each state's C_k, g_k/RT and h_k/RT in shared memory or a
// global workspace; k_jacobian_tm keeps h_k/RT in tensor memory (both call
// jacobian_state for one state per thread); k_jacobian_coop lets the warps
// of a block share a tile of 32 states.  Included by jacobian_inst.cu,
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

// ---------------------------------------------------------------------------
// Cooperative Jacobian: the W warps of a block evaluate one tile of 32 states
// together (lane l of every warp works on state 32*tile + l) and split the
// work of each state among themselves: the species of the thermo pass, the
// reactions (handed out one at a time from a shared counter), the species
// of the source-term pass and the columns of the energy and state rows.
// Each state's C_k,
// g_k/RT and h_k/RT sit once in shared memory ([array][k][lane]: a warp's
// access to one species is 32 consecutive doubles, conflict-free).
//
// Why: the Jacobian entries are accumulated by L2 reductions.  With one
// state per thread, every resident thread keeps a whole Jacobian live in L2
// for the length of its reaction loop; at 53 species that is ~1.4 GB across
// the GPU, so the reductions miss and each entry travels to DRAM and back
// several times.  Here a block keeps only 32 Jacobians live (one block of
// 16 warps per SM: ~90 MB for the 53-species CSR Jacobian, within L2; two
// blocks of 8 warps: twice that) with the same number of threads per SM.
//
// Cross-warp sums (the bath-gas concentration, the energy-equation
// denominator, the energy/state-row weights, the source-term sums) go
// through per-warp partials in shared memory added in warp order.  Jacobian
// entries and production rates receive L2 reductions from several warps, so
// their rounding can differ between runs by the order of the additions
// (the values agree to the accuracy of the sum, not bit for bit).
// ---------------------------------------------------------------------------
constexpr int kCoopTile = 32;  // states per block (one per lane)
constexpr int kCoopWarpsMax = 16;
// per-state scalars, [kCoopSc][32] doubles
enum CoopSc {
  cT, cV, cP, cInvT, cInvV, cLnT, cLnP, cCtot, cCdum, cCxB, cDcpB, cDen, cDdenT, cDdenS, cDCbT, cDCbS,
  // the energy and state rows' per-state values (JacRowVars)
  cIden, cTdot, cRtvp, cCT, cJ00, cJ01, cX0, cX1, cAT_T, cAT_S, cAS_T, cAS_S, cATB, cASB, kCoopSc
};
// per-warp partial sums, [W][kCoopPart][32] doubles
enum CoopPart { pAcc, pDen, pDden, pNum, pSum, pOm, pAT_T, pAT_S, pAS_T, pAS_S, pATB, pASB, pWb, kCoopPart };

// per-state flags (int): valid T, V, P; valid state
enum CoopFlag { fOk0, fOk, kCoopFlag };

// per-state arrays C_k, g_k/RT then Cx_k, h_k/RT of a tile: [3][Ns][32] doubles
__host__ __device__ constexpr size_t coop_arrays_bytes(int ns) {
  return (size_t)3 * ns * kCoopTile * sizeof(double);
}

__host__ __device__ constexpr size_t coop_smem_bytes(int ns, int warps, bool arrays_smem = true) {
  return (arrays_smem ? coop_arrays_bytes(ns) : 0) +
         (size_t)(kCoopSc + kCoopPart * warps) * kCoopTile * sizeof(double) +
         (size_t)(kCoopFlag * kCoopTile + 2) * sizeof(int);
}

// An L2 cache policy of priority evict_last for a whole access, and a store
// of zero with it (createpolicy / st.global.L2::cache_hint).
__device__ __forceinline__ uint64_t l2_policy_evict_last() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ void st_zero_evict_last(double* a, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.b64 [%0], 0, %1;" ::"l"(a), "l"(pol) : "memory");
}
__device__ __forceinline__ void st_zero_evict_last(float* a, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.b32 [%0], 0, %1;" ::"l"(a), "l"(pol) : "memory");
}

// MAXW: the most warps a block of this instance has (launch bound MAXW * 32
// threads, one block per SM guaranteed): 16 caps registers at 128 per
// thread, 8 allows 255.
// aws: the per-state arrays of each block's tile in a global workspace
// (mechanisms too large for shared memory), else null.  src.batches: tiles
// of several batches from a counter, else the tiles of (n, param, phi, ...).
template <int MODE, int FMT, typename DT, bool NEWTON, bool SPECIAL, int MAXW, bool BATCHED = false>
__global__ void __launch_bounds__(MAXW * 32, 1)
    k_jacobian_coop(DevMech m, int64_t n0, const double* __restrict__ param0, const double* __restrict__ phi0,
                    int64_t ld0, DT* __restrict__ J0, double* __restrict__ dphi0, int* status,
                    const double* __restrict__ hstep, double gamma, double* __restrict__ aws, CoopSrc src) {
  PJ_DYN_SMEM;
  __shared__ int64_t s_tile;
  load_exp_table(m.exp_tab);
  const uint64_t l2_last = l2_policy_evict_last();
  const int ns = m.ns, N = m.N, bath = m.ns - 1;
  // the warp index broadcast from lane 0, so that the compiler knows it (and
  // the reaction index derived from it) to be warp-uniform: reaction records
  // are then read and branched on as uniform values
  const int lane = threadIdx.x & 31, warp = __shfl_sync(0xffffffffu, (int)(threadIdx.x >> 5), 0);
  const int W = blockDim.x >> 5;
  const int64_t n_out = FMT == PJ_DENSE ? (int64_t)N * N : (int64_t)m.nnz;
  double* const tsm = aws ? smem : smem + 3 * ns * kCoopTile;                     // the tile's scalars and sums
  double* __restrict__ sc = tsm + lane;                                            // sc[v*32]
  double* __restrict__ part = tsm + kCoopSc * kCoopTile + lane;                    // part[(w*kCoopPart + v)*32]
  int* __restrict__ flags = reinterpret_cast<int*>(tsm + (kCoopSc + kCoopPart * W) * kCoopTile);
  int* __restrict__ next_rxn = flags + kCoopFlag * kCoopTile;  // the next reaction to hand out
  auto F = [&](int v) -> int& { return flags[v * kCoopTile + lane]; };
  auto S = [&](int v) -> double& { return sc[v * kCoopTile]; };
  auto Pw = [&](int w, int v) -> double& { return part[(w * kCoopPart + v) * kCoopTile]; };
  auto sum_parts = [&](int v) {
    double t = 0.0;
    for (int w = 0; w < W; w++) t += Pw(w, v);
    return t;
  };
  StateArrays A;
  A.ns = ns;
  A.base = aws ? aws + (int64_t)blockIdx.x * 3 * ns * kCoopTile + lane : smem + lane;
  A.stride = kCoopTile;
  enum { aC = 0, aG = 1, aH = 2 };

  for (int64_t it = blockIdx.x;; it += gridDim.x) {
    int64_t tile = it, n = n0, ld = ld0;
    const double* __restrict__ param = param0;
    const double* __restrict__ phi = phi0;
    DT* __restrict__ J = J0;
    double* __restrict__ dphi = dphi0;
    if constexpr (BATCHED) {
      // the next tile of the plan (read by every thread before the block's
      // next barrier, rewritten only after several more)
      if (threadIdx.x == 0) s_tile = (int64_t)atomicAdd(src.counter, 1ULL);
      __syncthreads();
      tile = s_tile;
      if (tile >= __ldg(src.tile_start + src.nb)) break;
      int lo = 0, hi = src.nb - 1;  // the batch holding it: the last b with tile_start[b] <= tile
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(src.tile_start + mid) <= tile) lo = mid;
        else hi = mid - 1;
      }
      const CoopBatch B = src.batches[lo];
      tile -= __ldg(src.tile_start + lo);
      n = B.n;
      ld = B.ld;
      param = B.param;
      phi = B.phi;
      J = reinterpret_cast<DT*>(B.out);
      dphi = B.dphi;
    } else if (tile * kCoopTile >= n) {
      break;
    }
    const int64_t s = tile * kCoopTile + lane;
    const bool act = s < n;
    double* __restrict__ wrow = dphi + 2 * ld + s;

    // A: the state's scalars (warp 0; a lane past the batch or with an
    // invalid T, V or P takes a dummy state); zero the outputs (all warps)
    if (warp == 0) {
      double T = 1000.0, V = 1.0, P = 1e5;
      bool ok0 = false;
      if (act) {
        const double T_ = phi[s], S_ = phi[ld + s], par = param[s];
        const double V_ = MODE == PJ_CONP ? S_ : par, P_ = MODE == PJ_CONP ? par : S_;
        ok0 = (T_ > 0.0) && (V_ > 0.0) && (P_ > 0.0) && isfinite(T_) && isfinite(V_) && isfinite(P_);
        if (ok0) {
          T = T_;
          V = V_;
          P = P_;
        }
      }
      S(cT) = T;
      S(cV) = V;
      S(cP) = P;
      S(cInvT) = 1.0 / T;
      S(cInvV) = 1.0 / V;
      S(cLnT) = log(T);
      S(cLnP) = m.has_pdep ? log(P) : 0.0;
      const double Ctot = P / (RU * T);
      S(cCtot) = Ctot;
      S(cCdum) = Ctot / ns;     // a dummy state's concentrations
      F(fOk0) = ok0;
      if (lane == 0) *next_rxn = W;  // reactions 0 .. W-1 go to warps 0 .. W-1
    }
    if (act) {
      // zeros stored with L2 priority evict_last: the tile's lines, which
      // its reductions will touch again, outlast the lines of finished
      // tiles (DRAM traffic per state at 53 species: 44 -> 34 KB at 16 x 1,
      // 73 -> 65 KB at 8 x 2, same speed); the reductions' own accesses
      // are of normal priority
      for (int64_t e = warp; e < n_out; e += W) st_zero_evict_last(J + e * ld + s, l2_last);
      for (int k = warp; k < ns - 1; k += W) wrow[(int64_t)k * ld] = 0.0;
    }
    __syncthreads();

    // B: concentrations and thermo of the warp's species
    {
      const double T = S(cT), V = S(cV), invT = S(cInvT), lnT = S(cLnT), cdum = S(cCdum);
      const bool ok0 = F(fOk0) != 0;
      double acc = 0.0, den = 0.0, dden = 0.0;
      for (int k = warp; k < ns; k += W) {
        const double* cb = nasa_block(m, k, T);
        double cp, h, sr, cp2, dcp;
        nasa_eval(cb, T, invT, lnT, cp, h, sr);
        nasa_cp(cb, T, cp2, dcp);
        A.at(aG, k) = h - sr;
        A.at(aH, k) = h;
        const double cx = MODE == PJ_CONP ? cp : cp - 1.0;
        if (k < bath) {
          const double c = ok0 ? phi[(int64_t)(k + 2) * ld + s] / V : cdum;
          A.at(aC, k) = c;
          acc += c;
          den = fma(c, cx, den);
          dden = fma(c, dcp, dden);
        } else {
          S(cCxB) = cx;
          S(cDcpB) = dcp;
        }
      }
      Pw(warp, pAcc) = acc;
      Pw(warp, pDen) = den;
      Pw(warp, pDden) = dden;
    }
    __syncthreads();

    // C: bath gas by subtraction, validity, denominator of the energy
    // equation and the bath-gas derivatives (warp 0)
    if (warp == 0) {
      const double Ctot = S(cCtot), P = S(cP), invT = S(cInvT), invV = S(cInvV);
      const double acc = sum_parts(pAcc);
      const double Cns = Ctot - acc;
      const bool ok = F(fOk0) != 0 && isfinite(acc) && isfinite(Cns) && !(Cns < -1e-12 * Ctot);
      A.at(aC, bath) = Cns;
      F(fOk) = ok;
      const double den = RU * (sum_parts(pDen) + Cns * S(cCxB));
      const double Cx_bath = RU * S(cCxB);
      const double dCb_T = -Ctot * invT;
      const double dCb_S = MODE == PJ_CONP ? (Ctot - Cns) * invV : Ctot / P;
      S(cDen) = den;
      S(cDCbT) = dCb_T;
      S(cDCbS) = dCb_S;
      S(cDdenT) = RU * (sum_parts(pDden) + Cns * S(cDcpB)) + Cx_bath * dCb_T;
      S(cDdenS) = MODE == PJ_CONP ? (Cx_bath * Ctot - den) * invV : Cx_bath * Ctot / P;
      if (__any_sync(0xffffffffu, act && !ok)) {
        if (act && !ok) {
          const DT qnan = DT(__longlong_as_double(0x7ff8000000000000ULL));
          for (int64_t e = 0; e < n_out; e++) J[e * ld + s] = qnan;
          write_nan_state(dphi, ld, s, ns + 1);
          if (status) atomicAdd(status, 1);
        }
      }
    }
    __syncthreads();

    // D: the warp's reactions (i = warp, warp + W, ...)
    const bool w = F(fOk) != 0;
    const JacOut<DT> o{J, wrow, ld, s, w, NEWTON && w ? DT(-hstep[s] * gamma) : DT(0)};
    {
      JacVars<DT> v;
      v.T = S(cT);
      v.V = S(cV);
      v.P = S(cP);
      v.invT = S(cInvT);
      v.lnT = S(cLnT);
      v.lnP = S(cLnP);
      v.Ctot = S(cCtot);
      v.invT2 = v.invT * v.invT;
      v.invV = S(cInvV);
      v.logPRT = m.log_pstd_over_r - v.lnT;
      v.dCb_T = S(cDCbT);
      v.dCb_S = S(cDCbS);
      v.AT_T = v.AT_S = v.AS_T = v.AS_S = v.ATB = v.ASB = DT(0);
      v.w_bath = 0.0;
      // reactions are handed out one at a time (a shared counter), so that
      // warps finish the phase within about one reaction of each other
      for (int i = warp; i < m.nr;) {
        if (!SPECIAL || i < m.nr_plain) jac_reaction<MODE, FMT, DT, false, false, NEWTON>(m, A, v, o, i, 0u);
        else jac_reaction<MODE, FMT, DT, true, false, NEWTON>(m, A, v, o, i, 0u);
        int nx = 0;
        if (lane == 0) nx = atomicAdd(next_rxn, 1);
        i = __shfl_sync(0xffffffffu, nx, 0);
      }
      Pw(warp, pAT_T) = double(v.AT_T);
      Pw(warp, pAT_S) = double(v.AT_S);
      Pw(warp, pAS_T) = double(v.AS_T);
      Pw(warp, pAS_S) = double(v.AS_S);
      Pw(warp, pATB) = double(v.ATB);
      Pw(warp, pASB) = double(v.ASB);
      Pw(warp, pWb) = v.w_bath;
    }
    __syncthreads();

    // E: source-term pass over the warp's species (G becomes Cx_k)
    {
      const double T = S(cT), V = S(cV);
      double num = 0.0, sumCxW = 0.0, Om = 0.0;
      for (int k = warp; k < ns; k += W) {
        const double wb = k == bath ? sum_parts(pWb) : 0.0;
        A.at(aG, k) = jac_species<MODE, FMT, DT, NEWTON>(m, k, T, V, A.at(aH, k), wb, o, num, sumCxW, Om);
      }
      Pw(warp, pNum) = num;
      Pw(warp, pSum) = sumCxW;
      Pw(warp, pOm) = Om;
    }
    __syncthreads();

    // F: totals of the per-warp sums; warp 0 also forms the source terms of T
    // and S and the per-state values of the energy and state rows
    if (warp == 0) {
      const double T = S(cT), V = S(cV), P = S(cP), invT = S(cInvT), den = S(cDen);
      const double num = sum_parts(pNum), sumCxW = sum_parts(pSum), Om = sum_parts(pOm);
      const double Tdot = -(num * (RU * T)) / den;
      if (w) {
        dphi[s] = Tdot;
        dphi[ld + s] = MODE == PJ_CONP ? V * Tdot * invT + (RU * T * V / P) * Om : P * Tdot * invT + RU * T * Om;
      }
      const JacRowVars<DT> x = jac_row_vars<MODE, DT>(T, V, P, invT, Tdot, Om, den, S(cDdenT), S(cDdenS), sumCxW,
                                                      A.at(aG, bath), DT(0), DT(0), DT(0), DT(0), DT(0), DT(0));
      S(cIden) = double(x.iden);
      S(cTdot) = double(x.Tdot);
      S(cRtvp) = double(x.rtvp);
      S(cCT) = double(x.cT);
      S(cJ00) = double(x.j00);
      S(cJ01) = double(x.j01);
      S(cX0) = double(x.x0);
      S(cX1) = double(x.x1);
    }
    for (int t = warp - 1; t >= 0 && t < 6; t += W - 1) {  // warps 1 .. W-1 (W >= 2)
      const int from[6] = {pAT_T, pAT_S, pAS_T, pAS_S, pATB, pASB};
      const int to[6] = {cAT_T, cAT_S, cAS_T, cAS_S, cATB, cASB};
      S(to[t]) = sum_parts(from[t]);
    }
    __syncthreads();

    // G: the warp's columns of rows 0 and 1
    {
      JacRowVars<DT> x;
      x.Cx_b = A.at(aG, bath);
      x.iden = DT(S(cIden));
      x.Tdot = DT(S(cTdot));
      x.invV = DT(S(cInvV));
      x.rtvp = DT(S(cRtvp));
      x.cT = DT(S(cCT));
      x.j00 = DT(S(cJ00));
      x.j01 = DT(S(cJ01));
      x.x0 = DT(S(cX0));
      x.x1 = DT(S(cX1));
      x.AT_T = DT(S(cAT_T));
      x.AT_S = DT(S(cAT_S));
      x.AS_T = DT(S(cAS_T));
      x.AS_S = DT(S(cAS_S));
      x.ATB = DT(S(cATB));
      x.ASB = DT(S(cASB));
      // columns j = warp, warp + W, ...: warps 0 and 1 take the T and S
      // columns first (W >= 4), every other column is a species column
      int j = warp;
      if (j == 0) {
        jac_ts_column<MODE, FMT, DT, NEWTON, 0>(m, 0, 0.0, x, o);
        j += W;
      } else if (j == 1) {
        jac_ts_column<MODE, FMT, DT, NEWTON, 1>(m, 1, 0.0, x, o);
        j += W;
      }
      for (; j < N; j += W) jac_ts_column<MODE, FMT, DT, NEWTON, 2>(m, j, A.at(aG, j - 2), x, o);
    }

    if (NEWTON) {
      // the identity on the species diagonal once every entry is complete
      __syncthreads();
      for (int k = warp + 2; k < N; k += W) newton_species_diagonal<FMT>(m, k, o);
    }
    __syncthreads();
  }
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

template <int MODE, int FMT, typename DT, bool NEWTON, bool SPECIAL>
static int launch_jac_coop_s(const DevMech& m, const CoopPlan& c, int64_t n, const JacArgs& a, double* ws,
                             cudaStream_t st) {
  // the batched plans' tile hand-out is an instance of its own (FP64
  // Jacobian, up to 16 warps), so that the other instances carry none of its
  // registers
  auto kern = a.src.batches ? k_jacobian_coop<MODE, FMT, DT, NEWTON, SPECIAL, kCoopWarpsMax, !NEWTON>
              : c.wide_regs ? k_jacobian_coop<MODE, FMT, DT, NEWTON, SPECIAL, 8>
                            : k_jacobian_coop<MODE, FMT, DT, NEWTON, SPECIAL, kCoopWarpsMax>;
  if (NEWTON && a.src.batches) return fail(PJ_ERR_UNSUPPORTED, "batched plans compute the FP64 Jacobian only");
  int rc;
  if ((rc = set_smem(kern, c.smem))) return rc;
  // n: the states of the launch's batch, or (batched) 32 x the plan's tiles
  const int64_t tiles = (n + kCoopTile - 1) / kCoopTile;
  const int64_t grid = tiles < c.grid ? (tiles < 1 ? 1 : tiles) : c.grid;
  kern<<<(unsigned)grid, c.warps * 32, c.smem, st>>>(m, n, a.param, a.phi, a.ld, static_cast<DT*>(a.J), a.dphi,
                                                     a.status, a.hstep, a.gamma, c.ws_bytes ? ws : nullptr,
                                                     a.src);
  return check_cuda(cudaGetLastError(), "k_jacobian_coop launch");
}
#endif  // PJ_NO_LAUNCHERS

}  // namespace pj
