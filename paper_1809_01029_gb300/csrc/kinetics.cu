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

#include "kinetics_device.cuh"

#ifndef PJ_DYN_SMEM
#define PJ_DYN_SMEM extern __shared__ double smem[]
#endif

namespace pj {

struct StateScalars {
  double T, V, P, invT, lnT, Ctot;
};

// Load one state, fill C_k (k < Ns-1 as n_k/V; the bath gas as C_tot minus
// the others summed in species order) and check validity.
template <int MODE>
__device__ __forceinline__ bool load_state(const DevMech& m, const double* __restrict__ phi,
                                           const double* __restrict__ param, int64_t ld, int64_t s,
                                           const StateArrays& A, int aC, StateScalars& st) {
  const int ns = m.ns;
  const double T = phi[s], S = phi[ld + s], par = param[s];
  const double V = MODE == PJ_CONP ? S : par;
  const double P = MODE == PJ_CONP ? par : S;
  bool ok = (T > 0.0) && (V > 0.0) && (P > 0.0) && isfinite(T) && isfinite(V) && isfinite(P);
  double acc = 0.0;
  for (int k = 0; k < ns - 1; k++) {
    const double c = phi[(int64_t)(k + 2) * ld + s] / V;
    A.at(aC, k) = c;
    acc += c;
  }
  const double Ctot = P / (RU * T);
  const double Cns = Ctot - acc;
  A.at(aC, ns - 1) = Cns;
  ok = ok && isfinite(acc) && isfinite(Cns) && !(Cns < -1e-12 * Ctot);
  st.T = T;
  st.V = V;
  st.P = P;
  st.invT = 1.0 / T;
  st.lnT = log(T);
  st.Ctot = Ctot;
  return ok;
}

// Troe / SRI broadening factor F(T, Pr).  With derivatives also returns
// FxPr = Pr dF/dPr (at fixed T) and FT = dF/dT (at fixed Pr).
template <bool DERIV>
__device__ __forceinline__ double falloff_F(const Rxn* __restrict__ r, int kind, double T, double invT,
                                            double lnT, double Pr, double& FxPr, double& FT) {
  FxPr = 0.0;
  FT = 0.0;
  if (kind == PJ_TROE) {
    const double a = __ldg(&r->fp[0]), iT3 = __ldg(&r->fp[1]), iT1 = __ldg(&r->fp[2]);
    const double T2 = __ldg(&r->fp[3]), has2 = __ldg(&r->fp[4]);
    const double e3 = exp(-T * iT3), e1 = exp(-T * iT1);
    const double e2 = has2 != 0.0 ? exp(-T2 * invT) : 0.0;
    const double Fcent = (1.0 - a) * e3 + a * e1 + e2;
    const double L = log10(Fcent);
    const double x = log10(Pr);
    const double cc = -0.4 - 0.67 * L;
    const double NN = 0.75 - 1.27 * L;
    const double xc = x + cc;
    const double D = NN - 0.14 * xc;
    const double f1 = xc / D;
    const double g = 1.0 / (1.0 + f1 * f1);
    const double F = exp(LN10 * (L * g));
    if (DERIV) {
      const double iD2 = 1.0 / (D * D);
      const double m2fg2 = -2.0 * f1 * g * g;
      const double dlg_dx = L * m2fg2 * NN * iD2;
      const double dlg_dL = g + L * m2fg2 * (-0.67 * D + 1.1762 * xc) * iD2;
      const double dFcent = -(1.0 - a) * iT3 * e3 - a * iT1 * e1 + T2 * invT * invT * e2;
      FxPr = F * dlg_dx;
      FT = F * dlg_dL * dFcent / Fcent;
    }
    return F;
  }
  if (kind == PJ_SRI) {
    const double a = __ldg(&r->fp[0]), b = __ldg(&r->fp[1]), ic = __ldg(&r->fp[2]);
    const double d = __ldg(&r->fp[3]), e = __ldg(&r->fp[4]);
    const double x = log10(Pr);
    const double X = 1.0 / (1.0 + x * x);
    const double eb = exp(-b * invT), ec = exp(-T * ic);
    const double Z = a * eb + ec;
    const double lnZ = log(Z);
    const double F = d * exp(X * lnZ + e * lnT);
    if (DERIV) {
      FxPr = F * (lnZ * (-2.0 * x * X * X)) * (1.0 / LN10);
      const double dZ = a * b * invT * invT * eb - ic * ec;
      FT = F * (X * dZ / Z + e * invT);
    }
    return F;
  }
  return 1.0;  // Lindemann
}

__device__ __forceinline__ double dneg(double x) {
  return __longlong_as_double(__double_as_longlong(x) ^ (long long)0x8000000000000000ULL);
}

// nu * x with the common nu = +-1 done as a sign flip (integer pipe)
__device__ __forceinline__ double nu_times(int nu, double nud, double x) {
  if (nu == 1) return x;
  if (nu == -1) return dneg(x);
  return nud * x;
}

// R = k * prod_a C_a^nu_a over one reaction side (positions off .. off+n-1)
// and, with DER, dR[a] = dR/dC_a.  The shape code selects the minimal
// multiply sequence; SH_GEN falls back to a general product.
template <bool DER>
__device__ __forceinline__ double side_rate(const StateArrays& A, int aC, const Rxn* __restrict__ r, int off,
                                            int shape, int n, double k, double (&dR)[PJ_MAX_SP]) {
  switch (shape) {
    case SH_1: {
      const double c0 = A.at(aC, __ldg(&r->sp[off]));
      if (DER) dR[0] = k;
      return k * c0;
    }
    case SH_2: {
      const double c0 = A.at(aC, __ldg(&r->sp[off]));
      const double t = k * c0;
      if (DER) dR[0] = t + t;
      return t * c0;
    }
    case SH_11: {
      const double c0 = A.at(aC, __ldg(&r->sp[off])), c1 = A.at(aC, __ldg(&r->sp[off + 1]));
      const double t = k * c1;
      if (DER) {
        dR[0] = t;
        dR[1] = k * c0;
      }
      return t * c0;
    }
    case SH_21: {
      const double c0 = A.at(aC, __ldg(&r->sp[off])), c1 = A.at(aC, __ldg(&r->sp[off + 1]));
      const double t = k * c0;
      const double t1 = t * c1;
      if (DER) {
        dR[0] = t1 + t1;
        dR[1] = t * c0;
      }
      return t1 * c0;
    }
    case SH_111: {
      const double c0 = A.at(aC, __ldg(&r->sp[off])), c1 = A.at(aC, __ldg(&r->sp[off + 1]));
      const double c2 = A.at(aC, __ldg(&r->sp[off + 2]));
      const double t2 = k * c2;
      const double t12 = t2 * c1;
      if (DER) {
        dR[0] = t12;
        dR[1] = t2 * c0;
        dR[2] = (k * c0) * c1;
      }
      return t12 * c0;
    }
    default: {
      double pw[PJ_MAX_SP], dpw[PJ_MAX_SP];
#pragma unroll
      for (int a = 0; a < PJ_MAX_SP; a++) {
        pw[a] = 1.0;
        dpw[a] = 0.0;
        if (a < n) {
          const int v = __ldg(&r->nu[off + a]);
          const double c = A.at(aC, __ldg(&r->sp[off + a]));
          const double cm = powi(c, v - 1);
          pw[a] = cm * c;
          dpw[a] = v * cm;
        }
      }
      double R = k;
#pragma unroll
      for (int a = 0; a < PJ_MAX_SP; a++)
        if (a < n) R *= pw[a];
      if (DER) {
#pragma unroll
        for (int a = 0; a < PJ_MAX_SP; a++) {
          if (a >= n) continue;
          double p = k * dpw[a];
#pragma unroll
          for (int b = 0; b < PJ_MAX_SP; b++)
            if (b != a && b < n) p *= pw[b];
          dR[a] = p;
        }
      }
      return R;
    }
  }
}

// Forward and reverse rate constants; the two exponentials sit in one basic
// block so their dependency chains interleave.
__device__ __forceinline__ void rate_constants(const StateArrays& A, int aG, const Rxn* __restrict__ r, int rev,
                                               int nre, int npr, double lnkf, double logPRT, double& kf,
                                               double& kr) {
  if (rev) {
    double dg = 0.0;
#pragma unroll
    for (int a = 0; a < PJ_MAX_SP; a++) {
      if (a < nre) dg = fma(-__ldg(&r->nud[a]), A.at(aG, __ldg(&r->sp[a])), dg);
      if (a < npr) dg = fma(__ldg(&r->nud[PJ_MAX_SP + a]), A.at(aG, __ldg(&r->sp[PJ_MAX_SP + a])), dg);
    }
    // kr = kf / Kc with Kc = exp(-dg) (P_std / R T)^dnu
    const double larg = lnkf + dg - __ldg(&r->dnu) * logPRT;
    kf = exp(lnkf);
    kr = exp(larg);
  } else {
    kf = exp(lnkf);
    kr = 0.0;
  }
}

// Third-body concentration [M] = C_tot + sum_e (alpha_e - 1) C_e.
__device__ __forceinline__ double third_body(const DevMech& m, const StateArrays& A, int aC, const Rxn* __restrict__ r,
                                             double Ctot) {
  double M = Ctot;
  for (int e = __ldg(&r->eff_lo), eh = __ldg(&r->eff_hi); e < eh; e++)
    M = fma(__ldg(m.eff_am1 + e), A.at(aC, __ldg(m.eff_sp + e)), M);
  return M;
}

__device__ __forceinline__ void red_add(double* p, double v) { atomicAdd(p, v); }  // result unused: red.global.add.f64

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
  const int ns = m.ns, bath = m.ns - 1;
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
  enum { aC = 0, aG = 1 };
  for (int64_t s = gtid; s < n; s += (int64_t)gridDim.x * blockDim.x) {
    StateScalars st;
    if (!load_state<MODE>(m, phi, param, ld, s, A, aC, st)) {
      write_nan_state(out, ld, s, ns + 1);
      if (status) atomicAdd(status, 1);
      continue;
    }
    const double T = st.T, invT = st.invT, lnT = st.lnT;
    double* __restrict__ wrow = out + 2 * ld + s;   // wdot_k accumulates at wrow[k*ld]
    for (int k = 0; k < ns - 1; k++) wrow[(int64_t)k * ld] = 0.0;
    double den = 0.0;
    for (int k = 0; k < ns; k++) {
      double cp, h, sr;
      nasa_eval(nasa_block(m, k, T), T, invT, lnT, cp, h, sr);
      A.at(aG, k) = h - sr;
      den = fma(A.at(aC, k), MODE == PJ_CONP ? cp : cp - 1.0, den);
    }
    den *= RU;
    const double logPRT = m.log_pstd_over_r - lnT;  // ln(P_std / (R T))
    double w_bath = 0.0;

    for (int i = 0; i < m.nr; i++) {
      const Rxn* __restrict__ r = m.rxn + i;
      const int kind = __ldg(&r->kind);
      const int nre = __ldg(&r->nreac), npr = __ldg(&r->nprod), rev = __ldg(&r->rev);
      const double lnkf = fma(__ldg(&r->beta), lnT, __ldg(&r->lnA)) - __ldg(&r->theta) * invT;
      double kf, kr;
      rate_constants(A, aG, r, rev, nre, npr, lnkf, logPRT, kf, kr);
      double dmy[PJ_MAX_SP];
      const double Rf = side_rate<false>(A, aC, r, 0, __ldg(&r->shape[0]), nre, kf, dmy);
      const double Rr = rev ? side_rate<false>(A, aC, r, PJ_MAX_SP, __ldg(&r->shape[1]), npr, kr, dmy) : 0.0;
      double c = 1.0;
      if (kind != PJ_ELEMENTARY) {
        const double M = third_body(m, A, aC, r, st.Ctot);
        if (kind == PJ_THIRD_BODY) {
          c = M;
        } else {
          const double lnk0 = fma(__ldg(&r->beta0), lnT, __ldg(&r->lnA0)) - __ldg(&r->theta0) * invT;
          const double Pr = exp(lnk0 - lnkf) * M;
          double d1, d2;
          const double F = falloff_F<false>(r, kind, T, invT, lnT, Pr, d1, d2);
          c = Pr / (1.0 + Pr) * F;
        }
      }
      const double q = c * (Rf - Rr);
#pragma unroll
      for (int a = 0; a < PJ_MAX_SP; a++) {
        if (a < nre) {
          const int k = __ldg(&r->sp[a]);
          const double v = nu_times(__ldg(&r->nu[a]), __ldg(&r->nud[a]), q);
          if (k == bath) w_bath -= v;
          else red_add(wrow + (int64_t)k * ld, dneg(v));
        }
        if (a < npr) {
          const int k = __ldg(&r->sp[PJ_MAX_SP + a]);
          const double v = nu_times(__ldg(&r->nu[PJ_MAX_SP + a]), __ldg(&r->nud[PJ_MAX_SP + a]), q);
          if (k == bath) w_bath += v;
          else red_add(wrow + (int64_t)k * ld, v);
        }
      }
    }

    // energy equation and ideal-gas state equation
    double num = 0.0, Om = 0.0;
    for (int k = 0; k < ns; k++) {
      double cp, h, sr;
      nasa_eval(nasa_block(m, k, T), T, invT, lnT, cp, h, sr);
      const double wk = k < bath ? __ldcg(wrow + (int64_t)k * ld) : w_bath;
      num = fma(MODE == PJ_CONP ? h : h - 1.0, wk, num);
      if (k < bath) {
        Om = fma(__ldg(m.wfac + k), wk, Om);
        wrow[(int64_t)k * ld] = st.V * wk;
      }
    }
    num *= RU * T;
    const double Tdot = -num / den;
    out[s] = Tdot;
    if (MODE == PJ_CONP)
      out[ld + s] = st.V * Tdot * invT + (RU * T * st.V / st.P) * Om;
    else
      out[ld + s] = st.P * Tdot * invT + RU * T * Om;
  }
}

// ---------------------------------------------------------------------------
// analytical Jacobian
// ---------------------------------------------------------------------------
template <int FMT>
__device__ __forceinline__ int64_t jpos(const DevMech& m, int row, int col) {
  if (FMT == PJ_DENSE) return (int64_t)row * m.N + col;
  const int32_t* p = FMT == PJ_CSR ? m.pos_csr : m.pos_csc;
  return __ldg(p + (int64_t)row * m.N + col);
}

__device__ __forceinline__ void jred(double* J, int64_t e, int64_t ld, int64_t s, double v) {
  if (e >= 0) red_add(J + e * ld + s, v);
}

// Shared memory holds C_k, g_k/RT and h_k/RT per state.  Production rates go
// to the source-term output by L2 reductions (bath gas in a register);
// Jacobian entries to the zero-initialised output by L2 reductions.
template <int MODE, int FMT>
__global__ void __launch_bounds__(128) k_jacobian(DevMech m, int64_t n, const double* __restrict__ param,
                                                  const double* __restrict__ phi, int64_t ld,
                                                  double* __restrict__ J, double* __restrict__ dphi,
                                                  int* status, double* ws, int64_t ws_stride) {
  PJ_DYN_SMEM;
  const int ns = m.ns, N = m.N, bath = m.ns - 1;
  const int64_t n_out = FMT == PJ_DENSE ? (int64_t)N * N : (int64_t)m.nnz;
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
  enum { aC = 0, aG = 1, aH = 2 };
  for (int64_t s = gtid; s < n; s += (int64_t)gridDim.x * blockDim.x) {
    StateScalars st;
    if (!load_state<MODE>(m, phi, param, ld, s, A, aC, st)) {
      write_nan_state(J, ld, s, (int)n_out);
      write_nan_state(dphi, ld, s, ns + 1);
      if (status) atomicAdd(status, 1);
      continue;
    }
    const double T = st.T, V = st.V, P = st.P, invT = st.invT, lnT = st.lnT, Ctot = st.Ctot;
    const double invT2 = invT * invT, invV = 1.0 / V;
    for (int64_t e = 0; e < n_out; e++) J[e * ld + s] = 0.0;
    double* __restrict__ wrow = dphi + 2 * ld + s;  // wdot_k accumulates at wrow[k*ld]
    for (int k = 0; k < ns - 1; k++) wrow[(int64_t)k * ld] = 0.0;

    // thermo, energy-equation denominator D = sum_k C_k Cx_k and dD/dT
    double den = 0.0, dden_T = 0.0, Cx_bath = 0.0;
    for (int k = 0; k < ns; k++) {
      const double* cb = nasa_block(m, k, T);
      double cp, h, sr, cp2, dcp;
      nasa_eval(cb, T, invT, lnT, cp, h, sr);
      nasa_cp(cb, T, cp2, dcp);
      A.at(aG, k) = h - sr;
      A.at(aH, k) = h;
      const double Ck = A.at(aC, k);
      const double cx = MODE == PJ_CONP ? cp : cp - 1.0;
      den = fma(Ck, cx, den);
      dden_T = fma(Ck, dcp, dden_T);
      if (k == bath) Cx_bath = RU * cx;
    }
    den *= RU;
    const double C_bath = A.at(aC, bath);
    // derivatives of the bath-gas concentration
    const double dCb_T = -Ctot * invT;
    const double dCb_S = MODE == PJ_CONP ? (Ctot - C_bath) * invV : Ctot / P;
    dden_T = RU * dden_T + Cx_bath * dCb_T;
    const double dden_S = MODE == PJ_CONP ? (Cx_bath * Ctot - den) * invV : Cx_bath * Ctot / P;
    const double logPRT = m.log_pstd_over_r - lnT;

    // accumulators of the energy row (T) and state row (S) for the T and S
    // columns and for the part common to every species column
    double AT_T = 0, AT_S = 0, AS_T = 0, AS_S = 0, ATB = 0, ASB = 0, w_bath = 0;

    for (int i = 0; i < m.nr; i++) {
      const Rxn* __restrict__ r = m.rxn + i;
      const int kind = __ldg(&r->kind);
      const int nre = __ldg(&r->nreac), npr = __ldg(&r->nprod);
      const int rev = __ldg(&r->rev);
      const double beta = __ldg(&r->beta), theta = __ldg(&r->theta);
      const double lnkf = fma(beta, lnT, __ldg(&r->lnA)) - theta * invT;
      const double dlnkf = fma(theta, invT2, beta * invT);
      double kf, kr;
      rate_constants(A, aG, r, rev, nre, npr, lnkf, logPRT, kf, kr);
      double dh = 0.0;
#pragma unroll
      for (int a = 0; a < PJ_MAX_SP; a++) {
        if (a < nre) dh = fma(-__ldg(&r->nud[a]), A.at(aH, __ldg(&r->sp[a])), dh);
        if (a < npr) dh = fma(__ldg(&r->nud[PJ_MAX_SP + a]), A.at(aH, __ldg(&r->sp[PJ_MAX_SP + a])), dh);
      }
      double dRf[PJ_MAX_SP], dRr[PJ_MAX_SP];
      const double Rf = side_rate<true>(A, aC, r, 0, __ldg(&r->shape[0]), nre, kf, dRf);
      double Rr = 0.0, dlnkr = 0.0;
      if (rev) {
        Rr = side_rate<true>(A, aC, r, PJ_MAX_SP, __ldg(&r->shape[1]), npr, kr, dRr);
        dlnkr = dlnkf - (dh - __ldg(&r->dnu)) * invT;
      }
      const double Rn = Rf - Rr;

      // pressure modification c and its derivatives
      double c = 1.0, dcdT = 0.0, dcdS = 0.0, dcdM = 0.0;
      if (kind != PJ_ELEMENTARY) {
        const double M = third_body(m, A, aC, r, Ctot);
        const double ab = __ldg(&r->alpha_bath);
        const double dMdT = ab * dCb_T;
        const double dMdS = MODE == PJ_CONP ? (ab * Ctot - M) * invV : ab * Ctot / P;
        if (kind == PJ_THIRD_BODY) {
          c = M;
          dcdM = 1.0;
          dcdT = dMdT;
          dcdS = dMdS;
        } else {
          const double beta0 = __ldg(&r->beta0), theta0 = __ldg(&r->theta0);
          const double lnk0 = fma(beta0, lnT, __ldg(&r->lnA0)) - theta0 * invT;
          const double dlnk0 = fma(theta0, invT2, beta0 * invT);
          const double rk = exp(lnk0 - lnkf);
          const double Pr = rk * M;
          double FxPr, FT;
          const double F = falloff_F<true>(r, kind, T, invT, lnT, Pr, FxPr, FT);
          const double i1p = 1.0 / (1.0 + Pr);
          const double fr = Pr * i1p;
          c = fr * F;
          const double cPr = F * i1p * i1p + FxPr * i1p;
          const double dPrdT = Pr * (dlnk0 - dlnkf) + rk * dMdT;
          dcdT = fr * FT + cPr * dPrdT;
          dcdM = cPr * rk;
          dcdS = dcdM * dMdS;
        }
      }

      // derivatives of the net rate in T and S (rate constants, and the bath
      // gas through C_Ns = C_tot - sum C_k)
      double dRdT = Rf * dlnkf - Rr * dlnkr;
      double dRdS = 0.0;
#pragma unroll
      for (int a = 0; a < PJ_MAX_SP; a++) {
        if (a < nre) {
          const int k = __ldg(&r->sp[a]);
          if (k == bath) {
            dRdT = fma(dRf[a], dCb_T, dRdT);
            dRdS = fma(dRf[a], dCb_S, dRdS);
          } else if (MODE == PJ_CONP) {
            dRdS = fma(dRf[a], -A.at(aC, k) * invV, dRdS);
          }
        }
        if (rev && a < npr) {
          const int k = __ldg(&r->sp[PJ_MAX_SP + a]);
          if (k == bath) {
            dRdT = fma(-dRr[a], dCb_T, dRdT);
            dRdS = fma(-dRr[a], dCb_S, dRdS);
          } else if (MODE == PJ_CONP) {
            dRdS = fma(dRr[a], A.at(aC, k) * invV, dRdS);
          }
        }
      }
      const double q = c * Rn;
      const double dqdT = fma(c, dRdT, Rn * dcdT);
      const double dqdS = fma(c, dRdS, Rn * dcdS);
#pragma unroll
      for (int a = 0; a < PJ_MAX_SP; a++) {
        if (a < nre) {
          const int k = __ldg(&r->sp[a]);
          const double v = nu_times(__ldg(&r->nu[a]), __ldg(&r->nud[a]), q);
          if (k == bath) w_bath -= v;
          else red_add(wrow + (int64_t)k * ld, dneg(v));
        }
        if (a < npr) {
          const int k = __ldg(&r->sp[PJ_MAX_SP + a]);
          const double v = nu_times(__ldg(&r->nu[PJ_MAX_SP + a]), __ldg(&r->nud[PJ_MAX_SP + a]), q);
          if (k == bath) w_bath += v;
          else red_add(wrow + (int64_t)k * ld, v);
        }
      }

      // energy-row and state-row weights of this reaction
      const double dE = RU * T * (MODE == PJ_CONP ? dh : dh - __ldg(&r->dnu));
      const double dW = __ldg(&r->dW);
      AT_T = fma(dE, dqdT, AT_T);
      AT_S = fma(dE, dqdS, AT_S);
      AS_T = fma(dW, dqdT, AS_T);
      AS_S = fma(dW, dqdS, AS_S);

      const int row_lo = __ldg(&r->row_lo), row_hi = __ldg(&r->row_hi);
      const double VdqdT = V * dqdT, VdqdS = V * dqdS;
      for (int q2 = row_lo; q2 < row_hi; q2++) {
        const RowNu rn = m.rows[q2];
        jred(J, jpos<FMT>(m, rn.k + 2, 0), ld, s, nu_times(rn.nu, rn.nud, VdqdT));
        jred(J, jpos<FMT>(m, rn.k + 2, 1), ld, s, nu_times(rn.nu, rn.nud, VdqdS));
      }

      // species columns: V dq/dn_j = c dR/dC_j + R dc/dM (alpha_j - 1) + B_i
      double Bi = 0.0;
      auto slot = [&](int j, double val) {
        if (j == bath) {
          Bi -= val;
          return;
        }
        for (int q2 = row_lo; q2 < row_hi; q2++) {
          const RowNu rn = m.rows[q2];
          jred(J, jpos<FMT>(m, rn.k + 2, j + 2), ld, s, nu_times(rn.nu, rn.nud, val));
        }
        jred(J, jpos<FMT>(m, 0, j + 2), ld, s, dE * val);
        jred(J, jpos<FMT>(m, 1, j + 2), ld, s, dW * val);
      };
#pragma unroll
      for (int a = 0; a < PJ_MAX_SP; a++) {
        if (a < nre) slot(__ldg(&r->sp[a]), c * dRf[a]);
        if (rev && a < npr) slot(__ldg(&r->sp[PJ_MAX_SP + a]), dneg(c * dRr[a]));
      }
      if (kind != PJ_ELEMENTARY) {
        const double t = Rn * dcdM;
        for (int e = __ldg(&r->eff_lo), eh = __ldg(&r->eff_hi); e < eh; e++)
          slot(__ldg(m.eff_sp + e), t * __ldg(m.eff_am1 + e));
      }
      if (__ldg(&r->dense)) {
        for (int q2 = row_lo; q2 < row_hi; q2++) {
          const RowNu rn = m.rows[q2];
          const double v = nu_times(rn.nu, rn.nud, Bi);
          for (int j = 0; j < ns - 1; j++) jred(J, jpos<FMT>(m, rn.k + 2, j + 2), ld, s, v);
        }
        ATB = fma(dE, Bi, ATB);
        ASB = fma(dW, Bi, ASB);
      }
    }

    // source terms; the G array now holds Cx_k = R (cp_k or cv_k)
    double num = 0.0, Om = 0.0, sumCxW = 0.0;
    for (int k = 0; k < ns; k++) {
      double cp, dcp;
      nasa_cp(nasa_block(m, k, T), T, cp, dcp);
      const double cx = RU * (MODE == PJ_CONP ? cp : cp - 1.0);
      A.at(aG, k) = cx;
      const double wk = k < bath ? __ldcg(wrow + (int64_t)k * ld) : w_bath;
      num = fma(MODE == PJ_CONP ? A.at(aH, k) : A.at(aH, k) - 1.0, wk, num);
      sumCxW = fma(cx, wk, sumCxW);
      if (k < bath) {
        Om = fma(__ldg(m.wfac + k), wk, Om);
        wrow[(int64_t)k * ld] = V * wk;
        if (MODE == PJ_CONP) jred(J, jpos<FMT>(m, k + 2, 1), ld, s, wk);
      }
    }
    num *= RU * T;
    const double Tdot = -num / den;
    const double Sdot = MODE == PJ_CONP ? V * Tdot * invT + (RU * T * V / P) * Om : P * Tdot * invT + RU * T * Om;
    dphi[s] = Tdot;
    dphi[ld + s] = Sdot;

    // energy row 0 and state row 1
    const double iden = 1.0 / den;
    const double Cx_b = A.at(aG, bath);
    const double rtvp = MODE == PJ_CONP ? RU * T * V / P : RU * T;
    for (int j = 0; j < N; j++) {
      const int64_t e0 = jpos<FMT>(m, 0, j), e1 = jpos<FMT>(m, 1, j);
      double jT, dOm;
      if (j == 0) {
        jT = -(AT_T + sumCxW + Tdot * dden_T) * iden;
        dOm = AS_T;
      } else if (j == 1) {
        jT = -(AT_S + Tdot * dden_S) * iden;
        dOm = AS_S;
      } else {
        const double accT = __ldcg(J + e0 * ld + s);
        const double accS = __ldcg(J + e1 * ld + s);
        jT = -(accT + ATB + Tdot * (A.at(aG, j - 2) - Cx_b)) * (invV * iden);
        dOm = (accS + ASB) * invV;
      }
      double jS;
      if (MODE == PJ_CONP) {
        jS = (V * invT) * jT + rtvp * dOm;
        if (j == 0) jS += -V * Tdot * invT2 + (RU * V / P) * Om;
        if (j == 1) jS += Tdot * invT + (RU * T / P) * Om;
      } else {
        jS = (P * invT) * jT + rtvp * dOm;
        if (j == 0) jS += -P * Tdot * invT2 + RU * Om;
        if (j == 1) jS += Tdot * invT;
      }
      J[e0 * ld + s] = jT;
      J[e1 * ld + s] = jS;
    }
  }
}

#ifndef PJ_NO_LAUNCHERS
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

// Per-state arrays: in shared memory when 128 threads fit, else in a global
// workspace with a fixed grid-stride grid.
LaunchPlan plan_for(int arrays, int ns, int64_t n) {
  LaunchPlan p{};
  const size_t per_thread = (size_t)arrays * ns * sizeof(double);
  const size_t smem_cap = 227 * 1024;  // opt-in dynamic shared memory per block on sm_100-class parts
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

template <int MODE, int FMT>
static int launch_jac_t(const DevMech& m, const LaunchPlan& p, int64_t n, const double* param, const double* phi,
                        int64_t ld, double* J, double* dphi, int* status, double* ws, cudaStream_t st) {
  int rc;
  if ((rc = set_smem(k_jacobian<MODE, FMT>, p.smem))) return rc;
  k_jacobian<MODE, FMT><<<p.grid, p.tpb, p.smem, st>>>(m, n, param, phi, ld, J, dphi, status, ws, p.ws_stride);
  return check_cuda(cudaGetLastError(), "k_jacobian launch");
}

int launch_jacobian(const DevMech& m, int mode, int fmt, int64_t n, const double* param, const double* phi,
                    int64_t ld, double* J, double* dphi, int* status, void* work, size_t work_bytes,
                    cudaStream_t st) {
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

size_t workspace_bytes(int arrays, int ns, int64_t n) { return plan_for(arrays, ns, n).ws_bytes; }

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
