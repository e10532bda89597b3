// Device helpers shared by the kernels of kinetics.cu and forms.cu: state
// loading, falloff broadening, reaction-side products, rate constants, third
// bodies, production-rate scatter and reductions.
#pragma once

#include <cuda_runtime.h>

#include "kinetics_device.cuh"

#ifndef PJ_DYN_SMEM
#define PJ_DYN_SMEM extern __shared__ double smem[]
#endif

namespace pj {

struct StateScalars {
  double T, V, P, invT, lnT, Ctot;
  double lnP;  // ln P [Pa], formed only when some reaction depends on pressure
};

__device__ __forceinline__ bool has_third_body(int kind) { return kind >= PJ_THIRD_BODY && kind <= PJ_SRI; }

// Load one state, fill C_k (k < Ns-1 as n_k/V; the bath gas as C_tot minus
// the others summed in species order) and check validity.
template <int MODE, class SA>
__device__ __forceinline__ bool load_state(const DevMech& m, const double* __restrict__ phi,
                                           const double* __restrict__ param, int64_t ld, int64_t s,
                                           const SA& A, int aC, StateScalars& st) {
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
  st.lnP = m.has_pdep ? log(P) : 0.0;
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

// Troe / SRI broadening factor F(T, Pr) in FP64.  With derivatives also
// returns FxPr = Pr dF/dPr (at fixed T) and FT = dF/dT (at fixed Pr),
// evaluated in the derivative type DT (FP64, or FP32 for the Newton form).
template <bool DERIV, typename DT = double>
__device__ __forceinline__ double falloff_F(const Rxn* __restrict__ r, int kind, double T, double invT,
                                            double lnT, double Pr, DT& FxPr, DT& FT) {
  FxPr = DT(0);
  FT = DT(0);
  if (kind == PJ_TROE) {
    const double a = __ldg(&r->fp[0]), iT3 = __ldg(&r->fp[1]), iT1 = __ldg(&r->fp[2]);
    const double T2 = __ldg(&r->fp[3]), has2 = __ldg(&r->fp[4]);
    const double e3 = pj_exp(-T * iT3), e1 = pj_exp(-T * iT1);
    const double e2 = has2 != 0.0 ? pj_exp(-T2 * invT) : 0.0;
    const double Fcent = (1.0 - a) * e3 + a * e1 + e2;
    const double L = log10(Fcent);
    const double x = log10(Pr);
    const double cc = -0.4 - 0.67 * L;
    const double NN = 0.75 - 1.27 * L;
    const double xc = x + cc;
    const double D = NN - 0.14 * xc;
    const double f1 = xc / D;
    const double g = 1.0 / (1.0 + f1 * f1);
    const double F = pj_exp(LN10 * (L * g));
    if (DERIV) {
      const DT Lt = DT(L), Dt = DT(D), f1t = DT(f1), gt = DT(g), Ft = DT(F), xct = DT(xc);
      const DT iD = DT(1) / Dt;
      const DT iD2 = iD * iD;
      const DT m2fg2 = DT(-2) * f1t * gt * gt;
      const DT dlg_dx = Lt * m2fg2 * DT(NN) * iD2;
      const DT dlg_dL = gt + Lt * m2fg2 * (DT(-0.67) * Dt + DT(1.1762) * xct) * iD2;
      const DT dFcent = DT(-(1.0 - a) * iT3) * DT(e3) - DT(a * iT1) * DT(e1) + DT(T2) * DT(invT * invT) * DT(e2);
      FxPr = Ft * dlg_dx;
      FT = Ft * dlg_dL * dFcent / DT(Fcent);
    }
    return F;
  }
  if (kind == PJ_SRI) {
    const double a = __ldg(&r->fp[0]), b = __ldg(&r->fp[1]), ic = __ldg(&r->fp[2]);
    const double d = __ldg(&r->fp[3]), e = __ldg(&r->fp[4]);
    const double x = log10(Pr);
    const double X = 1.0 / (1.0 + x * x);
    const double eb = pj_exp(-b * invT), ec = pj_exp(-T * ic);
    const double Z = a * eb + ec;
    const double lnZ = log(Z);
    const double F = d * pj_exp(X * lnZ + e * lnT);
    if (DERIV) {
      const DT Xt = DT(X), Ft = DT(F), xt = DT(x), it = DT(invT);
      FxPr = Ft * (DT(lnZ) * (DT(-2) * xt * Xt * Xt)) * DT(1.0 / LN10);
      const DT dZ = DT(a * b) * it * it * DT(eb) - DT(ic) * DT(ec);
      FT = Ft * (Xt * dZ / DT(Z) + DT(e) * it);
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
template <bool DER, class SA>
__device__ __forceinline__ double side_rate(const SA& A, int aC, const Rxn* __restrict__ r, int off,
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

// ln k of a P-log or Chebyshev reaction and, with DER, d ln k / dT and
// d ln k / d ln P.  P-log: Arrhenius rates at ascending ln P_m (table rows
// ln P, ln A, beta, theta), ln k linear in ln P on [ln P_m, ln P_m+1), held at
// the end values below the first and from the last pressure on.  Chebyshev:
// ln k = sum_t sum_p (ln10 a_tp) phi_t(T~) phi_p(P~) with T~ = cT1/T + cT0,
// P~ = cP1 ln P + cP0 and phi_n the Chebyshev polynomials (three-term
// recurrence, which also extends them outside [-1, 1]).
// Not inlined: it runs only for pressure-dependent reactions, and keeping it
// out of the reaction loop keeps that loop's register allocation unchanged.
template <bool DER>
__device__ __noinline__ double lnk_pdep(const DevMech& m, const Rxn* __restrict__ r, int kind, double lnT,
                                        double invT, double lnP, double& d_T, double& d_lnP) {
  const double* __restrict__ t = m.tab + __ldg(&r->tab_lo) + (__ldg(&r->rev) == 2 ? 3 : 0);
  if (kind == PJ_PLOG) {
    const int n = __ldg(&r->tab_n);
    auto lnk_at = [&](int j) { return fma(__ldg(t + 4 * j + 2), lnT, __ldg(t + 4 * j + 1)) - __ldg(t + 4 * j + 3) * invT; };
    auto dT_at = [&](int j) { return fma(__ldg(t + 4 * j + 3), invT * invT, __ldg(t + 4 * j + 2) * invT); };
    if (lnP < __ldg(t) || n == 1) {
      if (DER) { d_T = dT_at(0); d_lnP = 0.0; }
      return lnk_at(0);
    }
    if (lnP >= __ldg(t + 4 * (n - 1))) {
      if (DER) { d_T = dT_at(n - 1); d_lnP = 0.0; }
      return lnk_at(n - 1);
    }
    int j = 0;
    while (j + 2 < n && lnP >= __ldg(t + 4 * (j + 1))) j++;
    const double p0 = __ldg(t + 4 * j), p1 = __ldg(t + 4 * (j + 1));
    const double k0 = lnk_at(j), k1 = lnk_at(j + 1);
    const double slope = (k1 - k0) / (p1 - p0);
    if (DER) {
      const double w = (lnP - p0) / (p1 - p0);
      d_T = fma(w, dT_at(j + 1) - dT_at(j), dT_at(j));
      d_lnP = slope;
    }
    return fma(slope, lnP - p0, k0);
  }
  // Chebyshev
  const int nT = __ldg(&r->tab_n), nP = __ldg(&r->tab_m);
  const double x = fma(__ldg(t), invT, __ldg(t + 1));
  const double y = fma(__ldg(t + 2), lnP, __ldg(t + 3));
  const double* __restrict__ a = t + 4;
  double S = 0.0, Sx = 0.0, Sy = 0.0;
  double pt0 = 1.0, pt1 = x, dt0 = 0.0, dt1 = 1.0;  // phi_t(x) and phi_t'(x)
  for (int it = 0; it < nT; it++) {
    const double pt = it == 0 ? 1.0 : pt1, dpt = it == 0 ? 0.0 : dt1;
    double B = 0.0, By = 0.0;
    double pp0 = 1.0, pp1 = y, dp0 = 0.0, dp1 = 1.0;
    for (int ip = 0; ip < nP; ip++) {
      const double pp = ip == 0 ? 1.0 : pp1, dpp = ip == 0 ? 0.0 : dp1;
      const double c = __ldg(a + it * nP + ip);
      B = fma(c, pp, B);
      if (DER) By = fma(c, dpp, By);
      if (ip >= 1) {
        const double pn = fma(2.0 * y, pp1, -pp0), dn = fma(2.0 * y, dp1, fma(2.0, pp1, -dp0));
        pp0 = pp1; pp1 = pn; dp0 = dp1; dp1 = dn;
      }
    }
    S = fma(pt, B, S);
    if (DER) {
      Sx = fma(dpt, B, Sx);
      Sy = fma(pt, By, Sy);
    }
    if (it >= 1) {
      const double pn = fma(2.0 * x, pt1, -pt0), dn = fma(2.0 * x, dt1, fma(2.0, pt1, -dt0));
      pt0 = pt1; pt1 = pn; dt0 = dt1; dt1 = dn;
    }
  }
  if (DER) {
    d_T = -Sx * __ldg(t) * invT * invT;
    d_lnP = Sy * __ldg(t + 2);
  }
  return S;
}

// ln of reaction r's forward rate constant: the Arrhenius set for
// elementary, third-body and falloff reactions, the low-pressure set for
// chemically-activated ones, the P-log / Chebyshev forms otherwise.  lnkinf
// is the Arrhenius set itself (the high-pressure limit in Pr).  With DER:
// d_T, d_lnP of ln k_f and dinf_T of ln k_inf.
template <bool B>
struct BoolTag {
  static constexpr bool value = B;
};

template <bool DER, bool GEN = true>
__device__ __forceinline__ double ln_kf(const DevMech& m, const Rxn* __restrict__ r, int kind, double lnT,
                                        double invT, double lnP, double& lnkinf, double& d_T, double& d_lnP,
                                        double& dinf_T) {
  const double beta = __ldg(&r->beta), theta = __ldg(&r->theta);
  lnkinf = fma(beta, lnT, __ldg(&r->lnA)) - theta * invT;
  if (DER) {
    dinf_T = fma(theta, invT * invT, beta * invT);
    d_T = dinf_T;
    d_lnP = 0.0;
  }
  if (!GEN) return lnkinf;  // plain reactions: the Arrhenius set
  if (kind >= PJ_PLOG) return lnk_pdep<DER>(m, r, kind, lnT, invT, lnP, d_T, d_lnP);
  if (__ldg(&r->chem)) {
    const double beta0 = __ldg(&r->beta0), theta0 = __ldg(&r->theta0);
    if (DER) d_T = fma(theta0, invT * invT, beta0 * invT);
    return fma(beta0, lnT, __ldg(&r->lnA0)) - theta0 * invT;
  }
  return lnkinf;
}

// Forward and reverse rate constants; the two exponentials sit in one basic
// block so their dependency chains interleave.  rev == 2: explicit reverse
// Arrhenius set instead of k_f / K_c.
template <bool GEN = true, class SA>
__device__ __forceinline__ void rate_constants(const DevMech& m, const SA& A, int aG, const Rxn* __restrict__ r,
                                               int rev,
                                               int nre, int npr, double lnkf, double logPRT, double lnT,
                                               double invT, double& kf, double& kr) {
  if (GEN && rev == 2) {
    const double* __restrict__ rt = m.tab + __ldg(&r->tab_lo);
    const double larg = fma(__ldg(rt + 1), lnT, __ldg(rt)) - __ldg(rt + 2) * invT;
    kf = pj_exp(lnkf);
    kr = pj_exp(larg);
  } else if (rev) {
    double dg = 0.0;
#pragma unroll
    for (int a = 0; a < PJ_MAX_SP; a++) {
      if (a < nre) dg = fma(-__ldg(&r->nud[a]), A.at(aG, __ldg(&r->sp[a])), dg);
      if (a < npr) dg = fma(__ldg(&r->nud[PJ_MAX_SP + a]), A.at(aG, __ldg(&r->sp[PJ_MAX_SP + a])), dg);
    }
    // kr = kf / Kc with Kc = exp(-dg) (P_std / R T)^dnu
    const double larg = lnkf + dg - __ldg(&r->dnu) * logPRT;
    kf = pj_exp(lnkf);
    kr = pj_exp(larg);
  } else {
    kf = pj_exp(lnkf);
    kr = 0.0;
  }
}

// Third-body concentration [M] = C_tot + sum_e (alpha_e - 1) C_e.
template <class SA>
__device__ __forceinline__ double third_body(const DevMech& m, const SA& A, int aC, const Rxn* __restrict__ r,
                                             double Ctot) {
  double M = Ctot;
  for (int e = __ldg(&r->eff_lo), eh = __ldg(&r->eff_hi); e < eh; e++) {
    if (!PJ_DBG_OK(m.dbg, e >= 0 && e < m.n_eff && __ldg(m.eff_sp + e) >= 0 && __ldg(m.eff_sp + e) < m.ns,
                   PJ_DBG_EFF))
      break;
    M = fma(__ldg(m.eff_am1 + e), A.at(aC, __ldg(m.eff_sp + e)), M);
  }
  return M;
}

__device__ __forceinline__ void red_add(double* p, double v) { atomicAdd(p, v); }  // result unused: red.global.add.f64

// wdot_k += nu_k q for the reaction's species.  k < Ns-1: nu_k L2
// reductions of +-q into wrow[k*ld] (a repeated reduction instead of a
// multiply: no FP64 instruction, which the compiler would otherwise issue,
// predicated off, for the common nu = 1 too); skipped when !w.  The bath gas,
// in few reactions (Rxn::bath_in), into a register under a branch of its own.
__device__ __forceinline__ void scatter_wdot(const Rxn* __restrict__ r, int nre, int npr, int bath, double q,
                                             double* wrow, int64_t ld, double& w_bath, bool w = true) {
  const double nq = dneg(q);
#pragma unroll
  for (int a = 0; a < PJ_MAX_SP; a++) {
    if (a < nre) {
      const int k = __ldg(&r->sp[a]);
      if (k != bath && w)
        for (int u = __ldg(&r->nu[a]); u > 0; u--) red_add(wrow + (int64_t)k * ld, nq);
    }
    if (a < npr) {
      const int k = __ldg(&r->sp[PJ_MAX_SP + a]);
      if (k != bath && w)
        for (int u = __ldg(&r->nu[PJ_MAX_SP + a]); u > 0; u--) red_add(wrow + (int64_t)k * ld, q);
    }
  }
  if (__ldg(&r->bath_in)) {
    for (int a = 0; a < PJ_MAX_SP; a++) {
      if (a < nre && __ldg(&r->sp[a]) == bath) w_bath = fma(-__ldg(&r->nud[a]), q, w_bath);
      if (a < npr && __ldg(&r->sp[PJ_MAX_SP + a]) == bath) w_bath = fma(__ldg(&r->nud[PJ_MAX_SP + a]), q, w_bath);
    }
  }
}

}  // namespace pj
