// Per-state evaluation functions (source terms, analytical Jacobian and its
// FP32 Newton form) shared by the grid-stride kernels of kinetics.cu and the
// persistent batched kernels of batch.cu.
#pragma once

#include "kinetics_common.cuh"

namespace pj {

// One state of the source-term evaluation (s < n, arrays A of this thread).
template <int MODE, bool SPECIAL = true, class SA>
__device__ __forceinline__ void source_state(const DevMech& m, const SA& A, const double* __restrict__ param,
                                             const double* __restrict__ phi, int64_t ld, int64_t s,
                                             double* __restrict__ out, int* status) {
  const int ns = m.ns, bath = m.ns - 1;
  enum { aC = 0, aG = 1 };
  StateScalars st;
  if (!load_state<MODE>(m, phi, param, ld, s, A, aC, st)) {
    write_nan_state(out, ld, s, ns + 1);
    if (status) atomicAdd(status, 1);
    return;
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

  // Plain reactions (the first m.nr_plain in kernel order) run through a
  // body compiled without the special cases (chemically activated, explicit
  // reverse, P-log, Chebyshev), the rest through the general one; kernels for
  // mechanisms without special reactions are instantiated with SPECIAL =
  // false and carry no general body at all.
  auto reaction = [&](int i, auto gen_tag) {
    constexpr bool GEN = decltype(gen_tag)::value;
    const Rxn* __restrict__ r = m.rxn + i;
    const int kind = __ldg(&r->kind);
    const int nre = __ldg(&r->nreac), npr = __ldg(&r->nprod), rev = __ldg(&r->rev);
    double lnkinf, u0, u1, u2;
    const double lnkf = ln_kf<false, GEN>(m, r, kind, lnT, invT, st.lnP, lnkinf, u0, u1, u2);
    double kf, kr;
    rate_constants<GEN>(m, A, aG, r, rev, nre, npr, lnkf, logPRT, lnT, invT, kf, kr);
    double dmy[PJ_MAX_SP];
    const double Rf = side_rate<false>(A, aC, r, 0, __ldg(&r->shape[0]), nre, kf, dmy);
    const double Rr = rev ? side_rate<false>(A, aC, r, PJ_MAX_SP, __ldg(&r->shape[1]), npr, kr, dmy) : 0.0;
    double c = 1.0;
    if (has_third_body(kind)) {
      const double M = third_body(m, A, aC, r, st.Ctot);
      if (kind == PJ_THIRD_BODY) {
        c = M;
      } else {
        const double lnk0 = fma(__ldg(&r->beta0), lnT, __ldg(&r->lnA0)) - __ldg(&r->theta0) * invT;
        const double Pr = pj_exp(lnk0 - lnkinf) * M;
        double d1, d2;
        const double F = falloff_F<false>(r, kind, T, invT, lnT, Pr, d1, d2);
        // falloff: k_inf Pr/(1+Pr) F; chemically activated: k0 F/(1+Pr)
        c = ((GEN && __ldg(&r->chem)) ? 1.0 : Pr) / (1.0 + Pr) * F;
      }
    }
    const double q = c * (Rf - Rr);
    scatter_wdot(r, nre, npr, bath, q, wrow, ld, w_bath);
  };
  for (int i = 0; i < m.nr_plain; i++) reaction(i, BoolTag<false>{});
  if (SPECIAL)
    for (int i = m.nr_plain; i < m.nr; i++) reaction(i, BoolTag<true>{});


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

// ---------------------------------------------------------------------------
// analytical Jacobian
// ---------------------------------------------------------------------------
template <int FMT>
__device__ __forceinline__ int64_t jpos(const DevMech& m, int row, int col) {
  if (!PJ_DBG_OK(m.dbg, row >= 0 && row < m.N && col >= 0 && col < m.N, PJ_DBG_POSMAP)) return -1;
  if (FMT == PJ_DENSE) return (int64_t)row * m.N + col;
  const int32_t* p = FMT == PJ_CSR ? m.pos_csr : m.pos_csc;
  const int64_t e = __ldg(p + (int64_t)row * m.N + col);
  if (!PJ_DBG_OK(m.dbg, e >= -1 && e < m.nnz, PJ_DBG_POSMAP)) return -1;
  return e;
}

__device__ __forceinline__ void red_add(float* p, float v) { atomicAdd(p, v); }  // red.global.add.f32

template <typename DT>
__device__ __forceinline__ void jred(DT* J, int64_t e, int64_t ld, int64_t s, DT v) {
  if (e >= 0) red_add(J + e * ld + s, v);
}

__device__ __forceinline__ float dneg(float x) { return -x; }

// +-x for a row's unit coefficient (rows hold |nu| = 1, see RowNu): a sign
// flip, no FP64 instruction
template <typename DT>
__device__ __forceinline__ DT nu_times_t(int nu, double, DT x) {
  return nu > 0 ? x : dneg(x);
}

// ---------------------------------------------------------------------------
// Analytical Jacobian (Sec. 2.2, assembled as in Sec. 3.4).  Rates,
// equilibrium constants, exponentials and source terms are always FP64.  DT
// is the type of the derivative arithmetic, the entry accumulation and the
// output: double for J itself, float for the Newton-matrix form.
//
// The evaluation of one state has three parts, written as separate functions
// so that the one-state-per-thread kernels (jacobian_state) and the
// cooperative kernel (k_jacobian_coop: the warps of a block share 32 states
// and split the reactions, the species and the columns among themselves)
// run the same arithmetic:
//   jac_reaction   one reaction: rates, their derivatives, production rates
//                  and the Jacobian entries it changes (L2 reductions into
//                  the zero-initialised output), and its share of the
//                  energy-row (T) and state-row (S) weights;
//   jac_species    one species after all reactions: its heat capacity, its
//                  production rate (written as dn_k/dt = V wdot_k) and its
//                  terms of the energy and state equations;
//   jac_ts_column  column j of the energy row 0 and the state row 1.
// ---------------------------------------------------------------------------

// Per-state values the reaction body reads, and the accumulators it adds to.
template <typename DT>
struct JacVars {
  double T, V, P, invT, lnT, lnP, Ctot;
  double invT2, invV, logPRT, dCb_T, dCb_S;  // dCb_*: derivatives of the bath-gas concentration
  // energy-row (T) and state-row (S) weights for the T and S columns and for
  // the part common to every species column; bath-gas production rate
  DT AT_T, AT_S, AS_T, AS_S, ATB, ASB;
  double w_bath;
};

// Where a state's outputs go: J[e*ld + s], wrow[k*ld] = wdot_k (k < Ns-1);
// w = false masks every global write (a lane past the batch or an invalid
// state computing on a dummy).
template <typename DT>
struct JacOut {
  DT* __restrict__ J;
  double* __restrict__ wrow;
  int64_t ld, s;
  bool w;
  DT hg;  // Newton form: -h gamma, the factor every Jacobian contribution carries
};

// A Jacobian contribution as written: for the Newton form M = I - h gamma J
// scaled by -h gamma (the identity is added once every entry is complete).
template <bool NEWTON, typename DT>
__device__ __forceinline__ DT nscale(const JacOut<DT>& o, DT x) {
  return NEWTON ? o.hg * x : x;
}

template <int MODE, int FMT, typename DT, bool GEN, bool TM, bool NEWTON, class SA>
__device__ __forceinline__ void jac_reaction(const DevMech& m, const SA& A, JacVars<DT>& v, const JacOut<DT>& o,
                                             int i, uint32_t tm_row) {
  enum { aC = 0, aG = 1, aH = 2 };
  const int ns = m.ns, bath = m.ns - 1;
  DT* __restrict__ J = o.J;
  const int64_t ld = o.ld, s = o.s;
  const bool w = o.w;
  auto h_at = [&](int k) -> double {
    if (TM) return tmem_ld_f64(tm_row + 2u * (uint32_t)k);
    return A.at(aH, k);
  };
  const double T = v.T, P = v.P, invT = v.invT, lnT = v.lnT, Ctot = v.Ctot, invT2 = v.invT2, invV = v.invV;
  const DT invT_t = DT(invT), invV_t = DT(invV), V_t = DT(v.V);
  const DT dCb_T_t = DT(v.dCb_T), dCb_S_t = DT(v.dCb_S);

  const Rxn* __restrict__ r = m.rxn + i;
  const int kind = __ldg(&r->kind);
  const int nre = __ldg(&r->nreac), npr = __ldg(&r->nprod);
  const int rev = __ldg(&r->rev);
  double lnkinf, dlnkf_d, dlnP_d, dlnkinf_d;
  const double lnkf = ln_kf<true, GEN>(m, r, kind, lnT, invT, v.lnP, lnkinf, dlnkf_d, dlnP_d, dlnkinf_d);
  const DT dlnkf = DT(dlnkf_d);
  double kf, kr;
  rate_constants<GEN>(m, A, aG, r, rev, nre, npr, lnkf, v.logPRT, lnT, invT, kf, kr);
  double dh = 0.0;
  if (TM) __syncwarp();
#pragma unroll
  for (int a = 0; a < PJ_MAX_SP; a++) {
    if (a < nre) dh = fma(-__ldg(&r->nud[a]), h_at(__ldg(&r->sp[a])), dh);
    if (a < npr) dh = fma(__ldg(&r->nud[PJ_MAX_SP + a]), h_at(__ldg(&r->sp[PJ_MAX_SP + a])), dh);
  }
  double dRf[PJ_MAX_SP], dRr[PJ_MAX_SP];
  const double Rf = side_rate<true>(A, aC, r, 0, __ldg(&r->shape[0]), nre, kf, dRf);
  double Rr = 0.0;
  DT dlnkr = DT(0);
  if (rev) {
    Rr = side_rate<true>(A, aC, r, PJ_MAX_SP, __ldg(&r->shape[1]), npr, kr, dRr);
    if (GEN && rev == 2)
      dlnkr = DT(fma(__ldg(m.tab + __ldg(&r->tab_lo) + 2), invT2, __ldg(m.tab + __ldg(&r->tab_lo) + 1) * invT));
    else
      dlnkr = dlnkf - DT(dh - __ldg(&r->dnu)) * invT_t;
  }
  const double Rn = Rf - Rr;
  const DT Rn_t = DT(Rn);

  // pressure modification c (FP64) and its derivatives (DT)
  double c = 1.0;
  DT dcdT = 0, dcdS = 0, dcdM = 0;
  if (has_third_body(kind)) {
    const double M = third_body(m, A, aC, r, Ctot);
    const DT ab = DT(__ldg(&r->alpha_bath));
    const DT dMdT = ab * dCb_T_t;
    const DT dMdS = MODE == PJ_CONP ? (ab * DT(Ctot) - DT(M)) * invV_t : ab * DT(Ctot / P);
    if (kind == PJ_THIRD_BODY) {
      c = M;
      dcdM = DT(1);
      dcdT = dMdT;
      dcdS = dMdS;
    } else {
      const double beta0 = __ldg(&r->beta0), theta0 = __ldg(&r->theta0);
      const double lnk0 = fma(beta0, lnT, __ldg(&r->lnA0)) - theta0 * invT;
      const double dlnk0 = fma(theta0, invT2, beta0 * invT);
      // per-reaction scalars of the blending function, in FP64 whatever DT
      // (its derivative can subtract terms of similar size)
      const double rk = pj_exp(lnk0 - lnkinf);
      const double Pr = rk * M;
      double FxPr, FT;
      const double F = falloff_F<true, double>(r, kind, T, invT, lnT, Pr, FxPr, FT);
      const double i1p = 1.0 / (1.0 + Pr);
      const double ab_d = __ldg(&r->alpha_bath);
      const double dMdT_d = ab_d * v.dCb_T;
      const double dMdS_d = MODE == PJ_CONP ? (ab_d * Ctot - M) * invV : ab_d * Ctot / P;
      const double dPrdT = Pr * (dlnk0 - dlnkinf_d) + rk * dMdT_d;
      double cPr, dcdT_d;
      if (GEN && __ldg(&r->chem)) {
        // c = F / (1 + Pr): dc/dPr = (dF/dPr) / (1 + Pr) - F / (1 + Pr)^2
        c = F * i1p;
        cPr = i1p * (FxPr / Pr - F * i1p);
        dcdT_d = i1p * FT + cPr * dPrdT;
      } else {
        // c = F Pr / (1 + Pr)
        const double fr = Pr * i1p;
        c = fr * F;
        cPr = F * i1p * i1p + FxPr * i1p;
        dcdT_d = fr * FT + cPr * dPrdT;
      }
      dcdT = DT(dcdT_d);
      dcdM = DT(cPr * rk);
      dcdS = DT(cPr * rk * dMdS_d);
    }
  }
  const DT c_t = DT(c);
  DT dRf_t[PJ_MAX_SP], dRr_t[PJ_MAX_SP];
#pragma unroll
  for (int a = 0; a < PJ_MAX_SP; a++) {
    dRf_t[a] = a < nre ? DT(dRf[a]) : DT(0);
    dRr_t[a] = (rev && a < npr) ? DT(dRr[a]) : DT(0);
  }

  // derivatives of the net rate in T and S (rate constants, and the bath
  // gas through C_Ns = C_tot - sum C_k)
  // (the bath gas's terms only in reactions that have it, under a branch of
  // their own: FP64 work under a per-species condition is otherwise issued,
  // predicated off, for every species)
  DT dRdT = DT(Rf) * dlnkf - DT(Rr) * dlnkr;
  DT dRdS = DT(0);
  if (MODE == PJ_CONP) {
#pragma unroll
    for (int a = 0; a < PJ_MAX_SP; a++) {
      if (a < nre) {
        const int k = __ldg(&r->sp[a]);
        const double ck = k == bath ? 0.0 : A.at(aC, k);  // a select, not a branch
        dRdS = dRdS - dRf_t[a] * (DT(ck) * invV_t);
      }
      if (rev && a < npr) {
        const int k = __ldg(&r->sp[PJ_MAX_SP + a]);
        const double ck = k == bath ? 0.0 : A.at(aC, k);
        dRdS = dRdS + dRr_t[a] * (DT(ck) * invV_t);
      }
    }
  }
  if (__ldg(&r->bath_in)) {
    for (int a = 0; a < PJ_MAX_SP; a++) {
      if (a < nre && __ldg(&r->sp[a]) == bath) {
        dRdT = dRdT + dRf_t[a] * dCb_T_t;
        dRdS = dRdS + dRf_t[a] * dCb_S_t;
      }
      if (rev && a < npr && __ldg(&r->sp[PJ_MAX_SP + a]) == bath) {
        dRdT = dRdT - dRr_t[a] * dCb_T_t;
        dRdS = dRdS - dRr_t[a] * dCb_S_t;
      }
    }
  }
  if (GEN && MODE == PJ_CONV && kind >= PJ_PLOG) {
    // P-log / Chebyshev rates depend on P = S (held fixed in CONP); an
    // explicit reverse rate does not
    const DT dP = DT(dlnP_d / P);
    dRdS = dRdS + DT(Rf) * dP - (rev == 1 ? DT(Rr) * dP : DT(0));
  }
  const double q = c * Rn;
  const DT dqdT = c_t * dRdT + Rn_t * dcdT;
  const DT dqdS = c_t * dRdS + Rn_t * dcdS;
  scatter_wdot(r, nre, npr, bath, q, o.wrow, ld, v.w_bath, w);

  // energy-row and state-row weights of this reaction
  const DT dE = DT(RU * T * (MODE == PJ_CONP ? dh : dh - __ldg(&r->dnu)));
  const DT dW = DT(__ldg(&r->dW));
  v.AT_T = v.AT_T + dE * dqdT;
  v.AT_S = v.AT_S + dE * dqdS;
  v.AS_T = v.AS_T + dW * dqdT;
  v.AS_S = v.AS_S + dW * dqdS;

  int row_lo = __ldg(&r->row_lo), row_hi = __ldg(&r->row_hi);
  if (!PJ_DBG_OK(m.dbg, row_lo >= 0 && row_lo <= row_hi && row_hi <= m.n_rows, PJ_DBG_ROWS)) row_hi = row_lo = 0;
  const DT VdqdT = nscale<NEWTON>(o, V_t * dqdT), VdqdS = nscale<NEWTON>(o, V_t * dqdS);
  // sparse targets in the order of the reaction's target list (the host
  // builds it in exactly the order of the contributions below); dense
  // positions are plain arithmetic
  const int32_t* tg = FMT == PJ_CSR ? m.tgt_csr + __ldg(&r->tgt_lo) : m.tgt_csc + __ldg(&r->tgt_lo);
  auto target = [&](int row, int col) -> int64_t {
    if (FMT == PJ_DENSE) {
      if (!PJ_DBG_OK(m.dbg, row >= 0 && row < m.N && col >= 0 && col < m.N, PJ_DBG_POSMAP)) return -1;
      return (int64_t)row * m.N + col;
    }
#ifdef PJ_DEBUG_BOUNDS
    const int32_t* base = FMT == PJ_CSR ? m.tgt_csr : m.tgt_csc;
    if (!PJ_DBG_OK(m.dbg, tg >= base && tg < base + m.n_tgt, PJ_DBG_TARGET)) return -1;
#endif
    const int64_t e = __ldg(tg++);
    if (!PJ_DBG_OK(m.dbg, e >= -1 && e < m.nnz, PJ_DBG_TARGET)) return -1;
    return e;
  };
  for (int q2 = row_lo; q2 < row_hi; q2++) {
    const RowNu rn = m.rows[q2];
    const int64_t e0 = target(rn.k + 2, 0), e1 = target(rn.k + 2, 1);
    if (w) jred(J, e0, ld, s, nu_times_t<DT>(rn.nu, rn.nud, VdqdT));
    if (w) jred(J, e1, ld, s, nu_times_t<DT>(rn.nu, rn.nud, VdqdS));
  }

  // species columns: V dq/dn_j = c dR/dC_j + R dc/dM (alpha_j - 1) + B_i;
  // the bath gas's own terms make B_i (below, dense reactions only)
  auto slot = [&](int j, DT val) {
    if (j == bath) return;
    const DT vs = nscale<NEWTON>(o, val);
    for (int q2 = row_lo; q2 < row_hi; q2++) {
      const RowNu rn = m.rows[q2];
      const int64_t e = target(rn.k + 2, j + 2);
      if (w) jred(J, e, ld, s, nu_times_t<DT>(rn.nu, rn.nud, vs));
    }
    const int64_t eT = target(0, j + 2), eS = target(1, j + 2);
    if (w) jred(J, eT, ld, s, dE * vs);
    if (w) jred(J, eS, ld, s, dW * vs);
  };
#pragma unroll
  for (int a = 0; a < PJ_MAX_SP; a++) {
    if (a < nre) slot(__ldg(&r->sp[a]), c_t * dRf_t[a]);
    if (rev && a < npr) slot(__ldg(&r->sp[PJ_MAX_SP + a]), dneg(c_t * dRr_t[a]));
  }
  if (has_third_body(kind)) {
    const DT t = Rn_t * dcdM;
    for (int e = __ldg(&r->eff_lo), eh = __ldg(&r->eff_hi); e < eh; e++) {
      if (!PJ_DBG_OK(m.dbg, e >= 0 && e < m.n_eff, PJ_DBG_EFF)) break;
      slot(__ldg(m.eff_sp + e), t * DT(__ldg(m.eff_am1 + e)));
    }
  }
  if (__ldg(&r->dense)) {
    // B_i: minus the terms the slots above have for the bath gas, in their order
    DT Bi = DT(0);
    for (int a = 0; a < PJ_MAX_SP; a++) {
      if (a < nre && __ldg(&r->sp[a]) == bath) Bi = Bi - c_t * dRf_t[a];
      if (rev && a < npr && __ldg(&r->sp[PJ_MAX_SP + a]) == bath) Bi = Bi - dneg(c_t * dRr_t[a]);
    }
    if (has_third_body(kind)) {
      const DT t = Rn_t * dcdM;
      for (int e = __ldg(&r->eff_lo), eh = __ldg(&r->eff_hi); e < eh; e++) {
        if (!PJ_DBG_OK(m.dbg, e >= 0 && e < m.n_eff, PJ_DBG_EFF)) break;
        if (__ldg(m.eff_sp + e) == bath) Bi = Bi - t * DT(__ldg(m.eff_am1 + e));
      }
    }
    const DT Bs = nscale<NEWTON>(o, Bi);
    for (int q2 = row_lo; q2 < row_hi; q2++) {
      const RowNu rn = m.rows[q2];
      const DT val = nu_times_t<DT>(rn.nu, rn.nud, Bs);
      if (FMT == PJ_CSR) {
        // a dense row holds every species column, contiguous in CSR
        const int64_t e2 = jpos<FMT>(m, rn.k + 2, 2);
        if (!PJ_DBG_OK(m.dbg, e2 >= 0 && e2 + ns - 1 <= m.nnz, PJ_DBG_POSMAP)) continue;
        for (int j = 0; j < ns - 1; j++) if (w) jred(J, e2 + j, ld, s, val);
      } else {
        for (int j = 0; j < ns - 1; j++) if (w) jred(J, jpos<FMT>(m, rn.k + 2, j + 2), ld, s, val);
      }
    }
    v.ATB = v.ATB + dE * Bi;
    v.ASB = v.ASB + dW * Bi;
  }
}

// Species k after every reaction: Cx_k = R cp_k (CONP) or R cv_k (CONV) is
// returned; the production rate wdot_k (the bath gas: w_bath) is written as
// dn_k/dt = V wdot_k and, in CONP, added to J[k+2, 1]; its terms of the
// energy-equation numerator, of sum_k Cx_k wdot_k and of the state equation
// are added to num, sumCxW and Om.
template <int MODE, int FMT, typename DT, bool NEWTON>
__device__ __forceinline__ double jac_species(const DevMech& m, int k, double T, double V, double hk,
                                              double w_bath, const JacOut<DT>& o, double& num, double& sumCxW,
                                              double& Om) {
  const int bath = m.ns - 1;
  double cp, dcp;
  nasa_cp(nasa_block(m, k, T), T, cp, dcp);
  const double cx = RU * (MODE == PJ_CONP ? cp : cp - 1.0);
  const double wk = k < bath ? (o.w ? __ldcg(o.wrow + (int64_t)k * o.ld) : 0.0) : w_bath;
  num = fma(MODE == PJ_CONP ? hk : hk - 1.0, wk, num);
  sumCxW = fma(cx, wk, sumCxW);
  if (k < bath) {
    Om = fma(__ldg(m.wfac + k), wk, Om);
    if (o.w) o.wrow[(int64_t)k * o.ld] = V * wk;
    if (MODE == PJ_CONP) if (o.w) jred(o.J, jpos<FMT>(m, k + 2, 1), o.ld, o.s, nscale<NEWTON>(o, DT(wk)));
  }
  return cx;
}

// Per-state values the energy and state rows need once every reaction and
// species has been accumulated, formed once per state (jac_row_vars).
template <typename DT>
struct JacRowVars {
  double Cx_b;                     // Cx of the bath gas (differences Cx_j - Cx_b in FP64)
  DT iden, Tdot, invV, rtvp, cT;   // 1/D, dT/dt, 1/V, R T V/P (CONP) or R T (CONV), V/T or P/T
  DT j00, j01;                     // row 0, columns 0 and 1, less the accumulated weights
  DT x0, x1;                       // the state row's own terms in columns 0 and 1
  DT AT_T, AT_S, AS_T, AS_S, ATB, ASB;
};

template <int MODE, typename DT>
__device__ __forceinline__ JacRowVars<DT> jac_row_vars(double T, double V, double P, double invT, double Tdot,
                                                       double Om, double den, double dden_T, double dden_S,
                                                       double sumCxW, double Cx_b, DT AT_T, DT AT_S, DT AS_T,
                                                       DT AS_S, DT ATB, DT ASB) {
  JacRowVars<DT> x;
  const double invT2 = invT * invT;
  x.Cx_b = Cx_b;
  x.iden = DT(1.0 / den);
  x.Tdot = DT(Tdot);
  x.invV = DT(1.0 / V);
  x.rtvp = DT(MODE == PJ_CONP ? RU * T * V / P : RU * T);
  x.cT = DT(MODE == PJ_CONP ? V * invT : P * invT);
  x.j00 = DT(sumCxW) + x.Tdot * DT(dden_T);
  x.j01 = x.Tdot * DT(dden_S);
  if (MODE == PJ_CONP) {
    x.x0 = DT(-V * Tdot * invT2 + (RU * V / P) * Om);
    x.x1 = DT(Tdot * invT + (RU * T / P) * Om);
  } else {
    x.x0 = DT(-P * Tdot * invT2 + RU * Om);
    x.x1 = DT(Tdot * invT);
  }
  x.AT_T = AT_T;
  x.AT_S = AT_S;
  x.AS_T = AS_T;
  x.AS_S = AS_S;
  x.ATB = ATB;
  x.ASB = ASB;
  return x;
}

// Column j of the energy row 0 and the state row 1 (cx_j: Cx of species
// j-2 for a species column).  The species columns read the per-entry sums
// the reactions accumulated there and overwrite them with the final values.
// Newton form: the accumulated sums already carry -h gamma, the per-state
// terms take it here, and the diagonal entries (0,0) and (1,1) get the 1.
// COL: 0 and 1 for the T and S columns (j == COL), 2 for the species
// columns j >= 2, so that no column carries the other kinds' arithmetic (a
// runtime test of j leaves the branches' FP64 instructions in every column,
// predicated off).
template <int MODE, int FMT, typename DT, bool NEWTON, int COL>
__device__ __forceinline__ void jac_ts_column(const DevMech& m, int j, double cx_j, const JacRowVars<DT>& x,
                                              const JacOut<DT>& o) {
  const int64_t ld = o.ld, s = o.s;
  DT* __restrict__ J = o.J;
  const int64_t e0 = jpos<FMT>(m, 0, j), e1 = jpos<FMT>(m, 1, j);
#ifdef PJ_DEBUG_BOUNDS
  if (e0 < 0 || e1 < 0) return;  // a bad map entry (recorded by jpos)
#endif
  DT jT, dOm;
  if constexpr (COL == 0) {
    jT = -nscale<NEWTON>(o, x.AT_T + x.j00) * x.iden;
    dOm = nscale<NEWTON>(o, x.AS_T);
  } else if constexpr (COL == 1) {
    jT = -nscale<NEWTON>(o, x.AT_S + x.j01) * x.iden;
    dOm = nscale<NEWTON>(o, x.AS_S);
  } else {
    const DT accT = o.w ? __ldcg(J + e0 * ld + s) : DT(0);
    const DT accS = o.w ? __ldcg(J + e1 * ld + s) : DT(0);
    // differences Cx_j - Cx_b are formed in FP64 (they can cancel)
    jT = -(accT + nscale<NEWTON>(o, x.ATB + x.Tdot * DT(cx_j - x.Cx_b))) * (x.invV * x.iden);
    dOm = (accS + nscale<NEWTON>(o, x.ASB)) * x.invV;
  }
  DT jS = x.cT * jT + x.rtvp * dOm;
  if constexpr (COL == 0) {
    jS = jS + nscale<NEWTON>(o, x.x0);
    if (NEWTON) jT = jT + DT(1);
  }
  if constexpr (COL == 1) {
    jS = jS + nscale<NEWTON>(o, x.x1);
    if (NEWTON) jS = jS + DT(1);
  }
  if (o.w) {
    J[e0 * ld + s] = jT;
    J[e1 * ld + s] = jS;
  }
}

// Newton form: the identity on the species diagonal, once every entry of
// this state is complete (the T and S diagonal entries take it in
// jac_ts_column).
template <int FMT, typename DT>
__device__ __forceinline__ void newton_species_diagonal(const DevMech& m, int k, const JacOut<DT>& o) {
  if (!o.w) return;
  const int64_t e = jpos<FMT>(m, k, k);
#ifdef PJ_DEBUG_BOUNDS
  if (e < 0) return;
#endif
  DT* p = o.J + e * o.ld + o.s;
  *p = __ldcg(p) + DT(1);
}

// One state of the Jacobian evaluation (arrays A of this thread).  With
// NEWTON the output is M = I - h*gamma*J (h per state): every contribution
// carries -h gamma, and the identity is added at the end.
//
// Production rates go to the source-term output by L2 reductions (bath gas
// in a register); Jacobian entries to the zero-initialised output by L2
// reductions.
//
// TM = false: s < n, h_k/RT in A (array 2); an invalid state returns early.
// TM = true: h_k/RT lives in this thread's TMEM row at tm_row (columns
// 2k, 2k+1) and every lane of the warp runs the whole body convergently (the
// TMEM accesses are warp-collective): a lane past the batch (act = false) or
// with an invalid state computes on a harmless dummy state with every global
// read and write of the batch masked.
template <int MODE, int FMT, typename DT, bool NEWTON, bool TM = false, bool SPECIAL = true,
          class SA = StateArrays>
__device__ __forceinline__ void jacobian_state(const DevMech& m, const SA& A,
                                               const double* __restrict__ param, const double* __restrict__ phi,
                                               int64_t ld, int64_t s, DT* __restrict__ J, double* __restrict__ dphi,
                                               int* status, const double* __restrict__ hstep, double gamma,
                                               uint32_t tm_row = 0, bool act = true) {
  const int ns = m.ns, N = m.N, bath = m.ns - 1;
  const int64_t n_out = FMT == PJ_DENSE ? (int64_t)N * N : (int64_t)m.nnz;
  enum { aC = 0, aG = 1, aH = 2 };
  StateScalars st;
  const bool ok = act && load_state<MODE>(m, phi, param, ld, s, A, aC, st);
  if (act && !ok) {
    const DT qnan = DT(__longlong_as_double(0x7ff8000000000000ULL));
    for (int64_t e = 0; e < n_out; e++) J[e * ld + s] = qnan;
    write_nan_state(dphi, ld, s, ns + 1);
    if (status) atomicAdd(status, 1);
  }
  if (!ok) {
    if (!TM) return;
    st.T = 1000.0;
    st.V = 1.0;
    st.P = 1e5;
    st.invT = 1e-3;
    st.lnT = log(1000.0);
    st.lnP = log(1e5);
    st.Ctot = st.P / (RU * st.T);
    for (int k = 0; k < ns; k++) A.at(aC, k) = st.Ctot / ns;
  }
  const bool w = ok;  // this lane reads and writes the batch
  auto h_at = [&](int k) -> double {
    if (TM) return tmem_ld_f64(tm_row + 2u * (uint32_t)k);
    return A.at(aH, k);
  };
  const double T = st.T, V = st.V, P = st.P, invT = st.invT, lnT = st.lnT, Ctot = st.Ctot;
  const double invT2 = invT * invT, invV = 1.0 / V;
  if (w)
    for (int64_t e = 0; e < n_out; e++) J[e * ld + s] = DT(0);
  double* __restrict__ wrow = dphi + 2 * ld + s;  // wdot_k accumulates at wrow[k*ld]
  if (w)
    for (int k = 0; k < ns - 1; k++) wrow[(int64_t)k * ld] = 0.0;
  if (TM) __syncwarp();

  // thermo, energy-equation denominator D = sum_k C_k Cx_k and dD/dT
  double den = 0.0, dden_T = 0.0, Cx_bath = 0.0;
  for (int k = 0; k < ns; k++) {
    const double* cb = nasa_block(m, k, T);
    double cp, h, sr, cp2, dcp;
    nasa_eval(cb, T, invT, lnT, cp, h, sr);
    nasa_cp(cb, T, cp2, dcp);
    A.at(aG, k) = h - sr;
    if (TM) tmem_st_f64(tm_row + 2u * (uint32_t)k, h);
    else A.at(aH, k) = h;
    const double Ck = A.at(aC, k);
    const double cx = MODE == PJ_CONP ? cp : cp - 1.0;
    den = fma(Ck, cx, den);
    dden_T = fma(Ck, dcp, dden_T);
    if (k == bath) Cx_bath = RU * cx;
  }
  if (TM) tmem_wait_st();
  den *= RU;
  const double C_bath = A.at(aC, bath);
  JacVars<DT> v;
  v.T = T;
  v.V = V;
  v.P = P;
  v.invT = invT;
  v.lnT = lnT;
  v.lnP = st.lnP;
  v.Ctot = Ctot;
  v.invT2 = invT2;
  v.invV = invV;
  v.logPRT = m.log_pstd_over_r - lnT;
  // derivatives of the bath-gas concentration
  v.dCb_T = -Ctot * invT;
  v.dCb_S = MODE == PJ_CONP ? (Ctot - C_bath) * invV : Ctot / P;
  dden_T = RU * dden_T + Cx_bath * v.dCb_T;
  const double dden_S = MODE == PJ_CONP ? (Cx_bath * Ctot - den) * invV : Cx_bath * Ctot / P;
  v.AT_T = v.AT_S = v.AS_T = v.AS_S = v.ATB = v.ASB = DT(0);
  v.w_bath = 0.0;
  const JacOut<DT> o{J, wrow, ld, s, w, NEWTON && w ? DT(-hstep[s] * gamma) : DT(0)};

  // Plain reactions (the first m.nr_plain in kernel order) run through a
  // body compiled without the special cases (chemically activated, explicit
  // reverse, P-log, Chebyshev), the rest through the general one; kernels for
  // mechanisms without special reactions are instantiated with SPECIAL =
  // false and carry no general body at all.
  for (int i = 0; i < m.nr_plain; i++) jac_reaction<MODE, FMT, DT, false, TM, NEWTON>(m, A, v, o, i, tm_row);
  if (SPECIAL)
    for (int i = m.nr_plain; i < m.nr; i++) jac_reaction<MODE, FMT, DT, true, TM, NEWTON>(m, A, v, o, i, tm_row);

  // source terms; the G array now holds Cx_k = R (cp_k or cv_k)
  if (TM) __syncwarp();
  double num = 0.0, Om = 0.0, sumCxW = 0.0;
  for (int k = 0; k < ns; k++)
    A.at(aG, k) = jac_species<MODE, FMT, DT, NEWTON>(m, k, T, V, h_at(k), v.w_bath, o, num, sumCxW, Om);
  num *= RU * T;
  const double Tdot = -num / den;
  const double Sdot = MODE == PJ_CONP ? V * Tdot * invT + (RU * T * V / P) * Om : P * Tdot * invT + RU * T * Om;
  if (w) {
    dphi[s] = Tdot;
    dphi[ld + s] = Sdot;
  }

  // energy row 0 and state row 1
  const JacRowVars<DT> x = jac_row_vars<MODE, DT>(T, V, P, invT, Tdot, Om, den, dden_T, dden_S, sumCxW,
                                                  A.at(aG, bath), v.AT_T, v.AT_S, v.AS_T, v.AS_S, v.ATB, v.ASB);
  jac_ts_column<MODE, FMT, DT, NEWTON, 0>(m, 0, 0.0, x, o);
  jac_ts_column<MODE, FMT, DT, NEWTON, 1>(m, 1, 0.0, x, o);
  for (int j = 2; j < N; j++) jac_ts_column<MODE, FMT, DT, NEWTON, 2>(m, j, A.at(aG, j - 2), x, o);
  if (NEWTON)
    for (int k = 2; k < N; k++) newton_species_diagonal<FMT>(m, k, o);
}

}  // namespace pj
