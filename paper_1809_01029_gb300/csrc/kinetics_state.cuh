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
  if (FMT == PJ_DENSE) return (int64_t)row * m.N + col;
  const int32_t* p = FMT == PJ_CSR ? m.pos_csr : m.pos_csc;
  return __ldg(p + (int64_t)row * m.N + col);
}

__device__ __forceinline__ void red_add(float* p, float v) { atomicAdd(p, v); }  // red.global.add.f32

template <typename DT>
__device__ __forceinline__ void jred(DT* J, int64_t e, int64_t ld, int64_t s, DT v) {
  if (e >= 0) red_add(J + e * ld + s, v);
}

__device__ __forceinline__ float dneg(float x) { return -x; }

template <typename DT>
__device__ __forceinline__ DT nu_times_t(int nu, double nud, DT x) {
  if (nu == 1) return x;
  if (nu == -1) return dneg(x);
  return DT(nud) * x;
}

// Analytical Jacobian (Sec. 2.2, Sec. 3.4).  Rates, equilibrium constants,
// exponentials and source terms are always FP64.  DT is the type of the
// derivative arithmetic, the entry accumulation and the output: double for
// J itself, float for the Newton-matrix form.  With NEWTON the final pass
// turns the accumulated J into M = I - h*gamma*J in place (h per state).
//
// Shared memory holds C_k, g_k/RT and h_k/RT per state.  Production rates go
// to the source-term output by L2 reductions (bath gas in a register);
// Jacobian entries to the zero-initialised output by L2 reductions.
// One state of the Jacobian evaluation (arrays A of this thread).
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
  const DT invT_t = DT(invT), invT2_t = DT(invT2), invV_t = DT(invV), V_t = DT(V);
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
  // derivatives of the bath-gas concentration
  const double dCb_T = -Ctot * invT;
  const double dCb_S = MODE == PJ_CONP ? (Ctot - C_bath) * invV : Ctot / P;
  const DT dCb_T_t = DT(dCb_T), dCb_S_t = DT(dCb_S);
  dden_T = RU * dden_T + Cx_bath * dCb_T;
  const double dden_S = MODE == PJ_CONP ? (Cx_bath * Ctot - den) * invV : Cx_bath * Ctot / P;
  const double logPRT = m.log_pstd_over_r - lnT;

  // accumulators of the energy row (T) and state row (S) for the T and S
  // columns and for the part common to every species column
  DT AT_T = 0, AT_S = 0, AS_T = 0, AS_S = 0, ATB = 0, ASB = 0;
  double w_bath = 0;

  // Plain reactions (the first m.nr_plain in kernel order) run through a
  // body compiled without the special cases (chemically activated, explicit
  // reverse, P-log, Chebyshev), the rest through the general one; kernels for
  // mechanisms without special reactions are instantiated with SPECIAL =
  // false and carry no general body at all.
  auto reaction = [&](int i, auto gen_tag) {
    constexpr bool GEN = decltype(gen_tag)::value;
    const Rxn* __restrict__ r = m.rxn + i;
    const int kind = __ldg(&r->kind);
    const int nre = __ldg(&r->nreac), npr = __ldg(&r->nprod);
    const int rev = __ldg(&r->rev);
    double lnkinf, dlnkf_d, dlnP_d, dlnkinf_d;
    const double lnkf = ln_kf<true, GEN>(m, r, kind, lnT, invT, st.lnP, lnkinf, dlnkf_d, dlnP_d, dlnkinf_d);
    const DT dlnkf = DT(dlnkf_d);
    double kf, kr;
    rate_constants<GEN>(m, A, aG, r, rev, nre, npr, lnkf, logPRT, lnT, invT, kf, kr);
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
        const double dMdT_d = ab_d * dCb_T;
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
    DT dRdT = DT(Rf) * dlnkf - DT(Rr) * dlnkr;
    DT dRdS = DT(0);
#pragma unroll
    for (int a = 0; a < PJ_MAX_SP; a++) {
      if (a < nre) {
        const int k = __ldg(&r->sp[a]);
        if (k == bath) {
          dRdT = dRdT + dRf_t[a] * dCb_T_t;
          dRdS = dRdS + dRf_t[a] * dCb_S_t;
        } else if (MODE == PJ_CONP) {
          dRdS = dRdS - dRf_t[a] * (DT(A.at(aC, k)) * invV_t);
        }
      }
      if (rev && a < npr) {
        const int k = __ldg(&r->sp[PJ_MAX_SP + a]);
        if (k == bath) {
          dRdT = dRdT - dRr_t[a] * dCb_T_t;
          dRdS = dRdS - dRr_t[a] * dCb_S_t;
        } else if (MODE == PJ_CONP) {
          dRdS = dRdS + dRr_t[a] * (DT(A.at(aC, k)) * invV_t);
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
#pragma unroll
    for (int a = 0; a < PJ_MAX_SP; a++) {
      if (a < nre) {
        const int k = __ldg(&r->sp[a]);
        const double v = nu_times(__ldg(&r->nu[a]), __ldg(&r->nud[a]), q);
        if (k == bath) w_bath -= v;
        else if (w) red_add(wrow + (int64_t)k * ld, dneg(v));
      }
      if (a < npr) {
        const int k = __ldg(&r->sp[PJ_MAX_SP + a]);
        const double v = nu_times(__ldg(&r->nu[PJ_MAX_SP + a]), __ldg(&r->nud[PJ_MAX_SP + a]), q);
        if (k == bath) w_bath += v;
        else if (w) red_add(wrow + (int64_t)k * ld, v);
      }
    }

    // energy-row and state-row weights of this reaction
    const DT dE = DT(RU * T * (MODE == PJ_CONP ? dh : dh - __ldg(&r->dnu)));
    const DT dW = DT(__ldg(&r->dW));
    AT_T = AT_T + dE * dqdT;
    AT_S = AT_S + dE * dqdS;
    AS_T = AS_T + dW * dqdT;
    AS_S = AS_S + dW * dqdS;

    const int row_lo = __ldg(&r->row_lo), row_hi = __ldg(&r->row_hi);
    const DT VdqdT = V_t * dqdT, VdqdS = V_t * dqdS;
    // sparse targets in the order of the reaction's target list (the host
    // builds it in exactly the order of the contributions below); dense
    // positions are plain arithmetic
    const int32_t* tg = FMT == PJ_CSR ? m.tgt_csr + __ldg(&r->tgt_lo) : m.tgt_csc + __ldg(&r->tgt_lo);
    auto target = [&](int row, int col) -> int64_t {
      if (FMT == PJ_DENSE) return (int64_t)row * m.N + col;
      return __ldg(tg++);
    };
    for (int q2 = row_lo; q2 < row_hi; q2++) {
      const RowNu rn = m.rows[q2];
      const int64_t e0 = target(rn.k + 2, 0), e1 = target(rn.k + 2, 1);
      if (w) jred(J, e0, ld, s, nu_times_t<DT>(rn.nu, rn.nud, VdqdT));
      if (w) jred(J, e1, ld, s, nu_times_t<DT>(rn.nu, rn.nud, VdqdS));
    }

    // species columns: V dq/dn_j = c dR/dC_j + R dc/dM (alpha_j - 1) + B_i
    DT Bi = DT(0);
    auto slot = [&](int j, DT val) {
      if (j == bath) {
        Bi = Bi - val;
        return;
      }
      for (int q2 = row_lo; q2 < row_hi; q2++) {
        const RowNu rn = m.rows[q2];
        const int64_t e = target(rn.k + 2, j + 2);
        if (w) jred(J, e, ld, s, nu_times_t<DT>(rn.nu, rn.nud, val));
      }
      const int64_t eT = target(0, j + 2), eS = target(1, j + 2);
      if (w) jred(J, eT, ld, s, dE * val);
      if (w) jred(J, eS, ld, s, dW * val);
    };
#pragma unroll
    for (int a = 0; a < PJ_MAX_SP; a++) {
      if (a < nre) slot(__ldg(&r->sp[a]), c_t * dRf_t[a]);
      if (rev && a < npr) slot(__ldg(&r->sp[PJ_MAX_SP + a]), dneg(c_t * dRr_t[a]));
    }
    if (has_third_body(kind)) {
      const DT t = Rn_t * dcdM;
      for (int e = __ldg(&r->eff_lo), eh = __ldg(&r->eff_hi); e < eh; e++)
        slot(__ldg(m.eff_sp + e), t * DT(__ldg(m.eff_am1 + e)));
    }
    if (__ldg(&r->dense)) {
      for (int q2 = row_lo; q2 < row_hi; q2++) {
        const RowNu rn = m.rows[q2];
        const DT v = nu_times_t<DT>(rn.nu, rn.nud, Bi);
        if (FMT == PJ_CSR) {
          // a dense row holds every species column, contiguous in CSR
          const int64_t e2 = jpos<FMT>(m, rn.k + 2, 2);
          for (int j = 0; j < ns - 1; j++) if (w) jred(J, e2 + j, ld, s, v);
        } else {
          for (int j = 0; j < ns - 1; j++) if (w) jred(J, jpos<FMT>(m, rn.k + 2, j + 2), ld, s, v);
        }
      }
      ATB = ATB + dE * Bi;
      ASB = ASB + dW * Bi;
    }
  };
  for (int i = 0; i < m.nr_plain; i++) reaction(i, BoolTag<false>{});
  if (SPECIAL)
    for (int i = m.nr_plain; i < m.nr; i++) reaction(i, BoolTag<true>{});

  // source terms; the G array now holds Cx_k = R (cp_k or cv_k)
  if (TM) __syncwarp();
  double num = 0.0, Om = 0.0, sumCxW = 0.0;
  for (int k = 0; k < ns; k++) {
    double cp, dcp;
    nasa_cp(nasa_block(m, k, T), T, cp, dcp);
    const double cx = RU * (MODE == PJ_CONP ? cp : cp - 1.0);
    A.at(aG, k) = cx;
    const double wk = k < bath ? (w ? __ldcg(wrow + (int64_t)k * ld) : 0.0) : w_bath;
    const double hk = h_at(k);
    num = fma(MODE == PJ_CONP ? hk : hk - 1.0, wk, num);
    sumCxW = fma(cx, wk, sumCxW);
    if (k < bath) {
      Om = fma(__ldg(m.wfac + k), wk, Om);
      if (w) wrow[(int64_t)k * ld] = V * wk;
      if (MODE == PJ_CONP) if (w) jred(J, jpos<FMT>(m, k + 2, 1), ld, s, DT(wk));
    }
  }
  num *= RU * T;
  const double Tdot = -num / den;
  const double Sdot = MODE == PJ_CONP ? V * Tdot * invT + (RU * T * V / P) * Om : P * Tdot * invT + RU * T * Om;
  if (w) {
    dphi[s] = Tdot;
    dphi[ld + s] = Sdot;
  }

  // energy row 0 and state row 1
  const DT iden = DT(1.0 / den);
  const DT Tdot_t = DT(Tdot), Om_t = DT(Om);
  const double Cx_b = A.at(aG, bath);  // differences Cx_j - Cx_b are formed in FP64 (they can cancel)
  const DT rtvp = DT(MODE == PJ_CONP ? RU * T * V / P : RU * T);
  for (int j = 0; j < N; j++) {
    const int64_t e0 = jpos<FMT>(m, 0, j), e1 = jpos<FMT>(m, 1, j);
    DT jT, dOm;
    if (j == 0) {
      jT = -(AT_T + DT(sumCxW) + Tdot_t * DT(dden_T)) * iden;
      dOm = AS_T;
    } else if (j == 1) {
      jT = -(AT_S + Tdot_t * DT(dden_S)) * iden;
      dOm = AS_S;
    } else {
      const DT accT = w ? __ldcg(J + e0 * ld + s) : DT(0);
      const DT accS = w ? __ldcg(J + e1 * ld + s) : DT(0);
      jT = -(accT + ATB + Tdot_t * DT(A.at(aG, j - 2) - Cx_b)) * (invV_t * iden);
      dOm = (accS + ASB) * invV_t;
    }
    DT jS;
    if (MODE == PJ_CONP) {
      jS = DT(V * invT) * jT + rtvp * dOm;
      if (j == 0) jS = jS + DT(-V * Tdot * invT2 + (RU * V / P) * Om);
      if (j == 1) jS = jS + DT(Tdot * invT + (RU * T / P) * Om);
    } else {
      jS = DT(P * invT) * jT + rtvp * dOm;
      if (j == 0) jS = jS + DT(-P * Tdot * invT2 + RU * Om);
      if (j == 1) jS = jS + DT(Tdot * invT);
    }
    if (w) {
      J[e0 * ld + s] = jT;
      J[e1 * ld + s] = jS;
    }
  }

  if (NEWTON && w) {
    // M = I - h gamma J, in place (this thread's column only)
    const DT hg = DT(-hstep[s] * gamma);
    for (int64_t e = 0; e < n_out; e++) {
      DT* p = J + e * ld + s;
      *p = hg * __ldcg(p);
    }
    for (int k = 0; k < N; k++) {
      DT* p = J + jpos<FMT>(m, k, k) * ld + s;
      *p = *p + DT(1);
    }
  }
}

}  // namespace pj
