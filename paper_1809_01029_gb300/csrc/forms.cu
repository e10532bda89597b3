// Differentiation form: vector-Jacobian products of y = (wdot_0 .. wdot_{Ns-1},
// dT/dt) with respect to the state and to the per-reaction Arrhenius
// parameters theta_i = (ln A_i, beta_i, Ea_i) of the high-pressure (or only)
// rate, plus the forward evaluation of y.
//
// Adjoint structure (Sec. 2.2 rates): y depends on the state through the net
// rates q_i and, for dT/dt, through the species energies and the heat
// capacity sum D.  With cotangent u = (u_wdot, u_T),
//   ubar_i = sum_k nu_ki u_k - u_T dE_i / D        (adjoint of q_i)
//   g_Phi  = sum_i ubar_i grad q_i - u_T (delta_jT sum_k Cx_k wdot_k + Tdot grad D) / D
//   g_theta_i = sum_states ubar_i dq_i/dtheta_i,  dq_i/dtheta = (1, ln T, -1/(R_cal T)) Q_i
// with Q_i = q_i for non-falloff reactions and q_i - R_i Pr dc/dPr for falloff
// (k_inf scales R and divides Pr).  Parameter gradients are summed per warp
// by shuffles, per warp by L2 reductions into a workspace slot the warp owns,
// then over warps in a fixed order: deterministic for a given launch shape.
#include <cuda_runtime.h>

#include "kinetics_common.cuh"

namespace pj {

#ifndef PJ_WARP_SUM
constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
  return v;
}
#define PJ_LANE0(lane) ((lane) == 0)
#endif

// Forward values y = (wdot_0 .. wdot_{Ns-1}, dT/dt): y[k*ld + s].
template <int MODE, bool SPECIAL>
__global__ void __launch_bounds__(128) k_eval_y(DevMech m, int64_t n, const double* __restrict__ param,
                                                const double* __restrict__ phi, int64_t ld, double* __restrict__ y,
                                                int* status, double* ws, int64_t ws_stride) {
  PJ_DYN_SMEM;
  load_exp_table(m.exp_tab);
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
      write_nan_state(y, ld, s, ns + 1);
      if (status) atomicAdd(status, 1);
      continue;
    }
    const double T = st.T, invT = st.invT, lnT = st.lnT;
    double* __restrict__ wrow = y + s;
    for (int k = 0; k < ns - 1; k++) wrow[(int64_t)k * ld] = 0.0;
    double den = 0.0;
    for (int k = 0; k < ns; k++) {
      double cp, h, sr;
      nasa_eval(nasa_block(m, k, T), T, invT, lnT, cp, h, sr);
      A.at(aG, k) = h - sr;
      den = fma(A.at(aC, k), MODE == PJ_CONP ? cp : cp - 1.0, den);
    }
    den *= RU;
    const double logPRT = m.log_pstd_over_r - lnT;
    double w_bath = 0.0;
    // Plain reactions (the first m.nr_plain in kernel order) run through a
    // body compiled without the special cases (chemically activated, explicit
    // reverse, P-log, Chebyshev), the rest through the general one.
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
          c = ((GEN && __ldg(&r->chem)) ? 1.0 : Pr) / (1.0 + Pr) * F;
        }
      }
      const double q = c * (Rf - Rr);
      scatter_wdot(r, nre, npr, bath, q, wrow, ld, w_bath);
    };
    for (int i = 0; i < m.nr_plain; i++) reaction(i, BoolTag<false>{});
    if (SPECIAL)
      for (int i = m.nr_plain; i < m.nr; i++) reaction(i, BoolTag<true>{});

    double num = 0.0;
    for (int k = 0; k < ns; k++) {
      double cp, h, sr;
      nasa_eval(nasa_block(m, k, T), T, invT, lnT, cp, h, sr);
      const double wk = k < bath ? __ldcg(wrow + (int64_t)k * ld) : w_bath;
      num = fma(MODE == PJ_CONP ? h : h - 1.0, wk, num);
    }
    wrow[(int64_t)bath * ld] = w_bath;
    y[(int64_t)ns * ld + s] = -(num * RU * T) / den;
  }
}

// VJP.  Warps walk the batch 32 states at a time so that the per-reaction
// parameter gradients can be summed over the warp with shuffles.  The
// forward values y are produced on the way (needed for dT/dt's direct terms).
constexpr int kVjpCtas = 4;  // resident blocks of 128 threads per SM (at most 128 registers)

template <int MODE, bool SPECIAL>
__global__ void __launch_bounds__(128, kVjpCtas) k_vjp(DevMech m, int64_t n, const double* __restrict__ param,
                                             const double* __restrict__ phi, int64_t ld,
                                             const double* __restrict__ u_wdot, const double* __restrict__ u_T,
                                             double* __restrict__ y, double* __restrict__ g_phi,
                                             double* __restrict__ gth_part, int* status, double* ws,
                                             int64_t ws_stride) {
  PJ_DYN_SMEM;
  load_exp_table(m.exp_tab);
  const int ns = m.ns, bath = m.ns - 1, nr = m.nr;
  const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const int64_t warp = gtid >> 5;
  double* __restrict__ my_part = gth_part + warp * (int64_t)nr * 3;
  StateArrays A;
  A.ns = ns;
  if (ws) {
    A.base = ws + gtid;
    A.stride = ws_stride;
  } else {
    A.base = smem + threadIdx.x;
    A.stride = blockDim.x;
  }
  enum { aC = 0, aG = 1, aH = 2, aU = 3 };
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = gtid - lane; base < n; base += stride) {
    const int64_t s = base + lane;
    const bool in = s < n;
    StateScalars st;
    bool ok = false;
    if (in) {
      ok = load_state<MODE>(m, phi, param, ld, s, A, aC, st);
      if (!ok) {
        write_nan_state(g_phi, ld, s, ns + 1);
        write_nan_state(y, ld, s, ns + 1);
        if (status) atomicAdd(status, 1);
      }
    }
    // lanes without a valid state follow the same instruction stream on a
    // harmless state and contribute zero
    if (!ok) {
      st.T = 1000.0;
      st.V = 1.0;
      st.P = 1e5;
      st.invT = 1e-3;
      st.lnT = log(1000.0);
      st.lnP = log(1e5);
      st.Ctot = st.P / (RU * st.T);
      for (int k = 0; k < ns; k++) A.at(aC, k) = st.Ctot / ns;
    }
    const double T = st.T, V = st.V, P = st.P, invT = st.invT, lnT = st.lnT, Ctot = st.Ctot;
    const double invT2 = invT * invT, invV = 1.0 / V;
    const double uT = ok ? u_T[s] : 0.0;
    double* __restrict__ grow = g_phi + 2 * ld + s;  // d/dn_j accumulates at grow[j*ld]
    double* __restrict__ wrow = y + s;               // wdot_k accumulates at wrow[k*ld]
    if (ok)
      for (int k = 0; k < ns - 1; k++) {
        grow[(int64_t)k * ld] = 0.0;
        wrow[(int64_t)k * ld] = 0.0;
      }
    double den = 0.0, dden_T = 0.0, Cx_bath = 0.0;
    for (int k = 0; k < ns; k++) {
      const double* cb = nasa_block(m, k, T);
      double cp, h, sr, cp2, dcp;
      nasa_eval(cb, T, invT, lnT, cp, h, sr);
      nasa_cp(cb, T, cp2, dcp);
      A.at(aG, k) = h - sr;
      A.at(aH, k) = h;
      A.at(aU, k) = ok ? u_wdot[(int64_t)k * ld + s] : 0.0;
      const double Ck = A.at(aC, k);
      const double cx = MODE == PJ_CONP ? cp : cp - 1.0;
      den = fma(Ck, cx, den);
      dden_T = fma(Ck, dcp, dden_T);
      if (k == bath) Cx_bath = RU * cx;
    }
    den *= RU;
    const double iden = 1.0 / den;
    const double C_bath = A.at(aC, bath);
    const double dCb_T = -Ctot * invT;
    const double dCb_S = MODE == PJ_CONP ? (Ctot - C_bath) * invV : Ctot / P;
    dden_T = RU * dden_T + Cx_bath * dCb_T;
    const double dden_S = MODE == PJ_CONP ? (Cx_bath * Ctot - den) * invV : Cx_bath * Ctot / P;
    const double logPRT = m.log_pstd_over_r - lnT;
    const double mR_calT = -1.0 / (R_CAL * T);

    double gT = 0.0, gS = 0.0, gB = 0.0, w_bath = 0.0;
    // Plain reactions (the first m.nr_plain in kernel order) run through a
    // body compiled without the special cases (chemically activated, explicit
    // reverse, P-log, Chebyshev), the rest through the general one.
    auto reaction = [&](int i, auto gen_tag) {
      constexpr bool GEN = decltype(gen_tag)::value;
      const Rxn* __restrict__ r = m.rxn + i;
      const int kind = __ldg(&r->kind);
      const int nre = __ldg(&r->nreac), npr = __ldg(&r->nprod), rev = __ldg(&r->rev);
      double lnkinf, dlnkf, dlnP, dlnkinf;
      const double lnkf = ln_kf<true, GEN>(m, r, kind, lnT, invT, st.lnP, lnkinf, dlnkf, dlnP, dlnkinf);
      double kf, kr;
      rate_constants<GEN>(m, A, aG, r, rev, nre, npr, lnkf, logPRT, lnT, invT, kf, kr);
      double dh = 0.0, du = 0.0;
#pragma unroll
      for (int a = 0; a < PJ_MAX_SP; a++) {
        if (a < nre) {
          const int k = __ldg(&r->sp[a]);
          const double v = __ldg(&r->nud[a]);
          dh = fma(-v, A.at(aH, k), dh);
          du = fma(-v, A.at(aU, k), du);
        }
        if (a < npr) {
          const int k = __ldg(&r->sp[PJ_MAX_SP + a]);
          const double v = __ldg(&r->nud[PJ_MAX_SP + a]);
          dh = fma(v, A.at(aH, k), dh);
          du = fma(v, A.at(aU, k), du);
        }
      }
      double dRf[PJ_MAX_SP], dRr[PJ_MAX_SP];
      const double Rf = side_rate<true>(A, aC, r, 0, __ldg(&r->shape[0]), nre, kf, dRf);
      double Rr = 0.0, dlnkr = 0.0;
      if (rev) {
        Rr = side_rate<true>(A, aC, r, PJ_MAX_SP, __ldg(&r->shape[1]), npr, kr, dRr);
        if (GEN && rev == 2)
          dlnkr = fma(__ldg(m.tab + __ldg(&r->tab_lo) + 2), invT2, __ldg(m.tab + __ldg(&r->tab_lo) + 1) * invT);
        else
          dlnkr = dlnkf - (dh - __ldg(&r->dnu)) * invT;
      }
      const double Rn = Rf - Rr;
      double c = 1.0, dcdT = 0.0, dcdS = 0.0, dcdM = 0.0;
      // d q / d ln k_inf (k_inf: the Arrhenius set the parameter gradient is
      // taken for) = part through the base rate + part through Pr
      double Qpr = 0.0;
      if (has_third_body(kind)) {
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
          const double rk = pj_exp(lnk0 - lnkinf);
          const double Pr = rk * M;
          double FxPr, FT;
          const double F = falloff_F<true>(r, kind, T, invT, lnT, Pr, FxPr, FT);
          const double i1p = 1.0 / (1.0 + Pr);
          const double dPrdT = Pr * (dlnk0 - dlnkinf) + rk * dMdT;
          double cPr;
          if (GEN && __ldg(&r->chem)) {
            c = F * i1p;
            cPr = i1p * (FxPr / Pr - F * i1p);
            dcdT = i1p * FT + cPr * dPrdT;
          } else {
            const double fr = Pr * i1p;
            c = fr * F;
            cPr = F * i1p * i1p + FxPr * i1p;
            dcdT = fr * FT + cPr * dPrdT;
          }
          dcdM = cPr * rk;
          dcdS = dcdM * dMdS;
          Qpr = -Rn * cPr * Pr;  // k_inf divides Pr
        }
      }
      const double q = c * Rn;
      // the base rate is k_inf unless the reaction is chemically activated or
      // pressure-dependent; with an explicit reverse rate only R' scales
      const bool base_inf = !GEN || (kind < PJ_PLOG && !__ldg(&r->chem));
      const double Q = (base_inf ? c * ((GEN && rev == 2) ? Rf : Rn) : 0.0) + Qpr;
      if (ok) scatter_wdot(r, nre, npr, bath, q, wrow, ld, w_bath);
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
      if (GEN && MODE == PJ_CONV && kind >= PJ_PLOG) {
        // P-log / Chebyshev rates depend on P = S; an explicit reverse rate does not
        const double dP = dlnP / P;
        dRdS = fma(Rf, dP, dRdS) - (rev == 1 ? Rr * dP : 0.0);
      }
      const double dqdT = fma(c, dRdT, Rn * dcdT);
      const double dqdS = fma(c, dRdS, Rn * dcdS);

      // adjoint of q_i and its contributions to g_Phi
      const double dE = RU * T * (MODE == PJ_CONP ? dh : dh - __ldg(&r->dnu));
      const double ub = ok ? du - uT * dE * iden : 0.0;
      gT = fma(ub, dqdT, gT);
      gS = fma(ub, dqdS, gS);
      const double ubV = ub * invV;
      double Bi = 0.0;
#pragma unroll
      for (int a = 0; a < PJ_MAX_SP; a++) {
        if (a < nre) {
          const int j = __ldg(&r->sp[a]);
          const double val = c * dRf[a];
          if (j == bath) Bi -= val;
          else if (ok) red_add(grow + (int64_t)j * ld, ubV * val);
        }
        if (rev && a < npr) {
          const int j = __ldg(&r->sp[PJ_MAX_SP + a]);
          const double val = -c * dRr[a];
          if (j == bath) Bi -= val;
          else if (ok) red_add(grow + (int64_t)j * ld, ubV * val);
        }
      }
      if (has_third_body(kind)) {
        const double t = Rn * dcdM;
        for (int e = __ldg(&r->eff_lo), eh = __ldg(&r->eff_hi); e < eh; e++) {
          const int j = __ldg(m.eff_sp + e);
          const double val = t * __ldg(m.eff_am1 + e);
          if (j == bath) Bi -= val;
          else if (ok) red_add(grow + (int64_t)j * ld, ubV * val);
        }
      }
      gB = fma(ubV, Bi, gB);

      // parameter gradients summed over the warp, then by lane 0 into the
      // warp's own partial slot (program order: deterministic)
      const double wq = ub * Q;
      const double s0 = warp_sum(wq);
      const double s1 = warp_sum(wq * lnT);
      const double s2 = warp_sum(wq * mR_calT);
      if (PJ_LANE0(lane)) {
        red_add(my_part + 3 * i + 0, s0);
        red_add(my_part + 3 * i + 1, s1);
        red_add(my_part + 3 * i + 2, s2);
      }
    };
    for (int i = 0; i < m.nr_plain; i++) reaction(i, BoolTag<false>{});
    if (SPECIAL)
      for (int i = m.nr_plain; i < nr; i++) reaction(i, BoolTag<true>{});

    if (!ok) continue;

    // y, and the direct dependence of dT/dt on the state through E_k(T), D
    double num = 0.0, sumCxW = 0.0;
    for (int k = 0; k < ns; k++) {
      double cp, dcp;
      nasa_cp(nasa_block(m, k, T), T, cp, dcp);
      const double cx = RU * (MODE == PJ_CONP ? cp : cp - 1.0);
      A.at(aG, k) = cx;
      const double wk = k < bath ? __ldcg(wrow + (int64_t)k * ld) : w_bath;
      num = fma(MODE == PJ_CONP ? A.at(aH, k) : A.at(aH, k) - 1.0, wk, num);
      sumCxW = fma(cx, wk, sumCxW);
    }
    const double Tdot = -(num * RU * T) * iden;
    wrow[(int64_t)bath * ld] = w_bath;
    y[(int64_t)ns * ld + s] = Tdot;
    gT += uT * (-(sumCxW + Tdot * dden_T) * iden);
    gS += uT * (-(Tdot * dden_S) * iden);
    g_phi[s] = gT;
    g_phi[ld + s] = gS;
    const double Cxb = A.at(aG, bath);
    const double tv = uT * Tdot * invV * iden;
    for (int j = 0; j < ns - 1; j++) {
      const double acc = __ldcg(grow + (int64_t)j * ld);
      grow[(int64_t)j * ld] = acc + gB - tv * (A.at(aG, j) - Cxb);
    }
  }
}

// g_theta[perm[i]][p] = sum over warps of the partial sums, in warp order.
__global__ void k_vjp_reduce(int nr, int64_t n_warps, const double* __restrict__ part,
                             const int32_t* __restrict__ perm, double* __restrict__ g_theta) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)nr * 3) return;
  const int i = (int)(t / 3), p = (int)(t % 3);
  double acc = 0.0;
  for (int64_t w = 0; w < n_warps; w++) acc += part[w * (int64_t)nr * 3 + t];
  g_theta[(int64_t)perm[i] * 3 + p] = acc;
}

#ifndef PJ_NO_LAUNCHERS
}  // namespace pj
#include "launch.h"
namespace pj {
// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
struct FormPlan {
  int tpb, grid;
  size_t smem;
  bool global_ws;
  int64_t ws_stride;
  size_t ws_bytes;      // per-state arrays (global mode)
  size_t part_bytes;    // VJP per-warp partials
};


// The VJP kernel is compiled for four resident blocks of 128 threads; its
// arrays stay in shared memory only where that keeps those four blocks,
// else they go to an L1-cached global workspace (at 53 species: 16 warps per
// SM instead of 4, measured 1.4x faster).
static FormPlan form_plan(int arrays, const DevMech& m, int64_t n, bool vjp) {
  FormPlan p{};
  const size_t per_thread = (size_t)arrays * m.ns * sizeof(double);
  const size_t smem_cap = 225 * 1024;
  const int fit = (int)((smem_cap / per_thread) / 32 * 32);
  const int64_t cap_blocks = (int64_t)sm_count() * (vjp ? kVjpCtas : 8);
  if (fit >= (vjp ? kVjpCtas * 128 : 128)) {
    p.global_ws = false;
    p.tpb = fit >= 256 ? 128 : (fit % 64 == 0 ? 64 : 32);
    p.smem = per_thread * p.tpb;
  } else {
    p.global_ws = true;
    p.tpb = 128;
    p.smem = 0;
  }
  int64_t blocks = (n + p.tpb - 1) / p.tpb;
  if (blocks < 1) blocks = 1;
  // grid-stride: bounded grid (the VJP partials scale with the warp count)
  if (blocks > cap_blocks) blocks = cap_blocks;
  p.grid = (int)blocks;
  p.ws_stride = (int64_t)p.grid * p.tpb;
  p.ws_bytes = p.global_ws ? per_thread * (size_t)p.ws_stride : 0;
  p.part_bytes = vjp ? (size_t)(p.ws_stride / 32) * m.nr * 3 * sizeof(double) : 0;
  return p;
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

size_t form_workspace_bytes(int op, const DevMech& m, int64_t n) {
  if (op == PJ_OP_VJP) {
    FormPlan p = form_plan(4, m, n, true);
    return align256(p.ws_bytes) + p.part_bytes;
  }
  FormPlan p = form_plan(2, m, n, false);
  return p.ws_bytes;
}


int launch_eval_y(const DevMech& m, int mode, int64_t n, const double* param, const double* phi, int64_t ld,
                  double* y, int* status, void* work, size_t work_bytes, cudaStream_t st) {
  FormPlan p = form_plan(2, m, n, false);
  if (p.global_ws && (!work || work_bytes < p.ws_bytes))
    return fail(PJ_ERR_NOMEM, "workspace too small for pj_eval_y (see pj_workspace_size)");
  double* ws = p.global_ws ? static_cast<double*>(work) : nullptr;
  const bool special = m.nr_plain < m.nr;
  auto kern = mode == PJ_CONP ? (special ? k_eval_y<PJ_CONP, true> : k_eval_y<PJ_CONP, false>)
                              : (special ? k_eval_y<PJ_CONV, true> : k_eval_y<PJ_CONV, false>);
  int rc;
  if ((rc = set_smem(kern, p.smem))) return rc;
  kern<<<p.grid, p.tpb, p.smem, st>>>(m, n, param, phi, ld, y, status, ws, p.ws_stride);
  return check_cuda(cudaGetLastError(), "k_eval_y launch");
}

int launch_vjp(const DevMech& m, int mode, int64_t n, const double* param, const double* phi, int64_t ld,
               const double* u_wdot, const double* u_T, double* y, double* g_phi, double* g_theta, int* status,
               void* work, size_t work_bytes, cudaStream_t st) {
  FormPlan p = form_plan(4, m, n, true);
  const size_t need = align256(p.ws_bytes) + p.part_bytes;
  if (!work || work_bytes < need)
    return fail(PJ_ERR_NOMEM, "workspace too small for pj_vjp (see pj_workspace_size)");
  double* ws = p.global_ws ? static_cast<double*>(work) : nullptr;
  double* part = reinterpret_cast<double*>(static_cast<char*>(work) + align256(p.ws_bytes));
  cudaError_t e = cudaMemsetAsync(part, 0, p.part_bytes, st);
  if (e != cudaSuccess) return check_cuda(e, "cudaMemsetAsync(vjp partials)");
  const bool special = m.nr_plain < m.nr;
  auto kern = mode == PJ_CONP ? (special ? k_vjp<PJ_CONP, true> : k_vjp<PJ_CONP, false>)
                              : (special ? k_vjp<PJ_CONV, true> : k_vjp<PJ_CONV, false>);
  int rc;
  if ((rc = set_smem(kern, p.smem))) return rc;
  kern<<<p.grid, p.tpb, p.smem, st>>>(m, n, param, phi, ld, u_wdot, u_T, y, g_phi, part, status, ws, p.ws_stride);
  if ((rc = check_cuda(cudaGetLastError(), "k_vjp launch"))) return rc;
  const int64_t nt = (int64_t)m.nr * 3;
  if (nt > 0) {
    k_vjp_reduce<<<(unsigned)((nt + 127) / 128), 128, 0, st>>>(m.nr, p.ws_stride / 32, part, m.perm, g_theta);
    if ((rc = check_cuda(cudaGetLastError(), "k_vjp_reduce launch"))) return rc;
  }
  return PJ_OK;
}

#endif  // PJ_NO_LAUNCHERS

}  // namespace pj
