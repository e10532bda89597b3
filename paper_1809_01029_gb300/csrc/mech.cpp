// Host side of libpyjac_gb: mechanism validation, packing of the kernel
// constants, the fixed sparsity pattern of the exact Jacobian (Sec. 3.4) and
// the static full-index -> sparse-index maps the paper proposes in place of a
// per-entry search of the compressed row (Sec. 3.4, last paragraph).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <sstream>
#include <string>

#include "pj_internal.h"

namespace pj {

static thread_local std::string g_last_error;

int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

int check_cuda(int err, const char* what) {
  if (err == cudaSuccess) return PJ_OK;
  return fail(err == cudaErrorMemoryAllocation ? PJ_ERR_NOMEM : PJ_ERR_CUDA,
              std::string(what) + ": " + cudaGetErrorString((cudaError_t)err));
}

// Net stoichiometric coefficient of every species in reaction i.
static std::vector<int> net_nu(const pj_mech* m, int i) {
  std::vector<int> nu(m->ns, 0);
  for (int a = 0; a < PJ_MAX_SP; a++) {
    int k = m->reac_sp[i * PJ_MAX_SP + a];
    if (k >= 0) nu[k] -= m->reac_nu[i * PJ_MAX_SP + a];
    k = m->prod_sp[i * PJ_MAX_SP + a];
    if (k >= 0) nu[k] += m->prod_nu[i * PJ_MAX_SP + a];
  }
  return nu;
}

static inline bool is_falloff(int k) { return k == PJ_LINDEMANN || k == PJ_TROE || k == PJ_SRI; }
static inline bool has_third_body(int k) { return k == PJ_THIRD_BODY || is_falloff(k); }

static std::vector<double> alpha_of(const pj_mech* m, int i) {
  std::vector<double> a(m->ns, 1.0);
  for (int e = m->eff_ptr[i]; e < m->eff_ptr[i + 1]; e++) a[m->eff_sp[e]] = m->eff_val[e];
  return a;
}

// Species (< Ns-1) on which reaction i's rate depends, and whether that is
// every species (bath gas in the rate, or a non-unit bath-gas efficiency).
// The approximate form (Sec. 3.4) leaves out exactly those every-species
// derivatives: efficiencies then count against the default 1, and the result
// is never dense, so the kernels skip the bath-gas term of the reaction.
static bool rate_dependence(const pj_mech* m, int i, std::vector<char>& dep) {
  const bool approx = m->jac_form == PJ_JAC_APPROX;
  const int ns = m->ns, bath = ns - 1;
  dep.assign(ns - 1, 0);
  bool dense = false;
  auto member = [&](int k) {
    if (k == bath) dense = true;
    else if (k >= 0) dep[k] = 1;
  };
  for (int a = 0; a < PJ_MAX_SP; a++) member(m->reac_sp[i * PJ_MAX_SP + a]);
  if (m->rev[i])
    for (int a = 0; a < PJ_MAX_SP; a++) member(m->prod_sp[i * PJ_MAX_SP + a]);
  if (has_third_body(m->kind[i])) {
    std::vector<double> al = alpha_of(m, i);
    const double ref = approx ? 1.0 : al[bath];
    for (int k = 0; k < ns - 1; k++)
      if (al[k] != ref) dep[k] = 1;
    if (al[bath] != 1.0) dense = true;
  }
  if (approx) return false;
  if (dense) std::fill(dep.begin(), dep.end(), 1);
  return dense;
}

static int validate(const pj_mech* m) {
  const int ns = m->ns, nr = m->nr;
  if (ns < 2) return fail(PJ_ERR_MECH, "need at least 2 species");
  if (nr < 0) return fail(PJ_ERR_MECH, "negative reaction count");
  for (int k = 0; k < ns; k++) {
    if (!(m->W[k] > 0) || !std::isfinite(m->W[k])) return fail(PJ_ERR_MECH, "species " + std::to_string(k) + ": W must be > 0");
    if (!std::isfinite(m->T_mid[k])) return fail(PJ_ERR_MECH, "species " + std::to_string(k) + ": bad T_mid");
    for (int j = 0; j < 7; j++)
      if (!std::isfinite(m->nasa_low[k * 7 + j]) || !std::isfinite(m->nasa_high[k * 7 + j]))
        return fail(PJ_ERR_MECH, "species " + std::to_string(k) + ": non-finite NASA coefficient");
  }
  if (m->eff_ptr.size() != (size_t)nr + 1 || m->eff_ptr[0] != 0)
    return fail(PJ_ERR_MECH, "eff_ptr must have Nr+1 entries starting at 0");
  for (int i = 0; i < nr; i++) {
    std::string tag = "reaction " + std::to_string(i) + ": ";
    if (m->kind[i] < PJ_ELEMENTARY || m->kind[i] > PJ_CHEB) return fail(PJ_ERR_MECH, tag + "bad kind");
    int nre = 0, npr = 0;
    for (int a = 0; a < PJ_MAX_SP; a++) {
      for (int side = 0; side < 2; side++) {
        int k = side ? m->prod_sp[i * PJ_MAX_SP + a] : m->reac_sp[i * PJ_MAX_SP + a];
        int v = side ? m->prod_nu[i * PJ_MAX_SP + a] : m->reac_nu[i * PJ_MAX_SP + a];
        if (k < -1 || k >= ns) return fail(PJ_ERR_MECH, tag + "species index out of range");
        if (k >= 0) {
          if (v < 1 || v > 8) return fail(PJ_ERR_MECH, tag + "stoichiometric coefficient must be 1..8");
          (side ? npr : nre)++;
        }
      }
    }
    if (nre == 0 || npr == 0) return fail(PJ_ERR_MECH, tag + "needs at least one reactant and one product");
    const bool pdep = m->kind[i] == PJ_PLOG || m->kind[i] == PJ_CHEB;
    if (!pdep && (!(m->A[i] > 0) || !std::isfinite(m->A[i]))) return fail(PJ_ERR_MECH, tag + "A must be > 0");
    if (m->chem[i] && m->kind[i] < PJ_LINDEMANN) return fail(PJ_ERR_MECH, tag + "only falloff reactions can be chemically activated");
    if (m->chem[i] && m->kind[i] > PJ_SRI) return fail(PJ_ERR_MECH, tag + "only falloff reactions can be chemically activated");
    if (m->rev_explicit[i]) {
      if (!m->rev[i]) return fail(PJ_ERR_MECH, tag + "explicit reverse parameters on an irreversible reaction");
      if (!(m->rev_A[i] > 0) || !std::isfinite(m->rev_A[i]) || !std::isfinite(m->rev_beta[i]) || !std::isfinite(m->rev_Ea[i]))
        return fail(PJ_ERR_MECH, tag + "bad explicit reverse parameters");
    }
    if (m->plog_ptr[i + 1] < m->plog_ptr[i]) return fail(PJ_ERR_MECH, tag + "plog_ptr not monotone");
    const int np = m->plog_ptr[i + 1] - m->plog_ptr[i];
    if ((m->kind[i] == PJ_PLOG) != (np > 0)) return fail(PJ_ERR_MECH, tag + "P-log entries exactly for P-log reactions");
    for (int e = m->plog_ptr[i]; e < m->plog_ptr[i + 1]; e++) {
      const double* t = &m->plog[(size_t)e * 4];
      if (!(t[0] > 0) || !(t[1] > 0) || !std::isfinite(t[0]) || !std::isfinite(t[1]) || !std::isfinite(t[2]) ||
          !std::isfinite(t[3]))
        return fail(PJ_ERR_MECH, tag + "bad P-log entry");
      if (e > m->plog_ptr[i] && !(t[0] > t[-4])) return fail(PJ_ERR_MECH, tag + "P-log pressures must ascend strictly");
    }
    if (m->cheb_ptr[i + 1] < m->cheb_ptr[i]) return fail(PJ_ERR_MECH, tag + "cheb_ptr not monotone");
    const int ncf = m->cheb_ptr[i + 1] - m->cheb_ptr[i];
    if (m->kind[i] == PJ_CHEB) {
      const int nT = m->cheb_nT[i], nP = m->cheb_nP[i];
      const double* rg = &m->cheb_range[(size_t)i * 4];
      if (nT < 1 || nT > 16 || nP < 1 || nP > 16 || ncf != nT * nP) return fail(PJ_ERR_MECH, tag + "bad Chebyshev shape");
      if (!(rg[0] > 0) || !(rg[1] > rg[0]) || !(rg[2] > 0) || !(rg[3] > rg[2]) || !std::isfinite(rg[1]) ||
          !std::isfinite(rg[3]))
        return fail(PJ_ERR_MECH, tag + "bad Chebyshev range");
      for (int e = m->cheb_ptr[i]; e < m->cheb_ptr[i + 1]; e++)
        if (!std::isfinite(m->cheb_coef[e])) return fail(PJ_ERR_MECH, tag + "non-finite Chebyshev coefficient");
    } else if (ncf != 0) {
      return fail(PJ_ERR_MECH, tag + "Chebyshev coefficients on a non-Chebyshev reaction");
    }
    if (!pdep && (!std::isfinite(m->beta[i]) || !std::isfinite(m->Ea[i]))) return fail(PJ_ERR_MECH, tag + "bad beta/Ea");
    if (is_falloff(m->kind[i])) {
      if (!(m->A0[i] > 0) || !std::isfinite(m->A0[i])) return fail(PJ_ERR_MECH, tag + "A0 must be > 0");
      if (!std::isfinite(m->beta0[i]) || !std::isfinite(m->Ea0[i])) return fail(PJ_ERR_MECH, tag + "bad beta0/Ea0");
    }
    if (m->kind[i] == PJ_TROE) {
      int tn = m->troe_n[i];
      const double* t = &m->troe[i * 4];
      if (tn != 3 && tn != 4) return fail(PJ_ERR_MECH, tag + "Troe needs 3 or 4 parameters");
      if (t[1] == 0 || t[2] == 0 || !std::isfinite(t[0])) return fail(PJ_ERR_MECH, tag + "Troe T3/T1 must be nonzero");
    }
    if (m->kind[i] == PJ_SRI) {
      const double* s = &m->sri[i * 5];
      if (s[2] == 0 || !(s[3] > 0)) return fail(PJ_ERR_MECH, tag + "SRI needs c != 0 and d > 0");
    }
    if (m->eff_ptr[i + 1] < m->eff_ptr[i]) return fail(PJ_ERR_MECH, tag + "eff_ptr not monotone");
    for (int e = m->eff_ptr[i]; e < m->eff_ptr[i + 1]; e++) {
      if (m->eff_sp[e] < 0 || m->eff_sp[e] >= ns) return fail(PJ_ERR_MECH, tag + "efficiency species out of range");
      if (!std::isfinite(m->eff_val[e]) || m->eff_val[e] < 0) return fail(PJ_ERR_MECH, tag + "bad efficiency");
    }
  }
  return PJ_OK;
}

static void build_pattern(pj_mech* m) {
  const int ns = m->ns, N = ns + 1;
  std::vector<char> mask((size_t)N * N, 0);
  for (int j = 0; j < N; j++) {
    mask[0 * N + j] = mask[1 * N + j] = 1;
    mask[(size_t)j * N + 0] = mask[(size_t)j * N + 1] = 1;
    mask[(size_t)j * N + j] = 1;
  }
  std::vector<char> dep;
  for (int i = 0; i < m->nr; i++) {
    rate_dependence(m, i, dep);
    std::vector<int> nu = net_nu(m, i);
    for (int k = 0; k < ns - 1; k++) {
      if (nu[k] == 0) continue;
      for (int j = 0; j < ns - 1; j++)
        if (dep[j]) mask[(size_t)(k + 2) * N + (j + 2)] = 1;
    }
  }
  m->csr_ptr.assign(N + 1, 0);
  m->csr_idx.clear();
  m->pos_csr.assign((size_t)N * N, -1);
  for (int i = 0; i < N; i++) {
    for (int j = 0; j < N; j++)
      if (mask[(size_t)i * N + j]) {
        m->pos_csr[(size_t)i * N + j] = (int32_t)m->csr_idx.size();
        m->csr_idx.push_back(j);
      }
    m->csr_ptr[i + 1] = (int32_t)m->csr_idx.size();
  }
  m->csc_ptr.assign(N + 1, 0);
  m->csc_idx.clear();
  m->pos_csc.assign((size_t)N * N, -1);
  for (int j = 0; j < N; j++) {
    for (int i = 0; i < N; i++)
      if (mask[(size_t)i * N + j]) {
        m->pos_csc[(size_t)i * N + j] = (int32_t)m->csc_idx.size();
        m->csc_idx.push_back(i);
      }
    m->csc_ptr[j + 1] = (int32_t)m->csc_idx.size();
  }
  m->nnz = (int32_t)m->csr_idx.size();
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

int mech_build(pj_mech* m) {
  int rc = validate(m);
  if (rc) return rc;
  build_pattern(m);
  const int ns = m->ns, nr = m->nr, N = ns + 1, bath = ns - 1;

  // kernel order: the plain reactions first, then the special ones
  // (chemically activated, explicit reverse, P-log, Chebyshev), each part
  // stable-sorted by kind so that each kind's code runs as a block; the
  // kernels walk the plain part with a loop compiled without the special
  // cases
  auto special = [&](int i) { return m->chem[i] || m->rev_explicit[i] || m->kind[i] >= PJ_PLOG; };
  m->perm.resize(nr);
  for (int i = 0; i < nr; i++) m->perm[i] = i;
  std::stable_sort(m->perm.begin(), m->perm.end(), [&](int a, int b) {
    const int sa = special(a) ? 1 : 0, sb = special(b) ? 1 : 0;
    return sa != sb ? sa < sb : m->kind[a] < m->kind[b];
  });
  int nr_plain = 0;
  while (nr_plain < nr && !special(m->perm[nr_plain])) nr_plain++;

  // Within each group of equal kind, order reactions so that those writing
  // the same Jacobian entries run close together: the resident warps'
  // Jacobians far exceed L2, so an entry's reductions hit L2 only while its
  // line is recent.  Greedy: the next reaction is the one among the group's
  // next kLook candidates sharing the most entries with the last kRecent
  // reactions (ties: the earlier one).
  {
    constexpr int kLook = 256, kRecent = 6;
    auto entries = [&](int i) {
      std::vector<int> nu = net_nu(m, i);
      std::vector<int> rows, cols;
      for (int k = 0; k < bath; k++)
        if (nu[k] != 0) rows.push_back(k);
      for (int a = 0; a < PJ_MAX_SP; a++) {
        const int kr = m->reac_sp[i * PJ_MAX_SP + a], kp = m->prod_sp[i * PJ_MAX_SP + a];
        if (kr >= 0 && kr != bath) cols.push_back(kr);
        if (m->rev[i] && kp >= 0 && kp != bath) cols.push_back(kp);
      }
      if (has_third_body(m->kind[i]))
        for (int e = m->eff_ptr[i]; e < m->eff_ptr[i + 1]; e++)
          if (m->eff_sp[e] != bath && m->eff_val[e] != 1.0) cols.push_back(m->eff_sp[e]);
      std::vector<int64_t> ent;
      for (int k : rows) {
        ent.push_back((int64_t)(k + 2) * N + 0);
        ent.push_back((int64_t)(k + 2) * N + 1);
        for (int j : cols) ent.push_back((int64_t)(k + 2) * N + j + 2);
      }
      for (int j : cols) {
        ent.push_back(j + 2);
        ent.push_back((int64_t)N + j + 2);
      }
      std::sort(ent.begin(), ent.end());
      ent.erase(std::unique(ent.begin(), ent.end()), ent.end());
      return ent;
    };
    std::vector<std::vector<int64_t>> ent(nr);
    for (int i = 0; i < nr; i++) ent[i] = entries(i);
    auto shared = [](const std::vector<int64_t>& a, const std::vector<int64_t>& b) {
      int c = 0;
      size_t x = 0, y = 0;
      while (x < a.size() && y < b.size()) {
        if (a[x] < b[y]) x++;
        else if (b[y] < a[x]) y++;
        else { c++; x++; y++; }
      }
      return c;
    };
    for (int g0 = 0; g0 < nr;) {
      int g1 = g0 + 1;
      while (g1 < nr && special(m->perm[g1]) == special(m->perm[g0]) && m->kind[m->perm[g1]] == m->kind[m->perm[g0]])
        g1++;
      std::vector<int> rest(m->perm.begin() + g0, m->perm.begin() + g1), out;
      while (!rest.empty()) {
        size_t best = 0;
        int best_score = -1;
        for (size_t c = 0; c < rest.size() && c < (size_t)kLook; c++) {
          int score = 0;
          for (size_t q = out.size() > (size_t)kRecent ? out.size() - kRecent : 0; q < out.size(); q++)
            score += shared(ent[rest[c]], ent[out[q]]);
          if (score > best_score) {
            best_score = score;
            best = c;
          }
        }
        out.push_back(rest[best]);
        rest.erase(rest.begin() + (ptrdiff_t)best);
      }
      std::copy(out.begin(), out.end(), m->perm.begin() + g0);
      g0 = g1;
    }
  }

  std::vector<double> nasa((size_t)ns * NASA_STRIDE, 0.0), wfac(ns);
  for (int k = 0; k < ns; k++) {
    for (int r = 0; r < 2; r++) {
      const double* a = r == 0 ? &m->nasa_low[k * 7] : &m->nasa_high[k * 7];
      double* b = &nasa[(size_t)k * NASA_STRIDE + r * 16];
      for (int j = 0; j < 7; j++) b[j] = a[j];
      b[7] = a[1] / 2; b[8] = a[2] / 3; b[9] = a[3] / 4; b[10] = a[4] / 5;
      b[11] = a[2] / 2; b[12] = a[3] / 3; b[13] = a[4] / 4;
      b[14] = m->T_mid[k];
    }
    wfac[k] = 1.0 - m->W[k] / m->W[bath];
  }

  std::vector<Rxn> rx(nr);
  std::vector<int32_t> eff_sp;
  std::vector<double> eff_am1;
  std::vector<RowNu> rows;
  std::vector<char> dep;
  std::vector<double> tab;  // P-log entries and Chebyshev blocks
  bool has_pdep = false;
  for (int q = 0; q < nr; q++) {
    const int i = m->perm[q];
    Rxn& r = rx[q];
    std::memset(&r, 0, sizeof(Rxn));
    r.kind = m->kind[i];
    r.rev = m->rev[i] ? (m->rev_explicit[i] ? 2 : 1) : 0;
    const bool pdep = r.kind == PJ_PLOG || r.kind == PJ_CHEB;
    r.lnA = pdep ? 0.0 : std::log(m->A[i]);
    r.beta = pdep ? 0.0 : m->beta[i];
    r.theta = pdep ? 0.0 : m->Ea[i] / R_CAL;
    r.chem = m->chem[i] ? 1 : 0;
    r.tab_lo = (int32_t)tab.size();
    if (r.rev == 2) {
      tab.push_back(std::log(m->rev_A[i]));
      tab.push_back(m->rev_beta[i]);
      tab.push_back(m->rev_Ea[i] / R_CAL);
    }
    if (r.kind == PJ_PLOG) {
      // (ln P, ln A, beta, theta) per entry
      for (int e = m->plog_ptr[i]; e < m->plog_ptr[i + 1]; e++) {
        const double* t = &m->plog[(size_t)e * 4];
        tab.push_back(std::log(t[0]));
        tab.push_back(std::log(t[1]));
        tab.push_back(t[2]);
        tab.push_back(t[3] / R_CAL);
      }
      r.tab_n = (int16_t)(m->plog_ptr[i + 1] - m->plog_ptr[i]);
      has_pdep = true;
    } else if (r.kind == PJ_CHEB) {
      // T~ = cT1 / T + cT0, P~ = cP1 ln P + cP0, then ln10 * a_tp (ln k directly)
      const double* rg = &m->cheb_range[(size_t)i * 4];
      const double iTmin = 1.0 / rg[0], iTmax = 1.0 / rg[1];
      const double lPmin = std::log(rg[2]), lPmax = std::log(rg[3]);
      tab.push_back(2.0 / (iTmax - iTmin));
      tab.push_back(-(iTmin + iTmax) / (iTmax - iTmin));
      tab.push_back(2.0 / (lPmax - lPmin));
      tab.push_back(-(lPmin + lPmax) / (lPmax - lPmin));
      for (int e = m->cheb_ptr[i]; e < m->cheb_ptr[i + 1]; e++) tab.push_back(LN10 * m->cheb_coef[e]);
      r.tab_n = (int16_t)m->cheb_nT[i];
      r.tab_m = (int16_t)m->cheb_nP[i];
      has_pdep = true;
    }
    if (is_falloff(r.kind)) {
      r.lnA0 = std::log(m->A0[i]);
      r.beta0 = m->beta0[i];
      r.theta0 = m->Ea0[i] / R_CAL;
    }
    if (r.kind == PJ_TROE) {
      const double* t = &m->troe[i * 4];
      r.fp[0] = t[0]; r.fp[1] = 1.0 / t[1]; r.fp[2] = 1.0 / t[2];
      r.fp[3] = m->troe_n[i] == 4 ? t[3] : 0.0;
      r.fp[4] = m->troe_n[i] == 4 ? 1.0 : 0.0;
    } else if (r.kind == PJ_SRI) {
      const double* s = &m->sri[i * 5];
      r.fp[0] = s[0]; r.fp[1] = s[1]; r.fp[2] = 1.0 / s[2]; r.fp[3] = s[3]; r.fp[4] = s[4];
    }
    for (int a = 0; a < 2 * PJ_MAX_SP; a++) r.sp[a] = -1;
    for (int side = 0; side < 2; side++) {
      const int32_t* ssp = side ? &m->prod_sp[i * PJ_MAX_SP] : &m->reac_sp[i * PJ_MAX_SP];
      const int32_t* snu = side ? &m->prod_nu[i * PJ_MAX_SP] : &m->reac_nu[i * PJ_MAX_SP];
      std::vector<std::pair<int, int>> mem;  // (nu, species)
      for (int a = 0; a < PJ_MAX_SP; a++)
        if (ssp[a] >= 0) mem.push_back({snu[a], ssp[a]});
      // larger coefficients first, so 2A + B maps onto SH_21
      std::stable_sort(mem.begin(), mem.end(), [](auto x, auto y) { return x.first > y.first; });
      int32_t shape = SH_GEN;
      if (mem.size() == 1 && mem[0].first == 1) shape = SH_1;
      else if (mem.size() == 1 && mem[0].first == 2) shape = SH_2;
      else if (mem.size() == 2 && mem[0].first == 1 && mem[1].first == 1) shape = SH_11;
      else if (mem.size() == 2 && mem[0].first == 2 && mem[1].first == 1) shape = SH_21;
      else if (mem.size() == 3 && mem[0].first == 1 && mem[1].first == 1 && mem[2].first == 1) shape = SH_111;
      r.shape[side] = shape;
      for (size_t a = 0; a < mem.size(); a++) {
        r.sp[side * PJ_MAX_SP + a] = mem[a].second;
        r.nu[side * PJ_MAX_SP + a] = mem[a].first;
        r.nud[side * PJ_MAX_SP + a] = (double)mem[a].first;
      }
      (side ? r.nprod : r.nreac) = (int32_t)mem.size();
    }
    std::vector<int> nu = net_nu(m, i);
    double dnu = 0, dW = 0;
    for (int k = 0; k < ns; k++) {
      dnu += nu[k];
      if (k < bath) dW += nu[k] * wfac[k];
    }
    r.dnu = dnu;
    r.dW = dW;
    std::vector<double> al = alpha_of(m, i);
    r.alpha_bath = has_third_body(r.kind) ? al[bath] : 1.0;
    r.eff_lo = (int32_t)eff_sp.size();
    if (has_third_body(r.kind)) {
      for (int e = m->eff_ptr[i]; e < m->eff_ptr[i + 1]; e++) {
        if (m->eff_val[e] == 1.0) continue;  // default efficiency: no term
        eff_sp.push_back(m->eff_sp[e]);
        eff_am1.push_back(m->eff_val[e] - 1.0);
      }
    }
    r.eff_hi = (int32_t)eff_sp.size();
    // a row per unit of |nu|: every Jacobian contribution is then +-1 times
    // its value, a sign flip the kernels do without an FP64 instruction
    // (|nu| >= 2 is rare: 14 of 1262 rows at 53 species)
    r.row_lo = (int32_t)rows.size();
    for (int k = 0; k < bath; k++)
      for (int u = 0; u < std::abs(nu[k]); u++) rows.push_back(RowNu{k, nu[k] > 0 ? 1 : -1, nu[k] > 0 ? 1.0 : -1.0});
    r.row_hi = (int32_t)rows.size();
    r.dense = rate_dependence(m, i, dep) ? 1 : 0;
    r.bath_in = 0;
    for (int a = 0; a < 2 * PJ_MAX_SP; a++) r.bath_in |= r.sp[a] == bath && (a % PJ_MAX_SP) < (a < PJ_MAX_SP ? r.nreac : r.nprod);
  }

  // Every entry the Jacobian kernels accumulate into must be in the pattern
  // (the index maps hold -1 elsewhere): for each row a reaction changes, the
  // T and S columns, the columns of its reactants, reversible products and
  // non-unit efficiencies, and every species column when it is dense; rows T
  // and S and the diagonal in full.
  {
    auto in = [&](int i, int j) {
      return m->pos_csr[(size_t)i * N + j] >= 0 && m->pos_csc[(size_t)i * N + j] >= 0;
    };
    bool ok = true;
    for (int j = 0; j < N; j++) ok = ok && in(0, j) && in(1, j) && in(j, j);
    std::vector<int> cols;
    for (int q = 0; q < nr && ok; q++) {
      const Rxn& r = rx[q];
      cols.clear();
      for (int a = 0; a < r.nreac; a++) cols.push_back(r.sp[a]);
      if (r.rev)
        for (int a = 0; a < r.nprod; a++) cols.push_back(r.sp[PJ_MAX_SP + a]);
      for (int e = r.eff_lo; e < r.eff_hi; e++) cols.push_back(eff_sp[e]);
      if (r.dense)
        for (int j = 0; j < bath; j++) cols.push_back(j);
      for (int q2 = r.row_lo; q2 < r.row_hi && ok; q2++) {
        const int k = rows[q2].k;
        ok = ok && in(k + 2, 0) && in(k + 2, 1);
        for (int j : cols)
          if (j != bath) ok = ok && in(k + 2, j + 2);
      }
    }
    if (!ok) return fail(PJ_ERR_MECH, "internal: the sparsity pattern misses an entry the Jacobian kernel writes");
  }

  // The sparse targets of each reaction's Jacobian contributions, in the
  // order jacobian_state makes them: per row it changes the T and S columns;
  // then per slot (reactant a, reversible product a, a = 0, 1, ..., then the
  // non-unit efficiencies), skipping the bath gas, its column in each row and
  // in rows T and S.  Read sequentially by the kernels instead of looking up
  // the N x N index map per contribution.
  std::vector<int32_t> tgt_csr, tgt_csc;
  for (int q = 0; q < nr; q++) {
    Rxn& r = rx[q];
    r.tgt_lo = (int32_t)tgt_csr.size();
    auto push = [&](int i, int j) {
      tgt_csr.push_back(m->pos_csr[(size_t)i * N + j]);
      tgt_csc.push_back(m->pos_csc[(size_t)i * N + j]);
    };
    for (int q2 = r.row_lo; q2 < r.row_hi; q2++) {
      push(rows[q2].k + 2, 0);
      push(rows[q2].k + 2, 1);
    }
    auto slot = [&](int j) {
      if (j == bath) return;
      for (int q2 = r.row_lo; q2 < r.row_hi; q2++) push(rows[q2].k + 2, j + 2);
      push(0, j + 2);
      push(1, j + 2);
    };
    for (int a = 0; a < PJ_MAX_SP; a++) {
      if (a < r.nreac) slot(r.sp[a]);
      if (r.rev && a < r.nprod) slot(r.sp[PJ_MAX_SP + a]);
    }
    if (has_third_body(r.kind))
      for (int e = r.eff_lo; e < r.eff_hi; e++) slot(eff_sp[e]);
  }

  // one device allocation holding every constant array
  const size_t o_nasa = 0;
  const size_t o_wfac = align256(o_nasa + nasa.size() * sizeof(double));
  const size_t o_rxn = align256(o_wfac + wfac.size() * sizeof(double));
  const size_t o_esp = align256(o_rxn + rx.size() * sizeof(Rxn));
  const size_t o_eam = align256(o_esp + eff_sp.size() * sizeof(int32_t));
  const size_t o_rows = align256(o_eam + eff_am1.size() * sizeof(double));
  const size_t o_pcsr = align256(o_rows + rows.size() * sizeof(RowNu));
  const size_t o_pcsc = align256(o_pcsr + (size_t)N * N * sizeof(int32_t));
  const size_t o_perm = align256(o_pcsc + (size_t)N * N * sizeof(int32_t));
  const size_t o_etab = align256(o_perm + (size_t)nr * sizeof(int32_t));
  const size_t o_tab = align256(o_etab + 256 * sizeof(double));
  const size_t o_tcsr = align256(o_tab + tab.size() * sizeof(double));
  const size_t o_tcsc = align256(o_tcsr + tgt_csr.size() * sizeof(int32_t));
  const size_t o_dbg = align256(o_tcsc + tgt_csc.size() * sizeof(int32_t));
  const size_t total = align256(o_dbg + sizeof(uint32_t));
  // 2^(j/256) in extended precision, rounded once to double
  double etab[256];
  for (int j = 0; j < 256; j++) etab[j] = (double)std::exp2((long double)j / 256.0L);

  std::vector<char> blob(total, 0);
  auto put = [&](size_t off, const void* src, size_t bytes) { if (bytes) std::memcpy(blob.data() + off, src, bytes); };
  put(o_nasa, nasa.data(), nasa.size() * sizeof(double));
  put(o_wfac, wfac.data(), wfac.size() * sizeof(double));
  put(o_rxn, rx.data(), rx.size() * sizeof(Rxn));
  put(o_esp, eff_sp.data(), eff_sp.size() * sizeof(int32_t));
  put(o_eam, eff_am1.data(), eff_am1.size() * sizeof(double));
  put(o_rows, rows.data(), rows.size() * sizeof(RowNu));
  put(o_pcsr, m->pos_csr.data(), m->pos_csr.size() * sizeof(int32_t));
  put(o_pcsc, m->pos_csc.data(), m->pos_csc.size() * sizeof(int32_t));
  put(o_perm, m->perm.data(), m->perm.size() * sizeof(int32_t));
  put(o_etab, etab, sizeof etab);
  put(o_tab, tab.data(), tab.size() * sizeof(double));
  put(o_tcsr, tgt_csr.data(), tgt_csr.size() * sizeof(int32_t));
  put(o_tcsc, tgt_csc.data(), tgt_csc.size() * sizeof(int32_t));

  // Without any CUDA device the handle stays host-only: its pattern can be
  // queried, evaluation calls fail with PJ_ERR_CUDA.
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || count == 0) {
    cudaGetLastError();
    m->device = -1;
    return lu_build(m);
  }
  int dev = 0;
  if ((rc = check_cuda(cudaGetDevice(&dev), "cudaGetDevice"))) return rc;
  void* d = nullptr;
  if ((rc = check_cuda(cudaMalloc(&d, total), "cudaMalloc(mechanism constants)"))) return rc;
  if ((rc = check_cuda(cudaMemcpy(d, blob.data(), total, cudaMemcpyHostToDevice), "cudaMemcpy(mechanism constants)"))) {
    cudaFree(d);
    return rc;
  }
  m->device = dev;
  m->dev_blob = d;
  m->dev_bytes = total;
  char* b = static_cast<char*>(d);
  DevMech& dm = m->dm;
  dm.ns = ns;
  dm.nr = nr;
  dm.N = N;
  dm.nnz = m->nnz;
  dm.log_pstd_over_r = std::log(P_STD / RU);
  dm.nasa = reinterpret_cast<const double*>(b + o_nasa);
  dm.wfac = reinterpret_cast<const double*>(b + o_wfac);
  dm.rxn = reinterpret_cast<const Rxn*>(b + o_rxn);
  dm.eff_sp = reinterpret_cast<const int32_t*>(b + o_esp);
  dm.eff_am1 = reinterpret_cast<const double*>(b + o_eam);
  dm.rows = reinterpret_cast<const RowNu*>(b + o_rows);
  dm.pos_csr = reinterpret_cast<const int32_t*>(b + o_pcsr);
  dm.pos_csc = reinterpret_cast<const int32_t*>(b + o_pcsc);
  dm.perm = reinterpret_cast<const int32_t*>(b + o_perm);
  dm.exp_tab = reinterpret_cast<const double*>(b + o_etab);
  dm.tab = reinterpret_cast<const double*>(b + o_tab);
  dm.tgt_csr = reinterpret_cast<const int32_t*>(b + o_tcsr);
  dm.tgt_csc = reinterpret_cast<const int32_t*>(b + o_tcsc);
  dm.has_pdep = has_pdep ? 1 : 0;
  dm.nr_plain = nr_plain;
  dm.n_eff = (int32_t)eff_sp.size();
  dm.n_rows = (int32_t)rows.size();
  dm.n_tgt = (int32_t)tgt_csr.size();
  dm.dbg = reinterpret_cast<uint32_t*>(b + o_dbg);
  return lu_build(m);
}

void mech_release(pj_mech* m) {
  if (m && m->dev_blob) {
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != m->device) cudaSetDevice(m->device);
    cudaFree(m->dev_blob);
    if (m->lu_blob) cudaFree(m->lu_blob);
    if (cur != m->device && cur >= 0) cudaSetDevice(cur);
    m->dev_blob = nullptr;
    m->lu_blob = nullptr;
  }
}

}  // namespace pj

using namespace pj;

extern "C" const char* pj_last_error(void) { return g_last_error.c_str(); }

extern "C" const char* pj_version(void) { return "pyjac_gb 0.1 (sm_103a)"; }

extern "C" int pj_mech_create(const pj_mech_desc* d, pj_mech** out) {
  if (!d || !out) return fail(PJ_ERR_ARG, "pj_mech_create: null argument");
  *out = nullptr;
  const int ns = d->n_species, nr = d->n_reactions;
  if (ns < 2 || nr < 0) return fail(PJ_ERR_MECH, "pj_mech_create: bad sizes");
  if (!d->W || !d->T_mid || !d->nasa_low || !d->nasa_high || !d->eff_ptr ||
      (nr > 0 && (!d->kind || !d->reversible || !d->reac_sp || !d->reac_nu || !d->prod_sp ||
                  !d->prod_nu || !d->A || !d->beta || !d->Ea || !d->A0 || !d->beta0 ||
                  !d->Ea0 || !d->troe || !d->troe_n || !d->sri)))
    return fail(PJ_ERR_ARG, "pj_mech_create: null array in description");
  pj_mech* m = new (std::nothrow) pj_mech();
  if (!m) return fail(PJ_ERR_NOMEM, "pj_mech_create: out of host memory");
  try {
    m->ns = ns;
    m->nr = nr;
    m->W.assign(d->W, d->W + ns);
    m->T_mid.assign(d->T_mid, d->T_mid + ns);
    m->nasa_low.assign(d->nasa_low, d->nasa_low + 7 * ns);
    m->nasa_high.assign(d->nasa_high, d->nasa_high + 7 * ns);
    auto cp_i = [&](std::vector<int32_t>& v, const int32_t* s, size_t len) { v.assign(s, s + len); };
    auto cp_d = [&](std::vector<double>& v, const double* s, size_t len) { v.assign(s, s + len); };
    if (nr > 0) {
      cp_i(m->kind, d->kind, nr);
      cp_i(m->rev, d->reversible, nr);
      cp_i(m->reac_sp, d->reac_sp, (size_t)nr * PJ_MAX_SP);
      cp_i(m->reac_nu, d->reac_nu, (size_t)nr * PJ_MAX_SP);
      cp_i(m->prod_sp, d->prod_sp, (size_t)nr * PJ_MAX_SP);
      cp_i(m->prod_nu, d->prod_nu, (size_t)nr * PJ_MAX_SP);
      cp_d(m->A, d->A, nr);
      cp_d(m->beta, d->beta, nr);
      cp_d(m->Ea, d->Ea, nr);
      cp_d(m->A0, d->A0, nr);
      cp_d(m->beta0, d->beta0, nr);
      cp_d(m->Ea0, d->Ea0, nr);
      cp_d(m->troe, d->troe, (size_t)nr * 4);
      cp_i(m->troe_n, d->troe_n, nr);
      cp_d(m->sri, d->sri, (size_t)nr * 5);
    }
    cp_i(m->eff_ptr, d->eff_ptr, (size_t)nr + 1);
    const int ne = m->eff_ptr[nr];
    if (ne < 0) { delete m; return fail(PJ_ERR_MECH, "pj_mech_create: negative efficiency count"); }
    if (ne > 0 && (!d->eff_sp || !d->eff_val)) { delete m; return fail(PJ_ERR_ARG, "pj_mech_create: null efficiency arrays"); }
    if (ne > 0) {
      cp_i(m->eff_sp, d->eff_sp, ne);
      cp_d(m->eff_val, d->eff_val, ne);
    }
    // less common reaction types: absent arrays mean "none"
    auto opt_i = [&](std::vector<int32_t>& v, const int32_t* src, size_t len) {
      if (src) v.assign(src, src + len); else v.assign(len, 0);
    };
    auto opt_d = [&](std::vector<double>& v, const double* src, size_t len) {
      if (src) v.assign(src, src + len); else v.assign(len, 0.0);
    };
    opt_i(m->chem, d->chem, nr);
    opt_i(m->rev_explicit, d->rev_explicit, nr);
    opt_d(m->rev_A, d->rev_A, nr);
    opt_d(m->rev_beta, d->rev_beta, nr);
    opt_d(m->rev_Ea, d->rev_Ea, nr);
    opt_i(m->plog_ptr, d->plog_ptr, (size_t)nr + 1);
    opt_i(m->cheb_ptr, d->cheb_ptr, (size_t)nr + 1);
    opt_i(m->cheb_nT, d->cheb_nT, nr);
    opt_i(m->cheb_nP, d->cheb_nP, nr);
    opt_d(m->cheb_range, d->cheb_range, (size_t)nr * 4);
    const int npl = m->plog_ptr[nr], ncc = m->cheb_ptr[nr];
    if (npl < 0 || ncc < 0 || (npl > 0 && !d->plog) || (ncc > 0 && !d->cheb_coef)) {
      delete m;
      return fail(PJ_ERR_ARG, "pj_mech_create: P-log or Chebyshev counts without data");
    }
    opt_d(m->plog, d->plog, (size_t)npl * 4);
    opt_d(m->cheb_coef, d->cheb_coef, (size_t)ncc);
  } catch (...) {
    delete m;
    return fail(PJ_ERR_NOMEM, "pj_mech_create: out of host memory");
  }
  int rc = mech_build(m);
  if (rc) {
    mech_release(m);
    delete m;
    return rc;
  }
  *out = m;
  return PJ_OK;
}

extern "C" int pj_mech_free(pj_mech* m) {
  if (!m) return PJ_OK;
  mech_release(m);
  delete m;
  return PJ_OK;
}

extern "C" int pj_mech_info(const pj_mech* m, int32_t* ns, int32_t* nr, int32_t* nnz) {
  if (!m) return fail(PJ_ERR_ARG, "pj_mech_info: null mechanism");
  if (ns) *ns = m->ns;
  if (nr) *nr = m->nr;
  if (nnz) *nnz = m->nnz;
  return PJ_OK;
}

// A new handle holding a copy of src's mechanism description (not yet
// packed or uploaded); nullptr when host memory runs out.
static pj_mech* copy_description(const pj_mech* src) {
  pj_mech* m = new (std::nothrow) pj_mech();
  if (!m) return nullptr;
  try {
    m->ns = src->ns;
    m->nr = src->nr;
    m->W = src->W;
    m->T_mid = src->T_mid;
    m->nasa_low = src->nasa_low;
    m->nasa_high = src->nasa_high;
    m->A = src->A;
    m->beta = src->beta;
    m->Ea = src->Ea;
    m->A0 = src->A0;
    m->beta0 = src->beta0;
    m->Ea0 = src->Ea0;
    m->troe = src->troe;
    m->sri = src->sri;
    m->eff_val = src->eff_val;
    m->kind = src->kind;
    m->rev = src->rev;
    m->reac_sp = src->reac_sp;
    m->reac_nu = src->reac_nu;
    m->prod_sp = src->prod_sp;
    m->prod_nu = src->prod_nu;
    m->troe_n = src->troe_n;
    m->eff_ptr = src->eff_ptr;
    m->eff_sp = src->eff_sp;
    m->chem = src->chem;
    m->rev_explicit = src->rev_explicit;
    m->rev_A = src->rev_A;
    m->rev_beta = src->rev_beta;
    m->rev_Ea = src->rev_Ea;
    m->plog_ptr = src->plog_ptr;
    m->plog = src->plog;
    m->cheb_ptr = src->cheb_ptr;
    m->cheb_nT = src->cheb_nT;
    m->cheb_nP = src->cheb_nP;
    m->cheb_range = src->cheb_range;
    m->cheb_coef = src->cheb_coef;
  } catch (...) {
    delete m;
    return nullptr;
  }
  m->jac_form = src->jac_form;
  return m;
}

// Pack and upload a described handle; on failure release it.
static int finish_handle(pj_mech* m, pj_mech** out) {
  int rc = mech_build(m);
  if (rc) {
    mech_release(m);
    delete m;
    return rc;
  }
  *out = m;
  return PJ_OK;
}

extern "C" int pj_mech_with_jacobian_form(const pj_mech* src, int form, pj_mech** out) {
  if (!src || !out) return fail(PJ_ERR_ARG, "pj_mech_with_jacobian_form: null argument");
  *out = nullptr;
  if (form != PJ_JAC_EXACT && form != PJ_JAC_APPROX)
    return fail(PJ_ERR_ARG, "pj_mech_with_jacobian_form: form must be PJ_JAC_EXACT or PJ_JAC_APPROX");
  pj_mech* m = copy_description(src);
  if (!m) return fail(PJ_ERR_NOMEM, "pj_mech_with_jacobian_form: out of host memory");
  m->jac_form = form;
  return finish_handle(m, out);
}

extern "C" int pj_mech_arrhenius(const pj_mech* m, double* h_lnA, double* h_beta, double* h_Ea) {
  if (!m || !h_lnA || !h_beta || !h_Ea) return fail(PJ_ERR_ARG, "pj_mech_arrhenius: null argument");
  for (int i = 0; i < m->nr; i++) {
    h_lnA[i] = std::log(m->A[i]);
    h_beta[i] = m->beta[i];
    h_Ea[i] = m->Ea[i];
  }
  return PJ_OK;
}

extern "C" int pj_mech_with_arrhenius(const pj_mech* src, const double* h_lnA, const double* h_beta,
                                      const double* h_Ea, pj_mech** out) {
  if (!src || !h_lnA || !h_beta || !h_Ea || !out) return fail(PJ_ERR_ARG, "pj_mech_with_arrhenius: null argument");
  *out = nullptr;
  for (int i = 0; i < src->nr; i++)
    if (!std::isfinite(h_lnA[i]) || !std::isfinite(h_beta[i]) || !std::isfinite(h_Ea[i]))
      return fail(PJ_ERR_ARG, "pj_mech_with_arrhenius: non-finite parameter of reaction " + std::to_string(i));
  pj_mech* m = copy_description(src);
  if (!m) return fail(PJ_ERR_NOMEM, "pj_mech_with_arrhenius: out of host memory");
  for (int i = 0; i < m->nr; i++) {
    m->A[i] = std::exp(h_lnA[i]);
    m->beta[i] = h_beta[i];
    m->Ea[i] = h_Ea[i];
  }
  return finish_handle(m, out);
}

extern "C" int pj_mech_jacobian_form(const pj_mech* m, int32_t* form) {
  if (!m || !form) return fail(PJ_ERR_ARG, "pj_mech_jacobian_form: null argument");
  *form = m->jac_form;
  return PJ_OK;
}

extern "C" int pj_sparsity(const pj_mech* m, int fmt, int32_t* ptr, int32_t* idx) {
  if (!m || !ptr || !idx) return fail(PJ_ERR_ARG, "pj_sparsity: null argument");
  if (fmt != PJ_CSR && fmt != PJ_CSC) return fail(PJ_ERR_ARG, "pj_sparsity: fmt must be PJ_CSR or PJ_CSC");
  const auto& p = fmt == PJ_CSR ? m->csr_ptr : m->csc_ptr;
  const auto& x = fmt == PJ_CSR ? m->csr_idx : m->csc_idx;
  std::memcpy(ptr, p.data(), p.size() * sizeof(int32_t));
  std::memcpy(idx, x.data(), x.size() * sizeof(int32_t));
  return PJ_OK;
}

// ---- PJMECH text file ------------------------------------------------------
extern "C" int pj_mech_load(const char* path, pj_mech** out) {
  if (!path || !out) return fail(PJ_ERR_ARG, "pj_mech_load: null argument");
  std::ifstream in(path);
  if (!in) return fail(PJ_ERR_ARG, std::string("pj_mech_load: cannot open ") + path);
  std::string tok;
  auto expect = [&](const char* w) { return (in >> tok) && tok == w; };
  int version = 0;
  if (!expect("PJMECH") || !(in >> version) || (version != 1 && version != 2))
    return fail(PJ_ERR_MECH, "pj_mech_load: not a PJMECH 1 or 2 file");
  int ns = 0, nr = 0;
  if (!expect("SPECIES") || !(in >> ns) || ns < 2 || ns > 1000000) return fail(PJ_ERR_MECH, "pj_mech_load: bad SPECIES record");
  std::vector<double> W(ns), Tm(ns), lo(7 * ns), hi(7 * ns);
  for (int k = 0; k < ns; k++) {
    std::string name;
    int comp;
    if (!(in >> name >> W[k] >> Tm[k])) return fail(PJ_ERR_MECH, "pj_mech_load: truncated species record");
    for (int e = 0; e < 5; e++)
      if (!(in >> comp)) return fail(PJ_ERR_MECH, "pj_mech_load: truncated species composition");
    for (int j = 0; j < 7; j++) if (!(in >> lo[k * 7 + j])) return fail(PJ_ERR_MECH, "pj_mech_load: truncated NASA data");
    for (int j = 0; j < 7; j++) if (!(in >> hi[k * 7 + j])) return fail(PJ_ERR_MECH, "pj_mech_load: truncated NASA data");
  }
  if (!expect("REACTIONS") || !(in >> nr) || nr < 0 || nr > 10000000) return fail(PJ_ERR_MECH, "pj_mech_load: bad REACTIONS record");
  std::vector<int32_t> kind(nr), rev(nr), rsp((size_t)nr * PJ_MAX_SP, -1), rnu((size_t)nr * PJ_MAX_SP, 0),
      psp((size_t)nr * PJ_MAX_SP, -1), pnu((size_t)nr * PJ_MAX_SP, 0), tn(nr), eptr(nr + 1, 0), esp;
  std::vector<double> A(nr), b(nr), Ea(nr), A0(nr), b0(nr), Ea0(nr), troe((size_t)nr * 4), sri((size_t)nr * 5), eval;
  std::vector<int32_t> chem(nr, 0), revx(nr, 0), pptr(nr + 1, 0), cptr(nr + 1, 0), cnT(nr, 0), cnP(nr, 0);
  std::vector<double> rA(nr, 0.0), rb(nr, 0.0), rE(nr, 0.0), plog, crange((size_t)nr * 4, 0.0), ccoef;
  for (int i = 0; i < nr; i++) {
    int cnt;
    if (!(in >> kind[i] >> rev[i])) return fail(PJ_ERR_MECH, "pj_mech_load: truncated reaction record");
    for (int side = 0; side < 2; side++) {
      if (!(in >> cnt) || cnt < 0 || cnt > PJ_MAX_SP) return fail(PJ_ERR_MECH, "pj_mech_load: bad participant count");
      for (int a = 0; a < cnt; a++) {
        int32_t* sp = side ? &psp[(size_t)i * PJ_MAX_SP] : &rsp[(size_t)i * PJ_MAX_SP];
        int32_t* nu = side ? &pnu[(size_t)i * PJ_MAX_SP] : &rnu[(size_t)i * PJ_MAX_SP];
        if (!(in >> sp[a] >> nu[a])) return fail(PJ_ERR_MECH, "pj_mech_load: truncated participants");
      }
    }
    if (!(in >> A[i] >> b[i] >> Ea[i] >> A0[i] >> b0[i] >> Ea0[i] >> tn[i])) return fail(PJ_ERR_MECH, "pj_mech_load: truncated rate data");
    for (int j = 0; j < 4; j++) if (!(in >> troe[(size_t)i * 4 + j])) return fail(PJ_ERR_MECH, "pj_mech_load: truncated Troe data");
    for (int j = 0; j < 5; j++) if (!(in >> sri[(size_t)i * 5 + j])) return fail(PJ_ERR_MECH, "pj_mech_load: truncated SRI data");
    int ne;
    if (!(in >> ne) || ne < 0 || ne > 1000000) return fail(PJ_ERR_MECH, "pj_mech_load: bad efficiency count");
    for (int e = 0; e < ne; e++) {
      int32_t k;
      double v;
      if (!(in >> k >> v)) return fail(PJ_ERR_MECH, "pj_mech_load: truncated efficiencies");
      esp.push_back(k);
      eval.push_back(v);
    }
    eptr[i + 1] = (int32_t)esp.size();
    if (version >= 2) {
      int np;
      if (!(in >> chem[i] >> revx[i] >> rA[i] >> rb[i] >> rE[i])) return fail(PJ_ERR_MECH, "pj_mech_load: truncated reverse data");
      if (!(in >> np) || np < 0 || np > 1000000) return fail(PJ_ERR_MECH, "pj_mech_load: bad P-log count");
      for (int e = 0; e < 4 * np; e++) {
        double v;
        if (!(in >> v)) return fail(PJ_ERR_MECH, "pj_mech_load: truncated P-log data");
        plog.push_back(v);
      }
      if (!(in >> cnT[i] >> cnP[i]) || cnT[i] < 0 || cnP[i] < 0 || cnT[i] > 16 || cnP[i] > 16)
        return fail(PJ_ERR_MECH, "pj_mech_load: bad Chebyshev shape");
      if (cnT[i] * cnP[i] > 0) {
        for (int j = 0; j < 4; j++) if (!(in >> crange[(size_t)i * 4 + j])) return fail(PJ_ERR_MECH, "pj_mech_load: truncated Chebyshev range");
        for (int e = 0; e < cnT[i] * cnP[i]; e++) {
          double v;
          if (!(in >> v)) return fail(PJ_ERR_MECH, "pj_mech_load: truncated Chebyshev coefficients");
          ccoef.push_back(v);
        }
      }
    }
    pptr[i + 1] = (int32_t)(plog.size() / 4);
    cptr[i + 1] = (int32_t)ccoef.size();
  }
  if (!expect("END")) return fail(PJ_ERR_MECH, "pj_mech_load: missing END");
  pj_mech_desc d{};
  d.n_species = ns;
  d.n_reactions = nr;
  d.W = W.data(); d.T_mid = Tm.data(); d.nasa_low = lo.data(); d.nasa_high = hi.data();
  d.kind = kind.data(); d.reversible = rev.data();
  d.reac_sp = rsp.data(); d.reac_nu = rnu.data(); d.prod_sp = psp.data(); d.prod_nu = pnu.data();
  d.A = A.data(); d.beta = b.data(); d.Ea = Ea.data(); d.A0 = A0.data(); d.beta0 = b0.data(); d.Ea0 = Ea0.data();
  d.troe = troe.data(); d.troe_n = tn.data(); d.sri = sri.data();
  d.eff_ptr = eptr.data(); d.eff_sp = esp.data(); d.eff_val = eval.data();
  d.chem = chem.data(); d.rev_explicit = revx.data(); d.rev_A = rA.data(); d.rev_beta = rb.data(); d.rev_Ea = rE.data();
  d.plog_ptr = pptr.data(); d.plog = plog.data();
  d.cheb_ptr = cptr.data(); d.cheb_nT = cnT.data(); d.cheb_nP = cnP.data(); d.cheb_range = crange.data();
  d.cheb_coef = ccoef.data();
  return pj_mech_create(&d, out);
}
