// Internal definitions shared by the host-side mechanism code and the CUDA
// kernels of libpyjac_gb: packed mechanism constants and launch helpers.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "pyjac_gb.h"

namespace pj {

// physical constants, SI with kmol
constexpr double RU = 8314.46261815324;      // J / (kmol K)
constexpr double R_CAL = 1.98720425864083;   // cal / (mol K)
constexpr double P_STD = 101325.0;           // Pa
constexpr double LN10 = 2.302585092994045684;

// per-species NASA-7 block: two ranges of 16 doubles
//   [0..6]  a0..a6
//   [7..10] a1/2, a2/3, a3/4, a4/5   (enthalpy polynomial)
//   [11..13] a2/2, a3/3, a4/4        (entropy polynomial)
//   [14]    T_mid (same in both ranges), [15] unused
constexpr int NASA_STRIDE = 32;

// Stoichiometric pattern of one reaction side, chosen on the host so that the
// kernels form C-products and their derivatives with exactly the multiplies
// they need (species ordered to match the pattern).
enum : int32_t {
  SH_1 = 0,    // A
  SH_2 = 1,    // 2A
  SH_11 = 2,   // A + B
  SH_21 = 3,   // 2A + B
  SH_111 = 4,  // A + B + C
  SH_GEN = 5   // anything else (generic loop)
};

// One reaction, packed for warp-uniform loads (every thread of a warp reads
// the same record).  Reactions are stored in kernel order (see perm).
struct alignas(8) Rxn {
  double lnA, beta, theta;        // k = exp(lnA + beta lnT - theta/T), theta = Ea/R_cal [K]
  double lnA0, beta0, theta0;     // low-pressure limit (falloff)
  double dnu;                     // sum_k nu_k (equilibrium-constant pressure factor)
  double dW;                      // sum_{k<Ns-1} nu_k (1 - W_k/W_Ns)
  double alpha_bath;              // third-body efficiency of the bath gas
  double fp[5];                   // Troe: a, 1/T3, 1/T1, T2, has_T2 ; SRI: a, b, 1/c, d, e
  double nud[2 * PJ_MAX_SP];      // stoichiometric coefficients as doubles
  int32_t kind, rev;              // rev: 0 irreversible, 1 k_r = k_f / K_c, 2 explicit (DevMech::tab)
  int32_t nreac, nprod;
  int32_t shape[2];               // SH_* of the reactant and product sides
  int32_t sp[2 * PJ_MAX_SP];      // reactants [0, nreac), products [PJ_MAX_SP, PJ_MAX_SP + nprod)
  int32_t nu[2 * PJ_MAX_SP];
  int32_t eff_lo, eff_hi;         // non-default efficiencies in eff_sp / eff_am1
  int32_t row_lo, row_hi;         // species rows (k < Ns-1, net nu != 0) in rows[]
  int32_t dense;                  // rate depends on every species (bath gas involved)
  int32_t chem;                   // chemically-activated falloff
  int32_t tab_lo;                 // DevMech::tab: explicit reverse (ln A, beta, theta) when rev == 2,
                                  // then the P-log entries / Chebyshev block
  int16_t tab_n, tab_m;           // P-log entries / Chebyshev N_T, N_P
  int32_t tgt_lo;                 // first of this reaction's Jacobian targets in tgt_csr / tgt_csc
  int32_t bath_in;                // the bath gas is one of its reactants or products
};

// One unit of a reaction's net stoichiometric coefficient for species k: a
// species with |nu| = 2 has two such rows.
struct RowNu {
  int32_t k;      // species index (< Ns-1)
  int32_t nu;     // +1 or -1
  double nud;     // the same as a double
};

// Kernel view of a mechanism (POD, passed by value).
struct DevMech {
  int32_t ns, nr, N, nnz;
  double log_pstd_over_r;         // ln(P_std / R)
  const double* nasa;             // [ns * NASA_STRIDE]
  const double* wfac;             // [ns] 1 - W_k / W_{Ns-1}
  const Rxn* rxn;                 // [nr]
  const int32_t* eff_sp;          // [n_eff]
  const double* eff_am1;          // [n_eff] alpha - 1
  const RowNu* rows;              // [n_rows]
  const int32_t* pos_csr;         // [N*N] full -> CSR value index, -1 if absent
  const int32_t* pos_csc;         // [N*N] full -> CSC value index, -1 if absent
  const int32_t* tgt_csr;         // per reaction, the value indices its sparse contributions
  const int32_t* tgt_csc;         //   go to, in the order the Jacobian kernels make them
  const int32_t* perm;            // [nr] kernel order -> original reaction index
  const double* exp_tab;          // [256] 2^(j/256), correctly rounded (pj_exp)
  const double* tab;              // P-log entries (ln P, ln A, beta, theta) and Chebyshev
                                  // blocks (cT1, cT0, cP1, cP0, ln10 * a_tp row-major)
  int32_t has_pdep;               // some reaction depends on P (P-log, Chebyshev)
  int32_t nr_plain;               // plain reactions (kernel order): none chemically activated,
                                  // with explicit reverse parameters, P-log or Chebyshev
  int32_t n_eff, n_rows, n_tgt;   // lengths of eff_sp / rows / each target list array
  uint32_t* dbg;                  // error word of the bounds-checked build (PJ_DEBUG_BOUNDS)
};

// Index tables of the Newton-matrix LU (lu_symbolic.cpp, lu.cu); pivot
// order k, dense pivot-order positions r*N + c.
struct DevLu {
  int32_t N, nnz, lu_nnz, nl;  // nnz: CSR entries of M; nl: strictly lower factor entries
  int32_t NP;                  // row stride of the dense pivot-order arrays (N rounded up to odd)
  const int32_t* perm;         // [N] state-vector index of pivot k
  const int32_t* rptr;         // [N+1] rows i > k of column k ...
  const int32_t* ridx;         //   ... ascending
  const int32_t* cptr;         // [N+1] columns j > k of row k ...
  const int32_t* cidx;         //   ... ascending
  const int32_t* m2d;          // [nnz] CSR entry -> dense position r * NP + c
  const int32_t* l2d;          // [lu_nnz] factor entry (storage order) -> dense position
  const int32_t* xcol;         // [lu_nnz] state-vector index of the entry's column
  const int32_t* lptr;         // [N+1] lower row k in storage
  const int32_t* uptr;         // [N+1] upper row N-1-q in storage (diagonal first)
  uint32_t* dbg;               // error word of the bounds-checked build (the mechanism's)
};

}  // namespace pj

struct pj_mech {
  int32_t ns = 0, nr = 0, nnz = 0;
  int32_t jac_form = PJ_JAC_EXACT;  // Jacobian form of the pattern and kernels
  int device = -1;
  // host copies of the description
  std::vector<double> W, T_mid, nasa_low, nasa_high, A, beta, Ea, A0, beta0, Ea0, troe, sri, eff_val;
  std::vector<int32_t> kind, rev, reac_sp, reac_nu, prod_sp, prod_nu, troe_n, eff_ptr, eff_sp;
  // less common reaction types (empty when absent)
  std::vector<int32_t> chem, rev_explicit, plog_ptr, cheb_ptr, cheb_nT, cheb_nP;
  std::vector<double> rev_A, rev_beta, rev_Ea, plog, cheb_range, cheb_coef;
  // derived
  std::vector<int32_t> perm;          // kernel order -> original reaction index
  std::vector<int32_t> csr_ptr, csr_idx, csc_ptr, csc_idx;
  std::vector<int32_t> pos_csr, pos_csc;
  pj::DevMech dm{};
  void* dev_blob = nullptr;
  size_t dev_bytes = 0;
  // LU of the Newton matrix: pivot order, factor storage (pivot indices)
  std::vector<int32_t> lu_perm, lu_rows, lu_cols;
  pj::DevLu lu{};
  void* lu_blob = nullptr;
};

namespace pj {
// error reporting (thread-local message)
int fail(int code, const std::string& msg);
int check_cuda(int err, const char* what);
int mech_build(pj_mech* m);          // pack + pattern + upload
int lu_build(pj_mech* m);            // LU ordering, fill and tables (after the pattern)
void mech_release(pj_mech* m);
}  // namespace pj
