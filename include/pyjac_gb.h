/*
 * pyjac_gb.h -- C ABI of the GB300 library for thermochemical source terms
 * and analytical chemical-kinetic Jacobians (Curtis, Niemeyer & Sung,
 * "Using SIMD and SIMT vectorization to evaluate sparse chemical kinetic
 * Jacobian matrices and thermochemical source terms", arXiv:1809.01029).
 *
 * Conventions (every entry point):
 *  - Returns PJ_OK (0) or a PJ_ERR_* code; pj_last_error() gives a
 *    thread-local message for the last failure on the calling thread.  No
 *    C++ exception crosses this boundary.
 *  - Pointers named d_* are DEVICE pointers owned by the caller (e.g. PyTorch
 *    tensors); the library never frees them and never synchronises the
 *    stream.  Pointers named h_* are host pointers.  `stream` is a
 *    cudaStream_t passed as void* (NULL = legacy default stream).
 *  - State layout is structure-of-arrays (the paper's "F" ordering for
 *    shallow GPU vectorisation, Sec. 2.1): element v of state s is
 *    phi[v*ld + s] for v in [0, Ns] and s in [0, n), with ld >= n.  The state
 *    vector is Phi = [T, S, n_0 .. n_{Ns-2}] (Sec. 2.2): T in K; S = V [m^3]
 *    under constant pressure (PJ_CONP, P is the per-state parameter) or
 *    S = P [Pa] under constant volume (PJ_CONV, V is the parameter); n_k in
 *    kmol.  Species Ns-1 (the bath gas) is implicit through P V = n R T.
 *  - param[s] is P [Pa] (CONP) or V [m^3] (CONV), one per state.
 *  - Outputs use the same layout with the same ld: source terms
 *    dphi[v*ld + s]; sparse Jacobian values vals[e*ld + s] for e in [0, nnz)
 *    in the order of pj_sparsity(); dense Jacobian jac[(i*(Ns+1)+j)*ld + s]
 *    with i the source term (row) and j the state variable (column),
 *    Sec. 2.2 "Jacobian arrangement".
 *  - Units are SI with kmol: R = 8314.46261815324 J/(kmol K), activation
 *    energies in cal/mol (R_cal = 1.98720425864083 cal/(mol K)), standard
 *    pressure 101325 Pa.
 *  - Invalid states (T, V or P <= 0, any non-finite input, or a bath-gas
 *    concentration below -1e-12 of the total) get NaN outputs; if `d_status` (a device int)
 *    is non-NULL the number of such states is added to it atomically.
 *    Kernels never trap.
 *  - A mechanism handle is immutable after creation and may be used
 *    concurrently from several host threads on different streams.  Its
 *    constants live on the device that was current at creation; evaluation
 *    calls must run with that device current (PJ_ERR_ARG otherwise).
 */
#ifndef PYJAC_GB_H
#define PYJAC_GB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define PJ_OK 0
#define PJ_ERR_ARG 1          /* invalid argument (null pointer, ld < n, bad enum, ...) */
#define PJ_ERR_MECH 2         /* malformed mechanism (file or arrays) */
#define PJ_ERR_CUDA 3         /* a CUDA runtime call or launch failed */
#define PJ_ERR_NOMEM 4        /* host or device allocation failed / workspace too small */
#define PJ_ERR_UNSUPPORTED 5  /* valid request this build does not handle */
#define PJ_ERR_TIMEOUT 6      /* reserved for a bounded device-side wait that gives up; no entry point of
                                 this build returns it (its kernels wait only at block barriers and in
                                 tcgen05.alloc, whose columns are always available by construction) */

/* evaluation assumption (Sec. 2.2) */
#define PJ_CONP 0
#define PJ_CONV 1

/* Jacobian storage (Sec. 3.4: compressed row / column storage) */
#define PJ_CSR 0
#define PJ_CSC 1
#define PJ_DENSE 2

/* reaction kinds */
#define PJ_ELEMENTARY 0
#define PJ_THIRD_BODY 1
#define PJ_LINDEMANN 2
#define PJ_TROE 3
#define PJ_SRI 4
#define PJ_PLOG 5    /* pressure-dependent Arrhenius (P-log) */
#define PJ_CHEB 6    /* Chebyshev polynomial in 1/T and log P */

#define PJ_MAX_SP 4 /* distinct species per reaction side */

typedef struct pj_mech pj_mech;

/* Mechanism description: plain arrays, 0-based species indices, the last
 * species is the bath gas.  All arrays are host memory and are copied; the
 * caller keeps ownership.
 *   W[Ns]                 molecular weights, kg/kmol
 *   T_mid[Ns]             NASA-7 range switch: low coefficients iff T < T_mid
 *   nasa_low[Ns*7], nasa_high[Ns*7]  a0..a6 (cp/R = a0 + a1 T + .. + a4 T^4,
 *                         h/RT adds a5/T, s/R adds a6)
 *   kind[Nr]              PJ_ELEMENTARY .. PJ_CHEB
 *   reversible[Nr]        0/1; reverse rate from the equilibrium constant
 *   reac_sp/reac_nu[Nr*PJ_MAX_SP], prod_sp/prod_nu[...]: species (-1 pads)
 *                         and positive integer stoichiometric coefficients
 *   A, beta, Ea [Nr]      modified Arrhenius k = A T^beta exp(-Ea/(R_cal T));
 *                         the high-pressure limit for falloff reactions
 *   A0, beta0, Ea0 [Nr]   low-pressure limit (falloff kinds only)
 *   troe[Nr*4], troe_n[Nr]  a, T3, T1, T2 and the number of parameters (3|4)
 *   sri[Nr*5]             a, b, c, d, e
 *   eff_ptr[Nr+1], eff_sp[], eff_val[]  non-default third-body efficiencies
 *                         (CSR by reaction; default efficiency is 1)
 * Less common reaction types (Sec. 2.2 names them; standard forms).  Every
 * pointer below may be NULL when no reaction uses it:
 *   chem[Nr]              1: chemically-activated falloff (Lindemann / Troe /
 *                         SRI kinds): rate k0 F / (1 + Pr) instead of
 *                         k_inf F Pr / (1 + Pr)
 *   rev_explicit[Nr], rev_A/rev_beta/rev_Ea[Nr]  1: reverse rate
 *                         rev_A T^rev_beta exp(-rev_Ea/(R_cal T)) instead of
 *                         k_f / K_c (reversible reactions)
 *   plog_ptr[Nr+1], plog[n*4]  PJ_PLOG entries (P [Pa], A, beta, Ea), P
 *                         strictly ascending: ln k is linear in ln P between
 *                         neighbours, held at the end values outside
 *   cheb_ptr[Nr+1], cheb_nT/cheb_nP[Nr], cheb_range[Nr*4] (T_min, T_max [K],
 *                         P_min, P_max [Pa]), cheb_coef[] (row-major N_T x N_P
 *                         per reaction): PJ_CHEB, log10 k = sum a_tp
 *                         phi_t(T~) phi_p(P~), phi_n Chebyshev polynomials,
 *                         T~ = (2/T - 1/T_min - 1/T_max)/(1/T_max - 1/T_min),
 *                         P~ = (2 log P - log P_min - log P_max)/(log P_max
 *                         - log P_min); N_T, N_P in 1..16
 */
typedef struct {
  int32_t n_species, n_reactions;
  const double* W;
  const double* T_mid;
  const double* nasa_low;
  const double* nasa_high;
  const int32_t* kind;
  const int32_t* reversible;
  const int32_t* reac_sp;
  const int32_t* reac_nu;
  const int32_t* prod_sp;
  const int32_t* prod_nu;
  const double* A;
  const double* beta;
  const double* Ea;
  const double* A0;
  const double* beta0;
  const double* Ea0;
  const double* troe;
  const int32_t* troe_n;
  const double* sri;
  const int32_t* eff_ptr;
  const int32_t* eff_sp;
  const double* eff_val;
  const int32_t* chem;
  const int32_t* rev_explicit;
  const double* rev_A;
  const double* rev_beta;
  const double* rev_Ea;
  const int32_t* plog_ptr;
  const double* plog;
  const int32_t* cheb_ptr;
  const int32_t* cheb_nT;
  const int32_t* cheb_nP;
  const double* cheb_range;
  const double* cheb_coef;
} pj_mech_desc;

/* Thread-local message describing the last error on this thread. */
const char* pj_last_error(void);

/* Library version string. */
const char* pj_version(void);

/* Build a mechanism from arrays (copied), pack its constants for the
 * kernels, build the fixed sparsity pattern (Sec. 3.4) and upload both to the
 * current device.  *out receives a handle to release with pj_mech_free().
 * With no CUDA device present the handle is host-only: pj_mech_info and
 * pj_sparsity work, evaluation calls return PJ_ERR_CUDA.
 * Errors: PJ_ERR_ARG (null), PJ_ERR_MECH (index out of range, non-positive
 * A, bad kind, ...), PJ_ERR_CUDA / PJ_ERR_NOMEM (upload). */
int pj_mech_create(const pj_mech_desc* desc, pj_mech** out);

/* Same from a PJMECH text file (format documented in synth/mechfile.py:
 * one record per species and per reaction). */
int pj_mech_load(const char* path, pj_mech** out);

/* Release the handle and its device constants.  NULL is accepted. */
int pj_mech_free(pj_mech* mech);

/* Sizes: species, reactions, and nonzeros of the sparse Jacobian. */
int pj_mech_info(const pj_mech* mech, int32_t* n_species, int32_t* n_reactions, int32_t* nnz);

/* Jacobian forms (Sec. 3.4, "Sparsity patterns").  PJ_JAC_EXACT is the
 * derivative of the source terms.  PJ_JAC_APPROX leaves out, in the species
 * columns, the derivatives that reach a rate of progress through the bath
 * gas's concentration (C_Ns = C_tot - sum_k C_k depends on every n_j) and the
 * part of d[M]/dn_j that a non-unit bath-gas third-body efficiency spreads
 * over every species (the bath gas is counted at unit efficiency there); the
 * temperature and state columns, and the source terms, are unchanged.  Those
 * derivatives are what make whole species rows dense, so the approximate
 * pattern is sparser. */
#define PJ_JAC_EXACT 0
#define PJ_JAC_APPROX 1

/* New handle for the same mechanism data whose Jacobian entry points (sparse,
 * dense, Newton matrix, allocation-free, plans) and pj_sparsity / nnz use
 * `form`.  Source terms and the VJP (always the exact derivative) do not
 * depend on it.  Release *out with pj_mech_free().  Errors: PJ_ERR_ARG (null,
 * unknown form), PJ_ERR_CUDA / PJ_ERR_NOMEM (upload). */
int pj_mech_with_jacobian_form(const pj_mech* mech, int form, pj_mech** out);

/* The Jacobian form of a handle (PJ_JAC_EXACT for pj_mech_create/load). */
int pj_mech_jacobian_form(const pj_mech* mech, int32_t* form);

/* The high-pressure (or only) modified-Arrhenius parameters of every
 * reaction (the forward rate constant of Sec. 2.2, k = A T^beta
 * exp(-Ea / (R T))), in the reaction order of the description: host arrays
 * h_lnA[Nr] (ln A), h_beta[Nr], h_Ea[Nr] (cal/mol), written by the call.
 * These are the parameters theta of the VJP's g_theta (pj_vjp).  Errors:
 * PJ_ERR_ARG (null). */
int pj_mech_arrhenius(const pj_mech* mech, double* h_lnA, double* h_beta, double* h_Ea);

/* A new handle for the same mechanism (and Jacobian form) with reaction i's
 * high-pressure (or only) Arrhenius parameters replaced by (h_lnA[i],
 * h_beta[i], h_Ea[i]) (Sec. 2.2 rate constants; host arrays of Nr, read
 * only; the low-pressure, reverse, P-log and Chebyshev data stay as they
 * are).  For parameter fitting and sensitivity loops that evaluate the
 * source terms and the VJP at changing theta.  The source handle is not
 * modified; release *out with pj_mech_free().  Errors: PJ_ERR_ARG (null,
 * non-finite parameter), PJ_ERR_MECH (exp(ln A) not a positive finite
 * number), PJ_ERR_CUDA / PJ_ERR_NOMEM (upload). */
int pj_mech_with_arrhenius(const pj_mech* mech, const double* h_lnA, const double* h_beta, const double* h_Ea,
                           pj_mech** out);

/* Sparsity pattern of the Jacobian (Sec. 3.4), identical for CONP and
 * CONV: rows/columns of T and S dense, diagonal kept, species row k has
 * column j when a reaction that changes k has a rate depending on j (its
 * reactants, its products if reversible, species whose third-body efficiency
 * differs from the bath gas's, or every species when the bath gas takes part
 * in the rate; for PJ_JAC_APPROX handles, efficiencies differing from 1 and
 * no every-species clause).  fmt = PJ_CSR: h_ptr[Ns+2] row pointers, h_idx[nnz] column
 * indices ascending per row; PJ_CSC: column pointers / row indices. */
int pj_sparsity(const pj_mech* mech, int fmt, int32_t* h_ptr, int32_t* h_idx);

/* Source terms f = dPhi/dt (Sec. 2.2: molar source terms dn_k/dt = V wdot_k
 * with wdot_k = sum_i nu_ki R_i c_i; dT/dt from species enthalpies (CONP) or
 * internal energies (CONV); dV/dt or dP/dt from the ideal-gas law with the
 * bath gas closing the mass balance) for n states.  d_work / work_bytes: device
 * scratch of at least pj_workspace_size(PJ_OP_SOURCE) bytes (NULL when 0);
 * PJ_ERR_NOMEM if it is too small. */
int pj_eval_source_terms(const pj_mech* mech, int mode, int64_t n, const double* d_param,
                         const double* d_phi, int64_t ld, double* d_dphi, int* d_status,
                         void* d_work, size_t work_bytes, void* stream);

/* Exact analytical Jacobian J_ij = d f_i / d Phi_j (Sec. 2.2 "Jacobian
 * arrangement"; sparse storage Sec. 3.4) in CSR (fmt = PJ_CSR) or CSC
 * (PJ_CSC) value order: d_vals[e*ld + s].  d_dphi (required, same layout as
 * d_phi) receives the source terms, which the Jacobian kernel computes on the
 * way.  d_work must point to pj_workspace_size(PJ_OP_JACOBIAN) bytes of
 * device memory (may be NULL when that size is 0).  That size is the need of
 * the one-state-per-thread layouts, the largest of any layout; the
 * cooperative layout uses no workspace, so a short one is rejected
 * (PJ_ERR_NOMEM, nothing launched) only when the layout that runs needs it.
 *
 * Reproducibility: with the cooperative layout (pj_jacobian_layout) the
 * entries and production rates receive reductions from several warps in an
 * order that can change between runs, so results agree to the rounding of
 * those sums, not bit for bit; the one-state-per-thread layouts give the
 * same bits on every run.  The environment variable PYJAC_GB_JAC_LAYOUT
 * (read at every launch) forces a family: "percore" (bit-reproducible) or
 * "coop" (where its shared memory fits); PYJAC_GB_COOP_WARPS = 4, 8 or 16
 * sets the cooperative block's warps, PYJAC_GB_COOP_CTAS the blocks per
 * SM, and PYJAC_GB_COOP_ARRAYS = "global" puts a tile's per-state arrays in
 * the workspace instead of shared memory. */
int pj_eval_jacobian_sparse(const pj_mech* mech, int mode, int fmt, int64_t n,
                            const double* d_param, const double* d_phi, int64_t ld,
                            double* d_vals, double* d_dphi, int* d_status,
                            void* d_work, size_t work_bytes, void* stream);

/* Same, dense row-major (Ns+1)x(Ns+1) per state: d_jac[(i*(Ns+1)+j)*ld + s]. */
int pj_eval_jacobian_dense(const pj_mech* mech, int mode, int64_t n, const double* d_param,
                           const double* d_phi, int64_t ld, double* d_jac, double* d_dphi,
                           int* d_status, void* d_work, size_t work_bytes, void* stream);

/* Newton-iteration matrix M = I - h*gamma*J in FP32 (the matrix an implicit
 * integrator factors; the paper motivates the Jacobian by implicit
 * integration, Sec. 1, Sec. 3.4).  Rates, Gibbs-energy differences and
 * equilibrium constants, every exponential and the source terms are FP64;
 * the derivative arithmetic, the accumulation of J and the assembly of M are
 * FP32.  d_h[n] is the per-state step h (device), gamma a scalar; fmt is
 * PJ_CSR / PJ_CSC (values in pj_sparsity order, the diagonal is in the
 * pattern) or PJ_DENSE; d_M[e*ld + s] is float.  d_dphi (required) receives
 * the FP64 source terms.  Workspace as for pj_eval_jacobian_sparse
 * (PJ_OP_NEWTON). */
int pj_newton_matrix_f32(const pj_mech* mech, int mode, int fmt, int64_t n, const double* d_param,
                         const double* d_phi, int64_t ld, const double* d_h, double gamma, float* d_M,
                         double* d_dphi, int* d_status, void* d_work, size_t work_bytes, void* stream);

/* Allocation-free variant of pj_eval_jacobian_sparse (no counterpart in the
 * paper).  For callers that cannot allocate device memory or call an
 * allocating library routine, and so cannot supply d_work: the per-state
 * working arrays live in a fixed 64 MiB device array inside the library,
 * which every GPU that loads the library holds until the process exits.
 * Same arguments and outputs as pj_eval_jacobian_sparse minus the workspace.
 *  - Every call looks up that array's device address in the current
 *    device's context (cudaGetSymbolAddress, which does not allocate); the
 *    first call on a device loads the library's module there, so make it
 *    before any stream capture.
 *  - It runs the one-state-per-thread kernel with every per-state array in
 *    that global array (none of the shared-memory, tensor-memory or
 *    cooperative layouts pj_eval_jacobian_sparse picks), so it is slower
 *    than the regular entry on mechanisms those layouts serve (the
 *    benchmark's variants report both).
 *  - All calls on a device share the array and it keeps the last call's
 *    contents; calls that overlap on the GPU (different streams, or
 *    concurrent host threads) race on it, so serialise them.
 *  - Mechanisms whose arrays for 128 states exceed 64 MiB (about 21,800
 *    species) are rejected with PJ_ERR_UNSUPPORTED; n is unrestricted
 *    (states are processed in a grid-stride loop). */
int pj_eval_jacobian_sparse_noalloc(const pj_mech* mech, int mode, int fmt, int64_t n,
                                    const double* d_param, const double* d_phi, int64_t ld,
                                    double* d_vals, double* d_dphi, int* d_status, void* stream);

/* Source terms and sparse Jacobian (the operation of pj_eval_jacobian_sparse,
 * Sec. 2.2 and 3.4) of n states held in HOST memory, the transfers inside the
 * call.  h_param[s] and h_phi[v*n + s] in; h_vals[e*n + s] (pattern of fmt,
 * PJ_CSR or PJ_CSC) and h_dphi[v*n + s] out; the host arrays' leading
 * dimension is n.  The states go through the GPU in chunks of `chunk` states
 * (0: as many as fit 4 GiB of staging per chunk) and three device staging
 * slots, uploads, kernels and downloads on separate streams so that the
 * transfers of one chunk overlap the kernel of another.  Page-locked host
 * buffers (cudaHostAlloc or cudaHostRegister) let the copies run
 * asynchronously at full bandwidth; pageable ones work but serialise.
 * The call orders itself after the work queued on `stream`, allocates its
 * staging (3 slots of (2 (Ns+1) + 1 + nnz) x chunk doubles plus the
 * Jacobian workspace) and its streams, and returns once the outputs are on
 * the host.  h_status (host, nullable) receives the number of invalid
 * states.  Errors: PJ_ERR_ARG, PJ_ERR_NOMEM (staging does not fit: pass a
 * smaller chunk), PJ_ERR_UNSUPPORTED (n x 8 bytes beyond the device's copy
 * pitch limit), PJ_ERR_CUDA. */
int pj_eval_jacobian_sparse_host(const pj_mech* mech, int mode, int fmt, int64_t n, const double* h_param,
                                 const double* h_phi, double* h_vals, double* h_dphi, int* h_status, int64_t chunk,
                                 void* stream);

/* Bounds-checked build.  The library compiled with -DPJ_DEBUG_BOUNDS
 * (paper_1809_01029_gb300.build: debug_bounds=True, libpyjac_gb_dbg.so)
 * checks every lookup in the index tables derived at mechanism load (the
 * Jacobian kernels' per-reaction target lists and full -> sparse position
 * maps, the species-row and efficiency lists, the LU scatter and gather
 * maps) before use; a bad index sets a bit of the mechanism's device error
 * word and the access is skipped (no trap).  Bits: 1 target list, 2 position
 * map, 4 species-row list, 8 efficiency list, 16 LU map.  The paper has no
 * counterpart (it is a diagnostic of this library).
 *
 * pj_debug_word: *h_word = the error word (synchronous copy; clear != 0
 * resets it).  Always 0 in the regular build.  Errors: PJ_ERR_ARG,
 * PJ_ERR_CUDA.
 * pj_debug_build: *on = 1 in the bounds-checked build, else 0.
 * pj_debug_set_target: test hook of the bounds-checked build only -- writes
 * `value` into entry `index` of the device target list of fmt (PJ_CSR or
 * PJ_CSC), so that a test can show the checks catching a corrupt table.
 * PJ_ERR_UNSUPPORTED in the regular build; PJ_ERR_ARG for an index outside
 * the list. */
int pj_debug_word(const pj_mech* mech, uint32_t* h_word, int clear);
int pj_debug_build(int32_t* on);
int pj_debug_set_target(const pj_mech* mech, int fmt, int32_t index, int32_t value);

/* Kernel layouts of the Jacobian entries (pj_jacobian_layout) */
#define PJ_LAYOUT_PERCORE 0  /* one state per thread; state arrays in shared memory or a workspace */
#define PJ_LAYOUT_TMEM 1     /* one state per thread; h_k/RT in tensor memory */
#define PJ_LAYOUT_COOP 2     /* the warps of a block share 32 states and split the reactions */

/* The kernel layout the Jacobian entries (pj_eval_jacobian_sparse / dense,
 * fmt PJ_CSR, PJ_CSC or PJ_DENSE) and the FP32 Newton matrix (prec PJ_F32)
 * use for n states of this mechanism on the current device: *layout =
 * PJ_LAYOUT_*.  The choice was measured on GB300: the cooperative layout
 * for batches of at most one 32-state tile per SM, for batches below one
 * round of the one-state-per-thread kernels, and for the sparse Jacobians
 * and FP32 Newton matrices of mechanisms too large for per-thread shared
 * memory; tensor memory for the dense Jacobian of such mechanisms; shared
 * memory, one state per thread, for small mechanisms on large batches.  The
 * cooperative layout keeps few Jacobians live in L2 (a third to a half of
 * the DRAM traffic at 53 species) and is not bit-reproducible (see
 * pj_eval_jacobian_sparse).  Errors: PJ_ERR_ARG, PJ_ERR_CUDA (no device
 * copy). */
int pj_jacobian_layout(const pj_mech* mech, int fmt, int prec, int64_t n, int32_t* layout);

/* operation ids for pj_workspace_size */
#define PJ_OP_SOURCE 0
#define PJ_OP_JACOBIAN 1
#define PJ_OP_NEWTON 2
#define PJ_OP_VJP 3
#define PJ_OP_Y 4
#define PJ_OP_FD 5
#define PJ_OP_LU 6

/* Device scratch (bytes) an operation needs for a batch of n states; 0 when
 * the per-state working arrays fit in shared memory (PJ_OP_VJP always needs
 * room for its per-warp parameter-gradient partial sums). */
int pj_workspace_size(const pj_mech* mech, int op, int64_t n, size_t* bytes);

/* First-order forward finite-difference Jacobian, the comparator of
 * Sec. 3.5.2 (the analytical Jacobian's speedup over it): column j is
 * (f(Phi + h_j e_j) - f(Phi)) / h_j with delta_j = 2^-26 max(|Phi_j|,
 * 2^-26 n_tot), n_tot = P V / (R T), and h_j = (Phi_j + delta_j) - Phi_j
 * (the paper gives no step rule).  Same layout and formats as the
 * analytical entry points (fmt = PJ_CSR / PJ_CSC values in the handle's
 * pattern, PJ_DENSE rows); d_dphi (required) receives f(Phi).  Costs N + 1
 * source-term evaluations per state.  Workspace: pj_workspace_size(PJ_OP_FD)
 * bytes, always nonzero.  A column whose perturbed state is invalid is NaN
 * without counting in *d_status (the state itself is validated as usual). */
int pj_eval_jacobian_fd(const pj_mech* mech, int mode, int fmt, int64_t n, const double* d_param,
                        const double* d_phi, int64_t ld, double* d_vals, double* d_dphi, int* d_status,
                        void* d_work, size_t work_bytes, void* stream);

/* Forward values of the differentiation form: y = (wdot_0 .. wdot_{Ns-1},
 * dT/dt) per state, the species production rates of Sec. 2.2 (bath gas
 * included) and the temperature source term; d_y[k*ld + s], k in [0, Ns].
 * Workspace: pj_workspace_size(PJ_OP_Y). */
int pj_eval_y(const pj_mech* mech, int mode, int64_t n, const double* d_param, const double* d_phi,
              int64_t ld, double* d_y, int* d_status, void* d_work, size_t work_bytes, void* stream);

/* Vector-Jacobian product of y (see pj_eval_y) for sensitivity analysis:
 * with cotangents d_u_wdot[k*ld + s] (k < Ns) and d_u_T[s],
 *   d_g_phi[j*ld + s] = sum_y u_y dy/dPhi_j        (per state, j in [0, Ns])
 *   d_g_theta[3*i + p] = sum_s sum_y u_y dy/dtheta_ip  (summed over states)
 * for the per-reaction parameters theta_i = (ln A_i, beta_i, Ea_i) of the
 * high-pressure (or only) Arrhenius rate, reactions in description order
 * (Ea in cal/mol).  d_y receives y.  The state sum is deterministic for a
 * given (mechanism, n).  Workspace: pj_workspace_size(PJ_OP_VJP), required. */
int pj_vjp(const pj_mech* mech, int mode, int64_t n, const double* d_param, const double* d_phi, int64_t ld,
           const double* d_u_wdot, const double* d_u_T, double* d_y, double* d_g_phi, double* d_g_theta,
           int* d_status, void* d_work, size_t work_bytes, void* stream);

/* Diagnostic: the library's FP64 exponential (Tang's table-driven method,
 * used by every kernel for rate constants and falloff factors) and CUDA's
 * exp for the same n device inputs, so that its error can be verified. */
int pj_diag_exp(const pj_mech* mech, int64_t n, const double* d_x, double* d_y_ours, double* d_y_lib,
                void* stream);

/* ---- batching form: uneven batches, persistent kernels, CUDA graphs ----
 *
 * One batch of states: its own device buffers and leading dimension (the
 * layout of pj_eval_source_terms / pj_eval_jacobian_sparse).  d_out receives
 * the source terms (PJ_OP_SOURCE) or the Jacobian values in `fmt` order
 * (PJ_OP_JACOBIAN, FP64); d_dphi receives the source terms of a Jacobian
 * plan (required there, unused otherwise). */
typedef struct {
  const double* d_param;
  const double* d_phi;
  int64_t n;
  int64_t ld;
  double* d_out;
  double* d_dphi;
} pj_batch;

typedef struct pj_plan pj_plan;

/* Plan the evaluation of n_batches batches (op PJ_OP_SOURCE or
 * PJ_OP_JACOBIAN).  Consecutive batches are grouped into launches of at most
 * max_states_per_launch states (0: one launch); in each launch a persistent
 * kernel's warps take 32-state tiles of any batch of the group from a work
 * counter.  Batches of different groups may share output memory (groups run
 * one after another on the stream).  d_status (nullable) counts invalid
 * states.  Allocates device tables and, when the per-state arrays do not fit
 * shared memory, a workspace.  The default launch shape is the one
 * pj_workspace_size would imply; see pj_plan_autotune. */
int pj_plan_create(const pj_mech* mech, int op, int mode, int fmt, int n_batches, const pj_batch* batches,
                   int64_t max_states_per_launch, int* d_status, pj_plan** out);
int pj_plan_free(pj_plan* plan);

/* Launch shape: threads per block (32, 64, 128), resident blocks per SM
 * (1..16; the grid is blocks_per_sm x SMs), per-state arrays in shared
 * memory (use_shared = 1) or in the plan's global workspace. */
int pj_plan_set_config(pj_plan* plan, int threads_per_block, int blocks_per_sm, int use_shared);
int pj_plan_get_config(const pj_plan* plan, int* threads_per_block, int* blocks_per_sm, int* use_shared,
                       int* n_groups);

/* Time every admissible launch shape on the plan's own batches (reps runs
 * each, after one warm-up) and keep the fastest.  With cache_path non-NULL
 * the choice is read from / appended to that file (one JSON object per line,
 * keyed by GPU name, a hash of the mechanism constants, op, mode and fmt);
 * a cached entry is used without timing.  Synchronises the stream. */
int pj_plan_autotune(pj_plan* plan, void* stream, const char* cache_path, int reps);

/* Run the plan on `stream` (asynchronous). */
int pj_plan_run(pj_plan* plan, void* stream);

/* Capture one run into a CUDA graph on a non-default `stream`, then replay it
 * with pj_plan_launch (counters reset inside the graph).  Changing the launch
 * shape drops the graph. */
int pj_plan_capture(pj_plan* plan, void* stream);
int pj_plan_launch(pj_plan* plan, void* stream);

/* ------------------------------------------------------------------------
 * Linear algebra of the Newton matrix M = I - h gamma J: batched LU and solve
 * in the Jacobian's fixed pattern (Sec. 5 names these as the missing piece
 * for implicit integration, over many small matrices rather than one large).
 * Per handle (and Jacobian form) a symbolic phase fixes, at creation:
 *  - the pivot order perm: species by greedy minimum degree on the
 *    symmetrised species block (ties by lowest index), then T and S;
 *  - the fill of LU without pivoting of A = P M P^T (A[k][l] = M[perm[k]]
 *    [perm[l]]): L unit lower, U upper;
 *  - the storage order of the lu_nnz factor values per state: strictly lower
 *    rows k = 0..N-1 (columns ascending), then upper rows k = N-1..0, each as
 *    1/U_kk followed by U_kj, j > k ascending.
 * No pivoting: a state whose factors are not all finite (a zero pivot, or
 * overflow -- FP32's range is exceeded by very stiff states, whose unscaled
 * entries reach 1e20 and more) increments *d_status once; M of an implicit
 * step is the identity plus h gamma J.
 * ------------------------------------------------------------------------ */
#define PJ_F64 0
#define PJ_F32 1

/* lu_nnz and (h_perm non-NULL) perm[N]. */
int pj_lu_info(const pj_mech* mech, int32_t* lu_nnz, int32_t* h_perm);

/* Pivot-order (row, column) of each factor value, in storage order. */
int pj_lu_pattern(const pj_mech* mech, int32_t* h_rows, int32_t* h_cols);

/* Factor n matrices.  d_vals: [nnz x ld] CSR values (pj_sparsity order) of
 * M -- or, with d_h non-NULL, of J, and M = I - d_h[s] gamma J is formed on
 * the way in -- in double (PJ_F64) or float (PJ_F32, e.g. the output of
 * pj_newton_matrix_f32); d_lu: [lu_nnz x ld] factors of the same type.
 * Workspace: pj_workspace_size(PJ_OP_LU) bytes (0 unless N^2 values exceed
 * shared memory). */
int pj_lu_factor(const pj_mech* mech, int prec, int64_t n, const void* d_vals, int64_t ld, const double* d_h,
                 double gamma, void* d_lu, int* d_status, void* d_work, size_t work_bytes, void* stream);

/* Solve M x = b for n states with factors from pj_lu_factor: d_b, d_x
 * [N x ld] of the factors' type (d_x may equal d_b). */
int pj_lu_solve(const pj_mech* mech, int prec, int64_t n, const void* d_lu, int64_t ld, const void* d_b,
                void* d_x, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* PYJAC_GB_H */
