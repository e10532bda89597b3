"""GB300 (sm_103a) library for thermochemical source terms and analytical
chemical-kinetic Jacobians (arXiv:1809.01029), behind the C ABI of
include/pyjac_gb.h.  This package is the thin Python binding."""
from .api import (Mechanism, pj_mech_create, pj_mech_load, pj_sparsity, pj_workspace_size,
                  pj_mech_with_jacobian_form, pj_mech_jacobian_form, PJ_JAC_EXACT, PJ_JAC_APPROX,
                  pj_mech_arrhenius, pj_mech_with_arrhenius, pj_jacobian_layout,
                  pj_debug_word, pj_debug_build, pj_debug_set_target,
                  PJ_LAYOUT_PERCORE, PJ_LAYOUT_TMEM, PJ_LAYOUT_COOP,
                  pj_lu_factor, pj_lu_solve, lu_factor, lu_solve, PJ_OP_LU, PJ_F64, PJ_F32,
                  pj_eval_source_terms, pj_eval_jacobian_sparse, pj_eval_jacobian_dense,
                  pj_eval_jacobian_sparse_noalloc, pj_eval_jacobian_sparse_host, jacobian_sparse_host,
                  pj_newton_matrix_f32, newton_matrix_f32,
                  pj_eval_y, pj_vjp, eval_y, vjp, source_terms_y, arrhenius_parameters, PJ_OP_Y, Plan, pj_diag_exp,
                  source_terms, jacobian_sparse, jacobian_dense, jacobian_fd, pj_eval_jacobian_fd, PJ_OP_FD,
                  PJ_CONP, PJ_CONV, PJ_CSR, PJ_CSC, PJ_DENSE, PJ_OP_SOURCE, PJ_OP_JACOBIAN,
                  PJ_OP_NEWTON, PJ_OP_VJP)
from ._native import PJError, load as load_library
