"""CPU oracle (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It is a plain numpy float64 /
complex128 restatement of the method and shares no code with the CUDA path.
"""
from . import kinetics, forms
from .kinetics import (CONP, CONV, EXACT, APPROX, R, R_CAL, P_ATM, concentrations, nasa7, rates, source_terms,
                       source_terms_from_rates, jacobian, jacobian_columns, source_term_envelope, jacobian_envelope,
                       sparsity_pattern, csr_pattern, csc_pattern, dense_to_csr_values,
                       dense_to_csc_values, net_stoich, dependence_set)
from .forms import newton_matrix, vjp, outputs_y, y_jacobian, vjp_envelope, fd_jacobian, fd_steps
from . import linalg
