"""Seeded synthetic inputs (mechanisms, states, cotangents, step sizes).

Shared by the CPU oracle and the CUDA path; holds none of the evaluated
method's arithmetic.
"""
from .mechanism import (ELEMENTARY, THIRD_BODY, LINDEMANN, TROE, SRI, PLOG, CHEB, KIND_NAMES, MAX_SP,
                        ELEMENTS, ATOMIC_MASS, Mechanism, MechSpec, SPECS, make_mechanism,
                        build_mechanism)
from .states import (CONP, CONV, P_ATM, WORKLOADS, Workload, make_states, ragged_batch_sizes,
                     make_cotangents, make_step_sizes)
from .mechfile import write_mechanism, read_mechanism
