"""Hand-built tiny mechanisms that cover every reaction kind and the bath-gas
cases of the sparsity rules (Sec. 3.4).  Inputs only: no method arithmetic.

Species (last = bath gas N2): 0 H, 1 O, 2 H2, 3 O2, 4 OH, 5 H2O, 6 HO2, 7 N, 8 NO, 9 N2
"""
import numpy as np

import synth
from synth import ELEMENTARY, THIRD_BODY, LINDEMANN, TROE, SRI, PLOG, CHEB

SP = [(1, 0, 0, 0, 0), (0, 1, 0, 0, 0), (2, 0, 0, 0, 0), (0, 2, 0, 0, 0), (1, 1, 0, 0, 0),
      (2, 1, 0, 0, 0), (1, 2, 0, 0, 0), (0, 0, 0, 1, 0), (0, 1, 0, 1, 0), (0, 0, 0, 2, 0)]
H, O, H2, O2, OH, H2O, HO2, N, NO, N2 = range(10)


def all_kinds(seed=11):
    """Arbitrary (non-physical) parameters; one reaction of every kind."""
    rx = [
        dict(reac=[(H, 1), (O2, 1)], prod=[(OH, 1), (O, 1)], A=2.0e11, beta=-0.3, Ea=15000.0),
        dict(reac=[(O, 1), (H2, 1)], prod=[(OH, 1), (H, 1)], A=4.0e4, beta=2.5, Ea=6000.0, rev=False),
        dict(reac=[(OH, 2)], prod=[(O, 1), (H2O, 1)], A=3.0e1, beta=3.0, Ea=-1500.0),
        dict(reac=[(H, 2)], prod=[(H2, 1)], A=1.5e12, beta=-1.1, kind=THIRD_BODY,
             eff={H2: 0.0, H2O: 0.0}),
        dict(reac=[(H, 1), (OH, 1)], prod=[(H2O, 1)], A=2.0e16, beta=-1.9, kind=THIRD_BODY,
             eff={H2: 0.7, H2O: 3.5}),
        dict(reac=[(H, 1), (O2, 1)], prod=[(HO2, 1)], A=5.0e9, beta=0.4, kind=LINDEMANN,
             A0=6.0e14, beta0=-1.7, Ea0=500.0, eff={H2: 2.0, H2O: 12.0}),
        dict(reac=[(OH, 2)], prod=[(H2, 1), (O2, 1)], A=7.0e10, beta=-0.4, kind=TROE,
             A0=2.0e12, beta0=-0.8, Ea0=-1500.0, troe=(0.7, 90.0, 1800.0, 5000.0),
             eff={H2O: 6.0}),
        dict(reac=[(HO2, 1)], prod=[(H, 1), (O2, 1)], A=5.0e14, beta=0.0, Ea=40000.0, kind=TROE,
             A0=1.0e16, beta0=-1.0, Ea0=30000.0, troe=(0.5, 100.0, 2000.0), eff={H2: 1.5}),
        dict(reac=[(H, 1), (HO2, 1)], prod=[(H2, 1), (O2, 1)], A=2.0e10, beta=0.3, Ea=2000.0,
             kind=SRI, A0=3.0e14, beta0=-1.5, Ea0=1000.0, sri=(0.45, 800.0, 1000.0, 1.1, -0.2),
             eff={O2: 0.4}),
        dict(reac=[(N, 1), (NO, 1)], prod=[(N2, 1), (O, 1)], A=3.0e10, beta=0.0, Ea=400.0),
    ]
    return synth.build_mechanism("tiny_all_kinds", SP, rx, seed=seed)


def bath_efficiency(seed=12):
    """Pressure-dependent reactions where the bath gas has a non-unit efficiency."""
    rx = [
        dict(reac=[(H, 1), (O2, 1)], prod=[(OH, 1), (O, 1)], A=2.0e11, beta=-0.3, Ea=15000.0),
        dict(reac=[(O, 2)], prod=[(O2, 1)], A=6.0e12, beta=-0.5, kind=THIRD_BODY,
             eff={N2: 0.4, H2O: 5.0}),
        dict(reac=[(H, 1), (O2, 1)], prod=[(HO2, 1)], A=5.0e9, beta=0.4, kind=TROE,
             A0=6.0e14, beta0=-1.7, Ea0=500.0, troe=(0.5, 30.0, 90000.0, 90000.0),
             eff={N2: 1.8}),
    ]
    return synth.build_mechanism("tiny_bath_eff", SP, rx, seed=seed)


def all_types(seed=14):
    """One reaction of each less common type next to plain ones:
    chemically-activated falloff (Lindemann, Troe, SRI broadening), P-log
    (three and two pressures, reversible and not), Chebyshev (3 x 2) and
    explicit reverse Arrhenius parameters (elementary and third body)."""
    rx = [
        dict(reac=[(H, 1), (O2, 1)], prod=[(OH, 1), (O, 1)], A=2.0e11, beta=-0.3, Ea=15000.0),
        dict(reac=[(H, 1), (O2, 1)], prod=[(HO2, 1)], A=5.0e9, beta=0.4, kind=LINDEMANN, chem=True,
             A0=6.0e14, beta0=-1.7, Ea0=500.0, eff={H2: 2.0, H2O: 12.0}),
        dict(reac=[(OH, 2)], prod=[(H2O, 1), (O, 1)], A=7.0e10, beta=-0.4, kind=TROE, chem=True,
             A0=2.0e12, beta0=-0.8, Ea0=-1500.0, troe=(0.7, 90.0, 1800.0, 5000.0), eff={H2O: 6.0, N2: 1.4}),
        dict(reac=[(H, 1), (HO2, 1)], prod=[(H2, 1), (O2, 1)], A=2.0e10, beta=0.3, Ea=2000.0, kind=SRI,
             chem=True, A0=3.0e14, beta0=-1.5, Ea0=1000.0, sri=(0.45, 800.0, 1000.0, 1.1, -0.2)),
        dict(reac=[(H, 1), (HO2, 1)], prod=[(OH, 2)], A=1.0, kind=PLOG,
             plog=[(1.0e4, 7.0e10, 0.0, 300.0), (1.0e5, 2.0e11, -0.2, 500.0), (1.0e6, 9.0e11, -0.5, 900.0)]),
        dict(reac=[(O, 1), (H2, 1)], prod=[(OH, 1), (H, 1)], A=1.0, kind=PLOG, rev=False,
             plog=[(3.0e4, 4.0e4, 2.5, 6000.0), (3.0e6, 9.0e4, 2.3, 6500.0)]),
        dict(reac=[(OH, 1), (H2, 1)], prod=[(H2O, 1), (H, 1)], A=1.0, kind=CHEB,
             cheb=dict(T=(300.0, 3000.0), P=(1.0e3, 1.0e7),
                       coef=[[8.0, 0.3], [-0.7, 0.1], [0.05, -0.02]])),
        dict(reac=[(H, 1), (O2, 1)], prod=[(OH, 1), (O, 1)], A=2.0e11, beta=-0.3, Ea=15000.0,
             rev_arr=(1.5e10, 0.1, 800.0)),
        dict(reac=[(H, 2)], prod=[(H2, 1)], A=1.5e12, beta=-1.1, kind=THIRD_BODY, eff={H2: 0.0},
             rev_arr=(3.0e15, -0.5, 100000.0)),
        dict(reac=[(N, 1), (NO, 1)], prod=[(N2, 1), (O, 1)], A=3.0e10, beta=0.0, Ea=400.0),
    ]
    return synth.build_mechanism("tiny_all_types", SP, rx, seed=seed)


def single(reaction, species=None, seed=13):
    return synth.build_mechanism("tiny_single", species or SP, [reaction], seed=seed)


def constant_cp_nasa(ns, cp_R=3.5, a5=None, a6=None):
    """NASA-7 coefficient pairs with constant cp/R (identical ranges)."""
    low = np.zeros((ns, 7))
    low[:, 0] = cp_R
    low[:, 5] = 0.0 if a5 is None else a5
    low[:, 6] = 0.0 if a6 is None else a6
    return low, low.copy()
