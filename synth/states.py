"""Seeded synthetic thermochemical states and workload definitions.

The state vector of Sec. 2.2 is Phi = [T, S, n_1 .. n_{Ns-1}] with S = V for
constant pressure (CONP, P a per-state parameter) and S = P for constant
volume (CONV, V a per-state parameter).  States stand in for the paper's
partially-stirred-reactor databases: T ~ U[600, 2500] K,
P ~ logU[1, 50] atm, mass fractions Y ~ Dirichlet(0.5 * 1_Ns), V = 1 m^3,
n_k = Y_k rho V / W_k with rho = P Wbar / (R T).

Layout: structure of arrays, phi[v, s] for v in [0, Ns], s in [0, n).
Input generation only: no rates, source terms or Jacobians are computed here.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .mechanism import R_GAS, Mechanism

P_ATM = 101325.0
CONP, CONV = 0, 1


def make_states(mech: Mechanism, n: int, seed: int, mode: int = CONP,
                T_range=(600.0, 2500.0), P_atm_range=(1.0, 50.0), alpha=0.5):
    """Return (phi [Ns+1, n] float64, param [n] float64) for the given mode."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ns = mech.n_species
    T = rng.uniform(T_range[0], T_range[1], n)
    P = P_ATM * np.exp(rng.uniform(np.log(P_atm_range[0]), np.log(P_atm_range[1]), n))
    Y = rng.dirichlet(np.full(ns, alpha), size=n)  # [n, ns]
    V = np.ones(n)
    inv_w = Y @ (1.0 / mech.W)                      # sum_k Y_k / W_k  = 1 / Wbar
    ntot = P * V / (R_GAS * T)                       # kmol
    nk = (Y / mech.W[None, :]) * (ntot / inv_w)[:, None]
    phi = np.empty((ns + 1, n))
    phi[0] = T
    phi[1] = V if mode == CONP else P
    phi[2:] = nk[:, : ns - 1].T
    param = P if mode == CONP else V
    return np.ascontiguousarray(phi), np.ascontiguousarray(param)


@dataclass(frozen=True)
class Workload:
    key: str
    mech: str
    n_states: int
    seed: int
    description: str


WORKLOADS = {
    "h2co13_4k": Workload("h2co13_4k", "h2co13", 4096, 2018 + 1,
                          "13 species / 27 reactions, 4096 states, CONP source terms + CSR Jacobian"),
    "gri53_1m": Workload("gri53_1m", "gri53", 1048576, 2018 + 2,
                         "53 species / 325 reactions, 1,048,576 states, CONP+CONV source terms, "
                         "CSR and dense Jacobian"),
    "usc111_256k": Workload("usc111_256k", "usc111", 262144, 2018 + 3,
                            "111 species / 784 reactions, 262,144 states, FP32 Newton matrix"),
    "gri53_vjp64k": Workload("gri53_vjp64k", "gri53", 65536, 2018 + 4,
                             "53 species / 325 reactions, 65,536 states, adjoint VJP"),
    "ic5874_ragged": Workload("ic5874_ragged", "ic5874", 0, 2018 + 5,
                              "874 species / 3796 reactions, 32 ragged batches of 1024..65536 states"),
}


def ragged_batch_sizes(seed: int = 2018 + 5, n_batches: int = 32, lo: int = 1024, hi: int = 65536):
    """Log-uniform batch sizes in [lo, hi] (integers)."""
    rng = np.random.Generator(np.random.PCG64(seed + 1000))
    return np.floor(np.exp(rng.uniform(np.log(lo), np.log(hi + 1), n_batches))).astype(np.int64).clip(lo, hi)


def make_cotangents(ns: int, n: int, seed: int):
    """Random FP64 cotangents N(0,1) for (wdot_0..wdot_{Ns-1}, dT/dt)."""
    rng = np.random.Generator(np.random.PCG64(seed + 77))
    return rng.standard_normal((ns, n)), rng.standard_normal(n)


def make_step_sizes(n: int, seed: int):
    """Per-state implicit step sizes h ~ logU[1e-9, 1e-5] s."""
    rng = np.random.Generator(np.random.PCG64(seed + 99))
    return np.exp(rng.uniform(np.log(1e-9), np.log(1e-5), n))
