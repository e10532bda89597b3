"""CPU oracle: thermochemical source terms and chemical-kinetic Jacobian.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import or call anything in ``oracle/``.
The product path (``paper_1809_01029_gb300``) never imports it and shares no
code with it; both read the same mechanism *data* produced by ``synth``.

Plain, slow, obviously correct: numpy vectorised over states, Python loops
over species and reactions, IEEE float64 (or complex128 for complex-step
differentiation).  Every function names the passage it follows.  The paper's
equation bodies for the state vector, source terms and Jacobian are not in
the available text (Sec. 2.2 loads them from a supplement); the forms written
here are the standard published ones the section names (Sec. 2.2, Sec. 3.4):

* state Phi = [T, S, n_0 .. n_{Ns-2}], S = V (CONP, P fixed) or P (CONV, V
  fixed); the bath gas Ns-1 is implicit through the ideal-gas law (Sec. 2.2);
* production rates wdot_k = sum_i nu_ki R_i c_i (Sec. 2.2, production-rate
  equation);
* dT/dt from the species enthalpies (CONP) or internal energies (CONV), and
  dV/dt or dP/dt by differentiating P V = n R T with explicit mass
  conservation of the bath gas (Sec. 2.2, "volume and pressure source terms");
* Jacobian J_ij = d f_i / d Phi_j (Sec. 2.2, Jacobian arrangement), computed
  here by complex-step differentiation of f, i.e. exactly (to rounding) the
  derivative of the function defined above.

Parity pins (tests/test_oracle_*.py) tie this module to closed forms,
conservation laws, a computed chemical equilibrium and finite differences.
"""
from __future__ import annotations

import numpy as np

# physical constants (SI with kmol)
R = 8314.46261815324          # J / (kmol K)
R_CAL = 1.98720425864083      # cal / (mol K); activation energies are in cal/mol
P_ATM = 101325.0              # Pa, standard-state pressure of the equilibrium constant

CONP, CONV = 0, 1
ELEMENTARY, THIRD_BODY, LINDEMANN, TROE, SRI, PLOG, CHEB = 0, 1, 2, 3, 4, 5, 6
FALLOFF = (LINDEMANN, TROE, SRI)


def _re(x):
    return x.real if np.iscomplexobj(x) else x


# ---------------------------------------------------------------------------
# state -> concentrations (Sec. 2.2: [C]_k = n_k / V, ideal gas P V = n R T)
# ---------------------------------------------------------------------------
def concentrations(mech, mode, phi, param):
    """Return T, V, P, C[Ns, n], Ctot.

    The bath gas concentration is C_tot - sum_{k<Ns-1} C_k with the sum taken
    sequentially in species order (the implicit last species of Sec. 2.2).
    """
    ns = mech.n_species
    T = phi[0]
    if mode == CONP:
        V, P = phi[1], param
    else:
        P, V = phi[1], param
    C = np.empty((ns,) + np.shape(T), dtype=np.result_type(phi, param))
    for k in range(ns - 1):
        C[k] = phi[2 + k] / V
    Ctot = P / (R * T)
    acc = np.zeros_like(C[0])
    for k in range(ns - 1):
        acc = acc + C[k]
    C[ns - 1] = Ctot - acc
    return T, V, P, C, Ctot


# ---------------------------------------------------------------------------
# thermodynamics: NASA 7-coefficient polynomials, high/low range (Sec. 2.1)
# ---------------------------------------------------------------------------
def nasa7(mech, T):
    """cp/R, h/(RT), s/R for every species, shape [Ns, n].

    Low-temperature coefficients are used iff T < T_mid (real part).
    cp/R = a0 + a1 T + a2 T^2 + a3 T^3 + a4 T^4
    h/RT = a0 + a1 T/2 + a2 T^2/3 + a3 T^3/4 + a4 T^4/5 + a5/T
    s/R  = a0 ln T + a1 T + a2 T^2/2 + a3 T^3/3 + a4 T^4/4 + a6
    """
    ns = mech.n_species
    cp = np.empty((ns,) + np.shape(T), dtype=np.result_type(T, 1.0))
    h = np.empty_like(cp)
    s = np.empty_like(cp)
    lnT = np.log(T)
    for k in range(ns):
        low = _re(T) < mech.T_mid[k]
        a = [np.where(low, mech.nasa_low[k, j], mech.nasa_high[k, j]) for j in range(7)]
        cp[k] = a[0] + a[1] * T + a[2] * T ** 2 + a[3] * T ** 3 + a[4] * T ** 4
        h[k] = a[0] + a[1] * T / 2 + a[2] * T ** 2 / 3 + a[3] * T ** 3 / 4 + a[4] * T ** 4 / 5 + a[5] / T
        s[k] = a[0] * lnT + a[1] * T + a[2] * T ** 2 / 2 + a[3] * T ** 3 / 3 + a[4] * T ** 4 / 4 + a[6]
    return cp, h, s


# ---------------------------------------------------------------------------
# reaction rates (Sec. 2.2: R_i, c_i; modified Arrhenius; falloff forms)
# ---------------------------------------------------------------------------
def arrhenius(A, beta, Ea, T):
    """Modified Arrhenius k = A T^beta exp(-Ea / (R_cal T)), Ea in cal/mol,
    written in its logarithmic form exp(ln A + beta ln T - Ea / (R_cal T))."""
    return np.exp(np.log(A) + beta * np.log(T) - Ea / (R_CAL * T))


def net_stoich(mech):
    """nu[k, i] = nu''_ki - nu'_ki as a dense integer matrix [Ns, Nr]."""
    nu = np.zeros((mech.n_species, mech.n_reactions), dtype=np.int64)
    for i in range(mech.n_reactions):
        for k, v in mech.reactants(i):
            nu[k, i] -= v
        for k, v in mech.products(i):
            nu[k, i] += v
    return nu


def third_body_alpha(mech, i):
    """Dense efficiency vector alpha[k] of reaction i (default 1)."""
    a = np.ones(mech.n_species)
    for k, v in mech.efficiencies(i).items():
        a[k] = v
    return a


def troe_F(mech, i, T, Pr):
    """Troe broadening factor (Gilbert, Luther & Troe 1983)."""
    a, T3, T1, T2 = mech.troe[i]
    Fcent = (1 - a) * np.exp(-T / T3) + a * np.exp(-T / T1)
    if mech.troe_n[i] == 4:
        Fcent = Fcent + np.exp(-T2 / T)
    lF = np.log10(Fcent)
    c = -0.4 - 0.67 * lF
    N = 0.75 - 1.27 * lF
    x = np.log10(Pr)
    f1 = (x + c) / (N - 0.14 * (x + c))
    return 10.0 ** (lF / (1 + f1 * f1))


def sri_F(mech, i, T, Pr):
    """SRI broadening factor (Stewart, Larson & Golden 1989)."""
    a, b, c, d, e = mech.sri[i]
    x = np.log10(Pr)
    X = 1.0 / (1.0 + x * x)
    return d * (a * np.exp(-b / T) + np.exp(-T / c)) ** X * T ** e


def plog_lnk(mech, i, T, P):
    """ln k of a P-log reaction: the Arrhenius rates tabulated at pressures
    P_1 < .. < P_n, interpolated linearly in ln P between neighbours and held
    at the end values below P_1 and from P_n on.  Segment m covers
    [P_m, P_m+1), chosen by the real part of ln P."""
    tab = mech.plog_table(i)
    lnT = np.log(T)
    lnks = [np.log(A) + b * lnT - Ea / (R_CAL * T) for _, A, b, Ea in tab]
    lnPs = np.log(tab[:, 0])
    x = np.log(P)
    xr = _re(x) * np.ones(np.shape(T))
    out = lnks[0] * np.ones(np.shape(T), dtype=np.result_type(lnks[0], x))
    for m in range(len(tab) - 1):
        inside = (xr >= lnPs[m]) & (xr < lnPs[m + 1])
        w = (x - lnPs[m]) / (lnPs[m + 1] - lnPs[m])
        out = np.where(inside, lnks[m] + (lnks[m + 1] - lnks[m]) * w, out)
    return np.where(xr >= lnPs[-1], lnks[-1], out)


def cheb_log10k(mech, i, T, P):
    """log10 k of a Chebyshev reaction: sum_t sum_p a_tp phi_t(T~) phi_p(P~),
    phi_n the Chebyshev polynomials of the first kind (phi_0 = 1, phi_1 = x,
    phi_n = 2 x phi_{n-1} - phi_{n-2}), T~ = (2/T - 1/T_min - 1/T_max) /
    (1/T_max - 1/T_min), P~ = (2 log10 P - log10 P_min - log10 P_max) /
    (log10 P_max - log10 P_min)."""
    Tmin, Tmax, Pmin, Pmax = mech.cheb_range[i]
    a = mech.cheb_table(i)
    Tt = (2.0 / T - 1.0 / Tmin - 1.0 / Tmax) / (1.0 / Tmax - 1.0 / Tmin)
    Pt = (2.0 * np.log10(P) - np.log10(Pmin) - np.log10(Pmax)) / (np.log10(Pmax) - np.log10(Pmin))

    def basis(x, n):
        ph = [np.ones_like(x), x]
        while len(ph) < n:
            ph.append(2.0 * x * ph[-1] - ph[-2])
        return ph[:n]
    pt, pp = basis(Tt, a.shape[0]), basis(Pt * np.ones_like(Tt), a.shape[1])
    return sum(a[t, q] * pt[t] * pp[q] for t in range(a.shape[0]) for q in range(a.shape[1]))


def rates(mech, mode, phi, param, A=None, beta=None, Ea=None, dC=None, freeze_bath=False):
    """All intermediate quantities of the source-term evaluation.

    Returns a dict with T, V, P, C, Ctot, cp, h, s (NASA-7 forms), kf, kr,
    c (pressure modification), Rf = kf prod C^nu', Rr = kr prod C^nu'',
    qf = c Rf, qr = c Rr, q = qf - qr, wdot [Ns, n].

    A, beta, Ea optionally override the high-pressure (or only) Arrhenius
    parameters (used to differentiate with respect to them); dC is added to
    the concentrations after they are formed (used to differentiate with
    respect to a single concentration).

    freeze_bath=True gives the rates behind the approximate Jacobian
    (Sec. 3.4, "Sparsity patterns"): the values are unchanged, but the rates
    of progress see the bath gas through Re(C_Ns) only, and the third-body
    concentration is [M] = C_tot + sum_k (alpha_k - 1) C_rate,k, C_rate being
    C with Re(C_Ns) in the bath-gas slot (equal to alpha . C_rate + (C_Ns -
    Re C_Ns)): a perturbation of C_Ns enters [M] with unit efficiency.  Under a complex-step perturbation of a species amount
    n_j (C_tot real) the rates of progress then see no change of C_Ns and
    d[M]/dn_j = (alpha_j - 1)/V instead of (alpha_j - alpha_Ns)/V.
    """
    A = mech.A if A is None else A
    beta = mech.beta if beta is None else beta
    Ea = mech.Ea if Ea is None else Ea
    T, V, P, C, Ctot = concentrations(mech, mode, phi, param)
    if dC is not None:
        C = C + dC
    Cr = C                                      # concentrations seen by the rates of progress
    if freeze_bath:
        Cr = C.copy()
        Cr[-1] = _re(C[-1])
    cp, h, s = nasa7(mech, T)
    g = h - s                                   # g/RT
    nu = net_stoich(mech)
    nr, ns = mech.n_reactions, mech.n_species
    shape = (nr,) + np.shape(T)
    dt = np.result_type(C, A, beta, Ea)
    kf = np.empty(shape, dtype=dt)
    kr = np.empty(shape, dtype=dt)
    cmod = np.empty(shape, dtype=dt)
    Rf = np.empty(shape, dtype=dt)
    Rr = np.empty(shape, dtype=dt)
    for i in range(nr):
        kind = mech.kind[i]
        chem = kind in FALLOFF and bool(mech.chem[i])
        if kind == PLOG:
            kf[i] = np.exp(plog_lnk(mech, i, T, P))
        elif kind == CHEB:
            kf[i] = 10.0 ** cheb_log10k(mech, i, T, P)
        elif chem:                               # chemically activated: base rate k0
            kf[i] = arrhenius(mech.A0[i], mech.beta0[i], mech.Ea0[i], T)
        else:
            kf[i] = arrhenius(A[i], beta[i], Ea[i], T)
        if mech.reversible[i] and mech.rev_explicit[i]:
            kr[i] = arrhenius(*mech.rev_arr[i], T)
        elif mech.reversible[i]:
            # K_c = exp(-sum_k nu_k g_k/RT + (sum_k nu_k) ln(P_atm / RT)),
            # k_r = k_f / K_c = k_f exp(-ln K_c)
            dg = sum(nu[k, i] * g[k] for k in range(ns) if nu[k, i] != 0)
            dn = float(nu[:, i].sum())
            lnKc = -dg + dn * np.log(P_ATM / (R * T))
            kr[i] = kf[i] * np.exp(-lnKc)
        else:
            kr[i] = 0.0
        if kind in (ELEMENTARY, PLOG, CHEB):
            cmod[i] = 1.0
        else:
            # [M] = sum_k alpha_k C_k written as C_tot + sum_k (alpha_k - 1) C_k
            # (sum_k C_k = C_tot): only non-default efficiencies enter the sum.
            # With freeze_bath the rates see Re(C_Ns), and C_tot carries the
            # perturbation of C_Ns with unit efficiency.
            alpha = third_body_alpha(mech, i)
            M = Ctot * np.ones(np.shape(T))
            for k in range(ns):
                if alpha[k] != 1.0:
                    M = M + (alpha[k] - 1.0) * Cr[k]
            if kind == THIRD_BODY:
                cmod[i] = M
            else:
                k0 = arrhenius(mech.A0[i], mech.beta0[i], mech.Ea0[i], T)
                kinf = arrhenius(A[i], beta[i], Ea[i], T)
                Pr = k0 * M / kinf
                if kind == LINDEMANN:
                    F = 1.0
                elif kind == TROE:
                    F = troe_F(mech, i, T, Pr)
                else:
                    F = sri_F(mech, i, T, Pr)
                if chem:
                    # chemically activated: k = k0 F / (1 + Pr)
                    cmod[i] = F / (1 + Pr)
                else:
                    # Pr/(1+Pr) written as 1/(1+1/Pr): the same function, but
                    # its complex-step derivative avoids the cancellation
                    # (1+Pr) dPr - Pr dPr that loses digits for large Pr
                    cmod[i] = F / (1 + 1 / Pr)
        fwd = kf[i]
        for k, v in mech.reactants(i):
            fwd = fwd * Cr[k] ** v
        rev = kr[i]
        for k, v in mech.products(i):
            rev = rev * Cr[k] ** v
        Rf[i], Rr[i] = fwd, rev
    qf = cmod * Rf
    qr = cmod * Rr
    q = qf - qr
    wdot = np.zeros((ns,) + np.shape(T), dtype=dt)
    for i in range(nr):
        for k in range(ns):
            if nu[k, i] != 0:
                wdot[k] = wdot[k] + nu[k, i] * q[i]
    return dict(T=T, V=V, P=P, C=C, Ctot=Ctot, cp=cp, h=h, s=s, kf=kf, kr=kr, c=cmod,
                Rf=Rf, Rr=Rr, qf=qf, qr=qr, q=q, wdot=wdot, nu=nu)


def source_terms_from_rates(mech, mode, r):
    """f = [dT/dt, dS/dt, dn_0/dt .. dn_{Ns-2}/dt] (Sec. 2.2).

    CONP: dT/dt = -sum_k H_k wdot_k / sum_k C_k Cp_k,
          dV/dt = V dT/dt / T + (R T V / P) sum_{k<Ns-1} (1 - W_k/W_Ns) wdot_k
    CONV: dT/dt = -sum_k U_k wdot_k / sum_k C_k Cv_k,
          dP/dt = P dT/dt / T + R T sum_{k<Ns-1} (1 - W_k/W_Ns) wdot_k
    dn_k/dt = V wdot_k.  Sums over k run over all species, bath gas included.
    """
    ns = mech.n_species
    T, V, P, C, wdot = r["T"], r["V"], r["P"], r["C"], r["wdot"]
    if mode == CONP:
        E = R * T * r["h"]             # molar enthalpy H_k
        Cx = R * r["cp"]               # molar Cp_k
    else:
        E = R * T * (r["h"] - 1.0)     # molar internal energy U_k = H_k - R T
        Cx = R * (r["cp"] - 1.0)       # molar Cv_k = Cp_k - R
    num = sum(E[k] * wdot[k] for k in range(ns))
    den = sum(C[k] * Cx[k] for k in range(ns))
    Tdot = -num / den
    Om = sum((1.0 - mech.W[k] / mech.W[ns - 1]) * wdot[k] for k in range(ns - 1))
    f = np.empty((ns + 1,) + np.shape(T), dtype=wdot.dtype)
    f[0] = Tdot
    if mode == CONP:
        f[1] = V * Tdot / T + (R * T * V / P) * Om
    else:
        f[1] = P * Tdot / T + R * T * Om
    for k in range(ns - 1):
        f[2 + k] = V * wdot[k]
    return f, dict(E=E, Cx=Cx, num=num, den=den, Om=Om)


def source_terms(mech, mode, phi, param):
    """dPhi/dt for every state: array [Ns+1, n] (Sec. 2.2)."""
    r = rates(mech, mode, phi, param)
    return source_terms_from_rates(mech, mode, r)[0]


# ---------------------------------------------------------------------------
# Jacobian by complex-step differentiation (definition J_ij = df_i/dPhi_j)
# ---------------------------------------------------------------------------
def _cs_step(x):
    return 1e-30 * np.maximum(np.abs(x), 1.0)


EXACT, APPROX = "exact", "approx"


def _cs_columns(task):
    """Complex-step derivatives of f, of the forward / reverse parts and of
    the energy-equation denominator for the state columns `cols` (one task of
    jacobian's map), in the complex type matching phi's precision."""
    mech, mode, phi, param, cols, form = task
    ctype = np.clongdouble if phi.dtype == np.longdouble else np.complex128
    out = []
    for j in cols:
        ph = phi.astype(ctype)
        hj = _cs_step(phi[j])
        ph[j] = ph[j] + 1j * hj
        r = rates(mech, mode, ph, param.astype(ctype), freeze_bath=(form == APPROX and j >= 2))
        f, aux = source_terms_from_rates(mech, mode, r)
        out.append((f.imag / hj, r["qf"].imag / hj, r["qr"].imag / hj, aux["den"].imag / hj))
    return out


def _chunks(items, k):
    """items split into at most k contiguous, nearly equal runs."""
    k = max(1, min(k, len(items)))
    q, r = divmod(len(items), k)
    out, lo = [], 0
    for c in range(k):
        hi = lo + q + (c < r)
        out.append(items[lo:hi])
        lo = hi
    return out


def jacobian(mech, mode, phi, param, with_parts=False, form=EXACT, map_fn=map, chunks=1):
    """Dense Jacobian [Ns+1, Ns+1, n] of f with P (CONP) or V (CONV) fixed.

    Column j is Im f(Phi + i h e_j) / h with h = 1e-30 max(|Phi_j|, 1):
    complex-step differentiation, which carries no subtractive cancellation
    and equals the analytic derivative to rounding (the NASA-7 range choice
    follows the real part of T).
    With with_parts=True also returns the complex-step derivatives of the
    forward/reverse parts (qf, qr), of the energy-equation denominator and the
    values needed to bound rounding of a correct FP64 implementation.

    form=APPROX gives the approximate Jacobian of Sec. 3.4 ("Sparsity
    patterns"): in the species columns the derivatives that reach the rates
    of progress through the bath-gas concentration C_Ns = C_tot - sum C_k, and
    the pressure-modification derivatives that a non-unit bath-gas
    efficiency spreads over every species, are left out (rates(freeze_bath=
    True)).  The T and S columns, and every other use of C_Ns (the heat
    capacity of the mixture), stay exact.

    The columns are independent: map_fn (a parallel map, e.g. a process
    pool's) may evaluate them in `chunks` groups; the result is the same.
    With phi and param in np.longdouble the whole evaluation runs in that
    type (the extended-precision reference of the FP64 oracle).
    """
    if form not in (EXACT, APPROX):
        raise ValueError(f"unknown Jacobian form {form!r}")
    N = mech.n_species + 1
    n = phi.shape[1]
    rt = np.longdouble if phi.dtype == np.longdouble else np.float64
    J = np.empty((N, N, n), dtype=rt)
    parts = dict(dqf=np.empty((mech.n_reactions, N, n), dtype=rt), dqr=np.empty((mech.n_reactions, N, n), dtype=rt),
                 dden=np.empty((N, n), dtype=rt))
    groups = _chunks(list(range(N)), chunks)
    for cols, res in zip(groups, map_fn(_cs_columns, [(mech, mode, phi, param, c, form) for c in groups])):
        for j, (df, dqf, dqr, dden) in zip(cols, res):
            J[:, j] = df
            if with_parts:
                parts["dqf"][:, j] = dqf
                parts["dqr"][:, j] = dqr
                parts["dden"][j] = dden
    if with_parts:
        return J, parts
    return J


def jacobian_columns(mech, mode, phi, param, cols, form=EXACT):
    """Selected Jacobian columns [N, len(cols), n] by complex step (for large
    mechanisms where the full Jacobian is too slow for the oracle)."""
    N = mech.n_species + 1
    out = np.empty((N, len(cols), phi.shape[1]))
    for c, j in enumerate(cols):
        ph = phi.astype(np.complex128)
        hj = _cs_step(phi[j])
        ph[j] = ph[j] + 1j * hj
        r = rates(mech, mode, ph, param.astype(np.complex128), freeze_bath=(form == APPROX and j >= 2))
        out[:, c] = source_terms_from_rates(mech, mode, r)[0].imag / hj
    return out


# ---------------------------------------------------------------------------
# rounding envelopes for a conditioning-aware comparison (Sec. 3.2: net rates
# of progress lose accuracy where forward and reverse rates nearly cancel)
# ---------------------------------------------------------------------------
def source_term_envelope(mech, mode, phi, param):
    """Absolute envelope env[Ns+1, n]: the sum of magnitudes of the terms that
    make up each source term, so that a correct FP64 evaluation differs from
    another by at most a small multiple of u * env."""
    r = rates(mech, mode, phi, param)
    f, aux = source_terms_from_rates(mech, mode, r)
    ns = mech.n_species
    nu = r["nu"]
    ew = np.zeros_like(r["wdot"])
    for i in range(mech.n_reactions):
        t = np.abs(r["qf"][i]) + np.abs(r["qr"][i])
        for k in range(ns):
            if nu[k, i] != 0:
                ew[k] += abs(nu[k, i]) * t
    T, V, P = r["T"], r["V"], r["P"]
    den = np.abs(aux["den"])
    eT = sum(np.abs(aux["E"][k]) * ew[k] for k in range(ns)) / den
    eO = sum(abs(1.0 - mech.W[k] / mech.W[ns - 1]) * ew[k] for k in range(ns - 1))
    env = np.empty_like(f)
    env[0] = eT + np.abs(f[0])
    if mode == CONP:
        env[1] = V * env[0] / T + (R * T * V / P) * eO
    else:
        env[1] = P * env[0] / T + R * T * eO
    for k in range(ns - 1):
        env[2 + k] = V * ew[k]
    return f, np.maximum(env, np.abs(f))


def _dC_columns(task):
    """|dq'/dC_k| + |dq''/dC_k| per reaction for the species `species`, by
    complex step in C_k alone (one task of jacobian_envelope's map)."""
    mech, mode, phi, param, species = task
    ns = mech.n_species
    shape = (phi.shape[1],)
    _, _, _, C, _ = concentrations(mech, mode, phi, param)
    out = []
    for k in species:
        hk = 1e-30 * np.maximum(np.abs(C[k]), 1e-200)
        dC = np.zeros((ns,) + shape, dtype=np.complex128)
        dC[k] = 1j * hk
        rk = rates(mech, mode, phi.astype(np.complex128), param.astype(np.complex128), dC=dC)
        out.append((np.abs(rk["qf"].imag) + np.abs(rk["qr"].imag)) / hk)
    return out


def jacobian_envelope(mech, mode, phi, param, map_fn=map, chunks=1):
    """Jacobian J [N, N, n] and an absolute envelope of equal shape (map_fn,
    chunks: as for jacobian).

    Per reaction, the envelope of d q_i / d Phi_j sums the magnitudes of the
    forward and reverse parts and of the paths through the bath-gas
    concentration (which can cancel a species' own term):
      species columns: (|dqf/dC_j| + |dqr/dC_j| + |dqf/dC_b| + |dqr/dC_b|) / V
      T, S columns:    |dqf/dPhi| + |dqr/dPhi| + (|dqf/dC_b| + |dqr/dC_b|) |dC_b/dPhi|
                       (+ sum_k (|dqf/dC_k| + |dqr/dC_k|) C_k / V for V in CONP)
    Species rows combine these with |nu_ki|; energy / state rows follow the
    structure of the source terms.
    """
    J, parts = jacobian(mech, mode, phi, param, with_parts=True, map_fn=map_fn, chunks=chunks)
    r = rates(mech, mode, phi, param)
    f, aux = source_terms_from_rates(mech, mode, r)
    _, envf = source_term_envelope(mech, mode, phi, param)
    ns, N, nr = mech.n_species, mech.n_species + 1, mech.n_reactions
    nu = r["nu"]
    T, V, P, C, Ctot = r["T"], r["V"], r["P"], r["C"], r["Ctot"]
    shape = np.shape(T)
    # complex-step derivatives of the forward / reverse parts w.r.t. each C_k
    dC_mag = np.empty((nr, ns) + shape)
    groups = _chunks(list(range(ns)), chunks)
    for ks, res in zip(groups, map_fn(_dC_columns, [(mech, mode, phi, param, g) for g in groups])):
        for k, mag in zip(ks, res):
            dC_mag[:, k] = mag
    bath = dC_mag[:, ns - 1]                                   # [Nr, n]
    eq = np.empty((nr, N) + shape)                             # per-reaction envelope of dq_i/dPhi_j
    eq[:, 0] = np.abs(parts["dqf"][:, 0]) + np.abs(parts["dqr"][:, 0]) + bath * Ctot / T
    if mode == CONP:
        dCb_S = (Ctot - C[ns - 1]) / V
        eq[:, 1] = np.abs(parts["dqf"][:, 1]) + np.abs(parts["dqr"][:, 1]) + bath * np.abs(dCb_S)
        eq[:, 1] += sum(dC_mag[:, k] * np.abs(C[k]) for k in range(ns - 1)) / V
    else:
        eq[:, 1] = np.abs(parts["dqf"][:, 1]) + np.abs(parts["dqr"][:, 1]) + bath * Ctot / P
    for j in range(ns - 1):
        eq[:, 2 + j] = (dC_mag[:, j] + bath) / V
    ew = np.zeros((ns, N) + shape)
    ew_all = np.zeros((ns,) + shape)
    for i in range(nr):
        t = np.abs(r["qf"][i]) + np.abs(r["qr"][i])
        for k in range(ns):
            if nu[k, i] != 0:
                ew[k] += abs(nu[k, i]) * eq[i]
                ew_all[k] += abs(nu[k, i]) * t
    env = np.zeros_like(J)
    wd_env = envf[2:] / V
    for k in range(ns - 1):
        env[2 + k] = V * ew[k]
        if mode == CONP:
            env[2 + k, 1] += wd_env[k]
    den = np.abs(aux["den"])
    Tdot = f[0]
    eT = sum(np.abs(aux["E"][k]) * ew[k] for k in range(ns))      # [N, n]
    eT[0] += sum(np.abs(aux["Cx"][k]) * ew_all[k] for k in range(ns))
    eT += (np.abs(Tdot) + envf[0]) * np.abs(parts["dden"])
    env[0] = eT / den
    eO = sum(abs(1.0 - mech.W[k] / mech.W[ns - 1]) * ew[k] for k in range(ns - 1))
    eO0 = sum(abs(1.0 - mech.W[k] / mech.W[ns - 1]) * ew_all[k] for k in range(ns - 1))
    if mode == CONP:
        env[1] = (V / T) * env[0] + (R * T * V / P) * eO
        env[1, 0] += V / T ** 2 * (np.abs(Tdot) + envf[0]) + R * V / P * eO0
        env[1, 1] += (np.abs(Tdot) + envf[0]) / T + R * T / P * eO0
    else:
        env[1] = (P / T) * env[0] + R * T * eO
        env[1, 0] += P / T ** 2 * (np.abs(Tdot) + envf[0]) + R * eO0
        env[1, 1] += (np.abs(Tdot) + envf[0]) / T
    return J, np.maximum(env, np.abs(J))


# ---------------------------------------------------------------------------
# sparsity pattern (Sec. 3.4)
# ---------------------------------------------------------------------------
def dependence_set(mech, i, form=EXACT):
    """Species j < Ns-1 on which the rate of progress of reaction i depends.

    Reactants; products if reversible; for third-body / falloff reactions the
    species whose efficiency differs from the bath gas's; and every species
    when the bath gas takes part in the rate (as a reactant, as a product of a
    reversible reaction) or has a non-unit efficiency (Sec. 3.4).
    For the approximate form (Sec. 3.4) the last clause is dropped and the
    efficiencies are compared with the default 1 instead of the bath gas's.
    """
    ns = mech.n_species
    bath = ns - 1
    dep = set()
    members = [k for k, _ in mech.reactants(i)]
    if mech.reversible[i]:
        members += [k for k, _ in mech.products(i)]
    dep.update(k for k in members if k != bath)
    dense = bath in members
    if mech.kind[i] in (THIRD_BODY,) + FALLOFF:
        a = third_body_alpha(mech, i)
        ref = 1.0 if form == APPROX else a[bath]
        dep.update(k for k in range(ns - 1) if a[k] != ref)
        if a[bath] != 1.0:
            dense = True
    if dense and form != APPROX:
        dep.update(range(ns - 1))
    return dep


def sparsity_pattern(mech, form=EXACT):
    """Boolean mask [N, N] of the Jacobian's structural nonzeros.

    Rows/columns 0 (T) and 1 (V or P) are dense and the diagonal is kept; a
    species row k has column j when some reaction changes k (nu_ki != 0) and
    its rate depends on j (Sec. 3.4; for form=APPROX the dependence of
    Sec. 3.4's approximate form).  Identical for CONP and CONV.
    """
    ns, N = mech.n_species, mech.n_species + 1
    nu = net_stoich(mech)
    mask = np.zeros((N, N), dtype=bool)
    mask[0, :] = mask[1, :] = True
    mask[:, 0] = mask[:, 1] = True
    mask[np.arange(N), np.arange(N)] = True
    for i in range(mech.n_reactions):
        dep = dependence_set(mech, i, form)
        for k in range(ns - 1):
            if nu[k, i] != 0:
                for j in dep:
                    mask[2 + k, 2 + j] = True
    return mask


def csr_pattern(mech, form=EXACT):
    """(row_ptr [N+1], col_idx [nnz]) with columns ascending in each row."""
    mask = sparsity_pattern(mech, form)
    N = mask.shape[0]
    row_ptr = np.zeros(N + 1, dtype=np.int32)
    cols = []
    for i in range(N):
        c = [j for j in range(N) if mask[i, j]]
        cols += c
        row_ptr[i + 1] = row_ptr[i] + len(c)
    return row_ptr, np.array(cols, dtype=np.int32)


def csc_pattern(mech, form=EXACT):
    """(col_ptr [N+1], row_idx [nnz]) with rows ascending in each column."""
    mask = sparsity_pattern(mech, form)
    N = mask.shape[0]
    col_ptr = np.zeros(N + 1, dtype=np.int32)
    rows = []
    for j in range(N):
        r = [i for i in range(N) if mask[i, j]]
        rows += r
        col_ptr[j + 1] = col_ptr[j] + len(r)
    return col_ptr, np.array(rows, dtype=np.int32)


def dense_to_csr_values(mech, J, form=EXACT):
    """Values [nnz, n] of a dense Jacobian stack in CSR order."""
    row_ptr, col = csr_pattern(mech, form)
    rows = np.repeat(np.arange(len(row_ptr) - 1), np.diff(row_ptr))
    return J[rows, col]


def dense_to_csc_values(mech, J, form=EXACT):
    col_ptr, row = csc_pattern(mech, form)
    cols = np.repeat(np.arange(len(col_ptr) - 1), np.diff(col_ptr))
    return J[row, cols]
