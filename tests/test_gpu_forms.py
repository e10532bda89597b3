"""GPU parity of the derived forms: FP32 Newton matrix (precision form) and
the adjoint VJP with its torch.autograd.Function (differentiation form)."""
import numpy as np
import pytest

import oracle
import synth
from tests import tiny_mechs as tm
from tests.parity import RTOL_SRC, ATOL_SRC, check_close, y_envelope, newton_tol

pytestmark = pytest.mark.gpu

# stated accuracy of the FP32 Newton matrix against the FP64 oracle: per
# entry tests/parity.py's newton_tol; per state
NEWTON_FRO = 1e-6       # ||dM||_F <= 1e-6 ||M||_F per state
RTOL_VJP = 1e-8         # per output, relative to the envelope sum |u dy/dx|


@pytest.fixture(scope="module")
def pj():
    import paper_1809_01029_gb300 as pj
    from paper_1809_01029_gb300 import build
    build.build()
    pj.load_library()
    return pj


def _mech(mechs, name):
    if name in ("all_kinds", "bath_efficiency", "all_types"):
        return getattr(tm, name)()
    return mechs(name)


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("mode", [synth.CONP, synth.CONV])
@pytest.mark.parametrize("name,n,gamma", [("all_kinds", 40, 1.0), ("all_types", 35, 1.0), ("gri53", 48, 0.5),
                                           ("gri53_types", 40, 1.0), ("usc111", 16, 1.0)])
def test_newton_matrix_f32_against_fp64_oracle(pj, mechs, name, n, gamma, mode):
    import torch
    m = _mech(mechs, name)
    h = pj.pj_mech_create(m)
    phi, par = synth.make_states(m, n, 600 + n, mode)
    hs = synth.make_step_sizes(n, 600 + n)
    J, env = oracle.jacobian_envelope(m, mode, phi, par)
    N1 = m.n_species + 1
    M_ref = -(hs * gamma)[None, None, :] * J
    M_ref[np.arange(N1), np.arange(N1)] += 1.0
    scale = np.abs(M_ref) + (hs * gamma)[None, None, :] * env
    # the FP32 form's accuracy holds for states whose Newton matrix stays well
    # inside FP32's range (the tiny all-types mechanism's unphysical
    # thermochemistry drives some entries past 1e40)
    keep = ((hs * gamma)[None, None, :] * env).max(axis=(0, 1)) < 1e30
    assert keep.sum() >= n // 4
    sel = np.flatnonzero(keep)
    phi, par, hs, J, env, M_ref, scale = (phi[:, sel], par[sel], hs[sel], J[..., sel], env[..., sel],
                                          M_ref[..., sel], scale[..., sel])
    n = len(sel)
    f_ref, f_env = oracle.source_term_envelope(m, mode, phi, par)
    d_phi, d_par, d_h = dev(phi), dev(par), dev(hs)
    dphi = torch.empty((N1, n), dtype=torch.float64, device="cuda")
    Md = pj.newton_matrix_f32(h, mode, d_phi, d_par, d_h, gamma, fmt=pj.PJ_DENSE, dphi=dphi)
    assert Md.dtype == torch.float32
    Md = Md.cpu().numpy().astype(np.float64).reshape(N1, N1, n)
    err = np.abs(Md - M_ref)
    assert np.all(err <= newton_tol(scale)), float(np.max(err / newton_tol(scale)))
    fro = np.linalg.norm((Md - M_ref).reshape(-1, n), axis=0) / np.linalg.norm(M_ref.reshape(-1, n), axis=0)
    assert np.all(fro <= NEWTON_FRO), float(fro.max())
    check_close(dphi.cpu().numpy(), f_ref, f_env, RTOL_SRC, ATOL_SRC, "FP64 source terms of the Newton kernel")
    for fmt, conv in ((pj.PJ_CSR, oracle.dense_to_csr_values), (pj.PJ_CSC, oracle.dense_to_csc_values)):
        Ms = pj.newton_matrix_f32(h, mode, d_phi, d_par, d_h, gamma, fmt=fmt).cpu().numpy().astype(np.float64)
        e = np.abs(Ms - conv(m, M_ref))
        assert np.all(e <= newton_tol(conv(m, scale))), (fmt, float(np.max(e / newton_tol(conv(m, scale)))))


@pytest.mark.parametrize("mode", [synth.CONP, synth.CONV])
@pytest.mark.parametrize("name,n", [("all_kinds", 45), ("bath_efficiency", 33), ("all_types", 39), ("h2co13", 100), ("gri53", 70),
                                     ("gri53_types", 50)])
def test_vjp_against_oracle(pj, mechs, name, n, mode):
    m = _mech(mechs, name)
    h = pj.pj_mech_create(m)
    phi, par = synth.make_states(m, n, 700 + n, mode)
    uw, uT = synth.make_cotangents(m.n_species, n, 700 + n)
    y, g_phi, g_th = pj.vjp(h, mode, dev(phi), dev(par), dev(uw), dev(uT))
    y_ref = oracle.outputs_y(m, mode, phi, par)
    check_close(y.cpu().numpy(), y_ref, y_envelope(m, mode, phi, par), RTOL_SRC, ATOL_SRC, f"{name} y")
    g_ref, th_ref = oracle.vjp(m, mode, phi, par, uw, uT)
    e_phi, e_th = oracle.vjp_envelope(m, mode, phi, par, uw, uT)
    check_close(g_phi.cpu().numpy(), g_ref, e_phi, RTOL_VJP, 1e-300, f"{name} g_phi")
    check_close(g_th.cpu().numpy(), th_ref, e_th, RTOL_VJP, 1e-300, f"{name} g_theta")
    y2 = pj.eval_y(h, mode, dev(phi), dev(par)).cpu().numpy()
    check_close(y2, y_ref, y_envelope(m, mode, phi, par), RTOL_SRC, ATOL_SRC, f"{name} eval_y")


def test_vjp_deterministic_and_ragged(pj, mechs):
    m = mechs("gri53")
    h = pj.pj_mech_create(m)
    n = 1000 + 37
    phi, par = synth.make_states(m, n, 9, synth.CONP)
    uw, uT = synth.make_cotangents(m.n_species, n, 9)
    a = pj.vjp(h, synth.CONP, dev(phi), dev(par), dev(uw), dev(uT))
    b = pj.vjp(h, synth.CONP, dev(phi), dev(par), dev(uw), dev(uT))
    for x, z in zip(a, b):
        assert np.array_equal(x.cpu().numpy(), z.cpu().numpy())
    # sum over states equals the sum of two halves' gradients (to rounding)
    h1 = pj.vjp(h, synth.CONP, dev(phi[:, :500]), dev(par[:500]), dev(uw[:, :500]), dev(uT[:500]))[2]
    h2 = pj.vjp(h, synth.CONP, dev(phi[:, 500:]), dev(par[500:]), dev(uw[:, 500:]), dev(uT[500:]))[2]
    tot = (h1 + h2).cpu().numpy()
    ref = a[2].cpu().numpy()
    assert np.allclose(tot, ref, rtol=1e-9, atol=1e-9 * np.abs(ref).max())


def test_autograd_function_matches_finite_differences(pj, mechs):
    """Central differences (relative step 1e-6) of u.y through the GPU forward
    pass against the autograd backward, for the state and for parameters."""
    import torch
    m = mechs("gri53")
    h = pj.pj_mech_create(m)
    n = 8
    phi, par = synth.make_states(m, n, 21, synth.CONP, alpha=5.0)
    uw, uT = synth.make_cotangents(m.n_species, n, 21)
    u = np.concatenate([uw, uT[None, :]], axis=0)
    theta = pj.arrhenius_parameters(m).cuda().requires_grad_(True)
    d_phi = dev(phi).requires_grad_(True)
    y = pj.source_terms_y(h, synth.CONP, d_phi, dev(par), theta)
    (y * dev(u)).sum().backward()
    g_phi = d_phi.grad.cpu().numpy()
    g_th = theta.grad.cpu().numpy()
    d_par = dev(par)

    def uy(p_np):
        return float((pj.eval_y(h, synth.CONP, dev(p_np), d_par).cpu().numpy() * u).sum(axis=0).sum())

    e_phi, e_th = oracle.vjp_envelope(m, synth.CONP, phi, par, uw, uT)
    _, fenv = oracle.source_term_envelope(m, synth.CONP, phi, par)
    for j in (0, 1, 2, 5, 20, m.n_species):
        for s in range(n):
            hh = 1e-6 * abs(phi[j, s])
            p1, p2 = phi.copy(), phi.copy()
            p1[j, s] += hh
            p2[j, s] -= hh
            fd = (uy(p1) - uy(p2)) / (2 * hh)
            tol = 1e-4 * e_phi[j, s] + 1e-10 * np.sum(np.abs(u) * y_envelope(m, synth.CONP, phi, par)) / hh
            assert abs(fd - g_phi[j, s]) <= tol, (j, s, fd, g_phi[j, s])
    # parameters: perturb one reaction's ln A / beta / Ea in a new mechanism
    for i in (0, 7, int(np.flatnonzero(m.kind == synth.TROE)[0])):
        for p, (field, rel) in enumerate((("A", None), ("beta", 1e-6), ("Ea", 1e-6))):
            vals = []
            for sign in (1, -1):
                mm = m.copy()
                if field == "A":
                    mm.A = m.A.copy()
                    mm.A[i] = m.A[i] * np.exp(sign * 1e-6)
                    step = 1e-6
                else:
                    arr = getattr(m, field).copy()
                    step = rel * max(abs(arr[i]), 1.0)
                    arr[i] += sign * step
                    setattr(mm, field, arr)
                hm = pj.pj_mech_create(mm)
                vals.append(float((pj.eval_y(hm, synth.CONP, dev(phi), d_par).cpu().numpy() * u).sum()))
            fd = (vals[0] - vals[1]) / (2 * step)
            tol = 1e-4 * e_th[i, p] + 1e-10 * np.sum(np.abs(u) * y_envelope(m, synth.CONP, phi, par)) / step
            assert abs(fd - g_th[i, p]) <= tol, (i, p, fd, g_th[i, p])


def test_autograd_function_follows_theta(pj, mechs):
    """A theta that differs from the mechanism's parameters moves the
    evaluation point: y and both gradients equal the oracle's on a mechanism
    holding theta's (ln A, beta, Ea); theta equal to the mechanism's gives
    the mechanism's own values."""
    import torch
    m = mechs("gri53")
    h = pj.pj_mech_create(m)
    n = 40
    phi, par = synth.make_states(m, n, 23, synth.CONP)
    uw, uT = synth.make_cotangents(m.n_species, n, 23)
    u = np.concatenate([uw, uT[None, :]], axis=0)
    rng = np.random.default_rng(3)
    th0 = pj.arrhenius_parameters(m).numpy()
    th = th0.copy()
    th[:, 0] += rng.normal(0.0, 0.3, m.n_reactions)
    th[:, 1] += rng.normal(0.0, 0.05, m.n_reactions)
    th[:, 2] *= np.exp(rng.normal(0.0, 0.02, m.n_reactions))
    mp = m.copy()
    mp.A, mp.beta, mp.Ea = np.exp(th[:, 0]), th[:, 1].copy(), th[:, 2].copy()
    for theta_np, ref_m in ((th, mp), (th0, m)):
        theta = torch.from_numpy(theta_np.copy()).cuda().requires_grad_(True)
        d_phi = dev(phi).requires_grad_(True)
        y = pj.source_terms_y(h, synth.CONP, d_phi, dev(par), theta)
        (y * dev(u)).sum().backward()
        y_ref = oracle.outputs_y(ref_m, synth.CONP, phi, par)
        check_close(y.detach().cpu().numpy(), y_ref, y_envelope(ref_m, synth.CONP, phi, par), RTOL_SRC, ATOL_SRC,
                    "y at theta")
        g_phi, g_th = oracle.vjp(ref_m, synth.CONP, phi, par, uw, uT)
        e_phi, e_th = oracle.vjp_envelope(ref_m, synth.CONP, phi, par, uw, uT)
        check_close(d_phi.grad.cpu().numpy(), g_phi, e_phi, RTOL_VJP, 0.0, "g_phi at theta")
        check_close(theta.grad.cpu().numpy(), g_th, e_th, RTOL_VJP, 0.0, "g_theta at theta")
    # the perturbation is large enough to matter
    assert not np.allclose(oracle.outputs_y(mp, synth.CONP, phi, par), oracle.outputs_y(m, synth.CONP, phi, par),
                           rtol=1e-3)
