"""Python binding of the C ABI (include/pyjac_gb.h).

Functions named ``pj_*`` mirror the C entry points one to one (argument
marshalling only: torch tensors are passed by device pointer, ``stream``
defaults to torch's current stream).  The convenience wrappers below them
allocate outputs with torch and call the same entry points.  Every step of
the computation runs in the library's CUDA kernels.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _native as N
from ._native import (PJ_CONP, PJ_CONV, PJ_CSR, PJ_CSC, PJ_DENSE, PJ_OP_SOURCE, PJ_OP_JACOBIAN,
                      PJ_OP_NEWTON, PJ_OP_VJP, PJ_OP_Y, PJ_OP_FD, PJ_OP_LU, PJ_F64, PJ_F32, PJ_MAX_SP, PJ_JAC_EXACT, PJ_JAC_APPROX,
                      PJ_LAYOUT_PERCORE, PJ_LAYOUT_TMEM, PJ_LAYOUT_COOP, check)


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return C.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def _i32(a):
    return np.ascontiguousarray(np.asarray(a), dtype=np.int32)


def _f64(a):
    return np.ascontiguousarray(np.asarray(a), dtype=np.float64)


class Mechanism:
    """Owner of a ``pj_mech*`` handle (freed on garbage collection)."""

    def __init__(self, handle: C.c_void_p, name: str = ""):
        self._h = handle
        self.name = name
        ns, nr, nnz = C.c_int32(), C.c_int32(), C.c_int32()
        check(N.load().pj_mech_info(self._h, C.byref(ns), C.byref(nr), C.byref(nnz)), "pj_mech_info")
        self.n_species, self.n_reactions, self.nnz = ns.value, nr.value, nnz.value

    @property
    def handle(self):
        return self._h

    @property
    def jacobian_form(self):
        f = C.c_int32()
        check(N.load().pj_mech_jacobian_form(self._h, C.byref(f)), "pj_mech_jacobian_form")
        return f.value

    def with_jacobian_form(self, form) -> "Mechanism":
        """The same mechanism with the exact (PJ_JAC_EXACT) or approximate
        (PJ_JAC_APPROX, Sec. 3.4) Jacobian and its pattern."""
        h = C.c_void_p()
        check(N.load().pj_mech_with_jacobian_form(self._h, form, C.byref(h)), "pj_mech_with_jacobian_form")
        return Mechanism(h, self.name)

    def jacobian_layout(self, fmt=PJ_CSR, prec=PJ_F64, n=1 << 20):
        """PJ_LAYOUT_PERCORE / _TMEM / _COOP: the kernel layout of the
        Jacobian entries for n states of this mechanism on the current device."""
        lay = C.c_int32()
        check(N.load().pj_jacobian_layout(self._h, fmt, prec, int(n), C.byref(lay)), "pj_jacobian_layout")
        return lay.value

    def arrhenius(self):
        """(ln A, beta, Ea) [Nr] each: the high-pressure (or only) Arrhenius
        parameters of the handle, in reaction order (float64 numpy)."""
        nr = self.n_reactions
        a, b, e = (np.zeros(max(nr, 1)) for _ in range(3))
        check(N.load().pj_mech_arrhenius(self._h, a.ctypes.data_as(N._dp), b.ctypes.data_as(N._dp),
                                         e.ctypes.data_as(N._dp)), "pj_mech_arrhenius")
        return a[:nr], b[:nr], e[:nr]

    def with_arrhenius(self, lnA, beta, Ea) -> "Mechanism":
        """The same mechanism with the high-pressure (or only) Arrhenius
        parameters replaced (Sec. 2.2 rate constants)."""
        a, b, e = (np.ascontiguousarray(np.asarray(x, dtype=np.float64).reshape(-1)) for x in (lnA, beta, Ea))
        if not (a.shape == b.shape == e.shape == (self.n_reactions,)):
            raise ValueError(f"lnA, beta and Ea must each hold {self.n_reactions} values")
        h = C.c_void_p()
        check(N.load().pj_mech_with_arrhenius(self._h, a.ctypes.data_as(N._dp), b.ctypes.data_as(N._dp),
                                              e.ctypes.data_as(N._dp), C.byref(h)), "pj_mech_with_arrhenius")
        return Mechanism(h, self.name)

    def sparsity(self, fmt=PJ_CSR):
        ptr = np.zeros(self.n_species + 2, dtype=np.int32)
        idx = np.zeros(max(self.nnz, 1), dtype=np.int32)
        check(N.load().pj_sparsity(self._h, fmt, ptr.ctypes.data_as(N._ip), idx.ctypes.data_as(N._ip)),
              "pj_sparsity")
        return ptr, idx[: self.nnz]

    def lu_info(self):
        """(lu_nnz, perm [N]) of the Newton-matrix LU."""
        k = C.c_int32()
        perm = np.zeros(self.n_species + 1, dtype=np.int32)
        check(N.load().pj_lu_info(self._h, C.byref(k), perm.ctypes.data_as(N._ip)), "pj_lu_info")
        return k.value, perm

    def lu_pattern(self):
        """Pivot-order (rows, cols) of the factor values in storage order."""
        k, _ = self.lu_info()
        r = np.zeros(max(k, 1), dtype=np.int32)
        c = np.zeros(max(k, 1), dtype=np.int32)
        check(N.load().pj_lu_pattern(self._h, r.ctypes.data_as(N._ip), c.ctypes.data_as(N._ip)), "pj_lu_pattern")
        return r[:k], c[:k]

    def workspace_size(self, op, n):
        b = C.c_size_t()
        check(N.load().pj_workspace_size(self._h, op, n, C.byref(b)), "pj_workspace_size")
        return b.value

    def close(self):
        if self._h is not None and N._lib is not None:
            N._lib.pj_mech_free(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pj_mech_create(mech) -> Mechanism:
    """Create a device mechanism from a description object with the fields of
    ``pj_mech_desc`` (species data, reactions, efficiencies)."""
    lib = N.load()
    ns, nr = len(mech.W), len(mech.kind)
    keep = dict(
        W=_f64(mech.W), T_mid=_f64(mech.T_mid), nasa_low=_f64(mech.nasa_low).reshape(-1),
        nasa_high=_f64(mech.nasa_high).reshape(-1), kind=_i32(mech.kind),
        reversible=_i32(np.asarray(mech.reversible).astype(np.int32)),
        reac_sp=_i32(mech.reac_sp).reshape(-1), reac_nu=_i32(mech.reac_nu).reshape(-1),
        prod_sp=_i32(mech.prod_sp).reshape(-1), prod_nu=_i32(mech.prod_nu).reshape(-1),
        A=_f64(mech.A), beta=_f64(mech.beta), Ea=_f64(mech.Ea), A0=_f64(mech.A0),
        beta0=_f64(mech.beta0), Ea0=_f64(mech.Ea0), troe=_f64(mech.troe).reshape(-1),
        troe_n=_i32(mech.troe_n), sri=_f64(mech.sri).reshape(-1), eff_ptr=_i32(mech.eff_ptr),
        eff_sp=_i32(mech.eff_sp) if len(mech.eff_sp) else np.zeros(1, np.int32),
        eff_val=_f64(mech.eff_val) if len(mech.eff_val) else np.zeros(1))
    # less common reaction types (optional fields of the description object)
    z = lambda: np.zeros(nr)
    chem = getattr(mech, "chem", None)
    keep.update(
        chem=_i32(np.zeros(nr) if chem is None else np.asarray(chem).astype(np.int32)),
        rev_explicit=_i32(np.asarray(getattr(mech, "rev_explicit", z())).astype(np.int32)))
    rev_arr = np.asarray(getattr(mech, "rev_arr", np.zeros((nr, 3))), dtype=float).reshape(nr, 3)
    keep.update(rev_A=_f64(rev_arr[:, 0]), rev_beta=_f64(rev_arr[:, 1]), rev_Ea=_f64(rev_arr[:, 2]))
    plog = np.asarray(getattr(mech, "plog", np.zeros((0, 4))), dtype=float).reshape(-1)
    cheb = np.asarray(getattr(mech, "cheb_coef", np.zeros(0)), dtype=float).reshape(-1)
    shape = np.asarray(getattr(mech, "cheb_shape", np.zeros((nr, 2))), dtype=np.int64).reshape(nr, 2)
    keep.update(
        plog_ptr=_i32(getattr(mech, "plog_ptr", np.zeros(nr + 1))),
        plog=_f64(plog) if len(plog) else np.zeros(1),
        cheb_ptr=_i32(getattr(mech, "cheb_ptr", np.zeros(nr + 1))),
        cheb_nT=_i32(shape[:, 0]), cheb_nP=_i32(shape[:, 1]),
        cheb_range=_f64(np.asarray(getattr(mech, "cheb_range", np.zeros((nr, 4))), dtype=float).reshape(-1)),
        cheb_coef=_f64(cheb) if len(cheb) else np.zeros(1))
    d = N.pj_mech_desc()
    d.n_species, d.n_reactions = ns, nr
    for k, v in keep.items():
        setattr(d, k, v.ctypes.data_as(N._ip if v.dtype == np.int32 else N._dp))
    h = C.c_void_p()
    check(lib.pj_mech_create(C.byref(d), C.byref(h)), "pj_mech_create")
    return Mechanism(h, getattr(mech, "name", ""))


def pj_mech_load(path: str) -> Mechanism:
    h = C.c_void_p()
    check(N.load().pj_mech_load(path.encode(), C.byref(h)), "pj_mech_load")
    return Mechanism(h, path)


def pj_mech_with_jacobian_form(mech: Mechanism, form) -> Mechanism:
    return mech.with_jacobian_form(form)


def pj_debug_word(mech: Mechanism, clear=False) -> int:
    """The bounds-checked build's device error word of mech (0 when every
    index-table lookup stayed in range; always 0 in the regular build)."""
    w = C.c_uint32()
    check(N.load().pj_debug_word(mech.handle, C.byref(w), int(bool(clear))), "pj_debug_word")
    return w.value


def pj_debug_build() -> bool:
    on = C.c_int32()
    check(N.load().pj_debug_build(C.byref(on)), "pj_debug_build")
    return bool(on.value)


def pj_debug_set_target(mech: Mechanism, fmt, index, value):
    return check(N.load().pj_debug_set_target(mech.handle, fmt, int(index), int(value)), "pj_debug_set_target")


def pj_jacobian_layout(mech: Mechanism, fmt=PJ_CSR, prec=PJ_F64, n=1 << 20):
    return mech.jacobian_layout(fmt, prec, n)


def pj_mech_arrhenius(mech: Mechanism):
    return mech.arrhenius()


def pj_mech_with_arrhenius(mech: Mechanism, lnA, beta, Ea) -> Mechanism:
    return mech.with_arrhenius(lnA, beta, Ea)


def pj_mech_jacobian_form(mech: Mechanism):
    return mech.jacobian_form


def pj_sparsity(mech: Mechanism, fmt=PJ_CSR):
    return mech.sparsity(fmt)


def pj_workspace_size(mech: Mechanism, op, n):
    return mech.workspace_size(op, n)


def pj_eval_source_terms(mech, mode, n, param, phi, ld, dphi, status=None, work=None, work_bytes=0,
                         stream=None):
    return check(N.load().pj_eval_source_terms(mech.handle, mode, n, _ptr(param), _ptr(phi), ld, _ptr(dphi),
                                                _ptr(status), _ptr(work), work_bytes, _stream(stream)),
                 "pj_eval_source_terms")


def pj_eval_jacobian_sparse(mech, mode, fmt, n, param, phi, ld, vals, dphi=None, status=None, work=None,
                            work_bytes=0, stream=None):
    return check(N.load().pj_eval_jacobian_sparse(mech.handle, mode, fmt, n, _ptr(param), _ptr(phi), ld,
                                                   _ptr(vals), _ptr(dphi), _ptr(status), _ptr(work),
                                                   work_bytes, _stream(stream)),
                 "pj_eval_jacobian_sparse")


def pj_eval_jacobian_fd(mech, mode, fmt, n, param, phi, ld, vals, dphi=None, status=None, work=None,
                        work_bytes=0, stream=None):
    return check(N.load().pj_eval_jacobian_fd(mech.handle, mode, fmt, n, _ptr(param), _ptr(phi), ld,
                                               _ptr(vals), _ptr(dphi), _ptr(status), _ptr(work),
                                               work_bytes, _stream(stream)),
                 "pj_eval_jacobian_fd")


def pj_eval_jacobian_dense(mech, mode, n, param, phi, ld, jac, dphi=None, status=None, work=None,
                           work_bytes=0, stream=None):
    return check(N.load().pj_eval_jacobian_dense(mech.handle, mode, n, _ptr(param), _ptr(phi), ld, _ptr(jac),
                                                  _ptr(dphi), _ptr(status), _ptr(work), work_bytes,
                                                  _stream(stream)),
                 "pj_eval_jacobian_dense")


def pj_eval_y(mech, mode, n, param, phi, ld, y, status=None, work=None, work_bytes=0, stream=None):
    return check(N.load().pj_eval_y(mech.handle, mode, n, _ptr(param), _ptr(phi), ld, _ptr(y), _ptr(status),
                                     _ptr(work), work_bytes, _stream(stream)), "pj_eval_y")


def pj_vjp(mech, mode, n, param, phi, ld, u_wdot, u_T, y, g_phi, g_theta, status=None, work=None, work_bytes=0,
           stream=None):
    return check(N.load().pj_vjp(mech.handle, mode, n, _ptr(param), _ptr(phi), ld, _ptr(u_wdot), _ptr(u_T),
                                  _ptr(y), _ptr(g_phi), _ptr(g_theta), _ptr(status), _ptr(work), work_bytes,
                                  _stream(stream)), "pj_vjp")


def pj_newton_matrix_f32(mech, mode, fmt, n, param, phi, ld, h, gamma, M, dphi, status=None, work=None,
                         work_bytes=0, stream=None):
    return check(N.load().pj_newton_matrix_f32(mech.handle, mode, fmt, n, _ptr(param), _ptr(phi), ld, _ptr(h),
                                                float(gamma), _ptr(M), _ptr(dphi), _ptr(status), _ptr(work),
                                                work_bytes, _stream(stream)),
                 "pj_newton_matrix_f32")


def pj_diag_exp(mech, n, x, y_ours, y_lib, stream=None):
    return check(N.load().pj_diag_exp(mech.handle, n, _ptr(x), _ptr(y_ours), _ptr(y_lib), _stream(stream)),
                 "pj_diag_exp")


def pj_eval_jacobian_sparse_noalloc(mech, mode, fmt, n, param, phi, ld, vals, dphi, status=None, stream=None):
    """Sparse Jacobian without a workspace argument, for callers that cannot
    allocate device memory: the library's fixed per-device scratch array is
    used instead (calls overlapping on the GPU race on it)."""
    return check(N.load().pj_eval_jacobian_sparse_noalloc(mech.handle, mode, fmt, n, _ptr(param), _ptr(phi), ld,
                                                           _ptr(vals), _ptr(dphi), _ptr(status), _stream(stream)),
                 "pj_eval_jacobian_sparse_noalloc")


def _hptr(a):
    """Address of a host array: a CPU torch tensor or a numpy array."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if a.is_cuda:
            raise TypeError("host buffer expected, got a CUDA tensor")
        return C.c_void_p(a.data_ptr())
    return C.c_void_p(a.ctypes.data)


def pj_eval_jacobian_sparse_host(mech, mode, fmt, n, h_param, h_phi, h_vals, h_dphi, chunk=0, stream=None):
    """Source terms and sparse Jacobian of n states in host memory (leading
    dimension n), transfers inside the call, chunked and overlapped with the
    kernels; returns the number of invalid states.  Page-locked buffers
    (torch pin_memory) give the overlapped, full-bandwidth path."""
    st = C.c_int(0)
    check(N.load().pj_eval_jacobian_sparse_host(mech.handle, mode, fmt, n, _hptr(h_param), _hptr(h_phi),
                                                 _hptr(h_vals), _hptr(h_dphi), C.byref(st), int(chunk),
                                                 _stream(stream)),
          "pj_eval_jacobian_sparse_host")
    return st.value


# ---------------------------------------------------------------------------
# convenience wrappers (torch tensors in, torch tensors out)
# ---------------------------------------------------------------------------
def _check_batch(mech, phi, param):
    import torch
    if phi.dtype != torch.float64 or param.dtype != torch.float64:
        raise TypeError("phi and param must be float64")
    if not (phi.is_cuda and param.is_cuda):
        raise TypeError("phi and param must be CUDA tensors")
    if phi.dim() != 2 or phi.shape[0] != mech.n_species + 1 or phi.stride(1) != 1:
        raise ValueError("phi must be [Ns+1, n] with unit stride along states")
    if param.dim() != 1 or param.shape[0] != phi.shape[1] or param.stride(0) != 1:
        raise ValueError("param must be [n] contiguous")
    return phi.shape[1], max(phi.stride(0), 1)


def _check_out(t, rows, ld, n, dtype, what):
    """A caller-given output must be [rows, n] on the states' device with the
    states' leading dimension (the C ABI takes one ld for all arrays)."""
    if t is None:
        return
    if t.dtype != dtype or not t.is_cuda or t.dim() != 2 or t.shape[0] != rows or t.shape[1] != n:
        raise ValueError(f"{what} must be a CUDA {dtype} tensor of shape [{rows}, {n}]")
    if t.stride(1) != 1 or (rows > 1 and t.stride(0) != ld):
        raise ValueError(f"{what} must have unit stride along states and leading dimension {ld} (that of phi)")


def _workspace(mech, op, n, device):
    import torch
    b = mech.workspace_size(op, n)
    return (torch.empty(b, dtype=torch.uint8, device=device), b) if b else (None, 0)


def source_terms(mech, mode, phi, param, out=None, status=None, stream=None):
    import torch
    n, ld = _check_batch(mech, phi, param)
    _check_out(out, mech.n_species + 1, ld, n, torch.float64, "out")
    if out is None:
        out = torch.empty((mech.n_species + 1, ld), dtype=torch.float64, device=phi.device)[:, :n]
    work, wb = _workspace(mech, PJ_OP_SOURCE, n, phi.device)
    pj_eval_source_terms(mech, mode, n, param, phi, ld, out, status, work, wb, stream)
    return out


def _dphi_like(mech, phi, ld, n):
    import torch
    return torch.empty((mech.n_species + 1, ld), dtype=torch.float64, device=phi.device)[:, :n]


def jacobian_sparse(mech, mode, phi, param, fmt=PJ_CSR, out=None, dphi=None, status=None, stream=None):
    import torch
    n, ld = _check_batch(mech, phi, param)
    _check_out(out, mech.nnz, ld, n, torch.float64, "out")
    _check_out(dphi, mech.n_species + 1, ld, n, torch.float64, "dphi")
    if out is None:
        out = torch.empty((mech.nnz, ld), dtype=torch.float64, device=phi.device)[:, :n]
    if dphi is None:
        dphi = _dphi_like(mech, phi, ld, n)
    work, wb = _workspace(mech, PJ_OP_JACOBIAN, n, phi.device)
    pj_eval_jacobian_sparse(mech, mode, fmt, n, param, phi, ld, out, dphi, status, work, wb, stream)
    return out


def jacobian_sparse_host(mech, mode, phi, param, fmt=PJ_CSR, out=None, dphi=None, chunk=0, pin=True):
    """jacobian_sparse for host (CPU) float64 tensors phi [Ns+1, n] and param
    [n], both contiguous: returns (values [nnz, n], source terms [Ns+1, n],
    invalid-state count), the outputs in host memory (page-locked when
    allocated here with pin=True)."""
    import torch
    if phi.dtype != torch.float64 or param.dtype != torch.float64 or phi.is_cuda or param.is_cuda:
        raise TypeError("phi and param must be float64 CPU tensors")
    if phi.dim() != 2 or phi.shape[0] != mech.n_species + 1 or not phi.is_contiguous() or not param.is_contiguous():
        raise ValueError("phi must be a contiguous [Ns+1, n] tensor and param a contiguous [n] tensor")
    n = phi.shape[1]
    if out is None:
        out = torch.empty((mech.nnz, n), dtype=torch.float64, pin_memory=pin)
    if dphi is None:
        dphi = torch.empty((mech.n_species + 1, n), dtype=torch.float64, pin_memory=pin)
    bad = pj_eval_jacobian_sparse_host(mech, mode, fmt, n, param, phi, out, dphi, chunk)
    return out, dphi, bad


def jacobian_fd(mech, mode, phi, param, fmt=PJ_CSR, out=None, dphi=None, status=None, stream=None):
    """First-order forward finite-difference Jacobian (the comparator), in
    the layout of jacobian_sparse (fmt CSR/CSC) or jacobian_dense (PJ_DENSE)."""
    import torch
    n, ld = _check_batch(mech, phi, param)
    N1 = mech.n_species + 1
    _check_out(out, N1 * N1 if fmt == PJ_DENSE else mech.nnz, ld, n, torch.float64, "out")
    _check_out(dphi, N1, ld, n, torch.float64, "dphi")
    if out is None:
        rows = N1 * N1 if fmt == PJ_DENSE else mech.nnz
        out = torch.empty((rows, ld), dtype=torch.float64, device=phi.device)[:, :n]
    if dphi is None:
        dphi = _dphi_like(mech, phi, ld, n)
    work, wb = _workspace(mech, PJ_OP_FD, n, phi.device)
    pj_eval_jacobian_fd(mech, mode, fmt, n, param, phi, ld, out, dphi, status, work, wb, stream)
    return out


def jacobian_dense(mech, mode, phi, param, out=None, dphi=None, status=None, stream=None):
    import torch
    n, ld = _check_batch(mech, phi, param)
    N1 = mech.n_species + 1
    _check_out(out, N1 * N1, ld, n, torch.float64, "out")
    _check_out(dphi, N1, ld, n, torch.float64, "dphi")
    if out is None:
        out = torch.empty((N1 * N1, ld), dtype=torch.float64, device=phi.device)[:, :n]
    if dphi is None:
        dphi = _dphi_like(mech, phi, ld, n)
    work, wb = _workspace(mech, PJ_OP_JACOBIAN, n, phi.device)
    pj_eval_jacobian_dense(mech, mode, n, param, phi, ld, out, dphi, status, work, wb, stream)
    return out


def newton_matrix_f32(mech, mode, phi, param, h, gamma=1.0, fmt=PJ_CSR, out=None, dphi=None, status=None,
                      stream=None):
    """FP32 M = I - h*gamma*J (CSR/CSC values or dense rows) and FP64 source terms."""
    import torch
    n, ld = _check_batch(mech, phi, param)
    N1 = mech.n_species + 1
    rows = N1 * N1 if fmt == PJ_DENSE else mech.nnz
    _check_out(out, rows, ld, n, torch.float32, "out")
    _check_out(dphi, N1, ld, n, torch.float64, "dphi")
    if out is None:
        out = torch.empty((rows, ld), dtype=torch.float32, device=phi.device)[:, :n]
    if dphi is None:
        dphi = _dphi_like(mech, phi, ld, n)
    work, wb = _workspace(mech, PJ_OP_NEWTON, n, phi.device)
    pj_newton_matrix_f32(mech, mode, fmt, n, param, phi, ld, h, gamma, out, dphi, status, work, wb, stream)
    return out


def eval_y(mech, mode, phi, param, out=None, status=None, stream=None):
    """y = (wdot_0 .. wdot_{Ns-1}, dT/dt), shape [Ns+1, n]."""
    import torch
    n, ld = _check_batch(mech, phi, param)
    _check_out(out, mech.n_species + 1, ld, n, torch.float64, "out")
    if out is None:
        out = torch.empty((mech.n_species + 1, ld), dtype=torch.float64, device=phi.device)[:, :n]
    work, wb = _workspace(mech, PJ_OP_Y, n, phi.device)
    pj_eval_y(mech, mode, n, param, phi, ld, out, status, work, wb, stream)
    return out


def vjp(mech, mode, phi, param, u_wdot, u_T, status=None, stream=None):
    """(y, g_phi [Ns+1, n], g_theta [Nr, 3]) for cotangents u_wdot [Ns, n], u_T [n]."""
    import torch
    n, ld = _check_batch(mech, phi, param)
    if u_wdot.shape != (mech.n_species, n) or u_wdot.stride() != (ld, 1) or u_T.shape != (n,):
        raise ValueError("u_wdot must be [Ns, n] with the leading dimension of phi, u_T [n]")
    y = torch.empty((mech.n_species + 1, ld), dtype=torch.float64, device=phi.device)[:, :n]
    g_phi = torch.empty((mech.n_species + 1, ld), dtype=torch.float64, device=phi.device)[:, :n]
    g_theta = torch.empty((mech.n_reactions, 3), dtype=torch.float64, device=phi.device)
    work, wb = _workspace(mech, PJ_OP_VJP, n, phi.device)
    pj_vjp(mech, mode, n, param, phi, ld, u_wdot, u_T.contiguous(), y, g_phi, g_theta, status, work, wb, stream)
    return y, g_phi, g_theta


def arrhenius_parameters(mech_data):
    """theta [Nr, 3] = (ln A, beta, Ea) of the high-pressure (or only) rate of a
    mechanism description, as a float64 CPU tensor."""
    import torch
    return torch.tensor(np.stack([np.log(np.asarray(mech_data.A, float)), np.asarray(mech_data.beta, float),
                                  np.asarray(mech_data.Ea, float)], axis=1))


def _make_function():
    import torch

    class SourceTermsY(torch.autograd.Function):
        """y(phi, theta) = (wdot_0 .. wdot_{Ns-1}, dT/dt) with gradients by the
        adjoint kernel.  theta [Nr, 3] holds each reaction's high-pressure
        (or only) (ln A, beta, Ea): where it differs from the handle's, the
        evaluation and both gradients use a handle with theta's parameters
        (pj_mech_with_arrhenius; the last one is kept for the next call)."""

        @staticmethod
        def forward(ctx, phi, theta, mech, mode, param):
            ctx.mech, ctx.mode = _mech_at(mech, theta), mode
            ctx.save_for_backward(phi, param)
            return eval_y(ctx.mech, mode, phi.detach(), param)

        @staticmethod
        def backward(ctx, gy):
            phi, param = ctx.saved_tensors
            ns = ctx.mech.n_species
            gy = gy.contiguous()
            n = phi.shape[1]
            u_wdot = torch.empty((ns, max(phi.stride(0), 1)), dtype=torch.float64, device=phi.device)[:, :n]
            u_wdot.copy_(gy[:ns])
            _, g_phi, g_theta = vjp(ctx.mech, ctx.mode, phi.detach(), param, u_wdot, gy[ns])
            return g_phi, g_theta.to(phi.device), None, None, None

    return SourceTermsY


_Y = None


def _mech_at(mech, theta):
    """mech itself when theta [Nr, 3] equals its (ln A, beta, Ea), else a
    handle with theta's parameters (cached on mech for the last theta)."""
    t = theta.detach().to("cpu", dtype=__import__("torch").float64).numpy().reshape(mech.n_reactions, 3)
    if not hasattr(mech, "_theta0"):
        mech._theta0 = np.stack(mech.arrhenius(), axis=1)
        mech._theta_cache = (None, None)
    if np.array_equal(t, mech._theta0):
        return mech
    key = t.tobytes()
    if mech._theta_cache[0] != key:
        mech._theta_cache = (key, mech.with_arrhenius(t[:, 0], t[:, 1], t[:, 2]))
    return mech._theta_cache[1]


def source_terms_y(mech, mode, phi, param, theta):
    """Differentiable y = (wdot, dT/dt) (torch.autograd.Function)."""
    global _Y
    if _Y is None:
        _Y = _make_function()
    return _Y.apply(phi, theta, mech, mode, param)


# ---------------------------------------------------------------------------
# batching form
# ---------------------------------------------------------------------------
class Plan:
    """Owner of a ``pj_plan*``: uneven batches through persistent kernels,
    optionally replayed as a captured CUDA graph.  ``batches`` is a list of
    (param, phi, out, dphi) tensors; phi is [Ns+1, n] with unit stride along
    states, out/dphi as for the single-batch entry points."""

    def __init__(self, mech, op, mode, batches, fmt=PJ_CSR, max_states_per_launch=0, status=None):
        lib = N.load()
        self.mech = mech
        self._keep = batches
        arr = (N.pj_batch * max(len(batches), 1))()
        for i, (param, phi, out, dphi) in enumerate(batches):
            n = phi.shape[1]
            arr[i] = N.pj_batch(param.data_ptr(), phi.data_ptr(), n, max(phi.stride(0), 1), out.data_ptr(),
                                dphi.data_ptr() if dphi is not None else None)
        h = C.c_void_p()
        check(lib.pj_plan_create(mech.handle, op, mode, fmt, len(batches), arr, max_states_per_launch,
                                 _ptr(status), C.byref(h)), "pj_plan_create")
        self._h = h

    def config(self):
        t, b, s, g = C.c_int(), C.c_int(), C.c_int(), C.c_int()
        check(N.load().pj_plan_get_config(self._h, C.byref(t), C.byref(b), C.byref(s), C.byref(g)),
              "pj_plan_get_config")
        return dict(threads_per_block=t.value, blocks_per_sm=b.value, use_shared=s.value, groups=g.value)

    def set_config(self, threads_per_block, blocks_per_sm, use_shared):
        check(N.load().pj_plan_set_config(self._h, threads_per_block, blocks_per_sm, int(use_shared)),
              "pj_plan_set_config")

    def autotune(self, stream=None, cache_path=None, reps=2):
        check(N.load().pj_plan_autotune(self._h, _stream(stream), cache_path.encode() if cache_path else None,
                                        reps), "pj_plan_autotune")
        return self.config()

    def run(self, stream=None):
        check(N.load().pj_plan_run(self._h, _stream(stream)), "pj_plan_run")

    def capture(self, stream):
        check(N.load().pj_plan_capture(self._h, _stream(stream)), "pj_plan_capture")

    def launch(self, stream=None):
        check(N.load().pj_plan_launch(self._h, _stream(stream)), "pj_plan_launch")

    def close(self):
        if getattr(self, "_h", None) is not None and N._lib is not None:
            N._lib.pj_plan_free(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _prec(t):
    import torch
    if t.dtype == torch.float64:
        return PJ_F64
    if t.dtype == torch.float32:
        return PJ_F32
    raise TypeError("LU values must be float64 or float32")


def pj_lu_factor(mech, prec, n, vals, ld, lu, h=None, gamma=1.0, status=None, work=None, work_bytes=0,
                 stream=None):
    return check(N.load().pj_lu_factor(mech.handle, prec, n, _ptr(vals), ld, _ptr(h), float(gamma), _ptr(lu),
                                       _ptr(status), _ptr(work), work_bytes, _stream(stream)), "pj_lu_factor")


def pj_lu_solve(mech, prec, n, lu, ld, b, x, stream=None):
    return check(N.load().pj_lu_solve(mech.handle, prec, n, _ptr(lu), ld, _ptr(b), _ptr(x), _stream(stream)),
                 "pj_lu_solve")


def lu_factor(mech, vals, h=None, gamma=1.0, out=None, status=None, stream=None):
    """Factors [lu_nnz, n] of M (vals: CSR values of M, or of J with h given:
    M = I - h gamma J), in vals' precision."""
    import torch
    nnz, n = vals.shape
    ld = vals.stride(0) if n > 0 else 1
    if vals.stride(1) != 1 or nnz != mech.nnz:
        raise ValueError("vals must be [nnz, n] with unit stride along states")
    lu_nnz, _ = mech.lu_info()
    if out is None:
        out = torch.empty((lu_nnz, max(ld, 1)), dtype=vals.dtype, device=vals.device)[:, :n]
    wb = mech.workspace_size(PJ_OP_LU, n)
    work = torch.empty(wb, dtype=torch.uint8, device=vals.device) if wb else None
    pj_lu_factor(mech, _prec(vals), n, vals, max(ld, 1), out, h, gamma, status, work, wb, stream)
    return out


def lu_solve(mech, lu, b, out=None, stream=None):
    """x with M x = b per state ([N, n], lu's precision)."""
    import torch
    n = b.shape[1]
    ld = lu.stride(0)
    if b.stride(0) != ld or b.stride(1) != 1:
        raise ValueError("b must share lu's leading dimension")
    if out is None:
        out = torch.empty((b.shape[0], ld), dtype=b.dtype, device=b.device)[:, :n]
    pj_lu_solve(mech, _prec(lu), n, lu, ld, b, out, stream)
    return out
