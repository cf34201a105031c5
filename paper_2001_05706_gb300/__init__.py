"""Python binding of the GB300 Wilson-clover / overlap library (liblqcd.so).

Argument marshalling only: every operation runs in the CUDA kernels behind
the C ABI declared in ``include/lqcd.h``; this module converts numpy arrays
(host memory) and torch CUDA tensors (device memory) to plain pointers and
raises ``LqcdError`` for a non-zero status.  Importing it without the built
library raises ImportError: there is no CPU fallback.

Functions keep the C names (``lqcd_create``, ``lqcd_load_gauge``,
``lqcd_clover``, ``lqcd_dslash``, ``lqcd_solve``, ...).  ``Lattice`` bundles a
context with those calls for convenience.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

_HERE = os.path.dirname(os.path.abspath(__file__))

if not os.path.exists(_build.LIB):
    raise ImportError(
        f"{_build.LIB} is missing: build the CUDA library first "
        "(python -c 'import __graft_entry__ as g; g.build()' or python paper_2001_05706_gb300/build.py)")
_lib = ctypes.CDLL(_build.LIB)

# enums (include/lqcd.h)
LQCD_OK = 0
LQCD_ERR_ARG, LQCD_ERR_CUDA, LQCD_ERR_OOM, LQCD_ERR_NOCONV = -1, -2, -3, -4
LQCD_ERR_TIMEOUT, LQCD_ERR_STATE, LQCD_ERR_NOT_SU3, LQCD_ERR_SINGULAR = -5, -6, -7, -8
LQCD_F64, LQCD_F32, LQCD_F16, LQCD_BF16, LQCD_DF64 = 0, 1, 2, 3, 4
LQCD_RECON_18, LQCD_RECON_12, LQCD_RECON_8 = 18, 12, 8
LQCD_EVEN, LQCD_ODD, LQCD_FULL = 0, 1, 2
(LQCD_OP_M, LQCD_OP_MHAT, LQCD_OP_MHAT_DAG, LQCD_OP_MHAT_NORMAL, LQCD_OP_HOP_EO, LQCD_OP_HOP_OE, LQCD_OP_HW,
 LQCD_OP_K2A, LQCD_OP_M_DAG, LQCD_OP_MHAT_SYM, LQCD_OP_MHAT_SYM_DAG) = range(11)

PREC = {"f64": LQCD_F64, "f32": LQCD_F32, "f16": LQCD_F16, "bf16": LQCD_BF16, "df64": LQCD_DF64}
OPS = {"M": LQCD_OP_M, "MHAT": LQCD_OP_MHAT, "MHAT_DAG": LQCD_OP_MHAT_DAG, "MHAT_NORMAL": LQCD_OP_MHAT_NORMAL,
       "HOP_EO": LQCD_OP_HOP_EO, "HOP_OE": LQCD_OP_HOP_OE, "HW": LQCD_OP_HW, "K2A": LQCD_OP_K2A,
       "M_DAG": LQCD_OP_M_DAG, "MHAT_SYM": LQCD_OP_MHAT_SYM, "MHAT_SYM_DAG": LQCD_OP_MHAT_SYM_DAG}


class lqcd_solve_params(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_iter", ctypes.c_int), ("inner", ctypes.c_int),
                ("delta", ctypes.c_double), ("nrhs", ctypes.c_int), ("use_x0", ctypes.c_int),
                ("recon", ctypes.c_int), ("inner_recon", ctypes.c_int), ("check_every", ctypes.c_int),
                ("outer", ctypes.c_int), ("solver", ctypes.c_int), ("schur", ctypes.c_int),
                ("gcr_nkrylov", ctypes.c_int)]


class lqcd_overlap_params(ctypes.Structure):
    _fields_ = [("rho", ctypes.c_double), ("mass", ctypes.c_double), ("n_low", ctypes.c_int),
                ("max_degree", ctypes.c_int), ("sign_tol", ctypes.c_double), ("eig_tol", ctypes.c_double),
                ("max_filter", ctypes.c_int), ("seed", ctypes.c_ulonglong), ("high", ctypes.c_int),
                ("eig_method", ctypes.c_int)]


class lqcd_overlap_info(ctypes.Structure):
    _fields_ = [("n_low", ctypes.c_int), ("lambda_", ctypes.c_double * 64), ("resid", ctypes.c_double * 64),
                ("a", ctypes.c_double), ("b", ctypes.c_double), ("degree", ctypes.c_int),
                ("sign_error", ctypes.c_double), ("sweeps", ctypes.c_int), ("seconds", ctypes.c_double),
                ("degree_inner", ctypes.c_int), ("hw_applies", ctypes.c_double)]


LQCD_OV_APPLY, LQCD_OV_APPLY_DAG, LQCD_OV_SIGN, LQCD_OV_SOLVE, LQCD_OV_SOLVE_DEFLATED = 0, 1, 2, 3, 4
LQCD_OV_MAX_EV = 256


class lqcd_overlap_eigen_params(ctypes.Structure):
    _fields_ = [("n_ev", ctypes.c_int), ("sector", ctypes.c_int), ("tol", ctypes.c_double), ("basis", ctypes.c_int),
                ("max_restarts", ctypes.c_int), ("seed", ctypes.c_ulonglong)]


class lqcd_overlap_eigen_info(ctypes.Structure):
    _fields_ = [("n_ev", ctypes.c_int), ("n_partners", ctypes.c_int), ("mu", ctypes.c_double * LQCD_OV_MAX_EV),
                ("resid", ctypes.c_double * LQCD_OV_MAX_EV), ("lambda_re", ctypes.c_double * LQCD_OV_MAX_EV),
                ("lambda_im", ctypes.c_double * LQCD_OV_MAX_EV), ("restarts", ctypes.c_int),
                ("sign_applies", ctypes.c_double), ("seconds", ctypes.c_double)]


class lqcd_solve_info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("reliable_updates", ctypes.c_int), ("nrhs", ctypes.c_int),
                ("true_resid", ctypes.c_double * 64), ("seconds", ctypes.c_double),
                ("mhat_applies", ctypes.c_double)]


_vp = ctypes.c_void_p
_ip = ctypes.c_int
_sig = {
    "lqcd_create": [ctypes.POINTER(_vp), ctypes.POINTER(ctypes.c_int), _ip, _vp],
    "lqcd_destroy": [_vp],
    "lqcd_set_stream": [_vp, _vp],
    "lqcd_synchronize": [_vp],
    "lqcd_load_gauge": [_vp, _vp, _ip],
    "lqcd_clover": [_vp, ctypes.c_double, ctypes.c_double],
    "lqcd_set_rho": [_vp, ctypes.c_double],
    "lqcd_dslash": [_vp, _vp, _vp, _ip, _ip, _ip, _ip, _ip],
    "lqcd_field_create": [_vp, _ip, _ip, _ip, ctypes.POINTER(_vp)],
    "lqcd_field_destroy": [_vp],
    "lqcd_field_import": [_vp, _vp, _vp, _ip],
    "lqcd_field_export": [_vp, _vp, _vp, _ip],
    "lqcd_apply": [_vp, _ip, _ip, _vp, _vp],
    "lqcd_apply_schur": [_vp, _ip, _ip, _vp, _vp, _vp],
    "lqcd_field_norm2": [_vp, _vp, ctypes.POINTER(ctypes.c_double)],
    "lqcd_solve": [_vp, _vp, _vp, _ip, ctypes.POINTER(lqcd_solve_params), ctypes.POINTER(lqcd_solve_info)],
    "lqcd_norm2_noalloc": [_vp, ctypes.c_long, _ip, _vp, _vp],
    "lqcd_field_slices": [_vp, _vp, _ip, _ip, _ip, _vp, _ip, ctypes.c_double],
    "lqcd_k2a_slices": [_vp, _ip, _ip, _vp, _vp, _ip, _ip],
    "lqcd_k2b_slices": [_vp, _ip, _ip, _vp, _vp, _vp, _ip, _ip, _vp],
    "lqcd_field_axpby": [_vp, _vp, _vp, _vp, _vp],
    "lqcd_field_norm2s": [_vp, _vp, _vp],
    "lqcd_solve_batch": [ctypes.POINTER(_vp), _ip, ctypes.POINTER(_vp), ctypes.POINTER(_vp), _ip,
                         ctypes.POINTER(lqcd_solve_params), ctypes.POINTER(lqcd_solve_info)],
    "lqcd_overlap_setup": [_vp, ctypes.POINTER(lqcd_overlap_params), ctypes.POINTER(lqcd_overlap_info)],
    "lqcd_overlap_lowmodes": [_vp, _vp, _ip],
    "lqcd_overlap_eigen": [_vp, ctypes.POINTER(lqcd_overlap_eigen_params), ctypes.POINTER(lqcd_overlap_eigen_info)],
    "lqcd_overlap_eigvecs": [_vp, _vp, _ip, _ip],
    "lqcd_overlap": [_vp, _vp, _vp, _ip, _ip, _ip, ctypes.POINTER(lqcd_solve_params),
                     ctypes.POINTER(lqcd_solve_info)],
    "lqcd_mg_fine_stencil": [_vp, _vp, _vp, _vp],
    "lqcd_mg_apply": [_vp, ctypes.POINTER(ctypes.c_int), _ip, _vp, _vp, _vp, _vp, _vp],
    "lqcd_mg_orthonormalize": [_vp, ctypes.POINTER(ctypes.c_int), _ip, ctypes.POINTER(ctypes.c_int), _ip, _vp, _vp],
    "lqcd_mg_prolong": [_vp, ctypes.POINTER(ctypes.c_int), _ip, ctypes.POINTER(ctypes.c_int), _ip, _vp, _vp, _vp],
    "lqcd_mg_restrict": [_vp, ctypes.POINTER(ctypes.c_int), _ip, ctypes.POINTER(ctypes.c_int), _ip, _vp, _vp, _vp],
    "lqcd_mg_coarsen": [_vp, ctypes.POINTER(ctypes.c_int), _ip, ctypes.POINTER(ctypes.c_int), _ip, _vp, _vp, _vp,
                        _vp, _vp, _vp, _vp],
    "lqcd_mg_dots": [_vp, ctypes.c_long, _ip, _vp, _vp, ctypes.POINTER(ctypes.c_double)],
    "lqcd_mg_axpys": [_vp, ctypes.c_long, _ip, ctypes.POINTER(ctypes.c_double), _vp, _vp],
    "lqcd_mg_axpby": [_vp, ctypes.c_long, ctypes.POINTER(ctypes.c_double), _vp, ctypes.POINTER(ctypes.c_double), _vp],
}
for _name, _args in _sig.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = ctypes.c_int
_lib.lqcd_last_error.argtypes = []
_lib.lqcd_last_error.restype = ctypes.c_char_p


class LqcdError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"status {status}: {msg}")
        self.status = status


def lqcd_last_error() -> str:
    return _lib.lqcd_last_error().decode()


def _check(status):
    if status != LQCD_OK:
        raise LqcdError(status, lqcd_last_error())
    return status


def _buf(a):
    """(pointer, on_device) of a numpy array or a torch tensor (C-contiguous)."""
    if isinstance(a, np.ndarray):
        if not a.flags.c_contiguous:
            raise ValueError("array must be C-contiguous")
        return _vp(a.ctypes.data), 0
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return _vp(a.data_ptr()), 1 if a.is_cuda else 0
    raise TypeError(f"unsupported buffer type {type(a)}")


def _stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return _vp(stream)
    return _vp(stream.cuda_stream)


# ---- the C calls, same names ------------------------------------------------

def lqcd_create(dims, t_antiperiodic=1, stream=None):
    ctx = _vp()
    d = (ctypes.c_int * 4)(*[int(x) for x in dims])
    _check(_lib.lqcd_create(ctypes.byref(ctx), d, int(t_antiperiodic), _stream_ptr(stream)))
    return ctx


def lqcd_destroy(ctx):
    _check(_lib.lqcd_destroy(ctx))


def lqcd_set_stream(ctx, stream):
    _check(_lib.lqcd_set_stream(ctx, _stream_ptr(stream)))


def lqcd_synchronize(ctx):
    _check(_lib.lqcd_synchronize(ctx))


def lqcd_load_gauge(ctx, U):
    p, dev = _buf(U)
    _check(_lib.lqcd_load_gauge(ctx, p, dev))


def lqcd_clover(ctx, kappa, c_sw):
    _check(_lib.lqcd_clover(ctx, float(kappa), float(c_sw)))


def lqcd_set_rho(ctx, rho):
    _check(_lib.lqcd_set_rho(ctx, float(rho)))


def lqcd_dslash(ctx, out, inp, nrhs, op, prec, recon=LQCD_RECON_18):
    po, do = _buf(out)
    pi, di = _buf(inp)
    if do != di:
        raise ValueError("out and in must both be host or both be device buffers")
    _check(_lib.lqcd_dslash(ctx, po, pi, int(nrhs), int(op), int(prec), int(recon), do))


def lqcd_field_create(ctx, prec, subset, nrhs=1):
    f = _vp()
    _check(_lib.lqcd_field_create(ctx, int(prec), int(subset), int(nrhs), ctypes.byref(f)))
    return f


def lqcd_field_destroy(field):
    _check(_lib.lqcd_field_destroy(field))


def lqcd_field_import(ctx, field, canon):
    p, dev = _buf(canon)
    _check(_lib.lqcd_field_import(ctx, field, p, dev))


def lqcd_field_export(ctx, field, canon):
    p, dev = _buf(canon)
    _check(_lib.lqcd_field_export(ctx, field, p, dev))


def lqcd_apply(ctx, op, recon, out, inp):
    _check(_lib.lqcd_apply(ctx, int(op), int(recon), out, inp))


def lqcd_apply_schur(ctx, recon, dagger, out, x_odd, y_even):
    _check(_lib.lqcd_apply_schur(ctx, int(recon), int(dagger), out, x_odd, y_even))


def lqcd_field_norm2(ctx, field):
    r = ctypes.c_double(0)
    _check(_lib.lqcd_field_norm2(ctx, field, ctypes.byref(r)))
    return r.value


def lqcd_field_slices(ctx, field, parity, t0, t1, buf, to_field, factor=1.0):
    """Time slices [t0, t1) of one parity of a field to/from a device buffer (a CUDA tensor)."""
    pb, dev = _buf(buf)
    if not dev:
        raise ValueError("buf must be a CUDA tensor")
    _check(_lib.lqcd_field_slices(ctx, field, int(parity), int(t0), int(t1), pb, int(to_field), float(factor)))


def lqcd_k2a_slices(ctx, recon, dagger, y_even, x_odd, t0, t1):
    _check(_lib.lqcd_k2a_slices(ctx, int(recon), int(dagger), y_even, x_odd, int(t0), int(t1)))


def lqcd_k2b_slices(ctx, recon, dagger, z_odd, x_odd, y_even, t0, t1, nrhs=None):
    """z_o on time slices [t0, t1); returns the per-RHS ||z_o||^2 over them when nrhs is given."""
    if nrhs is None:
        _check(_lib.lqcd_k2b_slices(ctx, int(recon), int(dagger), z_odd, x_odd, y_even, int(t0), int(t1), None))
        return None
    out = (ctypes.c_double * int(nrhs))()
    _check(_lib.lqcd_k2b_slices(ctx, int(recon), int(dagger), z_odd, x_odd, y_even, int(t0), int(t1), out))
    return np.array(out[:])


def lqcd_field_axpby(ctx, y, a, b, x):
    """y = a[k] x + b[k] y per right-hand side."""
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    _check(_lib.lqcd_field_axpby(ctx, y, a.ctypes.data_as(_vp), b.ctypes.data_as(_vp), x))


def lqcd_field_norm2s(ctx, field, nrhs):
    out = (ctypes.c_double * int(nrhs))()
    _check(_lib.lqcd_field_norm2s(ctx, field, out))
    return np.array(out[:])


def lqcd_solve(ctx, x, b, params: lqcd_solve_params, raise_on_noconv=True):
    """Returns (status, info).  x holds the solution on return."""
    px, dx = _buf(x)
    pb, db = _buf(b)
    if dx != db:
        raise ValueError("x and b must both be host or both be device buffers")
    info = lqcd_solve_info()
    st = _lib.lqcd_solve(ctx, px, pb, dx, ctypes.byref(params), ctypes.byref(info))
    if st != LQCD_OK and (raise_on_noconv or st != LQCD_ERR_NOCONV):
        raise LqcdError(st, lqcd_last_error())
    return st, info


def lqcd_solve_batch(ctxs, xs, bs, params, raise_on_noconv=True):
    """Solve lattice i (context ctxs[i]) for xs[i] given bs[i]; returns (status, [info])."""
    n = len(ctxs)
    if not (len(xs) == len(bs) == n):
        raise ValueError("one x and one b per context")
    bufs_x = [_buf(a) for a in xs]
    bufs_b = [_buf(a) for a in bs]
    dev = {d for _, d in bufs_x + bufs_b}
    if len(dev) != 1:
        raise ValueError("all buffers must be host or all device")
    carr = (_vp * n)(*[c.value if isinstance(c, _vp) else c for c in ctxs])
    xarr = (_vp * n)(*[p.value for p, _ in bufs_x])
    barr = (_vp * n)(*[p.value for p, _ in bufs_b])
    infos = (lqcd_solve_info * n)()
    st = _lib.lqcd_solve_batch(carr, n, xarr, barr, dev.pop(), ctypes.byref(params), infos)
    if st != LQCD_OK and (raise_on_noconv or st != LQCD_ERR_NOCONV):
        raise LqcdError(st, lqcd_last_error())
    return st, list(infos)


def lqcd_norm2_noalloc(x, n, nrhs, result, stream=None):
    """result[k] = sum of squares of x[k*n:(k+1)*n] (device tensors of float64);
    allocates nothing (static library scratch), asynchronous on `stream`.
    The C side cannot see the tensors' sizes, so they are checked here: both
    float64, contiguous, on the current CUDA device, x holding n * nrhs values
    and result nrhs."""
    import torch
    for name, t in (("x", x), ("result", result)):
        if not isinstance(t, torch.Tensor) or not t.is_cuda:
            raise ValueError(f"{name} must be a CUDA tensor")
        if t.dtype != torch.float64:
            raise ValueError(f"{name} must be float64, not {t.dtype}")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
        if t.device.index != torch.cuda.current_device():
            raise ValueError(f"{name} is on {t.device}, not the current device cuda:{torch.cuda.current_device()}")
    n, nrhs = int(n), int(nrhs)
    if n >= 1 and nrhs >= 1 and x.numel() < n * nrhs:
        raise ValueError(f"x holds {x.numel()} values, fewer than n * nrhs = {n * nrhs}")
    if nrhs >= 1 and result.numel() < nrhs:
        raise ValueError(f"result holds {result.numel()} values, fewer than nrhs = {nrhs}")
    px, _ = _buf(x)
    pr, _ = _buf(result)
    _check(_lib.lqcd_norm2_noalloc(px, n, nrhs, pr, _stream_ptr(stream)))


LQCD_EIG_SUBSPACE, LQCD_EIG_LANCZOS = 0, 1
EIG_METHODS = {"subspace": LQCD_EIG_SUBSPACE, "lanczos": LQCD_EIG_LANCZOS}


def overlap_params(rho=1.5, mass=0.0, n_low=20, max_degree=4000, sign_tol=1e-10, eig_tol=1e-11, max_filter=200,
                   seed=7, high=LQCD_F64, eig_method=LQCD_EIG_SUBSPACE):
    if isinstance(high, str):
        high = PREC[high]
    if isinstance(eig_method, str):
        eig_method = EIG_METHODS[eig_method]
    return lqcd_overlap_params(rho, mass, n_low, max_degree, sign_tol, eig_tol, max_filter, seed, high, eig_method)


def lqcd_overlap_setup(ctx, params, raise_on_noconv=True):
    info = lqcd_overlap_info()
    st = _lib.lqcd_overlap_setup(ctx, ctypes.byref(params), ctypes.byref(info))
    if st != LQCD_OK and (raise_on_noconv or st != LQCD_ERR_NOCONV):
        raise LqcdError(st, lqcd_last_error())
    return st, info


def lqcd_overlap_lowmodes(ctx, vecs):
    p, dev = _buf(vecs)
    _check(_lib.lqcd_overlap_lowmodes(ctx, p, dev))


def overlap_eigen_params(n_ev=20, sector=1, tol=1e-9, basis=0, max_restarts=200, seed=11):
    return lqcd_overlap_eigen_params(n_ev, sector, tol, basis, max_restarts, seed)


def lqcd_overlap_eigen(ctx, params, raise_on_noconv=True):
    """The n_ev lowest eigenpairs of D_ov(0)^dag D_ov(0) in one chirality
    sector; returns (status, info)."""
    info = lqcd_overlap_eigen_info()
    st = _lib.lqcd_overlap_eigen(ctx, ctypes.byref(params), ctypes.byref(info))
    if st != LQCD_OK and (raise_on_noconv or st != LQCD_ERR_NOCONV):
        _check(st)
    return st, info


def lqcd_overlap_eigvecs(ctx, vecs, partners=False):
    p, dev = _buf(vecs)
    _check(_lib.lqcd_overlap_eigvecs(ctx, p, int(bool(partners)), dev))


def lqcd_overlap(ctx, out, inp, nrhs, op, cg=None, raise_on_noconv=True):
    po, do = _buf(out)
    pi, di = _buf(inp)
    if do != di:
        raise ValueError("out and in must both be host or both be device buffers")
    info = lqcd_solve_info()
    cgp = ctypes.byref(cg) if cg is not None else None
    st = _lib.lqcd_overlap(ctx, po, pi, int(nrhs), do, int(op), cgp, ctypes.byref(info))
    if st != LQCD_OK and (raise_on_noconv or st != LQCD_ERR_NOCONV):
        raise LqcdError(st, lqcd_last_error())
    return st, info


LQCD_SOLVER_CGLS, LQCD_SOLVER_BICGSTAB, LQCD_SOLVER_GCR = 0, 1, 2
SOLVERS = {"cgls": LQCD_SOLVER_CGLS, "bicgstab": LQCD_SOLVER_BICGSTAB, "gcr": LQCD_SOLVER_GCR}
LQCD_SCHUR_ASYM, LQCD_SCHUR_SYM = 0, 1
SCHUR = {"asym": LQCD_SCHUR_ASYM, "sym": LQCD_SCHUR_SYM}


def solve_params(tol=1e-10, max_iter=20000, inner=LQCD_F64, delta=0.1, nrhs=1, use_x0=0, recon=LQCD_RECON_18,
                 inner_recon=LQCD_RECON_12, check_every=8, outer=LQCD_F64, solver=LQCD_SOLVER_CGLS,
                 schur=LQCD_SCHUR_ASYM, gcr_nkrylov=0):
    if isinstance(solver, str):
        solver = SOLVERS[solver]
    if isinstance(schur, str):
        schur = SCHUR[schur]
    return lqcd_solve_params(tol, max_iter, inner, delta, nrhs, use_x0, recon, inner_recon, check_every, outer,
                             solver, schur, gcr_nkrylov)


# ---- convenience ------------------------------------------------------------

# ---- adaptive multigrid building blocks (complex128 CUDA tensors) -------------

def _mg_ptr(t, numel, name):
    """The device pointer of a contiguous complex128 CUDA tensor holding at
    least numel values (the C side cannot see sizes)."""
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != torch.complex128:
        raise ValueError(f"{name} must be complex128, not {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if t.numel() < numel:
        raise ValueError(f"{name} holds {t.numel()} values, fewer than {numel}")
    return _vp(t.data_ptr())


def _i4(v):
    v = [int(x) for x in v]
    if len(v) != 4:
        raise ValueError("four entries expected")
    return (ctypes.c_int * 4)(*v)


def _coarse(dims, block):
    if any(int(b) < 1 or int(d) % int(b) for d, b in zip(dims, block)):
        raise ValueError(f"blocks {tuple(block)} do not tile {tuple(dims)}")
    return tuple(int(d) // int(b) for d, b in zip(dims, block))


def lqcd_mg_fine_stencil(ctx, V, X, F, B):
    """X (V,12,12), F and B (4,V,12,12) of M = A - kappa D_W on the context's lattice."""
    _check(_lib.lqcd_mg_fine_stencil(ctx, _mg_ptr(X, V * 144, "X"), _mg_ptr(F, 4 * V * 144, "F"),
                                     _mg_ptr(B, 4 * V * 144, "B")))


def lqcd_mg_apply(ctx, dims, n, X, F, B, v, out):
    V = int(np.prod(dims))
    _check(_lib.lqcd_mg_apply(ctx, _i4(dims), int(n), _mg_ptr(X, V * n * n, "X"), _mg_ptr(F, 4 * V * n * n, "F"),
                              _mg_ptr(B, 4 * V * n * n, "B"), _mg_ptr(v, V * n, "in"), _mg_ptr(out, V * n, "out")))


def lqcd_mg_orthonormalize(ctx, dims, n, block, nv, vecs, P):
    V = int(np.prod(dims))
    _check(_lib.lqcd_mg_orthonormalize(ctx, _i4(dims), int(n), _i4(block), int(nv), _mg_ptr(vecs, nv * V * n, "vecs"),
                                       _mg_ptr(P, V * n * 2 * nv, "P")))


def lqcd_mg_prolong(ctx, dims, n, block, nc, P, w, out):
    V, Vc = int(np.prod(dims)), int(np.prod(_coarse(dims, block)))
    _check(_lib.lqcd_mg_prolong(ctx, _i4(dims), int(n), _i4(block), int(nc), _mg_ptr(P, V * n * nc, "P"),
                                _mg_ptr(w, Vc * nc, "w"), _mg_ptr(out, V * n, "out")))


def lqcd_mg_restrict(ctx, dims, n, block, nc, P, v, out):
    V, Vc = int(np.prod(dims)), int(np.prod(_coarse(dims, block)))
    _check(_lib.lqcd_mg_restrict(ctx, _i4(dims), int(n), _i4(block), int(nc), _mg_ptr(P, V * n * nc, "P"),
                                 _mg_ptr(v, V * n, "v"), _mg_ptr(out, Vc * nc, "out")))


def lqcd_mg_coarsen(ctx, dims, n, block, nc, X, F, B, P, Xc, Fc, Bc):
    V, Vc = int(np.prod(dims)), int(np.prod(_coarse(dims, block)))
    _check(_lib.lqcd_mg_coarsen(ctx, _i4(dims), int(n), _i4(block), int(nc), _mg_ptr(X, V * n * n, "X"),
                                _mg_ptr(F, 4 * V * n * n, "F"), _mg_ptr(B, 4 * V * n * n, "B"),
                                _mg_ptr(P, V * n * nc, "P"), _mg_ptr(Xc, Vc * nc * nc, "Xc"),
                                _mg_ptr(Fc, 4 * Vc * nc * nc, "Fc"), _mg_ptr(Bc, 4 * Vc * nc * nc, "Bc")))


def lqcd_mg_dots(ctx, k, Xv, y):
    """[<X_j, y> for j < k] (complex), X_j the first k rows of Xv (each y.numel() long)."""
    n = y.numel()
    out = (ctypes.c_double * (2 * int(k)))()
    _check(_lib.lqcd_mg_dots(ctx, n, int(k), _mg_ptr(Xv, k * n, "X"), _mg_ptr(y, n, "y"), out))
    a = np.array(out[:])
    return a[0::2] + 1j * a[1::2]


def lqcd_mg_axpys(ctx, coef, Xv, y):
    """y += sum_j coef[j] X_j."""
    coef = np.asarray(coef, dtype=np.complex128).reshape(-1)
    k, n = len(coef), y.numel()
    c = np.ascontiguousarray(coef.view(np.float64))
    _check(_lib.lqcd_mg_axpys(ctx, n, k, c.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), _mg_ptr(Xv, k * n, "X"),
                              _mg_ptr(y, n, "y")))


def lqcd_mg_axpby(ctx, a, x, b, y):
    """y = a x + b y (complex scalars)."""
    n = y.numel()
    ca = (ctypes.c_double * 2)(complex(a).real, complex(a).imag)
    cb = (ctypes.c_double * 2)(complex(b).real, complex(b).imag)
    _check(_lib.lqcd_mg_axpby(ctx, n, ca, _mg_ptr(x, n, "x"), cb, _mg_ptr(y, n, "y")))


class Lattice:
    """One context: geometry, gauge field, clover term (thin wrapper)."""

    def __init__(self, dims, t_antiperiodic=1, stream=None):
        self.dims = tuple(int(d) for d in dims)
        self.V = int(np.prod(self.dims))
        self.ctx = lqcd_create(self.dims, t_antiperiodic, stream)

    def close(self):
        if self.ctx is not None:
            lqcd_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def load_gauge(self, U):
        lqcd_load_gauge(self.ctx, U)

    def clover(self, kappa, c_sw):
        lqcd_clover(self.ctx, kappa, c_sw)

    def set_rho(self, rho):
        lqcd_set_rho(self.ctx, rho)

    def dslash(self, psi, op="MHAT", prec="f64", recon=18):
        """op(psi) on canonical complex128 arrays (numpy: host path; torch: device path)."""
        nrhs = psi.size // (12 * self.V) if isinstance(psi, np.ndarray) else psi.numel() // (24 * self.V)
        if isinstance(psi, np.ndarray):
            psi = np.ascontiguousarray(psi, dtype=np.complex128)
            out = np.empty_like(psi)
        else:
            out = psi.new_empty(psi.shape)
        lqcd_dslash(self.ctx, out, psi, nrhs, OPS[op] if isinstance(op, str) else op,
                    PREC[prec] if isinstance(prec, str) else prec, recon)
        return out

    def solve(self, b, tol=1e-10, inner="f64", nrhs=None, **kw):
        b = np.ascontiguousarray(b, dtype=np.complex128)
        if nrhs is None:
            nrhs = b.size // (12 * self.V)
        x = np.zeros_like(b)
        if isinstance(kw.get("outer"), str):
            kw["outer"] = PREC[kw["outer"]]
        prm = solve_params(tol=tol, inner=PREC[inner] if isinstance(inner, str) else inner, nrhs=nrhs, **kw)
        st, info = lqcd_solve(self.ctx, x, b, prm, raise_on_noconv=False)
        return x, st, info
