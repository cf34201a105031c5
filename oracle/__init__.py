"""FP64 CPU oracle for the Wilson-clover / overlap fermion hot path.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package; the library under
``paper_2001_05706_gb300`` never does, and this package never imports it.

The arithmetic is in ``oracle.c`` (plain C99 complex, FP64, full 4x4 spin
matrices, Gauss-Jordan inverses, sequential reductions).  This wrapper
marshals numpy arrays; the overlap-eigensystem functions at its end compose
oracle.c's H_W with numpy's dense Hermitian eigendecomposition (the exact
sign function and the chirality-sector spectrum, small lattices only).  The paper prints no formula; each function follows
the standard definition of the operator the paper names (Table 1:
QUDA_DIRAC_WILSON, QUDA_DIRAC_CLOVER; the overlap inverter of Secs. 1, 3, 4).
Conventions are listed at the top of ``oracle.c``.

Field shapes (complex128, canonical order, x fastest):
  links   (L3, L2, L1, L0, 4, 3, 3)
  spinor  (L3, L2, L1, L0, 4, 3)   -- one right-hand side
  clover  (V, 12, 12)              -- index 3*spin + colour
Parity-restricted vectors are full-lattice arrays that vanish on the other
parity.  ``dims`` is (L0, L1, L2, L3).

Parity pins: every routine here is checked against closed forms,
invariants or brute force by ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_c = np.complex128
_dp = ctypes.POINTER(ctypes.c_double)
_lp = ctypes.POINTER(ctypes.c_long)
_ip = ctypes.POINTER(ctypes.c_int)


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so beside it."""
    src = os.path.join(_HERE, "oracle.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-fopenmp", "-o", tmp, src, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            sig = {
                "or_gamma": ([ctypes.c_int, _dp], None),
                "or_hop": ([_ip, ctypes.c_int, _dp, _dp, _dp, ctypes.c_int], None),
                "or_hop_sites": ([_ip, ctypes.c_int, _dp, _dp, _lp, ctypes.c_long, _dp, ctypes.c_int], None),
                "or_field_strength": ([_ip, _dp, ctypes.c_long, ctypes.c_int, ctypes.c_int, _dp], None),
                "or_clover": ([_ip, _dp, ctypes.c_double, ctypes.c_double, _dp], None),
                "or_clover_sites": ([_ip, _dp, ctypes.c_double, ctypes.c_double, _lp, ctypes.c_long, _dp], None),
                "or_inverse": ([ctypes.c_int, _dp, _dp], ctypes.c_int),
                "or_clover_inverse": ([ctypes.c_long, _dp, _dp], ctypes.c_int),
                "or_site_mul": ([ctypes.c_long, _dp, _dp, _dp], None),
                "or_keep_parity": ([_ip, ctypes.c_int, _dp], None),
                "or_apply_M": ([_ip, ctypes.c_int, _dp, _dp, ctypes.c_double, _dp, _dp, ctypes.c_int], None),
                "or_apply_Mhat": ([_ip, ctypes.c_int, _dp, _dp, _dp, ctypes.c_double, _dp, _dp, ctypes.c_int], None),
                "or_apply_Mhat_sym": ([_ip, ctypes.c_int, _dp, _dp, _dp, ctypes.c_double, _dp, _dp, ctypes.c_int],
                                      None),
                "or_mhat_slab": ([_ip, ctypes.c_int, _dp, _dp, _dp, ctypes.c_double, _dp, ctypes.c_int, ctypes.c_int,
                                  _dp], None),
                "or_prepare_source": ([_ip, ctypes.c_int, _dp, _dp, ctypes.c_double, _dp, _dp], None),
                "or_reconstruct": ([_ip, ctypes.c_int, _dp, _dp, ctypes.c_double, _dp, _dp], None),
                "or_norm2": ([ctypes.c_long, _dp], ctypes.c_double),
                "or_true_residual": ([_ip, ctypes.c_int, _dp, _dp, ctypes.c_double, _dp, _dp], ctypes.c_double),
                "or_cgls": ([_ip, ctypes.c_int, _dp, _dp, _dp, ctypes.c_double, _dp, _dp, ctypes.c_double,
                             ctypes.c_int, _dp], ctypes.c_int),
                "or_solve": ([_ip, ctypes.c_int, _dp, _dp, _dp, ctypes.c_double, _dp, _dp, ctypes.c_double,
                              ctypes.c_int, _dp], ctypes.c_int),
                "or_apply_DW": ([_ip, ctypes.c_int, _dp, ctypes.c_double, _dp, _dp], None),
                "or_apply_gamma5": ([ctypes.c_long, _dp, _dp], None),
                "or_apply_HW": ([_ip, ctypes.c_int, _dp, ctypes.c_double, _dp, _dp], None),
                "or_cheb_coeffs": ([ctypes.c_double, ctypes.c_double, ctypes.c_int, _dp], None),
                "or_cheb_eval": ([ctypes.c_double, ctypes.c_double, ctypes.c_int, _dp, ctypes.c_double],
                                 ctypes.c_double),
                "or_sign_error": ([ctypes.c_double, ctypes.c_double, ctypes.c_int, _dp, ctypes.c_int],
                                  ctypes.c_double),
                "or_cheb_degree": ([ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                    _dp], ctypes.c_int),
                "or_apply_sign": ([_ip, ctypes.c_int, _dp, ctypes.c_double, ctypes.c_int, _dp, _dp, ctypes.c_double,
                                   ctypes.c_double, ctypes.c_int, _dp, _dp, _dp], None),
                "or_apply_overlap": ([_ip, ctypes.c_int, _dp, ctypes.c_double, ctypes.c_double, ctypes.c_int, _dp,
                                      _dp, ctypes.c_double, ctypes.c_double, ctypes.c_int, _dp, _dp, _dp,
                                      ctypes.c_int], None),
            }
            for name, (args, res) in sig.items():
                f = getattr(lib, name)
                f.argtypes = args
                f.restype = res
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    if not a.flags.c_contiguous:
        raise ValueError("array must be C-contiguous")
    if a.dtype == np.complex128:
        return a.ctypes.data_as(_dp)
    if a.dtype == np.float64:
        return a.ctypes.data_as(_dp)
    raise TypeError(a.dtype)


def _dims(dims):
    L = [int(d) for d in dims]
    return (ctypes.c_int * 4)(*L), L[0] * L[1] * L[2] * L[3]


def _field(psi, V):
    a = np.ascontiguousarray(psi, dtype=_c)
    if a.size != 12 * V:
        raise ValueError(f"spinor has {a.size} complex numbers, expected {12 * V}")
    return a


def _links(U, V):
    a = np.ascontiguousarray(U, dtype=_c)
    if a.size != 36 * V:
        raise ValueError("gauge field size mismatch")
    return a


def _opt(A):
    return None if A is None else _p(A)


# ----------------------------------------------------------------------------
# geometry helpers (pure index arithmetic)
# ----------------------------------------------------------------------------

def spinor_shape(dims):
    return (dims[3], dims[2], dims[1], dims[0], 4, 3)


def site_coords(dims, s):
    s = np.asarray(s)
    x0 = s % dims[0]
    x1 = (s // dims[0]) % dims[1]
    x2 = (s // (dims[0] * dims[1])) % dims[2]
    x3 = s // (dims[0] * dims[1] * dims[2])
    return x0, x1, x2, x3


def parity_mask(dims):
    """Boolean array (L3, L2, L1, L0): True on odd sites."""
    x3, x2, x1, x0 = np.meshgrid(*(np.arange(dims[k]) for k in (3, 2, 1, 0)), indexing="ij")
    return ((x0 + x1 + x2 + x3) & 1).astype(bool)


def keep_parity(dims, psi, parity):
    out = np.array(psi, dtype=_c, copy=True).reshape(spinor_shape(dims))
    odd = parity_mask(dims)
    out[odd != bool(parity)] = 0
    return out


def gamma(mu: int) -> np.ndarray:
    out = np.empty((4, 4), dtype=_c)
    _load().or_gamma(mu, _p(out))
    return out


# ----------------------------------------------------------------------------
# Wilson-clover operator
# ----------------------------------------------------------------------------

def hop(dims, U, psi, tbc=1, dagger=False):
    """(D psi)(x) = sum_mu (1-g_mu) U_mu(x) psi(x+mu) + (1+g_mu) U_mu(x-mu)^dag psi(x-mu)."""
    Ld, V = _dims(dims)
    U = _links(U, V)
    psi = _field(psi, V)
    out = np.empty(spinor_shape(dims), dtype=_c)
    _load().or_hop(Ld, int(tbc), _p(U), _p(psi), _p(out), int(dagger))
    return out


def hop_sites(dims, U, psi, sites, tbc=1, dagger=False):
    """(D psi) at the given lexicographic sites only: shape (n, 4, 3)."""
    Ld, V = _dims(dims)
    U = _links(U, V)
    psi = _field(psi, V)
    sites = np.ascontiguousarray(sites, dtype=np.int64)
    out = np.empty((len(sites), 4, 3), dtype=_c)
    _load().or_hop_sites(Ld, int(tbc), _p(U), _p(psi), sites.ctypes.data_as(_lp), len(sites), _p(out), int(dagger))
    return out


def field_strength(dims, U, s, mu, nu):
    Ld, V = _dims(dims)
    U = _links(U, V)
    out = np.empty((3, 3), dtype=_c)
    _load().or_field_strength(Ld, _p(U), int(s), int(mu), int(nu), _p(out))
    return out


def clover(dims, U, kappa, csw):
    """A(x) = 1 - csw*kappa*sum_{mu<nu} sigma_munu F_munu(x), shape (V, 12, 12)."""
    Ld, V = _dims(dims)
    U = _links(U, V)
    out = np.empty((V, 12, 12), dtype=_c)
    _load().or_clover(Ld, _p(U), float(kappa), float(csw), _p(out))
    return out


def clover_sites(dims, U, kappa, csw, sites):
    Ld, V = _dims(dims)
    U = _links(U, V)
    sites = np.ascontiguousarray(sites, dtype=np.int64)
    out = np.empty((len(sites), 12, 12), dtype=_c)
    _load().or_clover_sites(Ld, _p(U), float(kappa), float(csw), sites.ctypes.data_as(_lp), len(sites), _p(out))
    return out


def inverse(M):
    M = np.ascontiguousarray(M, dtype=_c)
    n = M.shape[0]
    out = np.empty_like(M)
    if _load().or_inverse(n, _p(M), _p(out)) != 0:
        raise np.linalg.LinAlgError("singular matrix")
    return out


def clover_inverse(A):
    A = np.ascontiguousarray(A, dtype=_c)
    out = np.empty_like(A)
    if _load().or_clover_inverse(A.shape[0], _p(A), _p(out)) != 0:
        raise np.linalg.LinAlgError("singular clover block")
    return out


def site_mul(A, psi):
    """out(x) = A(x) psi(x); A is (V,12,12) or None (identity)."""
    psi = np.ascontiguousarray(psi, dtype=_c)
    V = psi.size // 12
    out = np.empty_like(psi)
    _load().or_site_mul(V, _opt(A), _p(psi), _p(out))
    return out


def apply_M(dims, U, A, kappa, psi, tbc=1, dagger=False):
    """M psi = A psi - kappa D psi (A None means c_sw = 0)."""
    Ld, V = _dims(dims)
    U = _links(U, V)
    psi = _field(psi, V)
    out = np.empty(spinor_shape(dims), dtype=_c)
    _load().or_apply_M(Ld, int(tbc), _p(U), _opt(A), float(kappa), _p(psi), _p(out), int(dagger))
    return out


def apply_Mhat(dims, U, A, Ainv, kappa, psi, tbc=1, dagger=False):
    """Mhat psi_o = A_oo psi_o - kappa^2 D_oe A_ee^-1 D_eo psi_o (or its adjoint)."""
    Ld, V = _dims(dims)
    U = _links(U, V)
    psi = keep_parity(dims, _field(psi, V), 1)
    out = np.empty(spinor_shape(dims), dtype=_c)
    _load().or_apply_Mhat(Ld, int(tbc), _p(U), _opt(A), _opt(Ainv), float(kappa), _p(psi), _p(out), int(dagger))
    return out


def apply_Mhat_sym(dims, U, A, Ainv, kappa, psi, tbc=1, dagger=False):
    """Symmetric even-odd Schur complement A_oo^-1 Mhat psi_o (or its adjoint
    Mhat^dag A_oo^-1 psi_o); the standard alternative to the asymmetric form of
    the even-odd preconditioned clover operator in the QUDA inverters (Sec. 3)."""
    Ld, V = _dims(dims)
    U = _links(U, V)
    psi = keep_parity(dims, _field(psi, V), 1)
    out = np.empty(spinor_shape(dims), dtype=_c)
    _load().or_apply_Mhat_sym(Ld, int(tbc), _p(U), _opt(A), _opt(Ainv), float(kappa), _p(psi), _p(out), int(dagger))
    return out


def mhat_slab(dims, U, A, Ainv, kappa, psi, t0, t1, out=None, tbc=1):
    """Mhat psi_o on the odd sites of time slices t0 <= t < t1 only (a bounded
    piece of the full application; the other sites of ``out`` are untouched)."""
    Ld, V = _dims(dims)
    U = _links(U, V)
    psi = _field(psi, V)
    if out is None:
        out = np.zeros(spinor_shape(dims), dtype=_c)
    if not (0 <= t0 < t1 <= dims[3]):
        raise ValueError("need 0 <= t0 < t1 <= L3")
    _load().or_mhat_slab(Ld, int(tbc), _p(U), _opt(A), _opt(Ainv), float(kappa), _p(psi), int(t0), int(t1), _p(out))
    return out


def prepare_source(dims, U, Ainv, kappa, b, tbc=1):
    Ld, V = _dims(dims)
    U = _links(U, V)
    b = _field(b, V)
    out = np.empty(spinor_shape(dims), dtype=_c)
    _load().or_prepare_source(Ld, int(tbc), _p(U), _opt(Ainv), float(kappa), _p(b), _p(out))
    return out


def reconstruct(dims, U, Ainv, kappa, b, x_odd, tbc=1):
    Ld, V = _dims(dims)
    U = _links(U, V)
    b = _field(b, V)
    x = np.array(_field(x_odd, V), copy=True).reshape(spinor_shape(dims))
    _load().or_reconstruct(Ld, int(tbc), _p(U), _opt(Ainv), float(kappa), _p(b), _p(x))
    return x


def norm2(v):
    v = np.ascontiguousarray(v, dtype=_c)
    return _load().or_norm2(v.size, _p(v))


def true_residual(dims, U, A, kappa, x, b, tbc=1):
    """||b - M x|| / ||b|| on the full lattice."""
    Ld, V = _dims(dims)
    U = _links(U, V)
    x = _field(x, V)
    b = _field(b, V)
    return _load().or_true_residual(Ld, int(tbc), _p(U), _opt(A), float(kappa), _p(x), _p(b))


def cgls(dims, U, A, Ainv, kappa, bhat, x0=None, tol=1e-10, max_iter=10000, tbc=1):
    """CG on the normal equations of Mhat x = bhat.  Returns (x, iters, rel_resid)."""
    Ld, V = _dims(dims)
    U = _links(U, V)
    bhat = keep_parity(dims, _field(bhat, V), 1)
    x = np.zeros(spinor_shape(dims), dtype=_c) if x0 is None else keep_parity(dims, x0, 1)
    res = ctypes.c_double(0)
    it = _load().or_cgls(Ld, int(tbc), _p(U), _opt(A), _opt(Ainv), float(kappa), _p(bhat), _p(x), float(tol),
                         int(max_iter), ctypes.byref(res))
    return x, it, res.value


def solve(dims, U, A, Ainv, kappa, b, tol=1e-10, max_iter=10000, tbc=1):
    """M x = b via even-odd preconditioned CGLS.  Returns (x, iters, rel_resid_hat)."""
    Ld, V = _dims(dims)
    U = _links(U, V)
    b = _field(b, V)
    x = np.zeros(spinor_shape(dims), dtype=_c)
    res = ctypes.c_double(0)
    it = _load().or_solve(Ld, int(tbc), _p(U), _opt(A), _opt(Ainv), float(kappa), _p(b), _p(x), float(tol),
                          int(max_iter), ctypes.byref(res))
    return x, it, res.value


# ----------------------------------------------------------------------------
# overlap
# ----------------------------------------------------------------------------

def apply_DW(dims, U, m, psi, tbc=1):
    Ld, V = _dims(dims)
    U = _links(U, V)
    psi = _field(psi, V)
    out = np.empty(spinor_shape(dims), dtype=_c)
    _load().or_apply_DW(Ld, int(tbc), _p(U), float(m), _p(psi), _p(out))
    return out


def gamma5(psi):
    psi = np.ascontiguousarray(psi, dtype=_c)
    out = np.empty_like(psi)
    _load().or_apply_gamma5(psi.size // 12, _p(psi), _p(out))
    return out


def apply_HW(dims, U, rho, psi, tbc=1):
    """H_W psi = gamma5 D_W(-rho) psi."""
    Ld, V = _dims(dims)
    U = _links(U, V)
    psi = _field(psi, V)
    out = np.empty(spinor_shape(dims), dtype=_c)
    _load().or_apply_HW(Ld, int(tbc), _p(U), float(rho), _p(psi), _p(out))
    return out


def cheb_coeffs(a, b, n):
    c = np.empty(n + 1)
    _load().or_cheb_coeffs(float(a), float(b), int(n), _p(c))
    return c


def cheb_eval(a, b, c, y):
    c = np.ascontiguousarray(c, dtype=np.float64)
    return _load().or_cheb_eval(float(a), float(b), len(c) - 1, _p(c), float(y))


def sign_error(a, b, c, npts=100000):
    c = np.ascontiguousarray(c, dtype=np.float64)
    return _load().or_sign_error(float(a), float(b), len(c) - 1, _p(c), int(npts))


def cheb_degree(a, b, tol, nmax=20000, npts=100000):
    """Smallest degree whose sup |x P(x^2) - sign x| <= tol on [sqrt a, sqrt b]."""
    c = np.empty(nmax + 1)
    n = _load().or_cheb_degree(float(a), float(b), float(tol), int(nmax), int(npts), _p(c))
    if n < 0:
        raise ValueError("no degree below nmax reaches the tolerance")
    return n, c[: n + 1].copy()


def _lowmodes(nlow, lam, vecs, V):
    if nlow == 0:
        return np.zeros(1), np.zeros(12, dtype=_c)
    lam = np.ascontiguousarray(lam[:nlow], dtype=np.float64)
    vecs = np.ascontiguousarray(np.asarray(vecs[:nlow], dtype=_c).reshape(nlow, 12 * V))
    return lam, vecs


def apply_sign(dims, U, rho, psi, a, b, c, lam=(), vecs=(), tbc=1):
    """eps(H_W) psi with exact low modes and the Chebyshev series elsewhere."""
    Ld, V = _dims(dims)
    U = _links(U, V)
    psi = _field(psi, V)
    nlow = len(lam)
    lam_a, vec_a = _lowmodes(nlow, lam, vecs, V)
    c = np.ascontiguousarray(c, dtype=np.float64)
    out = np.empty(spinor_shape(dims), dtype=_c)
    _load().or_apply_sign(Ld, int(tbc), _p(U), float(rho), nlow, _p(lam_a), _p(vec_a), float(a), float(b),
                          len(c) - 1, _p(c), _p(psi), _p(out))
    return out


def apply_overlap(dims, U, rho, m, psi, a, b, c, lam=(), vecs=(), tbc=1, dagger=False):
    """D_ov(m) psi = (1 - m/(2 rho)) rho (1 + g5 eps(H_W)) psi + m psi."""
    Ld, V = _dims(dims)
    U = _links(U, V)
    psi = _field(psi, V)
    nlow = len(lam)
    lam_a, vec_a = _lowmodes(nlow, lam, vecs, V)
    c = np.ascontiguousarray(c, dtype=np.float64)
    out = np.empty(spinor_shape(dims), dtype=_c)
    _load().or_apply_overlap(Ld, int(tbc), _p(U), float(rho), float(m), nlow, _p(lam_a), _p(vec_a), float(a),
                             float(b), len(c) - 1, _p(c), _p(psi), _p(out), int(dagger))
    return out


def hw_dense(dims, U, rho, tbc=1):
    """The dense matrix of H_W, built column by column (small lattices only)."""
    V = int(np.prod(dims))
    N = 12 * V
    shape = spinor_shape(dims)
    H = np.empty((N, N), dtype=_c)
    e = np.zeros(N, dtype=_c)
    for j in range(N):
        e[j] = 1.0
        H[:, j] = apply_HW(dims, U, rho, e.reshape(shape), tbc).reshape(N)
        e[j] = 0.0
    return H


def low_modes_dense(dims, U, rho, k, tbc=1):
    """The k eigenpairs of H_W with smallest |lambda|, sorted by |lambda|, from
    a dense Hermitian eigendecomposition (numpy eigh) of the brute-force matrix.
    Small lattices only; larger eigenpairs are verified by their residuals
    (``eigen_residuals``) instead of being recomputed here."""
    H = hw_dense(dims, U, rho, tbc)
    H = 0.5 * (H + H.conj().T)
    lam, Vec = np.linalg.eigh(H)
    order = np.argsort(np.abs(lam), kind="stable")[:k]
    return lam[order], Vec[:, order].T.reshape((k,) + spinor_shape(dims)).copy()


def eigen_residuals(dims, U, rho, lam, vecs, tbc=1):
    """||H_W v_i - lam_i v_i|| for each pair, and max |<v_i, v_j> - delta_ij|."""
    k = len(lam)
    res = np.array([np.linalg.norm((apply_HW(dims, U, rho, vecs[i], tbc) - lam[i] * vecs[i]).ravel())
                    for i in range(k)])
    Z = np.asarray(vecs).reshape(k, -1)
    ortho = np.abs(Z.conj() @ Z.T - np.eye(k)).max()
    return res, ortho


# ---- overlap eigensystem (Sec. 4: the low eigenpairs of D_ov) ---------------
#
# D_ov(0) = rho (1 + g5 eps) is normal and g5-Hermitian, so D_ov(0)^dag D_ov(0)
# commutes with g5: its eigenvectors can be taken chiral, and on the chirality
# sector s (P_s = (1 + s g5)/2) it is 2 rho^2 P_s (1 + s eps) P_s.  A vector
# chi of sector s with eigenvalue mu belongs to the pair of D_ov(0)
# eigenvalues lambda = mu / (2 rho) +- i sqrt(mu - mu^2 / (4 rho^2)).

def chirality_indices(dims, sector):
    """Flattened canonical-spinor indices of chirality sector s: spins 0, 1
    (s = +1) or 2, 3 (s = -1), g5 = diag(1, 1, -1, -1) in the DeGrand-Rossi
    basis."""
    V = int(np.prod(dims))
    spin = np.tile(np.repeat(np.arange(4), 3), V)
    return np.nonzero(spin < 2 if sector > 0 else spin >= 2)[0]


def overlap_dense(dims, U, rho, m=0.0, tbc=1):
    """The dense matrix of D_ov(m) = (1 - m/(2 rho)) rho (1 + g5 eps(H_W)) + m
    with the exact sign function eps = Q sign(Lambda) Q^H of a dense
    eigendecomposition of H_W (small lattices only)."""
    H = hw_dense(dims, U, rho, tbc)
    H = 0.5 * (H + H.conj().T)
    lam, Q = np.linalg.eigh(H)
    eps = (Q * np.sign(lam)) @ Q.conj().T
    N = H.shape[0]
    g5 = np.ones(N)
    g5[chirality_indices(dims, -1)] = -1.0
    return (1.0 - m / (2.0 * rho)) * rho * (np.eye(N) + g5[:, None] * eps) + m * np.eye(N)


def overlap_sector_eigensystem(dims, U, rho, k, sector, tbc=1):
    """The k lowest eigenpairs (mu_i, chi_i) of D_ov(0)^dag D_ov(0) on the
    chirality-s subspace (dense Hermitian eigendecomposition of the restricted
    matrix), ascending; chi_i returned as full spinors, zero in the other
    chirality."""
    D = overlap_dense(dims, U, rho, 0.0, tbc)
    idx = chirality_indices(dims, sector)
    M = (D.conj().T @ D)[np.ix_(idx, idx)]
    M = 0.5 * (M + M.conj().T)
    mu, W = np.linalg.eigh(M)
    N = D.shape[0]
    vecs = np.zeros((k, N), dtype=_c)
    vecs[:, idx] = W[:, :k].T
    return mu[:k], vecs.reshape((k,) + spinor_shape(dims))


def apply_sector_normal(dims, U, rho, sector, chi, a, b, c, lam=(), vecs=(), tbc=1):
    """P_s D_ov(0)^dag D_ov(0) P_s chi = 2 rho^2 P_s (chi + s eps chi), with the
    polynomial sign function of apply_sign (the operator the GPU eigensolver
    uses)."""
    chi = np.array(chi, dtype=_c)
    keep = spinor_shape(dims)[-2]  # 4 spins
    mask = np.zeros(keep, dtype=bool)
    mask[[0, 1] if sector > 0 else [2, 3]] = True
    chi[..., ~mask, :] = 0
    e = apply_sign(dims, U, rho, chi, a, b, c, lam=lam, vecs=vecs, tbc=tbc)
    out = 2.0 * rho * rho * (chi + sector * e)
    out[..., ~mask, :] = 0
    return out


def overlap_pair_eigenvalues(mu, rho):
    """The eigenvalue pair lambda = re +- i im of D_ov(0) belonging to the
    D_ov(0)^dag D_ov(0) eigenvalue mu (0 <= mu <= 4 rho^2)."""
    mu = np.asarray(mu, dtype=np.float64)
    re = mu / (2.0 * rho)
    return re, np.sqrt(np.maximum(mu - re * re, 0.0))
