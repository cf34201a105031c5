"""GPU overlap operator against the FP64 oracle: low modes of H_W (vs dense
eigh), the polynomial sign function and D_ov (vs the oracle's evaluation with
the same projected modes and interval), the free-field closed form, the
Ginsparg-Wilson relation and the overlap solve (true residual recomputed by
the oracle).  Each runs with the FP64 parts in FP64 and in double-float
(high = LQCD_DF64), to the same tolerances."""
import numpy as np
import pytest

import gen
import oracle
from helpers import all_momenta, momenta, plane_wave, rel

pytestmark = pytest.mark.gpu
RHO = 1.5
BMAX = 6.5 ** 2


@pytest.fixture(scope="module")
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2001_05706_gb300 as L
    return L


def _setup(L, dims, U, n_low, mass=0.0, sign_tol=1e-12, high="f64", eig_method="subspace", max_filter=200):
    lat = L.Lattice(dims)
    lat.load_gauge(U.view(np.float64))
    prm = L.overlap_params(rho=RHO, mass=mass, n_low=n_low, sign_tol=sign_tol, eig_tol=1e-11, high=high,
                           eig_method=eig_method, max_filter=max_filter)
    st, info = L.lqcd_overlap_setup(lat.ctx, prm)
    vecs = np.zeros((n_low,) + oracle.spinor_shape(dims), dtype=np.complex128)
    if n_low:
        L.lqcd_overlap_lowmodes(lat.ctx, vecs)
    lam = np.array(info.lambda_[:n_low])
    return lat, info, lam, vecs


def _ov(L, lat, psi, op, nrhs=1, cg=None):
    out = np.zeros_like(psi)
    L.lqcd_overlap(lat.ctx, out, np.ascontiguousarray(psi), nrhs, op, cg)
    return out


@pytest.fixture(scope="module", params=[("f64", "subspace"), ("df64", "subspace"), ("f64", "lanczos"),
                                        ("df64", "lanczos")],
                ids=["f64-subspace", "df64-subspace", "f64-lanczos", "df64-lanczos"])
def rough(lib, request):
    dims = (4, 4, 4, 4)
    U = gen.gauge_field(dims, 0.3, 23)
    lat, info, lam, vecs = _setup(lib, dims, U, 8, high=request.param[0], eig_method=request.param[1])
    yield dims, U, lat, info, lam, vecs
    lat.close()


def test_low_modes_against_dense(rough):
    dims, U, lat, info, lam, vecs = rough
    lo, _ = oracle.low_modes_dense(dims, U, RHO, 8)
    assert np.allclose(np.abs(lam), np.abs(lo), atol=1e-10)
    assert np.allclose(np.sort(lam), np.sort(lo), atol=1e-10)  # signs too
    res, ortho = oracle.eigen_residuals(dims, U, RHO, lam, vecs)
    assert res.max() < 1e-10 and ortho < 1e-10
    assert info.degree > 0 and info.sign_error <= 1e-12
    # the FP32 sign function of the mixed CG stops at its rounding level
    assert 0 < info.degree_inner < info.degree


def test_sign_and_overlap_against_oracle(rough, lib):
    L = lib
    dims, U, lat, info, lam, vecs = rough
    psi = gen.gaussian_spinor(dims, 5)[0]
    a, b = info.a, info.b
    n, c = oracle.cheb_degree(a, b, 1e-12)
    eps_or = oracle.apply_sign(dims, U, RHO, psi, a, b, c, lam=lam, vecs=vecs)
    eps_gpu = _ov(L, lat, psi, L.LQCD_OV_SIGN)
    assert rel(eps_gpu, eps_or) < 1e-10
    # sign(H)^2 = 1 and the exact dense sign
    assert rel(_ov(L, lat, eps_gpu, L.LQCD_OV_SIGN), psi) < 1e-10
    H = oracle.hw_dense(dims, U, RHO)
    w, V = np.linalg.eigh(0.5 * (H + H.conj().T))
    exact = (V @ (np.sign(w) * (V.conj().T @ psi.reshape(-1)))).reshape(psi.shape)
    assert rel(eps_gpu, exact) < 1e-10
    # D_ov and its adjoint (massless here; the solve test uses a mass)
    d_or = oracle.apply_overlap(dims, U, RHO, 0.0, psi, a, b, c, lam=lam, vecs=vecs)
    assert rel(_ov(L, lat, psi, L.LQCD_OV_APPLY), d_or) < 1e-10
    dd_or = oracle.apply_overlap(dims, U, RHO, 0.0, psi, a, b, c, lam=lam, vecs=vecs, dagger=True)
    assert rel(_ov(L, lat, psi, L.LQCD_OV_APPLY_DAG), dd_or) < 1e-10


def test_ginsparg_wilson_on_gpu(rough, lib):
    L = lib
    dims, U, lat, info, lam, vecs = rough
    v = gen.gaussian_spinor(dims, 12)[0]
    D = lambda x: _ov(L, lat, x, L.LQCD_OV_APPLY)
    g5 = oracle.gamma5
    assert rel(g5(D(v)) + D(g5(v)), D(g5(D(v))) / RHO) < 1e-10


def test_multi_rhs_sign(rough, lib):
    L = lib
    dims, U, lat, info, lam, vecs = rough
    psi = gen.gaussian_spinor(dims, 31, nrhs=3)
    out = _ov(L, lat, psi, L.LQCD_OV_SIGN, nrhs=3)
    for k in range(3):
        assert rel(out[k], _ov(L, lat, psi[k], L.LQCD_OV_SIGN)) < 1e-12


@pytest.mark.parametrize("high", ["f64", "df64"])
def test_free_field_closed_form(lib, high):
    L = lib
    dims = (4, 4, 4, 4)
    U = gen.unit_gauge(dims)
    lat, info, lam, vecs = _setup(L, dims, U, 4, mass=0.05, high=high)
    # the low modes: |lambda| = min_p N(p), the bottom of a 24-fold cluster
    # (wider than the starting block, which must grow to hold it whole)
    nmin = min(np.sqrt((4 - RHO - np.cos(p).sum()) ** 2 + (np.sin(p) ** 2).sum()) for p in all_momenta(dims, 1))
    assert np.allclose(np.abs(lam), nmin, atol=1e-10)
    assert max(info.resid[:4]) <= 1e-11
    res, ortho = oracle.eigen_residuals(dims, U, RHO, lam, vecs)
    assert res.max() <= 1e-10 and ortho < 1e-10
    g = [oracle.gamma(mu) for mu in range(4)]
    m = 0.05
    rng = np.random.default_rng(2)
    for nn in [(0, 0, 0, 0), (1, 2, 0, 3), (2, 2, 2, 1)]:
        p = momenta(dims, nn, 1)
        u = rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))
        psi = plane_wave(dims, p, u)
        N = np.sqrt((4 - RHO - np.cos(p).sum()) ** 2 + (np.sin(p) ** 2).sum())
        DW = (4 - RHO - np.cos(p).sum()) * np.eye(4) + 1j * sum(g[mu] * np.sin(p[mu]) for mu in range(4))
        Dov = (1 - m / (2 * RHO)) * RHO * (np.eye(4) + DW / N) + m * np.eye(4)
        assert rel(_ov(L, lat, psi, L.LQCD_OV_APPLY), plane_wave(dims, p, Dov @ u)) < 1e-10
    lat.close()


@pytest.mark.parametrize("inner,high", [("f64", "f64"), ("f32", "f64"), ("f64", "df64"), ("f32", "df64")])
def test_overlap_solve(lib, inner, high):
    L = lib
    dims = (4, 4, 4, 8)
    U = gen.gauge_field(dims, 0.1, 5)
    m = 0.05
    lat, info, lam, vecs = _setup(L, dims, U, 6, mass=m, high=high)
    b = gen.gaussian_spinor(dims, 2005, nrhs=2)
    cg = L.solve_params(tol=1e-10, max_iter=2000, nrhs=2, inner=L.PREC[inner], delta=0.1)
    x = np.zeros_like(b)
    st, sinfo = L.lqcd_overlap(lat.ctx, x, b, 2, L.LQCD_OV_SOLVE, cg)
    assert st == L.LQCD_OK
    if inner == "f32":
        assert sinfo.reliable_updates >= 1
    n, c = oracle.cheb_degree(info.a, info.b, 1e-12)
    for k in range(2):
        r = b[k] - oracle.apply_overlap(dims, U, RHO, m, x[k], info.a, info.b, c, lam=lam, vecs=vecs)
        assert np.linalg.norm(r) / np.linalg.norm(b[k]) <= 1e-10
    lat.close()


def test_overlap_rejects_bad_high_precision(lib):
    L = lib
    dims = (4, 4, 4, 4)
    lat = L.Lattice(dims)
    lat.load_gauge(gen.gauge_field(dims, 0.3, 23).view(np.float64))
    prm = L.overlap_params(rho=RHO, n_low=2, high=L.LQCD_F32)
    with pytest.raises(L.LqcdError) as e:
        L.lqcd_overlap_setup(lat.ctx, prm)
    assert e.value.status == L.LQCD_ERR_ARG
    lat.close()


@pytest.mark.parametrize("high", ["f64", "df64"])
def test_lanczos_matches_subspace_iteration(lib, high):
    """Thick-restart Lanczos and block subspace iteration find the same 12 low
    modes of H_W on a smooth 8^4 field (clustered spectrum), each to an
    eigen-residual below 1e-10 recomputed by the oracle, and Lanczos applies
    H_W fewer times."""
    L = lib
    dims = (8, 8, 8, 8)
    U = gen.gauge_field(dims, 0.1, 31)
    res = {}
    for method in ("subspace", "lanczos"):
        lat, info, lam, vecs = _setup(L, dims, U, 12, sign_tol=1e-10, high=high, eig_method=method, max_filter=2000)
        r, ortho = oracle.eigen_residuals(dims, U, RHO, lam, vecs)
        assert r.max() < 1e-10 and ortho < 1e-10, method
        res[method] = (np.sort(lam), info.hw_applies, info.sweeps)
        lat.close()
    assert np.allclose(res["lanczos"][0], res["subspace"][0], atol=1e-10)
    assert 0 < res["lanczos"][1] < res["subspace"][1]


def test_overlap_rejects_bad_eig_method(lib):
    L = lib
    dims = (4, 4, 4, 4)
    lat = L.Lattice(dims)
    lat.load_gauge(gen.gauge_field(dims, 0.3, 23).view(np.float64))
    prm = L.overlap_params(rho=RHO, n_low=2, eig_method=5)
    with pytest.raises(L.LqcdError) as e:
        L.lqcd_overlap_setup(lat.ctx, prm)
    assert e.value.status == L.LQCD_ERR_ARG
    lat.close()


@pytest.mark.parametrize("high,method", [("f64", "subspace"), ("df64", "subspace"), ("f64", "lanczos"),
                                         ("df64", "lanczos")])
def test_twenty_mode_contract(lib, high, method):
    """20 low modes on a smooth 8^3x16 field (a clustered spectrum, as on the
    16^3x32 overlap workload): every returned mode meets eig_tol as an
    eigenpair of H_W itself, recomputed by the oracle, not only its H_W^2
    residual inside the solver."""
    L = lib
    dims = (8, 8, 8, 16)
    U = gen.gauge_field(dims, 0.1, 1005)
    eig_tol = 1e-10
    lat = L.Lattice(dims)
    lat.load_gauge(U.view(np.float64))
    prm = L.overlap_params(rho=RHO, mass=0.05, n_low=20, sign_tol=1e-10, eig_tol=eig_tol, high=high,
                           eig_method=method, max_filter=800)
    st, info = L.lqcd_overlap_setup(lat.ctx, prm)
    assert st == L.LQCD_OK
    vecs = np.zeros((20,) + oracle.spinor_shape(dims), dtype=np.complex128)
    L.lqcd_overlap_lowmodes(lat.ctx, vecs)
    lam = np.array(info.lambda_[:20])
    res, ortho = oracle.eigen_residuals(dims, U, RHO, lam, vecs)
    assert res.max() <= eig_tol, res
    assert max(info.resid[:20]) <= eig_tol
    assert ortho < 1e-10
    assert np.all(np.diff(np.abs(lam)) >= -1e-12)  # sorted by |lambda|
    lat.close()


def test_unconverged_setup_is_refused(lib):
    """A set-up that returns NOCONV leaves no usable state: the overlap
    operator and the low-mode export refuse to run on inexact eigenvectors."""
    L = lib
    dims = (4, 4, 4, 4)
    U = gen.gauge_field(dims, 0.3, 23)
    lat = L.Lattice(dims)
    lat.load_gauge(U.view(np.float64))
    prm = L.overlap_params(rho=RHO, n_low=8, sign_tol=1e-10, eig_tol=1e-13, max_filter=1)
    st, info = L.lqcd_overlap_setup(lat.ctx, prm, raise_on_noconv=False)
    assert st == L.LQCD_ERR_NOCONV
    psi = gen.gaussian_spinor(dims, 5)[0]
    with pytest.raises(L.LqcdError) as e:
        _ov(L, lat, psi, L.LQCD_OV_APPLY)
    assert e.value.status == L.LQCD_ERR_STATE
    with pytest.raises(L.LqcdError) as e:
        L.lqcd_overlap_lowmodes(lat.ctx, np.zeros((8,) + oracle.spinor_shape(dims), dtype=np.complex128))
    assert e.value.status == L.LQCD_ERR_STATE
    # a converged set-up on the same context makes it usable again
    prm = L.overlap_params(rho=RHO, n_low=8, sign_tol=1e-10, eig_tol=1e-11, max_filter=200)
    st, info = L.lqcd_overlap_setup(lat.ctx, prm)
    assert st == L.LQCD_OK
    assert np.isfinite(_ov(L, lat, psi, L.LQCD_OV_APPLY)).all()
    lat.close()
