"""The overlap eigensystem (the low eigenpairs of D_ov(0)^dag D_ov(0) in one
chirality sector, Sec. 4) and the deflated overlap CG, against the oracle:
eigenvalues against the dense chirality-sector spectrum, every vector and its
partner against the oracle's sector operator with the set-up's own sign
function (residuals recomputed on the CPU), chirality and orthonormality, and
deflated solves to an oracle-recomputed true residual in fewer iterations."""
import numpy as np
import pytest

import gen
import oracle

pytestmark = pytest.mark.gpu
RHO = 1.5


@pytest.fixture(scope="module")
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2001_05706_gb300 as L
    return L


def _setup(L, dims, U, n_low, mass=0.0, high="f64"):
    lat = L.Lattice(dims)
    lat.load_gauge(U.view(np.float64))
    prm = L.overlap_params(rho=RHO, mass=mass, n_low=n_low, sign_tol=1e-12, eig_tol=1e-11, high=high,
                           eig_method="lanczos", max_filter=400)
    st, info = L.lqcd_overlap_setup(lat.ctx, prm)
    vecs = np.zeros((n_low,) + oracle.spinor_shape(dims), dtype=np.complex128)
    L.lqcd_overlap_lowmodes(lat.ctx, vecs)
    n, c = oracle.cheb_degree(info.a, info.b, 1e-12)
    return lat, dict(a=info.a, b=info.b, c=c, lam=np.array(info.lambda_[:n_low]), vecs=vecs)


DIMS = (4, 4, 2, 4)  # 128 sites: the dense oracle's sector matrices are 768 x 768


@pytest.fixture(scope="module")
def field():
    U = gen.gauge_field(DIMS, 0.4, 61)
    dense = {s: oracle.overlap_sector_eigensystem(DIMS, U, RHO, 40, s) for s in (+1, -1)}
    return U, dense


@pytest.mark.parametrize("high", ["f64", "df64"])
@pytest.mark.parametrize("sector", [+1, -1])
def test_eigensystem_against_the_oracle(lib, field, sector, high):
    L = lib
    U, dense = field
    n_ev, tol = 24, 1e-9
    lat, sg = _setup(L, DIMS, U, 6, high=high)
    st, info = L.lqcd_overlap_eigen(lat.ctx, L.overlap_eigen_params(n_ev=n_ev, sector=sector, tol=tol))
    assert st == L.LQCD_OK and info.n_ev == n_ev
    mu = np.array(info.mu[:n_ev])
    assert np.all(np.diff(mu) >= -1e-12)
    assert np.allclose(mu, dense[sector][0][:n_ev], atol=1e-8, rtol=0)
    assert max(info.resid[:n_ev]) <= tol
    re, im = oracle.overlap_pair_eigenvalues(mu, RHO)
    assert np.allclose(info.lambda_re[:n_ev], re) and np.allclose(info.lambda_im[:n_ev], im)
    chi = np.zeros((n_ev,) + oracle.spinor_shape(DIMS), dtype=np.complex128)
    L.lqcd_overlap_eigvecs(lat.ctx, chi)
    npart = info.n_partners
    eta = np.zeros((npart,) + oracle.spinor_shape(DIMS), dtype=np.complex128)
    L.lqcd_overlap_eigvecs(lat.ctx, eta, partners=True)
    other = oracle.chirality_indices(DIMS, -sector)
    Z = chi.reshape(n_ev, -1)
    assert np.abs(Z[:, other]).max() == 0  # chiral
    assert np.abs(Z.conj() @ Z.T - np.eye(n_ev)).max() < 1e-10
    kw = dict(lam=sg["lam"], vecs=sg["vecs"])
    for i in range(n_ev):  # residual recomputed by the oracle with the set-up's sign function
        h = oracle.apply_sector_normal(DIMS, U, RHO, sector, chi[i], sg["a"], sg["b"], sg["c"], **kw)
        assert np.linalg.norm((h - mu[i] * chi[i]).ravel()) <= 2 * tol
    # partners: the other sector, the same eigenvalues, orthonormal; chiral
    # zero modes (a nonzero index) and mu = 4 rho^2 have none
    has = (mu > 1e-8) & (mu < 4 * RHO**2 - 1e-8)
    assert npart == int(has.sum())
    pmu = mu[has]
    Y = eta.reshape(npart, -1)
    assert np.abs(Y[:, oracle.chirality_indices(DIMS, sector)]).max() == 0
    assert np.abs(Y.conj() @ Y.T - np.eye(npart)).max() < 1e-9
    for i in range(npart):
        h = oracle.apply_sector_normal(DIMS, U, RHO, -sector, eta[i], sg["a"], sg["b"], sg["c"], **kw)
        assert np.linalg.norm((h - pmu[i] * eta[i]).ravel()) <= 4 * tol
    lat.close()


@pytest.mark.parametrize("inner", ["f64", "f32"])
def test_deflated_solve(lib, inner):
    """A smooth field and a light mass (m = 0.01), where the lowest modes of
    D^dag D set the CG's pace: the deflated CG reaches an oracle-recomputed
    true residual of 1e-10 in fewer iterations than the plain one."""
    L = lib
    dims = (4, 4, 4, 8)
    U = gen.gauge_field(dims, 0.1, 63)
    m = 0.01
    lat, sg = _setup(L, dims, U, 6, mass=m)
    st, info = L.lqcd_overlap_eigen(lat.ctx, L.overlap_eigen_params(n_ev=32, sector=1, tol=1e-9))
    assert st == L.LQCD_OK
    b = gen.gaussian_spinor(dims, 2063, nrhs=2)
    cg = L.solve_params(tol=1e-10, max_iter=3000, nrhs=2, inner=L.PREC[inner], delta=0.1)
    its = {}
    for op in (L.LQCD_OV_SOLVE, L.LQCD_OV_SOLVE_DEFLATED):
        x = np.zeros_like(b)
        st, sinfo = L.lqcd_overlap(lat.ctx, x, b, 2, op, cg)
        assert st == L.LQCD_OK
        its[op] = sinfo.iters
        for k in range(2):
            r = b[k] - oracle.apply_overlap(dims, U, RHO, m, x[k], sg["a"], sg["b"], sg["c"], lam=sg["lam"],
                                            vecs=sg["vecs"])
            assert np.linalg.norm(r) / np.linalg.norm(b[k]) <= 1e-10
    print("overlap CG iterations plain / deflated:", its[L.LQCD_OV_SOLVE], its[L.LQCD_OV_SOLVE_DEFLATED],
          "mu:", list(np.round(info.mu[:4], 5)))
    assert its[L.LQCD_OV_SOLVE_DEFLATED] < its[L.LQCD_OV_SOLVE]
    lat.close()


def test_eigensystem_state_and_arguments(lib):
    L = lib
    dims = (4, 4, 2, 4)
    U = gen.gauge_field(dims, 0.4, 65)
    lat = L.Lattice(dims)
    lat.load_gauge(U.view(np.float64))
    with pytest.raises(L.LqcdError):  # no overlap set-up
        L.lqcd_overlap_eigen(lat.ctx, L.overlap_eigen_params(n_ev=4))
    lat.close()
    lat, sg = _setup(L, dims, U, 4)
    b = gen.gaussian_spinor(dims, 3, nrhs=1)
    x = np.zeros_like(b)
    cg = L.solve_params(tol=1e-8, max_iter=500)
    with pytest.raises(L.LqcdError):  # nothing to deflate with yet
        L.lqcd_overlap(lat.ctx, x, b, 1, L.LQCD_OV_SOLVE_DEFLATED, cg)
    with pytest.raises(L.LqcdError):
        L.lqcd_overlap_eigvecs(lat.ctx, np.zeros((4,) + oracle.spinor_shape(dims), dtype=np.complex128))
    for bad in (dict(n_ev=0), dict(n_ev=300), dict(sector=0), dict(tol=0.0), dict(basis=5), dict(max_restarts=0)):
        with pytest.raises(L.LqcdError):
            L.lqcd_overlap_eigen(lat.ctx, L.overlap_eigen_params(**{"n_ev": 4, **bad}))
    # an unreachable tolerance within one restart: refused, nothing kept
    st, info = L.lqcd_overlap_eigen(lat.ctx, L.overlap_eigen_params(n_ev=8, tol=1e-14, max_restarts=1),
                                    raise_on_noconv=False)
    assert st == L.LQCD_ERR_NOCONV
    with pytest.raises(L.LqcdError):
        L.lqcd_overlap(lat.ctx, x, b, 1, L.LQCD_OV_SOLVE_DEFLATED, cg)
    st, info = L.lqcd_overlap_eigen(lat.ctx, L.overlap_eigen_params(n_ev=8, tol=1e-9))
    assert st == L.LQCD_OK
    st, _ = L.lqcd_overlap(lat.ctx, x, b, 1, L.LQCD_OV_SOLVE_DEFLATED, cg)
    assert st == L.LQCD_OK
    # a new set-up changes the sign function: the eigensystem is dropped
    L.lqcd_overlap_setup(lat.ctx, L.overlap_params(rho=RHO, n_low=4, sign_tol=1e-12, eig_tol=1e-11,
                                                   eig_method=L.LQCD_EIG_LANCZOS, max_filter=400))
    with pytest.raises(L.LqcdError):
        L.lqcd_overlap(lat.ctx, x, b, 1, L.LQCD_OV_SOLVE_DEFLATED, cg)
    lat.close()
