"""GPU solves checked by the FP64 oracle: true residual ||b - M x|| / ||b||
recomputed on the CPU from the returned x, and x against the oracle's own
solution."""
import numpy as np
import pytest

import gen
import oracle
from helpers import rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2001_05706_gb300 as L
    return L


def test_fp64_cg_wilson_8x4(lib):
    """Plain Wilson (c_sw = 0) even-odd CG in FP64 on 8^4, kappa = 0.12, eps = 0.3."""
    dims = (8, 8, 8, 8)
    U = gen.gauge_field(dims, 0.3, 1001)
    b = gen.gaussian_spinor(dims, 2001)[0]
    lat = lib.Lattice(dims)
    lat.load_gauge(U.view(np.float64))
    lat.clover(0.12, 0.0)
    x, st, info = lat.solve(b, tol=1e-10, inner="f64", recon=18)
    assert st == lib.LQCD_OK, lib.lqcd_last_error()
    r = oracle.true_residual(dims, U, None, 0.12, x, b)
    assert r <= 1e-10
    assert info.true_resid[0] <= 1e-10
    xo, it, _ = oracle.solve(dims, U, None, None, 0.12, b, tol=1e-12)
    assert rel(x, xo) < 1e-9
    lat.close()


@pytest.mark.parametrize("inner", ["f32", "f16", "bf16"])
def test_mixed_clover(lib, inner):
    dims = (8, 8, 8, 16)
    kappa, csw = 0.125, 1.0
    U = gen.gauge_field(dims, 0.2, 1003)
    b = gen.gaussian_spinor(dims, 2003)[0]
    lat = lib.Lattice(dims)
    lat.load_gauge(U.view(np.float64))
    lat.clover(kappa, csw)
    x, st, info = lat.solve(b, tol=1e-10, inner=inner, delta=0.1, recon=18, inner_recon=12)
    assert st == lib.LQCD_OK, lib.lqcd_last_error()
    A = oracle.clover(dims, U, kappa, csw)
    assert oracle.true_residual(dims, U, A, kappa, x, b) <= 1e-10
    assert info.reliable_updates >= 1
    lat.close()


def test_df64_cg_matches_fp64(lib):
    """Plain CGLS in double-float arithmetic reaches the same 1e-10 true
    residual (checked by the oracle) and the same solution as FP64 CGLS."""
    dims = (8, 8, 8, 16)
    kappa, csw = 0.125, 1.0
    U = gen.gauge_field(dims, 0.2, 1003)
    b = gen.gaussian_spinor(dims, 2003)[0]
    lat = lib.Lattice(dims)
    lat.load_gauge(U.view(np.float64))
    lat.clover(kappa, csw)
    xd, st, info = lat.solve(b, tol=1e-10, inner="df64", recon=18)
    assert st == lib.LQCD_OK, lib.lqcd_last_error()
    x64, st64, info64 = lat.solve(b, tol=1e-10, inner="f64", recon=18)
    assert st64 == lib.LQCD_OK
    A = oracle.clover(dims, U, kappa, csw)
    assert oracle.true_residual(dims, U, A, kappa, xd, b) <= 1e-10
    assert rel(xd, x64) < 1e-8
    # same recursion up to rounding: the iteration counts agree closely
    assert abs(info.iters - info64.iters) <= 0.05 * info64.iters + 8
    lat.close()


@pytest.mark.parametrize("inner", ["f16", "bf16"])
def test_mixed_with_df64_updates(lib, inner):
    """Mixed solve whose reliable updates and accumulated solution are DF64."""
    dims = (8, 8, 8, 16)
    kappa, csw = 0.125, 1.0
    U = gen.gauge_field(dims, 0.2, 1003)
    b = gen.gaussian_spinor(dims, 2003, nrhs=2)
    lat = lib.Lattice(dims)
    lat.load_gauge(U.view(np.float64))
    lat.clover(kappa, csw)
    x, st, info = lat.solve(b, tol=1e-10, inner=inner, delta=0.1, recon=18, inner_recon=12, outer="df64")
    assert st == lib.LQCD_OK, lib.lqcd_last_error()
    A = oracle.clover(dims, U, kappa, csw)
    for k in range(2):
        assert oracle.true_residual(dims, U, A, kappa, x[k], b[k]) <= 1e-10
    assert info.reliable_updates >= 1
    lat.close()


def test_solver_rejects_bad_outer(lib):
    dims = (4, 4, 4, 4)
    lat = lib.Lattice(dims)
    lat.load_gauge(gen.gauge_field(dims, 0.2, 5).view(np.float64))
    lat.clover(0.12, 1.0)
    b = gen.gaussian_spinor(dims, 6)[0]
    with pytest.raises(lib.LqcdError) as e:
        lat.solve(b, inner="f32", outer="f32")
    assert e.value.status == lib.LQCD_ERR_ARG
    with pytest.raises(lib.LqcdError) as e:
        lat.solve(b, inner="f32", schur=2)
    assert e.value.status == lib.LQCD_ERR_ARG
    lat.close()


def test_multi_rhs_point_sources(lib):
    """12 point sources, mixed FP16 inner solver, every one to 1e-10."""
    dims = (8, 8, 8, 8)
    kappa, csw = 0.125, 1.0
    U = gen.gauge_field(dims, 0.2, 1004)
    b = gen.point_sources(dims)
    lat = lib.Lattice(dims)
    lat.load_gauge(U.view(np.float64))
    lat.clover(kappa, csw)
    x, st, info = lat.solve(b, tol=1e-10, inner="f16", nrhs=12)
    assert st == lib.LQCD_OK, lib.lqcd_last_error()
    A = oracle.clover(dims, U, kappa, csw)
    for k in range(12):
        assert oracle.true_residual(dims, U, A, kappa, x[k], b[k]) <= 1e-10
    lat.close()


def test_solve_deterministic_and_x0(lib):
    dims = (4, 4, 4, 8)
    U = gen.gauge_field(dims, 0.3, 9)
    b = gen.gaussian_spinor(dims, 10)[0]
    lat = lib.Lattice(dims)
    lat.load_gauge(U.view(np.float64))
    lat.clover(0.12, 1.0)
    x1, st1, i1 = lat.solve(b, inner="f32")
    x2, st2, i2 = lat.solve(b, inner="f32")
    assert st1 == st2 == lib.LQCD_OK
    assert np.array_equal(x1, x2) and i1.iters == i2.iters
    # restart from the solution: converges immediately
    prm = lib.solve_params(tol=1e-10, inner=lib.LQCD_F64, use_x0=1)
    x3 = x1.copy()
    st, info = lib.lqcd_solve(lat.ctx, x3, b, prm)
    assert info.iters == 0
    lat.close()


def test_noconv_reports(lib):
    dims = (4, 4, 4, 8)
    U = gen.gauge_field(dims, 0.3, 9)
    b = gen.gaussian_spinor(dims, 10)[0]
    lat = lib.Lattice(dims)
    lat.load_gauge(U.view(np.float64))
    lat.clover(0.12, 1.0)
    x, st, info = lat.solve(b, max_iter=3, inner="f64")
    assert st == lib.LQCD_ERR_NOCONV
    assert info.iters == 3 and info.true_resid[0] > 1e-10
    lat.close()


@pytest.mark.parametrize("outer,schur", [("f64", "asym"), ("df64", "asym"), ("f64", "sym")])
def test_batch_of_uneven_lattices(lib, outer, schur):
    """Three lattices of different volumes in one graph-captured batch: each
    reaches 1e-10 (oracle) and equals the single-lattice solve bitwise, with
    FP64 or DF64 reliable updates, on either Schur form."""
    L = lib
    dims_list = [(4, 4, 4, 8), (6, 4, 4, 8), (8, 4, 6, 4)]
    kappa, csw = 0.125, 1.0
    lats, Us, bs = [], [], []
    for j, dims in enumerate(dims_list):
        U = gen.gauge_field(dims, 0.2, 3000 + j)
        lat = L.Lattice(dims)
        lat.load_gauge(U.view(np.float64))
        lat.clover(kappa, csw)
        lats.append(lat)
        Us.append(U)
        bs.append(np.ascontiguousarray(gen.gaussian_spinor(dims, 4000 + j, nrhs=2)))
    xs = [np.zeros_like(b) for b in bs]
    prm = L.solve_params(tol=1e-10, inner=L.LQCD_F16, nrhs=2, check_every=8, outer=L.PREC[outer], schur=schur)
    st, infos = L.lqcd_solve_batch([l.ctx for l in lats], xs, bs, prm)
    assert st == L.LQCD_OK
    for j, dims in enumerate(dims_list):
        A = oracle.clover(dims, Us[j], kappa, csw)
        for k in range(2):
            assert oracle.true_residual(dims, Us[j], A, kappa, xs[j][k], bs[j][k]) <= 1e-10
        x1 = np.zeros_like(bs[j])
        st1, info1 = L.lqcd_solve(lats[j].ctx, x1, bs[j], prm)
        assert np.array_equal(x1, xs[j]) and info1.iters == infos[j].iters
    for lat in lats:
        lat.close()


@pytest.mark.parametrize("inner,outer,nrhs", [("f64", "f64", 1), ("df64", "df64", 1), ("f32", "f64", 2),
                                              ("f16", "f64", 2), ("bf16", "f64", 1), ("f16", "df64", 1)])
def test_bicgstab(lib, inner, outer, nrhs):
    """BiCGStab on Mhat, plain and mixed with reliable updates: every right-hand
    side to a true residual of 1e-10 (recomputed by the oracle), and the same
    solution as the FP64 CGLS."""
    dims = (8, 8, 8, 16)
    kappa, csw = 0.125, 1.0
    U = gen.gauge_field(dims, 0.2, 1003)
    b = gen.gaussian_spinor(dims, 2003, nrhs=nrhs)
    lat = lib.Lattice(dims)
    lat.load_gauge(U.view(np.float64))
    lat.clover(kappa, csw)
    x, st, info = lat.solve(b, tol=1e-10, inner=inner, outer=outer, delta=0.1, recon=18, inner_recon=12,
                            solver="bicgstab")
    assert st == lib.LQCD_OK, lib.lqcd_last_error()
    A = oracle.clover(dims, U, kappa, csw)
    for k in range(nrhs):
        assert oracle.true_residual(dims, U, A, kappa, x[k], b[k]) <= 1e-10
        assert info.true_resid[k] <= 1e-10
    xc, stc, _ = lat.solve(b, tol=1e-10, inner="f64", recon=18)
    assert stc == lib.LQCD_OK
    assert rel(x, xc) < 1e-8
    if inner not in ("f64", "df64"):
        assert info.reliable_updates >= 1
    lat.close()


def test_bicgstab_point_sources_and_batch_rejects(lib):
    """Point sources (a very uneven residual) converge with the mixed BiCGStab;
    the batched entry point runs CGLS only and says so."""
    dims = (8, 8, 8, 8)
    kappa, csw = 0.125, 1.0
    U = gen.gauge_field(dims, 0.2, 1004)
    b = gen.point_sources(dims)[:3]
    lat = lib.Lattice(dims)
    lat.load_gauge(U.view(np.float64))
    lat.clover(kappa, csw)
    x, st, info = lat.solve(b, tol=1e-10, inner="f16", nrhs=3, solver="bicgstab")
    assert st == lib.LQCD_OK, lib.lqcd_last_error()
    A = oracle.clover(dims, U, kappa, csw)
    for k in range(3):
        assert oracle.true_residual(dims, U, A, kappa, x[k], b[k]) <= 1e-10
    prm = lib.solve_params(tol=1e-10, inner=lib.LQCD_F16, solver="bicgstab")
    with pytest.raises(lib.LqcdError) as e:
        lib.lqcd_solve_batch([lat.ctx], [np.zeros_like(b[0])], [np.ascontiguousarray(b[0])], prm)
    assert e.value.status == lib.LQCD_ERR_ARG
    lat.close()


def test_bicgstab_initial_guess(lib):
    """BiCGStab started from the solution of a looser solve: it converges in
    fewer iterations than from zero and to the same 1e-10 true residual."""
    dims = (8, 8, 8, 8)
    kappa, csw = 0.125, 1.0
    U = gen.gauge_field(dims, 0.2, 1006)
    b = gen.gaussian_spinor(dims, 2006)[0]
    lat = lib.Lattice(dims)
    lat.load_gauge(U.view(np.float64))
    lat.clover(kappa, csw)
    x0, st0, i0 = lat.solve(b, tol=1e-4, inner="f64", solver="bicgstab")
    assert st0 == lib.LQCD_OK
    prm = lib.solve_params(tol=1e-10, inner=lib.LQCD_F16, use_x0=1, solver="bicgstab")
    x = np.ascontiguousarray(x0.copy())
    st, info = lib.lqcd_solve(lat.ctx, x, np.ascontiguousarray(b), prm)
    assert st == lib.LQCD_OK
    _, _, cold = lat.solve(b, tol=1e-10, inner="f16", solver="bicgstab")
    assert info.iters < cold.iters
    A = oracle.clover(dims, U, kappa, csw)
    assert oracle.true_residual(dims, U, A, kappa, x, b) <= 1e-10
    lat.close()


@pytest.mark.parametrize("solver,inner,outer,nrhs", [("cgls", "f64", "f64", 1), ("cgls", "df64", "df64", 1),
                                                     ("cgls", "f32", "f64", 2), ("cgls", "f16", "f64", 1),
                                                     ("cgls", "f16", "df64", 1), ("bicgstab", "f64", "f64", 1),
                                                     ("bicgstab", "f16", "f64", 2)])
def test_symmetric_schur_solves(lib, solver, inner, outer, nrhs):
    """Solves on the symmetric Schur complement A_oo^-1 Mhat reach the 1e-10
    true residual of M x = b (recomputed by the oracle), although the recursion
    only sees A_oo^-1 times that residual, and give the asymmetric form's
    solution; on this rough field (eps = 1, c_sw = 2) the plain CGLS needs
    fewer iterations on the better-conditioned operator."""
    dims = (8, 8, 8, 8)
    kappa, csw = 0.14, 2.0
    U = gen.gauge_field(dims, 1.0, 1010)
    b = gen.gaussian_spinor(dims, 2010, nrhs=nrhs)
    lat = lib.Lattice(dims)
    lat.load_gauge(U.view(np.float64))
    lat.clover(kappa, csw)
    kw = dict(tol=1e-10, inner=inner, outer=outer, recon=18, inner_recon=12, solver=solver, max_iter=20000)
    xs, st, info = lat.solve(b, schur="sym", **kw)
    assert st == lib.LQCD_OK, lib.lqcd_last_error()
    A = oracle.clover(dims, U, kappa, csw)
    for k in range(nrhs):
        assert oracle.true_residual(dims, U, A, kappa, xs[k], b[k]) <= 1e-10
        assert info.true_resid[k] <= 1e-10
    xa, sta, infa = lat.solve(b, schur="asym", **kw)
    assert sta == lib.LQCD_OK
    assert rel(xs, xa) < 1e-8
    if solver == "cgls" and inner == "f64":
        assert info.iters < infa.iters
    lat.close()


@pytest.mark.parametrize("inner,outer,nrhs,nk", [("f64", "f64", 1, 8), ("df64", "df64", 1, 8), ("f32", "f64", 2, 8),
                                                 ("f16", "f64", 2, 8), ("bf16", "f64", 1, 16),
                                                 ("f16", "df64", 1, 4)])
def test_gcr(lib, inner, outer, nrhs, nk):
    """Restarted GCR(m) on Mhat, plain and mixed with a reliable update after
    each cycle: every right-hand side to a true residual of 1e-10 (recomputed
    by the oracle), and the FP64 CGLS solution."""
    dims = (8, 8, 8, 16)
    kappa, csw = 0.125, 1.0
    U = gen.gauge_field(dims, 0.2, 1003)
    b = gen.gaussian_spinor(dims, 2003, nrhs=nrhs)
    lat = lib.Lattice(dims)
    lat.load_gauge(U.view(np.float64))
    lat.clover(kappa, csw)
    x, st, info = lat.solve(b, tol=1e-10, inner=inner, outer=outer, delta=0.1, recon=18, inner_recon=12,
                            solver="gcr", gcr_nkrylov=nk, max_iter=4000)
    assert st == lib.LQCD_OK, lib.lqcd_last_error()
    A = oracle.clover(dims, U, kappa, csw)
    for k in range(nrhs):
        assert oracle.true_residual(dims, U, A, kappa, x[k], b[k]) <= 1e-10
        assert info.true_resid[k] <= 1e-10
    xc, stc, _ = lat.solve(b, tol=1e-10, inner="f64", recon=18)
    assert stc == lib.LQCD_OK
    assert rel(x, xc) < 1e-8
    if inner not in ("f64", "df64"):
        assert info.reliable_updates >= 1
    lat.close()


@pytest.mark.parametrize("inner", ["f64", "f16"])
def test_gcr_symmetric_schur_and_point_sources(lib, inner):
    """GCR on A_oo^-1 Mhat (rough field) and on point sources (uneven
    residuals), to the oracle's 1e-10; bad cycle lengths are refused."""
    dims = (8, 8, 8, 8)
    kappa, csw = 0.14, 2.0
    U = gen.gauge_field(dims, 1.0, 1010)
    b = gen.point_sources(dims)[:2]
    lat = lib.Lattice(dims)
    lat.load_gauge(U.view(np.float64))
    lat.clover(kappa, csw)
    A = oracle.clover(dims, U, kappa, csw)
    for schur in ("asym", "sym"):
        x, st, info = lat.solve(b, tol=1e-10, inner=inner, nrhs=2, solver="gcr", schur=schur, max_iter=6000)
        assert st == lib.LQCD_OK, lib.lqcd_last_error()
        for k in range(2):
            assert oracle.true_residual(dims, U, A, kappa, x[k], b[k]) <= 1e-10
    for bad in (-1, 65):
        with pytest.raises(lib.LqcdError):
            lat.solve(b[:1], tol=1e-10, solver="gcr", gcr_nkrylov=bad)
    lat.close()


@pytest.mark.parametrize("inner", ["f32", "f16"])
def test_mixed_solve_with_eight_real_inner_links(lib, inner):
    """The mixed CGLS with the 8-real form for the inner operator's links: the
    oracle's true residual of 1e-10."""
    dims = (8, 8, 8, 16)
    kappa, csw = 0.125, 1.0
    U = gen.gauge_field(dims, 0.2, 1003)
    b = gen.gaussian_spinor(dims, 2003, nrhs=1)
    lat = lib.Lattice(dims)
    lat.load_gauge(U.view(np.float64))
    lat.clover(kappa, csw)
    x, st, info = lat.solve(b, tol=1e-10, inner=inner, recon=18, inner_recon=8)
    assert st == lib.LQCD_OK, lib.lqcd_last_error()
    A = oracle.clover(dims, U, kappa, csw)
    assert oracle.true_residual(dims, U, A, kappa, x[0], b[0]) <= 1e-10
    lat.close()
