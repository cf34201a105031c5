"""The GPU multigrid building blocks (lqcd_mg_*) against the multigrid oracle
on the same inputs: the fine stencil built from the context's links and
clover term, stencil application, block orthonormalisation, prolongation,
restriction and the Galerkin coarse operator at two levels; the complex BLAS
against numpy; the coarse operator of a full 8^4 set-up against the oracle's
Galerkin product of the GPU's own prolongator; and a 3-level solve to the C
oracle's recomputed residual."""
import numpy as np
import pytest

import gen
import oracle
from oracle import multigrid as omg

pytestmark = pytest.mark.gpu
KAPPA, CSW = 0.12, 1.0
SMALL = (4, 4, 2, 4)


@pytest.fixture(scope="module")
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2001_05706_gb300 as L
    return L


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex128)).to("cuda")


def _host(t):
    return t.cpu().numpy()


def _rel(got, want):
    return np.abs(got - want).max() / max(np.abs(want).max(), 1e-300)


def _starts(nv, V, n, seed):
    return gen.gaussian(2 * nv * V * n, seed).view(np.complex128).reshape(nv, V, n)


def _lattice(L, dims, U, tbc, kappa, csw):
    lat = L.Lattice(dims, tbc)
    lat.load_gauge(U.view(np.float64))
    lat.clover(kappa, csw)
    return lat


@pytest.mark.parametrize("csw,tbc", [(CSW, 1), (0.0, 0)])
def test_fine_stencil_matches_the_oracle(lib, csw, tbc):
    from paper_2001_05706_gb300 import multigrid as gmg
    U = gen.gauge_field(SMALL, 0.5, 11)
    ref = omg.wilson_clover_stencil(SMALL, U, KAPPA, csw, tbc)
    with _lattice(lib, SMALL, U, tbc, KAPPA, csw) as lat:
        st = gmg.fine_stencil(lat)
        for got, want in ((st.X, ref.X), (st.F, ref.F), (st.B, ref.B)):
            assert _rel(_host(got), want) <= 1e-13


def test_kernels_match_the_oracle_on_its_inputs(lib):
    """apply, orthonormalize, prolong, restrict and coarsen at two levels,
    each given the oracle's own inputs."""
    from paper_2001_05706_gb300 import multigrid as gmg
    V = int(np.prod(SMALL))
    U = gen.gauge_field(SMALL, 0.5, 11)
    ref = omg.wilson_clover_stencil(SMALL, U, KAPPA, CSW, 1)
    with _lattice(lib, SMALL, U, 1, KAPPA, CSW) as lat:
        st = gmg.Stencil(lat.ctx, SMALL, 12, _dev(ref.X), _dev(ref.F), _dev(ref.B))
        v = gen.gaussian_spinor(SMALL, 12).reshape(V, 12)
        assert _rel(_host(st.apply(_dev(v))), ref.apply(v)) <= 1e-14
        levels = [(ref, st, (2, 2, 1, 2), 4, 41), (None, None, (2, 2, 2, 1), 3, 42)]
        fine_ref, fine = ref, st
        for _, _, block, nv, seed in levels:
            vecs = omg.near_null_vectors(fine_ref, _starts(nv, fine_ref.V, fine_ref.n, seed), 20)
            Pref = omg.Prolongator(fine_ref, block, vecs)
            P = gmg.Prolongator(fine, block, _dev(vecs))
            assert _rel(_host(P.P), Pref.Ps) <= 1e-11      # Gram-Schmidt against the QR
            P.P = _dev(Pref.Ps)                            # from here on, identical inputs
            w = _starts(1, Pref.Vc, Pref.nc, seed + 10)[0]
            u = _starts(1, fine_ref.V, fine_ref.n, seed + 20)[0]
            assert _rel(_host(P.prolong(_dev(w))), Pref.prolong(w)) <= 1e-14
            assert _rel(_host(P.restrict(_dev(u))), Pref.restrict(u)) <= 1e-14
            Dref = omg.coarsen(fine_ref, Pref)
            D = gmg.coarsen(fine, P)
            assert D.dims == Dref.dims and D.n == Dref.n
            for got, want in ((D.X, Dref.X), (D.F, Dref.F), (D.B, Dref.B)):
                assert _rel(_host(got), want) <= 1e-12
            assert _rel(_host(D.apply(_dev(w))), Dref.apply(w)) <= 1e-12
            fine_ref = Dref
            fine = gmg.Stencil(lat.ctx, Dref.dims, Dref.n, _dev(Dref.X), _dev(Dref.F), _dev(Dref.B))


@pytest.mark.parametrize("length", [1000, 300001])
def test_complex_blas_matches_numpy(lib, length):
    L = lib
    rng = np.random.default_rng(5)
    X = rng.standard_normal((5, length)) + 1j * rng.standard_normal((5, length))
    y = rng.standard_normal(length) + 1j * rng.standard_normal(length)
    coef = rng.standard_normal(5) + 1j * rng.standard_normal(5)
    with L.Lattice((4, 4, 4, 4)) as lat:
        ctx = lat.ctx
        want = X.conj() @ y
        assert np.abs(L.lqcd_mg_dots(ctx, 5, _dev(X), _dev(y)) - want).max() <= 1e-12 * np.abs(want).max()
        yd = _dev(y)
        L.lqcd_mg_axpys(ctx, coef, _dev(X), yd)
        assert _rel(_host(yd), y + coef @ X) <= 1e-14
        yd = _dev(y)
        L.lqcd_mg_axpby(ctx, 2 - 1j, _dev(X[0]), 0.5 + 0.25j, yd)
        assert _rel(_host(yd), (2 - 1j) * X[0] + (0.5 + 0.25j) * y) <= 1e-15
        L.lqcd_mg_axpby(ctx, 1.5, yd, -0.5j, yd)  # x and y the same array
        assert _rel(_host(yd), (1.5 - 0.5j) * ((2 - 1j) * X[0] + (0.5 + 0.25j) * y)) <= 1e-15


def test_arguments_are_checked(lib):
    import ctypes
    from paper_2001_05706_gb300 import multigrid as gmg
    L = lib
    V = int(np.prod(SMALL))
    U = gen.gauge_field(SMALL, 0.5, 11)
    with _lattice(L, SMALL, U, 1, KAPPA, CSW) as lat:
        st = gmg.fine_stencil(lat)
        v = _starts(1, V, 12, 1)
        with pytest.raises(L.LqcdError) as e:  # a vector and twice itself
            gmg.Prolongator(st, (2, 2, 1, 2), _dev(np.concatenate([v, 2 * v])))
        assert e.value.status == L.LQCD_ERR_SINGULAR
        with pytest.raises(ValueError):
            gmg.Prolongator(st, (3, 2, 1, 2), _dev(v))
        # the C side: blocks, sizes and host pointers refused before any launch
        dims = (ctypes.c_int * 4)(*SMALL)
        bad = (ctypes.c_int * 4)(3, 2, 1, 2)
        P = _dev(np.zeros((V, 12, 2)))
        vv = _dev(v)
        assert L._lib.lqcd_mg_orthonormalize(lat.ctx, dims, 12, bad, 1, ctypes.c_void_p(vv.data_ptr()),
                                             ctypes.c_void_p(P.data_ptr())) == L.LQCD_ERR_ARG
        assert L._lib.lqcd_mg_orthonormalize(lat.ctx, dims, 13, dims, 1, ctypes.c_void_p(vv.data_ptr()),
                                             ctypes.c_void_p(P.data_ptr())) == L.LQCD_ERR_ARG
        host = np.zeros(V * 12, dtype=np.complex128)
        assert L._lib.lqcd_mg_apply(lat.ctx, dims, 12, ctypes.c_void_p(st.X.data_ptr()),
                                    ctypes.c_void_p(st.F.data_ptr()), ctypes.c_void_p(st.B.data_ptr()),
                                    ctypes.c_void_p(host.ctypes.data), ctypes.c_void_p(vv.data_ptr())) == L.LQCD_ERR_ARG
    with L.Lattice(SMALL) as lat:  # no gauge field yet
        X = _dev(np.zeros((V, 12, 12)))
        F = _dev(np.zeros((4, V, 12, 12)))
        with pytest.raises(L.LqcdError) as e:
            L.lqcd_mg_fine_stencil(lat.ctx, V, X, F, F.clone())
        assert e.value.status == L.LQCD_ERR_STATE


def test_three_level_multigrid_solve_reaches_the_oracle_residual(lib):
    """Blocks (2,2,2,2) twice on 8^4 near the critical kappa.  The set-up's
    level-1 operator is checked against the oracle's P^H M P of the GPU's own
    prolongator, which is checked to be block-orthonormal; the solve must
    reach the C oracle's true residual <= 1e-10 in a fraction of plain
    GCR's steps."""
    from paper_2001_05706_gb300 import multigrid as gmg
    L = lib
    dims, kappa = (8, 8, 8, 8), 0.1285
    V = int(np.prod(dims))
    U = gen.gauge_field(dims, 0.3, 21)
    b = gen.gaussian_spinor(dims, 22).reshape(V, 12)
    with _lattice(L, dims, U, 1, kappa, CSW) as lat:
        st = gmg.fine_stencil(lat)
        mg = gmg.Multigrid(st, [(2, 2, 2, 2), (2, 2, 2, 2)], [_starts(8, V, 12, 23), _starts(8, V // 16, 16, 24)],
                           setup_iters=30)
        assert [op.dims for op in mg.ops] == [dims, (4, 4, 4, 4), (2, 2, 2, 2)]
        assert [op.n for op in mg.ops] == [12, 16, 16]
        ref = omg.wilson_clover_stencil(dims, U, kappa, CSW, 1)
        Pref = omg.Prolongator(ref, (2, 2, 2, 2), _starts(8, V, 12, 23))  # geometry; Ps replaced below
        Pref.Ps = _host(mg.P[0].P)
        w = _starts(1, Pref.Vc, Pref.nc, 25)[0]
        assert _rel(Pref.restrict(Pref.prolong(w)), w) <= 1e-12
        D1 = omg.coarsen(ref, Pref)
        for got, want in ((mg.ops[1].X, D1.X), (mg.ops[1].F, D1.F), (mg.ops[1].B, D1.B)):
            assert _rel(_host(got), want) <= 1e-12
        x, it_mg, rel = mg.solve(_dev(b), 1e-10)
        xh = _host(x)
        _, it_plain, _ = gmg.fgcr(st, _dev(b), 1e-10, 3000, nkrylov=32)
    A = oracle.clover(dims, U, kappa, CSW)
    canon = (dims[3], dims[2], dims[1], dims[0], 4, 3)
    assert rel <= 1e-10
    assert oracle.true_residual(dims, U, A, kappa, xh.reshape(canon), b.reshape(canon)) <= 1e-10
    assert it_mg <= 40 and it_mg * 4 <= it_plain, (it_mg, it_plain)
