"""Pins of the multigrid oracle (oracle/multigrid.py) against things other
than itself: the C oracle's Wilson-clover operator (pinned in
test_oracle_dirac.py), the free-field coarse operator in closed form, dense
products P^H M P, gamma5-hermiticity, the exact limit of full-rank
aggregation, Galerkin orthogonality of the coarse-grid correction, and a
3-level solve to the C oracle's recomputed residual."""
import numpy as np
import pytest

import gen
import oracle
from oracle import multigrid as mg

KAPPA, CSW = 0.12, 1.0
SMALL = (4, 4, 2, 4)


def _canon(dims, v):
    return np.asarray(v).reshape(dims[3], dims[2], dims[1], dims[0], 4, 3)


def _dense_M(dims, U, kappa, csw, tbc):
    """M column by column from the C oracle (independent of the stencil code)."""
    V = int(np.prod(dims))
    A = oracle.clover(dims, U, kappa, csw) if csw else None
    D = np.zeros((12 * V, 12 * V), dtype=np.complex128)
    e = np.zeros(12 * V, dtype=np.complex128)
    for j in range(12 * V):
        e[:] = 0
        e[j] = 1
        D[:, j] = oracle.apply_M(dims, U, A, kappa, _canon(dims, e), tbc).reshape(-1)
    return D


def _dense_P(P):
    n = P.Vc * P.nc
    return np.stack([P.prolong(np.eye(n, dtype=np.complex128)[k]).reshape(-1) for k in range(n)], axis=1)


def _starts(nv, V, n, seed):
    return gen.gaussian(2 * nv * V * n, seed).view(np.complex128).reshape(nv, V, n)


@pytest.mark.parametrize("csw,tbc", [(CSW, 1), (0.0, 0), (1.3, 0)])
def test_fine_stencil_is_the_wilson_clover_operator(csw, tbc):
    dims = SMALL
    V = int(np.prod(dims))
    U = gen.gauge_field(dims, 0.5, 11)
    psi = gen.gaussian_spinor(dims, 12)
    st = mg.wilson_clover_stencil(dims, U, KAPPA, csw, tbc)
    A = oracle.clover(dims, U, KAPPA, csw) if csw else None
    for dag, got in ((False, st.apply(psi)), (True, st.apply_adjoint(psi))):
        ref = oracle.apply_M(dims, U, A, KAPPA, psi, tbc, dagger=dag).reshape(V, 12)
        assert np.abs(got - ref).max() <= 1e-14 * np.abs(ref).max()
    # chi is the eigenvalue of gamma5 on each component
    assert np.array_equal(oracle.gamma5(psi).reshape(V, 12), st.chi[None, :] * psi.reshape(V, 12))


@pytest.mark.parametrize("tbc", [1, 0])
def test_free_field_coarse_operator_closed_form(tbc):
    """U = 1 (the clover term vanishes), null vectors constant in space:
    the coarse basis is the fine spin-colour basis and P^H M P has
    X_c = 1 - 2 kappa sum_mu (b_mu - 1) / b_mu (hops inside a block, both
    directions, each (1 - gamma) + (1 + gamma) = 2 on a constant field),
    F_c = -kappa (1 - gamma_mu) / b_mu and B_c = -kappa (1 + gamma_mu) / b_mu
    (one face site in b_mu), with -1 across the t boundary when tbc."""
    dims, block, kappa = (4, 6, 4, 8), (2, 3, 1, 4), 0.1
    V = int(np.prod(dims))
    st = mg.wilson_clover_stencil(dims, gen.unit_gauge(dims), kappa, CSW, tbc)
    vecs = np.zeros((6, V, 12), dtype=np.complex128)
    for k in range(6):
        vecs[k, :, k] = vecs[k, :, k + 6] = 1.0  # chirality + part e_k, - part e_{k+6}
    Dc = mg.coarsen(st, mg.Prolongator(st, block, vecs))
    assert Dc.dims == (2, 2, 4, 2) and Dc.n == 12 and list(Dc.chi) == [1] * 6 + [-1] * 6
    X = (1 - 2 * kappa * sum((b - 1) / b for b in block)) * np.eye(12)
    assert np.abs(Dc.X - X[None]).max() < 1e-14
    t = mg._coords(Dc.dims)[:, 3]
    for mu in range(4):
        sf = np.where((mu == 3) & bool(tbc) & (t == Dc.dims[3] - 1), -1.0, 1.0)
        sb = np.where((mu == 3) & bool(tbc) & (t == 0), -1.0, 1.0)
        F = -kappa * np.kron(np.eye(4) - oracle.gamma(mu), np.eye(3)) / block[mu]
        B = -kappa * np.kron(np.eye(4) + oracle.gamma(mu), np.eye(3)) / block[mu]
        assert np.abs(Dc.F[mu] - sf[:, None, None] * F[None]).max() < 1e-15
        assert np.abs(Dc.B[mu] - sb[:, None, None] * B[None]).max() < 1e-15


def test_prolongator_is_block_orthonormal_chiral_and_spans_its_vectors():
    dims = SMALL
    V = int(np.prod(dims))
    st = mg.wilson_clover_stencil(dims, gen.gauge_field(dims, 0.5, 11), KAPPA, CSW)
    vecs = _starts(4, V, 12, 31)
    P = mg.Prolongator(st, (2, 2, 1, 2), vecs)
    Pd = _dense_P(P)
    assert np.abs(Pd.conj().T @ Pd - np.eye(Pd.shape[1])).max() < 1e-14   # P^H P = 1
    for v in vecs:                                                      # P P^H v = v
        assert np.abs(P.prolong(P.restrict(v)) - v).max() < 1e-13 * np.abs(v).max()
    w = _starts(1, P.Vc, P.nc, 32)[0]                                   # gamma5 P = P Gamma5
    assert np.abs(st.chi[None, :] * P.prolong(w) - P.prolong(P.chi[None, :] * w)).max() < 1e-14
    # Gram-Schmidt order and phase: on each block and chirality the first
    # column is v_0 restricted there, divided by its (positive) norm
    for xc in range(P.Vc):
        sites = np.nonzero(P.c == xc)[0]
        for k, sign in enumerate((1, -1)):
            comps = st.chi == sign
            v0 = vecs[0][sites][:, comps]
            col = P.Ps[sites][:, comps, k * P.nv]
            assert np.abs(col - v0 / np.linalg.norm(v0)).max() < 1e-14


@pytest.mark.parametrize("tbc", [1, 0])
def test_coarse_operators_are_galerkin_products_and_gamma5_hermitian(tbc):
    """Two coarsenings, each against the dense P^H D P; D_c^H = G5 D_c G5
    at both levels (inherited from M^H = g5 M g5 through a P that commutes
    with gamma5)."""
    dims = SMALL
    V = int(np.prod(dims))
    U = gen.gauge_field(dims, 0.5, 11)
    st = mg.wilson_clover_stencil(dims, U, KAPPA, CSW, tbc)
    Md = _dense_M(dims, U, KAPPA, CSW, tbc)
    assert np.abs(st.dense() - Md).max() < 1e-15
    P1 = mg.Prolongator(st, (2, 2, 1, 2), mg.near_null_vectors(st, _starts(4, V, 12, 41), 20))
    D1 = mg.coarsen(st, P1)
    assert D1.dims == (2, 2, 2, 2) and D1.n == 8
    P2 = mg.Prolongator(D1, (2, 2, 2, 1), mg.near_null_vectors(D1, _starts(3, D1.V, D1.n, 42), 10))
    D2 = mg.coarsen(D1, P2)
    for D, fine_dense, P in ((D1, Md, P1), (D2, D1.dense(), P2)):
        Pd = _dense_P(P)
        G = Pd.conj().T @ fine_dense @ Pd
        Dd = D.dense()
        assert np.abs(Dd - G).max() <= 1e-13 * np.abs(G).max()
        g5 = np.tile(D.chi, D.V).astype(np.complex128)
        assert np.abs(Dd.conj().T - g5[:, None] * Dd * g5[None, :]).max() <= 1e-13 * np.abs(Dd).max()
        r = _starts(1, D.V, D.n, 43)[0]
        assert np.abs(D.apply_adjoint(r).reshape(-1) - Dd.conj().T @ r.reshape(-1)).max() <= 1e-13 * np.abs(Dd).max()


def test_full_rank_aggregation_makes_the_two_grid_cycle_exact():
    """With as many vectors as a block chirality has components P is
    unitary, D_c is M in another basis, and one cycle with an exact coarse
    solve and no smoothing is M^-1."""
    dims = SMALL
    V = int(np.prod(dims))
    st = mg.wilson_clover_stencil(dims, gen.gauge_field(dims, 0.5, 51), KAPPA, CSW)
    nv = 8 * 6  # 8 sites x 6 components of one chirality per (2,2,1,2) block
    M = mg.Multigrid(st, [(2, 2, 1, 2)], [_starts(nv, V, 12, 52)], setup_iters=5, pre=0, post=0,
                     coarsest_exact=True)
    r = _starts(1, V, 12, 53)[0]
    x = M.cycle(0, r)
    assert np.abs(st.apply(x) - r).max() <= 1e-12 * np.abs(r).max()


def test_coarse_grid_correction_is_a_galerkin_projection():
    """e = P D_c^-1 P^H r leaves a residual r - M e orthogonal to range(P),
    and C = 1 - P D_c^-1 P^H M is idempotent."""
    dims = SMALL
    V = int(np.prod(dims))
    st = mg.wilson_clover_stencil(dims, gen.gauge_field(dims, 0.5, 61), KAPPA, CSW)
    M = mg.Multigrid(st, [(2, 2, 1, 2)], [_starts(4, V, 12, 62)], setup_iters=20, pre=0, post=0,
                     coarsest_exact=True)
    P = M.P[0]
    r = _starts(1, V, 12, 63)[0]
    e = M.cycle(0, r)
    assert np.abs(P.restrict(r - st.apply(e))).max() <= 1e-12 * np.abs(r).max()

    def C(v):
        return v - M.cycle(0, st.apply(v))

    v = _starts(1, V, 12, 64)[0]
    assert np.abs(C(C(v)) - C(v)).max() <= 1e-12 * np.abs(v).max()


def test_krylov_pieces_on_block_diagonal_operators():
    """MR on c * 1 converges in one step; flexible GCR on a block-diagonal
    stencil (no hops) reaches the per-site dense solution."""
    dims = (2, 2, 2, 2)
    V = 16
    rng = np.random.default_rng(7)
    X = rng.standard_normal((V, 4, 4)) + 1j * rng.standard_normal((V, 4, 4)) + 6 * np.eye(4)
    Z = np.zeros((4, V, 4, 4))
    chi = np.array([1, 1, -1, -1])
    b = rng.standard_normal((V, 4)) + 1j * rng.standard_normal((V, 4))
    scal = mg.Stencil(dims, np.broadcast_to((2.5 - 1j) * np.eye(4), (V, 4, 4)), Z, Z, chi)
    assert np.abs(mg.mr(scal, b, 1) - b / (2.5 - 1j)).max() < 1e-15
    op = mg.Stencil(dims, X, Z, Z, chi)
    x, it, rel = mg.fgcr(op, b, 1e-13, 200)
    assert rel <= 1e-13
    assert np.abs(x - np.linalg.solve(X, b[..., None])[..., 0]).max() < 1e-12


def test_three_level_multigrid_reaches_the_oracle_residual():
    """Blocks (2,2,2,2) twice on 8^4 near the critical kappa: flexible GCR
    preconditioned by the K-cycle reaches a true residual <= 1e-10 as the C
    oracle recomputes it, in a fraction of plain GCR's steps."""
    dims, kappa = (8, 8, 8, 8), 0.1285
    V = int(np.prod(dims))
    U = gen.gauge_field(dims, 0.3, 21)
    st = mg.wilson_clover_stencil(dims, U, kappa, CSW, 1)
    b = gen.gaussian_spinor(dims, 22).reshape(V, 12)
    M = mg.Multigrid(st, [(2, 2, 2, 2), (2, 2, 2, 2)], [_starts(8, V, 12, 23), _starts(8, V // 16, 16, 24)],
                     setup_iters=30)
    assert [op.dims for op in M.ops] == [dims, (4, 4, 4, 4), (2, 2, 2, 2)] and [op.n for op in M.ops] == [12, 16, 16]
    x, it_mg, rel = M.solve(b, 1e-10)
    A = oracle.clover(dims, U, kappa, CSW)
    assert oracle.true_residual(dims, U, A, kappa, _canon(dims, x), _canon(dims, b)) <= 1e-10
    _, it_plain, _ = mg.fgcr(st, b, 1e-10, 3000, nkrylov=32)
    assert it_mg * 4 <= it_plain, (it_mg, it_plain)


def test_aggregation_rejects_bad_arguments():
    dims = SMALL
    V = int(np.prod(dims))
    st = mg.wilson_clover_stencil(dims, gen.gauge_field(dims, 0.5, 11), KAPPA, CSW)
    with pytest.raises(ValueError):
        mg.Prolongator(st, (3, 2, 1, 2), _starts(2, V, 12, 1))   # 3 does not divide 4
    with pytest.raises(ValueError):
        mg.Prolongator(st, (1, 1, 1, 1), _starts(7, V, 12, 1))   # 7 vectors, 6 components per chirality
    v = _starts(1, V, 12, 1)
    with pytest.raises(ValueError):
        mg.Prolongator(st, (2, 2, 1, 2), np.concatenate([v, 2 * v]))  # dependent vectors


def test_single_site_coarse_lattice_is_the_galerkin_product():
    """Blocks spanning the whole lattice: one coarse site, every hop across
    a block face wraps to the same block, and the coarse stencil's X + sum
    (F + B) must equal the dense P^H M P."""
    dims = SMALL
    V = int(np.prod(dims))
    U = gen.gauge_field(dims, 0.5, 71)
    st = mg.wilson_clover_stencil(dims, U, KAPPA, CSW, 1)
    P = mg.Prolongator(st, dims, mg.near_null_vectors(st, _starts(5, V, 12, 72), 15))
    D = mg.coarsen(st, P)
    assert D.dims == (1, 1, 1, 1) and D.n == 10
    Pd = _dense_P(P)
    G = Pd.conj().T @ _dense_M(dims, U, KAPPA, CSW, 1) @ Pd
    assert np.abs(D.dense() - G).max() <= 1e-13 * np.abs(G).max()
    # the t hops across the antiperiodic boundary keep their sign inside the single block
    assert np.abs(D.F[3]).max() > 0 and np.abs(D.B[3]).max() > 0
