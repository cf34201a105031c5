"""Pins of the oracle's Wilson-clover operator against closed forms, invariants
and brute force.  None of these compares the oracle with itself: each check
is a fact of the mathematics (Clifford algebra, free-field momentum space,
gamma5-hermiticity, gauge covariance, dense linear algebra) that a dropped
term, a wrong sign, a wrong index or a transposed operand would violate."""
import numpy as np
import pytest

import gen
import oracle
from helpers import (all_momenta, coords_grid, dense_matrix, momenta, parity_flat_indices, plane_wave,
                     random_gauge_transform, rel)

KAPPA = 0.12


def _gammas():
    return [oracle.gamma(mu) for mu in range(5)]


# ---------------------------------------------------------------------------
# gamma matrices: Clifford algebra, hermiticity, chirality
# ---------------------------------------------------------------------------

def test_gamma_clifford_and_chiral():
    g = _gammas()
    for mu in range(4):
        assert np.allclose(g[mu], g[mu].conj().T, atol=0)
        for nu in range(4):
            anti = g[mu] @ g[nu] + g[nu] @ g[mu]
            assert np.allclose(anti, 2.0 * (mu == nu) * np.eye(4), atol=1e-15)
    # gamma5 = g0 g1 g2 g3 is diagonal in a chiral basis
    assert np.allclose(g[4], g[0] @ g[1] @ g[2] @ g[3])
    assert np.allclose(g[4], np.diag([1, 1, -1, -1]))
    for mu in range(4):
        assert np.allclose(g[4] @ g[mu] + g[mu] @ g[4], 0)
    # sigma_munu is block diagonal (commutes with gamma5)
    for mu in range(4):
        for nu in range(4):
            sig = 0.5j * (g[mu] @ g[nu] - g[nu] @ g[mu])
            assert np.allclose(sig @ g[4], g[4] @ sig)


# ---------------------------------------------------------------------------
# free field: plane waves diagonalise the operator
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("dims,tbc", [((4, 4, 4, 4), 1), ((2, 2, 2, 2), 1), ((4, 2, 6, 4), 0), ((2, 4, 2, 6), 1)])
def test_free_field_plane_wave(dims, tbc):
    """Unit links: M e^{ipx} u = e^{ipx} [(1 - 2k sum cos p) + 2ik sum g_mu sin p_mu] u."""
    U = gen.unit_gauge(dims)
    g = _gammas()
    rng = np.random.default_rng(3)
    for n in [(0, 0, 0, 0), (1, 0, 0, 0), (0, 1, 1, 0), (1, 1, 1, 1), (0, 0, 1, 2)]:
        n = tuple(k % d for k, d in zip(n, dims))
        p = momenta(dims, n, tbc)
        u = rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))
        psi = plane_wave(dims, p, u)
        out = oracle.apply_M(dims, U, None, KAPPA, psi, tbc=tbc)
        Mp = (1 - 2 * KAPPA * np.cos(p).sum()) * np.eye(4) + 2j * KAPPA * sum(g[mu] * np.sin(p[mu]) for mu in range(4))
        expect = plane_wave(dims, p, Mp @ u)
        assert rel(out, expect) < 1e-13
        # gamma-independent form of the same statement (Clifford algebra only):
        # ||(M - (1 - 2k sum cos))psi||^2 = 4 k^2 sum sin^2 ||psi||^2
        d = out - (1 - 2 * KAPPA * np.cos(p).sum()) * psi
        assert abs(oracle.norm2(d) - 4 * KAPPA**2 * (np.sin(p) ** 2).sum() * oracle.norm2(psi)) < 1e-12 * oracle.norm2(psi)


def test_free_field_spectrum_dense_2x4():
    """Eigenvalues of the free M on 2^4 are 1 - 2k sum cos p +- 2ik sqrt(sum sin^2 p), each 6-fold."""
    dims = (2, 2, 2, 2)
    U = gen.unit_gauge(dims)
    shape = oracle.spinor_shape(dims)
    N = 12 * 16
    M = dense_matrix(lambda v: oracle.apply_M(dims, U, None, KAPPA, v), shape, np.arange(N))
    ev = np.linalg.eigvals(M)
    expect = []
    for p in all_momenta(dims, 1):
        re = 1 - 2 * KAPPA * np.cos(p).sum()
        im = 2 * KAPPA * np.sqrt((np.sin(p) ** 2).sum())
        expect += [re + 1j * im] * 6 + [re - 1j * im] * 6
    key = lambda z: (round(z.real, 9), round(z.imag, 9))
    assert np.allclose(sorted(ev, key=key), sorted(expect, key=key), atol=1e-12)


def test_free_field_solve_closed_form():
    """x = M(p)^-1 b exactly for a plane-wave source (even-odd CGLS path)."""
    dims = (4, 4, 4, 8)
    U = gen.unit_gauge(dims)
    g = _gammas()
    p = momenta(dims, (1, 0, 2, 3), 1)
    u = np.arange(12).reshape(4, 3) + 1j
    b = plane_wave(dims, p, u)
    A = oracle.clover(dims, U, KAPPA, 1.0)  # unit links: A = 1
    Ai = oracle.clover_inverse(A)
    x, it, _ = oracle.solve(dims, U, A, Ai, KAPPA, b, tol=1e-12)
    assert it > 0
    Mp = (1 - 2 * KAPPA * np.cos(p).sum()) * np.eye(4) + 2j * KAPPA * sum(g[mu] * np.sin(p[mu]) for mu in range(4))
    expect = plane_wave(dims, p, np.linalg.solve(Mp, u))
    assert rel(x, expect) < 1e-10


# ---------------------------------------------------------------------------
# adjoints and gamma5-hermiticity on random links
# ---------------------------------------------------------------------------

def _inner(a, b):
    return np.vdot(np.asarray(a).ravel(), np.asarray(b).ravel())


@pytest.fixture(scope="module")
def rough():
    dims = (4, 4, 2, 6)
    U = gen.gauge_field(dims, 0.6, 11)
    A = oracle.clover(dims, U, KAPPA, 1.3)
    Ai = oracle.clover_inverse(A)
    return dims, U, A, Ai


def test_adjoint_and_gamma5_hermiticity(rough):
    dims, U, A, Ai = rough
    u = gen.gaussian_spinor(dims, 21)[0]
    v = gen.gaussian_spinor(dims, 22)[0]
    g5 = oracle.gamma5
    # <u, D v> = <D^dag u, v>  and  D^dag = g5 D g5
    Dv = oracle.hop(dims, U, v)
    Ddu = oracle.hop(dims, U, u, dagger=True)
    assert abs(_inner(u, Dv) - _inner(Ddu, v)) < 1e-12 * abs(_inner(u, Dv))
    assert rel(Ddu, g5(oracle.hop(dims, U, g5(u)))) < 1e-14
    # full M with clover
    Mv = oracle.apply_M(dims, U, A, KAPPA, v)
    g5Mg5u = g5(oracle.apply_M(dims, U, A, KAPPA, g5(u)))
    assert abs(_inner(u, Mv) - _inner(g5Mg5u, v)) < 1e-12 * abs(_inner(u, Mv))
    # Schur complement
    uo = oracle.keep_parity(dims, u, 1)
    vo = oracle.keep_parity(dims, v, 1)
    Mh_v = oracle.apply_Mhat(dims, U, A, Ai, KAPPA, vo)
    Mhd_u = oracle.apply_Mhat(dims, U, A, Ai, KAPPA, uo, dagger=True)
    assert abs(_inner(uo, Mh_v) - _inner(Mhd_u, vo)) < 1e-12 * abs(_inner(uo, Mh_v))
    assert rel(Mhd_u, g5(oracle.apply_Mhat(dims, U, A, Ai, KAPPA, g5(uo)))) < 1e-13


def test_gauge_covariance(rough):
    """M[U^g](g psi) = g M[U] psi, F[U^g] = g F g^dag."""
    dims, U, _, _ = rough
    L = dims
    g = gen.su3_matrices(int(np.prod(L)), 1.0, 99).reshape(L[3], L[2], L[1], L[0], 3, 3)
    Ug = random_gauge_transform(dims, U, g)
    psi = gen.gaussian_spinor(dims, 5)[0]
    gpsi = np.einsum("tzyxab,tzyxsb->tzyxsa", g, psi)
    A = oracle.clover(dims, U, KAPPA, 1.0)
    Ag = oracle.clover(dims, Ug, KAPPA, 1.0)
    lhs = oracle.apply_M(dims, Ug, Ag, KAPPA, gpsi)
    rhs = np.einsum("tzyxab,tzyxsb->tzyxsa", g, oracle.apply_M(dims, U, A, KAPPA, psi))
    assert rel(lhs, rhs) < 1e-13
    gflat = g.reshape(-1, 3, 3)
    for s in (0, 7, 50):
        for mu, nu in ((0, 1), (1, 3), (2, 3)):
            F = oracle.field_strength(dims, U, s, mu, nu)
            Fg = oracle.field_strength(dims, Ug, s, mu, nu)
            assert np.allclose(Fg, gflat[s] @ F @ gflat[s].conj().T, atol=1e-13)


# ---------------------------------------------------------------------------
# clover term
# ---------------------------------------------------------------------------

def test_clover_structure(rough):
    dims, U, A, Ai = rough
    V = A.shape[0]
    # Hermitian, trace 12 (sigma traceless), block diagonal in the chiral basis
    assert np.abs(A - np.conj(np.swapaxes(A, 1, 2))).max() < 1e-14
    assert np.abs(np.trace(A, axis1=1, axis2=2) - 12).max() < 1e-13
    assert np.abs(A[:, :6, 6:]).max() < 1e-15 and np.abs(A[:, 6:, :6]).max() < 1e-15
    assert np.abs(A @ Ai - np.eye(12)).max() < 1e-13
    assert A.shape == (V, 12, 12)
    # c_sw = 0 and unit links both give A = 1
    assert np.abs(oracle.clover(dims, U, KAPPA, 0.0) - np.eye(12)).max() == 0
    assert np.abs(oracle.clover(dims, gen.unit_gauge(dims), KAPPA, 1.0) - np.eye(12)).max() < 1e-15


def test_clover_constant_abelian_field():
    """U_0(x) = exp(-i f x1 T), T = diag(1,-1,0), other links 1: every leaf of the
    (0,1) clover is exp(i f T), so F_01 = diag(sin f, -sin f, 0), all other F vanish,
    and A = 1 - c_sw kappa sigma_01 (x) F_01."""
    dims = (4, 6, 4, 4)
    f = 2 * np.pi * 2 / dims[1]
    U = gen.unit_gauge(dims)
    x0, x1, x2, x3 = coords_grid(dims)
    T = np.array([1.0, -1.0, 0.0])
    U[..., 0, :, :] = 0
    for k in range(3):
        U[..., 0, k, k] = np.exp(-1j * f * x1 * T[k])
    csw = 1.7
    A = oracle.clover(dims, U, KAPPA, csw)
    g = _gammas()
    sig01 = 0.5j * (g[0] @ g[1] - g[1] @ g[0])
    F01 = np.diag(np.sin(f * T))
    expect = np.eye(12) - csw * KAPPA * np.kron(sig01, F01)
    assert np.abs(A - expect[None]).max() < 1e-14
    for mu, nu in ((0, 2), (0, 3), (1, 2), (2, 3)):
        assert np.abs(oracle.field_strength(dims, U, 5, mu, nu)).max() < 1e-15
    assert np.allclose(oracle.field_strength(dims, U, 5, 0, 1), F01, atol=1e-15)


def test_gauss_jordan_inverse_against_library():
    rng = np.random.default_rng(0)
    M = rng.standard_normal((12, 12)) + 1j * rng.standard_normal((12, 12))
    assert np.abs(oracle.inverse(M) - np.linalg.inv(M)).max() < 1e-12


# ---------------------------------------------------------------------------
# dense 2^4 brute force: Schur complement, normal operator, exact solve
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def dense24():
    dims = (2, 2, 2, 2)
    U = gen.gauge_field(dims, 0.5, 4)
    A = oracle.clover(dims, U, 0.13, 1.0)
    Ai = oracle.clover_inverse(A)
    shape = oracle.spinor_shape(dims)
    full = np.arange(12 * 16)
    M = dense_matrix(lambda v: oracle.apply_M(dims, U, A, 0.13, v), shape, full)
    return dims, U, A, Ai, M


def test_dense_schur_complement(dense24):
    dims, U, A, Ai, M = dense24
    shape = oracle.spinor_shape(dims)
    e = parity_flat_indices(dims, 0)
    o = parity_flat_indices(dims, 1)
    schur = M[np.ix_(o, o)] - M[np.ix_(o, e)] @ np.linalg.solve(M[np.ix_(e, e)], M[np.ix_(e, o)])
    Mhat = dense_matrix(lambda v: oracle.apply_Mhat(dims, U, A, Ai, 0.13, v), shape, o)
    assert np.abs(Mhat - schur).max() < 1e-13
    Mhat_dag = dense_matrix(lambda v: oracle.apply_Mhat(dims, U, A, Ai, 0.13, v, dagger=True), shape, o)
    assert np.abs(Mhat_dag - Mhat.conj().T).max() < 1e-13
    N = Mhat.conj().T @ Mhat
    assert np.abs(N - N.conj().T).max() < 1e-13
    assert np.linalg.eigvalsh(N).min() > 0
    # the hop only couples opposite parities, so the same-parity blocks of M
    # are the clover matrices of those sites
    even_sites = e[::12] // 12
    blk = np.zeros((len(e), len(e)), dtype=np.complex128)
    for k, s in enumerate(even_sites):
        blk[12 * k:12 * k + 12, 12 * k:12 * k + 12] = A[s]
    assert np.abs(M[np.ix_(e, e)] - blk).max() < 1e-15


def test_dense_symmetric_schur_complement(dense24):
    """The symmetric form is M_oo^-1 times the Schur complement of M's even
    block (M_oo = A_oo: the hop couples opposite parities only), its adjoint
    is the conjugate transpose, and it solves for the same x_o as M x = b."""
    dims, U, A, Ai, M = dense24
    shape = oracle.spinor_shape(dims)
    e = parity_flat_indices(dims, 0)
    o = parity_flat_indices(dims, 1)
    Moo, Moe, Meo, Mee = M[np.ix_(o, o)], M[np.ix_(o, e)], M[np.ix_(e, o)], M[np.ix_(e, e)]
    schur = Moo - Moe @ np.linalg.solve(Mee, Meo)
    sym = np.linalg.solve(Moo, schur)
    assert np.abs(sym - (np.eye(len(o)) - np.linalg.solve(Moo, Moe) @ np.linalg.solve(Mee, Meo))).max() < 1e-13
    Ms = dense_matrix(lambda v: oracle.apply_Mhat_sym(dims, U, A, Ai, 0.13, v), shape, o)
    assert np.abs(Ms - sym).max() < 1e-13
    Msd = dense_matrix(lambda v: oracle.apply_Mhat_sym(dims, U, A, Ai, 0.13, v, dagger=True), shape, o)
    assert np.abs(Msd - sym.conj().T).max() < 1e-13
    # same solution: x_o of M x = b solves sym x_o = M_oo^-1 (b_o - M_oe M_ee^-1 b_e)
    b = gen.gaussian_spinor(dims, 9)[0].reshape(-1)
    x = np.linalg.solve(M, b)
    rhs = np.linalg.solve(Moo, b[o] - Moe @ np.linalg.solve(Mee, b[e]))
    assert rel(np.linalg.solve(Ms, rhs), x[o]) < 1e-12
    # the symmetric form is not gamma5-hermitian (unlike Mhat): g5 Ms g5 != Ms^dag
    g5 = np.diag(np.tile(np.repeat([1.0, 1.0, -1.0, -1.0], 3), len(o) // 12))
    assert np.abs(g5 @ Ms @ g5 - Msd).max() > 1e-3


def test_symmetric_schur_adjoint_and_wilson_limit(rough):
    dims, U, A, Ai = rough
    u = oracle.keep_parity(dims, gen.gaussian_spinor(dims, 31)[0], 1)
    v = oracle.keep_parity(dims, gen.gaussian_spinor(dims, 32)[0], 1)
    Msv = oracle.apply_Mhat_sym(dims, U, A, Ai, KAPPA, v)
    Msdu = oracle.apply_Mhat_sym(dims, U, A, Ai, KAPPA, u, dagger=True)
    assert abs(_inner(u, Msv) - _inner(Msdu, v)) < 1e-12 * abs(_inner(u, Msv))
    # Ms = 1 - kappa^2 A_oo^-1 D_oe A_ee^-1 D_eo, composed from the hop and the site matrices
    t = oracle.keep_parity(dims, oracle.hop(dims, U, v), 0)
    t = oracle.keep_parity(dims, oracle.hop(dims, U, oracle.site_mul(Ai, t)), 1)
    assert rel(Msv, v - KAPPA ** 2 * oracle.site_mul(Ai, t)) < 1e-13
    # c_sw = 0: A = 1 and the two forms coincide
    assert rel(oracle.apply_Mhat_sym(dims, U, None, None, KAPPA, v), oracle.apply_Mhat(dims, U, None, None, KAPPA, v)) \
        < 1e-15


def test_dense_solve(dense24):
    dims, U, A, Ai, M = dense24
    b = gen.gaussian_spinor(dims, 8)[0]
    x, it, _ = oracle.solve(dims, U, A, Ai, 0.13, b, tol=1e-13)
    xd = np.linalg.solve(M, b.reshape(-1)).reshape(b.shape)
    assert it > 0
    assert rel(x, xd) < 1e-11
    assert oracle.true_residual(dims, U, A, 0.13, x, b) < 1e-12


def test_hop_on_2x4_sums_both_directions():
    """On 2^4 the sites x+mu and x-mu coincide; unit links, periodic: D const = 8 const."""
    dims = (2, 2, 2, 2)
    U = gen.unit_gauge(dims)
    u = np.arange(12).reshape(4, 3) * (1 + 0.5j)
    psi = np.broadcast_to(u, oracle.spinor_shape(dims)).copy()
    assert rel(oracle.hop(dims, U, psi, tbc=0), 8 * psi) < 1e-15
    # antiperiodic t: at t=0 the backward hop wraps, so the mu=3 pair is
    # (1-g3)psi - (1+g3)psi = -2 g3 psi; at t=1 the forward hop wraps: +2 g3 psi
    g3 = oracle.gamma(3)
    expect = np.empty_like(psi)
    expect[0] = 6 * u - 2 * (g3 @ u)
    expect[1] = 6 * u + 2 * (g3 @ u)
    assert rel(oracle.hop(dims, U, psi, tbc=1), expect) < 1e-15


def test_cgls_interacting_clover():
    dims = (4, 4, 4, 8)
    U = gen.gauge_field(dims, 0.3, 1001)
    A = oracle.clover(dims, U, 0.125, 1.0)
    Ai = oracle.clover_inverse(A)
    b = gen.gaussian_spinor(dims, 2001)[0]
    x, it, r = oracle.solve(dims, U, A, Ai, 0.125, b, tol=0.5e-10)
    assert it > 0
    assert oracle.true_residual(dims, U, A, 0.125, x, b) <= 1e-10
    # the even-odd decomposition's own identities: Mhat x_o = bhat_o
    xo = oracle.keep_parity(dims, x, 1)
    bhat = oracle.prepare_source(dims, U, Ai, 0.125, b)
    assert rel(oracle.apply_Mhat(dims, U, A, Ai, 0.125, xo), bhat) < 1e-10


def test_mhat_slab_matches_full(rough):
    """The time-slab restriction of Mhat (used to bound CPU timings) equals the
    full application on those slices, including the t wrap."""
    dims, U, A, Ai = rough
    psi = gen.gaussian_spinor(dims, 31)[0]
    full = oracle.apply_Mhat(dims, U, A, Ai, KAPPA, psi)
    for t0, t1 in ((0, 1), (2, 4), (5, 6), (0, dims[3])):
        out = oracle.mhat_slab(dims, U, A, Ai, KAPPA, psi, t0, t1)
        assert np.abs(out[t0:t1] - full[t0:t1]).max() < 1e-14 * np.abs(full).max()
        rest = np.delete(out, range(t0, t1), axis=0)
        assert rest.size == 0 or np.abs(rest).max() == 0


# ---------------------------------------------------------------------------
# the checker of every solve: true_residual = ||b - M x|| / ||b||
# ---------------------------------------------------------------------------

def test_true_residual_free_field_closed_form():
    """Unit links, b a plane wave, x = M(p)^-1 b + eps v with v another plane
    wave: the residual is eps ||M(q) v|| / ||b|| with M(q) the momentum-space
    matrix 1 - 2k sum cos q + 2ik sum g sin q, computed here without the
    oracle's operator.  A missing square root, a wrong denominator or a sign
    error in b - M x changes the value."""
    dims = (4, 4, 4, 8)
    U = gen.unit_gauge(dims)
    g = _gammas()

    def Mmom(q):
        return (1 - 2 * KAPPA * np.cos(q).sum()) * np.eye(4) + 2j * KAPPA * sum(g[mu] * np.sin(q[mu]) for mu in range(4))

    p = momenta(dims, (1, 2, 0, 3), 1)
    q = momenta(dims, (0, 1, 3, 1), 1)
    u = (np.arange(12).reshape(4, 3) + 1.0) * (1 - 0.5j)
    w = np.cos(np.arange(12)).reshape(4, 3) + 1j * np.sin(3.0 * np.arange(12)).reshape(4, 3)
    b = plane_wave(dims, p, u)
    x0 = plane_wave(dims, p, np.linalg.solve(Mmom(p), u))
    assert oracle.true_residual(dims, U, None, KAPPA, x0, b) < 1e-14
    assert oracle.true_residual(dims, U, None, KAPPA, np.zeros_like(b), b) == 1.0
    for eps in (1e-3, 0.25):
        x = x0 + eps * plane_wave(dims, q, w)
        V = int(np.prod(dims))
        expect = eps * np.linalg.norm(Mmom(q) @ w) * np.sqrt(V) / (np.linalg.norm(u) * np.sqrt(V))
        assert abs(oracle.true_residual(dims, U, None, KAPPA, x, b) / expect - 1) < 1e-12


def test_true_residual_dense_clover(dense24):
    """With the clover term (2^4, dense M): x = M^-1 b + d gives ||M d|| / ||b||,
    the residual is invariant under (x, b) -> (c x, c b), and x = 0 gives 1."""
    dims, U, A, Ai, M = dense24
    b = gen.gaussian_spinor(dims, 41)[0]
    d = 1e-4 * gen.gaussian_spinor(dims, 42)[0]
    x = np.linalg.solve(M, b.reshape(-1)).reshape(b.shape) + d
    expect = np.linalg.norm(M @ d.reshape(-1)) / np.linalg.norm(b)
    r = oracle.true_residual(dims, U, A, 0.13, x, b)
    assert abs(r / expect - 1) < 1e-8
    assert abs(oracle.true_residual(dims, U, A, 0.13, (2.5 - 1j) * x, (2.5 - 1j) * b) / r - 1) < 1e-12
    assert oracle.true_residual(dims, U, A, 0.13, np.zeros_like(b), b) == 1.0
    # the clover term is part of the operator it checks: without it the value differs
    assert abs(oracle.true_residual(dims, U, None, 0.13, x, b) - r) > 1e-3


def test_site_list_variants_match_full(rough):
    """hop_sites and clover_sites (the per-site evaluations of the full-size
    parity test) equal the full-lattice hop and clover at any site list,
    including the boundary sites, both time boundary conditions and the
    adjoint hop."""
    dims, U, A, Ai = rough
    V = int(np.prod(dims))
    psi = gen.gaussian_spinor(dims, 51)[0]
    rng = np.random.default_rng(5)
    sites = np.concatenate([[0, V - 1, dims[0] - 1, V - dims[0]], rng.choice(V, 40, replace=False)])
    for tbc in (0, 1):
        for dag in (False, True):
            full = oracle.hop(dims, U, psi, tbc, dagger=dag).reshape(V, 4, 3)
            assert np.abs(oracle.hop_sites(dims, U, psi, sites, tbc, dagger=dag) - full[sites]).max() == 0
    Af = oracle.clover(dims, U, KAPPA, 1.3)
    assert np.abs(oracle.clover_sites(dims, U, KAPPA, 1.3, sites) - Af[sites]).max() == 0
    assert np.abs(Af - A).max() == 0
