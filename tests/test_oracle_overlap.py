"""Pins of the oracle's overlap pieces: the Chebyshev series for 1/sqrt(y),
the polynomial sign function, the overlap operator and the low-mode solver.
Checked against a library Chebyshev evaluator, the Bernstein-ellipse error
rate, free-field momentum space, dense eigendecompositions, sign(H)^2 = 1 and
the Ginsparg-Wilson relation."""
import numpy as np
import pytest

import gen
import oracle
from helpers import all_momenta, dense_matrix, momenta, plane_wave, rel

RHO = 1.5
B_MAX = 6.5**2  # ||H_W|| <= (4 - rho) + 4 for unitary links


def test_chebyshev_series_against_library():
    a, b, n = 0.3, B_MAX, 40
    c = oracle.cheb_coeffs(a, b, n)
    for y in (0.3, 1.0, 7.7, 20.0, 42.25):
        t = (2 * y - a - b) / (b - a)
        assert abs(oracle.cheb_eval(a, b, c, y) - np.polynomial.chebyshev.chebval(t, c)) < 1e-14
    # interpolation: exact at the Chebyshev-Gauss nodes
    nodes = 0.5 * ((b - a) * np.cos(np.pi * (np.arange(n + 1) + 0.5) / (n + 1)) + a + b)
    for y in nodes:
        assert abs(oracle.cheb_eval(a, b, c, y) - 1 / np.sqrt(y)) < 1e-12 / np.sqrt(y)


def test_chebyshev_error_rate_bernstein():
    """The error of the degree-n interpolant of 1/sqrt(y) decays like R^-n with
    R = |t0| + sqrt(t0^2 - 1), t0 the image of the singularity y = 0."""
    a, b = 0.5, B_MAX
    t0 = (a + b) / (b - a)
    R = t0 + np.sqrt(t0 * t0 - 1)
    ns = np.array([20, 40, 60, 80])
    errs = np.array([oracle.sign_error(a, b, oracle.cheb_coeffs(a, b, n), 20000) for n in ns])
    slope = np.polyfit(ns, np.log(errs), 1)[0]
    assert abs(slope + np.log(R)) < 0.1 * np.log(R)


def test_degree_search_is_minimal():
    a, b, tol = 0.8, B_MAX, 1e-10
    n, c = oracle.cheb_degree(a, b, tol)
    assert oracle.sign_error(a, b, c) <= tol
    assert oracle.sign_error(a, b, oracle.cheb_coeffs(a, b, n - 1)) > tol


def _free_N2(p):
    return (4 - RHO - np.cos(p).sum()) ** 2 + (np.sin(p) ** 2).sum()


def test_free_field_overlap_closed_form():
    """Unit links: gamma5 eps(H_W) = D_W(p)/N(p), so D_ov(p) = rho (1 + D_W(p)/N(p))."""
    dims = (4, 4, 4, 4)
    U = gen.unit_gauge(dims)
    g = [oracle.gamma(mu) for mu in range(4)]
    a = 0.99 * min(_free_N2(p) for p in all_momenta(dims, 1))
    n, c = oracle.cheb_degree(a, B_MAX, 1e-12)
    rng = np.random.default_rng(1)
    for m in (0.0, 0.05):
        for nn in [(0, 0, 0, 0), (1, 2, 0, 3), (2, 2, 2, 1)]:
            p = momenta(dims, nn, 1)
            u = rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))
            psi = plane_wave(dims, p, u)
            out = oracle.apply_overlap(dims, U, RHO, m, psi, a, B_MAX, c)
            DW = (4 - RHO - np.cos(p).sum()) * np.eye(4) + 1j * sum(g[mu] * np.sin(p[mu]) for mu in range(4))
            Dov = (1 - m / (2 * RHO)) * RHO * (np.eye(4) + DW / np.sqrt(_free_N2(p))) + m * np.eye(4)
            assert rel(out, plane_wave(dims, p, Dov @ u)) < 1e-10


@pytest.fixture(scope="module")
def dense_hw():
    dims = (2, 2, 2, 2)
    U = gen.gauge_field(dims, 0.4, 17)
    shape = oracle.spinor_shape(dims)
    H = dense_matrix(lambda v: oracle.apply_HW(dims, U, RHO, v), shape, np.arange(192))
    lam, Vec = np.linalg.eigh(H)
    return dims, U, H, lam, Vec


def test_polynomial_sign_against_dense_eigh(dense_hw):
    dims, U, H, lam, Vec = dense_hw
    assert np.abs(H - H.conj().T).max() < 1e-14  # H_W is Hermitian
    exact = Vec @ np.diag(np.sign(lam)) @ Vec.conj().T
    v = gen.gaussian_spinor(dims, 3)[0]
    ex = (exact @ v.reshape(-1)).reshape(v.shape)
    # no projection: interval from the smallest |lambda|
    order = np.argsort(np.abs(lam))
    a = 0.999 * lam[order[0]] ** 2
    n, c = oracle.cheb_degree(a, B_MAX, 1e-12)
    assert rel(oracle.apply_sign(dims, U, RHO, v, a, B_MAX, c), ex) < 1e-10
    # six low modes treated exactly, interval from the seventh
    k = 6
    low = order[:k]
    vecs = Vec[:, low].T.reshape((k,) + v.shape)
    a = 0.999 * lam[order[k]] ** 2
    n2, c2 = oracle.cheb_degree(a, B_MAX, 1e-12)
    assert n2 <= n
    out = oracle.apply_sign(dims, U, RHO, v, a, B_MAX, c2, lam=lam[low], vecs=vecs)
    assert rel(out, ex) < 1e-10


def test_low_modes_dense_pairs(dense_hw):
    dims, U, H, lam, Vec = dense_hw
    k = 10
    lo, vecs = oracle.low_modes_dense(dims, U, RHO, k)
    order = np.argsort(np.abs(lam))
    assert np.allclose(np.abs(lo), np.abs(lam[order[:k]]), atol=1e-12)
    res, ortho = oracle.eigen_residuals(dims, U, RHO, lo, vecs)
    assert res.max() < 1e-12 and ortho < 1e-12


def test_free_field_spectrum_closed_form():
    """Unit links: the eigenvalues of H_W are +-N(p), six-fold each."""
    dims = (2, 2, 4, 4)
    U = gen.unit_gauge(dims)
    V = int(np.prod(dims))
    lo, _ = oracle.low_modes_dense(dims, U, RHO, 12 * V)
    expect = []
    for p in all_momenta(dims, 1):
        expect += [np.sqrt(_free_N2(p))] * 6 + [-np.sqrt(_free_N2(p))] * 6
    assert np.allclose(np.sort(lo), np.sort(expect), atol=1e-12)


@pytest.fixture(scope="module")
def interacting():
    dims = (4, 2, 4, 4)
    U = gen.gauge_field(dims, 0.3, 23)
    k = 8
    lam, vecs = oracle.low_modes_dense(dims, U, RHO, k + 1)
    a = lam[k] ** 2
    n, c = oracle.cheb_degree(a, B_MAX, 1e-11)
    return dims, U, lam[:k], vecs[:k], a, c


def test_sign_squares_to_one(interacting):
    dims, U, lam, vecs, a, c = interacting
    v = gen.gaussian_spinor(dims, 9)[0]
    e1 = oracle.apply_sign(dims, U, RHO, v, a, B_MAX, c, lam=lam, vecs=vecs)
    e2 = oracle.apply_sign(dims, U, RHO, e1, a, B_MAX, c, lam=lam, vecs=vecs)
    assert rel(e2, v) < 1e-9
    # eps is Hermitian
    w = gen.gaussian_spinor(dims, 10)[0]
    ew = oracle.apply_sign(dims, U, RHO, w, a, B_MAX, c, lam=lam, vecs=vecs)
    assert abs(np.vdot(w, e1) - np.vdot(ew, v)) < 1e-9 * abs(np.vdot(w, e1))


def test_ginsparg_wilson(interacting):
    """g5 D + D g5 = (1/rho) D g5 D for the massless overlap operator."""
    dims, U, lam, vecs, a, c = interacting
    v = gen.gaussian_spinor(dims, 12)[0]
    D = lambda x: oracle.apply_overlap(dims, U, RHO, 0.0, x, a, B_MAX, c, lam=lam, vecs=vecs)
    g5 = oracle.gamma5
    lhs = g5(D(v)) + D(g5(v))
    rhs = D(g5(D(v))) / RHO
    assert rel(lhs, rhs) < 1e-9
    # adjoint: <u, D v> = <D^dag u, v>
    u = gen.gaussian_spinor(dims, 13)[0]
    Dd = oracle.apply_overlap(dims, U, RHO, 0.05, u, a, B_MAX, c, lam=lam, vecs=vecs, dagger=True)
    Dv = oracle.apply_overlap(dims, U, RHO, 0.05, v, a, B_MAX, c, lam=lam, vecs=vecs)
    assert abs(np.vdot(u, Dv) - np.vdot(Dd, v)) < 1e-9 * abs(np.vdot(u, Dv))


# ---- the overlap eigensystem: chirality sectors of D_ov(0)^dag D_ov(0) -----

def test_sector_spectrum_free_field_closed_form():
    """Unit links: per momentum D_ov(p) = rho (1 + D_W(p)/N(p)) (colour
    diagonal), so the sector-s spectrum is the union over p of the eigenvalues
    of the spin-s block of D_ov(p)^dag D_ov(p), three times each."""
    dims = (2, 2, 2, 4)
    U = gen.unit_gauge(dims)
    V = int(np.prod(dims))
    g = [oracle.gamma(mu) for mu in range(4)]
    for s in (+1, -1):
        blk = [0, 1] if s > 0 else [2, 3]
        expect = []
        for p in all_momenta(dims, 1):
            DW = (4 - RHO - np.cos(p).sum()) * np.eye(4) + 1j * sum(g[mu] * np.sin(p[mu]) for mu in range(4))
            D = RHO * (np.eye(4) + DW / np.sqrt(_free_N2(p)))
            M = (D.conj().T @ D)[np.ix_(blk, blk)]
            expect += list(np.linalg.eigvalsh(0.5 * (M + M.conj().T))) * 3
        mu, vecs = oracle.overlap_sector_eigensystem(dims, U, RHO, 6 * V, s)
        assert np.allclose(mu, np.sort(expect), atol=1e-11)
        # the vectors are chiral and orthonormal
        Z = vecs.reshape(6 * V, -1)
        assert np.abs(Z[:, oracle.chirality_indices(dims, -s)]).max() == 0
        assert np.abs(Z.conj() @ Z.T - np.eye(6 * V)).max() < 1e-11


def test_sector_spectra_pair_up_with_the_overlap_spectrum():
    """Interacting field: D_ov(0)'s eigenvalues lie on the Ginsparg-Wilson
    circle |lambda - rho| = rho, and the two sectors' spectra together are the
    moduli |lambda|^2 (each pair lambda, lambda* gives one value per sector;
    chiral zero modes and lambda = 2 rho only one)."""
    dims = (2, 2, 2, 2)
    U = gen.gauge_field(dims, 0.5, 41)
    V = int(np.prod(dims))
    D = oracle.overlap_dense(dims, U, RHO)
    lam = np.linalg.eigvals(D)
    assert np.abs(np.abs(lam - RHO) - RHO).max() < 1e-11
    mp, _ = oracle.overlap_sector_eigensystem(dims, U, RHO, 6 * V, +1)
    mm, _ = oracle.overlap_sector_eigensystem(dims, U, RHO, 6 * V, -1)
    assert np.allclose(np.sort(np.concatenate([mp, mm])), np.sort(np.abs(lam) ** 2), atol=1e-10)
    # away from 0 and 4 rho^2 the two sectors carry the same values
    inner = lambda m: np.sort(m[(m > 1e-8) & (m < 4 * RHO**2 - 1e-8)])
    assert np.allclose(inner(mp), inner(mm), atol=1e-10)
    # the pair formula reproduces D_ov(0)'s eigenvalues with Im >= 0
    re, im = oracle.overlap_pair_eigenvalues(mp, RHO)
    up = lam[lam.imag >= -1e-12]
    for r, i in zip(re[:20], im[:20]):
        assert np.abs(up - (r + 1j * i)).min() < 1e-8


def test_sector_vectors_against_the_polynomial_operator():
    """The dense sector eigenvectors are eigenvectors of the operator the GPU
    eigensolver applies, 2 rho^2 P_s (1 + s eps) P_s with the polynomial sign
    function, to the polynomial's accuracy; and D_ov(0) maps a sector vector to
    a D^dag D eigenvector of the same eigenvalue."""
    dims = (2, 2, 2, 4)
    U = gen.gauge_field(dims, 0.4, 43)
    k = 10
    lam_w, vecs_w = oracle.low_modes_dense(dims, U, RHO, 5)
    a = lam_w[4] ** 2
    n, c = oracle.cheb_degree(a, B_MAX, 1e-12)
    D = oracle.overlap_dense(dims, U, RHO)
    for s in (+1, -1):
        mu, chi = oracle.overlap_sector_eigensystem(dims, U, RHO, k, s)
        for i in range(k):
            h = oracle.apply_sector_normal(dims, U, RHO, s, chi[i], a, B_MAX, c, lam=lam_w[:4], vecs=vecs_w[:4])
            assert np.linalg.norm((h - mu[i] * chi[i]).ravel()) < 1e-9
            w = D @ chi[i].ravel()
            assert np.linalg.norm(D.conj().T @ (D @ w) - mu[i] * w) < 1e-9 * max(1.0, np.linalg.norm(w))


def test_overlap_acts_on_a_pair_as_a_two_by_two_matrix():
    """The deflated CG's identity: for a sector-s eigenvector chi with
    eps chi = c chi + n eta (eta of the other chirality, |eta| = 1),
    D_ov(0) chi = rho ((1 + s c) chi - s n eta) and
    D_ov(0) eta = rho (s n chi + (1 + s c) eta), checked on the dense D_ov."""
    dims = (2, 2, 2, 4)
    U = gen.gauge_field(dims, 0.4, 47)
    D = oracle.overlap_dense(dims, U, RHO)
    N = D.shape[0]
    g5 = np.ones(N)
    g5[oracle.chirality_indices(dims, -1)] = -1.0
    eps = g5[:, None] * (D / RHO - np.eye(N))  # D = rho (1 + g5 eps)
    for s in (+1, -1):
        mu, chi = oracle.overlap_sector_eigensystem(dims, U, RHO, 6, s)
        for i in range(6):
            x = chi[i].ravel()
            e = eps @ x
            c = np.vdot(x, e).real
            other = oracle.chirality_indices(dims, -s)
            y = np.zeros(N, dtype=np.complex128)
            y[other] = e[other]
            n = np.linalg.norm(y)
            eta = y / n
            assert abs(mu[i] - 2 * RHO**2 * (1 + s * c)) < 1e-10
            assert np.linalg.norm(D @ x - RHO * ((1 + s * c) * x - s * n * eta)) < 1e-10
            assert np.linalg.norm(D @ eta - RHO * (s * n * x + (1 + s * c) * eta)) < 1e-10
