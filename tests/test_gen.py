"""The seeded input generator: SU(3) links, Gaussian sources, determinism."""
import numpy as np
import scipy.linalg as sl

import gen


def test_links_are_su3_and_match_expm():
    U = gen.su3_matrices(2000, 0.3, 1001)
    I3 = np.eye(3)
    assert np.abs(U @ np.conj(np.swapaxes(U, 1, 2)) - I3).max() < 1e-14
    assert np.abs(np.linalg.det(U) - 1).max() < 1e-14
    for k in (0, 17, 1999):
        A = gen.su3_generator(k, 1001)
        assert np.abs(A - A.conj().T).max() == 0 and abs(np.trace(A)) < 1e-15
        assert np.abs(sl.expm(1j * 0.3 * A) - U[k]).max() < 1e-14


def test_generator_coefficients_are_unit_normal():
    # A = sum_a c_a lambda_a / 2 with tr(lambda_a lambda_b) = 2 delta_ab, so
    # tr(A^2) = sum c_a^2 / 2 has mean 4 for c_a ~ N(0, 1)
    t = np.array([np.trace(gen.su3_generator(k, 5) @ gen.su3_generator(k, 5)).real for k in range(4000)])
    assert abs(t.mean() - 4.0) < 0.15


def test_gaussian_moments_and_counters():
    g = gen.gaussian(200001, 7)
    assert abs(g.mean()) < 0.01 and abs(g.var() - 1) < 0.01
    # counter-based: the same seed gives the same stream, a prefix is a prefix
    assert np.array_equal(gen.gaussian(1000, 7), g[:1000])
    assert not np.array_equal(gen.gaussian(1000, 8), g[:1000])


def test_gauge_field_layout_and_determinism():
    dims = (4, 2, 2, 6)
    U = gen.gauge_field(dims, 0.2, 3)
    assert U.shape == (6, 2, 2, 4, 4, 3, 3)
    flat = gen.su3_matrices(4 * 96, 0.2, 3).reshape(U.shape)
    assert np.array_equal(U, flat)
    assert np.array_equal(U, gen.gauge_field(dims, 0.2, 3))


def test_point_sources():
    dims = (2, 2, 2, 4)
    P = gen.point_sources(dims)
    assert P.shape == (12, 4, 2, 2, 2, 4, 3)
    assert np.abs(P.reshape(12, -1).sum(axis=1) - 1).max() == 0
    assert P[5, 0, 0, 0, 0, 1, 2] == 1
