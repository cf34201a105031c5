"""Small helpers shared by the tests (index arithmetic and closed forms only)."""
import numpy as np


def coords_grid(dims):
    """Arrays x0..x3 of shape (L3, L2, L1, L0) in canonical order."""
    x3, x2, x1, x0 = np.meshgrid(*(np.arange(dims[k]) for k in (3, 2, 1, 0)), indexing="ij")
    return x0, x1, x2, x3


def momenta(dims, n, tbc=1):
    """Lattice momenta p_mu = 2 pi n_mu / L_mu, shifted by pi/L3 in t when antiperiodic."""
    p = [2.0 * np.pi * n[mu] / dims[mu] for mu in range(4)]
    if tbc:
        p[3] += np.pi / dims[3]
    return np.array(p)


def plane_wave(dims, p, u):
    """psi(x) = exp(i p.x) u with u a (4,3) spin-colour vector."""
    x0, x1, x2, x3 = coords_grid(dims)
    ph = np.exp(1j * (p[0] * x0 + p[1] * x1 + p[2] * x2 + p[3] * x3))
    return ph[..., None, None] * np.asarray(u)[None, None, None, None]


def all_momenta(dims, tbc=1):
    for n0 in range(dims[0]):
        for n1 in range(dims[1]):
            for n2 in range(dims[2]):
                for n3 in range(dims[3]):
                    yield momenta(dims, (n0, n1, n2, n3), tbc)


def dense_matrix(apply, shape, columns):
    """Matrix of a linear map, one column per basis vector index in ``columns``
    (flat indices into a field of ``shape``); rows restricted to the same set."""
    cols = []
    for j in columns:
        e = np.zeros(int(np.prod(shape)), dtype=np.complex128)
        e[j] = 1.0
        cols.append(apply(e.reshape(shape)).reshape(-1)[columns])
    return np.stack(cols, axis=1)


def parity_flat_indices(dims, parity):
    """Flat complex-component indices of all sites of the given parity."""
    x0, x1, x2, x3 = coords_grid(dims)
    par = ((x0 + x1 + x2 + x3) & 1).reshape(-1)
    sites = np.nonzero(par == parity)[0]
    return (sites[:, None] * 12 + np.arange(12)[None, :]).reshape(-1)


def random_gauge_transform(dims, U, g):
    """U'_mu(x) = g(x) U_mu(x) g(x+mu)^dag with g of shape (L3,L2,L1,L0,3,3)."""
    Up = np.empty_like(U)
    axes = {0: 3, 1: 2, 2: 1, 3: 0}
    for mu in range(4):
        gshift = np.roll(g, -1, axis=axes[mu])
        Up[..., mu, :, :] = g @ U[..., mu, :, :] @ np.conj(np.swapaxes(gshift, -1, -2))
    return Up


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300)


def site_max_rel(got, expect):
    """Largest per-site relative error: ||got_x - expect_x|| / ||expect_x|| over
    the sites, the denominator floored at a tenth of the rms site norm (a site
    whose exact value is near zero is held to an absolute bound instead)."""
    g = np.asarray(got).reshape(-1, 12)
    e = np.asarray(expect).reshape(-1, 12)
    ne = np.linalg.norm(e, axis=1)
    d = np.linalg.norm(g - e, axis=1)
    floor = 0.1 * np.sqrt(np.mean(ne**2))
    return float(np.max(d / np.maximum(ne, floor)))
