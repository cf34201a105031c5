"""The host side of the GPU multigrid (paper_2001_05706_gb300/multigrid.py:
flexible GCR, MR, near-null vectors, the K-cycle) on CPU.  Each lqcd_mg_*
call is replaced by the multigrid oracle's numpy arithmetic on CPU tensors,
so the sequencing of the calls -- which vectors each one reads and writes,
the Gram-Schmidt passes, restarts and the cycle -- is checked against the
oracle's own solver without a GPU."""
import types

import numpy as np
import pytest

import gen
import oracle
from oracle import multigrid as omg

torch = pytest.importorskip("torch")


def _np(t):
    return t.numpy()


def _chi(n):
    return np.array([1] * (n // 2) + [-1] * (n // 2))


def _stencil(dims, n, X, F, B):
    V = int(np.prod(dims))
    return omg.Stencil(dims, _np(X).reshape(V, n, n), _np(F).reshape(4, V, n, n), _np(B).reshape(4, V, n, n), _chi(n))


def _prolongator(dims, n, block, nc, P):
    """An oracle prolongator with the given matrices (geometry from random vectors)."""
    V = int(np.prod(dims))
    fine = types.SimpleNamespace(dims=tuple(dims), V=V, n=n, chi=_chi(n))
    rng = np.random.default_rng(0)
    pr = omg.Prolongator(fine, block, rng.standard_normal((nc // 2, V, n)) + 0j)
    pr.Ps = _np(P).reshape(V, n, nc)
    return pr


class _Shim:
    """torch with device arguments dropped and from_numpy(...).to(...) a no-op."""
    complex128 = torch.complex128

    @staticmethod
    def zeros(*a, device=None, **k):
        return torch.zeros(*a, **k)

    @staticmethod
    def empty(*a, device=None, **k):
        return torch.zeros(*a, **k)

    zeros_like = staticmethod(torch.zeros_like)
    empty_like = staticmethod(torch.zeros_like)

    @staticmethod
    def from_numpy(a):
        t = torch.from_numpy(a)
        return types.SimpleNamespace(to=lambda dev: t)


@pytest.fixture
def gmg(monkeypatch):
    from paper_2001_05706_gb300 import multigrid as m

    def apply(ctx, dims, n, X, F, B, v, out):
        _np(out).reshape(-1, n)[:] = _stencil(dims, n, X, F, B).apply(_np(v))

    def orthonormalize(ctx, dims, n, block, nv, vecs, P):
        V = int(np.prod(dims))
        fine = types.SimpleNamespace(dims=tuple(dims), V=V, n=n, chi=_chi(n))
        _np(P).reshape(V, n, 2 * nv)[:] = omg.Prolongator(fine, block, _np(vecs).reshape(nv, V, n)).Ps

    def prolong(ctx, dims, n, block, nc, P, w, out):
        _np(out).reshape(-1, n)[:] = _prolongator(dims, n, block, nc, P).prolong(_np(w))

    def restrict(ctx, dims, n, block, nc, P, v, out):
        _np(out).reshape(-1, nc)[:] = _prolongator(dims, n, block, nc, P).restrict(_np(v))

    def coarsen(ctx, dims, n, block, nc, X, F, B, P, Xc, Fc, Bc):
        D = omg.coarsen(_stencil(dims, n, X, F, B), _prolongator(dims, n, block, nc, P))
        _np(Xc).reshape(D.X.shape)[:] = D.X
        _np(Fc).reshape(D.F.shape)[:] = D.F
        _np(Bc).reshape(D.B.shape)[:] = D.B

    def dots(ctx, k, Xv, y):
        n = y.numel()
        return np.array([np.vdot(_np(Xv).reshape(-1)[j * n:(j + 1) * n], _np(y).reshape(-1)) for j in range(k)])

    def axpys(ctx, coef, Xv, y):
        coef = np.asarray(coef, dtype=np.complex128).reshape(-1)
        n = y.numel()
        yv = _np(y).reshape(-1)
        for j, c in enumerate(coef):
            yv += c * _np(Xv).reshape(-1)[j * n:(j + 1) * n]

    def axpby(ctx, a, x, b, y):
        yv = _np(y).reshape(-1)
        yv[:] = a * _np(x).reshape(-1).copy() + b * yv

    for name, f in dict(lqcd_mg_apply=apply, lqcd_mg_orthonormalize=orthonormalize, lqcd_mg_prolong=prolong,
                        lqcd_mg_restrict=restrict, lqcd_mg_coarsen=coarsen, lqcd_mg_dots=dots,
                        lqcd_mg_axpys=axpys, lqcd_mg_axpby=axpby).items():
        monkeypatch.setattr(m, name, f)
    monkeypatch.setattr(m, "_torch", lambda: _Shim)
    return m


def _starts(nv, V, n, seed):
    return gen.gaussian(2 * nv * V * n, seed).view(np.complex128).reshape(nv, V, n)


def test_gcr_and_mr_on_block_diagonal_operators(gmg):
    dims, V = (2, 2, 2, 2), 16
    rng = np.random.default_rng(3)
    X = rng.standard_normal((V, 4, 4)) + 1j * rng.standard_normal((V, 4, 4)) + 6 * np.eye(4)
    Z = np.zeros((4, V, 4, 4), dtype=np.complex128)
    b = rng.standard_normal((V, 4)) + 1j * rng.standard_normal((V, 4))
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex128))
    op = gmg.Stencil(None, dims, 4, T(X), T(Z), T(Z))
    x, it, rel = gmg.fgcr(op, T(b), 1e-13, 200, nkrylov=5)  # several restarts
    assert rel <= 1e-13 and it > 5
    assert np.abs(x.numpy() - np.linalg.solve(X, b[..., None])[..., 0]).max() < 1e-12
    scal = gmg.Stencil(None, dims, 4, T(np.broadcast_to((2.5 - 1j) * np.eye(4), (V, 4, 4))), T(Z), T(Z))
    assert np.abs(gmg.mr(scal, T(b), 1).numpy() - b / (2.5 - 1j)).max() < 1e-15


def test_host_driver_follows_the_oracle_solver(gmg):
    """Three levels on 8x8x4x8 near the critical kappa: the host code's set-up
    gives the oracle's coarse operators, and its solve the oracle's step count
    and a true residual <= 1e-10 recomputed by the C oracle."""
    dims, kappa = (8, 8, 4, 8), 0.1285
    V = int(np.prod(dims))
    U = gen.gauge_field(dims, 0.3, 21)
    ref = omg.wilson_clover_stencil(dims, U, kappa, 1.0, 1)
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex128))
    st = gmg.Stencil(None, dims, 12, T(ref.X), T(ref.F), T(ref.B))
    blocks = [(2, 2, 2, 2), (2, 2, 2, 2)]
    starts = [_starts(8, V, 12, 23), _starts(8, V // 16, 16, 24)]
    mg = gmg.Multigrid(st, blocks, starts, setup_iters=30)
    om = omg.Multigrid(ref, blocks, starts, setup_iters=30)
    for got, want in zip(mg.ops[1:], om.ops[1:]):
        assert got.dims == want.dims and got.n == want.n
        assert np.abs(got.X.numpy() - want.X).max() <= 1e-9 * np.abs(want.X).max()
    b = gen.gaussian_spinor(dims, 22).reshape(V, 12)
    x, it, rel = mg.solve(T(b), 1e-10)
    _, it_ref, _ = om.solve(b, 1e-10)
    assert abs(it - it_ref) <= 1 and rel <= 1e-10
    A = oracle.clover(dims, U, kappa, 1.0)
    canon = (dims[3], dims[2], dims[1], dims[0], 4, 3)
    assert oracle.true_residual(dims, U, A, kappa, x.numpy().reshape(canon), b.reshape(canon)) <= 1e-10
