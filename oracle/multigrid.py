"""Adaptive aggregation multigrid for the Wilson-clover operator: the FP64 oracle.

TEST INFRASTRUCTURE ONLY, like the rest of this package: the tests may import
it; the library never does.

The paper runs QUDA's multigrid inverter for the clover fermion: three
levels, aggregation blocks (4,4,4,4) and then (2,2,2,2), on a 96^3 x 192
lattice (Sec. 4; Table 1's caption: every part a clover multigrid needs was
ported).  It prints none of the method's steps and cites the GPU multigrid
of Clark et al. for them, so this module writes out the standard adaptive
aggregation multigrid of the lattice literature (Babich et al., PRL 105
(2010) 201602; Clark et al., SC16) from its definitions:

  operator     a nearest-neighbour stencil on a periodic 4-d lattice,
               D v(x) = X(x) v(x) + sum_mu F_mu(x) v(x+mu) + B_mu(x) v(x-mu),
               n components per site, each with a chirality chi = +-1 (the
               eigenvalue of gamma5, diagonal in the DeGrand-Rossi basis).
               The fine level is M = A - kappa D_W itself (full lattice).
  near-null    for each random start v0 (an input), v = v0 - e with e from
  vectors      a fixed number of GCR steps on D e = D v0: GCR minimises
               ||D v|| over v0 + Krylov space, which leaves v rich in the
               low modes of D.
  prolongator  the lattice is cut into blocks of b_mu sites; on each block
               and each chirality the near-null vectors' restrictions are
               orthonormalised by Gram-Schmidt (QR with a real positive
               diagonal), giving 2 nv coarse components per block, ordered
               [chi = +1: nv, chi = -1: nv].  P is block-orthonormal
               (P^H P = 1) and commutes with gamma5.
  coarse op    D_c = P^H D P (Galerkin), again a nearest-neighbour stencil:
               hops inside a block go to X_c, hops across a block face to
               F_c / B_c of that direction.
  cycle        K_l(r): nu_pre MR steps, restriction of the residual, the
               coarse system solved by flexible GCR to a relative tolerance
               preconditioned by K_{l+1} (the coarsest level: plain GCR, or
               an exact dense solve), prolongation of the correction,
               nu_post MR steps.
  solver       flexible GCR on the fine level preconditioned by K_0.

Every step is the plain definition, in numpy; no blocking or reordering
beyond it.  The choices the paper leaves open (smoother, setup iterations,
tolerances, the K-cycle) are parameters with the defaults stated above.
"""
from __future__ import annotations

import numpy as np

from . import clover as _clover
from . import gamma as _gamma

_c = np.complex128


def _coords(dims):
    """Coordinates (V, 4) of the lexicographic sites, x fastest."""
    L = [int(d) for d in dims]
    s = np.arange(int(np.prod(L)))
    return np.stack([s % L[0], (s // L[0]) % L[1], (s // (L[0] * L[1])) % L[2], s // (L[0] * L[1] * L[2])], axis=1)


def _index(dims, co):
    L = [int(d) for d in dims]
    return co[:, 0] + L[0] * (co[:, 1] + L[1] * (co[:, 2] + L[2] * co[:, 3]))


def _neighbours(dims):
    """fwd[mu][s], bwd[mu][s]: the sites s + mu and s - mu (periodic)."""
    co = _coords(dims)
    fwd, bwd = [], []
    for mu in range(4):
        for step, out in ((1, fwd), (-1, bwd)):
            c = co.copy()
            c[:, mu] = (c[:, mu] + step) % int(dims[mu])
            out.append(_index(dims, c))
    return np.array(fwd), np.array(bwd)


class Stencil:
    """D v(x) = X(x) v(x) + sum_mu F_mu(x) v(x + mu) + B_mu(x) v(x - mu) on the
    periodic lattice dims = (L0, L1, L2, L3); fields are (V, n) arrays in the
    lexicographic site order (x fastest).  Boundary phases are part of the
    matrices.  X (V, n, n), F and B (4, V, n, n), chi (n,) of +-1."""

    def __init__(self, dims, X, F, B, chi):
        self.dims = tuple(int(d) for d in dims)
        self.V = int(np.prod(self.dims))
        self.X = np.asarray(X, dtype=_c)
        self.F = np.asarray(F, dtype=_c)
        self.B = np.asarray(B, dtype=_c)
        self.n = self.X.shape[1]
        self.chi = np.asarray(chi, dtype=np.int64)
        if self.X.shape != (self.V, self.n, self.n) or self.F.shape != (4, self.V, self.n, self.n) \
                or self.B.shape != self.F.shape or self.chi.shape != (self.n,):
            raise ValueError("stencil arrays do not match the lattice")
        self.fwd, self.bwd = _neighbours(self.dims)

    def apply(self, v):
        v = np.asarray(v, dtype=_c).reshape(self.V, self.n)
        out = np.einsum("sij,sj->si", self.X, v)
        for mu in range(4):
            out += np.einsum("sij,sj->si", self.F[mu], v[self.fwd[mu]])
            out += np.einsum("sij,sj->si", self.B[mu], v[self.bwd[mu]])
        return out

    def apply_adjoint(self, v):
        """D^H v: D^H(x, y) = D(y, x)^H, so the forward matrix of x - mu and the
        backward matrix of x + mu act on v(x - mu) and v(x + mu)."""
        v = np.asarray(v, dtype=_c).reshape(self.V, self.n)
        out = np.einsum("sji,sj->si", self.X.conj(), v)
        for mu in range(4):
            b, f = self.bwd[mu], self.fwd[mu]
            out += np.einsum("sji,sj->si", self.F[mu][b].conj(), v[b])
            out += np.einsum("sji,sj->si", self.B[mu][f].conj(), v[f])
        return out

    def dense(self):
        """The (V n, V n) matrix, assembled from the stencil entries."""
        n, V = self.n, self.V
        D = np.zeros((V * n, V * n), dtype=_c)
        for s in range(V):
            D[s * n:(s + 1) * n, s * n:(s + 1) * n] += self.X[s]
            for mu in range(4):
                f, b = self.fwd[mu][s], self.bwd[mu][s]
                D[s * n:(s + 1) * n, f * n:(f + 1) * n] += self.F[mu][s]
                D[s * n:(s + 1) * n, b * n:(b + 1) * n] += self.B[mu][s]
        return D


def wilson_clover_stencil(dims, U, kappa, csw, tbc=1):
    """M = A - kappa D_W as a stencil (12 components, index 3 spin + colour):
    F_mu(x) = -kappa (1 - gamma_mu) U_mu(x), B_mu(x) = -kappa (1 + gamma_mu)
    U_mu(x - mu)^H, with -1 on the hops across the t boundary when tbc is
    set; X(x) = A(x), the clover term (the identity when csw = 0)."""
    dims = tuple(int(d) for d in dims)
    V = int(np.prod(dims))
    U = np.asarray(U, dtype=_c).reshape(V, 4, 3, 3)
    A = _clover(dims, U, kappa, csw) if csw else None
    X = np.broadcast_to(np.eye(12, dtype=_c), (V, 12, 12)).copy() if A is None else np.asarray(A, _c).reshape(V, 12, 12)
    fwd, bwd = _neighbours(dims)
    t = _coords(dims)[:, 3]
    F = np.empty((4, V, 12, 12), dtype=_c)
    B = np.empty((4, V, 12, 12), dtype=_c)
    one = np.eye(4, dtype=_c)
    for mu in range(4):
        sf = np.ones(V)
        sb = np.ones(V)
        if mu == 3 and tbc:
            sf[t == dims[3] - 1] = -1.0
            sb[t == 0] = -1.0
        Uf = U[:, mu]
        Ub = U[bwd[mu], mu].conj().transpose(0, 2, 1)
        F[mu] = -kappa * sf[:, None, None] * np.einsum("ab,sij->saibj", one - _gamma(mu), Uf).reshape(V, 12, 12)
        B[mu] = -kappa * sb[:, None, None] * np.einsum("ab,sij->saibj", one + _gamma(mu), Ub).reshape(V, 12, 12)
    chi = np.array([1] * 6 + [-1] * 6)  # gamma5 = diag(1, 1, -1, -1) in spin
    return Stencil(dims, X, F, B, chi)


# ---------------------------------------------------------------------------
# Krylov pieces
# ---------------------------------------------------------------------------

def _dot(a, b):
    return np.vdot(a.reshape(-1), b.reshape(-1))


def _nrm(a):
    return float(np.linalg.norm(a.reshape(-1)))


def mr(op, b, iters):
    """`iters` minimal-residual steps on op x = b from x = 0: each step adds
    alpha r with alpha = <D r, r> / <D r, D r>, the minimiser of ||r - alpha D r||."""
    x = np.zeros_like(b, dtype=_c)
    r = np.array(b, dtype=_c)
    for _ in range(iters):
        Ar = op.apply(r)
        den = _dot(Ar, Ar).real
        if den == 0:
            break
        a = _dot(Ar, r) / den
        x += a * r
        r -= a * Ar
    return x


def fgcr(op, b, tol, maxiter, precond=None, nkrylov=16):
    """Flexible GCR(nkrylov) on op x = b from x = 0: each step z = K(r) (or r),
    w = D z made orthonormal to the earlier w's (the z's follow the same
    combination), then x += <w, r> z, r -= <w, r> w.  At each restart and at
    the end r is recomputed as b - D x.  Returns (x, steps, ||b - D x|| / ||b||)."""
    b = np.asarray(b, dtype=_c)
    x = np.zeros_like(b)
    bn = _nrm(b)
    if bn == 0:
        return x, 0, 0.0
    r = b.copy()
    it = 0
    while True:
        Z, W = [], []
        for _ in range(nkrylov):
            z = precond(r) if precond is not None else r.copy()
            w = op.apply(z)
            for zi, wi in zip(Z, W):
                beta = _dot(wi, w)
                w = w - beta * wi
                z = z - beta * zi
            nw = _nrm(w)
            if nw == 0:
                break
            w, z = w / nw, z / nw
            alpha = _dot(w, r)
            x += alpha * z
            r -= alpha * w
            Z.append(z)
            W.append(w)
            it += 1
            if _nrm(r) <= tol * bn or it >= maxiter:
                break
        r = b - op.apply(x)
        rel = _nrm(r) / bn
        if rel <= tol or it >= maxiter or not W:
            return x, it, rel


def near_null_vectors(op, starts, iters):
    """v_k = v0_k - e_k, e_k from `iters` GCR steps on D e = D v0_k (e = 0 at
    the start): the component of the random start v0_k that GCR cannot
    remove, concentrated on the low modes of D.  starts (nv, V, n)."""
    out = []
    for v0 in np.asarray(starts, dtype=_c):
        e, _, _ = fgcr(op, op.apply(v0), 0.0, iters, nkrylov=iters)
        out.append(v0 - e)
    return np.array(out)


# ---------------------------------------------------------------------------
# aggregation
# ---------------------------------------------------------------------------

class Prolongator:
    """P: coarse fields (Vc, 2 nv) -> fine fields (V, n),
    (P w)(s) = Ps[s] w(c[s]), c[s] the block of fine site s.  On each block
    and chirality the columns are the Gram-Schmidt orthonormalisation (QR,
    real positive diagonal) of the near-null vectors restricted there, in
    their given order."""

    def __init__(self, fine: Stencil, block, vecs):
        self.block = tuple(int(b) for b in block)
        if any(L % b for L, b in zip(fine.dims, self.block)):
            raise ValueError(f"blocks {self.block} do not tile {fine.dims}")
        self.fine_dims = fine.dims
        self.coarse_dims = tuple(L // b for L, b in zip(fine.dims, self.block))
        vecs = np.asarray(vecs, dtype=_c).reshape(-1, fine.V, fine.n)
        nv = vecs.shape[0]
        co = _coords(fine.dims)
        self.fine_coords = co
        self.c = _index(self.coarse_dims, co // np.array(self.block))
        self.Vc = int(np.prod(self.coarse_dims))
        self.nv = nv
        self.nc = 2 * nv
        self.chi = np.array([1] * nv + [-1] * nv)
        self.Ps = np.zeros((fine.V, fine.n, self.nc), dtype=_c)
        for xc in range(self.Vc):
            sites = np.nonzero(self.c == xc)[0]
            for k, sign in enumerate((1, -1)):
                comps = np.nonzero(fine.chi == sign)[0]
                Mb = vecs[:, sites][:, :, comps].reshape(nv, -1).T  # (|block| * comps, nv)
                if Mb.shape[0] < nv:
                    raise ValueError(f"{nv} vectors exceed the {Mb.shape[0]} components of a block chirality")
                Q, R = np.linalg.qr(Mb)
                d = np.diag(R)
                if np.any(np.abs(d) <= 1e-12 * np.abs(d).max()):
                    raise ValueError("near-null vectors linearly dependent on a block")
                Q = Q * (d / np.abs(d))[None, :]
                self.Ps[sites[:, None], comps[None, :], k * nv:(k + 1) * nv] = Q.reshape(len(sites), len(comps), nv)

    def prolong(self, w):
        w = np.asarray(w, dtype=_c).reshape(self.Vc, self.nc)
        return np.einsum("sij,sj->si", self.Ps, w[self.c])

    def restrict(self, v):
        """P^H v: the sum over each block of Ps[s]^H v(s)."""
        v = np.asarray(v, dtype=_c).reshape(len(self.c), -1)
        out = np.zeros((self.Vc, self.nc), dtype=_c)
        np.add.at(out, self.c, np.einsum("sji,sj->si", self.Ps.conj(), v))
        return out


def coarsen(fine: Stencil, P: Prolongator) -> Stencil:
    """D_c = P^H D P as a stencil on the coarse lattice.  Each fine term
    Ps[s]^H T Ps[s'] (T = X(s), F_mu(s) with s' = s + mu, B_mu(s) with
    s' = s - mu) lands on the coarse site of s: in X_c when s' lies in the
    same block, in F_c[mu] / B_c[mu] when the hop crosses the block's face."""
    PsH = P.Ps.conj().transpose(0, 2, 1)
    Vc, nc = P.Vc, P.nc
    Xc = np.zeros((Vc, nc, nc), dtype=_c)
    Fc = np.zeros((4, Vc, nc, nc), dtype=_c)
    Bc = np.zeros((4, Vc, nc, nc), dtype=_c)
    np.add.at(Xc, P.c, PsH @ fine.X @ P.Ps)
    co = P.fine_coords
    for mu in range(4):
        b = P.block[mu]
        term = PsH @ fine.F[mu] @ P.Ps[fine.fwd[mu]]
        cross = co[:, mu] % b == b - 1
        np.add.at(Xc, P.c[~cross], term[~cross])
        np.add.at(Fc[mu], P.c[cross], term[cross])
        term = PsH @ fine.B[mu] @ P.Ps[fine.bwd[mu]]
        cross = co[:, mu] % b == 0
        np.add.at(Xc, P.c[~cross], term[~cross])
        np.add.at(Bc[mu], P.c[cross], term[cross])
    return Stencil(P.coarse_dims, Xc, Fc, Bc, P.chi)


# ---------------------------------------------------------------------------
# the hierarchy and the solver
# ---------------------------------------------------------------------------

class Multigrid:
    """Levels 0 (fine) .. len(blocks): op[l + 1] = P_l^H op[l] P_l, P_l built
    from near-null vectors of op[l] (setup_iters GCR steps from starts[l],
    each (nv_l, V_l, n_l)).  cycle(l, r) is the K-cycle of the module
    docstring."""

    def __init__(self, fine: Stencil, blocks, starts, setup_iters=30, pre=0, post=4, coarse_tol=0.25,
                 coarse_maxiter=200, coarsest_exact=False):
        self.ops = [fine]
        self.P = []
        for block, st in zip(blocks, starts):
            op = self.ops[-1]
            vecs = near_null_vectors(op, st, setup_iters)
            P = Prolongator(op, block, vecs)
            self.P.append(P)
            self.ops.append(coarsen(op, P))
        self.pre, self.post = pre, post
        self.coarse_tol, self.coarse_maxiter = coarse_tol, coarse_maxiter
        self.coarsest_exact = coarsest_exact
        self._dense_inv = None

    def _coarse_solve(self, l, rc):
        op = self.ops[l]
        if l == len(self.ops) - 1:
            if self.coarsest_exact:
                if self._dense_inv is None:
                    self._dense_inv = np.linalg.inv(op.dense())
                return (self._dense_inv @ rc.reshape(-1)).reshape(rc.shape)
            return fgcr(op, rc, self.coarse_tol, self.coarse_maxiter)[0]
        return fgcr(op, rc, self.coarse_tol, self.coarse_maxiter, precond=lambda v: self.cycle(l, v))[0]

    def cycle(self, l, r):
        """K_l r: pre-smoothing, coarse-grid correction, post-smoothing."""
        op, P = self.ops[l], self.P[l]
        r = np.asarray(r, dtype=_c).reshape(op.V, op.n)
        x = mr(op, r, self.pre) if self.pre else np.zeros_like(r)
        rc = P.restrict(r - op.apply(x) if self.pre else r)
        x = x + P.prolong(self._coarse_solve(l + 1, rc))
        if self.post:
            x = x + mr(op, r - op.apply(x), self.post)
        return x

    def solve(self, b, tol=1e-10, maxiter=500, nkrylov=16):
        """Flexible GCR on the fine level preconditioned by K_0; returns
        (x, outer steps, ||b - D x|| / ||b||)."""
        return fgcr(self.ops[0], b, tol, maxiter, precond=lambda v: self.cycle(0, v), nkrylov=nkrylov)
