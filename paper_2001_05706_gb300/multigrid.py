"""Adaptive aggregation multigrid for the Wilson-clover operator on the GPU.

The paper's clover inverter at scale is QUDA's 3-level multigrid (Sec. 4:
aggregation blocks (4,4,4,4) and then (2,2,2,2) on a 96^3 x 192 lattice;
Table 1: all parts a clover multigrid needs).  It gives no steps; this
module runs the standard adaptive aggregation method:

  levels     every level is a nearest-neighbour stencil (X, F_mu, B_mu) with
             n complex components per site, the first n/2 of chirality +1;
             the fine level is M = A - kappa D_W (lqcd_mg_fine_stencil);
  set-up     near-null vectors: for each random start v0 (an input), v =
             v0 - e with e from `setup_iters` GCR steps on D e = D v0; the
             prolongator orthonormalises them per block and chirality
             (lqcd_mg_orthonormalize) and the coarse level is P^H D P
             (lqcd_mg_coarsen);
  cycle      K_l r: `pre` MR steps, the restricted residual solved on level
             l + 1 by flexible GCR to a relative `coarse_tol` preconditioned
             by K_{l+1} (the coarsest level: plain GCR), the correction
             prolonged, `post` MR steps;
  solver     flexible GCR(nkrylov) on the fine level preconditioned by K_0,
             the residual recomputed as b - D x at each restart.

Every arithmetic step is a kernel of liblqcd.so (lqcd_mg_*): stencil
applications, restriction, prolongation, orthonormalisation, the Galerkin
product, inner products (fixed-order sums) and vector updates.  This module
owns the device arrays (torch tensors, used for memory only) and the Krylov
and cycle logic on the host.  Gram-Schmidt inside GCR is classical, applied
twice.  Fields are (V, n) complex128 CUDA tensors in lexicographic site order
(x fastest); a canonical spinor (L3, L2, L1, L0, 4, 3) is the same memory
as (V, 12).
"""
from __future__ import annotations

import numpy as np

from . import (lqcd_mg_apply, lqcd_mg_axpby, lqcd_mg_axpys, lqcd_mg_coarsen, lqcd_mg_dots,
               lqcd_mg_fine_stencil, lqcd_mg_orthonormalize, lqcd_mg_prolong, lqcd_mg_restrict)


def _torch():
    import torch
    return torch


class Stencil:
    """One level: D v(x) = X v(x) + sum_mu F_mu v(x + mu) + B_mu v(x - mu) on
    dims with n components; X (V, n, n), F and B (4, V, n, n) on the GPU."""

    def __init__(self, ctx, dims, n, X, F, B):
        self.ctx, self.dims, self.n = ctx, tuple(int(d) for d in dims), int(n)
        self.V = int(np.prod(self.dims))
        self.X, self.F, self.B = X, F, B

    def new(self):
        return _torch().zeros((self.V, self.n), dtype=_torch().complex128, device="cuda")

    def apply(self, v, out=None):
        out = self.new() if out is None else out
        lqcd_mg_apply(self.ctx, self.dims, self.n, self.X, self.F, self.B, v, out)
        return out


def fine_stencil(lattice):
    """M = A - kappa D_W of a Lattice with gauge field and clover term set."""
    torch = _torch()
    V = lattice.V
    X = torch.empty((V, 12, 12), dtype=torch.complex128, device="cuda")
    F = torch.empty((4, V, 12, 12), dtype=torch.complex128, device="cuda")
    B = torch.empty((4, V, 12, 12), dtype=torch.complex128, device="cuda")
    lqcd_mg_fine_stencil(lattice.ctx, V, X, F, B)
    return Stencil(lattice.ctx, lattice.dims, 12, X, F, B)


# ---- vector operations (each one kernel) ------------------------------------

def dot(ctx, x, y):
    return complex(lqcd_mg_dots(ctx, 1, x, y)[0])


def norm(ctx, x):
    return float(np.sqrt(max(dot(ctx, x, x).real, 0.0)))


def axpby(ctx, a, x, b, y):
    lqcd_mg_axpby(ctx, a, x, b, y)


def copy(ctx, x, y):
    lqcd_mg_axpby(ctx, 1.0, x, 0.0, y)


def mr(op, b, iters):
    """`iters` minimal-residual steps on op x = b from x = 0 (alpha = <D r, r> / <D r, D r>)."""
    x = op.new()
    r = op.new()
    copy(op.ctx, b, r)
    Ar = op.new()
    for _ in range(iters):
        op.apply(r, Ar)
        den = dot(op.ctx, Ar, Ar).real
        if den == 0:
            break
        a = dot(op.ctx, Ar, r) / den
        axpby(op.ctx, a, r, 1.0, x)
        axpby(op.ctx, -a, Ar, 1.0, r)
    return x


def fgcr(op, b, tol, maxiter, precond=None, nkrylov=16):
    """Flexible GCR(nkrylov) on op x = b from x = 0; returns (x, steps,
    ||b - D x|| / ||b||) with the residual recomputed at each restart."""
    torch = _torch()
    ctx = op.ctx
    x = op.new()
    bn = norm(ctx, b)
    if bn == 0:
        return x, 0, 0.0
    r = op.new()
    copy(ctx, b, r)
    Z = torch.zeros((nkrylov, op.V, op.n), dtype=torch.complex128, device="cuda")
    W = torch.zeros_like(Z)
    t = op.new()
    it = 0
    while True:
        k = 0
        while k < nkrylov:
            if precond is not None:
                copy(ctx, precond(r), Z[k])
            else:
                copy(ctx, r, Z[k])
            op.apply(Z[k], W[k])
            for _ in range(2):  # classical Gram-Schmidt, twice
                if k:
                    c = lqcd_mg_dots(ctx, k, W, W[k])
                    lqcd_mg_axpys(ctx, -c, W, W[k])
                    lqcd_mg_axpys(ctx, -c, Z, Z[k])
            nw = norm(ctx, W[k])
            if nw == 0:
                break
            axpby(ctx, 1.0 / nw, W[k], 0.0, W[k])
            axpby(ctx, 1.0 / nw, Z[k], 0.0, Z[k])
            alpha = dot(ctx, W[k], r)
            axpby(ctx, alpha, Z[k], 1.0, x)
            axpby(ctx, -alpha, W[k], 1.0, r)
            k += 1
            it += 1
            if norm(ctx, r) <= tol * bn or it >= maxiter:
                break
        op.apply(x, t)
        copy(ctx, b, r)
        axpby(ctx, -1.0, t, 1.0, r)
        rel = norm(ctx, r) / bn
        if rel <= tol or it >= maxiter or k == 0:
            return x, it, rel


def near_null_vectors(op, starts, iters):
    """v_k = v0_k - e_k, e_k from `iters` GCR steps on D e = D v0_k;
    starts (nv, V, n) CUDA tensor; returns an (nv, V, n) tensor."""
    torch = _torch()
    out = torch.empty_like(starts)
    for k in range(starts.shape[0]):
        rhs = op.apply(starts[k])
        e, _, _ = fgcr(op, rhs, 0.0, iters, nkrylov=iters)
        copy(op.ctx, starts[k], out[k])
        axpby(op.ctx, -1.0, e, 1.0, out[k])
    return out


class Prolongator:
    def __init__(self, fine: Stencil, block, vecs):
        torch = _torch()
        self.ctx, self.fine_dims, self.n = fine.ctx, fine.dims, fine.n
        self.block = tuple(int(b) for b in block)
        if any(L % b for L, b in zip(fine.dims, self.block)):
            raise ValueError(f"blocks {self.block} do not tile {fine.dims}")
        self.coarse_dims = tuple(L // b for L, b in zip(fine.dims, self.block))
        self.nv = int(vecs.shape[0])
        self.nc = 2 * self.nv
        self.P = torch.empty((fine.V, fine.n, self.nc), dtype=torch.complex128, device="cuda")
        lqcd_mg_orthonormalize(self.ctx, fine.dims, fine.n, self.block, self.nv, vecs.contiguous(), self.P)

    def prolong(self, w, out=None):
        torch = _torch()
        if out is None:
            out = torch.empty((int(np.prod(self.fine_dims)), self.n), dtype=torch.complex128, device="cuda")
        lqcd_mg_prolong(self.ctx, self.fine_dims, self.n, self.block, self.nc, self.P, w, out)
        return out

    def restrict(self, v, out=None):
        torch = _torch()
        if out is None:
            out = torch.empty((int(np.prod(self.coarse_dims)), self.nc), dtype=torch.complex128, device="cuda")
        lqcd_mg_restrict(self.ctx, self.fine_dims, self.n, self.block, self.nc, self.P, v, out)
        return out


def coarsen(fine: Stencil, P: Prolongator) -> Stencil:
    torch = _torch()
    Vc, nc = int(np.prod(P.coarse_dims)), P.nc
    Xc = torch.empty((Vc, nc, nc), dtype=torch.complex128, device="cuda")
    Fc = torch.empty((4, Vc, nc, nc), dtype=torch.complex128, device="cuda")
    Bc = torch.empty_like(Fc)
    lqcd_mg_coarsen(fine.ctx, fine.dims, fine.n, P.block, nc, fine.X, fine.F, fine.B, P.P, Xc, Fc, Bc)
    return Stencil(fine.ctx, P.coarse_dims, nc, Xc, Fc, Bc)


class Multigrid:
    """Levels 0 (fine) .. len(blocks); starts[l] (nv_l, V_l, n_l) complex
    numpy arrays of random start vectors, uploaded once."""

    def __init__(self, fine: Stencil, blocks, starts, setup_iters=30, pre=0, post=4, coarse_tol=0.25,
                 coarse_maxiter=200):
        torch = _torch()
        self.ops = [fine]
        self.P = []
        for block, st in zip(blocks, starts):
            op = self.ops[-1]
            st = np.ascontiguousarray(np.asarray(st, dtype=np.complex128).reshape(-1, op.V, op.n))
            vecs = near_null_vectors(op, torch.from_numpy(st).to("cuda"), setup_iters)
            P = Prolongator(op, block, vecs)
            self.P.append(P)
            self.ops.append(coarsen(op, P))
        self.pre, self.post = pre, post
        self.coarse_tol, self.coarse_maxiter = coarse_tol, coarse_maxiter

    def _coarse_solve(self, l, rc):
        op = self.ops[l]
        if l == len(self.ops) - 1:
            return fgcr(op, rc, self.coarse_tol, self.coarse_maxiter)[0]
        return fgcr(op, rc, self.coarse_tol, self.coarse_maxiter, precond=lambda v: self.cycle(l, v))[0]

    def cycle(self, l, r):
        op, P = self.ops[l], self.P[l]
        ctx = op.ctx
        if self.pre:
            x = mr(op, r, self.pre)
            t = op.apply(x)
            axpby(ctx, 1.0, r, -1.0, t)  # t = r - D x
            rc = P.restrict(t)
        else:
            x = op.new()
            rc = P.restrict(r)
        axpby(ctx, 1.0, P.prolong(self._coarse_solve(l + 1, rc)), 1.0, x)
        if self.post:
            t = op.apply(x)
            axpby(ctx, 1.0, r, -1.0, t)
            axpby(ctx, 1.0, mr(op, t, self.post), 1.0, x)
        return x

    def solve(self, b, tol=1e-10, maxiter=500, nkrylov=16):
        """Flexible GCR preconditioned by K_0; returns (x, outer steps, relative residual)."""
        return fgcr(self.ops[0], b, tol, maxiter, precond=lambda v: self.cycle(0, v), nkrylov=nkrylov)
