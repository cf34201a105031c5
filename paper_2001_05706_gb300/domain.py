"""Domain decomposition of the lattice along t: the multi-GPU form of the
Schur complement and of CG on its normal equations.

The paper's large runs (Sec. 4: the clover solve on a 96^3 x 192 lattice over
324 GPUs, the overlap eigensystem over 4 GPUs) split the lattice between
GPUs.  Here the global lattice (L0, L1, L2, L3) is cut into P domains of
Lt = L3 / P time slices each (Lt even), and each domain is an ordinary
library context on its slices plus HALO = 2 ghost slices on either side,
extended slice e holding global slice (t_off - HALO + e) mod L3.  Inside a
domain the lattice is periodic in t; the sign of the global antiperiodic
boundary is carried by the ghost data that crosses it (a factor -1 applied
on arrival, exact).

One application of Mhat = A_oo - kappa^2 D_oe A_ee^-1 D_eo on the interior
slices [HALO, HALO + Lt):
  1. exchange: each domain sends the odd-parity slices [HALO, 2 HALO) of x_o
     to the domain below and [Lt, Lt + HALO) to the domain above, and
     receives its ghost slices [0, HALO) and [Lt + HALO, Lt + 2 HALO);
  2. K2a, y_e = A_ee^-1 D_eo x_o, on slices [1, Lt + 3): the interior and the
     first ghost layer, whose values the second hop needs -- computed from the
     depth-2 ghosts of x_o instead of being exchanged a second time;
  3. K2b, z_o = A_oo x_o - kappa^2 D_oe y_e, on the interior, with the
     per-right-hand-side ||z_o||^2 of the interior fused.
One exchange of 2 slices per side per application (24 reals per site),
against the spin-projected single-slice faces (12 reals) of a two-exchange
scheme: fewer synchronisation points, twice the bytes.

With overlap=True the interior work runs while the halos are in flight:
after the sends are posted, K2a runs on slices [HALO + 1, Lt + HALO - 1)
(their t-neighbours of x_o are all interior) and K2b on
[HALO + 2, Lt + HALO - 2) (their t-neighbours of y_e are those slices);
once the ghosts have arrived K2a completes its two edge ranges and K2b the
interior's edges.  Every output slice is still computed once, by the same
kernel from the same values, so z is bit for bit the sequential result; the
norms are the sums of the pieces' fixed-order sums.

CG on the normal equations (CGLS) runs across domains with the global sums
(||q||^2; then ||r||^2 and ||s||^2 together) reduced by the exchange's
allreduce: two reductions and two halo exchanges per iteration.

Transport: `LocalExchange` routes halos between domains held by one process
(the one-GPU emulation of the tests), `DistExchange` one domain per rank
through torch.distributed (NCCL between GPUs, gloo on CPU).  The domain
objects (`GpuDomain` here; the tests add a CPU one) do the arithmetic: on the
GPU every step is a kernel of the library.
"""
from __future__ import annotations

import numpy as np

HALO = 2


class Partition:
    """Index logic of one domain of a t-split of the global lattice."""

    def __init__(self, global_dims, ndomains, rank, t_antiperiodic=1):
        L0, L1, L2, L3 = (int(v) for v in global_dims)
        if ndomains < 1 or L3 % ndomains:
            raise ValueError(f"{L3} time slices do not split into {ndomains} domains")
        lt = L3 // ndomains
        if lt % 2 or lt < 2:
            raise ValueError(f"each domain needs an even number >= 2 of time slices, not {lt}")
        if not 0 <= rank < ndomains:
            raise ValueError(f"rank {rank} outside 0..{ndomains - 1}")
        self.global_dims = (L0, L1, L2, L3)
        self.ndomains, self.rank, self.lt = ndomains, rank, lt
        self.t_off = rank * lt
        self.tbc = int(t_antiperiodic)
        self.local_dims = (L0, L1, L2, lt + 2 * HALO)
        self.interior = (HALO, HALO + lt)      # slices this domain owns
        self.k2a_slices = (1, lt + 2 * HALO - 1)  # y_e: interior plus the first ghost layer
        self.send_lo = (HALO, 2 * HALO)        # to the domain below (its upper ghosts)
        self.send_hi = (lt, lt + HALO)         # to the domain above (its lower ghosts)
        self.ghost_lo = (0, HALO)
        self.ghost_hi = (lt + HALO, lt + 2 * HALO)
        # the overlapped schedule: what needs no ghost data, and the rest
        a0, a1 = self.k2a_slices
        self.k2a_inner = (HALO + 1, max(HALO + 1, lt + HALO - 1))
        self.k2a_edges = _ranges((a0, self.k2a_inner[0]), (self.k2a_inner[1], a1))
        b0, b1 = self.interior
        self.k2b_inner = (HALO + 2, max(HALO + 2, lt + HALO - 2))
        self.k2b_edges = _ranges((b0, min(self.k2b_inner[0], b1)), (max(self.k2b_inner[1], b0 + 2), b1))
        # ghost data arriving across the global time boundary carries its sign
        self.factor_lo = -1.0 if (self.tbc and rank == 0) else 1.0
        self.factor_hi = -1.0 if (self.tbc and rank == ndomains - 1) else 1.0
        # global time slice held by each extended slice
        self.slab_t = [(self.t_off - HALO + e) % L3 for e in range(lt + 2 * HALO)]

    def slab(self, field_global):
        """The extended slab of a global canonical array (time is axis 0 of
        links [t][z][y][x][mu][3][3] and of spinors [t][z][y][x][4][3])."""
        return np.ascontiguousarray(np.asarray(field_global)[self.slab_t])

    def interior_of(self, field_local):
        a, b = self.interior
        return field_local[a:b]


def _ranges(*rs):
    """The non-empty ranges among rs, adjacent ones merged."""
    out = []
    for a, b in rs:
        if b <= a:
            continue
        if out and out[-1][1] == a:
            out[-1] = (out[-1][0], b)
        else:
            out.append((a, b))
    return out


class LocalExchange:
    """Halo routing and global sums between the domains held by one process
    (domain d's neighbours are d - 1 and d + 1, cyclically)."""

    def __init__(self, ndomains):
        self.n = ndomains

    def halo(self, sends):
        """sends[d] = (lo, hi) buffers of domain d; returns recv[d] = (for its
        lower ghosts: hi of d - 1, for its upper ghosts: lo of d + 1)."""
        if len(sends) != self.n:
            raise ValueError("one send pair per domain")
        return [(sends[(d - 1) % self.n][1], sends[(d + 1) % self.n][0]) for d in range(self.n)]

    def halo_start(self, sends):
        """Post the exchange; halo_finish returns what halo() does.  Within one
        process the routing is immediate (the send buffers are not written
        again before the next exchange)."""
        return self.halo(sends)

    def halo_finish(self, pending):
        return pending

    def allreduce(self, parts):
        """parts[d] = numpy array of domain d; the element-wise sum over domains."""
        return np.sum(np.stack([np.asarray(p, dtype=np.float64) for p in parts]), axis=0)


class DistExchange:
    """One domain per rank through torch.distributed (NCCL between GPUs, gloo
    on CPU).  Receive buffers are allocated like the send buffers.  With two
    ranks both neighbours are the same peer: the sends and receives are
    posted in an order that pairs each message with its buffer (first lo to
    the rank below / from the rank above, then hi)."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.rank = dist.get_rank(group)
        self.size = dist.get_world_size(group)

    def halo(self, sends):
        return self.halo_finish(self.halo_start(sends))

    def halo_start(self, sends):
        """Post the sends and receives and return without waiting.  With NCCL
        they run on the communicator's stream, ordered after the work already
        queued on torch's current stream (the domain's context stream must be
        that stream, the default); halo_finish makes the current stream wait
        for the receives."""
        import torch
        if len(sends) != 1:
            raise ValueError("one domain per rank")
        lo, hi = sends[0]
        if self.size == 1:
            return [], [(hi.clone(), lo.clone())]
        down = (self.rank - 1) % self.size
        up = (self.rank + 1) % self.size
        recv_hi = torch.empty_like(lo)  # the domain above's lo
        recv_lo = torch.empty_like(hi)  # the domain below's hi
        ops = [self.dist.P2POp(self.dist.isend, lo, down, self.group),
               self.dist.P2POp(self.dist.irecv, recv_hi, up, self.group),
               self.dist.P2POp(self.dist.isend, hi, up, self.group),
               self.dist.P2POp(self.dist.irecv, recv_lo, down, self.group)]
        return self.dist.batch_isend_irecv(ops), [(recv_lo, recv_hi)]

    def halo_finish(self, pending):
        reqs, recvs = pending
        for req in reqs:
            req.wait()
        return recvs

    def allreduce(self, parts):
        import torch
        if len(parts) != 1:
            raise ValueError("one domain per rank")
        backend = self.dist.get_backend(self.group)
        dev = torch.device("cuda", torch.cuda.current_device()) if backend == "nccl" else torch.device("cpu")
        t = torch.as_tensor(np.asarray(parts[0], dtype=np.float64), device=dev).clone()
        self.dist.all_reduce(t, group=self.group)
        return t.cpu().numpy()


class GpuDomain:
    """One domain on the GPU: a library context on the extended lattice,
    FP64 fields (ODD for the Krylov vectors, EVEN for the intermediate y_e),
    halos moved by the library's slice kernels.  Every arithmetic step is a
    kernel of liblqcd.so; this class only sequences the calls."""

    def __init__(self, part: Partition, stream=None, recon=18):
        from . import Lattice
        self.part = part
        self.recon = recon
        self.lat = Lattice(part.local_dims, 0, stream)  # periodic inside; the sign rides on the halos
        self.ctx = self.lat.ctx
        self.nrhs = None
        self._y = None
        self._buf = {}

    def close(self):
        self.lat.close()

    def load_gauge(self, U_global):
        self.lat.load_gauge(self.part.slab(U_global).view(np.float64))

    def clover(self, kappa, c_sw):
        self.lat.clover(kappa, c_sw)

    # ---- fields -----------------------------------------------------------
    def new_field(self, nrhs, subset=None):
        from . import LQCD_F64, LQCD_ODD, lqcd_field_create
        self.nrhs = nrhs
        return lqcd_field_create(self.ctx, LQCD_F64, LQCD_ODD if subset is None else subset, nrhs)

    def free(self, f):
        from . import lqcd_field_destroy
        lqcd_field_destroy(f)

    def import_global(self, f, canon_global):
        """The odd sites of this domain's interior from a global canonical
        array [rhs][t][z][y][x][4][3]; ghost slices zero."""
        from . import lqcd_field_import
        a = np.asarray(canon_global)
        slab = np.ascontiguousarray(a[:, self.part.slab_t])
        lo, hi = self.part.interior
        slab[:, :lo] = 0
        slab[:, hi:] = 0
        lqcd_field_import(self.ctx, f, slab)

    def export_interior(self, f, nrhs):
        """The interior slices of f as canonical [rhs][Lt][z][y][x][4][3]."""
        from . import lqcd_field_export
        L0, L1, L2, Le = self.part.local_dims
        out = np.zeros((nrhs, Le, L2, L1, L0, 4, 3), dtype=np.complex128)
        lqcd_field_export(self.ctx, f, out)
        lo, hi = self.part.interior
        return out[:, lo:hi]

    # ---- halos ------------------------------------------------------------
    def _halo_buffer(self, key, nrhs):
        import torch
        S = int(np.prod(self.part.local_dims[:3])) // 2  # sites of one parity per slice
        n = nrhs * 12 * HALO * S * 2  # 12 words of 16 bytes per FP64 site, as doubles
        if self._buf.get(key) is None or self._buf[key].numel() != n:
            self._buf[key] = torch.zeros(n, dtype=torch.float64, device="cuda")
        return self._buf[key]

    def pack(self, f, nrhs):
        from . import lqcd_field_slices
        lo, hi = self._halo_buffer("lo", nrhs), self._halo_buffer("hi", nrhs)
        lqcd_field_slices(self.ctx, f, 1, *self.part.send_lo, lo, 0)
        lqcd_field_slices(self.ctx, f, 1, *self.part.send_hi, hi, 0)
        return lo, hi

    def unpack(self, f, recv_lo, recv_hi):
        from . import lqcd_field_slices
        lqcd_field_slices(self.ctx, f, 1, *self.part.ghost_lo, recv_lo, 1, self.part.factor_lo)
        lqcd_field_slices(self.ctx, f, 1, *self.part.ghost_hi, recv_hi, 1, self.part.factor_hi)

    def clear_ghosts(self, f, nrhs):
        from . import lqcd_field_slices
        z = self._halo_buffer("zero", nrhs)
        z.zero_()
        lqcd_field_slices(self.ctx, f, 1, *self.part.ghost_lo, z, 1)
        lqcd_field_slices(self.ctx, f, 1, *self.part.ghost_hi, z, 1)

    # ---- operators and BLAS -------------------------------------------------
    def k2a(self, x, nrhs, t0, t1, dagger=False):
        """y_e = A_ee^-1 D_eo x_o (dagger: with g5 on x) on slices [t0, t1) of
        the domain's intermediate even field."""
        from . import LQCD_EVEN, LQCD_F64, lqcd_field_create, lqcd_k2a_slices
        if self._y is None or self._ynrhs != nrhs:
            if self._y is not None:
                self.free(self._y)
            self._y = lqcd_field_create(self.ctx, LQCD_F64, LQCD_EVEN, nrhs)
            self._ynrhs = nrhs
        lqcd_k2a_slices(self.ctx, self.recon, int(dagger), self._y, x, t0, t1)

    def k2b(self, out, x, nrhs, t0, t1, dagger=False):
        """out_o = A_oo x_o - kappa^2 D_oe y_e (dagger: g5 on the hop) on slices
        [t0, t1); returns the per-RHS ||out_o||^2 over them."""
        from . import lqcd_k2b_slices
        return lqcd_k2b_slices(self.ctx, self.recon, int(dagger), out, x, self._y, t0, t1, nrhs=nrhs)

    def axpby(self, y, a, b, x):
        from . import lqcd_field_axpby
        lqcd_field_axpby(self.ctx, y, a, b, x)

    def norm2s(self, f, nrhs):
        from . import lqcd_field_norm2s
        return lqcd_field_norm2s(self.ctx, f, nrhs)


# ---------------------------------------------------------------------------
# the distributed operator and solver (any domain objects with the methods above)
# ---------------------------------------------------------------------------

def _dd_apply(domains, exchange, outs, xs, nrhs, dagger, overlap):
    """outs[d] = Mhat xs[d] (or the adjoint) on each domain's interior, with one
    halo exchange; x's ghost slices are cleared again afterwards.  Returns each
    domain's per-RHS ||Mhat x||^2 over its interior (not yet reduced)."""
    sends = [d.pack(x, nrhs) for d, x in zip(domains, xs)]
    parts = [np.zeros(nrhs) for _ in domains]
    if overlap:
        pending = exchange.halo_start(sends)
        for i, (d, x, out) in enumerate(zip(domains, xs, outs)):
            if d.part.k2a_inner[1] > d.part.k2a_inner[0]:
                d.k2a(x, nrhs, *d.part.k2a_inner, dagger)
            if d.part.k2b_inner[1] > d.part.k2b_inner[0]:
                parts[i] = parts[i] + d.k2b(out, x, nrhs, *d.part.k2b_inner, dagger)
        recvs = exchange.halo_finish(pending)
        for i, (d, x, out, (rlo, rhi)) in enumerate(zip(domains, xs, outs, recvs)):
            d.unpack(x, rlo, rhi)
            for t0, t1 in d.part.k2a_edges:
                d.k2a(x, nrhs, t0, t1, dagger)
            for t0, t1 in d.part.k2b_edges:
                parts[i] = parts[i] + d.k2b(out, x, nrhs, t0, t1, dagger)
            d.clear_ghosts(x, nrhs)
        return parts
    recvs = exchange.halo(sends)
    for i, (d, x, out, (rlo, rhi)) in enumerate(zip(domains, xs, outs, recvs)):
        d.unpack(x, rlo, rhi)
        d.k2a(x, nrhs, *d.part.k2a_slices, dagger)
        parts[i] = d.k2b(out, x, nrhs, *d.part.interior, dagger)
        d.clear_ghosts(x, nrhs)
    return parts


def dd_mhat(domains, exchange, outs, xs, nrhs, dagger=False, overlap=False):
    """outs[d] = Mhat xs[d] (or the adjoint) on each domain's interior, with one
    halo exchange (overlapped with the interior work when overlap is set);
    returns the global per-RHS ||Mhat x||^2."""
    return exchange.allreduce(_dd_apply(domains, exchange, outs, xs, nrhs, dagger, overlap))


def dd_cgls(domains, exchange, xs, bs, nrhs, tol=1e-10, max_iter=10000, overlap=False):
    """CG on the normal equations of Mhat x = b across domains (x starts at 0;
    every right-hand side its own recursion, parked once converged).  Stops
    when the recomputed ||b - Mhat x|| <= tol ||b|| for every right-hand side.
    overlap: every operator application overlaps its halo exchange with the
    interior work.  Returns (iterations, relative residuals)."""
    D = list(zip(domains, xs, bs))
    one, zero = np.ones(nrhs), np.zeros(nrhs)
    mk = lambda: [d.new_field(nrhs) for d in domains]
    r, s, p, q = mk(), mk(), mk(), mk()
    try:
        for d, x, b in D:
            d.axpby(x, zero, zero, x)
        for d, rr_, (_, _, b) in zip(domains, r, D):
            d.axpby(rr_, one, zero, b)
        bn2 = exchange.allreduce([d.norm2s(b, nrhs) for d, _, b in D])
        gamma = dd_mhat(domains, exchange, s, r, nrhs, dagger=True, overlap=overlap)
        for d, pp, ss in zip(domains, p, s):
            d.axpby(pp, one, zero, ss)
        active = np.ones(nrhs, dtype=bool)
        target = (0.5 * tol) ** 2 * bn2  # iterate to half the tolerance (margin for the check)
        it = 0
        rel = np.ones(nrhs)
        while it < max_iter:
            it += 1
            qq = dd_mhat(domains, exchange, q, p, nrhs, overlap=overlap)
            alpha = np.where(active & (qq > 0), gamma / np.where(qq > 0, qq, 1.0), 0.0)
            for d, (_, x, _), pp, rr_, qv in zip(domains, D, p, r, q):
                d.axpby(x, alpha, one, pp)
                d.axpby(rr_, -alpha, one, qv)
            rparts = [d.norm2s(rr_, nrhs) for d, rr_ in zip(domains, r)]
            # s = Mhat^dag r, and the two sums reduced together
            gparts = _dd_apply(domains, exchange, s, r, nrhs, True, overlap)
            both = exchange.allreduce([np.concatenate([a, b]) for a, b in zip(rparts, gparts)])
            rr, gnew = both[:nrhs], both[nrhs:]
            if np.all(~active | (rr <= target)):
                # recompute the residual: q = b - Mhat x
                dd_mhat(domains, exchange, q, xs, nrhs, overlap=overlap)
                for d, qv, (_, _, b) in zip(domains, q, D):
                    d.axpby(qv, one, -one, b)
                rt = exchange.allreduce([d.norm2s(qv, nrhs) for d, qv in zip(domains, q)])
                rel = np.sqrt(rt / bn2)
                if np.all(rel <= tol):
                    return it, rel
                active = rel > tol
                target = np.where(active, target * 0.25, target)
            beta = np.where(active & (gamma > 0), gnew / np.where(gamma > 0, gamma, 1.0), 0.0)
            for d, pp, ss in zip(domains, p, s):
                d.axpby(pp, one, beta, ss)
            gamma = np.where(active, gnew, gamma)
            active &= rr > target
        return it, rel
    finally:
        for fs in (r, s, p, q):
            for d, f in zip(domains, fs):
                d.free(f)
