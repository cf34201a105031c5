"""The domain decomposition's index, exchange and solver logic on CPU.

`paper_2001_05706_gb300.domain` cuts the lattice along t, routes the halos
and runs CGLS across domains; the arithmetic of a domain is a pluggable
object.  Here that object is the FP64 oracle on the domain's extended
lattice (periodic in t, as the library context is), so the partition, the
ghost-slice routing, the antiperiodic sign carried by the halos, the
redundantly computed ghost layer of y_e and the distributed reductions are
checked against the oracle's operator on the whole lattice: with domains in
one process (LocalExchange) and with two gloo ranks (DistExchange)."""
import os
import socket

import numpy as np
import pytest

import gen
import oracle

KAPPA, CSW = 0.12, 1.0
DIMS = (4, 4, 2, 8)


class OracleDomain:
    """A domain computed by the oracle: fields are canonical complex arrays
    [rhs][extended t][z][y][x][4][3] of the odd sites."""

    def __init__(self, part, U_global):
        self.part = part
        self.U = part.slab(U_global)
        self.A = oracle.clover(part.local_dims, self.U, KAPPA, CSW)
        self.Ai = oracle.clover_inverse(self.A)
        lo, hi = part.interior
        self.mask = np.zeros(part.local_dims[3], dtype=bool)
        self.mask[lo:hi] = True
        self.y = None

    def new_field(self, nrhs):
        L0, L1, L2, Le = self.part.local_dims
        return np.zeros((nrhs, Le, L2, L1, L0, 4, 3), dtype=np.complex128)

    def free(self, f):
        pass

    def import_global(self, f, canon):
        slab = np.asarray(canon)[:, self.part.slab_t]
        for k in range(f.shape[0]):
            f[k] = oracle.keep_parity(self.part.local_dims, slab[k], 1)
        f[:, ~self.mask] = 0

    def export_interior(self, f, nrhs):
        lo, hi = self.part.interior
        return f[:nrhs, lo:hi].copy()

    def pack(self, f, nrhs):
        """The send slices; then x's ghost slices and all of y_e are set to NaN,
        so that a schedule reading either before it is rewritten (before the
        halo arrives, or before K2a has produced it) leaves NaN in the result."""
        import torch
        (a, b), (c, d) = self.part.send_lo, self.part.send_hi
        sends = (torch.from_numpy(np.ascontiguousarray(f[:, a:b]).view(np.float64).copy()),
                 torch.from_numpy(np.ascontiguousarray(f[:, c:d]).view(np.float64).copy()))
        f[:, ~self.mask] = np.nan
        self.y = np.full(f.shape, np.nan, dtype=np.complex128)
        return sends

    def unpack(self, f, rlo, rhi):
        (a, b), (c, d) = self.part.ghost_lo, self.part.ghost_hi
        f[:, a:b] = self.part.factor_lo * rlo.numpy().view(np.complex128).reshape(f[:, a:b].shape)
        f[:, c:d] = self.part.factor_hi * rhi.numpy().view(np.complex128).reshape(f[:, c:d].shape)

    def clear_ghosts(self, f, nrhs):
        f[:, ~self.mask] = 0

    def k2a(self, x, nrhs, t0, t1, dagger=False):
        """y_e = A_ee^-1 D_eo x_o (dagger: g5 x_o) on slices [t0, t1) (Sec. 3's
        even-odd factorisation), computed everywhere and kept on the slices."""
        dims = self.part.local_dims
        for k in range(nrhs):
            v = oracle.keep_parity(dims, x[k], 1)
            if dagger:
                v = oracle.gamma5(v)
            y = oracle.site_mul(self.Ai, oracle.keep_parity(dims, oracle.hop(dims, self.U, v, 0), 0))
            self.y[k, t0:t1] = y[t0:t1]

    def k2b(self, out, x, nrhs, t0, t1, dagger=False):
        """z_o = A_oo x_o - kappa^2 D_oe y_e (dagger: g5 on the hop) on slices
        [t0, t1); the per-RHS ||z_o||^2 over them."""
        dims = self.part.local_dims
        n2 = np.zeros(nrhs)
        for k in range(nrhs):
            h = oracle.keep_parity(dims, oracle.hop(dims, self.U, self.y[k], 0), 1)
            if dagger:
                h = oracle.gamma5(h)
            z = oracle.site_mul(self.A, oracle.keep_parity(dims, x[k], 1)) - KAPPA ** 2 * h
            out[k, t0:t1] = z[t0:t1]
            n2[k] = oracle.norm2(z[t0:t1])
        return n2

    def axpby(self, y, a, b, x):
        for k in range(y.shape[0]):
            y[k] = a[k] * x[k] + b[k] * y[k]

    def norm2s(self, f, nrhs):
        return np.array([oracle.norm2(f[k]) for k in range(nrhs)])


def _global_mhat(U, psi, tbc, dagger):
    A = oracle.clover(DIMS, U, KAPPA, CSW)
    Ai = oracle.clover_inverse(A)
    return np.stack([oracle.apply_Mhat(DIMS, U, A, Ai, KAPPA, oracle.keep_parity(DIMS, v, 1), tbc, dagger=dagger)
                     for v in psi])


def _run(domains, exchange, psi, b, tbc, dagger, overlap=False):
    from paper_2001_05706_gb300.domain import dd_cgls, dd_mhat
    xs = [d.new_field(2) for d in domains]
    zs = [d.new_field(2) for d in domains]
    for d, x in zip(domains, xs):
        d.import_global(x, psi)
    n2 = dd_mhat(domains, exchange, zs, xs, 2, dagger=dagger, overlap=overlap)
    z = [d.export_interior(zf, 2) for d, zf in zip(domains, zs)]
    bs = [d.new_field(2) for d in domains]
    sol = [d.new_field(2) for d in domains]
    for d, bf in zip(domains, bs):
        d.import_global(bf, b)
    it, res = dd_cgls(domains, exchange, sol, bs, 2, tol=1e-10, overlap=overlap)
    return z, n2, [d.export_interior(s, 2) for d, s in zip(domains, sol)], it, res


@pytest.mark.parametrize("ndom,tbc,dagger,overlap", [(2, 1, False, False), (4, 1, True, False), (2, 0, True, False),
                                                     (1, 1, False, False), (2, 1, True, True), (4, 1, False, True),
                                                     (1, 0, True, True)])
def test_domains_in_one_process_match_the_oracle(ndom, tbc, dagger, overlap):
    from paper_2001_05706_gb300.domain import LocalExchange, Partition
    U = gen.gauge_field(DIMS, 0.4, 71)
    psi = gen.gaussian_spinor(DIMS, 72, nrhs=2)
    b = np.stack([oracle.keep_parity(DIMS, v, 1) for v in gen.gaussian_spinor(DIMS, 73, nrhs=2)])
    doms = [OracleDomain(Partition(DIMS, ndom, r, tbc), U) for r in range(ndom)]
    z, n2, x, it, res = _run(doms, LocalExchange(ndom), psi, b, tbc, dagger, overlap)
    expect = _global_mhat(U, psi, tbc, dagger)
    got = np.concatenate(z, axis=1)
    assert np.abs(got - expect).max() <= 1e-13 * np.abs(expect).max()
    assert np.allclose(n2, [oracle.norm2(e) for e in expect], rtol=1e-12)
    xg = np.concatenate(x, axis=1)
    r = b - _global_mhat(U, xg, tbc, False)
    assert all(np.linalg.norm(r[k]) <= 1e-10 * np.linalg.norm(b[k]) for k in range(2))
    assert np.all(res <= 1e-10)


def test_partition_rejects_bad_splits():
    from paper_2001_05706_gb300.domain import Partition
    with pytest.raises(ValueError):
        Partition((4, 4, 4, 8), 3, 0)  # 8 slices do not split in 3
    with pytest.raises(ValueError):
        Partition((4, 4, 4, 6), 2, 0)  # 3 slices per domain: odd
    with pytest.raises(ValueError):
        Partition((4, 4, 4, 8), 2, 2)
    p = Partition((4, 4, 4, 16), 4, 3, 1)
    assert p.local_dims == (4, 4, 4, 8) and p.t_off == 12
    assert p.slab_t == [10, 11, 12, 13, 14, 15, 0, 1]
    assert p.factor_hi == -1.0 and p.factor_lo == 1.0  # the top domain's upper ghosts cross t = L3


@pytest.mark.parametrize("lt", [2, 4, 6, 8, 12])
def test_overlapped_schedule_covers_each_slice_once(lt):
    """The overlapped schedule's K2a ranges tile the sequential K2a range and
    its K2b ranges the interior, each slice once; the pieces that run before
    the halo arrives read x_o only on the interior (K2a at t reads t - 1 and
    t + 1) and y_e only where the early K2a wrote it."""
    from paper_2001_05706_gb300.domain import HALO, Partition
    p = Partition((4, 4, 4, 4 * lt), 4, 1)

    def cover(ranges):
        return sorted(t for a, b in ranges for t in range(a, b))

    inner_a, inner_b = p.k2a_inner, p.k2b_inner
    assert cover([inner_a] + p.k2a_edges) == list(range(*p.k2a_slices))
    assert cover([inner_b] + p.k2b_edges) == list(range(*p.interior))
    interior = set(range(*p.interior))
    assert all({t - 1, t + 1} <= interior for t in range(*inner_a))
    assert all({t - 1, t + 1} <= set(range(*inner_a)) for t in range(*inner_b))
    if lt > 4:  # something is left to hide the exchange behind
        assert inner_b[1] - inner_b[0] == lt - 2 * HALO


# ---- two gloo ranks ---------------------------------------------------------

def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, tbc, dagger, overlap, q):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
    import torch.distributed as dist
    from paper_2001_05706_gb300.domain import DistExchange, Partition
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        U = gen.gauge_field(DIMS, 0.4, 71)
        psi = gen.gaussian_spinor(DIMS, 72, nrhs=2)
        b = np.stack([oracle.keep_parity(DIMS, v, 1) for v in gen.gaussian_spinor(DIMS, 73, nrhs=2)])
        dom = OracleDomain(Partition(DIMS, world, rank, tbc), U)
        z, n2, x, it, res = _run([dom], DistExchange(), psi, b, tbc, dagger, overlap)
        q.put((rank, z[0], n2, x[0], it, res))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,tbc,dagger,overlap", [(2, 1, False, False), (2, 1, True, False), (2, 1, True, True),
                                                      (4, 1, False, True)])
def test_gloo_ranks_match_the_oracle(world, tbc, dagger, overlap):
    """Two ranks (both neighbours the same peer) and four (distinct peers
    below and above) against the oracle on the whole lattice."""
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, tbc, dagger, overlap, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted((q.get(timeout=300) for _ in range(world)), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    U = gen.gauge_field(DIMS, 0.4, 71)
    psi = gen.gaussian_spinor(DIMS, 72, nrhs=2)
    b = np.stack([oracle.keep_parity(DIMS, v, 1) for v in gen.gaussian_spinor(DIMS, 73, nrhs=2)])
    expect = _global_mhat(U, psi, tbc, dagger)
    got = np.concatenate([o[1] for o in out], axis=1)
    assert np.abs(got - expect).max() <= 1e-13 * np.abs(expect).max()
    for o in out:  # the reduced norms are the global ones on every rank
        assert np.allclose(o[2], [oracle.norm2(e) for e in expect], rtol=1e-12)
        assert o[4] == out[0][4]  # the same iteration count on both ranks
    xg = np.concatenate([o[3] for o in out], axis=1)
    r = b - _global_mhat(U, xg, tbc, False)
    assert all(np.linalg.norm(r[k]) <= 1e-10 * np.linalg.norm(b[k]) for k in range(2))
