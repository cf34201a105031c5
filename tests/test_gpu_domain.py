"""Domain decomposition along t on one GPU: several domains held by one
process, their halos exchanged by copies (LocalExchange), must reproduce the
single-domain operator bit for bit, and CG across the domains must solve the
Schur system to an oracle-recomputed residual.

Bit for bit: every output site of a domain is computed by the same kernel
from the same link, clover and neighbour values as on the full lattice; the
global antiperiodic sign arrives as an exact negation of the ghost data
(the redundantly computed ghost layer of y_e is then uniformly negated,
which is the sign the second hop across the boundary needs)."""
import numpy as np
import pytest

import gen
import oracle

pytestmark = pytest.mark.gpu
KAPPA, CSW = 0.12, 1.0


@pytest.fixture(scope="module")
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2001_05706_gb300 as L
    return L


def _domains(L, dims, ndom, U, tbc):
    from paper_2001_05706_gb300.domain import GpuDomain, LocalExchange, Partition
    doms = []
    for r in range(ndom):
        d = GpuDomain(Partition(dims, ndom, r, tbc))
        d.load_gauge(U)
        d.clover(KAPPA, CSW)
        doms.append(d)
    return doms, LocalExchange(ndom)


@pytest.mark.parametrize("ndom,tbc,overlap", [(2, 1, False), (4, 1, False), (2, 0, False), (1, 1, False),
                                              (2, 1, True), (4, 1, True), (1, 0, True)])
@pytest.mark.parametrize("dagger", [False, True])
def test_domains_reproduce_mhat_bitwise(lib, ndom, tbc, overlap, dagger):
    """Sequential and overlapped schedules (the interior slices computed
    before the halo is unpacked) both give the single-domain operator."""
    from paper_2001_05706_gb300.domain import dd_mhat
    L = lib
    dims = (8, 6, 4, 16)
    U = gen.gauge_field(dims, 0.3, 1201)
    psi = gen.gaussian_spinor(dims, 1202, nrhs=2)
    # single domain: the library's Mhat on the whole lattice
    with L.Lattice(dims, tbc) as lat:
        lat.load_gauge(U.view(np.float64))
        lat.clover(KAPPA, CSW)
        full = lat.dslash(psi, "MHAT_DAG" if dagger else "MHAT", "f64", 18)
    doms, ex = _domains(L, dims, ndom, U, tbc)
    try:
        xs = [d.new_field(2) for d in doms]
        zs = [d.new_field(2) for d in doms]
        for d, x in zip(doms, xs):
            d.import_global(x, psi)
        n2 = dd_mhat(doms, ex, zs, xs, 2, dagger=dagger, overlap=overlap)
        got = np.concatenate([d.export_interior(z, 2) for d, z in zip(doms, zs)], axis=1)
        odd = oracle.keep_parity(dims, np.ones(oracle.spinor_shape(dims)), 1) != 0
        assert np.array_equal(got[:, odd], full[:, odd])
        assert np.all(got[:, ~odd] == 0)
        for k in range(2):
            assert abs(n2[k] - oracle.norm2(full[k])) <= 1e-12 * n2[k]
        for d, x, z in zip(doms, xs, zs):
            d.free(x)
            d.free(z)
    finally:
        for d in doms:
            d.close()


@pytest.mark.parametrize("overlap", [False, True])
def test_domains_cgls_solves_the_schur_system(lib, overlap):
    from paper_2001_05706_gb300.domain import dd_cgls
    L = lib
    dims = (8, 6, 4, 16)
    U = gen.gauge_field(dims, 0.3, 1211)
    b = np.stack([oracle.keep_parity(dims, v, 1) for v in gen.gaussian_spinor(dims, 1212, nrhs=2)])
    doms, ex = _domains(L, dims, 2, U, 1)
    try:
        xs = [d.new_field(2) for d in doms]
        bs = [d.new_field(2) for d in doms]
        for d, bf in zip(doms, bs):
            d.import_global(bf, b)
        it, res = dd_cgls(doms, ex, xs, bs, 2, tol=1e-10, overlap=overlap)
        assert np.all(res <= 1e-10)
        x = np.concatenate([d.export_interior(xf, 2) for d, xf in zip(doms, xs)], axis=1)
        for d, xf, bf in zip(doms, xs, bs):
            d.free(xf)
            d.free(bf)
    finally:
        for d in doms:
            d.close()
    A = oracle.clover(dims, U, KAPPA, CSW)
    Ai = oracle.clover_inverse(A)
    for k in range(2):
        r = b[k] - oracle.apply_Mhat(dims, U, A, Ai, KAPPA, oracle.keep_parity(dims, x[k], 1))
        assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(b[k])
    assert it > 10


def test_slices_reject_bad_arguments(lib):
    import torch
    L = lib
    dims = (4, 4, 4, 8)
    with L.Lattice(dims) as lat:
        f = L.lqcd_field_create(lat.ctx, L.LQCD_F64, L.LQCD_ODD, 1)
        h = L.lqcd_field_create(lat.ctx, L.LQCD_F16, L.LQCD_ODD, 1)
        buf = torch.zeros(4096, dtype=torch.float64, device="cuda")
        try:
            for parity, t0, t1 in ((0, 0, 1), (1, 1, 9), (1, 3, 2)):  # even sites absent, past the end, empty
                with pytest.raises(L.LqcdError):
                    L.lqcd_field_slices(lat.ctx, f, parity, t0, t1, buf, 0)
            with pytest.raises(L.LqcdError):
                L.lqcd_field_slices(lat.ctx, f, 1, 0, 1, buf, 0, 2.0)  # factor not +-1
            with pytest.raises(L.LqcdError):
                L.lqcd_field_slices(lat.ctx, h, 1, 0, 1, buf, 0)  # FP16 scales live apart
        finally:
            L.lqcd_field_destroy(f)
            L.lqcd_field_destroy(h)
