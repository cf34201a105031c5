"""GPU parity of the operator kernels against the FP64 oracle, through the C ABI.

Tolerances (relative 2-norm over the output sites): 1e-12 for FP64 storage
and for double-float (DF64: two FP32 numbers per real, ~2^-47 relative
rounding per operation, a few hundred operations per output), 1e-5 for FP32,
1e-2 for FP16/BF16 storage with FP32 arithmetic."""
import numpy as np
import pytest

import gen
import oracle
from helpers import rel, site_max_rel

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "df64": 1e-12, "f32": 1e-5, "f16": 1e-2, "bf16": 1e-2}
# the largest error of any single site, relative to that site (floored at a
# tenth of the rms site norm): FP16 rounds each stored real to 2^-11, BF16 to
# 2^-8 of its site's scale, accumulated over the eight neighbours
SITE_TOL = {"f64": 1e-11, "df64": 1e-11, "f32": 1e-5, "f16": 1e-2, "bf16": 3e-2}
KAPPA, CSW, RHO = 0.12, 1.0, 1.5


@pytest.fixture(scope="module")
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2001_05706_gb300 as L
    return L


def _setup(L, dims, eps, seed, csw=CSW, tbc=1):
    U = gen.gauge_field(dims, eps, seed)
    lat = L.Lattice(dims, tbc)
    lat.load_gauge(U.view(np.float64))
    lat.clover(KAPPA, csw)
    lat.set_rho(RHO)
    A = oracle.clover(dims, U, KAPPA, csw) if csw != 0 else None
    Ai = oracle.clover_inverse(A) if A is not None else None
    return lat, U, A, Ai


def _oracle_op(op, dims, U, A, Ai, psi, tbc=1):
    e = lambda v: oracle.keep_parity(dims, v, 0)
    o = lambda v: oracle.keep_parity(dims, v, 1)
    if op == "HOP_EO":
        return e(oracle.hop(dims, U, o(psi), tbc))
    if op == "HOP_OE":
        return o(oracle.hop(dims, U, e(psi), tbc))
    if op == "K2A":
        return e(oracle.site_mul(Ai, oracle.hop(dims, U, o(psi), tbc)))
    if op == "M":
        return oracle.apply_M(dims, U, A, KAPPA, psi, tbc)
    if op == "M_DAG":
        return oracle.apply_M(dims, U, A, KAPPA, psi, tbc, dagger=True)
    if op == "MHAT":
        return oracle.apply_Mhat(dims, U, A, Ai, KAPPA, o(psi), tbc)
    if op == "MHAT_DAG":
        return oracle.apply_Mhat(dims, U, A, Ai, KAPPA, o(psi), tbc, dagger=True)
    if op == "MHAT_NORMAL":
        t = oracle.apply_Mhat(dims, U, A, Ai, KAPPA, o(psi), tbc)
        return oracle.apply_Mhat(dims, U, A, Ai, KAPPA, t, tbc, dagger=True)
    if op == "HW":
        return oracle.apply_HW(dims, U, RHO, psi, tbc)
    if op == "MHAT_SYM":
        return oracle.apply_Mhat_sym(dims, U, A, Ai, KAPPA, o(psi), tbc)
    if op == "MHAT_SYM_DAG":
        return oracle.apply_Mhat_sym(dims, U, A, Ai, KAPPA, o(psi), tbc, dagger=True)
    raise ValueError(op)


OPS = ["HOP_EO", "HOP_OE", "K2A", "M", "M_DAG", "MHAT", "MHAT_DAG", "MHAT_NORMAL", "HW", "MHAT_SYM", "MHAT_SYM_DAG"]
# (8,6,4,10): 960 sites per parity = 7.5 blocks of 128 threads (ragged tail)
DIMS = (8, 6, 4, 10)


@pytest.fixture(scope="module")
def clover_lattice(lib):
    lat, U, A, Ai = _setup(lib, DIMS, 0.3, 1001)
    yield lat, U, A, Ai
    lat.close()


@pytest.mark.parametrize("op", OPS)
@pytest.mark.parametrize("prec,recon", [("f64", 18), ("f64", 12), ("df64", 18), ("f32", 18), ("f32", 12), ("f16", 12),
                                        ("bf16", 12), ("f32", 8), ("f16", 8)])
def test_ops_clover(clover_lattice, op, prec, recon):
    lat, U, A, Ai = clover_lattice
    psi = gen.gaussian_spinor(DIMS, 2001)[0]
    out = lat.dslash(psi, op, prec, recon)
    expect = _oracle_op(op, DIMS, U, A, Ai, psi)
    assert rel(out, expect) < TOL[prec], f"{op} {prec} r{recon}"
    assert site_max_rel(out, expect) < SITE_TOL[prec], f"{op} {prec} r{recon} per site"


@pytest.mark.parametrize("op", ["K2A", "MHAT", "MHAT_DAG", "M", "MHAT_SYM_DAG"])
@pytest.mark.parametrize("prec", ["f64", "df64", "f32", "bf16"])
def test_ops_wilson(lib, op, prec):
    dims = (4, 4, 6, 8)
    lat, U, A, Ai = _setup(lib, dims, 0.3, 7, csw=0.0)
    psi = gen.gaussian_spinor(dims, 8)[0]
    recon = 18 if prec == "df64" else 12  # DF64 keeps all 18 reals of a link
    out = lat.dslash(psi, op, prec, recon)
    expect = _oracle_op(op, dims, U, None, None, psi)
    assert rel(out, expect) < TOL[prec]
    assert site_max_rel(out, expect) < SITE_TOL[prec]
    lat.close()


@pytest.mark.parametrize("nrhs", [2, 3, 4, 12])
@pytest.mark.parametrize("prec", ["f64", "df64", "f32", "f16"])
def test_multi_rhs(clover_lattice, nrhs, prec):
    lat, U, A, Ai = clover_lattice
    psi = gen.gaussian_spinor(DIMS, 3000 + nrhs, nrhs=nrhs)
    out = lat.dslash(psi, "MHAT", prec, 18 if prec == "df64" else 12)
    for k in range(nrhs):
        expect = _oracle_op("MHAT", DIMS, U, A, Ai, psi[k])
        assert rel(out[k], expect) < TOL[prec]
        assert site_max_rel(out[k], expect) < SITE_TOL[prec]


@pytest.mark.parametrize("op", ["MHAT_SYM", "MHAT_SYM_DAG"])
@pytest.mark.parametrize("prec", ["f64", "f32", "f16"])
def test_multi_rhs_symmetric_schur(clover_lattice, op, prec):
    lat, U, A, Ai = clover_lattice
    psi = gen.gaussian_spinor(DIMS, 3001, nrhs=4)
    out = lat.dslash(psi, op, prec, 18 if prec == "f64" else 12)
    for k in range(4):
        assert rel(out[k], _oracle_op(op, DIMS, U, A, Ai, psi[k])) < TOL[prec]


def test_periodic_time_and_2x4(lib):
    """Periodic t, and the 2^4 lattice where x+mu and x-mu coincide."""
    for dims, tbc in [((2, 2, 2, 2), 1), ((4, 2, 2, 4), 0)]:
        lat, U, A, Ai = _setup(lib, dims, 0.5, 5, tbc=tbc)
        psi = gen.gaussian_spinor(dims, 6)[0]
        for op in ("M", "MHAT"):
            out = lat.dslash(psi, op, "f64", 18)
            assert rel(out, _oracle_op(op, dims, U, A, Ai, psi, tbc)) < 1e-12
        lat.close()


def test_device_buffers_match_host(clover_lattice):
    import torch
    lat, U, A, Ai = clover_lattice
    psi = gen.gaussian_spinor(DIMS, 44, nrhs=2)
    host = lat.dslash(psi, "MHAT", "f32", 12)
    t = torch.from_numpy(psi.view(np.float64).copy()).cuda()
    dev = lat.dslash(t, "MHAT", "f32", 12)
    assert np.array_equal(dev.cpu().numpy().view(np.complex128).reshape(host.shape), host)


@pytest.mark.parametrize("dims,nrhs,prec", [((4, 4, 4, 8), 1, "f32"), ((4, 6, 4, 16), 2, "f16"),
                                            ((6, 4, 4, 12), 1, "f64")])
def test_pipelined_host_mhat(lib, dims, nrhs, prec):
    """Mhat on host buffers runs as a chunked copy/compute/copy pipeline over
    whole time slices (16, 8 or 4 chunks, the wrap chunk first): it must match
    the device-buffer path bit for bit, zero the even sites, and match the
    oracle."""
    import os
    import torch
    U = gen.gauge_field(dims, 0.3, 77)
    lat = lib.Lattice(dims)
    lat.load_gauge(U.view(np.float64))
    lat.clover(KAPPA, CSW)
    psi = gen.gaussian_spinor(dims, 78, nrhs=nrhs)
    host = lat.dslash(psi, "MHAT", prec, 12)
    t = torch.from_numpy(psi.view(np.float64).copy()).cuda()
    dev = lat.dslash(t, "MHAT", prec, 12).cpu().numpy().view(np.complex128).reshape(host.shape)
    assert np.array_equal(dev, host)
    os.environ["LQCD_NO_PIPELINE"] = "1"
    try:
        plain = lat.dslash(psi, "MHAT", prec, 12)
    finally:
        del os.environ["LQCD_NO_PIPELINE"]
    assert np.array_equal(plain, host)
    A = oracle.clover(dims, U, KAPPA, CSW)
    Ai = oracle.clover_inverse(A)
    for k in range(nrhs):
        expect = oracle.apply_Mhat(dims, U, A, Ai, KAPPA, oracle.keep_parity(dims, psi.reshape((nrhs,) + psi.shape[-6:])[k], 1), 1)
        got = host.reshape((nrhs,) + psi.shape[-6:])[k]
        assert rel(got, expect) < TOL[prec]
        assert np.all(oracle.keep_parity(dims, got, 0) == 0)
    lat.close()


def test_field_api_and_schur_split(clover_lattice, lib):
    L = lib
    lat, U, A, Ai = clover_lattice
    ctx = lat.ctx
    psi = gen.gaussian_spinor(DIMS, 91)[0]
    xo = oracle.keep_parity(DIMS, psi, 1)
    fx = L.lqcd_field_create(ctx, L.LQCD_F64, L.LQCD_ODD, 1)
    fy = L.lqcd_field_create(ctx, L.LQCD_F64, L.LQCD_EVEN, 1)
    fz = L.lqcd_field_create(ctx, L.LQCD_F64, L.LQCD_ODD, 1)
    try:
        L.lqcd_field_import(ctx, fx, np.ascontiguousarray(psi))
        back = np.zeros_like(psi)
        L.lqcd_field_export(ctx, fx, back)
        assert np.array_equal(back, xo)  # exact round trip of the odd sites
        L.lqcd_apply(ctx, L.LQCD_OP_K2A, 18, fy, fx)
        L.lqcd_apply_schur(ctx, 18, 0, fz, fx, fy)
        z = np.zeros_like(psi)
        L.lqcd_field_export(ctx, fz, z)
        assert rel(z, _oracle_op("MHAT", DIMS, U, A, Ai, psi)) < 1e-12
        # dagger split: y from g5 x, then the g5 on the hop result
        fg = L.lqcd_field_create(ctx, L.LQCD_F64, L.LQCD_ODD, 1)
        L.lqcd_field_import(ctx, fg, np.ascontiguousarray(oracle.gamma5(psi)))
        L.lqcd_apply(ctx, L.LQCD_OP_K2A, 18, fy, fg)
        L.lqcd_apply_schur(ctx, 18, 1, fz, fx, fy)
        L.lqcd_field_export(ctx, fz, z)
        assert rel(z, _oracle_op("MHAT_DAG", DIMS, U, A, Ai, psi)) < 1e-12
        L.lqcd_field_destroy(fg)
        # deterministic FP64 norm
        n1 = L.lqcd_field_norm2(ctx, fz)
        n2 = L.lqcd_field_norm2(ctx, fz)
        assert n1 == n2
        assert abs(n1 - oracle.norm2(z)) < 1e-12 * n1
    finally:
        for f in (fx, fy, fz):
            L.lqcd_field_destroy(f)


def test_rejects_non_su3_and_bad_args(lib):
    L = lib
    dims = (4, 4, 4, 4)
    U = gen.gauge_field(dims, 0.3, 1)
    U[1, 2, 3, 0, 2] *= 1.001
    lat = L.Lattice(dims)
    with pytest.raises(L.LqcdError) as e:
        lat.load_gauge(U.view(np.float64))
    assert e.value.status == L.LQCD_ERR_NOT_SU3
    psi = gen.gaussian_spinor(dims, 1)[0]
    with pytest.raises(L.LqcdError) as e:
        lat.dslash(psi, "MHAT", "f64", 18)
    assert e.value.status == L.LQCD_ERR_STATE
    lat.load_gauge(gen.gauge_field(dims, 0.3, 1).view(np.float64))
    with pytest.raises(L.LqcdError) as e:
        lat.dslash(psi, "MHAT", "f64", 18)  # kappa not set yet
    assert e.value.status == L.LQCD_ERR_STATE
    lat.clover(0.12, 1.0)
    with pytest.raises(L.LqcdError) as e:
        lat.dslash(psi, "MHAT", "f16", 18)  # half links are 12-real only
    assert e.value.status == L.LQCD_ERR_ARG
    with pytest.raises(L.LqcdError):
        L.lqcd_create((4, 3, 4, 4))
    lat.close()


# ---------------------------------------------------------------------------
# full size: 32^3 x 64, the configuration the benchmark times, sampled sites
# ---------------------------------------------------------------------------

def _mhat_at_sites(dims, U, kappa, csw, x, sites):
    """Mhat x at the given odd sites, from per-site oracle evaluations only."""
    V = int(np.prod(dims))
    xo = oracle.keep_parity(dims, x, 1)
    # the even neighbours of each sample, and y = A^-1 D x there
    L0, L1, L2, L3 = dims
    x0, x1, x2, x3 = oracle.site_coords(dims, np.asarray(sites))
    nb = set()
    for mu, Lm in enumerate(dims):
        for d in (1, -1):
            c = [x0.copy(), x1.copy(), x2.copy(), x3.copy()]
            c[mu] = (c[mu] + d) % Lm
            nb.update((c[0] + L0 * (c[1] + L1 * (c[2] + L2 * c[3]))).tolist())
    nb = np.array(sorted(nb))
    Dx = oracle.hop_sites(dims, U, xo, nb)
    An = oracle.clover_sites(dims, U, kappa, csw, nb)
    y = np.zeros((V, 12), dtype=np.complex128)
    for k, s in enumerate(nb):
        y[s] = np.linalg.solve(An[k], Dx[k].reshape(12))
    Dy = oracle.hop_sites(dims, U, y.reshape(oracle.spinor_shape(dims)), sites)
    As = oracle.clover_sites(dims, U, kappa, csw, sites)
    xf = xo.reshape(V, 12)
    return np.stack([As[k] @ xf[s] - kappa**2 * Dy[k].reshape(12) for k, s in enumerate(sites)])


@pytest.mark.parametrize("prec,recon", [("f32", 12), ("f64", 18), ("df64", 18), ("f16", 12)])
def test_full_size_sampled(lib, prec, recon):
    L = lib
    dims = (32, 32, 32, 64)
    kappa, csw = 0.125, 1.0
    U = gen.gauge_field(dims, 0.2, 1002)
    lat = L.Lattice(dims)
    lat.load_gauge(U.view(np.float64))
    lat.clover(kappa, csw)
    psi = gen.gaussian_spinor(dims, 2002)[0]
    ctx = lat.ctx
    P = L.PREC[prec]
    fx = L.lqcd_field_create(ctx, P, L.LQCD_ODD, 1)
    fz = L.lqcd_field_create(ctx, P, L.LQCD_ODD, 1)
    L.lqcd_field_import(ctx, fx, psi)
    L.lqcd_apply(ctx, L.LQCD_OP_MHAT, recon, fz, fx)  # the call the benchmark times
    z = np.zeros_like(psi)
    L.lqcd_field_export(ctx, fz, z)
    L.lqcd_field_destroy(fx)
    L.lqcd_field_destroy(fz)
    lat.close()
    V = int(np.prod(dims))
    rng = np.random.default_rng(0)
    cand = rng.choice(V, 400, replace=False)
    par = np.array([sum(c) % 2 for c in zip(*oracle.site_coords(dims, cand))])
    # odd sites on the t boundaries and the x, y, z wraps, plus random ones
    edge = []
    for c in [(31, 0, 0, 0), (0, 31, 0, 0), (0, 0, 31, 0), (0, 0, 0, 63), (31, 31, 31, 63), (1, 0, 0, 0),
              (30, 0, 0, 63), (31, 0, 1, 0), (0, 0, 0, 1)]:
        if sum(c) % 2 == 1:
            edge.append(c[0] + 32 * (c[1] + 32 * (c[2] + 32 * c[3])))
    sites = np.array(sorted(set(edge) | set(cand[par == 1][:64].tolist())))
    expect = _mhat_at_sites(dims, U, kappa, csw, psi, sites)
    got = z.reshape(V, 12)[sites]
    assert rel(got, expect) < TOL[prec]
    assert site_max_rel(got, expect) < SITE_TOL[prec]


def test_df64_rejects_12_real_links(clover_lattice, lib):
    lat, U, A, Ai = clover_lattice
    psi = gen.gaussian_spinor(DIMS, 2001)[0]
    with pytest.raises(lib.LqcdError) as e:
        lat.dslash(psi, "MHAT", "df64", 12)
    assert e.value.status == lib.LQCD_ERR_ARG and "18-real" in str(e.value)


def test_df64_beats_fp32_and_tracks_fp64(clover_lattice):
    """DF64 is not FP32 in disguise: its error against the oracle is orders
    of magnitude below FP32's and within a small factor of FP64's."""
    lat, U, A, Ai = clover_lattice
    psi = gen.gaussian_spinor(DIMS, 2011)[0]
    expect = _oracle_op("MHAT", DIMS, U, A, Ai, psi)
    e32 = rel(lat.dslash(psi, "MHAT", "f32", 18), expect)
    e64 = rel(lat.dslash(psi, "MHAT", "f64", 18), expect)
    edf = rel(lat.dslash(psi, "MHAT", "df64", 18), expect)
    assert edf < 1e-5 * e32
    assert edf < 1e-13 and e64 < 1e-14


def test_eight_real_links_refused_for_unit_links(lib):
    """The 8-real rebuild divides by 1 - |U00|^2: unit links (the free field)
    are refused for it, and still run with 12 reals."""
    dims = (4, 4, 4, 4)
    lat = lib.Lattice(dims)
    lat.load_gauge(gen.unit_gauge(dims).view(np.float64))
    lat.clover(KAPPA, CSW)
    psi = gen.gaussian_spinor(dims, 5)[0]
    with pytest.raises(lib.LqcdError) as e:
        lat.dslash(psi, "MHAT", "f32", 8)
    assert e.value.status == lib.LQCD_ERR_ARG
    lat.dslash(psi, "MHAT", "f32", 12)
    for prec in ("f64", "bf16"):  # no FP64 8-real form; BF16 cannot hold the angles
        with pytest.raises(lib.LqcdError):
            lat.dslash(psi, "MHAT", prec, 8)
    lat.close()
