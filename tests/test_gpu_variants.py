"""Every dslash kernel variant against the FP64 oracle, element by element.

Per launch the library picks one of: dslash_kernel with 1, 2 or 4 right-hand
sides per thread (variant codes 1, 2, 4), or the tiled many-right-hand-side
kernel with g = 1, 2, 3, 6 warps of two right-hand sides per block sharing
one staged tile of links and clover (codes 101, 102, 103, 106).  The
autotuner keeps whichever was fastest on the device, so without a way to
force one the others would go untested; LQCD_FORCE_VARIANT forces it.

Each right-hand side is checked twice: the relative 2-norm over all sites
against the operator tolerance (1e-12 FP64 and DF64, 1e-5 FP32, 1e-2
FP16/BF16 storage) and the largest per-site relative error against a
per-site bound, so a single wrong site cannot hide in the norm."""
import os

import numpy as np
import pytest

import gen
import oracle
from helpers import rel, site_max_rel

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "df64": 1e-12, "f32": 1e-5, "f16": 1e-2, "bf16": 1e-2}
# per-site bounds: storage rounding of one site's inputs and output (FP16 2^-11,
# BF16 2^-8 relative per component) accumulated over its eight neighbours
SITE_TOL = {"f64": 1e-11, "df64": 1e-11, "f32": 1e-5, "f16": 1e-2, "bf16": 3e-2}
KAPPA, CSW, RHO = 0.12, 1.0, 1.5
DIMS = (8, 6, 4, 10)  # 960 sites per parity: 30 tiles of 32, 7.5 blocks of 128
OPS = ["MHAT", "MHAT_DAG", "M_DAG", "HOP_OE", "HW", "MHAT_SYM"]
PRECS = [("f32", 12), ("f32", 18), ("f16", 12), ("bf16", 12), ("f64", 18), ("df64", 18)]
VARIANTS = [1, 2, 4, 101, 102, 103, 106]


def admissible(v, prec, nrhs):
    """Whether the variant runs the main launches of an operator at this size."""
    if v < 100:
        return nrhs % v == 0 and not (prec == "df64" and v == 4)
    return prec in ("f32", "f16", "bf16") and nrhs >= 2 and v - 100 <= (nrhs + 1) // 2


@pytest.fixture(scope="module")
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2001_05706_gb300 as L
    return L


@pytest.fixture(scope="module")
def setup(lib):
    U = gen.gauge_field(DIMS, 0.3, 1101)
    lat = lib.Lattice(DIMS)
    lat.load_gauge(U.view(np.float64))
    lat.clover(KAPPA, CSW)
    lat.set_rho(RHO)
    A = oracle.clover(DIMS, U, KAPPA, CSW)
    Ai = oracle.clover_inverse(A)
    yield lat, U, A, Ai, {}
    lat.close()


def _oracle(op, U, A, Ai, psi):
    o = lambda v: oracle.keep_parity(DIMS, v, 1)
    e = lambda v: oracle.keep_parity(DIMS, v, 0)
    if op == "MHAT":
        return oracle.apply_Mhat(DIMS, U, A, Ai, KAPPA, o(psi))
    if op == "MHAT_DAG":
        return oracle.apply_Mhat(DIMS, U, A, Ai, KAPPA, o(psi), dagger=True)
    if op == "M_DAG":
        return oracle.apply_M(DIMS, U, A, KAPPA, psi, dagger=True)
    if op == "HOP_OE":
        return o(oracle.hop(DIMS, U, e(psi)))
    if op == "HW":
        return oracle.apply_HW(DIMS, U, RHO, psi)
    if op == "MHAT_SYM":
        return oracle.apply_Mhat_sym(DIMS, U, A, Ai, KAPPA, o(psi))
    raise ValueError(op)


@pytest.fixture
def force():
    def set_variant(v):
        os.environ["LQCD_FORCE_VARIANT"] = str(v)
    yield set_variant
    os.environ.pop("LQCD_FORCE_VARIANT", None)


@pytest.mark.parametrize("nrhs", [3, 12])
@pytest.mark.parametrize("prec,recon", PRECS)
@pytest.mark.parametrize("variant", VARIANTS)
def test_variant_ops(setup, force, variant, prec, recon, nrhs):
    if not admissible(variant, prec, nrhs):
        pytest.skip("variant cannot run this launch")
    lat, U, A, Ai, cache = setup
    psi = gen.gaussian_spinor(DIMS, 4000 + nrhs, nrhs=nrhs)
    force(variant)
    for op in OPS:
        out = lat.dslash(psi, op, prec, recon)
        for k in range(nrhs):
            key = (op, nrhs, k)
            if key not in cache:
                cache[key] = _oracle(op, U, A, Ai, psi[k])
            expect = cache[key]
            assert rel(out[k], expect) < TOL[prec], f"{op} rhs {k}"
            assert site_max_rel(out[k], expect) < SITE_TOL[prec], f"{op} rhs {k} per site"


@pytest.mark.parametrize("variant", [1, 2, 4, 101, 102])
@pytest.mark.parametrize("inner", ["f16", "f32"])
def test_variant_mixed_solve(setup, force, variant, inner):
    """A four-right-hand-side mixed CGLS under each variant: the fused
    ||Mhat p||^2 of the forced kernel drives the recursion, and every
    right-hand side reaches an oracle-recomputed true residual of 1e-10."""
    import paper_2001_05706_gb300 as L
    lat, U, A, Ai, _ = setup
    b = gen.gaussian_spinor(DIMS, 4100, nrhs=4)
    force(variant)
    x, st, info = lat.solve(b, tol=1e-10, inner=inner, nrhs=4)
    assert st == L.LQCD_OK, L.lqcd_last_error()
    for k in range(4):
        assert oracle.true_residual(DIMS, U, A, KAPPA, x[k], b[k]) <= 1e-10
