"""The allocation-free reduction entry point, lqcd_norm2_noalloc.

It exists for callers that cannot call cudaMalloc (device memory owned by
another allocator, latency-critical loops where an allocation would
synchronise the device): its scratch is a static array of the library.  This
file is named to be collected last, so a run that stops at the first failure
has already run every other test.  Each check compares the new entry point
with the existing lqcd_field_norm2 on the same data, through the C ABI, on
two calls in a row (the shared scratch must be reusable)."""
import numpy as np
import pytest

import gen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2001_05706_gb300 as L
    return L


def _existing_norms(L, ctx, canon, nrhs):
    """Per right-hand side ||v||^2 from the existing entry point (one field each)."""
    out = []
    for k in range(nrhs):
        f = L.lqcd_field_create(ctx, L.LQCD_F64, L.LQCD_FULL, 1)
        try:
            L.lqcd_field_import(ctx, f, np.ascontiguousarray(canon[k]))
            out.append(L.lqcd_field_norm2(ctx, f))
        finally:
            L.lqcd_field_destroy(f)
    return np.array(out)


def test_noalloc_norm2_matches_field_norm2_twice(lib):
    import torch
    L = lib
    dims = (8, 6, 4, 10)
    V = int(np.prod(dims))
    nrhs = 3
    stream = torch.cuda.current_stream()
    with L.Lattice(dims, stream=stream) as lat:
        for call, seed in enumerate((501, 502)):
            canon = gen.gaussian_spinor(dims, seed, nrhs=nrhs) * (1.0 + call)
            expect = _existing_norms(L, lat.ctx, canon, nrhs)
            x = torch.from_numpy(canon.view(np.float64).reshape(-1).copy()).cuda()
            res = torch.full((nrhs,), -1.0, dtype=torch.float64, device="cuda")
            L.lqcd_norm2_noalloc(x, 24 * V, nrhs, res, stream)
            torch.cuda.synchronize()
            got = res.cpu().numpy()
            assert np.all(np.abs(got - expect) <= 1e-12 * expect), (call, got, expect)
            # bitwise reproducible from call to call on the same data
            res2 = torch.zeros_like(res)
            L.lqcd_norm2_noalloc(x, 24 * V, nrhs, res2, stream)
            torch.cuda.synchronize()
            assert torch.equal(res, res2)


def test_noalloc_rejects_sizes_beyond_the_scratch(lib):
    import torch
    L = lib
    x = torch.zeros(16 * 65, dtype=torch.float64, device="cuda")
    r = torch.zeros(65, dtype=torch.float64, device="cuda")
    with pytest.raises(L.LqcdError) as e:
        L.lqcd_norm2_noalloc(x, 16, 65, r)
    assert e.value.status == L.LQCD_ERR_ARG and "64" in str(e.value)
    with pytest.raises(L.LqcdError):
        L.lqcd_norm2_noalloc(x, 0, 1, r)


@pytest.mark.parametrize("n,nrhs", [(3_000_000, 2), (100, 64)])
def test_noalloc_capped_grid_and_full_scratch(lib, n, nrhs):
    """Beyond 2048 x 1024 values the grid is capped at 1024 blocks and the
    kernel strides over the rest; 64 right-hand sides fill the static scratch.
    Checked against numpy's FP64 sum of squares on the host and against the
    existing entry point on canonical spinors, on two calls in a row."""
    import torch
    L = lib
    rng = np.random.default_rng(n + nrhs)
    for call in range(2):
        xh = rng.standard_normal(n * nrhs) * (1.0 + call)
        x = torch.from_numpy(xh).cuda()
        res = torch.full((nrhs,), -1.0, dtype=torch.float64, device="cuda")
        L.lqcd_norm2_noalloc(x, n, nrhs, res)
        torch.cuda.synchronize()
        expect = np.array([np.dot(xh[k * n:(k + 1) * n], xh[k * n:(k + 1) * n]) for k in range(nrhs)])
        assert np.all(np.abs(res.cpu().numpy() - expect) <= 1e-12 * expect), call


def test_noalloc_binding_checks_what_the_c_side_cannot(lib):
    """The C entry point sees bare pointers: the binding rejects a wrong dtype,
    too-short arrays and host tensors before any launch, and the C side
    rejects a host pointer."""
    import ctypes
    import torch
    L = lib
    x = torch.zeros(64, dtype=torch.float64, device="cuda")
    r = torch.zeros(2, dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        L.lqcd_norm2_noalloc(x.float(), 32, 2, r)
    with pytest.raises(ValueError):
        L.lqcd_norm2_noalloc(x, 33, 2, r)  # needs 66 values
    with pytest.raises(ValueError):
        L.lqcd_norm2_noalloc(x, 32, 3, r)  # result too short
    with pytest.raises(ValueError):
        L.lqcd_norm2_noalloc(x.cpu(), 32, 2, r)
    host = np.zeros(64)
    st = L._lib.lqcd_norm2_noalloc(host.ctypes.data_as(ctypes.c_void_p), 32, 2, ctypes.c_void_p(r.data_ptr()), None)
    assert st == L.LQCD_ERR_ARG
