"""Failures made on the host, never on the GPU: a simulated out-of-memory
(LQCD_FAULT_ALLOC_AFTER makes library allocations fail before cudaMalloc is
called), non-finite inputs, non-SU(3) links, an iteration cap.  Each must come
back as a status code with a message, leaving the context usable."""
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest

import gen

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2001_05706_gb300 as L
    return L


def test_simulated_oom_is_reported_and_recoverable(lib):
    child = textwrap.dedent("""
        import sys, numpy as np
        sys.path.insert(0, %r)
        import gen, paper_2001_05706_gb300 as L
        dims = (4, 4, 4, 4)
        lat = L.Lattice(dims)                       # 3 allocations
        lat.load_gauge(gen.gauge_field(dims, 0.3, 1).view(np.float64))   # 1
        lat.clover(0.12, 1.0)                       # 1: the 5th
        psi = gen.gaussian_spinor(dims, 2)[0]
        try:
            lat.dslash(psi, "MHAT", "f32", 12)      # packed links: the 6th fails
            print("NO-ERROR")
        except L.LqcdError as e:
            print("STATUS", e.status, str(e).replace(chr(10), " "))
        lat.close()
        print("CLOSED")
    """ % ROOT)
    env = dict(os.environ, LQCD_FAULT_ALLOC_AFTER="5")
    out = subprocess.run([sys.executable, "-c", child], env=env, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr
    assert "STATUS -3" in out.stdout and "cannot allocate" in out.stdout, out.stdout
    assert "CLOSED" in out.stdout


def test_non_finite_source_and_links(lib):
    L = lib
    dims = (4, 4, 4, 4)
    U = gen.gauge_field(dims, 0.3, 1)
    lat = L.Lattice(dims)
    bad = U.copy()
    bad[0, 0, 0, 0, 1, 0, 0] = np.nan
    with pytest.raises(L.LqcdError) as e:
        lat.load_gauge(bad.view(np.float64))
    assert e.value.status == L.LQCD_ERR_NOT_SU3
    lat.load_gauge(U.view(np.float64))
    lat.clover(0.12, 1.0)
    b = gen.gaussian_spinor(dims, 3)[0]
    b[1, 1, 1, 1, 0, 0] = np.inf
    with pytest.raises(L.LqcdError) as e:
        lat.solve(b, tol=1e-10, inner="f16")
    assert e.value.status == L.LQCD_ERR_ARG and "not finite" in str(e.value)
    # the context still works
    x, st, info = lat.solve(gen.gaussian_spinor(dims, 3)[0], tol=1e-10, inner="f16")
    assert st == L.LQCD_OK
    lat.close()


def test_bad_solver_arguments(lib):
    L = lib
    dims = (4, 4, 4, 4)
    lat = L.Lattice(dims)
    lat.load_gauge(gen.gauge_field(dims, 0.3, 1).view(np.float64))
    lat.clover(0.12, 1.0)
    b = gen.gaussian_spinor(dims, 3)[0]
    for kw, msg in ((dict(tol=0.0), "tol"), (dict(max_iter=0), "max_iter"), (dict(delta=1.5, inner="f32"), "delta")):
        with pytest.raises(L.LqcdError) as e:
            lat.solve(b, **{"tol": 1e-10, **kw})
        assert e.value.status == L.LQCD_ERR_ARG and msg in str(e.value)
    lat.close()
