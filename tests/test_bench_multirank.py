"""The multi-rank path of bench.py on CPU: two gloo ranks, max-over-ranks
timing and the whole-job (weak-scaling) throughput rank 0 reports."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms_local = 1.0 + rank  # rank 1 is the slow one
    dist.barrier()
    ms = bench.max_over_ranks(ms_local, dist, "cpu")
    gbs = bench.weak_gbs(1e9, ms, world)
    q.put((rank, ms, gbs))
    dist.destroy_process_group()


def test_two_gloo_ranks_report_the_slowest_rank():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, gbs in out:
        assert ms == 2.0  # the max over ranks, on every rank
        assert abs(gbs - 2 * 1e9 / 2e-3 / 1e9) < 1e-9  # both ranks' bytes over the slowest time


def test_single_process_helpers():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert abs(bench.weak_gbs(2e9, 1.0, 1) - 2000.0) < 1e-9
    assert bench.site_bytes("f32", 12, "k2a") == 864 and bench.site_bytes("f32", 12, "k2b") == 960
    assert bench.site_bytes("f64", 18, "k2a") == 2112 and bench.site_bytes("f16", 12, "k2b") == 496


def test_committed_profile_matches_the_kernel_source():
    """The ncu summary the bench reads its DRAM traffic from was captured on the
    current dslash source (same hash), so roofline.traffic is reported."""
    import bench
    for kernel in ("k2a", "k2b"):
        t = bench.profiled_traffic("dslash_f32_r12_mhat", kernel)
        assert t is not None and t > 0, kernel
        # compulsory bytes of one full-size launch; the measured traffic is within a few percent
        compulsory = 1048576 * bench.site_bytes("f32", 12, kernel)
        assert 0.9 < t / compulsory < 1.1
