"""Benchmark: Wilson-clover even-odd dslash HBM throughput on GB300, and
mixed-precision vs FP64 solve time to a true residual of 1e-10.

Workload (one "step"): one application of the Schur complement
Mhat = A_oo - kappa^2 D_oe A_ee^-1 D_eo (kernels K2a: y = A^-1 D x and
K2b: z = A x - kappa^2 D y) on a 32^3 x 64 lattice, c_sw = 1.0,
kappa = 0.125, links exp(i 0.2 A) (seeded synthetic), FP32 storage and
arithmetic, 12-real links, one right-hand side, fields resident in HBM.
Throughput uses the compulsory byte model: per output site 8 links, the
input spinor, the output spinor, the clover block pair (and the local
spinor for K2b) -- 864 + 960 bytes per site in FP32 with 12-real links.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl lqcd|reference]
                  [--no-solve] [--no-batch] [--kernel-only k2a|k2b|mhat --lattice X,Y,Z,T]
                  [--solver-iteration]
  python bench.py --overlap [--high df64] [--eig lanczos]   (overlap set-up and 12-RHS solve on 16^3x32)
  python bench.py --solve-lattice 48,48,48,96   (mixed vs FP64 solve only, on that lattice)

--impl reference times the FP64 CPU oracle on the same workload (bounded
time-slab samples per step).  --kernel-only runs just that kernel (for ncu).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

DIMS = (32, 32, 32, 64)
KAPPA, CSW, EPS = 0.125, 1.0, 0.2
GAUGE_SEED, SRC_SEED = 1002, 2002
METRIC = "Wilson-clover dslash HBM GB/s (% of peak); mixed vs FP64 solve time to 1e-10"
WORKLOAD = ("Wilson-clover even-odd Mhat = K2a (A^-1 D) + K2b (A x - kappa^2 D y), 32^3x64, c_sw=1.0, "
            "kappa=0.125, links exp(i*0.2*A) seeded, FP32 storage+math, 12-real links, 1 RHS")
FLOPS = {"k2a": 1824, "k2b": 1872}
PB = {"f64": 8, "df64": 8, "f32": 4, "f16": 2, "bf16": 2}


def bench_config(world: int) -> dict:
    """The workload description both arms print (same keys, same values)."""
    return {"workload": WORKLOAD, "lattice": list(DIMS), "prec": "f32", "recon": 12, "nrhs": 1,
            "kappa": KAPPA, "c_sw": CSW, "eps": EPS, "parallelism": f"replicas x{world}",
            "l2": "inputs larger than L2: each step streams ~1.2 GB (links 403 MB, clover 604 MB, spinors)"}


def site_bytes(prec: str, recon: int, kernel: str) -> int:
    """Compulsory bytes per output site: 8 links, input spinor, output spinor,
    clover block pair (+ the local spinor for K2b); FP16/BF16 add a 4-byte
    scale per spinor and clover site."""
    b = PB[prec]
    half = prec in ("f16", "bf16")
    link = 8 * recon * b
    sp = 24 * b + (4 if half else 0)
    cl = 72 * b + (4 if half else 0)
    k2a = link + 2 * sp + cl
    return k2a if kernel == "k2a" else k2a + sp


def mhat_bytes(prec, recon):
    return site_bytes(prec, recon, "k2a") + site_bytes(prec, recon, "k2b")


def mhat_bytes_per_rhs(prec, recon, nrhs):
    """Compulsory bytes per output site and right-hand side of an nrhs-RHS Mhat:
    links and clover once per site for all right-hand sides, spinors per RHS
    (K2a: input and output; K2b: input, local and output)."""
    b = PB[prec]
    half = prec in ("f16", "bf16")
    sp = 24 * b + (4 if half else 0)
    lc = 8 * recon * b + 72 * b + (4 if half else 0)
    return 2 * lc / nrhs + 5 * sp


# ---------------------------------------------------------------------------
# helpers
# ---------------------------------------------------------------------------

def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "MEASURED_PEAKS.json hbm_gbs (of measured)"
    except Exception:
        return 6800.0, "recipe fallback 6.8 TB/s (of fallback)"


def kernel_source_hash():
    h = hashlib.sha256()
    for f in ("dslash.cuh", "common.cuh", "reduce.cuh", "dslash_inst.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2001_05706_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def profiled_traffic(name, kernel):
    """Per-launch DRAM bytes recorded in profiles/<name>.md, if the kernel
    source has not changed since the capture (else None)."""
    p = os.path.join(ROOT, "profiles", name + ".md")
    if not os.path.exists(p):
        return None
    vals = {}
    for line in open(p):
        if ":" in line and line.strip().startswith("- "):
            k, v = line.strip()[2:].split(":", 1)
            vals[k.strip()] = v.strip().strip("`")
    if vals.get("source_sha256") != kernel_source_hash():
        return None
    key = "traffic_bytes_per_launch_full_size" + ("_k2a" if kernel == "k2a" else "")
    try:
        return int(float(vals[key]))
    except (KeyError, ValueError):
        return None


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200", "-i",
                 str(gpu_index)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def max_over_ranks(x, dist=None, device="cpu"):
    """The largest x over all ranks (x itself without a process group)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_gbs(bytes_per_rank_step, ms, world):
    """Whole-job GB/s of a weak-scaled step: every rank moves the same bytes and
    the step takes the slowest rank's time."""
    return world * bytes_per_rank_step / (ms * 1e-3) / 1e9


def gpu_index(local_rank):
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        ids = [v for v in vis.split(",") if v.strip()]
        if local_rank < len(ids):
            return ids[local_rank].strip()
    return str(local_rank)


# ---------------------------------------------------------------------------
# CPU oracle pieces (cpu_baseline leg and the reference arm only)
# ---------------------------------------------------------------------------

def oracle_setup(U):
    import oracle
    A = oracle.clover(DIMS, U, KAPPA, CSW)
    Ai = oracle.clover_inverse(A)
    return A, Ai


def oracle_slab_rate(U, A, Ai, psi, target_s=8.0):
    """Time the oracle Mhat on whole time slices, repeating passes over the
    lattice until ~target_s of wall time; returns (sites per second, slices
    timed, seconds)."""
    import oracle
    out = np.zeros_like(psi)
    t0 = time.perf_counter()
    oracle.mhat_slab(DIMS, U, A, Ai, KAPPA, psi, 0, 1, out)
    one = time.perf_counter() - t0
    n = max(1, int(target_s / max(one, 1e-4)))
    done = 0
    t0 = time.perf_counter()
    while done < n:
        t = done % DIMS[3]
        k = min(n - done, DIMS[3] - t)
        oracle.mhat_slab(DIMS, U, A, Ai, KAPPA, psi, t, t + k, out)
        done += k
    dt = time.perf_counter() - t0
    sites = n * DIMS[0] * DIMS[1] * DIMS[2] // 2
    return sites / dt, n, dt


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def make_inputs():
    import gen
    U = gen.gauge_field(DIMS, EPS, GAUGE_SEED)
    psi = gen.gaussian_spinor(DIMS, SRC_SEED)[0]
    return U, psi


# ---------------------------------------------------------------------------
# reference arm: the FP64 oracle on the host cores
# ---------------------------------------------------------------------------

def run_reference(args, rank):
    if rank != 0:
        return 0
    U, psi = make_inputs()
    A, Ai = oracle_setup(U)
    import oracle
    out = np.zeros_like(psi)
    # bounded per-step sample: whole time slices, sized so K+W steps take ~2 min
    t0 = time.perf_counter()
    oracle.mhat_slab(DIMS, U, A, Ai, KAPPA, psi, 0, 1, out)
    one = time.perf_counter() - t0
    per_step = max(1, min(DIMS[3], int(120.0 / max(1, args.steps + args.warmup) / max(one, 1e-3))))
    for w in range(args.warmup):
        t = (w * per_step) % DIMS[3]
        oracle.mhat_slab(DIMS, U, A, Ai, KAPPA, psi, t, min(DIMS[3], t + per_step), out)
    t0 = time.perf_counter()
    for k in range(args.steps):
        t = (k * per_step) % DIMS[3]
        oracle.mhat_slab(DIMS, U, A, Ai, KAPPA, psi, t, min(DIMS[3], t + per_step), out)
    dt = time.perf_counter() - t0
    sites = args.steps * per_step * DIMS[0] * DIMS[1] * DIMS[2] // 2
    gbs = sites * mhat_bytes("f32", 12) / dt / 1e9
    sample = (f"oracle Mhat (FP64, full 4x4 spin matrices, 12x12 clover) on {per_step} of {DIMS[3]} time slices "
              f"per step of the 32^3x64 workload; GB/s counts the workload's FP32 12-real compulsory bytes "
              f"({mhat_bytes('f32', 12)} B per output site)")
    line = {
        "impl": "reference", "metric": METRIC, "value": gbs, "unit": "GB/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": bench_config(args.gpus),
        "cpu_baseline": {"value": gbs, "unit": "GB/s", "cores": cpu_cores(), "kind": "oracle", "sample": sample,
                         "sites_per_s": sites / dt},
        "e2e": {"value": gbs, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def time_ms(torch, fn, steps, stream):
    s = torch.cuda.Event(enable_timing=True)
    e = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    s.record(stream)
    for _ in range(steps):
        fn()
    e.record(stream)
    e.synchronize()
    return s.elapsed_time(e) / steps


def kernel_only(args):
    """A few launches of one kernel for an ncu capture."""
    import torch
    import gen
    import paper_2001_05706_gb300 as L
    dims = tuple(int(v) for v in args.lattice.split(","))
    torch.cuda.set_device(0)
    U = gen.gauge_field(dims, EPS, GAUGE_SEED)
    psi = gen.gaussian_spinor(dims, SRC_SEED)[0]
    P = L.PREC[args.prec]
    with L.Lattice(dims, stream=torch.cuda.current_stream()) as lat:
        lat.load_gauge(U.view(np.float64))
        lat.clover(KAPPA, CSW)
        ctx = lat.ctx
        fx = L.lqcd_field_create(ctx, P, L.LQCD_ODD, args.nrhs)
        fy = L.lqcd_field_create(ctx, P, L.LQCD_EVEN, args.nrhs)
        fz = L.lqcd_field_create(ctx, P, L.LQCD_ODD, args.nrhs)
        L.lqcd_field_import(ctx, fx, np.ascontiguousarray(np.broadcast_to(psi, (args.nrhs,) + psi.shape)))
        L.lqcd_apply(ctx, L.LQCD_OP_K2A, args.recon, fy, fx)
        L.lqcd_synchronize(ctx)
        for _ in range(args.warmup + args.steps):
            if args.kernel_only in ("k2a", "mhat"):
                L.lqcd_apply(ctx, L.LQCD_OP_K2A, args.recon, fy, fx)
            if args.kernel_only in ("k2b", "mhat"):
                L.lqcd_apply_schur(ctx, args.recon, 0, fz, fx, fy)
        L.lqcd_synchronize(ctx)
        for f in (fx, fy, fz):
            L.lqcd_field_destroy(f)
    print(json.dumps({"kernel_only": args.kernel_only, "lattice": list(dims), "launches": args.steps + args.warmup}))
    return 0


def solver_iteration(args):
    """One inner iteration of each solver on the benchmark lattice, run
    eagerly (max_iter = 1 stops before the graph-captured loop), twice: the
    first pass fills the autotuner, the second shows one iteration's kernels
    in a launch list.  CGLS and BiCGStab with the 12 point sources, CGLS on
    one Gaussian RHS in both Schur forms; FP16 inner, DF64 updates."""
    import torch
    import gen
    import paper_2001_05706_gb300 as L
    torch.cuda.set_device(0)
    U = gen.gauge_field(DIMS, EPS, GAUGE_SEED)
    b12 = torch.from_numpy(gen.point_sources(DIMS).view(np.float64).reshape(-1).copy()).cuda()
    b1 = torch.from_numpy(gen.gaussian_spinor(DIMS, 2003)[0].view(np.float64).reshape(-1).copy()).cuda()
    out = []
    with L.Lattice(DIMS, stream=torch.cuda.current_stream()) as lat:
        lat.load_gauge(U.view(np.float64))
        lat.clover(KAPPA, CSW)
        for rep in range(2):
            for tag, b, n, solver, schur in (("cgls_12rhs", b12, 12, "cgls", "asym"),
                                             ("bicgstab_12rhs", b12, 12, "bicgstab", "asym"),
                                             ("cgls_1rhs", b1, 1, "cgls", "asym"), ("cgls_1rhs_sym", b1, 1, "cgls", "sym")):
                prm = L.solve_params(tol=1e-10, max_iter=1, inner=L.LQCD_F16, outer=L.LQCD_DF64, nrhs=n, recon=18,
                                     inner_recon=12, check_every=1, solver=solver, schur=schur)
                st, info = L.lqcd_solve(lat.ctx, torch.zeros_like(b), b, prm, raise_on_noconv=False)
                out.append({"pass": rep, "solve": tag, "iters": info.iters})
    print(json.dumps({"solver_iteration": out}))
    return 0


SOLVE_SET = ("fp64", "mixed_f32", "mixed_f16", "mixed_bf16", "df64", "mixed_f16_df64", "bicgstab_fp64",
             "bicgstab_mixed_f16", "bicgstab_mixed_f16_df64", "gcr_mixed_f16", "mixed_f16_r8")


def run_solves(L, torch, lat, U, rank, want_oracle, oracle_AAi, dims=None, which=SOLVE_SET, src_seed=2003):
    """FP64 CG vs mixed precision on one lattice, one Gaussian RHS."""
    import gen
    dims = tuple(dims or DIMS)
    b = gen.gaussian_spinor(dims, src_seed)[0]
    bt = torch.from_numpy(b.view(np.float64).copy()).cuda()
    res = {"lattice": list(dims), "kappa": KAPPA, "c_sw": CSW, "tol": 1e-10, "source": f"Gaussian, seed {src_seed}"}
    xs = {}
    cg, bi, gc = L.LQCD_SOLVER_CGLS, L.LQCD_SOLVER_BICGSTAB, L.LQCD_SOLVER_GCR
    for name, inner, outer, solver in (
            ("fp64", L.LQCD_F64, L.LQCD_F64, cg), ("mixed_f32", L.LQCD_F32, L.LQCD_F64, cg),
            ("mixed_f16", L.LQCD_F16, L.LQCD_F64, cg), ("mixed_bf16", L.LQCD_BF16, L.LQCD_F64, cg),
            ("df64", L.LQCD_DF64, L.LQCD_DF64, cg), ("mixed_f16_df64", L.LQCD_F16, L.LQCD_DF64, cg),
            ("bicgstab_fp64", L.LQCD_F64, L.LQCD_F64, bi), ("bicgstab_mixed_f16", L.LQCD_F16, L.LQCD_F64, bi),
            ("bicgstab_mixed_f16_df64", L.LQCD_F16, L.LQCD_DF64, bi), ("gcr_mixed_f16", L.LQCD_F16, L.LQCD_F64, gc),
            ("mixed_f16_r8", L.LQCD_F16, L.LQCD_F64, cg)):
        if name not in which:
            continue
        xt = torch.zeros_like(bt)
        prm = L.solve_params(tol=1e-10, max_iter=40000 if solver == cg else 4000, inner=inner, delta=0.1, recon=18,
                             inner_recon=8 if name.endswith("_r8") else 12, check_every=0, outer=outer,
                             solver=solver, gcr_nkrylov=8)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st, info = L.lqcd_solve(lat.ctx, xt, bt, prm, raise_on_noconv=False)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        res[name] = {"seconds": wall, "iters": info.iters, "reliable_updates": info.reliable_updates,
                     "mhat_applies": info.mhat_applies, "true_resid_gpu_fp64": info.true_resid[0],
                     "status": "ok" if st == L.LQCD_OK else L.lqcd_last_error()}
        xs[name] = xt.cpu().numpy().view(np.complex128).reshape(b.shape)
    # the headline pair: FP64 reliable updates against the FP64 CG
    best = min((k for k in ("mixed_f32", "mixed_f16", "mixed_bf16") if k in res and res[k]["status"] == "ok"),
               key=lambda k: res[k]["seconds"], default=None)
    if best and res["fp64"]["status"] == "ok":
        res["best_mixed"] = best
        res["speedup_vs_fp64"] = res["fp64"]["seconds"] / res[best]["seconds"]
    if "df64" in res and res["df64"]["status"] == "ok" and res["fp64"]["status"] == "ok":
        res["df64_cg_speedup_vs_fp64_cg"] = res["fp64"]["seconds"] / res["df64"]["seconds"]
    ok = [k for k in res if isinstance(res[k], dict) and res[k].get("status") == "ok" and k != "fp64"]
    if ok and res["fp64"]["status"] == "ok":
        fastest = min(ok, key=lambda k: res[k]["seconds"])
        res["fastest"] = fastest
        res["fastest_speedup_vs_fp64_cg"] = res["fp64"]["seconds"] / res[fastest]["seconds"]
    if want_oracle and oracle_AAi is not None:
        import oracle
        A = oracle_AAi[0]
        for name, x in xs.items():
            res[name]["true_resid_oracle"] = oracle.true_residual(dims, U, A, KAPPA, x, b)
    return res


def headline(res):
    """FP64 CGLS against the best mixed CGLS (FP64 updates) and the fastest
    solve of any kind, with the oracle's residuals of those solves."""
    if not res or res.get("fp64", {}).get("status") != "ok":
        return None
    h = {"lattice": res["lattice"], "fp64_cgls_s": res["fp64"]["seconds"]}
    for key, name in (("best_mixed", res.get("best_mixed")), ("fastest", res.get("fastest"))):
        if name:
            h[key] = name
            h[key + "_s"] = res[name]["seconds"]
            h[key + "_speedup_vs_fp64_cgls"] = res["fp64"]["seconds"] / res[name]["seconds"]
    ok = [k for k in res if isinstance(res[k], dict) and "true_resid_oracle" in res[k]]
    if ok:
        h["max_true_resid_oracle"] = max(res[k]["true_resid_oracle"] for k in ok)
        h["oracle_checked_solves"] = len(ok)
    return h


def run_config3(L, torch, stream, want_oracle):
    """Config 3: 48^3x96 (10.6 M sites), eps 0.2, c_sw 1.0, kappa 0.125, one
    Gaussian RHS: plain FP64 CGLS against mixed FP16 CGLS (FP64 updates, and
    DF64 updates) and mixed FP16 BiCGStab with DF64 updates, each to an
    oracle-recomputed true residual of 1e-10."""
    import gen
    dims = (48, 48, 48, 96)
    U = gen.gauge_field(dims, EPS, 1003)
    AAi = None
    if want_oracle:
        import oracle
        A = oracle.clover(dims, U, KAPPA, CSW)
        AAi = (A, None)
    with L.Lattice(dims, stream=stream) as lat:
        lat.load_gauge(U.view(np.float64))
        lat.clover(KAPPA, CSW)
        return run_solves(L, torch, lat, U, 0, want_oracle, AAi, dims=dims,
                          which=("fp64", "mixed_f16", "mixed_f16_df64", "bicgstab_mixed_f16_df64"), src_seed=2003)


def run_multi_rhs(L, torch, lat, U, want_oracle, oracle_AAi):
    """Config 4 (i): the 12 spin-colour point sources on the benchmark lattice,
    mixed precision (FP16 inner), one multi-RHS solve: CGLS with FP64 updates
    (the headline configuration), CGLS with DF64 updates, BiCGStab with DF64
    updates."""
    import gen
    b = gen.point_sources(DIMS)
    bt = torch.from_numpy(b.view(np.float64).reshape(-1).copy()).cuda()
    res = {"rhs": "12 point sources at the origin", "inner": "f16",
           "tuning": "autotuner warmed by an untimed one-iteration solve per outer precision"}
    # the first launch of each (precision, mode, nrhs, volume) times every
    # RHS-per-thread choice; a one-iteration solve does that outside the timed region
    for outer in (L.LQCD_F64, L.LQCD_DF64):
        prm = L.solve_params(tol=1e-10, max_iter=1, inner=L.LQCD_F16, delta=0.1, nrhs=12, recon=18, inner_recon=12,
                             check_every=0, outer=outer)
        L.lqcd_solve(lat.ctx, torch.zeros_like(bt), bt, prm, raise_on_noconv=False)
    for name, outer, solver in (("cgls", L.LQCD_F64, L.LQCD_SOLVER_CGLS),
                                ("cgls_df64_updates", L.LQCD_DF64, L.LQCD_SOLVER_CGLS),
                                ("bicgstab_df64_updates", L.LQCD_DF64, L.LQCD_SOLVER_BICGSTAB)):
        xt = torch.zeros_like(bt)
        prm = L.solve_params(tol=1e-10, max_iter=40000, inner=L.LQCD_F16, delta=0.1, nrhs=12, recon=18,
                             inner_recon=12, check_every=0, outer=outer, solver=solver)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st, info = L.lqcd_solve(lat.ctx, xt, bt, prm, raise_on_noconv=False)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        r = {"seconds": wall, "iters": info.iters, "reliable_updates": info.reliable_updates,
             "mhat_applies": info.mhat_applies, "max_true_resid_gpu_fp64": max(info.true_resid[:12]),
             "status": "ok" if st == L.LQCD_OK else L.lqcd_last_error()}
        if want_oracle and oracle_AAi is not None:
            import oracle
            x = xt.cpu().numpy().view(np.complex128).reshape(b.shape)
            rr = [oracle.true_residual(DIMS, U, oracle_AAi[0], KAPPA, x[k], b[k]) for k in range(12)]
            r["true_resid_oracle"] = rr
            r["max_true_resid_oracle"] = max(rr)
        if name == "cgls":
            res.update(r)
        else:
            res[name] = r
    return res


def run_schur_rough(L, torch, stream, want_oracle):
    """Asymmetric (Mhat) against symmetric (A_oo^-1 Mhat) Schur complement on a
    rough 32^3x64 field: eps 0.45 (mean plaquette ~0.59, as a quenched beta = 6
    ensemble), c_sw 1.77, kappa 0.13, one Gaussian RHS to 1e-10."""
    import gen
    eps, kappa, csw = 0.45, 0.13, 1.77
    U = gen.gauge_field(DIMS, eps, GAUGE_SEED)
    b = gen.gaussian_spinor(DIMS, 2003)[0]
    bt = torch.from_numpy(b.view(np.float64).copy()).cuda()
    res = {"lattice": list(DIMS), "eps": eps, "kappa": kappa, "c_sw": csw, "tol": 1e-10}
    cg, bi = L.LQCD_SOLVER_CGLS, L.LQCD_SOLVER_BICGSTAB
    xs = {}
    with L.Lattice(DIMS, stream=stream) as lat:
        lat.load_gauge(U.view(np.float64))
        lat.clover(kappa, csw)
        for name, inner, outer, solver, schur in (
                ("fp64_asym", L.LQCD_F64, L.LQCD_F64, cg, "asym"), ("fp64_sym", L.LQCD_F64, L.LQCD_F64, cg, "sym"),
                ("mixed_f16_asym", L.LQCD_F16, L.LQCD_F64, cg, "asym"),
                ("mixed_f16_sym", L.LQCD_F16, L.LQCD_F64, cg, "sym"),
                ("bicgstab_mixed_f16_df64_asym", L.LQCD_F16, L.LQCD_DF64, bi, "asym"),
                ("bicgstab_mixed_f16_df64_sym", L.LQCD_F16, L.LQCD_DF64, bi, "sym")):
            xt = torch.zeros_like(bt)
            prm = L.solve_params(tol=1e-10, max_iter=40000 if solver == cg else 8000, inner=inner, delta=0.1,
                                 recon=18, inner_recon=12, check_every=0, outer=outer, solver=solver, schur=schur)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st, info = L.lqcd_solve(lat.ctx, xt, bt, prm, raise_on_noconv=False)
            torch.cuda.synchronize()
            res[name] = {"seconds": time.perf_counter() - t0, "iters": info.iters,
                         "reliable_updates": info.reliable_updates, "mhat_applies": info.mhat_applies,
                         "true_resid_gpu_fp64": info.true_resid[0],
                         "status": "ok" if st == L.LQCD_OK else L.lqcd_last_error()}
            xs[name] = xt.cpu().numpy().view(np.complex128).reshape(b.shape)
    for pre in ("fp64", "mixed_f16", "bicgstab_mixed_f16_df64"):
        a, y = res[pre + "_asym"], res[pre + "_sym"]
        if a["status"] == "ok" and y["status"] == "ok":
            res[pre + "_sym_speedup"] = a["seconds"] / y["seconds"]
    if want_oracle:
        import oracle
        A = oracle.clover(DIMS, U, kappa, csw)
        for name, x in xs.items():
            res[name]["true_resid_oracle"] = oracle.true_residual(DIMS, U, A, kappa, x, b)
    return res


def run_batch(L, torch, stream, want_oracle):
    """Config 4 (ii): 24 lattices of uneven volume (8 each of 16^3x32, 20^3x40,
    24^3x48; eps 0.2, kappa 0.125, c_sw 1.0), 4 Gaussian RHS each, mixed
    precision, one graph-captured batched solve; every one of the 96 solutions
    is checked by the oracle's full-lattice true residual."""
    import gen
    shapes = [(16, 16, 16, 32)] * 8 + [(20, 20, 20, 40)] * 8 + [(24, 24, 24, 48)] * 8
    lats, bs, xs, Us, bh = [], [], [], [], []
    for j, d in enumerate(shapes):
        U = gen.gauge_field(d, EPS, 3000 + j)
        lat = L.Lattice(d, stream=stream)
        lat.load_gauge(U.view(np.float64))
        lat.clover(KAPPA, CSW)
        lats.append(lat)
        bnp = gen.gaussian_spinor(d, 4000 + j, nrhs=4)
        b = torch.from_numpy(bnp.view(np.float64).reshape(-1).copy()).cuda()
        bs.append(b)
        xs.append(torch.zeros_like(b))
        Us.append(U)
        bh.append(bnp)
    sites = sum(int(np.prod(d)) for d in shapes)
    res = {"lattices": "8 x 16^3x32 + 8 x 20^3x40 + 8 x 24^3x48", "sites": sites, "rhs_per_lattice": 4,
           "inner": "f16", "tuning": "autotuner warmed by an untimed one-iteration batch per outer precision"}
    for outer in (L.LQCD_F64, L.LQCD_DF64):
        prm = L.solve_params(tol=1e-10, max_iter=1, inner=L.LQCD_F16, delta=0.1, nrhs=4, recon=18, inner_recon=12,
                             check_every=0, outer=outer)
        L.lqcd_solve_batch([l.ctx for l in lats], [torch.zeros_like(b) for b in bs], bs, prm, raise_on_noconv=False)
    sols = {}
    for name, outer in (("fp64_updates", L.LQCD_F64), ("df64_updates", L.LQCD_DF64)):
        for x in xs:
            x.zero_()
        prm = L.solve_params(tol=1e-10, max_iter=40000, inner=L.LQCD_F16, delta=0.1, nrhs=4, recon=18,
                             inner_recon=12, check_every=0, outer=outer)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st, infos = L.lqcd_solve_batch([l.ctx for l in lats], xs, bs, prm, raise_on_noconv=False)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        r = {"seconds": wall, "max_iters": max(i.iters for i in infos),
             "max_true_resid_gpu_fp64": max(max(i.true_resid[:4]) for i in infos),
             "status": "ok" if st == L.LQCD_OK else L.lqcd_last_error()}
        sols[name] = [x.cpu().numpy().view(np.complex128).reshape(b.shape) for x, b in zip(xs, bh)]
        if name == "fp64_updates":
            res.update(r)
        else:
            res[name] = r
    for lat in lats:
        lat.close()
    if want_oracle:
        import oracle
        worst = {k: 0.0 for k in sols}
        n = 0
        for j, d in enumerate(shapes):
            A = oracle.clover(d, Us[j], KAPPA, CSW)
            for k in range(4):
                n += 1
                for name in sols:
                    r = oracle.true_residual(d, Us[j], A, KAPPA, sols[name][j][k], bh[j][k])
                    worst[name] = max(worst[name], r)
        res["max_true_resid_oracle"] = worst["fp64_updates"]
        res["df64_updates"]["max_true_resid_oracle"] = worst["df64_updates"]
        res["oracle_checked_rhs"] = n
    return res


def mrhs_mhat(L, torch, ctx, psi, stream, steps):
    """The many-right-hand-side Schur complement: 12 RHS against one, per
    storage precision (autotuned kernel variant), with the per-RHS compulsory
    bytes (links and clover read once for all right-hand sides)."""
    out = {}
    Vh = int(np.prod(DIMS)) // 2
    for prec in ("f16", "bf16", "f32"):
        P = L.PREC[prec]
        r = {}
        for n in (1, 12):
            fx = L.lqcd_field_create(ctx, P, L.LQCD_ODD, n)
            fy = L.lqcd_field_create(ctx, P, L.LQCD_EVEN, n)
            fz = L.lqcd_field_create(ctx, P, L.LQCD_ODD, n)
            L.lqcd_field_import(ctx, fx, np.ascontiguousarray(np.broadcast_to(psi, (n,) + psi.shape)))
            f = lambda: L.lqcd_apply(ctx, L.LQCD_OP_MHAT, 12, fz, fx)
            for _ in range(5):
                f()
            ms = time_ms(torch, f, max(10, steps // (4 * n)), stream)
            for g in (fx, fy, fz):
                L.lqcd_field_destroy(g)
            bpr = mhat_bytes_per_rhs(prec, 12, n)
            r[f"nrhs{n}"] = {"ms": ms, "ms_per_rhs": ms / n, "bytes_per_site_rhs": bpr,
                             "GBps": n * Vh * bpr / (ms * 1e-3) / 1e9}
        r["speedup_per_rhs"] = r["nrhs1"]["ms"] / r["nrhs12"]["ms_per_rhs"]
        out[prec] = r
    return out


def run_solve_only(args):
    """Mixed vs FP64 solve comparison on another lattice (config 3: 48^3x96)."""
    global DIMS
    import torch
    import gen
    import paper_2001_05706_gb300 as L
    torch.cuda.set_device(0)
    DIMS = tuple(int(v) for v in args.solve_lattice.split(","))
    U = gen.gauge_field(DIMS, EPS, GAUGE_SEED)
    oracle_AAi = None if args.no_cpu_baseline else oracle_setup(U)
    with L.Lattice(DIMS, stream=torch.cuda.current_stream()) as lat:
        lat.load_gauge(U.view(np.float64))
        lat.clover(KAPPA, CSW)
        res = run_solves(L, torch, lat, U, 0, oracle_AAi is not None, oracle_AAi)
    print(json.dumps({"metric": "mixed vs FP64 solve time to 1e-10", "config": {
        "workload": f"Wilson-clover even-odd CG, {'x'.join(map(str, DIMS))}, c_sw=1.0, kappa=0.125, eps 0.2, "
                    f"one Gaussian RHS"}, "solve": res}))
    return 0


def overlap_workload(L, torch, high, eig, want_oracle, stream):
    """Config 5: overlap operator on 16^3x32 (eps 0.1, rho 1.5, m 0.05), 20
    exact low modes, Chebyshev sign to 1e-10, 12 RHS, mixed-precision CG; the
    low modes and every right-hand side's true residual checked by the oracle
    (its own FP64 sign function, with the returned modes and interval)."""
    import gen
    dims = (16, 16, 16, 32)
    U = gen.gauge_field(dims, 0.1, 1005)
    b = gen.gaussian_spinor(dims, 2005, nrhs=12)
    out = {"high": high, "eig_method": eig, "config": {
        "workload": "overlap D_ov(m) = rho[1 + g5 sign(H_W)] + ..., 16^3x32, eps 0.1, rho 1.5, m 0.05, 20 low modes, "
                    "sign to 1e-10 (FP32 sign inside the CG to 1e-6), 12 Gaussian RHS, CG on the normal "
                    "equations with FP64 (or DF64) reliable updates every two decades (delta 0.01)"}}
    with L.Lattice(dims, stream=stream) as lat:
        lat.load_gauge(U.view(np.float64))
        prm = L.overlap_params(rho=1.5, mass=0.05, n_low=20, sign_tol=1e-10, eig_tol=1e-10, max_filter=400,
                               high=high, eig_method=eig)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st, info = L.lqcd_overlap_setup(lat.ctx, prm, raise_on_noconv=False)
        torch.cuda.synchronize()
        out["setup"] = {"seconds": time.perf_counter() - t0, "status": "ok" if st == 0 else L.lqcd_last_error(),
                        "sweeps_or_restarts": info.sweeps, "hw_applications": info.hw_applies,
                        "degree": info.degree, "degree_inner_fp32": info.degree_inner,
                        "a": info.a, "b": info.b, "eig_tol": 1e-10,
                        "sign_error": info.sign_error, "max_eig_resid": max(info.resid[:20]),
                        "lambda_min_max": [min(abs(v) for v in info.lambda_[:20]),
                                           max(abs(v) for v in info.lambda_[:20])]}
        if st != 0:
            return out
        x = np.zeros_like(b)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        L.lqcd_overlap(lat.ctx, x, b, 12, L.LQCD_OV_APPLY)
        t_apply = time.perf_counter() - t0
        out["apply_fp64_12rhs"] = {"seconds": t_apply, "hw_applications": 2 * info.degree + 1,
                                   "wilson_rhs_applications_per_s": 12 * (2 * info.degree + 1) / t_apply}
        # delta 0.01: the inner FP32 sign function is good to ~1e-6, so an update per
        # two decades costs fewer FP64/DF64 sign functions than one per decade
        cg = L.solve_params(tol=1e-10, max_iter=4000, nrhs=12, inner=L.LQCD_F32, delta=0.01)
        t0 = time.perf_counter()
        st, si = L.lqcd_overlap(lat.ctx, x, b, 12, L.LQCD_OV_SOLVE, cg, raise_on_noconv=False)
        out["solve_mixed_12rhs"] = {"seconds": time.perf_counter() - t0, "iters": si.iters,
                                    "reliable_updates": si.reliable_updates, "status": "ok" if st == 0 else
                                    L.lqcd_last_error(), "max_true_resid_gpu_fp64": max(si.true_resid[:12])}
        if want_oracle:
            import oracle
            vecs = np.zeros((20,) + oracle.spinor_shape(dims), dtype=np.complex128)
            L.lqcd_overlap_lowmodes(lat.ctx, vecs)
            lam = np.array(info.lambda_[:20])
            res, ortho = oracle.eigen_residuals(dims, U, 1.5, lam, vecs)
            out["oracle_eig_resid_max"] = float(res.max())
            out["oracle_eig_ortho"] = float(ortho)
            n, c = oracle.cheb_degree(info.a, info.b, 1e-10)
            rr = []
            for k in range(12):
                r = b[k] - oracle.apply_overlap(dims, U, 1.5, 0.05, x[k], info.a, info.b, c, lam=lam, vecs=vecs)
                rr.append(float(np.linalg.norm(r) / np.linalg.norm(b[k])))
            out["oracle_true_resid"] = rr
            out["max_true_resid_oracle"] = max(rr)
    return out


def overlap_eigen_workload(L, torch, dims, n_ev, want_oracle, stream, nrhs=2, basis=0, hw_eig_tol=1e-10,
                           max_filter=400):
    """The overlap eigensystem (Sec. 4: 200 pairs on a 24^3x64 lattice; here a
    synthetic stand-in, eps 0.1, rho 1.5, m 0.01): the n_ev lowest eigenpairs
    of D_ov(0)^dag D_ov(0) in the + chirality sector (and their partners) by
    thick-restart Lanczos, then the plain and the deflated mixed-precision
    overlap CG on nrhs Gaussian sources.  The oracle recomputes three
    eigenvectors' residuals (lowest, middle, highest) with its own sign
    function on the returned low modes and interval, and every deflated
    solve's true residual."""
    import gen
    U = gen.gauge_field(dims, 0.1, 1009)
    b = gen.gaussian_spinor(dims, 2009, nrhs=nrhs)
    name = "x".join(str(d) for d in dims)
    out = {"config": {"workload": f"overlap eigensystem {name}, eps 0.1, rho 1.5, m 0.01, 20 H_W low modes to "
                                  f"{hw_eig_tol:g}, sign to 1e-10 (double-float), {n_ev} eigenpairs of D_ov^dag D_ov "
                                  f"in the + sector to 1e-8, then {nrhs} Gaussian RHS by the mixed overlap CG to "
                                  f"1e-10 plain and deflated"}}
    with L.Lattice(dims, stream=stream) as lat:
        lat.load_gauge(U.view(np.float64))
        prm = L.overlap_params(rho=1.5, mass=0.01, n_low=20, sign_tol=1e-10, eig_tol=hw_eig_tol,
                               max_filter=max_filter, high="df64", eig_method="lanczos")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st, oinfo = L.lqcd_overlap_setup(lat.ctx, prm, raise_on_noconv=False)
        out["setup_seconds"] = time.perf_counter() - t0
        if st != 0:
            out["status"] = L.lqcd_last_error()
            return out
        st, info = L.lqcd_overlap_eigen(lat.ctx, L.overlap_eigen_params(n_ev=n_ev, sector=1, tol=1e-8,
                                                                        basis=basis, max_restarts=400),
                                        raise_on_noconv=False)
        mu = np.array(info.mu[:n_ev])
        out["eigensystem"] = {"status": "ok" if st == 0 else L.lqcd_last_error(), "seconds": info.seconds,
                              "restarts": info.restarts, "sign_applications": info.sign_applies,
                              "pairs": n_ev, "partners": info.n_partners,
                              "mu_min_max": [float(mu.min()), float(mu.max())],
                              "lambda_min": [info.lambda_re[0], info.lambda_im[0]],
                              "max_resid_gpu": max(info.resid[:n_ev])}
        if st != 0:
            return out
        cg = L.solve_params(tol=1e-10, max_iter=8000, nrhs=nrhs, inner=L.LQCD_F32, delta=0.1)
        xs = {}
        for op, key in ((L.LQCD_OV_SOLVE, "solve_mixed"), (L.LQCD_OV_SOLVE_DEFLATED, "solve_mixed_deflated")):
            x = np.zeros_like(b)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st, si = L.lqcd_overlap(lat.ctx, x, b, nrhs, op, cg, raise_on_noconv=False)
            out[key] = {"seconds": time.perf_counter() - t0, "iters": si.iters,
                        "reliable_updates": si.reliable_updates, "status": "ok" if st == 0 else L.lqcd_last_error(),
                        "max_true_resid_gpu_fp64": max(si.true_resid[:nrhs])}
            xs[key] = x
        out["deflation_speedup"] = out["solve_mixed"]["seconds"] / out["solve_mixed_deflated"]["seconds"]
        if want_oracle:
            import oracle
            vecs = np.zeros((20,) + oracle.spinor_shape(dims), dtype=np.complex128)
            L.lqcd_overlap_lowmodes(lat.ctx, vecs)
            lam = np.array(oinfo.lambda_[:20])
            n, c = oracle.cheb_degree(oinfo.a, oinfo.b, 1e-10)
            chi = np.zeros((n_ev,) + oracle.spinor_shape(dims), dtype=np.complex128)
            L.lqcd_overlap_eigvecs(lat.ctx, chi)
            res = {}
            for i in sorted({0, n_ev // 2, n_ev - 1}):
                h = oracle.apply_sector_normal(dims, U, 1.5, 1, chi[i], oinfo.a, oinfo.b, c, lam=lam, vecs=vecs)
                res[i] = float(np.linalg.norm((h - mu[i] * chi[i]).ravel()))
            out["oracle_eig_resid_sampled"] = res
            rr = []
            for k in range(nrhs):
                x = xs["solve_mixed_deflated"][k]
                r = b[k] - oracle.apply_overlap(dims, U, 1.5, 0.01, x, oinfo.a, oinfo.b, c, lam=lam, vecs=vecs)
                rr.append(float(np.linalg.norm(r) / np.linalg.norm(b[k])))
            out["oracle_true_resid_deflated"] = rr
    return out


def run_ov_eigen(args):
    """The overlap eigensystem on its own (--ov-eigen L0,L1,L2,L3 --n-ev N)."""
    import torch
    import paper_2001_05706_gb300 as L
    torch.cuda.set_device(0)
    dims = tuple(int(v) for v in args.ov_eigen.split(","))
    out = {"metric": "overlap eigensystem and deflated overlap solve time"}
    out.update(overlap_eigen_workload(L, torch, dims, args.n_ev, not args.no_cpu_baseline,
                                      torch.cuda.current_stream(), basis=args.ev_basis, hw_eig_tol=args.hw_eig_tol,
                                      max_filter=args.max_filter))
    print(json.dumps(out))
    return 0


def run_overlap(args):
    """Config 5 on its own (--overlap), either low-mode method and precision."""
    import torch
    import paper_2001_05706_gb300 as L
    torch.cuda.set_device(0)
    out = {"metric": "overlap set-up and mixed-precision 12-RHS solve time to 1e-10"}
    out.update(overlap_workload(L, torch, args.high, args.eig, not args.no_cpu_baseline, torch.cuda.current_stream()))
    print(json.dumps(out))
    return 0


def multigrid_cpu_baseline(dims, U, kappa, csw, seconds=15.0):
    """The oracle's fine-level stencil application (the multigrid kernel with
    the largest share) timed on the host over a bounded number of
    applications; numpy's batched einsum runs on one core."""
    import gen
    from oracle import multigrid as omg
    st = omg.wilson_clover_stencil(dims, U, kappa, csw, 1)
    v = gen.gaussian_spinor(dims, 2012).reshape(st.V, 12)
    st.apply(v)
    reps, t0 = 0, time.perf_counter()
    while True:
        st.apply(v)
        reps += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    return {"value": reps / el, "unit": "fine-level stencil applications/s", "cores": 1, "kind": "oracle",
            "sample": f"{reps} applications of the {'x'.join(map(str, dims))} fine stencil (oracle/multigrid.py)"}


def run_multigrid(args):
    """The 3-level multigrid solve on its own (--multigrid L0,L1,L2,L3): the
    paper's aggregation layout, blocks (4,4,4,4) and then (2,2,2,2), with 24
    near-null vectors per level, against the library's FP64 and mixed CGLS
    on the same full-lattice system; the solution checked by the oracle."""
    import torch
    import gen
    import paper_2001_05706_gb300 as L
    from paper_2001_05706_gb300 import multigrid as gmg
    torch.cuda.set_device(0)
    dims = tuple(int(v) for v in args.multigrid.split(","))
    V = int(np.prod(dims))
    kappa, csw, eps, nv = 0.1285, 1.0, 0.3, 24
    blocks = [(4, 4, 4, 4), (2, 2, 2, 2)]
    U = gen.gauge_field(dims, eps, 1011)
    b = gen.gaussian_spinor(dims, 2011)
    cfg = {"workload": f"Wilson-clover M x = b on {'x'.join(map(str, dims))}, eps {eps}, kappa {kappa}, c_sw {csw}, "
                       f"Gaussian source, tol 1e-10; 3-level multigrid, blocks {blocks[0]} and {blocks[1]}, "
                       f"{nv} near-null vectors per level (30 GCR steps each), K-cycle (0 pre / 4 post MR, coarse "
                       "GCR to 0.25), outer flexible GCR(16)"}
    out = {"metric": "multigrid set-up and solve time to 1e-10", "config": cfg}
    with L.Lattice(dims, 1) as lat:
        lat.load_gauge(U.view(np.float64))
        lat.clover(kappa, csw)
        starts = []
        n, Vl = 12, V
        for k, blk in enumerate(blocks):
            starts.append(gen.gaussian(2 * nv * Vl * n, 2100 + k).view(np.complex128).reshape(nv, Vl, n))
            Vl, n = Vl // int(np.prod(blk)), 2 * nv
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = gmg.fine_stencil(lat)
        mg = gmg.Multigrid(st, blocks, starts, setup_iters=30)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        bd = torch.from_numpy(b.reshape(V, 12).copy()).to("cuda")
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        x, it, rel = mg.solve(bd, 1e-10, maxiter=300)
        torch.cuda.synchronize()
        t3 = time.perf_counter()
        xh = x.cpu().numpy().reshape(b.shape)
        out["multigrid"] = {"setup_seconds": t1 - t0, "solve_seconds": t3 - t2, "outer_iters": it,
                            "rel_resid_gpu": rel, "levels": [{"dims": list(op.dims), "n": op.n} for op in mg.ops]}
        # roofline of the stencil application at each level (CUDA events on the
        # launching stream): algorithmic bytes per site = 9 n^2 matrix entries
        # + n read + n written, 16 B each
        peak, _ = load_peaks()
        roof = []
        for op in mg.ops:
            v = op.new()
            w = op.new()
            for _ in range(3):
                op.apply(v, w)
            reps = 20
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            for _ in range(reps):
                op.apply(v, w)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            nbytes = op.V * (9 * op.n * op.n + 2 * op.n) * 16
            roof.append({"dims": list(op.dims), "n": op.n, "ms": ms, "bytes": nbytes, "gbs": nbytes / ms / 1e6,
                         "frac": nbytes / ms / 1e6 / peak, "l2_resident": nbytes < 120e6})
        out["multigrid"]["apply_roofline"] = roof
        if args.kernel_shares:
            # device time per kernel over a second set-up and solve, from
            # CUPTI activity records (torch.profiler): shares, not bench values
            from torch.profiler import ProfilerActivity, profile
            with profile(activities=[ProfilerActivity.CUDA]) as prof:
                mg2 = gmg.Multigrid(st, blocks, starts, setup_iters=30)
                mg2.solve(bd, 1e-10, maxiter=300)
                torch.cuda.synchronize()
            tot = {}
            for ev in prof.events():
                if getattr(ev.device_type, "name", "") == "CUDA":
                    name = ev.name.replace("(anonymous namespace)::", "").replace("lqcd::", "")
                    name = name.replace("void ", "").split("(")[0].split("<")[0]
                    c, t = tot.get(name, (0, 0.0))
                    tot[name] = (c + 1, t + ev.time_range.elapsed_us())
            all_us = sum(t for _, t in tot.values()) or 1.0
            out["kernel_shares"] = sorted(({"kernel": k, "launches": c, "total_ms": t / 1e3, "share": t / all_us}
                                           for k, (c, t) in tot.items()), key=lambda r: -r["total_ms"])
        for name, inner in (("cgls_fp64", "f64"), ("cgls_mixed_f16", "f16")):
            lat.solve(b, 1e-10, inner)  # warm the autotuner
            xs, stt, info = lat.solve(b, 1e-10, inner)
            out[name] = {"seconds": info.seconds, "iters": info.iters, "status": int(stt)}
    out["multigrid"]["apply_per_s"] = 1e3 / out["multigrid"]["apply_roofline"][0]["ms"]
    if not args.no_cpu_baseline:  # the oracle, after the timed regions: its check of the solution, its timing
        import oracle
        A = oracle.clover(dims, U, kappa, csw)
        out["multigrid"]["oracle_true_resid"] = oracle.true_residual(dims, U, A, kappa, xh, b)
        out["cpu_baseline"] = multigrid_cpu_baseline(dims, U, kappa, csw)
    print(json.dumps(out))
    return 0


def run_gpu(args, rank, world, local_rank):
    import torch
    import paper_2001_05706_gb300 as L
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    stream = torch.cuda.current_stream()
    U, psi = make_inputs()
    V = int(np.prod(DIMS))
    Vh = V // 2
    lat = L.Lattice(DIMS, stream=stream)
    lat.load_gauge(U.view(np.float64))
    lat.clover(KAPPA, CSW)
    ctx = lat.ctx

    def fields(prec):
        P = L.PREC[prec]
        fx = L.lqcd_field_create(ctx, P, L.LQCD_ODD, 1)
        fy = L.lqcd_field_create(ctx, P, L.LQCD_EVEN, 1)
        fz = L.lqcd_field_create(ctx, P, L.LQCD_ODD, 1)
        L.lqcd_field_import(ctx, fx, psi)
        return fx, fy, fz

    fx, fy, fz = fields("f32")
    mhat = lambda: L.lqcd_apply(ctx, L.LQCD_OP_MHAT, 12, fz, fx)
    for _ in range(args.warmup):
        mhat()
    torch.cuda.synchronize()
    clocks = ClockSampler(gpu_index(local_rank))
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ms = time_ms(torch, mhat, args.steps, stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
        ms = max_over_ranks(ms, dist, "cuda")
    # per-kernel launch durations (same stream, events around K launches)
    k2a_ms = time_ms(torch, lambda: L.lqcd_apply(ctx, L.LQCD_OP_K2A, 12, fy, fx), args.steps, stream)
    k2b_ms = time_ms(torch, lambda: L.lqcd_apply_schur(ctx, 12, 0, fz, fx, fy), args.steps, stream)
    clk = clocks.stop()
    for f in (fx, fy, fz):
        L.lqcd_field_destroy(f)

    peak, peak_src = load_peaks()
    gbs = weak_gbs(Vh * mhat_bytes("f32", 12), ms, world)
    k2a_gbs = Vh * site_bytes("f32", 12, "k2a") / (k2a_ms * 1e-3) / 1e9
    k2b_gbs = Vh * site_bytes("f32", 12, "k2b") / (k2b_ms * 1e-3) / 1e9
    dom = "k2b" if k2b_ms >= k2a_ms else "k2a"
    dom_ms, dom_gbs = (k2b_ms, k2b_gbs) if dom == "k2b" else (k2a_ms, k2a_gbs)
    traffic = profiled_traffic("dslash_f32_r12_mhat", dom)

    # precision / link-format variants of the full Mhat
    variants = {}
    vsteps = max(50, min(args.steps, 1000))
    for prec, recon in (("f64", 18), ("f64", 12), ("df64", 18), ("f32", 18), ("f32", 12), ("f16", 12), ("bf16", 12)):
        a, y, z = fields(prec)
        f = lambda: L.lqcd_apply(ctx, L.LQCD_OP_MHAT, recon, z, a)
        for _ in range(5):
            f()
        vms = time_ms(torch, f, vsteps if prec not in ("f64", "df64") else max(20, vsteps // 4), stream)
        for g in (a, y, z):
            L.lqcd_field_destroy(g)
        b_site = mhat_bytes(prec, recon)
        flops = (FLOPS["k2a"] + FLOPS["k2b"]) * Vh / (vms * 1e-3) / 1e12
        variants[f"{prec}_r{recon}"] = {"ms": vms, "GBps": Vh * b_site / (vms * 1e-3) / 1e9,
                                        "pct_hbm": 100 * Vh * b_site / (vms * 1e-3) / 1e9 / peak,
                                        "TFLOPs": flops, "bytes_per_site": b_site}

    # end to end through the C ABI with pinned host buffers
    hin = torch.from_numpy(psi.view(np.float64).copy()).pin_memory()
    hout = torch.empty_like(hin).pin_memory()
    e2e_steps = 5
    L.lqcd_dslash(ctx, hout, hin, 1, L.LQCD_OP_MHAT, L.LQCD_F32, 12)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        L.lqcd_dslash(ctx, hout, hin, 1, L.LQCD_OP_MHAT, L.LQCD_F32, 12)
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    if dist:
        e2e_s = max_over_ranks(e2e_s, dist, "cuda")
    nbytes = hin.numel() * 8
    e2e = {"value": world * Vh * mhat_bytes("f32", 12) / e2e_s / 1e9, "unit": "GB/s",
           "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes, "ms_per_step": e2e_s * 1e3,
           "path": "lqcd_dslash(op=MHAT, prec=F32, recon=12) on pinned host canonical FP64 arrays: H2D copy, "
                   "pack, K2a, K2b, unpack, D2H copy, pipelined over 32 time-slice chunks on three streams"}

    need_oracle = rank == 0 and world == 1 and not args.no_cpu_baseline
    oracle_AAi = oracle_setup(U) if need_oracle else None
    solve = None
    mrhs = None
    if world == 1:
        mrhs = mrhs_mhat(L, torch, ctx, psi, stream, args.steps)
    solve = None
    solve_head = None
    if not args.no_solve and world == 1:
        solve = run_solves(L, torch, lat, U, rank, need_oracle, oracle_AAi)
        solve["schur_forms_rough_field"] = run_schur_rough(L, torch, stream, need_oracle)
        solve_head = {"lattice_32x32x32x64": headline(solve)}
        if not args.no_config3:
            solve["lattice_48x48x48x96"] = run_config3(L, torch, stream, need_oracle)
            solve_head["lattice_48x48x48x96"] = headline(solve["lattice_48x48x48x96"])
    multi = None
    if not args.no_batch and world == 1:
        multi = {"point_sources_32x32x32x64": run_multi_rhs(L, torch, lat, U, need_oracle, oracle_AAi),
                 "batch_24_lattices": run_batch(L, torch, stream, need_oracle)}
    overlap = None
    if not args.no_overlap and world == 1:
        overlap = overlap_workload(L, torch, "df64", "lanczos", need_oracle, stream)
        overlap["eigensystem_12x12x12x24"] = overlap_eigen_workload(L, torch, (12, 12, 12, 24), 50, need_oracle,
                                                                    stream)
    cpu = None
    if need_oracle:
        rate, nsl, dt = oracle_slab_rate(U, oracle_AAi[0], oracle_AAi[1], psi)
        cpu = {"value": rate * mhat_bytes("f32", 12) / 1e9, "unit": "GB/s", "cores": cpu_cores(), "kind": "oracle",
               "sample": f"oracle Mhat (FP64) on {nsl} time slices (passes over the {DIMS[3]}) of the 32^3x64 workload "
                         f"({dt:.1f} s); GB/s counts the workload's {mhat_bytes('f32', 12)} compulsory bytes "
                         f"per output site", "sites_per_s": rate}
    lat.close()
    if dist:
        dist.destroy_process_group()
    if rank != 0:
        return 0
    line = {
        "metric": METRIC, "value": gbs, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": bench_config(world),
        "pct_of_peak": 100.0 * gbs / world / peak,
        # the literature's "no-reuse" convention (8 neighbour spinors read per site; K2a 1536 B,
        # K2b 1632 B for FP32 12-real) and the flop rate, for comparison with published tables
        "effective_no_reuse_GBps": Vh * (1536 + 1632) / (ms * 1e-3) / 1e9,
        "TFLOPs": Vh * (FLOPS["k2a"] + FLOPS["k2b"]) / (ms * 1e-3) / 1e12,
        "roofline": {"bound": "hbm", "achieved": dom_gbs, "peak": peak, "unit": "GB/s", "frac": dom_gbs / peak,
                     "traffic": traffic, "kernel": f"dslash_kernel {dom} (FP32, 12-real)",
                     "bytes_per_launch": Vh * site_bytes("f32", 12, dom), "ms_per_launch": dom_ms,
                     "traffic_over_compulsory": (traffic / (Vh * site_bytes("f32", 12, dom))) if traffic else None,
                     "peak_source": peak_src},
        "kernels": {"k2a_ms": k2a_ms, "k2a_GBps": k2a_gbs, "k2b_ms": k2b_ms, "k2b_GBps": k2b_gbs},
        "variants": variants,
        "e2e": e2e,
        "gpu_launches": 2 * args.steps,
        "clocks": clk,
        "cpu_baseline": cpu,
        "solve_headline": solve_head,
        "multi_rhs_mhat_32x32x32x64": mrhs,
        "solve": solve,
        "multi_rhs_and_batch": multi,
        "overlap_16x16x16x32": overlap,
    }
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--impl", default="lqcd", choices=["lqcd", "reference"])
    ap.add_argument("--no-solve", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-config3", action="store_true", help="skip the 48^3x96 solve comparison")
    ap.add_argument("--no-overlap", action="store_true", help="skip the overlap workload in the default run")
    ap.add_argument("--ov-eigen", default=None, help="run only the overlap eigensystem on lattice L0,L1,L2,L3")
    ap.add_argument("--n-ev", type=int, default=200, help="eigenpairs for --ov-eigen")
    ap.add_argument("--ev-basis", type=int, default=0, help="Lanczos basis for --ov-eigen (0: automatic)")
    ap.add_argument("--hw-eig-tol", type=float, default=1e-10, help="H_W low-mode tolerance for --ov-eigen")
    ap.add_argument("--max-filter", type=int, default=400, help="H_W low-mode restart cap for --ov-eigen")
    ap.add_argument("--overlap", action="store_true", help="run the overlap workload (16^3x32) instead")
    ap.add_argument("--multigrid", default=None, help="run only the multigrid solve on lattice L0,L1,L2,L3")
    ap.add_argument("--kernel-shares", action="store_true",
                    help="with --multigrid: device time per kernel of a second set-up and solve (CUPTI records)")
    ap.add_argument("--solve-lattice", default=None, help="run only the solve comparison on this lattice")
    ap.add_argument("--high", default="f64", choices=["f64", "df64"],
                    help="--overlap: arithmetic of the FP64 parts (FP64 or double-float)")
    ap.add_argument("--eig", default="lanczos", choices=["subspace", "lanczos"],
                    help="--overlap: low-mode solver (block subspace iteration or thick-restart Lanczos)")
    ap.add_argument("--kernel-only", choices=["k2a", "k2b", "mhat"])
    ap.add_argument("--lattice", default="32,32,32,64")
    ap.add_argument("--prec", default="f32")
    ap.add_argument("--recon", type=int, default=12)
    ap.add_argument("--nrhs", type=int, default=1)
    ap.add_argument("--solver-iteration", action="store_true",
                    help="one eager inner iteration of each solver, twice (for a launch list)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank)
    if args.kernel_only:
        return kernel_only(args)
    if args.solver_iteration:
        return solver_iteration(args) if rank == 0 else 0
    if args.overlap:
        return run_overlap(args) if rank == 0 else 0
    if args.ov_eigen:
        return run_ov_eigen(args) if rank == 0 else 0
    if args.multigrid:
        return run_multigrid(args) if rank == 0 else 0
    if args.solve_lattice:
        return run_solve_only(args) if rank == 0 else 0
    return run_gpu(args, rank, world, local_rank)


if __name__ == "__main__":
    sys.exit(main())
