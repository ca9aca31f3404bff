#!/usr/bin/env python
"""Benchmark of the k.p hole eigensolve on one B300: converged eigenpairs/s
on the 160x48x48 FinFET-shaped grid (2.21M complex unknowns, plain FP64,
lowest 16 states, B = 0.5 T along [110], smooth strain), with the stencil's
roofline.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints ONE JSON line on rank 0.  One step = one cold-start eigensolve
(random start, fixed seed) through the C-ABI with every input resident in
HBM; the working set (four 849 MB blocks) is far larger than L2, so no L2
flush is needed between steps.  Under torchrun each rank solves its own
replica (the single-problem solve has no data-parallel split): weak scaling.

`--impl reference` times the FP64 CPU oracle (block Lanczos on the host
cores) on a bounded sample of the same workload: the same physics on a
cropped 32x12x12 box, its eigenpairs/s scaled by the unknowns ratio.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "converged k·p eigenpairs/s at 2.2M unknowns; stencil HBM GB/s vs peak"
UNIT = "eigenpairs/s"
WORKLOAD = ("c2: 160x48x48 grid h=0.5nm (2.21M unknowns), FP64, lowest 16 of block 24, degree 180, "
            "tol 1e-10 eV, coarse-grid start")
# filter degrees measured at C2 (B300): from the coarse-grid start plain
# FP64 is fastest at degree 180 (4 outer iterations; 120 takes 6) and the
# defect-corrected FP32 filter at 250 (3; 200 takes 4); from a random start
# 120 and 200; warm-started solves (SP loop, CI, sweeps) keep 200
SOLVE_KW = dict(n_states=16, block_m=24, degree=180, precision=0, tol=1e-10, seed=1, max_iter=600, start="coarse")
RANDOM_START_DEGREE = 120
MIXED_DEGREE = 250        # defect-corrected FP32 filter (precision 2), coarse-grid start
# SP loops: every solve after the first starts from the previous
# iteration's whole Ritz block (eigenvectors and guard columns); measured
# over 24 relaxed-occupation iterations at C2 (B300, s per SP iteration,
# identical iterates): coarse-grid start at 24 columns 0.683, at 28
# columns 0.562 (32: 0.685); block start at 28 columns degree 250 0.398,
# degree 160 0.391, degree 100 0.422; at 24 columns degree 160 0.516.
# The linear-mixing loop at 1.5 K oscillates (max |dV| ~1e-2 eV per
# iteration): there the previous block is a poor start (0.578 against
# 0.471 s per iteration from the coarse grid at 24 columns, degree 250)
SP_BLOCK_M = 28
SP_DEGREE = 160
MIXED_DEGREE_WARM = 200   # the same filter from warm or random starts
CROP = (32, 12, 12)
# DRAM bytes per point-vector of the FP64 fused stencil launch, from ncu
# (dram__bytes_read.sum + dram__bytes_write.sum = 2.463 GB + 0.829 GB over
# 24 x 368640 point-vectors, one ncu capture of a full-width FP64 filter
# launch at C2).  Valid for the kernel version profiled there; set to None
# when the kernel changes.
NCU_TRAFFIC_FP64_PER_PV = (2.463422464e9 + 0.829164544e9) / (24 * 368640)


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--e2e-steps", type=int, default=None,
                    help="end-to-end steps through host buffers (default: --steps)")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--sweep", type=int, default=0,
                    help="batched-sweep form: solve this many detuning points of the 64-point "
                         "sweep (uneven 96..160 x 40..48 x 40..48 grids, 12 states each) with "
                         "khp_eigensolve_batched in chunks, against sequential single solves")
    ap.add_argument("--sweep-chunk", type=int, default=8)
    ap.add_argument("--sweep-plain", type=int, default=4,
                    help="sweep points also solved in plain FP64 for the mixed-vs-plain speed-up")
    ap.add_argument("--profile", choices=["plain", "mixed", "dc", "poisson"], default=None,
                    help="one short C2 solve (6 outer iterations; 'poisson': one Poisson solve from zero on the "
                         "C2 grid with gates on the x faces) for profiler captures; prints its stats")
    ap.add_argument("--sweep-start", choices=["coarse", "random"], default="coarse",
                    help="start block of the sweep's solves (coarse-grid start or random)")
    ap.add_argument("--profile-start", choices=["random", "coarse"], default="random",
                    help="start block of the --profile solve (the timed solves use the coarse-grid start)")
    return ap.parse_args()


# ------------------------------------------------------------------ helpers
class Clocks:
    """nvidia-smi sampling (200 ms) during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None
        return self

    def __exit__(self, *exc):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()

    def summary(self):
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except OSError:
        return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0}, "fallback"


def _fp64_peak_tflops(torch):
    """FP64 peak of this GPU, measured: cuBLAS DGEMM 8192^3 (best of 5)."""
    a = torch.randn(8192, 8192, dtype=torch.float64, device="cuda")
    b = torch.randn(8192, 8192, dtype=torch.float64, device="cuda")
    for _ in range(2):
        torch.matmul(a, b)
    best = 1e30
    for _ in range(5):
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record()
        torch.matmul(a, b)
        e.record()
        e.synchronize()
        best = min(best, s.elapsed_time(e))
    del a, b
    return 2 * 8192 ** 3 / (best * 1e-3) / 1e12


# FP64 ALU issue rate of a B300 SM: 2 DFMA per clock (a DFMA-only probe on
# this GPU runs at 1.202 TFLOP/s at 2032 MHz = 148 SMs x 2 x 2 flop x clock;
# FP64 tensor instructions, mma.sync m8n8k4 f64, share these units: 1.05
# TFLOP/s alone, 1.07 mixed with DFMA)
FP64_DFMA_PER_CLOCK_SM = 2


def _fp64_alu_peak_tflops(torch, sm_mhz):
    """FP64 ALU peak from unit counts and the SM clock sampled in the run."""
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    return sms * FP64_DFMA_PER_CLOCK_SM * 2 * sm_mhz * 1e6 / 1e12


def _fp32_peak_tflops(torch):
    """FP32 (non-tensor) peak of this GPU, measured: cuBLAS SGEMM 8192^3 with
    TF32 off (best of 5)."""
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    a = torch.randn(8192, 8192, dtype=torch.float32, device="cuda")
    b = torch.randn(8192, 8192, dtype=torch.float32, device="cuda")
    for _ in range(2):
        torch.matmul(a, b)
    best = 1e30
    for _ in range(5):
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record()
        torch.matmul(a, b)
        e.record()
        e.synchronize()
        best = min(best, s.elapsed_time(e))
    del a, b
    torch.backends.cuda.matmul.allow_tf32 = prev
    return 2 * 8192 ** 3 / (best * 1e-3) / 1e12


def _crop(p, size=CROP):
    """The workload's physics on a bounded box of `size` points (cpu
    baseline sample), centred in the full grid."""
    nx, ny, nz = size
    x0, y0, z0 = (p.nx - nx) // 2, (p.ny - ny) // 2, (p.nz - nz) // 2
    sl = (slice(z0, z0 + nz), slice(y0, y0 + ny), slice(x0, x0 + nx))
    V = np.ascontiguousarray(p.V[sl])
    eps = None if p.strain is None else np.ascontiguousarray(p.strain[(slice(None),) + sl])
    return p.with_(nx=nx, ny=ny, nz=nz, V=V, strain=eps, name=p.name + "_crop")


def _oracle_solve(q, n):
    from oracle import eig, kp
    H = kp.assemble(q)
    t0 = time.perf_counter()
    w, v, res, cyc = eig.lowest_block_lanczos(H, n, tol=1e-10, return_residuals=True)
    return w, time.perf_counter() - t0


def _arpack_baseline(q, n, full_unknowns):
    """Second CPU baseline: SciPy eigsh (ARPACK, which='SA') on the oracle's
    CSR matrix of the same crop; the paper compares its solver with ARPACK."""
    from oracle import kp
    from scipy.sparse.linalg import eigsh
    H = kp.assemble(q).tocsr()
    t0 = time.perf_counter()
    eigsh(H, k=n, which="SA", tol=1e-10, return_eigenvectors=True)
    t = time.perf_counter() - t0
    scale = q.n_unknowns / full_unknowns
    return {"value": n / t * scale, "unit": UNIT, "cores": os.cpu_count(), "kind": "scipy eigsh (ARPACK)",
            "sample": (f"eigsh(k={n}, which='SA', tol=1e-10) on the oracle CSR of the {CROP[0]}x{CROP[1]}x"
                       f"{CROP[2]} crop: {t:.2f} s, scaled by the unknowns ratio {scale:.4g}")}


def _oracle_next_rows(p):
    """The oracle timed beside the NEXT rows, each on a stated crop
    (centred), unscaled: the H0 (block Lanczos, 16 states) and three SP
    iterations (dense eigensolver, direct Poisson) on the C2 physics; the
    two-hole CI (2 orbitals) and the g-tensors (dense, 7 assembled
    operators) on the double dot."""
    import inputs
    from oracle import ci as ci_o
    from oracle import eig, kp
    from oracle import gtensor as gt_o
    from oracle import poisson as po_o
    out = {}

    def gates(q):
        g = np.zeros((q.nz, q.ny, q.nx), dtype=np.uint8)
        g[:, :, 0] = 1
        g[:, :, -1] = 1
        return g

    q = _crop(p).with_(B=np.zeros(3))
    H = kp.assemble_h0(q)
    t0 = time.perf_counter()
    eig.lowest_block_lanczos(H, 16, tol=1e-10)
    out["h0"] = {"s": time.perf_counter() - t0, "sample": f"{CROP[0]}x{CROP[1]}x{CROP[2]} crop, "
                 f"{H.shape[0]} unknowns, 16 states, block Lanczos"}
    q = _crop(p, (10, 6, 6))
    t0 = time.perf_counter()
    po_o.sp_loop(q, q.V, gates(q), np.zeros_like(q.V), 8, 2.0, 1.5, 0.3, 3, bands=6)
    out["sp"] = {"s_per_iteration": (time.perf_counter() - t0) / 3,
                 "sample": f"10x6x6 crop, {q.n_unknowns} unknowns, 8 states, 2 holes, 3 iterations"}
    pdd = inputs.double_dot(p.nx, p.ny, p.nz, p.h)
    q = _crop(pdd, (14, 6, 6))
    t0 = time.perf_counter()
    ci_o.ci_pipeline(q, 2, gates(q))
    out["ci"] = {"s": time.perf_counter() - t0, "sample": "14x6x6 crop, 2 H0 orbitals, K = 6"}
    q = _crop(pdd, (12, 6, 6))
    t0 = time.perf_counter()
    gt_o.dqd_g_tensors(q)
    out["gtensor"] = {"s": time.perf_counter() - t0, "sample": f"12x6x6 crop, {q.n_unknowns} unknowns"}
    return out


def _cpu_baseline(p, n, full_unknowns):
    q = _crop(p)
    _, t = _oracle_solve(q, n)
    scale = q.n_unknowns / full_unknowns
    return {"value": n / t * scale, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": (f"FP64 oracle (CSR + thick-restart block Lanczos, tol 1e-10 eV) on the same physics "
                       f"cropped to {CROP[0]}x{CROP[1]}x{CROP[2]} ({q.n_unknowns} unknowns): {t:.2f} s for "
                       f"{n} eigenpairs, scaled by the unknowns ratio {scale:.4g} to the full grid; "
                       f"sparse matvec single-threaded, BLAS on all cores.  The linear scaling flatters "
                       f"the oracle: its iterations grow with the box as the levels crowd")}


# --------------------------------------------------------------- reference
def run_reference(args, rank):
    if rank != 0:
        return
    import inputs
    p = inputs.config2()
    n = SOLVE_KW["n_states"]
    q = _crop(p)
    for _ in range(args.warmup):
        _oracle_solve(q, n)
    ts = []
    for _ in range(args.steps):
        _, t = _oracle_solve(q, n)
        ts.append(t)
    T = sum(ts)
    scale = q.n_unknowns / p.n_unknowns
    value = n * args.steps / T * scale
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * T / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": f"cropped {CROP}", "l2": "inputs larger than L2 n/a (CPU)"},
            "impl": "reference",
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                             "sample": f"oracle block Lanczos on the workload cropped to {CROP}, "
                                       f"scaled by unknowns ratio {scale:.4g}"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------- ours
def run_ours(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist
    import inputs
    import paper_2607_08447_b300 as khp

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    p = inputs.config2()
    grid = khp.KPGrid.from_problem(p, device=dev)
    stream = grid.stream
    n = SOLVE_KW["n_states"]

    def barrier():
        if world > 1:
            dist.barrier()

    # warm-up
    for _ in range(args.warmup):
        r = grid.eigensolve(**SOLVE_KW)
    torch.cuda.synchronize()

    # timed region: K cold-start solves
    stats = []
    barrier()
    torch.cuda.synchronize()
    with Clocks(local_rank) as clk:
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(args.steps):
            r = grid.eigensolve(**SOLVE_KW)
            stats.append(r.stats)
        ev1.record(stream)
        torch.cuda.synchronize()
    barrier()
    ms = ev0.elapsed_time(ev1)
    clocks = clk.summary()
    t_all = torch.tensor([ms], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t_all, op=dist.ReduceOp.MAX)
    ms_max = float(t_all.item())
    conv = min(s["converged"] for s in stats)
    value = world * conv * args.steps / (ms_max * 1e-3)
    evals_plain = r.evals.copy()

    # warm start: the previous solve starts the solve for a potential
    # changed by 0.1 meV of smooth noise (one Schroedinger-Poisson update),
    # from its whole Ritz block (degree 180) and from its eigenvectors alone
    # (degree 120, the remaining columns random); the original fields are
    # restored afterwards
    lev = getattr(p, "levers", None)
    alpha0 = None if lev is None else np.zeros(lev.shape[0])
    blk = torch.empty((grid.N, SOLVE_KW["block_m"]), dtype=torch.complex128, device=dev)
    grid.eigensolve(**SOLVE_KW, block_out=blk)          # the unperturbed solve's block (untimed)
    dV = 1e-4 * inputs.smooth_noise(np.random.Generator(np.random.PCG64(99)), (p.nz, p.ny, p.nx))
    grid.set_fields(p.V + dV, p.strain, lev, alpha0, p.B, p.gauge)

    def timed_solve(kw, ws):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = grid.eigensolve(**kw, warm_start=ws)
        e1.record(stream)
        torch.cuda.synchronize()
        return out, e0.elapsed_time(e1)

    rw, ms_warm = timed_solve(dict(SOLVE_KW), blk)
    rwe, ms_warm_evecs = timed_solve(dict(SOLVE_KW, degree=RANDOM_START_DEGREE), r.evecs)
    del blk
    grid.set_fields(p.V, p.strain, lev, alpha0, p.B, p.gauge)

    # the same solve from a random start block (the coarse-grid start's gain)
    er0, er1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    er0.record(stream)
    rr = grid.eigensolve(**dict(SOLVE_KW, start="random", degree=RANDOM_START_DEGREE))
    er1.record(stream)
    torch.cuda.synchronize()
    ms_random = er0.elapsed_time(er1)

    peaks, peak_kind = _peaks()
    hbm = float(peaks["hbm_gbs"])
    fp64_dgemm = _fp64_peak_tflops(torch)
    sm_mhz = clocks.get("sm_mhz") or clocks.get("sm_max_mhz") or 2032.0
    fp64_peak = _fp64_alu_peak_tflops(torch, sm_mhz)
    fp32_peak = _fp32_peak_tflops(torch)

    # dominant kernel: the fused FP64 Chebyshev stencil.  Its device time is
    # taken from CUDA events the library records on this stream around every
    # filter (stencil launches only); point-vectors counted per launch.
    l64 = sum(s["launches_fp64"] for s in stats)
    ms64 = sum(s["ms_filter_fp64"] for s in stats)
    pv64 = sum(s["pv_fp64"] for s in stats)
    st0 = stats[0]
    t64 = ms64 / max(l64, 1)                          # ms per launch
    pv_launch = pv64 / max(l64, 1)                    # point-vectors per launch
    flops_launch = st0["flops_per_pv"] * pv_launch
    bytes_launch64 = st0["bytes_per_pv_fp64"] * pv_launch
    achieved_tf = flops_launch / (t64 * 1e-3) / 1e12
    roofline = {"bound": "alu", "kernel": "stencil_kernel<double> (fused Chebyshev step)",
                "achieved": achieved_tf, "peak": fp64_peak, "unit": "TFLOP/s",
                "frac": achieved_tf / fp64_peak,
                "traffic": (NCU_TRAFFIC_FP64_PER_PV * pv_launch if NCU_TRAFFIC_FP64_PER_PV else None),
                "traffic_note": "ncu DRAM bytes of a full-width launch scaled to this run's mean launch width",
                "peak_source": ("FP64 ALU from unit counts: SMs x 2 DFMA/clock x 2 flop x the SM clock "
                                "sampled in the timed region"),
                "dgemm_tflops": fp64_dgemm, "frac_of_dgemm": achieved_tf / fp64_dgemm,
                "frac_note": ("the stencil mixes DFMA (2 flop) with DADD/DMUL (1 flop) issues, so the "
                              "flop fraction sits below its FP64-pipe occupancy (88 % in ncu)"),
                "algorithmic_flops_per_launch": flops_launch, "ms_per_launch": t64,
                "point_vectors_per_launch": pv_launch,
                "hbm_gbs": bytes_launch64 / (t64 * 1e-3) / 1e9,
                "hbm_frac": bytes_launch64 / (t64 * 1e-3) / 1e9 / hbm,
                "share_of_step": ms64 / ms}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "grid": [p.nx, p.ny, p.nz], "unknowns": p.n_unknowns,
                       "n_states": n, "block_m": SOLVE_KW["block_m"], "degree": SOLVE_KW["degree"],
                       "tol_ev": SOLVE_KW["tol"], "start": SOLVE_KW["start"],
                       "start_ms": st0["ms_start"], "start_iterations": st0["start_iterations"],
                       "parallelism": f"replicas x{world}",
                       "l2": "inputs larger than L2 (4 x 849 MB blocks), no flush",
                       "iterations": st0["iterations"], "peaks": peak_kind}}
    # the steps around the eigensolve first (the driver keeps the end of
    # the line: the headline evidence goes last)
    line["h0"] = _h0_bench(p, dev, torch, khp)
    line["sp"] = _sp_bench(p, dev, torch, khp)
    # the CI and the g-tensors on the mirror-symmetric double dot of the
    # same grid, where t and J are a tunnel coupling and an exchange energy
    pdd = inputs.double_dot(p.nx, p.ny, p.nz, p.h)
    line["ci"] = _ci_bench(pdd, dev, torch, khp)
    line["gtensor"] = _gtensor_bench(pdd, dev, torch, khp, line["ci"].get("exchange_ev"))
    line["random_start"] = {"value": rr.stats["converged"] / (ms_random * 1e-3), "unit": UNIT,
                            "ms_per_solve": ms_random, "iterations": rr.stats["iterations"],
                            "max_abs_dE_vs_coarse_start_ev": float(np.abs(rr.evals - evals_plain).max()),
                            "degree": RANDOM_START_DEGREE,
                            "note": "the same solve from a random start block instead of the coarse-grid start, "
                                    "at the degree that is fastest from a random start"}
    line["warm"] = {"value": rw.stats["converged"] / (ms_warm * 1e-3), "unit": UNIT, "ms_per_solve": ms_warm,
                    "iterations": rw.stats["iterations"],
                    "note": "warm start from the previous solve's whole Ritz block (block_out), V changed by 0.1 meV "
                            "smooth noise",
                    "max_abs_dE_vs_evecs_start_ev": float(np.abs(rw.evals - rwe.evals).max()),
                    "evecs_only": {"value": rwe.stats["converged"] / (ms_warm_evecs * 1e-3), "unit": UNIT,
                                   "ms_per_solve": ms_warm_evecs, "iterations": rwe.stats["iterations"],
                                   "degree": RANDOM_START_DEGREE}}
    line["projections"] = _projections_bench(grid, p.n_unknowns, SOLVE_KW["block_m"], hbm, torch)
    step32 = _fp32_step_bench(grid, p, SOLVE_KW["block_m"], hbm, torch)

    # mixed precision to the same tolerance: every filter apply in FP32,
    # defect-corrected by the FP64 residual; FP64 H Y and Rayleigh-Ritz
    if not args.no_mixed:
        kw = dict(SOLVE_KW, precision=2, degree=MIXED_DEGREE)
        grid.eigensolve(**kw)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rm = grid.eigensolve(**kw)
        e1.record(stream)
        torch.cuda.synchronize()
        msm = e0.elapsed_time(e1)
        sm = rm.stats
        t32 = sm["ms_filter_fp32"] / max(sm["launches_fp32"], 1)
        pv32 = sm["pv_fp32"] / max(sm["launches_fp32"], 1)
        # defect-corrected steps also read the FP32 residual block (48 B/pv)
        b32 = (sm["bytes_per_pv_fp32"] + 48.0) * pv32
        line["mixed"] = {"value": rm.stats["converged"] / (msm * 1e-3), "unit": UNIT, "ms_per_solve": msm,
                         "speedup_vs_fp64": (rm.stats["converged"] / (msm * 1e-3)) / (value / world),
                         "max_abs_dE_vs_fp64_ev": float(np.abs(rm.evals - evals_plain).max()),
                         "iterations_fp32": sm["iterations_fp32"], "iterations": sm["iterations"],
                         "max_residual": sm["max_residual"], "precision": "fp32 filter (defect-corrected) + FP64-accurate Rayleigh-Ritz on the tensor cores",
                         "degree": MIXED_DEGREE,
                         "phase_ms": {"fp32_filter": sm["ms_filter_fp32"], "combine_and_fp64_HY": sm["ms_between"],
                                      "gram": sm["ms_gram"], "small_eig": sm["ms_small"], "rotation": sm["ms_rotate"]},
                         "residual_history_ev": [float(f"{x:.3g}") for x in sm["res_history"]]}
        line["stencil_fp32"] = {"bound": "hbm", "kernel": "stencil_plane_kernel (FP32, TMA-staged planes) defect-corrected step (reads Z_k, Z_k-1, R; writes Z_k+1)",
                                "achieved": b32 / (t32 * 1e-3) / 1e9, "peak": hbm,
                                "unit": "GB/s", "frac": b32 / (t32 * 1e-3) / 1e9 / hbm,
                                "frac_of_nominal_8tbs": b32 / (t32 * 1e-3) / 1e9 / 8000.0,
                                "ms_per_launch": t32, "algorithmic_bytes_per_launch": b32,
                                "tflops": sm["flops_per_pv"] * pv32 / (t32 * 1e-3) / 1e12,
                                "fp32_peak_tflops": fp32_peak,
                                "flop_frac": sm["flops_per_pv"] * pv32 / (t32 * 1e-3) / 1e12 / fp32_peak,
                                "fp32_peak_source": "cuBLAS SGEMM 8192^3, TF32 off, measured in this run"}


    # end to end through host buffers: H2D of V and strain, solve, D2H of
    # eigenvalues and eigenvectors, every step
    Vh = torch.from_numpy(p.V.reshape(-1)).pin_memory()
    Sh = torch.from_numpy(p.strain.reshape(-1)).pin_memory()
    Vd = torch.empty_like(Vh, device=dev)
    Sd = torch.empty_like(Sh, device=dev)
    out_h = torch.empty((p.n_unknowns, n), dtype=torch.complex128).pin_memory()
    e2e_steps = args.e2e_steps or args.steps
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        Vd.copy_(Vh, non_blocking=True)
        Sd.copy_(Sh, non_blocking=True)
        grid.set_fields(Vd, Sd, None, None, p.B, p.gauge)
        re = grid.eigensolve(**SOLVE_KW)
        out_h.copy_(re.evecs, non_blocking=True)
        torch.cuda.synchronize()
    te = time.perf_counter() - t0
    line["e2e"] = {"value": world * re.stats["converged"] * e2e_steps / te, "unit": UNIT, "steps": e2e_steps,
                   "h2d_bytes_per_step": int(Vh.numel() * 8 + Sh.numel() * 8),
                   "d2h_bytes_per_step": int(out_h.numel() * 16 + n * 8)}

    if rank == 0 and not args.no_cpu_baseline:
        for key, v in _oracle_next_rows(p).items():
            if key in line:
                line[key]["oracle_cpu"] = dict(v, cores=os.cpu_count(), kind="oracle")
        line["cpu_baseline_arpack"] = _arpack_baseline(_crop(p), n, p.n_unknowns)
        line["cpu_baseline"] = _cpu_baseline(p, n, p.n_unknowns)
    # headline evidence at the end of the line
    for key in ("mixed", "stencil_fp32"):
        if key in line:
            line[key] = line.pop(key)
    line["stencil_fp32_step"] = step32
    line["roofline"] = roofline
    line["clocks"] = clocks
    line["gpu_launches"] = int(sum(s["kernel_launches"] for s in stats))
    if rank == 0:
        print(json.dumps(line), flush=True)
    grid.close()


def _h0_bench(p, dev, torch, khp):
    """The spin-independent H0 (three bands, B = 0) on the same grid and
    fields: lowest 16 states, plain FP64 and defect-corrected FP32 filter,
    one cold solve each after one warm-up."""
    g = khp.KPGrid.from_problem(p, device=dev, bands=3)
    out = {"unknowns": 3 * p.n_points}
    for name, kw in (("fp64", dict(SOLVE_KW)), ("mixed", dict(SOLVE_KW, precision=2, degree=MIXED_DEGREE_WARM))):
        g.eigensolve(**kw)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(g.stream)
        r = g.eigensolve(**kw)
        e1.record(g.stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        out[name] = {"value": r.stats["converged"] / (ms * 1e-3), "unit": UNIT, "ms_per_solve": ms,
                     "iterations": r.stats["iterations"], "max_residual": r.stats["max_residual"]}
        if name == "fp64":
            e64 = r.evals
        else:
            out[name]["max_abs_dE_vs_fp64_ev"] = float(np.abs(r.evals - e64).max())
    g.close()
    return out


def _sp_bench(p, dev, torch, khp):
    """Schroedinger-Poisson loop on the C2 grid and fields: grounded gates on
    the two x faces, 2 holes at 1.5 K, linear mixing 0.3, defect-corrected
    solves from the coarse-grid start, up to 12 iterations or max |dV| <=
    1e-6 eV; then Anderson mixing at 20 K and the loop with relaxed
    occupations at 1.5 K, whose solves after the first start from the
    previous iteration's whole Ritz block."""
    from paper_2607_08447_b300.poisson import Poisson, sp_solve
    gate = np.zeros((p.nz, p.ny, p.nx), dtype=np.uint8)
    gate[:, :, 0] = 1
    gate[:, :, -1] = 1
    g = khp.KPGrid.from_problem(p, device=dev)
    P = Poisson(p.nx, p.ny, p.nz, p.h, gate, np.zeros_like(p.V), device=dev)
    kw_lin = dict(block_m=SOLVE_KW["block_m"], degree=MIXED_DEGREE, precision=2, tol=1e-10, seed=1, start="coarse")
    kw = dict(block_m=SP_BLOCK_M, degree=SP_DEGREE, precision=2, tol=1e-10, seed=1, start="coarse")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    r = sp_solve(g, P, p.V, SOLVE_KW["n_states"], 2.0, T=1.5, mix=0.3, iters=12, tol_v=1e-6, strain=p.strain,
                 B=p.B, gauge=p.gauge, solve_kw=kw_lin, warm=False)
    torch.cuda.synchronize()
    t = time.perf_counter() - t0
    # the Poisson solve alone, from zero, on the final density
    f = 0.5 * (1.0 - np.tanh(0.5 * (r.evals - r.mu) / (8.617333262e-5 * 1.5)))
    rho = g.density(r.evecs, f / p.h ** 3)
    phi = torch.zeros(p.n_points, dtype=torch.float64, device=dev)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    P.solve(rho, phi, tol=1e-10)
    torch.cuda.synchronize()
    tp = time.perf_counter() - t1
    cold_iterations = P.last_iterations
    # the same solve with the Jacobi preconditioner
    P.set_preconditioner("jacobi")
    phi.zero_()
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    P.solve(rho, phi, tol=1e-10)
    torch.cuda.synchronize()
    tj = time.perf_counter() - t1
    jacobi_iterations = P.last_iterations
    P.set_preconditioner("multigrid")
    out = {"iterations": len(r.history), "s_total": t, "s_per_iteration": t / len(r.history),
           "final_max_dV_ev": r.history[-1], "poisson_cg_iterations": r.poisson_iterations,
           "poisson_ms_cold": 1e3 * tp, "poisson_cold_iterations": cold_iterations,
           "poisson_multigrid_levels": P.mg_levels,
           "poisson_ms_cold_jacobi": 1e3 * tj, "poisson_cold_iterations_jacobi": jacobi_iterations,
           "workload": "C2 grid and fields, grounded gates on both x faces, 2 holes, T 1.5 K, mix 0.3",
           "solves": f"defect-corrected, {SOLVE_KW['block_m']} columns, degree {MIXED_DEGREE}, coarse-grid start; "
                     f"the runs below: {SP_BLOCK_M} columns, degree {SP_DEGREE}, coarse-grid start then the "
                     "previous iteration's Ritz block"}
    # Anderson mixing (library history, depth 6, damping 0.5) at 20 K, where
    # kT exceeds the splittings of the random wells and the density responds
    # smoothly to V; then the loop with relaxed occupations at 1.5 K, with
    # linear mixing 0.5 and with Anderson mixing (damping 0.8, depth 4)
    runs = (("anderson_20k", 20.0, dict(mix=0.5, anderson_depth=6)),
            ("relaxed_1p5k_linear", 1.5, dict(mix=0.5, relax=True)),
            ("relaxed_1p5k_anderson", 1.5, dict(mix=0.8, anderson_depth=4, relax=True)))
    for name, T, opt in runs:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ra = sp_solve(g, P, p.V, SOLVE_KW["n_states"], 2.0, T=T, iters=24, tol_v=1e-6, strain=p.strain,
                      B=p.B, gauge=p.gauge, solve_kw=kw, warm="block", **opt)
        torch.cuda.synchronize()
        out[name] = {"T_K": T, "iterations": len(ra.history), "s_total": time.perf_counter() - t0,
                     "converged": ra.history[-1] <= 1e-6,
                     "max_dV_last_ev": [float(f"{x:.3g}") for x in ra.history[-4:]]}
        if ra.occupations is not None:
            out[name]["occupations"] = [float(f"{x:.4g}") for x in ra.occupations[:6]]
    P.close()
    g.close()
    return out


def _ci_bench(p, dev, torch, khp):
    """Two-hole CI of the double dot on the 160x48x48 grid: the lowest 4
    orbitals of the spin-independent H0 (defect-corrected solve), 16
    Coulomb potentials (32 Poisson solves, grounded gates on both x faces),
    K = 28 determinants; J = E_T - E_S."""
    from paper_2607_08447_b300.ci import ci_exchange
    from paper_2607_08447_b300.poisson import Poisson
    gate = np.zeros((p.nz, p.ny, p.nx), dtype=np.uint8)
    gate[:, :, 0] = 1
    gate[:, :, -1] = 1
    g = khp.KPGrid.from_problem(p, device=dev, bands=3)
    P = Poisson(p.nx, p.ny, p.nz, p.h, gate, np.zeros_like(p.V), device=dev)
    # H0 solve from the coarse grid at 12 columns, degree 250; measured on
    # B300 (s per CI, the same J to 1e-12 eV): random start 16 columns
    # degree 200 0.206, 12 columns 0.168; coarse start 16 columns degree
    # 250 0.182, 160 0.204; 12 columns degree 250 0.149
    kw = dict(block_m=12, degree=MIXED_DEGREE, precision=2, tol=1e-10, seed=1, start="coarse")
    ci_exchange(g, P, 4, p.material["delta_so"], solve_kw=kw)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    r = ci_exchange(g, P, 4, p.material["delta_so"], solve_kw=kw)
    torch.cuda.synchronize()
    t = time.perf_counter() - t0
    out = {"s_total": t, "determinants": len(r.energies), "exchange_ev": r.exchange,
           "lowest_two_hole_ev": [float(x) for x in r.energies[:4]],
           "spin2_lowest4": [float(f"{x:.4g}") for x in r.spin2[:4]],
           "lowest4_spread_ev": float(r.energies[3] - r.energies[0]),
           "workload": "mirror-symmetric double dot (hw = 5 meV wells at 0.3 and 0.7 L_x) on the 160x48x48 "
                       "grid, device frame, no strain, B = 0; H0 lowest 4 orbitals, grounded gates on both x faces"}
    P.close()
    g.close()
    return out


def _gtensor_bench(p, dev, torch, khp, j_ci):
    """g-matrices of the bonding/anti-bonding doublets and the left/right
    g-tensors of the double dot on the 160x48x48 grid (B = 0): the 4-state
    defect-corrected solve, then the responses
    (6 operator applies at B = +-d e_j, 6 tensor-core projections) and the
    position moments.  Then the host maps of Eq. 17 on a 91 x 181 grid of
    field directions, with the CI's J and a stated spin-orbit rotation
    (theta_so = 0.2 about y: the paper takes it from experiment)."""
    from paper_2607_08447_b300 import exchange as ex
    from paper_2607_08447_b300.gtensor import g_tensors
    g = khp.KPGrid.from_problem(p, device=dev)
    # measured on B300 (s per call, the same t to 1e-17 eV): random start
    # degree 200 0.259; coarse start degree 250 0.231, degree 160 0.218
    kw = dict(block_m=12, degree=160, precision=2, tol=1e-10, seed=1, start="coarse")
    g_tensors(g, solve_kw=kw)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    r = g_tensors(g, solve_kw=kw)
    torch.cuda.synchronize()
    t_total = time.perf_counter() - t0
    g.set_B(np.zeros(3))
    st = g.eigensolve(4, **kw)
    g.set_B(p.B)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g_tensors(g, states=(st.evals, st.evecs))
    torch.cuda.synchronize()
    t_resp = time.perf_counter() - t0
    out = {"s_total": t_total, "s_response_and_moments": t_resp, "delta_ev": r.delta, "tunnel_ev": r.tunnel,
           "g_left_principal": [float(x) for x in np.sqrt(np.linalg.eigvalsh(r.g_left.T @ r.g_left))],
           "g_right_principal": [float(x) for x in np.sqrt(np.linalg.eigvalsh(r.g_right.T @ r.g_right))],
           "workload": "mirror-symmetric double dot on the 160x48x48 grid at B = 0, lowest 4 states "
                       "(bonding + anti-bonding doublets), d = 0.01 T"}
    if j_ci:
        th, ph = np.linspace(0, np.pi, 91), np.linspace(0, 2 * np.pi, 181)
        t0 = time.perf_counter()
        jp, jl, dz = ex.exchange_maps(j_ci, r.gsym_left, r.gsym_right, 0.2, [0.0, 1.0, 0.0], 0.1, th, ph)
        out["maps_ms"] = (time.perf_counter() - t0) * 1e3
        out["u_minus_eps_ev"] = 2 * r.tunnel ** 2 / j_ci
        out["jperp_range_ev"] = [float(jp.min()), float(jp.max())]
        out["jpar_range_ev"] = [float(jl.min()), float(jl.max())]
    g.close()
    return out


def _fp32_step_bench(grid, p, m, hbm, torch):
    """The FP32 filter step alone at full width (khp_filter_step: the
    defect-corrected form y = alpha H x + beta x + gamma prev + c_col src
    on all m columns of the C2 blocks), 20 launches timed with CUDA events
    on the handle's stream after 3 warm-up launches.  Algorithmic bytes per
    point-vector: x, prev and src read and y written (4 x 48 B) plus the
    per-point field tables (onsite 24 B, phases 72 B) over the m columns."""
    gen = torch.Generator(device="cuda").manual_seed(11)
    blocks = [torch.randn((p.n_unknowns, m), dtype=torch.complex64, device="cuda", generator=gen) for _ in range(4)]
    x, prev, src, y = blocks
    coef = np.linspace(-1.0, 1.0, m)
    for _ in range(3):
        grid.filter_step(x, y, 0.3, -0.2, -0.5, prev=prev, src=src, src_coef=coef)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(grid.stream)
    K = 20
    for _ in range(K):
        grid.filter_step(x, y, 0.3, -0.2, -0.5, prev=prev, src=src, src_coef=coef)
    e1.record(grid.stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / K
    bpv = 4 * 48.0 + 96.0 / m
    byts = p.n_points * m * bpv
    del blocks, x, prev, src, y
    return {"bound": "hbm", "kernel": "stencil_plane_kernel, defect-corrected FP32 step, full width",
            "achieved": byts / (ms * 1e-3) / 1e9, "peak": hbm, "unit": "GB/s",
            "frac": byts / (ms * 1e-3) / 1e9 / hbm, "frac_of_nominal_8tbs": byts / (ms * 1e-3) / 1e9 / 8000.0,
            "ms_per_launch": ms, "algorithmic_bytes_per_launch": byts, "bytes_per_pv": bpv,
            "point_vectors_per_launch": p.n_points * m}


def _projections_bench(grid, N, m, hbm, torch):
    """The Rayleigh-Ritz contractions at the bench's block size: Gram
    (G = Y^H Y, S = Y^H HY; reads 2 blocks) and rotation (X = Y Q, HX = W Q;
    reads 2, writes 2 blocks), as split-digit BF16 products (28 digit
    pairs) on the tcgen05 tensor cores ("tensor", the solver's default) and
    through mma.sync ("mma"), and on the FP64 ALUs.  CUDA events on the
    handle's stream around 5 calls after 2 warm-up calls."""
    gen = torch.Generator(device="cuda").manual_seed(7)
    Y = torch.randn((N, m), dtype=torch.complex128, device="cuda", generator=gen)
    W = grid.apply(Y)
    X = torch.empty_like(Y)
    HX = torch.empty_like(Y)
    rng = np.random.default_rng(7)
    Q = rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m))
    blk = N * m * 16.0
    out = {}

    def t(fn):
        for _ in range(2):
            fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(grid.stream)
        for _ in range(5):
            fn()
        e1.record(grid.stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 5

    for name, method in (("tensor", 0), ("mma", 2), ("fp64", 1)):
        tg = t(lambda: grid.project(Y, W, method=method))
        tr = t(lambda: grid.rotate(Y, Q, W, method=method, out=X, out_w=HX))
        out[name] = {"gram_ms": tg, "rotate_ms": tr,
                     "gram_gbs": 2 * blk / (tg * 1e-3) / 1e9, "rotate_gbs": 4 * blk / (tr * 1e-3) / 1e9}
    mma_flop = 28 * 2.0 * (2 * m) ** 2 * N * 2          # per contraction pair (G and S, or X and HX)
    for name in ("tensor", "mma"):
        tc = out[name]
        tc["gram_hbm_frac"] = tc["gram_gbs"] / hbm
        tc["rotate_hbm_frac"] = tc["rotate_gbs"] / hbm
        tc["gram_bf16_tflops"] = mma_flop / (tc["gram_ms"] * 1e-3) / 1e12
        tc["rotate_bf16_tflops"] = mma_flop / (tc["rotate_ms"] * 1e-3) / 1e12
    tc = out["tensor"]
    out["speedup_gram"] = out["fp64"]["gram_ms"] / tc["gram_ms"]
    out["speedup_rotate"] = out["fp64"]["rotate_ms"] / tc["rotate_ms"]
    out["tcgen05_vs_mma_gram"] = out["mma"]["gram_ms"] / tc["gram_ms"]
    out["tcgen05_vs_mma_rotate"] = out["mma"]["rotate_ms"] / tc["rotate_ms"]
    out["note"] = ("times include the library's stream synchronisation and the m x m host copy; "
                   "algorithmic bytes: Gram 2 blocks read, rotation 2 read + 2 written (N x m complex128)")
    return out


def run_profile(args):
    """Short solve on the full C2 grid for ncu: a few outer iterations."""
    import torch
    import inputs
    import paper_2607_08447_b300 as khp
    p = inputs.config2()
    if args.profile == "poisson":
        from paper_2607_08447_b300.poisson import Poisson
        gate = np.zeros((p.nz, p.ny, p.nx), dtype=np.uint8)
        gate[:, :, 0] = 1
        gate[:, :, -1] = 1
        P = Poisson(p.nx, p.ny, p.nz, p.h, gate, np.zeros_like(p.V))
        rho = torch.from_numpy(np.random.default_rng(5).random(p.n_points) * 1e-3).cuda()
        phi = P.solve(rho, tol=1e-10)
        torch.cuda.synchronize()
        print(json.dumps({"profile": "poisson", "multigrid_levels": P.mg_levels, "iterations": P.last_iterations,
                          "rel_residual": P.last_residual, "phi_max": float(phi.abs().max())}), flush=True)
        P.close()
        return
    g = khp.KPGrid.from_problem(p)
    prec = {"plain": 0, "mixed": 1, "dc": 2}[args.profile]
    # a random start by default: then every captured launch is the full
    # grid's own; --profile-start coarse gives the timed solves' sequence
    kw = dict(SOLVE_KW, max_iter=6, precision=prec, refine_sweeps=0, start=args.profile_start)
    coarse = args.profile_start == "coarse"
    if prec == 2:
        kw["degree"] = MIXED_DEGREE if coarse else MIXED_DEGREE_WARM
    elif not coarse:
        kw["degree"] = RANDOM_START_DEGREE
    r = g.eigensolve(**kw, allow_not_converged=True)
    torch.cuda.synchronize()
    print(json.dumps({"profile": args.profile, "stats": r.stats}), flush=True)
    g.close()


def run_sweep(args):
    """Batching form: many sweep points per call (lock-step rounds, one CUDA
    graph per round, block width autotuned once, one grouped filter launch
    per step across the chunk's problems), against the same rounds with
    per-problem filter launches and the same points solved one by one.  Defect-corrected FP32 filter, tol 1e-10 eV.  Under
    torchrun the points are sharded over the ranks (greedy by unknowns, no
    data-path collective) and the time is the maximum over ranks."""
    import torch
    import torch.distributed as dist
    import inputs
    import paper_2607_08447_b300 as khp
    from paper_2607_08447_b300.sweep import shard_of
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local_rank)
    allp = inputs.config4()[: args.sweep]
    mine = shard_of([p.n_unknowns for p in allp], rank, world)
    probs = [allp[i] for i in mine]
    coarse = args.sweep_start == "coarse"
    n, kw = 12, dict(degree=MIXED_DEGREE if coarse else MIXED_DEGREE_WARM, precision=2, tol=1e-10, seed=1,
                     start=args.sweep_start)
    unknowns = sum(p.n_unknowns for p in allp)
    # tuned once on the first chunk, reused for the rest
    grids = [khp.KPGrid.from_problem(p) for p in probs[: args.sweep_chunk]]
    rs = khp.solve_batched(grids, n, autotune=True, **kw)
    bm = rs[0].stats["block_m"]
    tune_ms = sum(r.stats["autotune_ms"] for r in rs)
    for g in grids:
        g.close()
    del grids, rs

    def timed(fn):
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = fn()
        torch.cuda.synchronize()
        t = torch.tensor([time.perf_counter() - t0], dtype=torch.float64, device="cuda")
        if world > 1:
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return out, float(t.item())

    def batched(grouped=True):
        ev = []
        for c in range(0, len(probs), args.sweep_chunk):
            grids = [khp.KPGrid.from_problem(p) for p in probs[c: c + args.sweep_chunk]]
            rs = khp.solve_batched(grids, n, block_m=bm, graph=True, grouped=grouped, **kw)
            ev += [r.evals for r in rs]
            for g in grids:
                g.close()
        return ev

    def sequential():
        ev = []
        for p in probs:
            g = khp.KPGrid.from_problem(p)
            ev.append(g.eigensolve(n, block_m=bm, **kw).evals)
            g.close()
        return ev

    evals_b, tb = timed(batched)
    evals_u, tu = timed(lambda: batched(grouped=False))
    evals_s, ts = timed(sequential)
    # the same grouped batches from random start blocks (the coarse start's gain)
    kw_coarse = kw
    kw = dict(kw, start="random", degree=MIXED_DEGREE_WARM)
    evals_r, tr = timed(batched)
    kw = kw_coarse
    dgr = max(float(np.abs(a - b).max()) for a, b in zip(evals_b, evals_r)) if probs else 0.0
    dmax = max(float(np.abs(a - b).max()) for a, b in zip(evals_b, evals_s)) if probs else 0.0
    dgu = max(float(np.abs(a - b).max()) for a, b in zip(evals_b, evals_u)) if probs else 0.0

    # plain FP64 (the same tolerance) on a sample of this rank's points,
    # batched the same way, against the defect-corrected batched solve
    sample = probs[: args.sweep_plain]

    def batched_sample(kws):
        grids = [khp.KPGrid.from_problem(p) for p in sample]
        rs = khp.solve_batched(grids, n, block_m=bm, graph=True, **kws)
        ev = [r.evals for r in rs]
        for g in grids:
            g.close()
        return ev

    plain_kw = dict(degree=SOLVE_KW["degree"] if coarse else RANDOM_START_DEGREE, precision=0, tol=1e-10, seed=1,
                    start=args.sweep_start)
    ev_dc, t_dc = timed(lambda: batched_sample(kw))
    ev_fp64, t_fp64 = timed(lambda: batched_sample(plain_kw))
    d_plain = max(float(np.abs(a - b).max()) for a, b in zip(ev_dc, ev_fp64)) if sample else 0.0
    line = {"metric": "sweep eigenpairs/s (batched detuning sweep)", "value": n * len(allp) / tb,
            "unit": "eigenpairs/s", "n_gpus": world, "higher_is_better": True, "scaling": "strong",
            "dtype": "fp32 filter + fp64 RR", "data": "synthetic",
            "config": {"workload": f"config-4 sweep: {len(allp)} points, {unknowns} unknowns in total, "
                                   f"12 states each, chunks of {args.sweep_chunk}, degree {kw['degree']}, "
                                   f"{args.sweep_start} start, block_m autotuned = {bm}", "autotune_ms": tune_ms,
                       "parallelism": f"sweep sharded over {world} rank(s), no collective"},
            "sequential": {"value": n * len(allp) / ts, "unit": "eigenpairs/s", "s": ts},
            "batched_s": tb, "speedup_vs_sequential": ts / tb, "max_abs_dE_batched_vs_single_ev": dmax,
            "ungrouped": {"s": tu, "speedup_vs_sequential": ts / tu, "max_abs_dE_vs_grouped_ev": dgu,
                          "note": "the same batched rounds with one filter launch per problem and step"},
            "random_start": {"s": tr, "value": n * len(allp) / tr, "max_abs_dE_vs_grouped_ev": dgr,
                             "note": f"the same grouped batches from random start blocks at degree {MIXED_DEGREE_WARM}"},
            "vs_plain_fp64": {"points": len(sample), "mixed_batched_s": t_dc, "fp64_batched_s": t_fp64,
                              "speedup": t_fp64 / t_dc if t_dc > 0 else None,
                              "max_abs_dE_ev": d_plain,
                              "note": "same points, start, block width and tolerance (1e-10 eV); plain FP64 at "
                                      f"degree {plain_kw['degree']}, mixed = defect-corrected FP32 filter at degree "
                                      f"{kw['degree']}"}}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    args = _args()
    if args.profile:
        run_profile(args)
        return
    if args.sweep:
        run_sweep(args)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    run_ours(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
