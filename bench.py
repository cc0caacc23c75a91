#!/usr/bin/env python3
"""Benchmark of the GB300 sFLSQR / sFLSMR solvers.

One step = one complete solve (initialisation, sketched flexible Golub-Kahan
steps up to the discrepancy stop, x = Z y) of a synthetic CT workload.  The
default workload is sFLSMR with an unmatched pixel-driven back-projector on a
256x256 image (180 angles x 363 bins, A: 15.0M nonzeros, B: 23.6M nonzeros,
5%-sparse phantom, 2% noise, reweighting flexible operator, sketch s = 400,
window 2, maxit 200), FP64 path.  Its operator bytes (about 464 MB per step)
exceed the 129 MB L2, so no L2 flush is needed between timed steps.

Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle
on the host cores instead (a bounded sample per step).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

DEFAULT_WORKLOAD = "ct1024_sflsqr"
# Oracle steps per bounded CPU sample (None: the whole solve), sized so one
# sample takes about 5-30 s on one host core.
ORACLE_SAMPLE_STEPS = {"ct1024_sflsqr": 4, "ct256_sflsmr_unmatched": None, "ct64_sflsqr": None}
REFERENCE_SAMPLE_STEPS = {"ct1024_sflsqr": 1, "ct256_sflsmr_unmatched": 10, "ct64_sflsqr": 10}
METRIC = "sFLSQR/sFLSMR iters/s, time to discrepancy stop, HBM roofline fraction"


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-tiles", action="store_true",
                    help="store the rows of A^T / B in natural order instead of 16x16 pixel tiles")
    ap.add_argument("--slot-layout", default="interleaved", choices=["interleaved", "operator"],
                    help="entry order inside the chunk slots of the single-solve plans (main and mixed legs)")
    ap.add_argument("--only-batched", action="store_true",
                    help="run only the batched multi-sinogram leg (64 x 512^2, FP32) and print its JSON")
    ap.add_argument("--only-mixed", action="store_true",
                    help="run only the mixed-precision leg (1024^2, BF16 / FP32 values) and print its JSON")
    ap.add_argument("--mixed-size", type=int, default=1024,
                    help="image size of the mixed-precision leg (1024: the configured workload; smaller sizes keep "
                         "its geometry recipe, for profiling)")
    ap.add_argument("--only-decay", action="store_true",
                    help="run only the residual-size study (dense 1024 x 512, Gaussian sketches) and print its JSON")
    ap.add_argument("--only-matfree", action="store_true",
                    help="only the matrix-free 256x256 unmatched solve (FP64 and FP32 projectors)")
    ap.add_argument("--only-deblur", action="store_true",
                    help="only the low-rank deblurring timing comparison (512x512, rank 30, 50 steps)")
    ap.add_argument("--only-flsqr", action="store_true",
                    help="only the FLSQR / sFLSQR comparison at equal step counts (1024x1024, FP64)")
    ap.add_argument("--only-diff", action="store_true",
                    help="run only the differentiable leg (16 x 256^2, fixed k, forward + adjoint) and print its JSON")
    ap.add_argument("--driver", default="graph", choices=["graph", "host_loop"],
                    help="graph: one CUDA graph per solve (the measured configuration); host_loop: the same "
                         "kernels launched one by one from the host, for profilers that cannot see inside "
                         "graphs with conditional nodes (skips the end-to-end leg)")
    ap.add_argument("--sketch-apply", default="auto", choices=["auto", "fused", "kernel"],
                    help="how the main workload's solver applies the sparse-sign sketch (auto: the library's choice)")
    ap.add_argument("--image", type=int, default=0,
                    help="profiling only: build the main workload at this image size (same angles and recipe); "
                         "the line's config.workload then carries the size")
    ap.add_argument("--oracle-sample", type=int, default=0, help=argparse.SUPPRESS)
    return ap.parse_args()


# ---------------------------------------------------------------- helpers

def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return {"hbm_gbs": float(d["hbm_gbs"]), "source": "measured"}
    return {"hbm_gbs": 6800.0, "source": "fallback"}


class ClockSampler:
    """nvidia-smi clock/throttle samples every 50 ms while the timed region runs."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1])); smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def img(args, p):
    """The n-side image shape of a CT workload (pixel tiles for A^T / B), unless --no-tiles."""
    return None if getattr(args, "no_tiles", False) else (p.N, p.N)


def adjoint_mismatch(p, np):
    """|y^T A x - x^T B y| for seeded random unit x, y: how far an unmatched
    back-projector B is from A^T (None when the plan uses A^T itself)."""
    if p.B is None:
        return None
    rng = np.random.default_rng(12)
    x = rng.standard_normal(p.A.shape[1]); x /= np.linalg.norm(x)
    y = rng.standard_normal(p.A.shape[0]); y /= np.linalg.norm(y)
    return float(abs(y @ (p.A.scipy() @ x) - x @ (p.B.scipy() @ y)))


def kernel_source_hash() -> str:
    """Hash of the product kernels' code: kernels.cuh and common.cuh with
    comments and blank lines removed, so that comment edits keep a recorded
    ncu measurement valid and code edits do not."""
    h = hashlib.sha256()
    for name in ("kernels.cuh", "common.cuh"):
        for line in open(os.path.join(ROOT, "paper_2605_22281_gb300", "csrc", name), encoding="utf-8"):
            code = line.split("//", 1)[0].rstrip()
            if code:
                h.update(code.encode() + b"\n")
    return h.hexdigest()[:16]


def recorded_traffic(kernel: str, workload: str):
    """DRAM bytes per launch from a committed ncu summary, if it matches the current kernel source."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.json")
    if not os.path.exists(path):
        return None
    d = json.load(open(path))
    e = d.get(workload, {}).get(kernel)
    if not e or e.get("kernel_source_sha") != kernel_source_hash():
        return None
    return e.get("bytes_per_launch")


def spmv_bytes(nnz, rows, cols, vbytes, xbytes, ndots, table_bytes, ibytes=4):
    """Compulsory bytes of one fused SpMV launch: values + column indices
    (ibytes per entry: 4, or 2 for 16-bit column deltas, which add one 4-byte
    base column per row) + row pointers, the gathered input vector once, the
    output vector, the window vectors read by the fused dots, and the sketch
    table."""
    base = 4 * rows if ibytes == 2 else 0
    return (nnz * (vbytes + ibytes) + 4 * (rows + 1) + base + xbytes * (cols + rows) + xbytes * rows * ndots
            + table_bytes)


# ---------------------------------------------------------------- oracle (CPU) legs

def oracle_solve(workload: str, maxit_cap: int | None, problem=None):
    import numpy as np
    import oracle as O
    import workloads as wl
    p = problem or wl.make(workload)
    st = p.settings
    tol = O.discrepancy_tol(st["eta"], p.noise_norm[0], float(np.linalg.norm(p.b)))
    maxit = st["maxit"] if maxit_cap is None else min(maxit_cap, st["maxit"])
    if not hasattr(p, "_sp"):          # SciPy views built once per problem (not timed)
        p._sp = (p.A.scipy(), p.B.scipy() if p.B is not None else None)
    A, AT = p._sp
    tau = {"identity": O.Identity(), "irw": O.Reweighting(st.get("irw_eps", 1e-4))}.get(st["precond"])
    t0 = time.perf_counter()
    if st["method"] == "sflsqr":
        S = O.SparseSign(st["seed"], st["s"], st["zeta"], A.shape[0])
        r = O.sflsqr(A, p.b, S, maxit=maxit, tol=tol, ell=st["window"], tau=tau, AT=AT, keep_basis=False)
    else:
        Sn = O.SparseSign(st["seed"], st["s"], st["zeta"], A.shape[1])
        Sm = O.SparseSign(st["seed"] + 1, st["s"], st["zeta"], A.shape[0])
        r = O.sflsmr(A, p.b, Sn, S_stop=Sm, maxit=maxit, tol=tol, ell=st["window"], tau=tau, AT=AT, keep_basis=False)
    return r, time.perf_counter() - t0


def cpu_baseline_subprocess(workload: str, maxit_cap: int | None, threads: int = 1) -> dict:
    """Time the oracle in a child process with `threads` BLAS/OpenMP threads."""
    t = str(threads)
    env = dict(os.environ, OMP_NUM_THREADS=t, OPENBLAS_NUM_THREADS=t, MKL_NUM_THREADS=t)
    cmd = [sys.executable, os.path.abspath(__file__), "--workload", workload, "--oracle-sample",
           str(maxit_cap if maxit_cap else -1)]
    out = subprocess.run(cmd, env=env, capture_output=True, text=True, timeout=1200)
    if out.returncode != 0:
        return {"error": out.stderr[-400:]}
    return json.loads(out.stdout.strip().splitlines()[-1])


def oracle_sample_main(workload: str, cap: int):
    r, dt = oracle_solve(workload, None if cap < 0 else cap)
    print(json.dumps({"iters": r.iters, "seconds": dt, "status": int(r.status)}))


def run_reference(args):
    """The oracle as it stands on the host cores; each step a bounded sample."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import workloads as wl
    cap = REFERENCE_SAMPLE_STEPS.get(args.workload, 10)
    p = wl.make(args.workload)
    for _ in range(args.warmup):
        oracle_solve(args.workload, cap, p)
    iters, secs = 0, 0.0
    for _ in range(args.steps):
        r, dt = oracle_solve(args.workload, cap, p)
        iters += r.iters
        secs += dt
    value = iters / secs
    sample = f"each step: the first {cap} sFLSMR/sFLSQR steps of the {args.workload} workload (oracle, FP64, 1 thread)"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * secs / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "l2": "inputs larger than L2 (CPU run)"},
            "cpu_baseline": {"value": value, "unit": "iters/s", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "iters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- GPU leg

def gather_rank_values(vals, world: int, device) -> list:
    """Every rank's list of values (all_gather over the default process
    group); with one rank, [vals]."""
    if world <= 1:
        return [list(vals)]
    import torch
    import torch.distributed as dist
    tt = torch.tensor([float(v) for v in vals], dtype=torch.float64, device=device)
    out = [torch.zeros_like(tt) for _ in range(world)]
    dist.all_gather(out, tt)
    return [[float(v) for v in o] for o in out]


def aggregate(per_rank: list, steps: int) -> tuple:
    """Weak scaling over independent problems: (max time over ranks in ms,
    iterations of all ranks, whole-job iterations per second) from per-rank
    (time ms, iterations per solve)."""
    t_max = max(r[0] for r in per_rank)
    total = sum(int(round(r[1])) * steps for r in per_rank)
    return t_max, total, total / (t_max / 1000.0)


def rank_problem(p, rank: int, wl, np):
    """Rank r > 0 solves its own problem: the same operator and phantom, fresh
    noise at the same level (seed 1000 + r)."""
    if rank == 0:
        return p
    rng = np.random.default_rng(1000 + rank)
    b_true = p.A.matvec(p.x_true)
    p.b, en = wl.add_noise(b_true, float(p.noise_norm[0] / np.linalg.norm(b_true)), rng)
    p.noise_norm = np.array([en])
    return p


def batched_variant(args, G, wl, np, torch):
    """The multi-sinogram form: 64 sinograms of 512x512 ellipse phantoms through
    one 360 x 725 Siddon operator (120M nonzeros), noise levels log-uniform in
    [0.5%, 5%], batched sFLSQR with FP32 values and vectors (FP64 small
    problems), against the plain FP64 single-solve path on a sample of the
    same right-hand sides; errors are ||x - x_true|| / ||x_true||."""
    p = wl.make("ct512_batch64")
    st = p.settings
    R = p.b.shape[1]
    kw = dict(s=st["s"], zeta=st["zeta"], seed=st["seed"], window=st["window"], maxit=st["maxit"], eta=st["eta"])
    B = torch.as_tensor(np.ascontiguousarray(p.b.T), device="cuda")
    # batched solves: rows in the operator's entry order, no pixel tiles (the SpMM walks one row per warp)
    plan32 = G.Plan(p.A, value_dtype="f32", slot_layout="operator")
    t0 = time.perf_counter()
    X, infos = G.solve_batched(plan32, B, p.noise_norm, **kw)       # builds and tunes the session
    torch.cuda.synchronize()
    t_first = time.perf_counter() - t0
    stream = torch.cuda.current_stream()
    reps = max(1, min(args.steps, 3))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        G.solve_batched(plan32, B, p.noise_norm, sync=False, out=X, **kw)
    e1.record(stream)
    torch.cuda.synchronize()
    t_batch = e0.elapsed_time(e1) / reps
    Xh = X.cpu().numpy()
    xt = p.x_true.T
    err32 = [float(np.linalg.norm(Xh[j] - xt[j]) / np.linalg.norm(xt[j])) for j in range(R)]
    iters = [i.iters for i in infos]
    tiles = G.batched_tiles(plan32)
    plan32.close()
    # algorithmic bytes of the batch: the matrix twice per batched step, the active right-hand sides' vectors
    m, n = p.A.shape
    alg = sum(2 * int(p.A.nnz) * 8 + sum(1 for i in iters if i >= k) * 9 * (m + n) * 4
              for k in range(1, max(iters) + 1))
    pk = load_peaks()
    # plain FP64 path, one solve per right-hand side, on a sample of columns
    plan64 = G.Plan(p.A, value_dtype="f64", image_shape=img(args, p))
    sample = list(range(R))   # every right-hand side of the batch
    for j in sample[:1]:
        plan64.solve("sflsqr", torch.as_tensor(p.b[:, j], device="cuda"), noise_norm=float(p.noise_norm[j]), **kw)
    torch.cuda.synchronize()
    t64 = 0.0
    eq = 0
    err64 = []
    for j in sample:
        bj = torch.as_tensor(np.ascontiguousarray(p.b[:, j]), device="cuda")
        e0.record(stream)
        x64, i64, _ = plan64.solve("sflsqr", bj, noise_norm=float(p.noise_norm[j]), **kw)
        e1.record(stream)
        torch.cuda.synchronize()
        t64 += e0.elapsed_time(e1)
        e = float(np.linalg.norm(x64.cpu().numpy() - xt[j]) / np.linalg.norm(xt[j]))
        err64.append(e)
        eq += abs(err32[j] - e) <= 0.01 * e
    plan64.close()
    fp64_solves = len(sample) / (t64 / 1000)
    value = R / (t_batch / 1000)
    return {"value": value, "unit": "solves/s", "batch_ms": t_batch, "nrhs": R, "m": p.A.shape[0], "n": p.A.shape[1],
            "nnz": int(p.A.nnz), "values": "f32", "vectors": "f32", "small_problems": "f64",
            "iters_min_median_max": [min(iters), int(statistics.median(iters)), max(iters)],
            "rel_error_median": statistics.median(err32), "spmm_tiles": {"A": tiles[0], "At": tiles[1]},
            "roofline": {"bound": "hbm", "achieved": alg / (t_batch / 1000) / 1e9, "peak": pk["hbm_gbs"],
                         "unit": "GB/s", "frac": alg / (t_batch / 1000) / 1e9 / pk["hbm_gbs"], "traffic": None,
                         "algorithmic_bytes_per_batch": alg, "peak_source": pk["source"],
                         "scope": "whole batched solve: 2 nnz (V + I) per batched step + 9 (m + n) X per active RHS; "
                                  "the SpMMs are bound by L2 gathers (nnz x 64 RHS x 4 B per product), not HBM"},
            "first_call_s_incl_session_and_tuning": t_first,
            "plain_fp64": {"solves_per_s": fp64_solves, "columns": len(sample),
                           "rel_error_min_median_max": [min(err64), statistics.median(err64), max(err64)],
                           "worst_relative_gap_to_batched_error": max(abs(err32[j] - e) / e for j, e in zip(sample, err64)),
                           "equal_error_columns": f"{eq}/{len(sample)} within 1% (relative) of the FP64 error"},
            "speedup_vs_plain_fp64": value / fp64_solves}


def mixed_variant(args, G, wl, np, torch, x_fp64=None):
    """sFLSQR at scale: 1024x1024 image, 360 angles x 1449 bins (481M nonzeros),
    1% noise, s = 600, window 4, maxit 300, with BF16 or FP32 operator values
    (FP32 vectors and accumulation, FP64 small problem and coefficients), and
    the FP64 path on the same problem for the error comparison."""
    N = args.mixed_size
    p = wl.make("ct1024_sflsqr") if N == 1024 else wl.make("ct1024_sflsqr", N=N, n_angles=max(1, 360 * N // 1024))
    st = p.settings
    kw = dict(s=st["s"], zeta=st["zeta"], seed=st["seed"], window=st["window"], maxit=st["maxit"],
              noise_norm=float(p.noise_norm[0]), eta=st["eta"])
    b = torch.as_tensor(p.b, device="cuda")
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = {"image": f"{N}x{N}", "m": p.A.shape[0], "n": p.A.shape[1], "nnz": int(p.A.nnz)}
    xs = {}
    dtypes = ("bf16", "f32") if x_fp64 is not None and N == 1024 else ("bf16", "f32", "f64")
    if len(dtypes) == 2:
        xs["f64"] = x_fp64
    for vdt in dtypes:
        plan = G.Plan(p.A, value_dtype=vdt, image_shape=img(args, p), slot_layout=args.slot_layout)
        x, info, _ = plan.solve("sflsqr", b, driver=args.driver, **kw)
        reps = max(1, min(args.steps, 3))
        e0.record(stream)
        for _ in range(reps):
            plan.solve("sflsqr", b, out=x, sync=False, driver=args.driver, **kw)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        xh = x.cpu().numpy()
        xs[vdt] = xh
        leg = {"iters": info.iters, "stop": info.status_name, "time_to_stop_ms": ms,
               "iters_per_s": info.iters / (ms / 1000),
               "rel_error_vs_x_true": float(np.linalg.norm(xh - p.x_true) / np.linalg.norm(p.x_true))}
        if vdt != "f64":
            _, _, hp = plan.solve("sflsqr", b, driver="profiled", **kw)
            kms, kl = hp["kernel_ms"], hp["kernel_launches"]
            vb = 2 if vdt == "bf16" else 4
            pst = plan.stats()
            for name, nnz, rows, cols, ib in (("spmv_fwd", p.A.nnz, p.A.shape[0], p.A.shape[1], pst["index_bytes_A"]),
                                              ("spmv_bwd", p.A.nnz, p.A.shape[1], p.A.shape[0], pst["index_bytes_At"])):
                avg = kms[name] / max(kl[name], 1)
                nbytes = spmv_bytes(int(nnz), rows, cols, vb, 4, st["window"] + 1, 0, ib)
                leg[name] = {"avg_us": 1000 * avg, "bytes": nbytes, "gbs": nbytes / (avg * 1e-3) / 1e9,
                             "hbm_frac_of_measured": nbytes / (avg * 1e-3) / 1e9 / load_peaks()["hbm_gbs"]}
        out[vdt] = leg
        plan.close()
    for vdt in ("bf16", "f32"):
        out[vdt]["rel_diff_vs_fp64_path_x"] = float(np.linalg.norm(xs[vdt] - xs["f64"]) / np.linalg.norm(xs["f64"]))
    out["value"] = out["bf16"]["iters_per_s"]
    out["unit"] = "iters/s"
    return out


def flsqr_variant(args, G, wl, np, torch, steps: int = 30):
    """The paper's FLSQR-against-sFLSQR timing comparison, on the GPU at
    1024x1024 (FP64, 481M nonzeros), at equal step counts: FLSQR (full
    orthogonalization by block CGS2, exact projected problem through H, no
    sketch) and sFLSQR (window 4, sparse-sign sketch s = 600), both run for
    `steps` steps with the discrepancy stop off, plus sFLSMR with a full window.
    Also the relative residual each reaches at the last step."""
    p = wl.make("ct1024_sflsqr")
    st = p.settings
    plan = G.Plan(p.A, value_dtype="f64", image_shape=img(args, p), slot_layout=args.slot_layout)
    b = torch.as_tensor(p.b, device="cuda")
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = {"image": "1024x1024", "steps": steps, "values": "f64"}
    legs = {"flsqr_full": ("flsqr", dict(s=0, window=-1)),
            "sflsqr_window4": ("sflsqr", dict(s=st["s"], zeta=st["zeta"], seed=st["seed"], window=st["window"])),
            "sflsqr_full": ("sflsqr", dict(s=st["s"], zeta=st["zeta"], seed=st["seed"], window=-1))}
    for name, (method, kw) in legs.items():
        x, info, _ = plan.solve(method, b, maxit=steps, **kw)
        torch.cuda.synchronize()
        e0.record(stream)
        plan.solve(method, b, maxit=steps, out=x, sync=False, **kw)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        xh = x.cpu().numpy()
        res = float(np.linalg.norm(p.A.matvec(xh) - p.b) / np.linalg.norm(p.b))
        out[name] = {"iters": info.iters, "stop": info.status_name, "ms": ms, "ms_per_step": ms / max(info.iters, 1),
                     "rel_residual": res,
                     "rel_error_vs_x_true": float(np.linalg.norm(xh - p.x_true) / np.linalg.norm(p.x_true))}
    plan.close()
    out["flsqr_over_sflsqr_time"] = out["flsqr_full"]["ms"] / out["sflsqr_window4"]["ms"]
    return out


def deblur_variant(args, G, wl, np, torch, N: int = 512):
    """The timing experiment of Section 4.1 on the GPU: deblurring and
    inpainting of a 512x512 image (Gaussian PSF of variance 0.25, half of the
    pixels kept, 5% noise, synthetic block image), 50 steps of each method
    with no stop, rank-30 truncation by the randomized SVD (oversampling 10,
    one subspace-iteration step), CountSketch with s = 101, window 2.  FP64
    operator and vectors; the truncation itself is FP32."""
    p = wl.make("deblur512_lowrank", N=N) if N != 512 else wl.make("deblur512_lowrank")
    st = p.settings
    plan = G.Plan(p.A, value_dtype="f64", image_shape=(p.N, p.N))
    b = torch.as_tensor(p.b, device="cuda")
    om = torch.as_tensor(st["omega"], device="cuda")
    lr = dict(precond="lowrank", lowrank_rank=st["rank"], lowrank_oversample=st["oversample"],
              lowrank_power=st["power"], lowrank_omega=om)
    sk = dict(s=st["s"], zeta=st["zeta"], seed=st["seed"], window=st["window"])
    legs = {"flsqr_identity": ("flsqr", dict(s=0, window=-1)),
            "sflsqr_identity": ("sflsqr", dict(sk)),
            "flsqr_rnd": ("flsqr", dict(s=0, window=-1, **lr)),
            "sflsqr_rnd": ("sflsqr", dict(sk, **lr)),
            "sflsmr_rnd": ("sflsmr", dict(sk, **lr))}
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = {"image": f"{p.N}x{p.N}", "m": p.A.shape[0], "n": p.A.shape[1], "nnz": int(p.A.nnz), "steps": st["maxit"],
           "rank": st["rank"], "oversample": st["oversample"], "power": st["power"], "s": st["s"], "zeta": st["zeta"]}
    for name, (method, kw) in legs.items():
        x, info, _ = plan.solve(method, b, maxit=st["maxit"], **kw)
        torch.cuda.synchronize()
        reps = 3
        e0.record(stream)
        for _ in range(reps):
            plan.solve(method, b, maxit=st["maxit"], out=x, sync=False, **kw)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        xh = x.cpu().numpy()
        leg = {"iters": info.iters, "stop": info.status_name, "ms": ms, "ms_per_step": ms / max(info.iters, 1),
               "rel_residual": float(np.linalg.norm(p.A.matvec(xh) - p.b) / np.linalg.norm(p.b)),
               "rel_error_vs_x_true": float(np.linalg.norm(xh - p.x_true) / np.linalg.norm(p.x_true))}
        if name == "sflsqr_rnd":
            _, _, hp = plan.solve(method, b, maxit=st["maxit"], driver="profiled", **kw)
            leg["kernel_ms_per_step"] = {c: hp["kernel_ms"][c] / max(info.iters, 1) for c in hp["kernel_ms"]
                                         if hp["kernel_launches"][c] > 0}
        out[name] = leg
    plan.close()
    return out


def matfree_variant(args, G, wl, np, torch):
    """The 256x256 unmatched sFLSMR workload solved with no stored operator: the
    matrix-free plan computes A z by Siddon's ray walk and B w by the
    pixel-driven interpolation on the fly (FP64, and FP32 geometry with FP32
    vectors), against the stored-operator FP64 solve of the same problem.
    Reports the products' launch times and the stored operator's bytes per
    launch they replace (the products are bound by arithmetic, not memory)."""
    p = wl.make("ct256_sflsmr_unmatched")
    st = p.settings
    kw = dict(s=st["s"], zeta=st["zeta"], seed=st["seed"], window=st["window"], maxit=st["maxit"],
              noise_norm=float(p.noise_norm[0]), eta=st["eta"], precond="reweight", irw_eps=st["irw_eps"])
    b = torch.as_tensor(p.b, device="cuda")
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ref = G.Plan(p.A, p.B, image_shape=(p.N, p.N))
    x_ref, i_ref, _ = ref.solve("sflsmr", b, **kw)
    x_ref = x_ref.cpu().numpy()
    ref.close()
    out = {"image": f"{p.N}x{p.N}", "angles": p.n_angles, "bins": p.n_bins,
           "stored_iters": i_ref.iters, "stored_nnz": {"A": int(p.A.nnz), "B": int(p.B.nnz)}}
    for vdt in ("f64", "f32"):
        plan = G.Plan.ct(p.N, p.n_angles, p.n_bins, back="unmatched", value_dtype=vdt)
        x, info, _ = plan.solve("sflsmr", b, **kw)
        reps = max(3, min(args.steps, 10))
        e0.record(stream)
        for _ in range(reps):
            plan.solve("sflsmr", b, out=x, sync=False, **kw)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        xh = x.cpu().numpy()
        _, _, hp = plan.solve("sflsmr", b, driver="profiled", **kw)
        kms, kl = hp["kernel_ms"], hp["kernel_launches"]
        vb = 8 if vdt == "f64" else 4
        leg = {"iters": info.iters, "stop": info.status_name, "time_to_stop_ms": ms, "iters_per_s": info.iters / (ms / 1000),
               "rel_diff_vs_stored_fp64_x": float(np.linalg.norm(xh - x_ref) / np.linalg.norm(x_ref)),
               "rel_error_vs_x_true": float(np.linalg.norm(xh - p.x_true) / np.linalg.norm(p.x_true))}
        for name, nnz in (("spmv_fwd", p.A.nnz), ("spmv_bwd", p.B.nnz)):
            avg = kms[name] / max(kl[name], 1)
            leg[name] = {"avg_us": 1000 * avg, "entries_per_s": nnz / (avg * 1e-3),
                         "stored_bytes_replaced": int(nnz) * (vb + 4)}
        out[vdt] = leg
        plan.close()
    return out


def diff_variant(args, G, wl, np, torch):
    """The differentiable form: 16 sinograms of 256x256 phantoms, fixed k = 30
    steps of sFLSQR with a diagonal weight (s = 61, window 2), FP32 values and
    vectors; one forward plus one hand-written adjoint per timed step."""
    p = wl.make("ct256_diff16")
    st = p.settings
    plan = G.Plan(p.A, value_dtype="f32", image_shape=img(args, p))
    B = torch.as_tensor(np.ascontiguousarray(p.b.T), device="cuda")
    d = torch.as_tensor(st["weight"], device="cuda")
    kw = dict(s=st["s"], zeta=st["zeta"], seed=st["seed"], window=st["window"], maxit=st["maxit"])
    Xbar = torch.randn((B.shape[0], p.A.shape[1]), dtype=torch.float64, device="cuda",
                       generator=torch.Generator(device="cuda").manual_seed(0))
    X, infos, _ = G.fixed_batched(plan, B, d, **kw)
    G.adjoint(plan, Xbar)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    reps = max(1, min(args.steps, 5))
    fwd = bwd = 0.0
    for _ in range(reps):
        e0.record(stream)
        G.fixed_batched(plan, B, d, out=X, **kw)
        e1.record(stream)
        G.adjoint(plan, Xbar)
        e2.record(stream)
        torch.cuda.synchronize()
        fwd += e0.elapsed_time(e1)
        bwd += e1.elapsed_time(e2)
    fwd /= reps
    bwd /= reps
    R = B.shape[0]
    plan.close()
    return {"value": R / ((fwd + bwd) / 1000), "unit": "differentiated solves/s", "nrhs": R, "k": st["maxit"],
            "forward_ms": fwd, "adjoint_ms": bwd, "values": "f32", "vectors": "f32",
            "note": "gradients checked in tests (FP64 oracle autograd, finite differences)"}


def small_variant(args, G, wl, np, torch):
    """The 64x64 workload (60 angles x 91 bins, sFLSQR, FP64, s = 200, window 2):
    L2-resident and latency-bound, reported as iterations/s and time to stop."""
    p = wl.make("ct64_sflsqr")
    st = p.settings
    kw = dict(s=st["s"], zeta=st["zeta"], seed=st["seed"], window=st["window"], maxit=st["maxit"],
              noise_norm=float(p.noise_norm[0]), eta=st["eta"])
    plan = G.Plan(p.A, image_shape=(p.N, p.N))
    b = torch.as_tensor(p.b, device="cuda")
    x, info, _ = plan.solve("sflsqr", b, **kw)
    for _ in range(2):
        plan.solve("sflsqr", b, out=x, **kw)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 20
    e0.record(stream)
    for _ in range(reps):
        plan.solve("sflsqr", b, out=x, sync=False, **kw)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    err = float(np.linalg.norm(x.cpu().numpy() - p.x_true) / np.linalg.norm(p.x_true))
    plan.close()
    return {"iters": info.iters, "stop": info.status_name, "time_to_stop_ms": ms,
            "iters_per_s": info.iters / (ms / 1000), "rel_error_vs_x_true": err}


def decay_variant(args, G, wl, np, torch):
    """The paper's residual-size study through the GPU path: A (1024 x 512) with
    singular values rho^(1-i), x_true = ones, ||b_true|| = 1, 10% noise; 20 steps of
    sLSQR and sLSMR with Gaussian sketches of s = 2k + 1 = 41 rows (explicit dense
    sketch matrices, identity operator, window 8), against the optimal residual of
    the same Krylov space (LSQR: SciPy's lsqr, 20 iterations, on the host).  Per rho:
    LSQR's ||A x - b|| / ||b|| and the sketched residuals relative to it, averaged
    over 5 sketches; again with the Gaussian and SRHT sketches the kernel
    regenerates from the seed ("generated")."""
    import scipy.sparse.linalg as spla
    k, s, m, n, draws = 20, 41, 1024, 512, 5
    Sm = torch.empty((s, m), dtype=torch.float64, device="cuda")
    Sn = torch.empty((s, n), dtype=torch.float64, device="cuda")
    out = {"m": m, "n": n, "k": k, "s": s, "noise": 0.10, "sketches": draws, "window": 8, "rho": {}}
    for rho in (1.01, 1.03, 1.05, 1.08, 1.10, 1.15):
        A, b, _, _ = wl.decaying(m, n, rho, 70, 0.10)
        x_opt = spla.lsqr(A, b, atol=0.0, btol=0.0, conlim=0.0, iter_lim=k)[0]
        r_opt = float(np.linalg.norm(A @ x_opt - b))
        plan = G.Plan(wl.dense_csr(A))
        bd = torch.as_tensor(b, device="cuda")
        rq, rm = [], []
        for t in range(draws):
            g = np.random.default_rng(500 + t)
            Sm.copy_(torch.as_tensor(g.standard_normal((s, m))))
            Sn.copy_(torch.as_tensor(g.standard_normal((s, n))))
            xq, _, _ = plan.solve("sflsqr", bd, s=s, window=8, maxit=k, sketch_matrix=Sm)
            xm, _, _ = plan.solve("sflsmr", bd, s=s, window=8, maxit=k, sketch_matrix=Sn, sketch_matrix_stop=Sm)
            rq.append(float(np.linalg.norm(A @ xq.cpu().numpy() - b)) / r_opt)
            rm.append(float(np.linalg.norm(A @ xm.cpu().numpy() - b)) / r_opt)
        # the same with sketches the kernel regenerates from the seed (no matrices)
        gen = {}
        for kind in ("gaussian", "srht"):
            gq, gm = [], []
            for t in range(draws):
                xq, _, _ = plan.solve("sflsqr", bd, s=s, seed=500 + t, window=8, maxit=k, sketch_kind=kind)
                xm, _, _ = plan.solve("sflsmr", bd, s=s, seed=500 + t, window=8, maxit=k, sketch_kind=kind)
                gq.append(float(np.linalg.norm(A @ xq.cpu().numpy() - b)) / r_opt)
                gm.append(float(np.linalg.norm(A @ xm.cpu().numpy() - b)) / r_opt)
            gen[kind] = {"slsqr_over_lsqr": statistics.mean(gq), "slsmr_over_lsqr": statistics.mean(gm)}
        plan.close()
        out["rho"][f"{rho:.2f}"] = {"lsqr_rel_residual": r_opt / float(np.linalg.norm(b)),
                                    "slsqr_over_lsqr": statistics.mean(rq), "slsmr_over_lsqr": statistics.mean(rm),
                                    "generated": gen}
    return out


def single_leg(args, G, wl, np, torch, p, vdt: str, *, steps: int, warmup: int, world: int = 1,
               barrier=None, sampler=None, e2e: bool = False, workload: str = ""):
    """One single-solve workload on one value precision: warm-up solves (which
    also build the session and its CUDA graph), `steps` timed solves with CUDA
    events on the launching stream, the per-launch times of the two products
    from the profiled driver (same kernels, same stream), and optionally the
    same solve end to end through the host-buffer C ABI.  Returns a dict."""
    st = p.settings
    method = st["method"]
    precond = {"identity": "identity", "irw": "reweight", "diag": "diag"}[st["precond"]]
    kw = dict(s=st["s"], zeta=st["zeta"], seed=st["seed"], window=st["window"], maxit=st["maxit"],
              noise_norm=float(p.noise_norm[0]), eta=st["eta"], precond=precond, irw_eps=st.get("irw_eps", 1e-4),
              sketch_apply=getattr(args, "sketch_apply", "auto"))
    barrier = barrier or (lambda: None)
    t_plan = time.perf_counter()
    plan = G.Plan(p.A, p.B, value_dtype=vdt, image_shape=img(args, p), slot_layout=args.slot_layout)
    torch.cuda.synchronize()
    t_plan = time.perf_counter() - t_plan
    stats = plan.stats()
    b_dev = torch.as_tensor(p.b, device="cuda")
    x_dev = torch.empty(p.A.shape[1], dtype=torch.float64, device="cuda")
    for _ in range(max(warmup, 3)):
        x_dev, info, _ = plan.solve(method, b_dev, out=x_dev, driver=args.driver, **kw)
    iters = info.iters
    xh = x_dev.cpu().numpy()
    err = float(np.linalg.norm(xh - p.x_true) / np.linalg.norm(p.x_true))
    stream = torch.cuda.current_stream()
    barrier()
    torch.cuda.synchronize()
    if sampler:
        sampler.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(steps):
        plan.solve(method, b_dev, out=x_dev, sync=False, driver=args.driver, **kw)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop() if sampler else None
    t_ms = ev0.elapsed_time(ev1)
    _, info_chk, _ = plan.solve(method, b_dev, out=x_dev, **kw)
    assert info_chk.iters == iters, "solve is not deterministic"
    # per-kernel launch durations (CUDA events around every launch, same solve)
    _, _, hp = plan.solve(method, b_dev, out=x_dev, driver="profiled", **kw)
    kms, kl = hp["kernel_ms"], hp["kernel_launches"]
    m, n = p.A.shape
    ell = st["window"]
    vb = {"f64": 8, "f32": 4, "bf16": 2}[vdt]
    xb = 8 if vdt == "f64" else 4
    fwd_bytes = spmv_bytes(stats["nnz_A"], m, n, vb, xb, ell + 1, 0, stats["index_bytes_A"])
    bwd_bytes = spmv_bytes(stats["nnz_At"], n, m, vb, xb, ell, 0, stats["index_bytes_At"])
    peaks = load_peaks()
    kern = {}
    for name, nbytes, nnz in (("spmv_fwd", fwd_bytes, stats["nnz_A"]), ("spmv_bwd", bwd_bytes, stats["nnz_At"])):
        avg_ms = kms[name] / max(kl[name], 1)
        gbs = nbytes / (avg_ms * 1e-3) / 1e9
        kern[name] = {"avg_us": 1000 * avg_ms, "launches": kl[name], "bytes": nbytes, "gbs": gbs,
                      "hbm_frac_of_measured": gbs / peaks["hbm_gbs"],
                      "tflops": 2 * nnz / (avg_ms * 1e-3) / 1e12,
                      "share": kms[name] / max(sum(kms.values()), 1e-12)}
    breakdown = {c: {"avg_us": 1000 * kms[c] / kl[c], "launches": kl[c], "share": kms[c] / max(sum(kms.values()), 1e-12)}
                 for c in kms if kl[c] > 0}
    dom = max(kern, key=lambda k: kern[k]["share"])
    roof = {"bound": "hbm", "achieved": kern[dom]["gbs"], "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": kern[dom]["gbs"] / peaks["hbm_gbs"],
            "traffic": recorded_traffic(dom, workload) if vdt == "f64" else None,
            "kernel": dom, "peak_source": peaks["source"],
            "algorithmic_bytes_per_launch": kern[dom]["bytes"], "avg_launch_us": kern[dom]["avg_us"]}
    out = {"workload": workload, "values": vdt, "vectors": "f64" if vdt == "f64" else "f32", "method": method,
           "t_ms": t_ms, "steps": steps, "iters": iters, "stop": info.status_name,
           "time_to_stop_ms": t_ms / steps, "iters_per_s": iters * steps / (t_ms / 1000),
           "rel_error_vs_x_true": err, "plan_build_s": t_plan, "stats": stats, "precond": precond,
           "roofline": roof, "kernels": kern, "kernel_breakdown": breakdown, "clocks": clocks, "x": xh}
    if e2e and args.driver == "graph":
        b_host = torch.from_numpy(np.ascontiguousarray(p.b)).pin_memory().numpy()
        x_host = torch.empty(n, dtype=torch.float64).pin_memory().numpy()
        for _ in range(2):
            plan.solve_host(method, b_host, x_out=x_host, **kw)
        barrier()
        t0 = time.perf_counter()
        for _ in range(steps):
            plan.solve_host(method, b_host, x_out=x_host, **kw)
        out["e2e_s"] = time.perf_counter() - t0
        out["e2e_bytes"] = (8 * m, 8 * n)
    plan.close()
    return out


def leg_summary(leg: dict) -> dict:
    """A single-solve leg as reported among the variants (no arrays)."""
    keep = ("values", "vectors", "method", "iters", "stop", "time_to_stop_ms", "iters_per_s", "rel_error_vs_x_true",
            "plan_build_s", "roofline", "kernels")
    d = {k: leg[k] for k in keep}
    d["value"], d["unit"] = leg["iters_per_s"], "iters/s"
    return d


def ct256_variants(args, G, wl, np, torch):
    """The 256x256 unmatched sFLSMR workload (A: 15.0M, B: 23.6M nonzeros,
    reweighting operator, s = 400, window 2, 2% noise): FP64, and FP32 values
    and vectors (FP64 coefficients and small QR)."""
    p = wl.make("ct256_sflsmr_unmatched")
    out = {}
    for vdt in ("f64", "f32"):
        leg = single_leg(args, G, wl, np, torch, p, vdt, steps=args.steps, warmup=3, workload="ct256_sflsmr_unmatched")
        out[vdt] = leg_summary(leg)
    out["unmatched_adjoint_mismatch"] = adjoint_mismatch(p, np)
    return out


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    import workloads as wl
    from paper_2605_22281_gb300 import api as G

    for flag, leg in (("only_batched", batched_variant), ("only_mixed", mixed_variant), ("only_diff", diff_variant),
                      ("only_decay", decay_variant), ("only_flsqr", flsqr_variant), ("only_deblur", deblur_variant),
                      ("only_matfree", matfree_variant)):
        if getattr(args, flag):
            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
            print(json.dumps(leg(args, G, wl, np, torch)), flush=True)
            return

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if not torch.cuda.is_available():
        raise RuntimeError("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    p = rank_problem(wl.make(args.workload, **({"N": args.image} if args.image else {})), rank, wl, np)
    st = p.settings
    leg = single_leg(args, G, wl, np, torch, p, "f64", steps=args.steps, warmup=args.warmup, world=world,
                     barrier=barrier, sampler=ClockSampler(local), e2e=True,
                     workload=args.workload if not args.image else f"{args.workload}@{args.image}")
    iters = leg["iters"]
    method = leg["method"]
    t_max_ms, total_iters, value = aggregate(gather_rank_values([leg["t_ms"], iters], world, "cuda"), args.steps)
    ms_per_step = t_max_ms / args.steps
    m, n = p.A.shape
    e2e = None
    if "e2e_s" in leg:
        e2e_all = [r[0] for r in gather_rank_values([leg["e2e_s"]], world, "cuda")]
        e2e = {"value": total_iters / max(e2e_all), "unit": "iters/s", "h2d_bytes_per_step": leg["e2e_bytes"][0],
               "d2h_bytes_per_step": leg["e2e_bytes"][1]}

    variants = {}
    if not args.no_variants:
        if args.workload == "ct1024_sflsqr":
            variants["mixed_ct1024_sflsqr"] = mixed_variant(args, G, wl, np, torch, x_fp64=leg["x"])
            variants["flsqr_vs_sflsqr_ct1024_30_steps"] = flsqr_variant(args, G, wl, np, torch)
        if args.workload != "ct256_sflsmr_unmatched":
            variants["ct256_sflsmr_unmatched"] = ct256_variants(args, G, wl, np, torch)
        variants["batched_ct512_64rhs_f32"] = batched_variant(args, G, wl, np, torch)
        variants["diff_ct256_16rhs_fixed_k"] = diff_variant(args, G, wl, np, torch)
        variants["deblur512_lowrank_rnd_50_steps"] = deblur_variant(args, G, wl, np, torch)
        variants["matrix_free_ct256_sflsmr_unmatched"] = matfree_variant(args, G, wl, np, torch)
        variants["decay_study_gaussian"] = decay_variant(args, G, wl, np, torch)
        variants["ct64_sflsqr"] = small_variant(args, G, wl, np, torch)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cap = ORACLE_SAMPLE_STEPS.get(args.workload)
        res = cpu_baseline_subprocess(args.workload, cap)
        if "iters" in res:
            host = os.cpu_count() or 1
            what = f"the first {res['iters']} steps" if cap else f"one full solve ({res['iters']} steps)"
            cpu = {"value": res["iters"] / res["seconds"], "unit": "iters/s", "cores": 1, "kind": "oracle",
                   "sample": f"{what} of the {args.workload} oracle solve ({res['seconds']:.1f} s, FP64, 1 thread; "
                             f"workload generation not timed)", "host_cores": host}
            # the same sample with every host core for BLAS (the sparse products stay single-threaded)
            res_all = cpu_baseline_subprocess(args.workload, cap, host)
            if "iters" in res_all:
                cpu["all_cores"] = {"value": res_all["iters"] / res_all["seconds"], "cores": host,
                                    "seconds": res_all["seconds"]}
        else:
            cpu = {"value": None, "unit": "iters/s", "cores": 1, "kind": "oracle", "sample": res.get("error", "")}

    # reset + ||b|| pass + A^T w_1 + initial sketch(es), six kernels per step, x = Z y
    launches_per_step = 1 + 2 + (2 if method == "sflsmr" else 1) + 6 * iters + 1
    if rank == 0:
        stats = leg["stats"]
        opnd = stats["nnz_A"] * 12 + stats["nnz_At"] * 12
        line = {"metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": args.workload + (f" at {p.N}x{p.N} (profiling size)" if args.image else ""),
                           "method": method, "image": f"{p.N}x{p.N}",
                           "angles": p.n_angles, "bins": p.n_bins, "m": m, "n": n, "nnz_A": stats["nnz_A"],
                           "nnz_B_or_At": stats["nnz_At"], "s": st["s"], "zeta": st["zeta"], "window": st["window"],
                           "maxit": st["maxit"], "precond": leg["precond"], "iters_to_stop": iters,
                           "stop": leg["stop"], "time_to_stop_ms": ms_per_step,
                           "rel_error_vs_x_true": leg["rel_error_vs_x_true"], "plan_build_s": leg["plan_build_s"],
                           "l2": f"inputs larger than L2 (operators {opnd / 1e6:.0f} MB > 129 MB); no flush",
                           "parallelism": f"replicas x{world} (independent problems)",
                           "driver": args.driver, "unmatched_adjoint_mismatch": adjoint_mismatch(p, np)},
                "roofline": leg["roofline"], "kernels": leg["kernels"], "kernel_breakdown": leg["kernel_breakdown"],
                "clocks": leg["clocks"], "e2e": e2e,
                "gpu_launches": launches_per_step * args.steps,
                "cpu_baseline": cpu, "variants": variants}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse_args()
    if args.oracle_sample:
        oracle_sample_main(args.workload, args.oracle_sample)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
