"""Benchmark: eigenpairs/s of the DACG-Newton solve on the 100^3 variable-
coefficient diffusion matrix (n = 1e6, 7-point, p = 10, IC(10, 1e-3),
relative residual 1e-8), with the inner-PCG HBM roofline.

A "step" is one complete nle_solve: DACG + Newton with every inner PCG
iteration for all p eigenpairs, inputs (factored matrix, start vectors)
resident on the device.  The IC factorisation is set-up and is reported
separately (``ic_seconds``), as the paper reports its "IC CPU" column.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision mixed|fp64]
  python bench.py --impl reference ...    # the oracle on the host cores

Under torchrun (N > 1) every rank solves its own replica of the problem (a
single problem does not shard: the IC triangular solves are one global
recurrence) and rank 0 prints the line.
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "diff3d7_100"
WORKLOAD_P = 10
CPU_SAMPLE_PAIRS = 3  # bounded oracle sample of the CPU baseline: the first eigenpairs of the workload
REF_STEP_PAIRS = 1    # the reference arm's step: the first eigenpair (a few seconds of oracle work)
FP64_STEPS = 3        # timed steps of the plain FP64 arm (its warm-up: 1 step)
METRIC = "eigenpairs/s at n=1e6, rel. residual 1e-8"
DESCRIPTION = {
    "diff3d7_100": "3D 7-point diffusion 100^3, exp(Gaussian field) faces",
    "diff2d5_600x700": "2D 5-point diffusion 600x700, lognormal cells, harmonic-mean faces",
    "hex27_96": "27-point trilinear hex stiffness, 96^3 interior nodes, lognormal elements",
}
UNIT = "eigenpairs/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default=None, choices=["mixed", "fp64"], help="default: mixed")
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 arm (profiling runs)")
    ap.add_argument("--skip-e2e", action="store_true", help="profiling runs: skip the host-buffer pass")
    ap.add_argument("--no-ic-host", action="store_true", help="skip the host IC factor timed for comparison")
    ap.add_argument("--pairs", type=int, default=0, help="profiling runs: solve only the first P eigenpairs")
    ap.add_argument("--trsv-warps", type=int, default=0, help="0 = library default")
    ap.add_argument("--ordering", default="natural", choices=["natural", "mc1", "mc2"],
                    help="symmetric ordering before the IC factor (natural = the paper's)")
    ap.add_argument("--bfgs", default="simplified", choices=["simplified", "full"],
                    help="BFGS update of the preconditioner (simplified = the paper's eq. lastprec)")
    ap.add_argument("--max-newton", type=int, default=0,
                    help="outer step cap; 0 = the workload's (the paper's ITMAX = 100; 400 for workloads with "
                         "eigenvalue clusters)")
    ap.add_argument("--spin-timeout", type=float, default=0.0, help="0 = library default (seconds)")
    ap.add_argument("--batch-ctas", type=int, default=0, help="graph batch: CTAs per problem (0: 4 mixed, 8 FP64)")
    ap.add_argument("--schedule", default="auto", choices=["auto", "level", "chain"],
                    help="schedule of the triangular solves (auto = timed at set-up, the faster kept)")
    ap.add_argument("--cpu-sample", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--sample-eigenpairs", type=int, default=1, help=argparse.SUPPRESS)
    return ap.parse_args()


# ---------------------------------------------------------------------------
# oracle timing (CPU baseline and the reference arm)
# ---------------------------------------------------------------------------

def cpu_sample(workload: str, npairs: int) -> dict:
    """Time the oracle, as it stands, on the first `npairs` eigenpairs of the
    workload (IC set-up excluded).  Runs in this process: the caller starts
    it as a single-threaded subprocess."""
    import oracle as O
    import workloads as W

    A, st = W.workload(workload)
    ic = O.ic_factor(A, st["lfil"], st["tau_ic"])
    X0 = W.start_vectors(A.n, npairs, st["seed"])
    opt = O.OracleOptions(tol=st["tol"], lfil=st["lfil"], tau_ic=st["tau_ic"], max_newton=st.get("max_newton", 100))
    t0 = time.perf_counter()
    lam, V, stats = O.dacg_newton(A, npairs, X0, opt, ic=ic)
    sec = time.perf_counter() - t0
    return dict(seconds=sec, eigenpairs=npairs, lam=[float(x) for x in lam])


BATCH = "graph_batch"
BATCH_P = 4
BATCH_SAMPLE = 10  # problems of the batch timed on the oracle (at most ~25 s)
# the larger graphs have lambda_2 and lambda_3 within 0.4 % of each other; the
# oracle needs up to ~170 Newton steps there
BATCH_MAX_NEWTON = 400


def batch_problem_start(A, b: int):
    import workloads as W

    return W.graph_batch_start(A, b, BATCH_P)


def cpu_sample_batch() -> dict:
    """The oracle, as it stands, on the first problems of the batched
    workload (up to BATCH_SAMPLE problems or about 25 s)."""
    import oracle as O
    import workloads as W

    mats = W.graph_batch(count=BATCH_SAMPLE)
    sec, pairs = 0.0, 0
    for b, A in enumerate(mats):
        ic = O.ic_factor(A, 30, 1e-2)
        t0 = time.perf_counter()
        O.dacg_newton(A, BATCH_P, batch_problem_start(A, b),
                      O.OracleOptions(tol=1e-8, lfil=30, tau_ic=1e-2, max_newton=BATCH_MAX_NEWTON), ic=ic)
        sec += time.perf_counter() - t0
        pairs += BATCH_P
        if sec > 25.0:
            break
    return dict(seconds=sec, eigenpairs=pairs, problems=pairs // BATCH_P)


def run_cpu_sample(workload: str, npairs: int) -> dict:
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-sample", "--workload", workload,
                        "--sample-eigenpairs", str(npairs)], env=env, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("oracle sample failed: " + r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def golden(workload: str):
    """The stored oracle run of a workload (tests/golden/<name>.json, written
    by tests/golden/make_golden.py from the oracle alone), or None."""
    try:
        with open(os.path.join(ROOT, "tests", "golden", f"{workload}.json")) as fh:
            return json.load(fh)
    except Exception:
        return None


def cpu_baseline_entry(res: dict, workload: str) -> dict:
    e = dict(value=res["eigenpairs"] / res["seconds"], unit=UNIT, cores=1, nproc=os.cpu_count(), kind="oracle",
             sample=f"oracle (numpy + plain C, FP64, 1 thread) on eigenpairs 1-{res['eigenpairs']} of {workload} "
                    f"({res['seconds']:.1f} s, IC set-up excluded); later eigenpairs cost more (more deflation "
                    f"columns, more Newton steps), so the sample overstates the oracle's rate for all pairs")
    g = golden(workload)
    if g and g.get("oracle_seconds"):
        e["full_run"] = dict(value=g["p"] / g["oracle_seconds"], seconds=g["oracle_seconds"], eigenpairs=g["p"],
                             where="the stored oracle run of tests/golden (all pairs, 1 process; measured on the "
                                   "development host, not on this machine)")
    return e


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    times = []
    for i in range(args.warmup + args.steps):
        res = run_cpu_sample(args.workload, REF_STEP_PAIRS)
        if i >= args.warmup:
            times.append(res["seconds"])
    total = sum(times)
    value = REF_STEP_PAIRS * args.steps / total
    line = dict(impl="reference", metric=METRIC, value=value, unit=UNIT, n_gpus=args.gpus, steps=args.steps,
                warmup=args.warmup, ms_per_step=1000 * total / args.steps, higher_is_better=True, scaling="weak",
                vs_baseline=None, dtype="f64", data="synthetic",
                config=dict(workload=args.workload,
                            sample=f"eigenpair 1-{REF_STEP_PAIRS} per step (DACG + Newton), IC set-up excluded"),
                cpu_baseline=dict(value=value, unit=UNIT, cores=1, nproc=os.cpu_count(), kind="oracle",
                                  sample=f"eigenpair 1-{REF_STEP_PAIRS} of the workload per step, 1 thread (the "
                                         f"cheapest eigenpair: this overstates the rate over all pairs)"),
                e2e=dict(value=value, unit=UNIT, h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        import tempfile

        fd, self.path = tempfile.mkstemp(prefix=f"nle_clocks_rank{index}_", suffix=".csv")
        os.close(fd)

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return dict(sm_mhz=None, sm_max_mhz=None, reasons=["nvidia-smi unavailable"])
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1]))
                    smax.append(float(f[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, f[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        return dict(sm_mhz=statistics.median(sm) if sm else None, sm_max_mhz=max(smax) if smax else None,
                    reasons=sorted(reasons), samples=len(sm))


# ---------------------------------------------------------------------------
# roofline accounting
# ---------------------------------------------------------------------------

def alg_bytes(n, nnz_a, nnz_l, w, its, sum_m, sum_k, kind):
    """Algorithmic HBM bytes of `its` iterations.

    Matrix terms: B_A = nnz_A (w + 4) + 4 (n + 1), B_L = nnz_L (w + 4) + 4 (n + 1)
    (values + int32 column indices + row pointers).
    Inner PCG iteration (fused schedule): B_A + 2 B_L + (16 + 4k + 4m) n w.
    DACG iteration: B_A + 2 B_L + (16 + 2m) n w.
    """
    BA = nnz_a * (w + 4) + 4 * (n + 1)
    BL = nnz_l * (w + 4) + 4 * (n + 1)
    V = n * w
    if kind == "pcg":
        return its * (BA + 2 * BL + 16 * V) + 4 * V * (sum_k + sum_m)
    return its * (BA + 2 * BL + 16 * V) + 2 * V * sum_m


def kernel_hash() -> str:
    """Hash of the code the solver kernels and their data layout come from
    (every source except the device IC factor's own translation unit, which
    they do not include), comments and blank space removed, so that a
    captured traffic figure stays valid across comment-only edits."""
    import re

    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_1312_1553_gb300", "csrc")
    for f in sorted(os.listdir(d)):
        if f.startswith("nle_ict."):
            continue
        with open(os.path.join(d, f), encoding="utf-8") as fh:
            code = fh.read()
        code = re.sub(r"/\*.*?\*/", " ", code, flags=re.S)
        code = re.sub(r"//[^\n]*", " ", code)
        h.update(f.encode() + b"\0" + " ".join(code.split()).encode())
    return h.hexdigest()[:16]


def load_traffic(kernel: str, workload: str):
    """ncu dram bytes per launch of `kernel` on `workload` (the bench's
    launch configuration), if captured for the current sources."""
    p = os.path.join(ROOT, "profiles", "traffic.txt")
    try:
        with open(p) as fh:
            t = json.load(fh)
    except Exception:
        return None
    e = t.get(kernel)
    if not e or e.get("kernel_hash") != kernel_hash() or e.get("workload") != workload:
        return None
    return e.get("bytes_per_launch")


def max_over_ranks(values, device="cuda"):
    """Element-wise maximum of per-rank timings (seconds) over all ranks of
    the default process group; the values themselves when there is none.
    Replicas run independently, so the job's time is the slowest rank's."""
    import torch

    if not (torch.distributed.is_available() and torch.distributed.is_initialized()):
        return [float(v) for v in values]
    tt = torch.tensor([float(v) for v in values], device=device, dtype=torch.float64)
    torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
    return [float(v) for v in tt]


def replica_throughput(world: int, units_per_rank_step: int, steps: int, t_max: float) -> float:
    """Whole-job throughput of `world` independent replicas (weak scaling):
    all units processed by all ranks over the slowest rank's time."""
    return world * units_per_rank_step * steps / t_max


def peak_hbm():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def batch_main(args, world, rank, local, cpu):
    """Batched workload: 256 grounded geometric-graph Laplacians, p = 4 each,
    solved by one nle_batch_solve per step (one persistent launch, groups
    of 4 CTAs taking problems from a device queue)."""
    import torch

    import workloads as W
    from paper_1312_1553_gb300 import _build, nle

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    _build.build()
    nle.load_library()
    mats = W.graph_batch(count=256)
    max_newton = args.max_newton or BATCH_MAX_NEWTON
    prec = nle.NLE_FP64 if args.precision == "fp64" else nle.NLE_MIXED
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        t0 = time.perf_counter()
        solvers = []
        for A in mats:
            # FP64 needs 8 CTAs per problem for the largest graphs (n = 60,000)
            ctas = args.batch_ctas or (4 if prec == nle.NLE_MIXED else 8)
            s = nle.Eigensolver(A, dict(precision=prec, grid_ctas=ctas, trsv_schedule=nle.NLE_SCHED_LEVEL),
                                stream=stream)
            s.factor_ic(30, 1e-2)
            solvers.append(s)
        ic_seconds = time.perf_counter() - t0
        ics = [s.last_stats()["ic"] for s in solvers]
        ic_info = dict(on_device=sum(i["on_device"] for i in ics), problems=len(ics),
                       factor_ms=sum(i["factor_ms"] for i in ics), kernel_ms=sum(i["kernel_ms"] for i in ics))
        nnz_l = [int(s.get_factor()["Lrowptr"][-1]) for s in solvers]
        X0h = [torch.tensor(batch_problem_start(A, b), dtype=torch.float64).pin_memory() for b, A in enumerate(mats)]
        X0d = [x.to("cuda") for x in X0h]
        count = len(solvers)
        H = (ctypes.c_void_p * count)(*[s.h.value for s in solvers])
        lams = [torch.empty(BATCH_P, dtype=torch.float64, device="cuda") for _ in solvers]
        Vs = [torch.empty((BATCH_P, s.n), dtype=torch.float64, device="cuda") for s in solvers]
        L = (ctypes.c_void_p * count)(*[t.data_ptr() for t in lams])
        V = (ctypes.c_void_p * count)(*[t.data_ptr() for t in Vs])
        X = (ctypes.c_void_p * count)(*[t.data_ptr() for t in X0d])
        per = (ctypes.c_int * count)()

        def step():
            rc = nle.nle_batch_solve(count, H, BATCH_P, 1e-8, max_newton, 20, X, L, V, per)
            if rc not in (0, 5):  # 5 = NLE_ERR_NOCONV: counted below, outputs written
                raise nle.NLEError(rc, nle.nle_last_error(solvers[0].h))

        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        clk = ClockSampler(local)
        clk.start()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        ms_kernel = 0.0
        for _ in range(args.steps):
            step()
            ms_kernel += solvers[0].last_stats()["ms_batch"]
        ev1.record(stream)
        torch.cuda.synchronize()
        clocks = clk.stop()
        ms = ev0.elapsed_time(ev1)
        stats = [s.last_stats() for s in solvers]
        unconverged = [b for b in range(count) if per[b] != 0]
        # end to end: start vectors from pinned host memory in, eigenvalues out
        lam_h = torch.empty((count, BATCH_P), dtype=torch.float64).pin_memory()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        if not args.skip_e2e:
            for _ in range(args.steps):
                for b in range(count):
                    X0d[b].copy_(X0h[b], non_blocking=True)
                step()
                for b in range(count):
                    lam_h[b].copy_(lams[b], non_blocking=True)
                torch.cuda.synchronize()
        e2e_sec = max(time.perf_counter() - t0, 1e-9)
        for s in solvers:
            s.close()
    t_max, e2e_max = max_over_ranks([ms / 1000.0, e2e_sec])
    if args.skip_e2e:
        e2e_max = float("inf")
    pairs = count * BATCH_P
    w = 4 if prec == nle.NLE_MIXED else 8
    b_step = sum(alg_bytes(A.n, A.nnz, nl, w, st["pcg_iterations"], st["pcg_sum_m"], st["pcg_sum_k"], "pcg") +
                 alg_bytes(A.n, A.nnz, nl, w, st["dacg_iterations"], st["dacg_sum_m"], 0, "dacg")
                 for A, nl, st in zip(mats, nnz_l, stats))
    ms_launch = ms_kernel / args.steps
    peak, peak_kind = peak_hbm()
    achieved = (b_step / 1e9) / (ms_launch / 1e3)
    line = dict(metric=f"eigenpairs/s, {count} graph Laplacians batched, rel. residual 1e-8",
                value=replica_throughput(world, pairs, args.steps, t_max), unit=UNIT, n_gpus=world, steps=args.steps,
                warmup=args.warmup, ms_per_step=1000 * t_max / args.steps, higher_is_better=True, scaling="weak",
                vs_baseline=None, dtype="f32" if prec == nle.NLE_MIXED else "f64", data="synthetic",
                config=dict(workload=f"{BATCH}: {count} random geometric graph Laplacians + 1e-3 I, "
                                     f"n ~ U[2000, 60000], p = {BATCH_P}",
                            n_total=sum(A.n for A in mats), nnz_total=sum(A.nnz for A in mats), lfil=30, tau_ic=1e-2,
                            tol=1e-8, ic_seconds=ic_seconds, ic_factor=ic_info, l2="working set > 129 MB L2 (no flush needed)",
                            parallelism=f"replicas{world}" if world > 1 else
                            f"single GPU, groups of {args.batch_ctas or (4 if prec == nle.NLE_MIXED else 8)} CTAs"),
                roofline=dict(bound="hbm", achieved=achieved, peak=peak, unit="GB/s", frac=achieved / peak,
                              traffic=load_traffic("k_batch", BATCH), kernel="k_batch",
                              peak_source=f"{peak_kind} hbm_gbs (MEASURED_PEAKS.json)" if peak_kind == "measured"
                              else "fallback 6.8 TB/s", alg_bytes_per_launch=b_step, ms_per_launch=ms_launch),
                cpu_baseline=cpu,
                e2e=None if args.skip_e2e else dict(
                    value=replica_throughput(world, pairs, args.steps, e2e_max), unit=UNIT,
                    h2d_bytes_per_step=sum(x.numel() * 8 for x in X0h), d2h_bytes_per_step=count * BATCH_P * 8),
                clocks=clocks, gpu_launches=args.steps * (1 + count * (BATCH_P + 1)),
                iterations=dict(pcg=sum(st["pcg_iterations"] for st in stats),
                                dacg=sum(st["dacg_iterations"] for st in stats)),
                unconverged=dict(problems=len(unconverged), max_newton=max_newton,
                                 detail=[dict(problem=b, n=mats[b].n, outer_its=stats[b]["outer_its"],
                                              final_res=stats[b]["final_res"]) for b in unconverged[:8]]))
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.cpu_sample:
        print(json.dumps(cpu_sample_batch() if args.workload == BATCH else
                         cpu_sample(args.workload, args.sample_eigenpairs)))
        return 0
    if args.impl == "reference":
        return reference_arm(args)
    if args.warmup < 3:
        print("warning: --warmup < 3 is below the timing rules", file=sys.stderr)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    # CPU baseline before any GPU work (rank 0, N = 1 only)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            if args.workload == BATCH:
                r = run_cpu_sample(BATCH, 0)
                cpu = dict(value=r["eigenpairs"] / r["seconds"], unit=UNIT, cores=1, kind="oracle",
                           sample=f"oracle (numpy + plain C, FP64, 1 thread) on problems 1-{r['problems']} of the "
                                  f"batch, p = {BATCH_P} each ({r['seconds']:.1f} s, IC set-up excluded)")
            else:
                cpu = cpu_baseline_entry(run_cpu_sample(args.workload, CPU_SAMPLE_PAIRS), args.workload)
        except Exception as e:  # reported, not fatal
            cpu = dict(value=None, unit=UNIT, cores=1, kind="oracle", sample=f"failed: {e}")
    if args.workload == BATCH:
        return batch_main(args, world, rank, local, cpu)

    import numpy as np
    import torch

    import workloads as W
    from paper_1312_1553_gb300 import _build, nle

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    _build.build()
    nle.load_library()

    A, st = W.workload(args.workload)
    p = args.pairs if args.pairs > 0 else st["p"]
    max_newton = args.max_newton or st.get("max_newton", 100)
    X0 = W.start_vectors(A.n, p, st["seed"])
    prec = nle.NLE_FP64 if args.precision == "fp64" else nle.NLE_MIXED
    opts = dict(precision=prec)
    if args.trsv_warps > 0:
        opts["trsv_warps"] = args.trsv_warps
    if args.spin_timeout > 0:
        opts["spin_timeout_s"] = args.spin_timeout
    opts["ordering"] = {"natural": nle.NLE_ORDER_NATURAL, "mc1": nle.NLE_ORDER_MULTICOLOR1,
                        "mc2": nle.NLE_ORDER_MULTICOLOR2}[args.ordering]
    opts["bfgs_update"] = nle.NLE_BFGS_FULL if args.bfgs == "full" else nle.NLE_BFGS_SIMPLIFIED
    opts["trsv_schedule"] = {"auto": nle.NLE_SCHED_AUTO, "level": nle.NLE_SCHED_LEVEL,
                             "chain": nle.NLE_SCHED_CHAIN}[args.schedule]
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        s = nle.Eigensolver(A, opts, stream=stream)
        t0 = time.perf_counter()
        s.factor_ic(st["lfil"], st["tau_ic"])
        ic_seconds = time.perf_counter() - t0
        ic_stats = s.last_stats()["ic"]
        ic_info = dict(where="device" if ic_stats["on_device"] else "host", factor_ms=ic_stats["factor_ms"],
                       kernel_ms=ic_stats["kernel_ms"], setup_ms=ic_stats["setup_ms"])
        if ic_stats["on_device"] and not args.no_ic_host and rank == 0:
            # the same factor computed on the host, for comparison (set-up only)
            sh = nle.Eigensolver(A, dict(opts, ic_device=nle.NLE_IC_HOST, trsv_schedule=nle.NLE_SCHED_LEVEL),
                                 stream=stream)
            sh.factor_ic(st["lfil"], st["tau_ic"])
            ic_info["host_factor_ms"] = sh.last_stats()["ic"]["factor_ms"]
            sh.close()
        F = s.get_factor()
        nnz_l = int(F["Lrowptr"][-1])
        x0 = torch.tensor(X0, dtype=torch.float64, device="cuda")
        lam = torch.empty(p, dtype=torch.float64, device="cuda")
        V = torch.empty((p, A.n), dtype=torch.float64, device="cuda")

        def step():
            stats = nle.nle_stats()
            rc = nle.nle_solve(s.h, p, st["tol"], max_newton, 20, nle._dptr(x0), nle._dptr(lam), nle._dptr(V), stats, 1)
            if rc != 0:
                raise nle.NLEError(rc, nle.nle_last_error(s.h))
            return nle.stats_dict(stats)

        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        clk = ClockSampler(local)
        clk.start()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev0.record(stream)
        all_stats = [step() for _ in range(args.steps)]
        ev1.record(stream)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        clocks = clk.stop()
        ms = ev0.elapsed_time(ev1)
        # end to end through the C ABI with host buffers (pinned), copies inside
        x0_h = torch.tensor(X0, dtype=torch.float64).pin_memory()
        lam_h = torch.empty(p, dtype=torch.float64).pin_memory()
        V_h = torch.empty((p, A.n), dtype=torch.float64).pin_memory()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(0 if args.skip_e2e else args.steps):
            stats = nle.nle_stats()
            rc = nle.nle_solve(s.h, p, st["tol"], max_newton, 20, nle._dptr(x0_h), nle._dptr(lam_h), nle._dptr(V_h),
                               stats, 0)
            if rc != 0:
                raise nle.NLEError(rc, nle.nle_last_error(s.h))
            _ = float(lam_h[0])
        e2e_sec = max(time.perf_counter() - t0, 1e-9)
        lam_dev = lam.cpu().numpy()
        V_dev = V.cpu().numpy()
        s.close()
        # the plain FP64 form of the same solve (the baseline of the mixed
        # form's speed-up), same schedule option, fewer steps
        fp64 = None
        if prec == nle.NLE_MIXED and not args.no_fp64:
            o64 = dict(opts, precision=nle.NLE_FP64)
            s64 = nle.Eigensolver(A, o64, stream=stream)
            s64.factor_ic(st["lfil"], st["tau_ic"])
            lam64 = torch.empty(p, dtype=torch.float64, device="cuda")
            V64 = torch.empty((p, A.n), dtype=torch.float64, device="cuda")

            def step64():
                stats = nle.nle_stats()
                rc = nle.nle_solve(s64.h, p, st["tol"], max_newton, 20, nle._dptr(x0), nle._dptr(lam64),
                                   nle._dptr(V64), stats, 1)
                if rc != 0:
                    raise nle.NLEError(rc, nle.nle_last_error(s64.h))
                return nle.stats_dict(stats)

            step64()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st64 = [step64() for _ in range(FP64_STEPS)]
            e1.record(stream)
            torch.cuda.synchronize()
            ms64 = e0.elapsed_time(e1)
            fp64 = dict(value=p * FP64_STEPS / (ms64 / 1000.0), unit=UNIT, ms_per_step=ms64 / FP64_STEPS,
                        steps=FP64_STEPS, warmup=1, trsv_schedule=st64[-1]["trsv_schedule"],
                        iterations=dict(pcg=st64[-1]["pcg_iterations"], dacg=st64[-1]["dacg_iterations"]))
            lam64_h = lam64.cpu().numpy()
            s64.close()

    # max over ranks
    t_max, e2e_max = max_over_ranks([ms / 1000.0, e2e_sec])
    if args.skip_e2e:
        e2e_max = float("inf")
    value = replica_throughput(world, p, args.steps, t_max)
    e2e_value = replica_throughput(world, p, args.steps, e2e_max)

    # roofline of the dominant kernel (Newton phase or DACG phase)
    w = 4 if prec == nle.NLE_MIXED else 8
    ms_newton = sum(x["ms_newton"] for x in all_stats)
    ms_dacg = sum(x["ms_dacg"] for x in all_stats)
    its = sum(x["pcg_iterations"] for x in all_stats)
    b_newton = alg_bytes(A.n, A.nnz, nnz_l, w, its, sum(x["pcg_sum_m"] for x in all_stats),
                         sum(x["pcg_sum_k"] for x in all_stats), "pcg")
    dits = sum(x["dacg_iterations"] for x in all_stats)
    b_dacg = alg_bytes(A.n, A.nnz, nnz_l, w, dits, sum(x["dacg_sum_m"] for x in all_stats), 0, "dacg")
    peak, peak_kind = peak_hbm()
    launches_per_step = p  # one persistent launch of each phase kernel per eigenpair
    kern = "k_newton" if ms_newton >= ms_dacg else "k_dacg"
    b, msk = (b_newton, ms_newton) if kern == "k_newton" else (b_dacg, ms_dacg)
    achieved = (b / 1e9) / (msk / 1e3)
    nlaunch = launches_per_step * args.steps
    traffic = load_traffic(kern, args.workload) if not (args.ordering != "natural" or args.bfgs != "simplified" or
                                                       prec != nle.NLE_MIXED or args.pairs) else None
    roof = dict(bound="hbm", achieved=achieved, peak=peak, unit="GB/s", frac=achieved / peak, traffic=traffic,
                kernel=kern, peak_source=f"{peak_kind} hbm_gbs (MEASURED_PEAKS.json)" if peak_kind == "measured" else
                "fallback 6.8 TB/s", alg_bytes_per_launch=b / nlaunch, ms_per_launch=msk / nlaunch,
                other=dict(kernel="k_dacg" if kern == "k_newton" else "k_newton",
                           achieved=((b_dacg if kern == "k_newton" else b_newton) / 1e9) /
                           (max(ms_dacg if kern == "k_newton" else ms_newton, 1e-9) / 1e3)))
    # error against the stored FP64 oracle run: eigenvalues (relative) and
    # eigenvectors (CountSketch estimate of ||v - v_oracle||, which is the
    # angle between them to first order)
    accuracy = None
    g = golden(args.workload)
    if g and g["p"] == p and "sketch_V" in g:
        lam_g = np.array(g["lam"])
        bucket, sign = W.count_sketch_hash(A.n, g["sketch_K"], g["sketch_seed"])
        ang = []
        for j in range(p):
            sk = W.count_sketch(V_dev[j], bucket, sign, g["sketch_K"])
            ref = np.array(g["sketch_V"][j])
            ang.append(float(min(np.linalg.norm(sk - ref), np.linalg.norm(sk + ref))))
        accuracy = dict(vs="stored FP64 oracle run (tests/golden)", max_rel_eig_err=float(np.max(np.abs(lam_dev - lam_g) / lam_g)),
                        max_vec_angle_sketch=max(ang), vec_angle_sketch=ang)
        if fp64 is not None:
            fp64["max_rel_eig_err"] = float(np.max(np.abs(lam64_h - lam_g) / lam_g))
    metric = METRIC if args.workload == WORKLOAD else f"eigenpairs/s, {args.workload}, rel. residual {st['tol']:g}"
    line = dict(metric=metric, value=value, unit=UNIT, n_gpus=world, steps=args.steps, warmup=args.warmup,
                ms_per_step=1000 * t_max / args.steps, higher_is_better=True, scaling="weak", vs_baseline=None,
                dtype="f32" if prec == nle.NLE_MIXED else "f64", data="synthetic",
                config=dict(workload=f"{args.workload}: {DESCRIPTION.get(args.workload, args.workload)}",
                            n=A.n, nnz=A.nnz, p=p, lfil=st["lfil"], tau_ic=st["tau_ic"], tol=st["tol"],
                            precision="FP32 bulk + FP64 outer step" if prec == nle.NLE_MIXED else "FP64",
                            nnz_L=nnz_l, nlev_L=F["nlevL"], ordering=args.ordering, bfgs=args.bfgs, ic_seconds=ic_seconds,
                            ic_factor=ic_info,
                            trsv_schedule=all_stats[-1]["trsv_schedule"], schedule_request=args.schedule,
                            tune_ms=all_stats[-1]["tune_ms"], strands=all_stats[-1]["strands"],
                            l2="working set > 129 MB L2 (no flush needed)",
                            parallelism=f"replicas{world}" if world > 1 else "single GPU"),
                roofline=roof, cpu_baseline=cpu,
                e2e=None if args.skip_e2e else dict(value=e2e_value, unit=UNIT, h2d_bytes_per_step=p * A.n * 8,
                                                    d2h_bytes_per_step=p * A.n * 8 + p * 8),
                clocks=clocks, gpu_launches=int(sum(x["kernel_launches"] for x in all_stats)),
                phase_ms=dict(dacg=ms_dacg / args.steps, newton=ms_newton / args.steps),
                pass_ms={k: sum(x["ms_phase"][k] for x in all_stats) / args.steps for k in nle.PHASES},
                iterations=dict(pcg=its / args.steps, dacg=dits / args.steps),
                lambda_first=float(lam_dev[0]), accuracy=accuracy, fp64=fp64,
                mixed_over_fp64=(value / fp64["value"]) if fp64 else None)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
