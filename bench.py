#!/usr/bin/env python3
"""Time-to-tolerance of IterativeCUR (arXiv 2509.21963, Algorithm 1) on GB300.

Default workload (one "step" = one complete cur_run to tolerance):
  A = U diag(i^-2) V^T + noise, 20000 x 20000 FP64 (U, V thin orthonormal factors
  of rank 2000 from QR of seeded Gaussians; i.i.d. N(0, (1e-8)^2) noise),
  tol 1e-2, block size b = 50, sketch rows c = floor(1.1 b) = 55, seed 0, the
  FP64 form of the sketch on the tensor cores (CUR_SKETCH_F64_TC: exact sketch
  of the 52-bit fixed point of A by the 8-bit Gaussian sketch; every later step
  FP64).  With this noise (1.85e-4 of ||A||_F) the cross approximation stalls
  near rho ~ 1.2e-3, so 1e-2 is the tolerance of the family that the method
  reaches; the line also reports the same step with the FP64-pipe Gaussian
  sketch, tol 1e-3 and 1e-4 on the same spectrum with N(0, (1e-10)^2) noise,
  and the FP32 matrix with the FP64 sketch and with the two-digit tensor-core
  sketch.  A (3.2 GB) is resident in HBM and larger than L2, so no L2 flush is
  needed.

Prints ONE JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle
instead (the reference arm: one whole oracle run per step on the host cores).
Under torchrun every rank runs an independent replica (the method has no
data-parallel exchange): value = max-over-ranks time / (ranks x steps).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import re
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# dram bytes (read + write) of one sketch launch, from the committed ncu capture
# summarised in profiles/; valid only while the kernel source is unchanged.
# profiles/sketch_f64_simt_8000x4000.md: 259.5 MB read + 65.8 MB written at 8000 x 4000
# (split-K 50); at 20000^2 (split-K 12) reads scale with m*n (3244 MB) and the partial
# writes with ks*c*n at the measured write ratio (79 MB).  The fingerprint is of the
# file's code with // comments removed; it was moved once since the capture, when
# host-side row-block launchers were appended to the file (the kernel unchanged).
TRAFFIC = {"sketch_simt.cu": {"sha1": "31824a3eff0a3f330025c2a908a52893a001d576",
                              "bytes_per_launch_full": 3.323e9},
           # profiles/sketch_fx_8192x4096_c55.md: 277.4 MB read + 4.1 MB written at 8192 x 4096;
           # at 20000^2 reads scale with m*n (3307 MB) and the int64 sum writes with c*n (20 MB)
           "sketch_fx.cu": {"sha1": "340702b5a6bcfaeedd52420c55205b9dc38e1f06", "bytes_per_launch_full": 3.327e9}}
FP64_PEAK_TFLOPS = 1.25  # GB300 nominal FP64 rate; the line reports the measured one beside it


def hbm_peak():
    """Measured copy bandwidth of the GB300s this runs on (MEASURED_PEAKS.json),
    else 6800 GB/s, an earlier copy measurement on a GB300."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


HBM_GBS, HBM_SRC = hbm_peak()


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--m", type=int, default=20000)
    p.add_argument("--n", type=int, default=20000)
    p.add_argument("--dtype", choices=["f64", "f32"], default="f64")
    p.add_argument("--sketch-mode", type=int, default=None,
                   help="0 FP64-pipe Gaussian sketch; 1-4 tensor-core precision form with 1-4 "
                        "digits (FP32 A); 5 FP64 tensor-core form (FP64 A).  Default: 5 for "
                        "FP64 A, 0 for FP32 A")
    p.add_argument("--tol", type=float, default=1e-2)
    p.add_argument("--block", type=int, default=50)
    p.add_argument("--sketch", type=int, default=55)
    p.add_argument("--noise", type=float, default=1e-8)
    p.add_argument("--seed", type=int, default=0)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-second-form", action="store_true")
    p.add_argument("--no-extra-forms", action="store_true",
                   help="skip the FP64-pipe, tol 1e-4 and FP32 forms")
    p.add_argument("--second-tol", type=float, default=1e-3)
    p.add_argument("--second-noise", type=float, default=1e-10)
    p.add_argument("--e2e-steps", type=int, default=3)
    p.add_argument("--paper-workload", action="store_true",
                   help="time the Low-Rank matrix of Sec. 5.1 (30000^2 FP64, G1 G2^T of rank "
                        "2000, tol 1e-6, b = 250; the paper reports 12 s on a 48-core CPU) even with "
                        "--no-extra-forms (it runs with the other forms by default)")
    p.add_argument("--workload", choices=["primary", "batch", "serve", "precision", "sketch"],
                   default="primary",
                   help="batch: 4096 independent FP32 matrices (m, n log-uniform in [64, 2048], "
                        "spectra exp(-i/20) / i^-1.5 / exact rank U[5,200]), tol 1e-4, b = c = 8, "
                        "all in one persistent launch; one step = the whole batch")
    p.add_argument("--batch-jobs", type=int, default=4096)
    p.add_argument("--batch-uniform", type=int, default=0,
                   help="every job N x N (with --batch-kind) instead of the mixed recipe")
    p.add_argument("--batch-kind", choices=["exp20", "poly1.5", "rank"], default="poly1.5")
    p.add_argument("--serve-requests", type=int, default=300)
    p.add_argument("--serve-rate", type=float, default=200.0, help="Poisson arrival rate (1/s)")
    p.add_argument("--serve-pool", type=int, default=0,
                   help="distinct matrices of the stream (0: one per request); request k uses "
                        "matrix k mod pool, with its own sketch seed and tolerance, so that a "
                        "stream whose matrices do not fit in HBM together can still be played")
    p.add_argument("--serve-deadline", type=float, default=0.0,
                   help="stop submitting after this many seconds of the stream (0: none); the "
                        "requests not yet submitted are reported as the backlog")
    p.add_argument("--serve-min", type=int, default=512)
    p.add_argument("--serve-max", type=int, default=4096)
    p.add_argument("--serve-team", type=int, default=8)
    p.add_argument("--serve-streams", type=int, default=4)
    p.add_argument("--serve-budget-gb", type=float, default=120.0)
    p.add_argument("--serve-big", type=int, default=500000,
                   help="requests with m*n at or above this run on the whole GPU (single-matrix path)")
    p.add_argument("--serve-lanes", type=int, default=2,
                   help="large requests that may run at once, each on its own stream")
    p.add_argument("--no-plain-serial", action="store_true")
    p.add_argument("--batch-teams", type=str, default="2,4,8",
                   help="team sizes the batch autotuner tries (CTAs per job)")
    p.add_argument("--verbose", action="store_true", help="stage timestamps on stderr")
    p.add_argument("--watchdog", type=float, default=0.0,
                   help="dump all Python stacks to stderr and exit after this many seconds")
    return p.parse_args()


_T0 = time.perf_counter()
_VERBOSE = False


def log(msg):
    if _VERBOSE:
        print(f"[bench {time.perf_counter() - _T0:8.2f}s] {msg}", file=sys.stderr, flush=True)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def aggregate(elapsed_ms, steps, ws, device=None):
    """Max-over-ranks elapsed time of the timed region and the whole-job value
    (ms per decomposition = max time / (ranks x steps)); ranks are replicas."""
    if ws > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([elapsed_ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        elapsed_ms = float(t.item())
    return elapsed_ms, elapsed_ms / (steps * ws)


SKETCH_FORMS = {0: "FP64-pipe Gaussian sketch", 5: "FP64 tensor-core sketch (52-bit fixed point)"}


def workload_name(a):
    dt = "FP64" if a.dtype == "f64" else "FP32"
    form = ", " + SKETCH_FORMS.get(a.sketch_mode,
                                   f"tensor-core precision sketch with {a.sketch_mode} digit(s)")
    return (f"{a.m}x{a.n} {dt} A=U diag(i^-2) V^T + N(0,({a.noise:g})^2) noise, tol {a.tol:g}, "
            f"b={a.block}, c={a.sketch}{form}")


def make_matrix(a, device, dtype):
    from paper_2509_21963_gb300 import inputs
    return inputs.decay_matrix_torch(a.m, a.n, "poly2", seed=11, noise=a.noise, rank_cap=2000,
                                     dtype=dtype, device=device)


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix="clocks", suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = max(mx, float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def source_sha1(name):
    src = os.path.join(ROOT, "paper_2509_21963_gb300", "csrc", name)
    code = re.sub(r"//[^\n]*", "", open(src).read())
    return hashlib.sha1(code.encode()).hexdigest()


def traffic_for(name):
    """DRAM bytes per full-size launch from the committed ncu capture, or None
    once the kernel source has changed since the counters were taken."""
    rec = TRAFFIC[name]
    if rec["sha1"] == source_sha1(name) and rec["bytes_per_launch_full"] is not None:
        return rec["bytes_per_launch_full"]
    return None


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    import platform
    return platform.processor() or platform.machine()


def oracle_run_for(a, A_host, tol=None):
    """The oracle's run of the same method on the same matrix, for the sketch
    form a.sketch_mode (FP64 data; FP32 inputs upcast exactly)."""
    import numpy as np
    import oracle
    tol = a.tol if tol is None else tol
    m = A_host.shape[0]
    if a.sketch_mode == 5:
        return oracle.run_fx(A_host, tol, a.block, a.sketch, seed=a.seed)
    if a.sketch_mode == 0:
        return oracle.run(A_host, tol, a.block, a.sketch, seed=a.seed, mode=1)
    Gq = oracle.gaussian_sketch_q8(a.seed, a.sketch, m)
    Y = oracle.sketch(Gq, oracle.fixed_point(A_host, a.sketch_mode))
    return oracle.run_y(A_host, tol, a.block, a.sketch, Y)


def timed_oracle(a, A_host, threads):
    import oracle
    oracle.set_threads(threads)
    t0 = time.perf_counter()
    r = oracle_run_for(a, A_host)
    return (time.perf_counter() - t0) * 1000.0, r


def run_reference(a, ws, rank):
    """The reference arm: the FP64 CPU oracle as it stands (the same method,
    sketch form and matrix), one whole run per step on all host cores."""
    if rank != 0:
        return 0
    import torch
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    dtype = torch.float64 if a.dtype == "f64" else torch.float32
    A = make_matrix(a, dev, dtype)
    A_host = A.to(torch.float64).cpu().numpy()
    del A
    cores = os.cpu_count() or 1
    for _ in range(a.warmup):
        timed_oracle(a, A_host, cores)
    vals = []
    for _ in range(a.steps):
        ms, r = timed_oracle(a, A_host, cores)
        vals.append(ms)
    value = sum(vals) / len(vals)
    sample = (f"one whole oracle run per step on the {a.m}x{a.n} matrix ({cores} threads, "
              f"rank {r.rank}, rho {r.rho:.3e}); {a.steps} steps after {a.warmup} warm-up runs")
    line = {"impl": "reference", "metric": "time-to-tolerance per CUR", "value": value, "unit": "ms",
            "n_gpus": ws, "steps": a.steps, "warmup": a.warmup, "ms_per_step": value,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": workload_name(a)},
            "cpu_baseline": {"value": value, "unit": "ms", "cores": cores, "kind": "oracle",
                             "sample": sample, "cpu_model": cpu_model()},
            "e2e": {"value": value, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# Batched workload
# ---------------------------------------------------------------------------
BATCH_TOL, BATCH_B, BATCH_C = 1e-4, 8, 8


def batch_rank_model(spec):
    """Rank a job reaches (for work estimates when no run is available):
    exp(-i/20) needs ~184 indices for 1e-4, i^-1.5 runs to full rank, exact
    rank r stops at r; all rounded up to whole blocks of 8, capped at min(m,n)."""
    k = min(spec["m"], spec["n"])
    r = {"exp20": 192, "poly1.5": k, "rank": spec["r"]}[spec["kind"]]
    return min(k, -(-r // BATCH_B) * BATCH_B)


def batch_flops(m, n, r):
    """FP64 operations of one job: the sketch 2cmn, the Lemma 1 residual
    products (m + n) r^2 summed over the blocks, the core QR 4/3 r^3 and its
    solve 3 r^3 (Q^T applied to the identity, then back substitution)."""
    return 2.0 * BATCH_C * m * n + (m + n) * r * r + (4.0 / 3.0 + 3.0) * r ** 3


def batch_job_specs(a, seed):
    from paper_2509_21963_gb300 import inputs
    if a.batch_uniform:
        return [dict(m=a.batch_uniform, n=a.batch_uniform, kind=a.batch_kind, r=100,
                     seed=seed * 100003 + j) for j in range(a.batch_jobs)]
    return inputs.batch_specs(a.batch_jobs, seed)


def batch_workload_name(a):
    if a.batch_uniform:
        return (f"{a.batch_jobs} independent FP32 matrices of {a.batch_uniform} x {a.batch_uniform}, "
                f"spectrum {a.batch_kind}, tol {BATCH_TOL:g}, b={BATCH_B}, c={BATCH_C}")
    return (f"{a.batch_jobs} independent FP32 matrices, m, n log-uniform in [64, 2048], spectra "
            f"exp(-i/20) / i^-1.5 / exact rank r~U[5,200] (one third each), tol {BATCH_TOL:g}, "
            f"b={BATCH_B}, c={BATCH_C}")


def batch_oracle_sample(specs, seconds, seed):
    """Run the FP64 oracle on jobs in a fixed random order until `seconds` of
    CPU time are spent; return (wall seconds, sampled work by the rank model,
    jobs run)."""
    import numpy as np
    import oracle
    from paper_2509_21963_gb300 import inputs
    order = np.random.default_rng(seed).permutation(len(specs))
    t_all, work, done = 0.0, 0.0, 0
    for j in order:
        s = specs[j]
        A = inputs.batch_matrix(s).astype(np.float32).astype(np.float64)
        t0 = time.perf_counter()
        oracle.run(A, BATCH_TOL, BATCH_B, BATCH_C, seed=s["seed"], mode=1)
        t_all += time.perf_counter() - t0
        work += batch_flops(s["m"], s["n"], batch_rank_model(s))
        done += 1
        if t_all >= seconds:
            break
    return t_all, work, done


def run_batch_reference(a, ws, rank):
    if rank != 0:
        return 0
    specs = batch_job_specs(a, a.seed)
    total = sum(batch_flops(s["m"], s["n"], batch_rank_model(s)) for s in specs)
    vals = []
    for k in range(a.warmup + a.steps):
        t, w, done = batch_oracle_sample(specs, 8.0, seed=k)
        if k >= a.warmup:
            vals.append(t * 1000.0 * total / w)
    value = sum(vals) / len(vals)
    sample = (f"oracle on random jobs of the batch until 8 s of CPU time per step, scaled by "
              f"the batch's FP64 work (rank model) over the sample's")
    line = {"impl": "reference", "metric": "time per batch of CURs", "value": value, "unit": "ms",
            "n_gpus": ws, "steps": a.steps, "warmup": a.warmup, "ms_per_step": value,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": batch_workload_name(a)},
            "cpu_baseline": {"value": value, "unit": "ms", "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_batch(a, ws, rank, local):
    import numpy as np
    import torch
    import paper_2509_21963_gb300 as cur
    from paper_2509_21963_gb300 import inputs

    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = f"cuda:{local}"
    log("batch: generating matrices")
    specs = batch_job_specs(a, a.seed + 1000 * rank)
    mats = [inputs.batch_matrix_torch(s, device=dev) for s in specs]
    torch.cuda.synchronize()
    log("batch: matrices ready")
    ctx = cur.Context(local)
    stream = torch.cuda.current_stream()
    B = cur.Batch(ctx, mats, BATCH_TOL, BATCH_B, BATCH_C, seed=[s["seed"] for s in specs])
    cands = [int(x) for x in a.batch_teams.split(",")]
    team, tune_ms = B.tune(cands)
    log(f"batch: tuner chose team {team} ({tune_ms:.1f} ms)")
    for _ in range(max(a.warmup, 3)):
        B.run()

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.4)
    barrier()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(a.steps):
        B.run()
    t1.record(stream)
    barrier()
    clk = clocks.stop()
    elapsed_ms = t0.elapsed_time(t1)
    elapsed_ms, value = aggregate(elapsed_ms, a.steps, ws, device=dev)
    info = [B.info(j) for j in range(len(specs))]
    statuses = np.bincount([x[3] for x in info], minlength=8).tolist()
    flops = sum(batch_flops(s["m"], s["n"], x[0]) for s, x in zip(specs, info))
    achieved = flops / (value * 1e-3) / 1e12
    ph = B.phase_cycles()
    tot = sum(v for k, v in ph.items() if k != "jobs")
    fp64_meas = ctx.fp64_tflops()
    roofline = {"bound": "alu", "achieved": achieved, "peak": fp64_meas, "unit": "TFLOP/s",
                "frac": achieved / fp64_meas, "traffic": None,
                "peak_source": "measured FP64 FMA rate (cur_probe_fp64_tflops); nominal 1.25",
                "kernel": "batch_kernel (whole batch, FP64 SIMT pipe)", "kernel_ms": value,
                "flops_per_launch": flops,
                "phase_share": {k: v / tot for k, v in ph.items() if k != "jobs"}}

    e2e = None
    if not a.no_e2e:
        # every step: all matrices host -> device (pinned), the batch, per-job records
        # and every job's I, J and U device -> host
        log("batch e2e: pinning host copies")
        host = [m.cpu().pin_memory() for m in mats]
        ranks = [x[0] for x in info]
        outI = [torch.empty(r, dtype=torch.int64).pin_memory() for r in ranks]
        outJ = [torch.empty(r, dtype=torch.int64).pin_memory() for r in ranks]
        outU = [torch.empty(r * r, dtype=torch.float64).pin_memory() for r in ranks]
        L = cur.lib()

        def e2e_step():
            for hm, dm in zip(host, mats):
                dm.copy_(hm, non_blocking=True)
            B.run()
            for j, r in enumerate(ranks):
                rj = B.info(j)[0]
                if rj:
                    st = L.cur_batch_copy_job(B.ptr, j, outI[j].data_ptr(), outJ[j].data_ptr(),
                                              outU[j].data_ptr(), None)
                    if st != cur.CUR_OK:
                        raise cur.CurError(st, ctx.last_error())
        e2e_step()
        torch.cuda.synchronize()
        w0 = time.perf_counter()
        for _ in range(a.e2e_steps):
            e2e_step()
        torch.cuda.synchronize()
        e2e_ms = (time.perf_counter() - w0) * 1000.0 / a.e2e_steps
        e2e = {"value": e2e_ms, "unit": "ms",
               "h2d_bytes_per_step": int(sum(m.numel() * 4 for m in mats)),
               "d2h_bytes_per_step": int(sum(16 * r + 8 * r * r for r in ranks) + 48 * len(ranks))}
        del host

    cpu = None
    if rank == 0 and ws == 1 and not a.no_cpu_baseline:
        log("batch cpu baseline: oracle on sampled jobs")
        total = sum(batch_flops(s["m"], s["n"], batch_rank_model(s)) for s in specs)
        t, w, done = batch_oracle_sample(specs, 20.0, seed=0)
        cpu = {"value": t * 1000.0 * total / w, "unit": "ms", "cores": 1, "kind": "oracle",
               "sample": f"{done} random jobs of the batch ({t:.1f} s of oracle time), scaled by the "
                         f"batch's FP64 work over the sample's (rank model)"}

    if rank == 0:
        line = {
            "metric": "time per batch of CURs", "value": value, "unit": "ms", "n_gpus": ws,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": elapsed_ms / a.steps,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64 (FP32 A)", "data": "synthetic",
            "config": {"workload": batch_workload_name(a), "jobs": len(specs),
                       "team": team, "schedule": B.schedule(), "statuses": statuses,
                       "sum_rank": int(sum(x[0] for x in info)),
                       "l2": "inputs (5.3 GB) larger than L2",
                       "parallelism": f"replicas x{ws}"},
            "gpu_launches": a.steps, "clocks": clk, "e2e": e2e, "roofline": roofline,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    B.close()
    ctx.close()
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


# ---------------------------------------------------------------------------
# Serving workload
# ---------------------------------------------------------------------------
SERVE_B, SERVE_C = 50, 55
SERVE_TOLS = (1e-2, 1e-4, 1e-6)


def serve_stream(a, seed):
    """Arrival times (s), shapes/spectra and tolerances of the request stream."""
    import numpy as np
    from paper_2509_21963_gb300 import inputs
    rng = np.random.default_rng(seed)
    arrivals = np.cumsum(rng.exponential(1.0 / a.serve_rate, a.serve_requests))
    specs = inputs.batch_specs(a.serve_requests, seed + 1, a.serve_min, a.serve_max)
    tols = [float(t) for t in rng.choice(SERVE_TOLS, a.serve_requests)]
    return arrivals, specs, tols


def serve_rank_model(spec, tol, b):
    """Rank a request reaches: exp(-i/20) needs 20 ln(1/tol), i^-1.5 about
    0.65 / tol, exact rank r stops at r; whole blocks of b, capped at min(m, n)."""
    import math
    k = min(spec["m"], spec["n"])
    r = {"exp20": 20 * math.log(1 / tol), "poly1.5": 0.65 / tol, "rank": spec["r"]}[spec["kind"]]
    return int(min(k, -(-int(r) // b) * b))


def serve_flops(m, n, r, b=SERVE_B, c=SERVE_C):
    return 2.0 * c * m * n + (m + n) * r * r + (4.0 / 3.0 + 3.0) * r ** 3


def serve_workload_name(a):
    return (f"{a.serve_requests} requests, Poisson {a.serve_rate:g}/s, FP32 A with m, n "
            f"log-uniform in [{a.serve_min}, {a.serve_max}], spectra exp(-i/20) / i^-1.5 / exact "
            f"rank r~U[5,200], tol uniform over {{1e-2, 1e-4, 1e-6}}, b={SERVE_B}, c={SERVE_C}, "
            f"{a.serve_budget_gb:g} GB admission budget"
            + (f", {a.serve_pool} distinct matrices (request k uses matrix k mod {a.serve_pool} "
               f"with its own sketch seed and tolerance)"
               if 0 < getattr(a, "serve_pool", 0) < a.serve_requests else ""))


def pct(xs, q):
    import numpy as np
    return float(np.percentile(np.asarray(xs, dtype=np.float64), q)) if len(xs) else None


def serve_oracle_sample(specs, tols, seconds, seed):
    import numpy as np
    import oracle
    from paper_2509_21963_gb300 import inputs
    order = np.random.default_rng(seed).permutation(len(specs))
    t_all, work, done = 0.0, 0.0, 0
    for j in order:
        s = specs[j]
        w = serve_flops(s["m"], s["n"], serve_rank_model(s, tols[j], SERVE_B))
        if w > 5e10 and done > 0:
            continue  # keep the sample bounded: skip jobs of more than ~1 min on one core
        A = inputs.batch_matrix(s).astype(np.float32).astype(np.float64)
        t0 = time.perf_counter()
        oracle.run(A, tols[j], SERVE_B, SERVE_C, seed=s["seed"], mode=1)
        t_all += time.perf_counter() - t0
        work += w
        done += 1
        if t_all >= seconds:
            break
    return t_all, work, done


def run_serve_reference(a, ws, rank):
    if rank != 0:
        return 0
    arrivals, specs, tols = serve_stream(a, a.seed)
    total = sum(serve_flops(s["m"], s["n"], serve_rank_model(s, t, SERVE_B)) for s, t in zip(specs, tols))
    vals = []
    for k in range(a.warmup + a.steps):
        t, w, done = serve_oracle_sample(specs, tols, 8.0, seed=k)
        if k >= a.warmup:
            vals.append(t * 1000.0 * total / w / len(specs))
    value = sum(vals) / len(vals)
    line = {"impl": "reference", "metric": "served latency p50 per request", "value": value,
            "unit": "ms", "n_gpus": ws, "steps": a.steps, "warmup": a.warmup, "ms_per_step": value,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": serve_workload_name(a)},
            "cpu_baseline": {"value": value, "unit": "ms", "cores": 1, "kind": "oracle",
                             "sample": "mean oracle time per request over random requests of the "
                                       "stream (8 s per step), scaled by FP64 work (rank model)"},
            "e2e": {"value": value, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_serve(a, ws, rank, local):
    import numpy as np
    import torch
    import paper_2509_21963_gb300 as cur
    from paper_2509_21963_gb300 import inputs

    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = f"cuda:{local}"
    arrivals, specs, tols = serve_stream(a, a.seed + 1000 * rank)
    pool = a.serve_pool if 0 < a.serve_pool < len(specs) else len(specs)
    if pool < len(specs):   # request k: matrix k mod pool, its own sketch seed and tolerance
        specs = [dict(specs[k % pool], seed=specs[k % pool]["seed"], sketch_seed=specs[k]["seed"])
                 for k in range(len(specs))]
    log(f"serve: generating {pool} matrices")
    uniq = [inputs.batch_matrix_torch(s, device=dev) for s in specs[:pool]]
    mats = [uniq[k % pool] for k in range(len(specs))]
    for s in specs:
        s.setdefault("sketch_seed", s["seed"])
    torch.cuda.synchronize()
    log("serve: matrices ready")
    ctx = cur.Context(local)
    budget = int(a.serve_budget_gb * (1 << 30))
    S = cur.Server(ctx, budget, "float32", team=a.serve_team, streams=a.serve_streams,
                   big_elements=a.serve_big, big_lanes=a.serve_lanes)

    # warm-up: a few small requests through the server and the plain path
    small = sorted(range(len(specs)), key=lambda j: specs[j]["m"] * specs[j]["n"])[:4]
    for j in small:
        S.wait(S.submit(mats[j], tols[j], SERVE_B, SERVE_C, seed=specs[j]["sketch_seed"]))
        ctx.run(mats[j], tols[j], SERVE_B, SERVE_C, specs[j]["sketch_seed"])
    S.drain()
    for st in list(S._keep):
        S.release(st)

    def play(host):
        """Submit every request at its arrival time; returns per-request
        (latency, queue, rank, status) and the makespan in s."""
        if host:
            hs = [m.cpu().numpy() for m in uniq]
            srcs = [hs[k % len(hs)] for k in range(len(mats))]
        else:
            srcs = mats
        barrier_sync()
        t0 = time.perf_counter()
        tickets = []
        for k in range(len(specs)):
            if a.serve_deadline > 0 and time.perf_counter() - t0 > a.serve_deadline:
                break   # the rest is the backlog at the deadline
            delay = arrivals[k] - (time.perf_counter() - t0)
            if delay > 0:
                time.sleep(delay)
            tickets.append(S.submit(srcs[k], tols[k], SERVE_B, SERVE_C,
                                    seed=specs[k]["sketch_seed"]))
        out = []
        for tk in tickets:
            S.wait(tk)
            r, it, rho, st, lat, q = S.info(tk)
            if st not in (cur.CUR_OK, cur.CUR_TOL_UNREACHED):
                log(f"serve: request {tk} failed with status {st}: {ctx.last_error()}")
            out.append((lat, q, r, st))
            S.release(tk)
        return out, time.perf_counter() - t0

    def barrier_sync():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.4)
    log("serve: playing the stream (device-resident requests)")
    launches0 = S.stats()["launches"]
    res, makespan = play(False)
    clk = clocks.stop()
    backlog = len(specs) - len(res)
    lat = [x[0] for x in res]
    stats = S.stats()
    flops = sum(serve_flops(s["m"], s["n"], x[2]) for s, x in zip(specs, res))
    offered = sum(serve_flops(s["m"], s["n"], serve_rank_model(s, t, SERVE_B))
                  for s, t in zip(specs, tols))
    statuses = np.bincount([x[3] for x in res], minlength=8).tolist()
    met = sum(1 for x in res if x[3] == cur.CUR_OK)
    log(f"serve: p50 {pct(lat, 50):.1f} ms p99 {pct(lat, 99):.1f} ms makespan {makespan:.2f} s")

    e2e = None
    if not a.no_e2e:
        log("serve: playing the stream again with host-resident requests")
        res_h, makespan_h = play(True)
        lat_h = [x[0] for x in res_h]
        e2e = {"value": pct(lat_h, 50), "unit": "ms", "p99_ms": pct(lat_h, 99),
               "throughput_rps": len(res_h) / makespan_h,
               "h2d_bytes_per_step": int(sum(m.numel() * 4 for m in mats)),
               "d2h_bytes_per_step": 0,
               "note": "requests carry host memory; the server copies each A at admission"}

    plain = None
    if not a.no_plain_serial:
        # the plain single-matrix path (cur_run), one request at a time in arrival order:
        # each starts when it has arrived and the previous one has finished
        log("serve: plain path, serially")
        end, lat_p = 0.0, []
        for k in range(len(specs)):
            if a.serve_deadline > 0 and end > a.serve_deadline:
                break   # the same deadline on the simulated clock
            torch.cuda.synchronize()
            w0 = time.perf_counter()
            ctx.run(mats[k], tols[k], SERVE_B, SERVE_C, specs[k]["sketch_seed"])
            torch.cuda.synchronize()
            d = time.perf_counter() - w0
            start = max(arrivals[k], end)
            end = start + d
            lat_p.append((end - arrivals[k]) * 1000.0)
        plain = {"p50_ms": pct(lat_p, 50), "p99_ms": pct(lat_p, 99),
                 "throughput_rps": len(lat_p) / end, "busy_s": end, "served": len(lat_p),
                 "backlog_at_deadline": len(specs) - len(lat_p)}

    fp64_meas = ctx.fp64_tflops()
    cpu = None
    if rank == 0 and ws == 1 and not a.no_cpu_baseline:
        log("serve: cpu baseline")
        total = sum(serve_flops(s["m"], s["n"], serve_rank_model(s, t, SERVE_B))
                    for s, t in zip(specs, tols))
        t, w, done = serve_oracle_sample(specs, tols, 20.0, seed=0)
        cpu = {"value": t * 1000.0 * total / w / len(specs), "unit": "ms per request", "cores": 1,
               "kind": "oracle",
               "sample": f"{done} random requests of the stream ({t:.1f} s of oracle time); mean "
                         f"time per request scaled by FP64 work (rank model)"}

    if rank == 0:
        line = {
            "metric": "served latency p50 per request", "value": pct(lat, 50), "unit": "ms",
            "n_gpus": ws, "steps": 1, "warmup": 1, "ms_per_step": makespan * 1000.0,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64 (FP32 A)", "data": "synthetic",
            "p99_ms": pct(lat, 99), "throughput_rps": len(res) / makespan,
            "queue_p50_ms": pct([x[1] for x in res], 50), "met_tolerance": met,
            "served": len(res), "backlog_at_deadline": backlog,
            "offered_load": {"tflop_model": offered / 1e12,
                             "arrival_span_s": float(arrivals[-1]),
                             "tflops_needed_model": offered / 1e12 / float(arrivals[-1])},
            "config": {"workload": serve_workload_name(a), "team": a.serve_team,
                       "streams": a.serve_streams, "big_elements": a.serve_big,
                       "big_lanes": a.serve_lanes,
                       "statuses": statuses,
                       "waves": stats["waves"], "bytes_peak": stats["bytes_peak"],
                       "parallelism": f"replicas x{ws}"},
            "gpu_launches": stats["launches"] - launches0, "clocks": clk, "e2e": e2e,
            "roofline": {"bound": "alu", "achieved": flops / makespan / 1e12,
                         "peak": fp64_meas, "unit": "TFLOP/s",
                         "frac": flops / makespan / 1e12 / fp64_meas, "traffic": None,
                         "peak_source": "measured FP64 FMA rate (cur_probe_fp64_tflops); nominal 1.25",
                         "kernel": "serve_kernel waves over the makespan (FP64 SIMT pipe)"},
            "plain_serial": plain, "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    S.close()
    ctx.close()
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


# ---------------------------------------------------------------------------
# Precision-form workload
# ---------------------------------------------------------------------------
PREC_M, PREC_N, PREC_RANK = 65536, 32768, 4096
PREC_CASES = (  # (tol, b, c, (sketch mode, residual planes) forms, rank cap); mode 0 = FP64
    # sketch, S = digits; planes 0 = FP64 residual products, 2 / 3 = BF16 planes on tcgen05
    (1e-2, 100, 110, ((0, 0), (1, 0), (1, 2)), 2048),   # one digit: its sketch error (~0.1
    (1e-3, 100, 110, ((0, 0), (2, 0), (2, 2), (2, 3)), 4096),   # here) bounds its reach
    (1e-6, 56, 62, ((0, 0), (3, 0), (4, 0)), 6144),  # CUR needs ~1.4x the SVD rank here; c <= 64
)                                                    # for four digits; planes stall near 2e-6


def precision_workload_name():
    return (f"{PREC_M}x{PREC_N} FP32 A = U diag(exp(-i/200)) V^T (built in FP64, stored FP32), "
            f"U, V from QR of seeded Gaussian factors of rank {PREC_RANK}; tol 1e-2 and 1e-3 "
            f"(b=100, c=110), 1e-6 (b=56, c=62); FP64 sketch vs tensor-core sketches with 1/2/3/4 "
            f"base-256 digits")


def true_rel_error(A, I, J, U, chunk=4096):
    """||A - A(:,J) U A(I,:)||_F / ||A||_F in FP64, in row chunks."""
    import torch
    Jt = torch.from_numpy(J).to(A.device)
    It = torch.from_numpy(I).to(A.device)
    Ut = torch.from_numpy(U).to(A.device)
    W = Ut @ A[It, :].double()                       # U R  (r x n)
    num, den = 0.0, 0.0
    for r0 in range(0, A.shape[0], chunk):
        blk = A[r0:r0 + chunk].double()
        E = blk - blk[:, Jt] @ W
        num += float((E * E).sum())
        den += float((blk * blk).sum())
        del E, blk
    return (num / den) ** 0.5


def run_precision(a, ws, rank, local):
    import torch
    import paper_2509_21963_gb300 as cur
    from paper_2509_21963_gb300 import inputs
    torch.cuda.set_device(local)
    dev = f"cuda:{local}"
    log("precision: generating A")
    A = inputs.decay_matrix_torch(PREC_M, PREC_N, "exp200", seed=23, noise=0.0,
                                  rank_cap=PREC_RANK, dtype=torch.float32, device=dev,
                                  factor_dtype=torch.float64)
    torch.cuda.synchronize()
    log("precision: A ready")
    ctx = cur.Context(local)
    stream = torch.cuda.current_stream()
    forms = []
    for tol, b, c, modes, cap in PREC_CASES:
        for mode, planes in modes:
            kw = dict(sketch_mode=mode, timing=True, max_rank=cap, residual_planes=planes)
            st, out = ctx.run_raw(A, tol, b, c, a.seed, **kw)   # warm
            cur.lib().cur_result_free(out)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            st, out = ctx.run_raw(A, tol, b, c, a.seed, **kw)
            e1.record(stream)
            torch.cuda.synchronize()
            if st not in (cur.CUR_OK, cur.CUR_TOL_UNREACHED) or not out:
                msg = ctx.last_error()
                log(f"precision: tol {tol:g} mode {mode}: status {st}: {msg}")
                forms.append({"tol": tol, "b": b, "c": c, "sketch_mode": mode,
                              "residual_planes": planes, "status": int(st),
                              "error": msg, "meets_tol": False})
                continue
            res = cur._result_from(out)
            cur.lib().cur_result_free(out)
            err = true_rel_error(A, res.I, res.J, res.U) if res.rank else 1.0
            sk = max(res.phase_ms["sketch"], 1e-9)
            row = {"tol": tol, "b": b, "c": c,
                   "sketch": "FP64" if mode == 0 else f"tensor-core, {mode} digit(s)",
                   "residual_products": "FP64" if planes == 0 else
                                        f"tensor cores, {planes} BF16 planes",
                   "time_to_tolerance_ms": e0.elapsed_time(e1), "rank": res.rank,
                   "iterations": res.iterations, "rho": res.rho, "status": int(st),
                   "true_rel_error": err, "meets_tol": bool(st == cur.CUR_OK and err <= tol),
                   "sketch_ms": sk, "phase_ms": res.phase_ms}
            if mode == 0:
                row["sketch_fp64_tflops"] = 2.0 * c * PREC_M * PREC_N / (sk * 1e-3) / 1e12
            else:
                row["sketch_hbm_gbs_two_passes"] = 2.0 * PREC_M * PREC_N * 4 / (sk * 1e-3) / 1e9
            forms.append(row)
            log(f"precision: tol {tol:g} mode {mode} planes {planes}: "
                f"{row['time_to_tolerance_ms']:.1f} ms, "
                f"rank {res.rank}, rho {res.rho:.2e}, true error {err:.2e}, status {st}")
    if rank == 0:
        cands = [f for f in forms if f["tol"] == 1e-3 and f.get("meets_tol")
                 and "sketch_hbm_gbs_two_passes" in f]
        head = min(cands, key=lambda f: f["time_to_tolerance_ms"]) if cands else next(
            f for f in forms if f["tol"] == 1e-3 and f.get("sketch", "").startswith("tensor-core, 2"))
        line = {"metric": "time-to-tolerance per CUR", "value": head["time_to_tolerance_ms"],
                "unit": "ms", "n_gpus": ws, "steps": 1, "warmup": 1,
                "ms_per_step": head["time_to_tolerance_ms"], "higher_is_better": False,
                "scaling": "weak", "vs_baseline": None,
                "dtype": f"bf16 digit slices in the sketch ({head.get('sketch')}), residual products "
                         f"{head.get('residual_products')}, f64 LUPP, core and norms",
                "data": "synthetic",
                "config": {"workload": precision_workload_name(),
                           "headline": "tol 1e-3, the fastest form that meets it"},
                "forms": forms,
                "roofline": {"bound": "hbm", "achieved": head["sketch_hbm_gbs_two_passes"],
                             "peak": HBM_GBS, "unit": "GB/s",
                             "frac": head["sketch_hbm_gbs_two_passes"] / HBM_GBS, "traffic": None,
                             "kernel": "sketch phase (column scales + tensor-core pass)"}}
        print(json.dumps(line), flush=True)
    ctx.close()
    return 0


# ---------------------------------------------------------------------------
# The sketch step alone (for kernel profiles)
# ---------------------------------------------------------------------------
def run_sketch_step(a, ws, rank, local):
    """cur_step_sketch (FP64 pipe), cur_step_sketch_fx (FP64 tensor-core form) or
    cur_step_sketch_q (digits) on a Gaussian A of
    m x n, c = --sketch rows: W warm-up calls, then K timed calls."""
    import torch
    import paper_2509_21963_gb300 as cur
    torch.cuda.set_device(local)
    dtype = torch.float64 if a.dtype == "f64" else torch.float32
    g = torch.Generator(device=f"cuda:{local}")
    g.manual_seed(a.seed + 1)
    A = torch.randn(a.m, a.n, device=f"cuda:{local}", generator=g, dtype=dtype)
    ctx = cur.Context(local)
    G = ctx.gaussian(a.seed, a.sketch, a.m)
    if a.sketch_mode == 0:
        call = lambda: ctx.sketch(G, A)
    elif a.sketch_mode == 5:
        call = lambda: ctx.sketch_fx(G, A)
    else:
        call = lambda: ctx.sketch_q(G, A, a.sketch_mode)
    for _ in range(max(a.warmup, 3)):
        call()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(a.steps):
        call()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / a.steps
    if rank == 0:
        es = A.element_size()
        line = {"metric": "sketch step time", "value": ms, "unit": "ms", "n_gpus": ws,
                "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms,
                "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
                "dtype": {0: a.dtype, 5: "f64 data, bf16 digits"}.get(a.sketch_mode,
                                                                        f"bf16x{a.sketch_mode}"),
                "data": "synthetic",
                "config": {"workload": f"sketch Y = G A, A {a.m}x{a.n} {a.dtype} Gaussian, c={a.sketch}",
                           "sketch_mode": a.sketch_mode},
                "one_pass_gbs": a.m * a.n * es / ms / 1e6,
                "fp64_tflops": 2.0 * a.sketch * a.m * a.n / ms / 1e9}
        print(json.dumps(line), flush=True)
    ctx.close()
    return 0


def main():
    global _VERBOSE
    a = parse()
    if a.sketch_mode is None:
        a.sketch_mode = 5 if a.dtype == "f64" else 0
    _VERBOSE = a.verbose
    if a.watchdog > 0:
        import faulthandler
        faulthandler.dump_traceback_later(a.watchdog, exit=True)
    ws, rank, local = dist_env()
    if a.workload == "batch":
        if a.impl == "reference":
            return run_batch_reference(a, ws, rank)
        return run_batch(a, ws, rank, local)
    if a.workload == "sketch":
        if a.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "kernel-profile mode only"}))
            return 0
        return run_sketch_step(a, ws, rank, local)
    if a.workload == "precision":
        if a.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable":
                              "the oracle would need hours on a 65536 x 32768 matrix; the "
                              "precision forms are compared with the FP64 GPU path instead"}))
            return 0
        return run_precision(a, ws, rank, local)
    if a.workload == "serve":
        if a.impl == "reference":
            return run_serve_reference(a, ws, rank)
        return run_serve(a, ws, rank, local)
    if a.impl == "reference":
        return run_reference(a, ws, rank)

    import copy
    import numpy as np
    import torch
    import paper_2509_21963_gb300 as cur

    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dtype = torch.float64 if a.dtype == "f64" else torch.float32
    log("generating A")
    A = make_matrix(a, f"cuda:{local}", dtype)
    torch.cuda.synchronize()
    log("A ready")
    ctx = cur.Context(local)
    L = cur.lib()
    stream = torch.cuda.current_stream()

    last_phases = [None]

    def one_step(timing, AA=None, tol=None, mode=None):
        AA = A if AA is None else AA
        st, out = ctx.run_raw(AA, a.tol if tol is None else tol, a.block, a.sketch, a.seed,
                              timing=timing, sketch_mode=a.sketch_mode if mode is None else mode)
        if st not in (cur.CUR_OK, cur.CUR_TOL_UNREACHED):
            raise cur.CurError(st, ctx.last_error())
        last_phases[0] = {p: float(L.cur_result_phase_ms(out, i)) for i, p in enumerate(cur.PHASES)}
        info = (int(L.cur_result_rank(out)), int(L.cur_result_iterations(out)),
                float(L.cur_result_err(out)), float(L.cur_result_phase_ms(out, 1)),
                int(L.cur_result_kernel_launches(out)), int(st))
        L.cur_result_free(out)
        return info

    def time_form(AA, tol, mode, reps, warm=2):
        """Time-to-tolerance of one form (CUDA events on the library's stream)."""
        for _ in range(warm):
            one_step(True, AA, tol, mode)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            info = one_step(True, AA, tol, mode)
        e1.record(stream)
        torch.cuda.synchronize()
        return {"time_to_tolerance_ms": e0.elapsed_time(e1) / reps, "rank": info[0],
                "iterations": info[1], "rho": info[2], "status": info[5],
                "sketch_mode": mode, "phase_ms": last_phases[0]}

    for _ in range(max(a.warmup, 3)):
        info = one_step(True)
        log(f"warm-up step: rank {info[0]}, iterations {info[1]}, rho {info[2]:.3e}, sketch {info[3]:.2f} ms")

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.4)
    barrier()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    infos = []
    phases = []
    ev_step = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(a.steps)]
    for k in range(a.steps):
        ev_step[k][0].record(stream)
        infos.append(one_step(True))
        ev_step[k][1].record(stream)
        phases.append(last_phases[0])
    t1.record(stream)
    barrier()
    clk = clocks.stop()
    elapsed_ms = t0.elapsed_time(t1)
    per_step = [e0.elapsed_time(e1) for e0, e1 in ev_step]
    step_ms = {"median": float(np.median(per_step)), "p10": float(np.percentile(per_step, 10)),
               "p90": float(np.percentile(per_step, 90)), "n": len(per_step)}
    log(f"timed {a.steps} steps: {elapsed_ms:.2f} ms")
    elapsed_ms, value = aggregate(elapsed_ms, a.steps, ws, device=f"cuda:{local}")
    rank_r, iters, rho, _, launches, status = infos[-1]
    phase_ms = {p: sum(ph[p] for ph in phases) / len(phases) for p in cur.PHASES}
    sketch_ms = phase_ms["sketch"]
    ms_per_step = elapsed_ms / a.steps

    # accuracy of the timed configuration: ||A - C U R||_F / ||A||_F in FP64 on
    # the device (outside the timed region), C = A(:, J), R = A(I, :)
    res = ctx.run(A, a.tol, a.block, a.sketch, a.seed, sketch_mode=a.sketch_mode)
    A64 = A if A.dtype == torch.float64 else A.to(torch.float64)
    Jt = torch.from_numpy(res.J).to(A.device)
    It = torch.from_numpy(res.I).to(A.device)
    Ut = torch.from_numpy(res.U.reshape(res.rank, res.rank)).to(A.device)
    E = A64 - (A64[:, Jt] @ Ut) @ A64[It, :]
    true_err = float(torch.linalg.norm(E) / torch.linalg.norm(A64))
    del E, A64
    torch.cuda.empty_cache()
    log(f"true relative error {true_err:.3e} (rho {res.rho:.3e})")

    # end-to-end: the host-buffer C ABI call, H2D of A and D2H of I, J, U inside
    e2e = None
    A_host = None
    if not a.no_e2e or (rank == 0 and ws == 1 and not a.no_cpu_baseline):
        log("copying A to pinned host memory")
        Ah = A.cpu().pin_memory()
        A_host = Ah.numpy()
    if not a.no_e2e:
        ctx.run_host(A_host, a.tol, a.block, a.sketch, a.seed, sketch_mode=a.sketch_mode)  # warm
        torch.cuda.synchronize()
        w0 = time.perf_counter()
        for _ in range(a.e2e_steps):
            r = ctx.run_host(A_host, a.tol, a.block, a.sketch, a.seed, sketch_mode=a.sketch_mode)
        torch.cuda.synchronize()
        e2e_ms = (time.perf_counter() - w0) * 1000.0 / a.e2e_steps
        log(f"e2e: {e2e_ms:.2f} ms per step")
        es = A_host.itemsize
        e2e = {"value": e2e_ms, "unit": "ms", "h2d_bytes_per_step": a.m * a.n * es,
               "d2h_bytes_per_step": 16 * r.rank + 8 * r.rank * r.rank + 8 * (r.iterations + 8)}
        # the copy floor on this machine: the same bytes, one plain pinned copy
        # into a device buffer (the host link's rate varies between machines)
        Ad = torch.empty_like(A)
        cms = []
        for _ in range(3):
            c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            c0.record()
            Ad.copy_(Ah, non_blocking=True)
            c1.record()
            c1.synchronize()
            cms.append(c0.elapsed_time(c1))
        del Ad
        copy_ms = sorted(cms)[1]
        e2e["h2d_copy_ms"] = copy_ms
        e2e["h2d_gbs"] = a.m * a.n * es / (copy_ms * 1e-3) / 1e9
        e2e["after_copy_ms"] = e2e_ms - copy_ms
        log(f"plain H2D copy of A: {copy_ms:.2f} ms ({e2e['h2d_gbs']:.1f} GB/s)")

    # roofline of the dominant kernel: the sketch of A (the one full pass)
    fp64_meas = ctx.fp64_tflops()
    a_bytes = float(a.m) * a.n * A.element_size()
    if a.sketch_mode == 5:
        achieved = a_bytes / (sketch_ms * 1e-3) / 1e9
        scales_ms = phase_ms["scales"]
        roofline = {"bound": "hbm", "achieved": achieved, "peak": HBM_GBS, "unit": "GB/s",
                    "frac": achieved / HBM_GBS, "traffic": traffic_for("sketch_fx.cu"),
                    "peak_source": f"{HBM_SRC} copy bandwidth",
                    "kernel": "sketch_fx_kernel<64> (FP64 tensor-core sketch, tcgen05 + TMA) "
                              "+ its 20 us reduction; algorithmic bytes m*n*8 per launch",
                    "kernel_ms": sketch_ms,
                    "sketch_phase": {"column_scales_ms": scales_ms, "total_ms": scales_ms + sketch_ms,
                                     "hbm_frac_over_two_reads":
                                         2 * a_bytes / ((scales_ms + sketch_ms) * 1e-3) / 1e9 / HBM_GBS}}
    elif a.sketch_mode == 0:
        flops = 2.0 * a.sketch * a.m * a.n
        achieved = flops / (sketch_ms * 1e-3) / 1e12
        roofline = {"bound": "alu", "achieved": achieved, "peak": fp64_meas, "unit": "TFLOP/s",
                    "frac": achieved / fp64_meas, "traffic": traffic_for("sketch_simt.cu"),
                    "peak_source": "measured FP64 FMA rate (cur_probe_fp64_tflops)",
                    "kernel": "sketch_kernel<FP64 A> (Y = G A, FP64 SIMT pipe)",
                    "kernel_ms": sketch_ms,
                    "hbm_frac_of_measured": a_bytes / (sketch_ms * 1e-3) / 1e9 / HBM_GBS}
    else:
        byts = 2.0 * a_bytes   # two reads of A: column scales, then the sketch pass
        achieved = byts / (sketch_ms * 1e-3) / 1e9
        roofline = {"bound": "hbm", "achieved": achieved, "peak": HBM_GBS, "unit": "GB/s",
                    "frac": achieved / HBM_GBS, "traffic": None,
                    "peak_source": f"{HBM_SRC} copy bandwidth",
                    "kernel": f"sketch phase, precision form ({a.sketch_mode} digits): colmax + "
                              "sketch_tc_kernel + reduce", "kernel_ms": sketch_ms}

    # the CPU oracle on the same matrix: all host cores and one core
    cpu = None
    if rank == 0 and ws == 1 and not a.no_cpu_baseline:
        cores = os.cpu_count() or 1
        log(f"cpu baseline: oracle on the whole matrix, {cores} threads")
        ms_all, ro = timed_oracle(a, A_host, cores)
        log(f"cpu baseline: {ms_all:.0f} ms ({cores} threads); one core next")
        ms_one, _ = timed_oracle(a, A_host, 1)
        log(f"cpu baseline: {ms_one:.0f} ms (1 thread)")
        cpu = {"value": ms_all, "unit": "ms", "cores": cores, "kind": "oracle",
               "one_core_ms": ms_one, "nproc": cores, "cpu_model": cpu_model(),
               "sample": f"one oracle run of the same method (same sketch form) on the whole "
                         f"{a.m}x{a.n} matrix with {cores} threads; one_core_ms: the same run "
                         "on one thread",
               "oracle_rank": ro.rank, "oracle_rho": ro.rho,
               "same_indices_as_gpu": bool(np.array_equal(np.asarray(ro.I), res.I) and
                                           np.array_equal(np.asarray(ro.J), res.J))}
    del A_host

    extra = {}
    if not a.no_extra_forms and a.dtype == "f64" and a.sketch_mode == 5:
        log("FP64-pipe Gaussian sketch on the same matrix")
        extra["fp64_pipe_sketch"] = time_form(A, a.tol, 0, 2, warm=1)

    # further forms of the configuration: tighter tolerances on the low-noise
    # spectrum, then the FP32 matrix
    second = None
    if not a.no_second_form:
        b2 = copy.copy(a)
        b2.tol, b2.noise = a.second_tol, a.second_noise
        del A
        torch.cuda.empty_cache()
        log("second form: generating A")
        A = make_matrix(b2, f"cuda:{local}", dtype)
        torch.cuda.synchronize()
        second = time_form(A, b2.tol, a.sketch_mode, max(2, a.steps // 2))
        second["workload"] = workload_name(b2)
        log(f"second form: {second['time_to_tolerance_ms']:.2f} ms, rank {second['rank']}")
        if not a.no_extra_forms:
            b3 = copy.copy(b2)
            b3.tol = 1e-4
            extra["tol_1e-4"] = time_form(A, 1e-4, a.sketch_mode, 2, warm=1)
            extra["tol_1e-4"]["workload"] = workload_name(b3)
            log(f"tol 1e-4: {extra['tol_1e-4']['time_to_tolerance_ms']:.2f} ms")
    if not a.no_extra_forms and a.dtype == "f64":
        b4 = copy.copy(a)
        b4.dtype = "f32"
        del A
        torch.cuda.empty_cache()
        log("FP32 forms: generating A")
        A = make_matrix(b4, f"cuda:{local}", torch.float32)
        torch.cuda.synchronize()
        for mode, key in ((0, "fp32_fp64_pipe_sketch"), (2, "fp32_tensor_core_2_digits")):
            b4.sketch_mode = mode
            extra[key] = time_form(A, a.tol, mode, 3)
            extra[key]["workload"] = workload_name(b4)
            log(f"{key}: {extra[key]['time_to_tolerance_ms']:.2f} ms")

    # the paper's own threshold experiment (Sec. 5.1), with the other forms
    paper = None
    if a.paper_workload or (not a.no_extra_forms and a.dtype == "f64"):
        from paper_2509_21963_gb300 import inputs
        del A
        torch.cuda.empty_cache()
        log("paper workload: generating the 30000^2 Low-Rank matrix")
        A = inputs.low_rank_gaussian_torch(30000, 30000, 2000, seed=5, device=f"cuda:{local}")
        torch.cuda.synchronize()
        pmode = 5
        st3, out3 = ctx.run_raw(A, 1e-6, 250, 275, a.seed, timing=True, sketch_mode=pmode)   # warm
        L.cur_result_free(out3)
        p0 = torch.cuda.Event(enable_timing=True)
        p1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        p0.record(stream)
        st3, out3 = ctx.run_raw(A, 1e-6, 250, 275, a.seed, timing=True, sketch_mode=pmode)
        p1.record(stream)
        torch.cuda.synchronize()
        r3 = int(L.cur_result_rank(out3))
        res3 = cur._result_from(out3)
        L.cur_result_free(out3)
        # true relative error ||A - C U R||_F / ||A||_F on the device (FP64)
        Jt = torch.from_numpy(res3.J).to(A.device)
        It = torch.from_numpy(res3.I).to(A.device)
        Ut = torch.from_numpy(res3.U).to(A.device)
        E = A - (A[:, Jt] @ Ut) @ A[It, :]
        terr = float(torch.linalg.norm(E) / torch.linalg.norm(A))
        del E
        ms3 = p0.elapsed_time(p1)
        paper = {"workload": "Low-Rank 30000x30000 FP64 (G1 G2^T, rank 2000), tol 1e-6, b=250, c=275, "
                             + SKETCH_FORMS[pmode],
                 "time_to_tolerance_ms": ms3, "rank": r3, "rho": res3.rho,
                 "true_rel_error": terr, "phase_ms": res3.phase_ms,
                 "paper_ms_48core_cpu": 12000.0, "ratio_vs_paper": ms3 / 12000.0}
        log(f"paper workload: {ms3:.1f} ms, rank {r3}, true error {terr:.2e}")

    if rank == 0:
        line = {
            "metric": "time-to-tolerance per CUR", "value": value, "unit": "ms", "n_gpus": ws,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms_per_step,
            "step_ms": step_ms,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": {0: "f64", 5: "f64 loop; sketch on bf16 tensor cores, exact 52-bit fixed point"}.get(
                a.sketch_mode, f"bf16x{a.sketch_mode} sketch, f64 loop"),
            "data": "synthetic",
            "config": {"workload": workload_name(a), "m": a.m, "n": a.n, "tol": a.tol,
                       "block_size": a.block, "sketch_size": a.sketch, "a_dtype": a.dtype,
                       "sketch_mode": a.sketch_mode,
                       "rank": rank_r, "iterations": iters, "rho": rho, "status": status,
                       "true_rel_error": true_err,
                       "l2": "inputs larger than L2 (A is resident in HBM)",
                       "parallelism": f"replicas x{ws}"},
            "gpu_launches": launches * a.steps,
            "clocks": clk, "e2e": e2e, "roofline": roofline, "cpu_baseline": cpu,
            "fp64_peak": {"measured_tflops": fp64_meas, "nominal_tflops": FP64_PEAK_TFLOPS},
            "phase_ms": phase_ms, "second_form": second, "forms": extra, "paper_workload": paper,
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
