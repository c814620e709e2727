#!/usr/bin/env python
"""Throughput of the PSWF fast Ewald hot path on GB300 (one JSON line on rank 0).

Workload: n = 100,000 uniform neutral charges (rho ~ U[-1,1] minus the mean) in the
unit box, relative tolerance 1e-6, mixed precision (the metric's headline form).  One
"step" is one full evaluation: bin/sort, spread, FFT, scale, inverse FFT, interpolate
(phi and forces), real-space sum, self term and energy.  Inputs are resident in HBM when
the timed region starts; L2 is flushed (256 MB write) between timed steps, outside the
events that bracket each step.  Under torchrun every rank evaluates its own independent
system (replicas, weak scaling); the time reported is the max over ranks.

--impl reference times the FP64 CPU oracle (the converged Ewald sum) on the host cores
on a bounded sample of the same workload; it never touches the GPU.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle evals/s (phi+forces) at rel tol 1e-6/1e-10, mixed vs FP64 GPU form"
UNIT = "particle evals/s"
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12     # SMs x FP32 lanes x 2 (FMA) x max SM clock
FP64_PEAK_TFLOPS = 1.25                               # nominal GB300 FP64 (non-tensor)
REF_TARGETS = 8                                       # oracle sample per reference step


def _env_int(k, d):
    try:
        return int(os.environ.get(k, d))
    except ValueError:
        return d


def workload_config(n, tol, precision):
    return {
        "workload": "uniform neutral charges n=%d, rho~U[-1,1] minus mean, L=1, rel tol %g, %s" % (n, tol, precision),
        "n": n, "tol": tol, "precision": precision, "L": 1.0,
        "l2": "flushed between timed steps (256 MB write, outside the step events)",
        "parallelism": "replicas (one independent system per GPU)",
    }


# ------------------------------------------------------------------ oracle timing (CPU) --
# The oracle runs as it stands in worker processes started with "spawn" (the parent may already hold a
# CUDA context), one per host core, each with one BLAS/OpenMP thread.

def _oracle_exact_sample(args):
    """Worker: the converged PSWF Ewald sum (O-exact) of the n-particle system for the given targets."""
    n, targets, seed = args
    import numpy as np
    from oracle import exact
    from workloads import uniform_neutral
    x, rho, L = uniform_neutral(n, seed=seed)
    t = time.perf_counter()
    exact.pswf_exact(x, rho, L, targets=np.asarray(targets, dtype=np.int64))
    return time.perf_counter() - t


def _oracle_alg2_sample(args):
    """Worker: Alg. 2 restated on the CPU (O-alg2) with a plan's parameters: spread and FFTs over all n,
    potential and forces at the given targets (real-space sum included)."""
    n, seed, prm, targets = args
    import numpy as np
    from oracle.alg2 import Alg2
    from workloads import uniform_neutral
    x, rho, L = uniform_neutral(n, seed=seed)
    A = Alg2(L, prm["m"], prm["P"], prm["cs"], prm["cw"], prm["rc"])
    t = time.perf_counter()
    A.total(x, rho, targets=np.asarray(targets, dtype=np.int64))
    return time.perf_counter() - t


class OraclePool:
    """A pool of `cores` spawned worker processes running the oracle on the host cores."""

    def __init__(self, cores=None):
        import multiprocessing as mp
        from concurrent.futures import ProcessPoolExecutor
        self.cores = int(cores or os.cpu_count() or 1)
        for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            os.environ[k] = "1"
        self.ex = ProcessPoolExecutor(self.cores, mp_context=mp.get_context("spawn"))

    def exact_round(self, n, per_worker, seed=0):
        """Every core evaluates its own `per_worker` targets (structure factor included); wall seconds."""
        step = max(1, n // (self.cores * per_worker))
        jobs = [(n, [(w * per_worker + k) * step % n for k in range(per_worker)], seed) for w in range(self.cores)]
        t = time.perf_counter()
        list(self.ex.map(_oracle_exact_sample, jobs))
        return time.perf_counter() - t

    def alg2(self, n, prm, targets, seed=0):
        return self.ex.submit(_oracle_alg2_sample, (n, seed, prm, list(targets))).result()

    def close(self):
        self.ex.shutdown()


def host_cpu():
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                if line.lower().startswith(("model name", "cpu part")):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    n = args.n
    pool = OraclePool()
    times = []
    for k in range(args.warmup + args.steps):
        s = pool.exact_round(n, REF_TARGETS)
        if k >= args.warmup:
            times.append(s)
    pool.close()
    t = sum(times) / len(times)
    value = pool.cores * REF_TARGETS / t
    sample = ("phi+F at %d targets per core per step, %d cores in parallel, of the %d-particle system (oracle: "
              "FP64 converged PSWF Ewald sum, c_s=34, r_c=L/2, all-source structure factor, k-sphere |k|<=14)"
              % (REF_TARGETS, pool.cores, n))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * t, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(n, args.tol, args.precision),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": pool.cores, "kind": "oracle", "sample": sample,
                         "cpu": host_cpu()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------- clocks --
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return None
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [v.strip() for v in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------------------------------- work models --
def algorithmic_flops(stage, p, n, pairs):
    """Algorithmic flops of one launch (FMA = 2 flops): window Horner + tensor-product stencil for
    spread / interp, 100 flop per pair inside r_c for the real-space sum (rsqrt, two radial Horners)."""
    P, dw, dr = p.P, p.deg_w, p.deg_r
    if stage == "spread":
        return n * 2 * (P ** 3 + P ** 2 + 3 * P * (dw + 1))
    if stage == "interp":
        return n * 2 * (2 * P ** 3 + 6 * P ** 2 + 6 * P * (dw + 1))
    if stage == "short":
        return pairs * 100
    return None


def hbm_peak():
    """Measured copy bandwidth (GB/s) from MEASURED_PEAKS.json, else the fallback figure."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured (MEASURED_PEAKS.json)"
    except (OSError, ValueError, KeyError, TypeError):
        return 6800.0, "fallback 6.8 TB/s"


def algorithmic_bytes(stage, p, n, precision):
    """Algorithmic bytes of one launch: the minimum data a stage must read and write once."""
    grid = [int(v) for v in p.grid]
    m3 = grid[0] * grid[1] * grid[2]
    word = 4 if precision == "f32" else 8                    # grid value (float-float grids: float2)
    rec = {"f32": 24, "f64": 40, "ff": 40}[precision]       # sorted spreading record + index per particle
    if stage == "sort":
        out = {"f32": 64, "f64": 96, "ff": 84}[precision]
        return n * (32 + 32 + out)                          # x, rho in; keys out and back; records out
    if stage == "spread":
        return n * rec + m3 * word
    if stage == "halo":
        return slab_values(p) * word + m3 * word            # tile slabs in, grid out
    if stage == "scale":
        nspec = grid[0] * grid[1] * (grid[2] // 2 + 1)
        return nspec * 2 * (8 if precision == "f32" else 16)
    if stage == "interp":
        return n * rec + m3 * word + n * 32                 # records and grid in, phi and F out
    if stage == "short":
        return n * ({"f32": 32, "f64": 48, "ff": 36}[precision] + (16 if precision == "f32" else 32))
    if stage == "energy":
        return n * (88 if precision == "f32" else 104)
    return None


def stage_rooflines(stages_serial, p, n, pairs, precision):
    """Per-stage achieved bandwidth and flop rate against the HBM and ALU peaks (serialised stage times)."""
    try:
        hbm, hbm_src = hbm_peak()
        alu = FP64_PEAK_TFLOPS if precision == "f64" else FP32_PEAK_TFLOPS
        out = []
        for st in ("sort", "spread", "halo", "scale", "interp", "short", "energy"):
            t = stages_serial.get(st)
            if not t or t <= 0:
                continue
            b = algorithmic_bytes(st, p, n, precision)
            fl = algorithmic_flops(st, p, n, pairs)
            row = {"stage": st, "us": 1000.0 * t}
            if b:
                gbs = b / (t / 1000.0) / 1e9
                row.update({"bytes": b, "GB/s": gbs, "frac_hbm": gbs / hbm})
            if fl:
                tf = fl / (t / 1000.0) / 1e12
                row.update({"flops": fl, "TFLOP/s": tf, "frac_alu": tf / alu})
            out.append(row)
        return {"hbm_peak_gbs": hbm, "hbm_peak_source": hbm_src, "alu_peak_tflops": alu, "stages": out}
    except Exception as e:   # reporting only: never fail the bench line
        return {"error": repr(e)}


# device.cuh section (first line prefix) holding each stage's kernel; the float-float kernels live in
# ff_kernels.cuh
SECTION_OF = {"short": "// ---- real-space sum", "interp": "// ---- Alg. 2 step 5", "spread": "// ---- Alg. 2 step 1:",
              "halo": "// ---- Alg. 2 step 1 (continued)"}


def source_digest(stage, precision):
    """sha1 prefix of the source a stage's kernel is compiled from (its device.cuh section)."""
    csrc = os.path.join(ROOT, "paper_2602_16591_gb300", "csrc")
    if precision == "ff":
        text = open(os.path.join(csrc, "ff_kernels.cuh")).read()
    else:
        text = open(os.path.join(csrc, "device.cuh")).read()
        marker = SECTION_OF.get(stage)
        if marker is None or marker not in text:
            return None
        i = text.index(marker)
        j = text.find("\n// ---- ", i + 1)
        text = text[i:j if j >= 0 else len(text)]
    return hashlib.sha1(text.encode()).hexdigest()[:12]


def traffic_for(stage, n, p, precision):
    """Per-launch DRAM bytes from the committed ncu summary, if taken on the current kernel source."""
    path = os.path.join(ROOT, "profiles", "roofline_traffic.txt")
    if not os.path.exists(path):
        return None
    digest = source_digest(stage, precision)
    for line in open(path):
        f = line.split()
        if len(f) >= 6 and not line.startswith("#") and f[0] == stage and int(f[1]) == n and int(f[2]) == p.P \
                and f[3] == precision and f[5] == digest:
            return float(f[4])
    return None


# ---------------------------------------------------------------------- multi-rank --
def max_over_ranks(value, dist=None, device="cuda"):
    """Max of a host float over all ranks (replica timing); identity without a process group."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_value(n_per_rank, world, ms_max):
    """Whole-job throughput: every rank evaluates n_per_rank particles per step."""
    return world * n_per_rank / (ms_max / 1000.0)


# ------------------------------------------------------------------ stored oracle values --
GOLDEN = {100_000: "uniform1e5_seed0.txt", 10_000_000: "uniform1e7_seed0.txt"}
VARIANTS = ((1e-4, "mixed"), (1e-6, "fp64"), (1e-8, "mixed"), (1e-10, "mixed"), (1e-10, "fp64"), (1e-12, "mixed"))
LARGE_N, LARGE_TOL, LARGE_DENSITIES = 10_000_000, 1e-8, (1.0, 4.0, 13.0)
LARGE_SCRATCH_GB = 60.0          # plans whose workspace would exceed this are reported, not run
CPU_TARGETS = 16                 # O-exact targets per host core in the CPU baseline


def read_golden(n):
    """Stored oracle values (targets, phi, F, E or None) of uniform_neutral(n, seed=0), when committed.
    They are written by tests/golden/make_reference_values.py, which calls only the oracle."""
    name = GOLDEN.get(n)
    path = os.path.join(ROOT, "tests", "golden", name) if name else None
    if not path or not os.path.exists(path):
        return None
    import numpy as np
    E, rows = None, []
    with open(path) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            f = line.split()
            if f[0] == "E":
                E = float(f[1])
            else:
                rows.append([float(v) for v in f])
    a = np.array(rows)
    return a[:, 0].astype(np.int64), a[:, 1], a[:, 2:5], E


def result_errors(phi, F, E, gold):
    """Errors of one evaluation against the stored oracle values: relative l2 of phi and of F over the
    stored targets, relative energy error (when stored), worst particle relative to the RMS."""
    if gold is None:
        return None
    import numpy as np
    tg, rphi, rF, rE = gold
    import torch
    ti = torch.as_tensor(tg, device=phi.device)
    p = phi[ti].double().cpu().numpy()
    f = F[ti].double().cpu().numpy()
    rel = lambda a, r: float(np.linalg.norm(a - r) / np.linalg.norm(r))   # noqa: E731
    out = {"err_phi": rel(p, rphi), "err_F": rel(f, rF),
           "err_E": abs(E - rE) / abs(rE) if (rE is not None and E is not None) else None,
           "worst_phi": float(np.max(np.abs(p - rphi)) / np.sqrt(np.mean(rphi ** 2))),
           "worst_F": float(np.max(np.linalg.norm(f - rF, axis=1)) / np.sqrt(np.mean(np.sum(rF ** 2, axis=1)))),
           "targets": int(len(tg)), "reference": "stored oracle values (converged PSWF Ewald sum)"}
    return out


def slab_values(p):
    """Tile-slab values of a plan: a head of T x-planes per tile and a tail of E - T planes per x-chain of
    K tiles (K the largest divisor of the x tile count with K T <= 32), E x E values per plane."""
    grid = [int(v) for v in p.grid]
    T, E = p.tile, p.tile + p.P - 1
    nt = [g // T for g in grid]
    K = max(k for k in range(1, 32 // T + 1) if nt[0] % k == 0)
    ntiles = nt[0] * nt[1] * nt[2]
    return ntiles * T * E * E + (ntiles // K) * (E - T) * E * E


def plan_workspace_gb(p, n):
    """Device workspace of a plan (the tile slabs dominate), in GB."""
    word = 4 if p.precision == 1 else 8
    grid = [int(v) for v in p.grid]
    m3 = grid[0] * grid[1] * grid[2]
    return (slab_values(p) * word + 4 * m3 * word + n * 400) / 1e9


# ------------------------------------------------------------------------- main run --
def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch

    import paper_2602_16591_gb300 as pe
    from workloads import uniform_neutral

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))

    def barrier():
        if dist is not None:
            dist.barrier()

    def reduce_max(v):
        return max_over_ranks(v, dist, "cuda")

    n = args.n
    x_np, rho_np, L = uniform_neutral(n, seed=rank)
    x = torch.tensor(x_np, device="cuda")
    rho = torch.tensor(rho_np, device="cuda")
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    gold = read_golden(n) if rank == 0 else None

    def timed(plan, steps, warmup, profile=False, xr=None, serial=False):
        xx, rr = (x, rho) if xr is None else xr
        nn = len(rr)
        phi = torch.empty(nn, dtype=torch.float64, device="cuda")
        F = torch.empty(nn, 3, dtype=torch.float64, device="cuda")
        for _ in range(warmup):
            plan.eval(xx, rr, phi, F, energy=False)
        torch.cuda.synchronize()
        if profile:
            plan.profile(True, serial=serial)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        torch.cuda.synchronize()
        barrier()
        for k in range(steps):
            flush.zero_()
            ev[k][0].record(stream)
            plan.eval(xx, rr, phi, F, energy=False)
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        barrier()
        ms = sum(a.elapsed_time(b) for a, b in ev)
        stages = None
        if profile:
            stages, cnt = plan.profile_read()
            plan.profile(False)
            stages = {k: v / cnt for k, v in stages.items()}
        plan.check()
        return ms / steps, stages

    def errors_of(plan, g, xr=None):
        """One more evaluation of the timed plan (with the energy) against the stored oracle values."""
        if g is None:
            return None
        xx, rr = (x, rho) if xr is None else xr
        phi, F, E = plan.eval(xx, rr)
        torch.cuda.synchronize()
        return result_errors(phi, F, E, g)

    gpu_index = local_rank
    cvd = os.environ.get("CUDA_VISIBLE_DEVICES")
    if cvd:
        try:
            gpu_index = int(cvd.split(",")[local_rank])
        except (ValueError, IndexError):
            pass

    # the plan's grid density (the real-space / Alg. 2 balance) is tuned at plan creation unless given
    popts = {"autotune": 0, "grid_density": args.grid_density} if args.grid_density is not None else \
        {"autotune": 0 if args.no_autotune else 1}
    plan = pe.Plan(L, n, args.tol, precision=args.precision, **popts)
    with ClockSampler(gpu_index) as clk:
        ms_local, _ = timed(plan, args.steps, args.warmup, profile=False)
    clocks = clk.summary()
    # per-stage event times (concurrent, as in the timed steps) from a separate profiled run
    _, stages = timed(plan, min(60, args.steps), 2, profile=True)
    ms = reduce_max(ms_local)
    value = aggregate_value(n, world, ms)
    headline_err = errors_of(plan, gold)

    # end to end through the public API with host buffers (pinned), copies inside the timed region
    xh = torch.empty((n, 3), dtype=torch.float64, pin_memory=True).numpy()
    rh = torch.empty(n, dtype=torch.float64, pin_memory=True).numpy()
    xh[:] = x_np
    rh[:] = rho_np
    # results into page-locked host arrays owned by the caller
    outs = (torch.empty(n, dtype=torch.float64, pin_memory=True).numpy(),
            torch.empty((n, 3), dtype=torch.float64, pin_memory=True).numpy())
    try:
        plan.eval_host(xh, rh, *outs)
        e2e_outputs = "page-locked"
    except (TypeError, ValueError):
        outs = ()
        e2e_outputs = "allocated per call"
    for _ in range(args.warmup):
        plan.eval_host(xh, rh, *outs)
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        plan.eval_host(xh, rh, *outs)
    e2e_s = (time.perf_counter() - t0) / args.steps
    e2e_s = reduce_max(e2e_s)

    p = plan.params
    # dominant kernel of the step and its roofline
    rc = p.rc
    pairs = n * (n - 1) * (4.0 / 3.0) * np.pi * rc ** 3 / L ** 3
    # kernel durations without overlap for the roofline: a few more steps with the real-space sum and
    # Alg. 2 serialised on one stream (same kernels; the concurrent stage times above include waiting)
    _, stages_serial = timed(plan, 5, 2, profile=True, serial=True)
    ours = {k: v for k, v in stages_serial.items() if k not in ("fft_fwd", "fft_inv")}
    dom = max(ours, key=ours.get)
    fl = algorithmic_flops(dom, p, n, pairs)
    prec_tag = pe.PATH_NAMES[p.precision]
    peak = FP64_PEAK_TFLOPS if prec_tag == "f64" else FP32_PEAK_TFLOPS
    roofline = None
    if fl is not None:
        ach = fl / (stages_serial[dom] / 1000.0) / 1e12
        roofline = {"bound": "alu", "kernel": dom, "timing": "stage events with the stages serialised (ewald_profile 2)",
                    "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                    "frac": ach / peak, "traffic": traffic_for(dom, n, p, prec_tag),
                    "flops_per_launch": fl, "count": "100 flop per pair inside r_c" if dom == "short" else
                    "window Horner + tensor-product stencil per particle",
                    "peak_source": "nominal GB300 FP64 1.25 TFLOP/s" if prec_tag == "f64"
                    else "derived: 152 SMs x 128 FP32 lanes x 2 x 2.07 GHz"}

    variants = []
    if not args.no_variants:
        for tol, prec in VARIANTS:
            vp = pe.Plan(L, n, tol, precision=prec, **popts)
            vms, vst = timed(vp, min(60, max(5, args.steps // 3)), 2, profile=True)
            vms = reduce_max(vms)
            variants.append({"tol": tol, "precision": prec,
                             "path": pe.PATH_NAMES[vp.params.precision],
                             "m": vp.params.m, "P": vp.params.P, "ms_per_step": vms,
                             "value": world * n / (vms / 1000.0), "stages_ms": vst,
                             "errors": errors_of(vp, gold)})
            del vp

    if not args.no_variants:
        # cuboid box (Remark on cuboid domains): the headline density in a 1 x 1 x 2 box, twice the particles
        from workloads import uniform_neutral_box
        cb = (1.0, 1.0, 2.0)
        cxn, crn, _ = uniform_neutral_box(2 * n, cb, seed=rank)
        cxr = (torch.tensor(cxn, device="cuda"), torch.tensor(crn, device="cuda"))
        cp = pe.Plan(cb, 2 * n, args.tol, precision=args.precision, **popts)
        cms, cst = timed(cp, min(60, max(5, args.steps // 3)), 3, profile=True, xr=cxr)
        cms = reduce_max(cms)
        variants.append({"tol": args.tol, "precision": args.precision, "box": list(cb), "n": 2 * n,
                         "path": pe.PATH_NAMES[cp.params.precision], "grid": list(cp.params.grid), "P": cp.params.P,
                         "ms_per_step": cms, "value": world * 2 * n / (cms / 1000.0), "stages_ms": cst})
        del cp, cxr

    batch = None
    if not args.no_variants:
        # batched workload: 256 independent systems, n log-uniform in [500, 20000], L = (n/100)^(1/3).  With
        # several ranks the ONE batch is split over them (cost-model bin packing, no exchange while
        # evaluating; the timed region covers each rank's own share, max over ranks)
        from workloads import batched_systems
        from paper_2602_16591_gb300 import shard
        systems = batched_systems(nsys=256, seed=0)
        bLs = np.array([sy[2] for sy in systems])
        bns = np.array([len(sy[1]) for sy in systems], dtype=np.int64)
        t0 = time.perf_counter()
        if world > 1:
            sp = shard.ShardedBatchPlan(bLs, bns, 1e-6, rank=rank, world=world, precision="mixed")
            mine = sp.share[rank]
            bp = sp.plan
        else:
            mine = list(range(len(systems)))
            bp = pe.BatchPlan(bLs, bns, 1e-6, precision="mixed")
        plan_s = time.perf_counter() - t0
        bx = torch.tensor(np.concatenate([systems[i][0] for i in mine]), device="cuda")
        brho = torch.tensor(np.concatenate([systems[i][1] for i in mine]), device="cuda")
        bphi = torch.empty(len(brho), dtype=torch.float64, device="cuda")
        bF = torch.empty(len(brho), 3, dtype=torch.float64, device="cuda")
        for _ in range(3):
            bp.eval(bx, brho, bphi, bF)
        reps = min(60, max(5, args.steps // 3))
        torch.cuda.synchronize()
        barrier()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            flush.zero_()
            bp.eval(bx, brho, bphi, bF)
        b.record(stream)
        torch.cuda.synchronize()
        bms = reduce_max(a.elapsed_time(b) / reps)
        N = int(bns.sum())
        batch = {"workload": "256 independent systems, n log-uniform in [500, 20000] (total %d), L = (n/100)^(1/3), "
                             "rel tol 1e-6, mixed; one call per step, energies copied back" % N,
                 "ms_per_step": bms, "value": N / (bms / 1000.0), "unit": UNIT,
                 "systems_per_s": 256 / (bms / 1000.0), "plan_seconds": plan_s,
                 "scaling": "strong" if world > 1 else None,
                 "sharding": "one batch split over %d ranks by cost (shard.py)" % world if world > 1 else None}
        del bp, bx, brho, bphi, bF

    large = None
    if not args.no_large:
        large = run_large(pe, torch, np, timed, errors_of, reduce_max, world, rank)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        pool = OraclePool()
        pool.exact_round(n, 1)                         # start-up (imports, first structure factor)
        s = pool.exact_round(n, CPU_TARGETS)
        tg = np.linspace(0, n - 1, 256).astype(np.int64)
        prm = {"m": p.m, "P": p.P, "cs": p.cs, "cw": p.cw, "rc": p.rc}
        s2 = pool.alg2(n, prm, tg)
        pool.close()
        cv = pool.cores * CPU_TARGETS / s
        cpu = {"value": cv, "unit": UNIT, "cores": pool.cores, "per_core": cv / pool.cores, "kind": "oracle",
               "cpu": host_cpu(),
               "sample": "O-exact (FP64 converged PSWF Ewald sum incl. the all-source structure factor): phi+F at "
                         "%d targets of the %d-particle system on each of %d cores in parallel, %.1f s wall"
                         % (CPU_TARGETS, n, pool.cores, s),
               "o_alg2": {"value": 256 / s2, "unit": UNIT, "cores": 1, "seconds": s2,
                          "sample": "Alg. 2 restated on the CPU with the headline plan (m=%d, P=%d): spread and "
                                    "FFTs over all %d particles, phi+F at 256 targets, one process" % (p.m, p.P, n)}}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": prec_tag, "data": "synthetic",
            "config": dict(workload_config(n, args.tol, args.precision), m=p.m, P=p.P, rc=p.rc, cs=p.cs, cw=p.cw,
                           deg_w=p.deg_w, deg_r=p.deg_r, tile=p.tile, plan=dict(popts)),
            "errors": headline_err,
            "roofline": roofline, "cpu_baseline": cpu,
            "e2e": {"value": world * n / e2e_s, "unit": UNIT, "h2d_bytes_per_step": 32 * n,
                    "d2h_bytes_per_step": 32 * n + 8, "host_buffers": "page-locked inputs, results " + e2e_outputs},
            # own kernels per step: prep, scan, place, rerank, scatter, real-space, spread, halo, scale,
            # (float-float: grid conversion,) interpolation, combine + energy; cuFFT's kernels are not counted
            "gpu_launches": (12 if prec_tag == "ff" else 11) * args.steps,
            "stages_serial_ms": stages_serial,
            "stage_rooflines": stage_rooflines(stages_serial, p, n, pairs, prec_tag),
            "clocks": clocks, "stages_ms": stages, "variants": variants,
            "batched": batch, "large": large,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def run_large(pe, torch, np, timed, errors_of, reduce_max, world, rank):
    """The large configuration: n = 1e7 uniform neutral charges, tol 1e-8, grid densities 1, 4, 13 (m up to
    512), float64 grid + FFT with float64 particles vs float-float particles (the MIXED path at this tol).
    Inputs exceed L2 (320 MB), so no flush is needed.  Per-stage rooflines from serialised stage events."""
    from workloads import uniform_neutral
    xn, rn, L = uniform_neutral(LARGE_N, seed=rank)
    xr = (torch.tensor(xn, device="cuda"), torch.tensor(rn, device="cuda"))
    del xn, rn
    gold = read_golden(LARGE_N) if rank == 0 else None
    runs = []
    for g in LARGE_DENSITIES:
        for prec in ("fp64", "mixed"):
            q = pe.plan_params(L, LARGE_N, LARGE_TOL, precision=prec, grid_density=g)
            gb = plan_workspace_gb(q, LARGE_N)
            row = {"grid_density": g, "precision": prec, "path": pe.PATH_NAMES[q.precision], "m": q.m, "P": q.P,
                   "tile": q.tile, "rc": q.rc, "workspace_gb": gb}
            if gb > LARGE_SCRATCH_GB:
                row["skipped"] = "workspace %.0f GB above the bench's %.0f GB bound" % (gb, LARGE_SCRATCH_GB)
                runs.append(row)
                continue
            lp = pe.Plan(L, LARGE_N, LARGE_TOL, precision=prec, grid_density=g, autotune=0)
            lms, _ = timed(lp, 3, 2, xr=xr)
            _, lst = timed(lp, 2, 1, xr=xr, profile=True, serial=True)
            lms = reduce_max(lms)
            tag = pe.PATH_NAMES[lp.params.precision]
            row.update({"ms_per_step": lms, "value": world * LARGE_N / (lms / 1000.0), "stages_serial_ms": lst,
                        "stage_rooflines": stage_rooflines(lst, lp.params, LARGE_N,
                                                           LARGE_N * (LARGE_N - 1) * 4.0 / 3.0 * np.pi * q.rc ** 3,
                                                           tag),
                        "errors": errors_of(lp, gold, xr)})
            runs.append(row)
            del lp
            torch.cuda.empty_cache()
    return {"workload": "n=%d uniform neutral charges, rho~U[-1,1] minus mean, L=1, rel tol %g; grid densities "
                        "%s; fp64 = float64 particles, grid and FFT; mixed = float-float particles (float32 "
                        "pipes, ~48 bits) with float64 grid and FFT" % (LARGE_N, LARGE_TOL, list(LARGE_DENSITIES)),
            "unit": UNIT, "runs": runs}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                help="timed steps (default: 1000 for this implementation, 3 oracle samples for --impl reference)")
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=("ours", "reference"))
    ap.add_argument("--n", type=int, default=100_000)
    ap.add_argument("--tol", type=float, default=1e-6)
    ap.add_argument("--precision", default="mixed", choices=("mixed", "fp64", "floatfloat"))
    ap.add_argument("--grid-density", type=float, default=None, help="m^3/n target of the cutoff rule")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="plan with the default grid density")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-large", action="store_true", help="skip the n = 1e7 configuration")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.steps is None:
        # enough steps that the clock sampler sees the timed region several times (~0.5 s at 0.45 ms a step)
        args.steps = 3 if args.impl == "reference" else 1000
    rank = _env_int("RANK", 0)
    world = _env_int("WORLD_SIZE", 1)
    local_rank = _env_int("LOCAL_RANK", 0)
    if args.impl == "reference":
        return run_reference(args, rank, world)
    return run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    sys.exit(main())
