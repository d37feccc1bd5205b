"""Benchmark of the QED Monte-Carlo particle step on GB300.

Workload (one bench "step" = one complete job): head-on collision of 1e6 electrons
(gamma0 ~ N(2000, 5%), 1e-3 rad divergence) with a linearly polarised plane-wave pulse
(lambda = 1 um, a0 = 100, sin^2 envelope of 30 fs intensity FWHM), dt = lambda/(100 c),
4000 time steps, photon emission and pair production on, mixed precision (FP32 state and push,
FP64 optical depth).  Every time step runs the whole hot path: field evaluation, Boris push,
eta/chi, rate look-up, optical-depth advance, sampling, recoil, append, ordered merge, ledgers.

Metric: particle-steps/s (alive particles pushed per second, all species).
  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "QED MC particle-steps/s (mixed FP32/FP64 vs plain FP64) at <=1e-5 rel err; p50/p99 latency"
UNIT = "particle-steps/s"
# algorithmic bytes per particle-step of the step kernel (read + write), mixed precision:
# e+-: x,u (6 x 4 B) + tau (8 B) read and written;  photons: x,k,tau read (32 B), x written (12 B),
# and tau written (8 B) when the photon is in a field (its optical depth changed); each created
# particle: one append-slot write (6 x 4 + 8 + 4 B).  FP64: 8-byte positions and momenta.
BYTES = {"mixed": {"lepton": 64, "photon": 44, "tau": 8, "child": 36},
         "fp64": {"lepton": 112, "photon": 72, "tau": 8, "child": 60}}


def algorithmic_bytes(b, lep, ph, tau_ph, created):
    """Bytes the per-step kernel must move for these pushes and children (see BYTES)."""
    return lep * b["lepton"] + ph * b["photon"] + tau_ph * b["tau"] + created * b["child"]


def env_rank():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


def workload_name(n, steps):
    return f"head_on_LP_a0=100_gamma0=2000_lambda=1um_fwhm=30fs_{n:.0e}_electrons_{steps}_steps"


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------- our arm
class Job:
    """One complete collision run on the GPU through the C ABI."""

    def __init__(self, qed, tables, w, precision, rank, torch, multistep=0):
        self.qed, self.tables, self.w, self.torch = qed, tables, w, torch
        self.multistep = multistep
        n = w.n
        prec = qed.MIXED if precision == "mixed" else qed.FP64
        self.prec = prec
        # capacities: photons grow to ~50 per electron in this pulse; pairs are rare
        self.e = qed.Species(qed.ELECTRON, prec, 2 * n + 4096, n + 4096)
        self.p = qed.Species(qed.POSITRON, prec, n + 4096, n + 4096)
        self.g = qed.Species(qed.PHOTON, prec, 80 * n + 4096, 2 * n + 4096)
        dt = torch.float32 if prec == qed.MIXED else torch.float64
        xr = w.x.copy()
        xr[:, 0] -= w.window_x0
        # pristine initial state resident in HBM (device columns), copied in at the start of a job
        self.cols = [torch.tensor(np.ascontiguousarray(a[:, c]), dtype=dt, device="cuda")
                     for a in (xr, w.u) for c in range(3)]
        self.empty = qed.Soa(*([None] * 8))
        self.params = qed.StepParams(dt=w.dt, seed=w.seed, scenario=rank, field=qed.Field(**w.field.as_dict()),
                                     emit_photons=True, make_pairs=True, window_x0=w.window_x0, window_v=w.window_v)
        self.rank = rank

    def reset(self, stream=None):
        qed = self.qed
        soa = qed.Soa(*[c.data_ptr() for c in self.cols], None, None)
        self.e.upload_soa(soa, self.w.n, self.w.n, stream)
        self.e.init_tau(self.w.seed, self.rank, stream)
        self.p.upload_soa(self.empty, 0, 0, stream)
        self.g.upload_soa(self.empty, 0, 0, stream)

    step_log = None  # list of per-step work counters, when requested (profiling runs only)

    def run(self, stream=None):
        sp = [self.e, self.p, self.g]
        if self.step_log is None:
            if self.multistep:
                self.qed.run_multistep(self.tables, sp, self.params, 0, self.w.n_steps, self.multistep, stream)
            else:
                self.qed.run(self.tables, sp, self.params, 0, self.w.n_steps, stream)
            return
        # same steps, one call each, with the cumulative work counters read after every step and
        # the device time of each call (step kernel and finalisation) from events around it
        import torch

        st = torch.cuda.current_stream() if stream is None else stream
        for k in range(self.w.n_steps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(st)
            self.qed.run(self.tables, sp, self.params, k, 1, stream)
            b.record(st)
            b.synchronize()
            self.step_log.append(tuple(self.qed.work_read(self.e, stream=stream)) + (a.elapsed_time(b),))


def flush_l2(torch, buf):
    buf.add_(1.0)  # 256 MiB write, larger than the 129 MB L2


def our_arm(args):
    import torch

    from paper_1311_5551_gb300 import build as qbuild
    from paper_1311_5551_gb300 import qed, workloads as W

    rank, world, local = env_rank()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    qbuild.build()
    qed.load_library()
    tables = qed.Tables()
    w = W.head_on(n=args.n, n_steps=args.time_steps, seed=2)
    job = Job(qed, tables, w, args.precision, rank, torch, args.multistep)
    flush_buf = torch.zeros(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    # the warm-up jobs run with the kernel timers on, so that their event pools are filled before
    # the timed jobs (which then reuse them: no event is created inside a timed job)
    qed.timing_enable(True)
    for _ in range(args.warmup):
        job.reset()
        job.run()
        qed.timing_read(reset=True)
        qed.timing_read_multistep(reset=True)
    barrier()
    if args.step_log:
        job.step_log = []

    # ---------------- timed region: K complete jobs, device time by CUDA events per job
    qed.work_read(job.e, reset=True)
    qed.timing_read(reset=True)
    qed.timing_read_multistep(reset=True)
    launches0 = qed.launch_count()
    step_ms, step_launches, multi_ms, multi_passes = 0.0, 0, 0.0, 0
    clocks = ClockSampler(local)
    clocks.start()
    ev = []
    for _ in range(args.steps):
        job.reset()
        flush_l2(torch, flush_buf)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        job.run()
        e1.record(stream)
        ev.append((e0, e1))
        # the kernel timers of this job (waits for it; the next job's events start after)
        m, n = qed.timing_read(reset=True)
        step_ms, step_launches = step_ms + m, step_launches + n
        m, n = qed.timing_read_multistep(reset=True)
        multi_ms, multi_passes = multi_ms + m, multi_passes + n
    barrier()
    clk = clocks.stop()
    qed.timing_enable(False)
    launches = qed.launch_count() - launches0
    job_ms = [a.elapsed_time(b) for a, b in ev]
    lep, ph, created, lep_multi, ph_multi, tau_ph = qed.work_read_split(job.e, reset=True)
    if args.step_log and rank == 0:
        write_step_log(args.step_log, job.step_log)
        job.step_log = None
    # jobs' own kernels only: reset copies (init_tau, counters) are outside the events
    total_ms, units_all = aggregate_ranks(float(sum(job_ms)), float(lep + ph), world, "cuda")
    value = units_all / (total_ms * 1e-3)

    b = BYTES[args.precision]
    # the per-step kernel's own work: multi-step passes are timed with the job, not with it
    alg_bytes = algorithmic_bytes(b, lep - lep_multi, ph - ph_multi, tau_ph, created)
    achieved_gbs = alg_bytes / (step_ms * 1e-3) / 1e9 if step_ms > 0 else None
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
        peak = float(peaks["hbm_gbs"])
        peak_src = "measured"
    except (OSError, KeyError, ValueError):
        peak, peak_src = 6800.0, "fallback"
    traffic = read_traffic(args.precision, step_launches, lep - lep_multi + ph - ph_multi, created)

    # ---------------- e2e through the C ABI with pinned host buffers
    e2e = None if args.no_e2e else e2e_run(args, qed, tables, w, torch, job, rank, world)

    # ---------------- FP64 path (one scenario at a time) vs mixed on the same job
    fp64_cmp = None if args.no_fp64 else fp64_compare(args, qed, tables, W, torch, rank)
    del job
    torch.cuda.empty_cache()

    if rank != 0:
        return
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / max(1, args.steps), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64" if args.precision == "mixed" else "f64", "data": "synthetic",
        "config": {"workload": workload_name(args.n, args.time_steps), "n_electrons": args.n,
                   "time_steps": args.time_steps, "precision": args.precision,
                   "particle_steps_per_job": units_all / max(1, args.steps) / world,
                   "particles_created_per_job": created / max(1, args.steps),
                   "l2": "256 MiB buffer written between jobs (outside the job events); state exceeds L2 after the collision",
                   "parallelism": "replicas" if world > 1 else "single"},
        "roofline": {"bound": "hbm", "kernel": "step_kernel", "achieved": achieved_gbs, "peak": peak, "unit": "GB/s",
                     "frac": (achieved_gbs / peak) if achieved_gbs else None, "traffic": traffic,
                     "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)" if peak_src == "measured" else
                     "fallback 6.8 TB/s", "step_kernel_ms": step_ms, "step_kernel_launches": step_launches,
                     "algorithmic_bytes_per_launch": alg_bytes / max(1, step_launches),
                     "step_kernel_share_of_job_time": step_ms / total_ms if total_ms else None},
        "clocks": clk,
        "e2e": e2e,
        "gpu_launches": launches,
        "multi_step": {"chunk": args.multistep, "share_of_particle_steps": (lep_multi + ph_multi) / max(1, lep + ph),
                       "passes": multi_passes, "ms": multi_ms, "share_of_job_time": multi_ms / total_ms if total_ms else None,
                       "particle_steps_per_s": (lep_multi + ph_multi) / (multi_ms * 1e-3) if multi_ms else None,
                       "note": "event-free stretches of up to `chunk` steps taken in one pass over the particles "
                               "(probe + commit); the roofline above is the per-step kernel's"},
        "fp64_path": fp64_cmp,
    }
    if not args.no_cpu_baseline and world == 1:  # the host baseline is quoted at one GPU only
        out["cpu_baseline"], oracle_sample = cpu_baseline(args, W)
        out["mixed_vs_oracle_energy"] = sample_vs_oracle(args, qed, tables, W, torch, oracle_sample)
    # the batched scan and the serving loop, at one GPU (they use the whole device)
    if world == 1 and not args.no_batched:
        out["batched"] = batched_run(args, qed, tables, W, torch)
    if world == 1 and not args.no_serving:
        out["serving"] = serving_run(args, qed, tables, W, torch)
    print(json.dumps(out))


def aggregate_ranks(ms, units, world, device):
    """Whole-job figures over the ranks: the slowest rank's time and the sum of the units (weak
    scaling; the ranks run independent replicas, so this is the only collective)."""
    if world <= 1:
        return ms, units
    import torch
    import torch.distributed as dist

    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    c = torch.tensor([units], dtype=torch.float64, device=device)
    dist.all_reduce(c)
    return float(t.item()), float(c.item())


def e2e_run(args, qed, tables, w, torch, job, rank, world):
    """Same metric through the public API with host buffers: pinned H2D of the initial state,
    the run, D2H of the ledger (the job's result); host wall clock with synchronisation."""
    dt = torch.float32 if job.prec == qed.MIXED else torch.float64
    xr = w.x.copy()
    xr[:, 0] -= w.window_x0
    host = [torch.tensor(np.ascontiguousarray(a[:, c]), dtype=dt).pin_memory() for a in (xr, w.u) for c in range(3)]
    ids = torch.arange(w.n, dtype=torch.int32).pin_memory()
    tau = torch.zeros(w.n, dtype=torch.float64).pin_memory()
    h2d = sum(t.numel() * t.element_size() for t in host) + ids.numel() * 4 + tau.numel() * 8
    soa = qed.Soa(*[t.data_ptr() for t in host], tau.data_ptr(), ids.data_ptr())
    reps = max(1, args.steps)
    flush = torch.zeros(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    qed.work_read(job.e, reset=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(reps):
        flush_l2(torch, flush)  # as in the device-timed loop: every job starts with a cold L2
        job.e.upload_soa(soa, w.n, w.n)
        job.e.init_tau(w.seed, rank)
        job.p.upload_soa(job.empty, 0, 0)
        job.g.upload_soa(job.empty, 0, 0)
        job.run()
        led = qed.read_ledger([job.e, job.p, job.g])  # D2H of the result, synchronises
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    lep, ph, _ = qed.work_read(job.e, reset=True)
    del led
    return {"value": (lep + ph) * world / el, "unit": UNIT, "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": 13 * 8 + 6 * 8, "reps": reps}


def fp64_compare(args, qed, tables, W, torch, rank):
    """The same job (the workload at its full size) once in mixed precision and once on the
    plain FP64 path: the FP64 path's rate and the two paths' energies."""
    n = args.n
    w = W.head_on(n=n, n_steps=args.time_steps, seed=2)
    out = {"workload": workload_name(n, args.time_steps)}
    for prec in ("mixed", "fp64"):
        job = Job(qed, tables, w, prec, rank, torch, args.multistep)
        job.reset()
        qed.work_read(job.e, reset=True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        job.run()
        e1.record()
        torch.cuda.synchronize()
        lep, ph, _ = qed.work_read(job.e, reset=True)
        out[prec] = (lep + ph) / (e0.elapsed_time(e1) * 1e-3)
        led = qed.read_ledger([job.e, job.p, job.g])
        out[prec + "_energy_per_electron"] = [v / n for v in led["energy"]]
        del job
        torch.cuda.empty_cache()
    out["speedup_mixed_over_fp64"] = out["mixed"] / out["fp64"]
    out["mixed_vs_fp64_rel_err_energy"] = [abs(a / b - 1) if b else 0.0 for a, b in
                                           zip(out["mixed_energy_per_electron"], out["fp64_energy_per_electron"])]
    return out


def energy_errors(pairs):
    """Mixed-precision results against FP64 ones, from (value, reference) pairs of per-species
    energy triples: the relative error of the summed energies of all the results per species
    ("ensemble"), and the largest relative error of one result ("max_per_result"; the absolute
    value where the reference is 0).  The two paths take the same random numbers, but a rounding
    difference near a threshold can turn an event on or off, after which a particle's history
    differs: results with few particles differ by that much, the ensemble agrees statistically.
    None without pairs."""
    if not pairs:
        return None
    rel = lambda a, b: abs(a / b - 1) if b else abs(a)
    errs = [[rel(a, b) for a, b in zip(x, y)] for x, y in pairs]
    tot = [rel(sum(x[c] for x, _ in pairs), sum(y[c] for _, y in pairs)) for c in range(3)]
    return {"ensemble": tot, "max_per_result": [max(e[c] for e in errs) for c in range(3)], "results": len(pairs)}


def write_step_log(path, log):
    """Per time step of the first timed job: e+- pushes, photon pushes, particles created
    (differences of the cumulative work counters) and the device time of the step's call."""
    with open(path, "w") as f:
        f.write("step,lepton_pushes,photon_pushes,created,step_us\n")
        prev = (0, 0, 0)
        for k, cur in enumerate(log):
            f.write(f"{k},{cur[0] - prev[0]},{cur[1] - prev[1]},{cur[2] - prev[2]},{cur[3] * 1e3:.2f}\n")
            prev = cur[:3]


TRAFFIC_FILE = os.path.join(ROOT, "profiles", "step_kernel_traffic_head_on.md")


def read_traffic(precision, launches, units, created):
    """DRAM bytes per launch, from the DRAM bytes per particle-step that the committed ncu summary
    records, if the summary was taken on this kernel source and precision."""
    rec = None
    try:
        with open(TRAFFIC_FILE) as f:
            for line in f:
                if line.startswith("traffic-record:"):
                    rec = json.loads(line.split(":", 1)[1])
    except (OSError, ValueError):
        return None
    if rec is None:
        return None
    if rec.get("source_digest") != kernel_digest() or rec.get("precision") != precision:
        return None
    per_unit = rec.get("dram_bytes_per_particle_step")
    if per_unit is None or launches == 0:
        return None
    return per_unit * units / launches


def kernel_digest():
    """Digest of the step kernel's sources and build defines (a traffic record applies only to it)."""
    h = hashlib.sha256()
    for f in ("qed_kernels.cu", "qed_device.cuh", "qed_internal.h"):
        with open(os.path.join(ROOT, "paper_1311_5551_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    defines = " ".join(f for f in os.environ.get("QED_NVCC_DEFINES", "").split() if f.startswith("-D"))
    if defines:
        h.update(defines.encode())
    return h.hexdigest()[:16]


# ----------------------------------------------------------------------------- CPU oracle
def oracle_sample_run(W, n_sample, time_steps, chunk=0, n_total=1_000_000, energies=False):
    """The FP64 oracle on electrons [chunk*n_sample, (chunk+1)*n_sample) of the same workload (all
    species), as a job of their own (ids from 0, scenario 0)."""
    import oracle as o

    w = W.head_on(n=max(n_total, (chunk + 1) * n_sample), n_steps=time_steps, seed=2)
    x, u = w.x[chunk * n_sample:(chunk + 1) * n_sample], w.u[chunk * n_sample:(chunk + 1) * n_sample]
    path = os.path.join(ROOT, "oracle", "_build", "tables_default.npz")
    tables = o.Tables.load(path) if os.path.exists(path) else o.Tables()
    e = o.Species(4 * n_sample + 64)
    e.set(x, u)
    e.init_tau(o.ELECTRON, w.seed)
    p, g = o.Species(4 * n_sample + 64), o.Species(120 * n_sample + 64)
    sp = o.StepParams(dt=w.dt, seed=w.seed, field=o.Field(**w.field.as_dict()))
    units = 0
    t0 = time.perf_counter()
    for k in range(time_steps):
        units += e.n + p.n + g.n
        o.step(tables, sp, k, e, p, g)
    el = time.perf_counter() - t0
    if not energies:
        return units, el
    alive = np.isfinite(g.get("tau"))
    return units, el, [e.energy().tolist(), p.energy().tolist(), g.energy(photon=True)[alive].tolist()]


def _oracle_chunk(job):
    W_mod, n_sample, time_steps, chunk = job
    from paper_1311_5551_gb300 import workloads as W

    return oracle_sample_run(W, n_sample, time_steps, chunk=chunk, energies=chunk == 0)


def cpu_baseline(args, W):
    """The FP64 oracle on the host cores: one sample of cpu_sample electrons per core (the first
    of them is the sample the GPU's error figures are taken against).  Returns the baseline and
    that first sample's final particle energies."""
    import multiprocessing as mp

    import oracle as o

    o.build()
    path = os.path.join(ROOT, "oracle", "_build", "tables_default.npz")
    if not os.path.exists(path):
        o.Tables().save(path)
    cores = max(1, min(os.cpu_count() or 1, args.cpu_cores))
    t0 = time.perf_counter()
    with mp.get_context("spawn").Pool(cores) as pool:
        res = pool.map(_oracle_chunk, [(None, args.cpu_sample, args.time_steps, c) for c in range(cores)], chunksize=1)
    wall = time.perf_counter() - t0
    units = sum(r[0] for r in res)
    single = res[0][0] / res[0][1]
    return ({"value": units / wall, "unit": UNIT, "cores": cores, "kind": "oracle",
             "single_core_value": single,
             "sample": f"{cores} samples of {args.cpu_sample} electrons of the workload (electrons "
                       f"[c*{args.cpu_sample}, (c+1)*{args.cpu_sample}) for core c), all {args.time_steps} steps, "
                       f"all species, one process per core: {units} particle-steps in {wall:.1f} s "
                       f"(FP64 C oracle)"}, res[0][2])


def sample_vs_oracle(args, qed, tables, W, torch, oracle_energies):
    """The cpu_baseline's first sample (the workload's first cpu_sample electrons as a job of their
    own) on the GPU in mixed precision and on the FP64 path, against the oracle: per species the
    relative error of the total energy and the statistical standard error of the oracle's total."""
    w = W.head_on(n=args.n, n_steps=args.time_steps, seed=2)
    m = args.cpu_sample
    w.x, w.u = w.x[:m].copy(), w.u[:m].copy()
    out = {"sample": f"first {m} electrons of the workload, all {args.time_steps} steps"}
    ores = [(0, 0, 0.0, oracle_energies)]
    for prec in ("mixed", "fp64"):
        job = Job(qed, tables, w, prec, 0, torch, args.multistep)
        job.reset()
        job.run()
        led = qed.read_ledger([job.e, job.p, job.g])
        out[prec] = energy_vs_oracle([led["energy"]], ores)
        del job
    return out


# ----------------------------------------------------------------------------- batched scan
SCAN_N = 256


def scan_workloads(W, scale, time_steps, first=0):
    """The scan's scenarios (the first `first` of them when it is > 0: a smaller case of the same
    batch for profiling), each under its own scenario index."""
    only = list(range(first)) if first else None
    return W.scan(n_scenarios=SCAN_N, n_steps=time_steps, scale=scale, only=only)


def measured_hbm_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback 6.8 TB/s"


def _oracle_scenario(job):
    """One whole scenario of the scan, or one request of the serving stream, on the FP64 oracle
    (a worker of cpu_baseline_scan's process pool): returns its key, its particle-steps, the
    seconds it took and the final energies of its particles."""
    kind, k, a, b, c = job
    import oracle as o
    from paper_1311_5551_gb300 import workloads as W

    if kind == "scan":  # (scale, time steps)
        w = W.scan(n_scenarios=SCAN_N, n_steps=b, scale=a, only=[k])[0]
    else:  # a request: (rate, arrival window, scale)
        w = W.request_specs(rate_hz=a, duration_s=b, scale=c)[k][1].workload()
    tables = o.Tables.load(os.path.join(ROOT, "oracle", "_build", "tables_default.npz"))
    n = w.n
    e, p, g = o.Species(8 * n + 64), o.Species(8 * n + 64), o.Species(1200 * n + 4096)
    e.set(w.x, w.u)
    e.init_tau(o.ELECTRON, w.seed, k)
    sp = o.StepParams(dt=w.dt, seed=w.seed, scenario=k, field=o.Field(**w.field.as_dict()))
    units = 0
    t0 = time.perf_counter()
    for step in range(w.n_steps):
        units += e.n + p.n + g.n
        o.step(tables, sp, step, e, p, g)
    el = time.perf_counter() - t0
    energies = [e.energy().tolist(), p.energy().tolist()]
    alive = np.isfinite(g.get("tau"))  # converted photons stay as holes (tau = +inf)
    energies.append(g.energy(photon=True)[alive].tolist())
    return k, units, el, energies


def cpu_baseline_scan(jobs, cores):
    """The FP64 oracle on whole scenarios of the scan (or requests of the serving stream), one
    per host core at a time (the baseline of the batched line, and the reference that its error
    figures are taken against).  ``jobs``: _oracle_scenario's arguments."""
    import multiprocessing as mp

    import oracle as o

    o.build()
    path = os.path.join(ROOT, "oracle", "_build", "tables_default.npz")
    if not os.path.exists(path):
        o.Tables().save(path)
    t0 = time.perf_counter()
    with mp.get_context("spawn").Pool(cores) as pool:
        res = pool.map(_oracle_scenario, jobs, chunksize=1)
    wall = time.perf_counter() - t0
    return res, wall


def energy_vs_oracle(gpu_energy, oracle_res):
    """Relative error of each species' total energy (summed over the compared scenarios), GPU
    against the oracle, beside the statistical standard error of the oracle's total (the spread
    of its particles' energies times sqrt(count)); and the same per scenario, largest value."""
    out = {"species": ["electron", "positron", "photon"], "scenarios": len(oracle_res),
           "sigma": "electrons: sqrt(N) x the spread of their energies; positrons and photons, whose number "
                    "is itself random: sqrt(sum of their squared energies)"}
    rel, sig, per = [], [], []
    for c in range(3):
        ref = sum(float(np.sum(r[3][c])) for r in oracle_res)
        got = sum(gpu_energy[r[0]][c] for r in oracle_res)
        allv = np.concatenate([np.asarray(r[3][c], dtype=np.float64) for r in oracle_res]) if oracle_res else np.zeros(0)
        if c == 0:
            sd = float(np.std(allv) * math.sqrt(len(allv))) if len(allv) > 1 else 0.0
        else:
            sd = float(math.sqrt(np.sum(allv * allv)))
        rel.append(abs(got / ref - 1.0) if ref else abs(got))
        sig.append(sd / ref if ref else 0.0)
        per.append(max((abs(gpu_energy[r[0]][c] / float(np.sum(r[3][c])) - 1.0) if float(np.sum(r[3][c])) else 0.0)
                       for r in oracle_res) if oracle_res else None)
    out["rel_err"] = rel
    out["rel_sigma"] = sig
    out["err_over_sigma"] = [r / s if s else None for r, s in zip(rel, sig)]
    out["max_rel_err_per_scenario"] = per
    return out


def batched_run(args, qed, tables, W, torch):
    """Config of the scan: 256 head-on scenarios (log-uniform particle counts in [1e3, 1e6], a0,
    gamma0 and pulse FWHM drawn per scenario) in one batch, mixed precision, autotuned launch
    configuration, graph-replayed batch steps.  Capacities from a pilot run; the whole scan at the
    stated size when it fits in device memory, else the largest scale that does (recorded)."""
    from paper_1311_5551_gb300.serving import footprint, make_species, pilot_capacities

    prec = qed.MIXED
    stream = torch.cuda.current_stream()
    torch.cuda.empty_cache()
    scale, reason = args.scan_scale, "stated size"
    ws = scan_workloads(W, scale, args.time_steps, args.scan_first)
    caps, pstat = pilot_capacities(qed, tables, ws, prec, sample=args.pilot_sample)
    need = sum(footprint(w, 4, c) for w, c in zip(ws, caps)) + 2 * sum(w.n for w in ws) * 4 * 8
    free, total = torch.cuda.mem_get_info()
    budget = free - (6 << 30)
    if need > budget:
        scale = math.floor(scale * budget / need * 100) / 100
        reason = f"stores of the stated size need {need / 1e9:.0f} GB, {budget / 1e9:.0f} GB free: scaled to fit"
        ws = scan_workloads(W, scale, args.time_steps, args.scan_first)
        caps, pstat = pilot_capacities(qed, tables, ws, prec, sample=args.pilot_sample)
        need = sum(footprint(w, 4, c) for w, c in zip(ws, caps))
    sps = [make_species(qed, w, prec, c) for w, c in zip(ws, caps)]
    batch = qed.Batch(tables, prec, len(ws))
    # initial states in pinned host memory (the end-to-end figure copies them in)
    host = []
    for w in ws:
        xr = w.x.copy()
        xr[:, 0] -= w.window_x0
        cols = [torch.tensor(np.ascontiguousarray(a[:, c]), dtype=torch.float32).pin_memory() for a in (xr, w.u)
                for c in range(3)]
        host.append(cols)
    h2d = sum(t.numel() * 4 for cols in host for t in cols)
    empty = qed.Soa(*([None] * 8))

    def load():
        for k, (sp, w) in enumerate(zip(sps, ws)):
            sp[0].upload_soa(qed.Soa(*[t.data_ptr() for t in host[k]], None, None), w.n, w.n)
            sp[0].init_tau(w.seed, k)
            sp[1].upload_soa(empty, 0, 0)
            sp[2].upload_soa(empty, 0, 0)
            p = qed.StepParams(dt=w.dt, seed=w.seed, scenario=k, field=qed.Field(**w.field.as_dict()),
                               window_x0=w.window_x0, window_v=w.window_v)
            batch.attach(k, sp, p, 0, w.n_steps)
            qed.work_read(sp[0], reset=True)

    load()
    tb, gs = batch.tune(trial_steps=4)
    flush = torch.zeros(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    # ---- timed: the end-to-end region (H2D of the initial states, the run, D2H of every
    # scenario's ledger) around the device-timed run
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    launches0 = qed.launch_count()
    t0 = time.perf_counter()
    load()
    flush_l2(torch, flush)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    batch.run(args.time_steps)
    e1.record(stream)
    ledgers = [qed.read_ledger(sp) for sp in sps]
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    clk = clocks.stop()
    launches = qed.launch_count() - launches0
    ms = e0.elapsed_time(e1)
    qed.check([s for sp in sps for s in sp])
    assert np.all(batch.remaining() == 0)
    work = np.array([qed.work_read_split(sp[0]) for sp in sps], dtype=np.float64)
    units = float(work[:, 0].sum() + work[:, 1].sum())
    b = BYTES["mixed"]
    alg = float(algorithmic_bytes(b, work[:, 0].sum(), work[:, 1].sum(), work[:, 5].sum(), work[:, 2].sum()))
    peak, peak_src = measured_hbm_peak()
    gpu_energy = [led["energy"] for led in ledgers]
    held = [[s.count() for s in sp] for sp in sps]
    for sp in sps:
        for s in sp:
            s.close()
    batch.close()
    del sps, flush
    torch.cuda.empty_cache()

    # ---- one scenario at a time on the plain FP64 path: scenarios at the 10/30/50/70/90 %
    # quantiles of the size, a rate; and the mixed-precision batch against it
    order = sorted(range(len(ws)), key=lambda k: ws[k].n)
    picks = sorted({order[int(q * (len(ws) - 1))] for q in (0.1, 0.3, 0.5, 0.7, 0.9)})
    if args.no_fp64:
        picks = []
    fp_units, fp_ms, pairs = 0.0, 0.0, []
    for k in picks:
        w = ws[k]
        s64 = make_species(qed, w, qed.FP64, caps[k])
        xr = w.x.copy()
        xr[:, 0] -= w.window_x0
        s64[0].upload(xr, w.u)
        s64[0].init_tau(w.seed, k)
        p = qed.StepParams(dt=w.dt, seed=w.seed, scenario=k, field=qed.Field(**w.field.as_dict()),
                           window_x0=w.window_x0, window_v=w.window_v)
        a, bb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        qed.run(tables, s64, p, 0, w.n_steps)
        bb.record(stream)
        torch.cuda.synchronize()
        fp_ms += a.elapsed_time(bb)
        fp_units += sum(qed.work_read(s64[0])[:2])
        pairs.append((gpu_energy[k], qed.read_ledger(s64)["energy"]))
        for q in s64:
            q.close()
    fp64_rate = fp_units / (fp_ms * 1e-3) if fp_ms else None

    # ---- the oracle on the smallest whole scenarios (host cores): CPU baseline and reference
    cores = max(1, min(os.cpu_count() or 1, args.cpu_cores))
    est = [(k, w.n * (w.n_steps + caps[k][2] / max(1, w.n) * w.n_steps / 2)) for k, w in enumerate(ws)]
    est.sort(key=lambda t: t[1])
    picks_o, budget_ps = [], args.oracle_budget_s * 3e7 * cores
    for k, ps in est:
        if ps > budget_ps / cores or len(picks_o) >= 4 * cores:
            break
        if args.no_cpu_baseline:
            break
        picks_o.append(k)
        budget_ps -= ps
        if budget_ps <= 0:
            break
    ores, owall = (cpu_baseline_scan([("scan", k, scale, args.time_steps, None) for k in picks_o], cores)
                   if picks_o else ([], 0.0))
    o_units = sum(r[1] for r in ores)

    value = units / (ms * 1e-3)
    out = {
        "workload": f"scan_{len(ws)}_head_on_LP_lambda=1um_a0=U[10,500]_gamma0=U[200,4000]_fwhm=U[15,60]fs_"
                    f"N=logU[1e3,1e6]x{scale:g}_{args.time_steps}_steps",
        "metric": METRIC, "value": value, "unit": UNIT, "scenarios": len(ws), "scale": scale, "scale_reason": reason,
        "electrons_total": int(sum(w.n for w in ws)), "time_steps": args.time_steps, "precision": "mixed",
        "ms": ms, "particle_steps": units, "particles_created": float(work[:, 2].sum()),
        "particles_held_at_end": [int(sum(h[c] for h in held)) for c in range(3)],
        "l2": "256 MiB buffer written before the run; the state exceeds L2 from the first steps",
        "autotuned": {"target_blocks": tb, "graph_steps": gs},
        "capacity_plan": {"method": "pilot run of every scenario's first electrons on the GPU", **pstat,
                          "stores_GB": need / 1e9},
        "gpu_launches": launches,
        "roofline": {"bound": "hbm", "kernel": "whole batch run (all kernels)", "unit": "GB/s",
                     "achieved": alg / (ms * 1e-3) / 1e9, "peak": peak, "frac": alg / (ms * 1e-3) / 1e9 / peak,
                     "peak_source": peak_src, "algorithmic_bytes": alg, "traffic": None},
        "clocks": clk,
        "e2e": {"value": units / wall, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": len(ws) * 19 * 8,
                "note": "H2D of every scenario's initial state from pinned memory, the run and the D2H of every ledger"},
        "fp64_one_at_a_time": {"value": fp64_rate, "unit": UNIT, "scenarios": picks,
                               "note": "the scenarios at the 10/30/50/70/90 % size quantiles, one qed_run each"},
        "speedup_vs_fp64_one_at_a_time": (value / fp64_rate) if fp64_rate else None,
        "mixed_vs_fp64_rel_err_energy": energy_errors(pairs),
        "mixed_vs_oracle_energy": energy_vs_oracle(gpu_energy, ores),
        "cpu_baseline": {"value": o_units / owall if owall else None, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{len(ores)} whole scenarios of the scan (the smallest), one per core at a time, "
                                   f"{o_units:.3e} particle-steps in {owall:.1f} s"},
    }
    return out


def scan_arm(args):
    """The batched scan on its own line."""
    import torch

    from paper_1311_5551_gb300 import build as qbuild
    from paper_1311_5551_gb300 import qed, workloads as W

    torch.cuda.set_device(0)
    qbuild.build()
    tables = qed.Tables()
    print(json.dumps(batched_run(args, qed, tables, W, torch)))


# ----------------------------------------------------------------------------- serving
def serving_run(args, qed, tables, W, torch):
    """Config of the serving loop: Poisson arrivals at args.rate of head-on requests (particle
    counts log-uniform in [1e3, 2e6], a0, gamma0 and steps drawn per request), continuous
    batching under a device-memory budget; p50/p99 latency beside served throughput, a point at
    a sustainable rate, and the same stream served one request at a time on the FP64 path."""
    from paper_1311_5551_gb300.serving import make_species, serve

    torch.cuda.empty_cache()
    free, _ = torch.cuda.mem_get_info()
    budget = int(free * 0.85)
    out = {"workload": f"serve_head_on_poisson_{args.rate:g}_per_s_N=logU[1e3,2e6]x{args.serve_scale:g}_"
                       f"steps=U[2000,8000]", "unit": UNIT, "scale": args.serve_scale, "budget_GB": budget / 1e9}

    def one(rate, precision, slots, window, wall, tag):
        reqs = W.request_specs(rate_hz=rate, duration_s=window, scale=args.serve_scale)
        fin, st = serve(qed, tables, reqs, precision, slots=slots, chunk=args.chunk, max_wall=wall,
                        admit_until=window, budget_bytes=budget)
        st["rate_hz"] = rate
        st["arrival_window_s"] = window
        st["offered_requests"] = len(reqs)
        st["offered_electron_steps_per_s"] = sum(r.n * r.n_steps for _, r in reqs) / window
        out[tag] = st
        torch.cuda.empty_cache()
        return fin, st, reqs

    fin, st, reqs = one(args.rate, qed.MIXED, args.slots, args.serve_window, args.max_wall, "batched_mixed")
    # particle-steps of a request: electron-steps times the mean ratio of all particle-steps to
    # electron-steps over the finished requests; the sustainable rate offers 0.7 of what was served
    if fin:
        ratio = np.sum([r.result["particle_steps"] for r in fin]) / np.sum([r.n * r.steps for r in fin])
        per_req = ratio * np.mean([r.n * r.steps for r in fin])
        sus = 0.7 * st["served_particle_steps_per_s"] / per_req if per_req > 0 else None
        out["offered_load_ratio"] = st["offered_electron_steps_per_s"] * ratio / max(1.0, st["served_particle_steps_per_s"])
        if sus:
            one(sus, qed.MIXED, args.slots, args.sustain_window, args.max_wall, "batched_mixed_sustainable")
    fin64, _, _ = one(args.rate, qed.FP64, 1, args.serve_window, args.fp64_wall, "one_at_a_time_fp64")
    b, f = out["batched_mixed"], out["one_at_a_time_fp64"]
    out["speedup_vs_fp64_one_at_a_time"] = (b["processed_particle_steps_per_s"] / f["processed_particle_steps_per_s"]
                                            if f["processed_particle_steps_per_s"] else None)
    out["speedup_note"] = ("particle-steps processed per second (finished and unfinished requests) by the batched "
                           "loop and by one-request-at-a-time FP64 launches on the same arrival stream")

    # every finished request's energies against the same request alone on the FP64 path (the
    # smallest ones, up to 5) and against the oracle (the smallest ones the host cores finish
    # within the budget)
    mixed = {r.rid: r.result["ledger"]["energy"] for r in fin}
    pairs = [(mixed[r.rid], r.result["ledger"]["energy"]) for r in fin64 if r.rid in mixed]
    small = sorted(fin, key=lambda r: r.result["particle_steps"])
    stream = torch.cuda.current_stream()
    for r in small[:5]:
        w = reqs[r.rid][1].workload()
        s64 = make_species(qed, w, qed.FP64)
        xr = w.x.copy()
        xr[:, 0] -= w.window_x0
        s64[0].upload(xr, w.u)
        s64[0].init_tau(w.seed, r.rid)
        p = qed.StepParams(dt=w.dt, seed=w.seed, scenario=r.rid, field=qed.Field(**w.field.as_dict()),
                           window_x0=w.window_x0, window_v=w.window_v)
        qed.run(tables, s64, p, 0, w.n_steps, stream=stream)
        pairs.append((mixed[r.rid], qed.read_ledger(s64)["energy"]))
        for q in s64:
            q.close()
    out["mixed_vs_fp64_rel_err_energy"] = energy_errors(pairs)
    cores = max(1, min(os.cpu_count() or 1, args.cpu_cores))
    picks_o, left = [], args.oracle_budget_s * 3e7 * cores
    for r in small:
        ps = r.result["particle_steps"]
        if ps > args.oracle_budget_s * 3e7 or ps > left or len(picks_o) >= 4 * cores or args.no_cpu_baseline:
            break
        picks_o.append(r.rid)
        left -= ps
    jobs = [("serve", k, args.rate, args.serve_window, args.serve_scale) for k in picks_o]
    ores, _ = cpu_baseline_scan(jobs, cores) if jobs else ([], 0.0)
    out["mixed_vs_oracle_energy"] = energy_vs_oracle(mixed, ores)
    return out


def cascade_arm(args):
    """Rotating electric field (the node of a circularly polarised standing wave), |E| = 1e-3 E_s,
    lambda = 0.8 um, dt = lambda/(200 c), 1e4 electrons at rest; every photon and pair is kept and
    the run goes on until the live particles reach --cascade-live (or --cascade-max-steps)."""
    import torch

    from paper_1311_5551_gb300 import build as qbuild
    from paper_1311_5551_gb300 import qed, workloads as W

    torch.cuda.set_device(0)
    qbuild.build()
    tables = qed.Tables()
    prec = qed.MIXED if args.precision == "mixed" else qed.FP64
    w = W.rotating_e(n=args.cascade_n, n_steps=args.cascade_max_steps, seed=3)
    cap = int(args.cascade_live * 1.1) + 4096
    lep_cap = cap // 8  # pairs are rare at this field strength: the photons hold most of the particles
    # append regions: the children of one step, at most one per parent and never more than the store
    e = qed.Species(qed.ELECTRON, prec, lep_cap, lep_cap)
    p = qed.Species(qed.POSITRON, prec, lep_cap, lep_cap)
    g = qed.Species(qed.PHOTON, prec, cap, 2 * lep_cap)
    e.upload(w.x, w.u)
    e.init_tau(w.seed)
    params = qed.StepParams(dt=w.dt, seed=w.seed, field=qed.Field(**w.field.as_dict()))
    sp = [e, p, g]
    qed.work_read(e, reset=True)
    qed.timing_read(reset=True)
    qed.timing_enable(True)
    launches0 = qed.launch_count()
    flush_l2(torch, torch.zeros(64 * 1024 * 1024, dtype=torch.float32, device="cuda"))
    clocks = ClockSampler(0)
    clocks.start()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    step, live, compactions = 0, w.n, 0
    step_ms, step_launches = 0.0, 0
    e0.record(stream)
    merges, merged_groups, merge_ms = 0, 0, 0.0
    while step < args.cascade_max_steps and live < args.cascade_live:
        k = min(args.chunk_steps, args.cascade_max_steps - step)
        qed.run(tables, sp, params, step, k)
        step += k
        counts = [s.count() for s in sp]  # synchronises
        m, nl = qed.timing_read(reset=True)  # the chunk's kernel timers (their events are reused)
        step_ms, step_launches = step_ms + m, step_launches + nl
        led = qed.read_ledger(sp)
        live = int(sum(led["n"]))
        if counts[2] - led["n"][2] > 0.1 * counts[2]:  # converted photons leave holes
            g.compact()
            compactions += 1
        if args.merge_above and led["n"][2] > args.merge_above:
            m0, m1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            m0.record(stream)
            span = step * w.dt + 3e6  # the merging grid covers every photon emitted so far (they fly at c)
            merged_groups += g.merge(origin=(-span,) * 3, cell=(span / 4,) * 3, n_cells=(8, 8, 8), n_face=6, n_sub=2,
                                     min_group=4)
            m1.record(stream)
            torch.cuda.synchronize()
            merge_ms += m0.elapsed_time(m1)
            merges += 1
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    qed.timing_enable(False)
    ms = e0.elapsed_time(e1)
    lep, ph, created, _, _, tau_ph = qed.work_read_split(e)
    qed.check(sp)
    led = qed.read_ledger(sp)
    b = BYTES[args.precision]
    alg = algorithmic_bytes(b, lep, ph, tau_ph, created)
    peak, src = measured_hbm_peak()
    achieved = alg / (step_ms * 1e-3) / 1e9 if step_ms else None
    out = {"workload": "cascade", "metric": METRIC, "value": (lep + ph) / (ms * 1e-3), "unit": UNIT, "n_gpus": 1,
           "higher_is_better": True, "dtype": "f32+f64" if args.precision == "mixed" else "f64", "data": "synthetic",
           "config": {"workload": f"rotating_E_1e-3Es_lambda=0.8um_{args.cascade_n:.0e}_electrons_to_"
                                  f"{args.cascade_live:.0e}_live", "time_steps": step, "precision": args.precision,
                      "l2": "state exceeds L2 after the first steps (photons accumulate)"},
           "ms": ms, "particle_steps": lep + ph, "final_counts": led["n"], "created": created,
           "compactions": compactions,
           "merging": {"above_photons": args.merge_above, "merges": merges, "groups": merged_groups,
                       "ms": merge_ms, "photon_totals": list(g.totals()[:2]) if args.merge_above else None},
           "roofline": {"bound": "hbm", "kernel": "step_kernel", "achieved": achieved, "peak": peak, "unit": "GB/s",
                        "frac": achieved / peak if achieved else None, "traffic": None, "peak_source": src,
                        "step_kernel_ms": step_ms, "step_kernel_launches": step_launches,
                        "step_kernel_share_of_run_time": step_ms / ms if ms else None},
           "clocks": clk, "gpu_launches": qed.launch_count() - launches0}
    print(json.dumps(out))


def serve_arm(args):
    """The serving loop on its own line."""
    import torch

    from paper_1311_5551_gb300 import build as qbuild
    from paper_1311_5551_gb300 import qed, workloads as W

    torch.cuda.set_device(0)
    qbuild.build()
    tables = qed.Tables()
    out = serving_run(args, qed, tables, W, torch)
    out["metric"] = METRIC
    print(json.dumps(out))


def reference_arm(args):
    """The FP64 oracle as it stands, timed on the host cores: every bench step runs one sample of
    --ref-sample electrons (with all their children, all steps) per core, in a process pool (spawn);
    a step takes as long as its slowest sample's oracle run (building the initial state is not
    timed).  Under torchrun rank 0 alone runs it."""
    rank, world, _ = env_rank()
    if rank != 0:
        return
    import multiprocessing as mp

    import oracle as o

    o.build()
    path = os.path.join(ROOT, "oracle", "_build", "tables_default.npz")
    if not os.path.exists(path):
        o.Tables().save(path)
    cores = max(1, min(os.cpu_count() or 1, args.cpu_cores))
    jobs = [(None, args.ref_sample, args.time_steps, c + 1) for c in range(cores)]
    tot_u, tot_t = 0, 0.0
    with mp.get_context("spawn").Pool(cores) as pool:
        for k in range(args.warmup + args.steps):
            res = pool.map(_oracle_chunk, jobs, chunksize=1)
            el = max(r[1] for r in res)  # the cores run side by side: the slowest sample's oracle time
            if k >= args.warmup:
                tot_u += sum(r[0] for r in res)
                tot_t += el
    v = tot_u / tot_t
    sample = (f"{cores} samples of {args.ref_sample} electrons of the workload (one per core, electrons "
              f"[c*{args.ref_sample}, (c+1)*{args.ref_sample}) for c = 1..{cores}), all {args.time_steps} steps, "
              f"all species, per bench step")
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": tot_t * 1e3 / max(1, args.steps), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": workload_name(args.n, args.time_steps), "sample": sample},
           "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["mixed", "fp64"], default="mixed")
    ap.add_argument("--n", type=int, default=1_000_000)
    ap.add_argument("--time-steps", type=int, default=4000)
    ap.add_argument("--cpu-sample", type=int, default=1000)
    ap.add_argument("--ref-sample", type=int, default=250)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="leave the batched scan out of the default line")
    ap.add_argument("--no-serving", action="store_true", help="leave the serving loop out of the default line")
    ap.add_argument("--cpu-cores", type=int, default=16, help="host cores for the oracle baselines")
    ap.add_argument("--scan-scale", type=float, default=1.0, help="particle counts of the scan x this")
    ap.add_argument("--scan-first", type=int, default=0,
                    help="the scan's first N scenarios only (a smaller case of the batch, for profiling)")
    ap.add_argument("--pilot-sample", type=int, default=1024, help="electrons per scenario in the capacity pilot")
    ap.add_argument("--oracle-budget-s", type=float, default=20.0,
                    help="seconds of oracle work per core for the batched line's oracle comparison")
    ap.add_argument("--serve-scale", type=float, default=1.0, help="particle counts of the requests x this")
    ap.add_argument("--serve-window", type=float, default=60.0, help="seconds of arrivals at --rate")
    ap.add_argument("--sustain-window", type=float, default=40.0, help="seconds of arrivals at the sustainable rate")
    ap.add_argument("--fp64-wall", type=float, default=30.0, help="wall seconds of one-at-a-time FP64 serving")
    ap.add_argument("--workload", choices=["head_on", "scan", "serve", "cascade"], default="head_on")
    ap.add_argument("--multistep", type=int, default=64,
                    help="take event-free stretches of up to this many steps in one pass (0: per-step only)")
    ap.add_argument("--batch-multistep", type=int, default=0,
                    help="multi-step stretch per batch step in the scan and serve workloads (0: off; their "
                         "high-a0 scenarios keep emitting to the end, so it does not pay there)")
    ap.add_argument("--step-log", default=None,
                    help="write per-step work counters of the first timed job to this CSV (profiling)")
    ap.add_argument("--cascade-n", type=int, default=10_000)
    ap.add_argument("--cascade-live", type=float, default=2e8)
    ap.add_argument("--cascade-max-steps", type=int, default=400_000)
    ap.add_argument("--chunk-steps", type=int, default=1000)
    ap.add_argument("--merge-above", type=float, default=0,
                    help="cascade: merge photons whenever more than this many are live (0: never)")
    ap.add_argument("--rate", type=float, default=200.0)
    ap.add_argument("--slots", type=int, default=256)
    ap.add_argument("--chunk", type=int, default=50)
    ap.add_argument("--max-wall", type=float, default=60.0,
                    help="serving: wall seconds of a run; requests unfinished by then give latency lower bounds")
    args = ap.parse_args()
    if args.impl == "reference":
        reference_arm(args)
    elif args.workload == "scan":
        scan_arm(args)
    elif args.workload == "serve":
        serve_arm(args)
    elif args.workload == "cascade":
        cascade_arm(args)
    else:
        our_arm(args)


if __name__ == "__main__":
    main()
