#!/usr/bin/env python
"""Layered-field benchmark.

The default line is the batching form: one bench step = 64 tessellation jobs
(icosphere or noisy torus, 10k-600k vertices each, 10.0 M in all; 32-2048
seeds; FP32 or BF16 field storage) seeded and advanced 1000 time-iterations
together by lf_step_batch.  The metric is nnz-updates/s: the
interest-skeleton entries advanced per second, summed over all jobs; the line
carries the same jobs stepped one at a time (vs_plain), the roofline of the
step kernel, the end-to-end figure through the C ABI from host buffers and
the FP64 oracle timed on the host cores (cpu_baseline).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload NAME]

Under torchrun every rank runs its own jobs on its own GPU (independent jobs,
no data-path collective: weak scaling); rank 0 prints one JSON line.
--impl reference times the FP64 CPU oracle on a bounded sample of the same
jobs on every host core.

Other workloads (--workload): grid512 (one 512 x 512 jittered grid, 1024
seeds, 2000 steps), torus1024 and torus3300 (noisy tori of 1 M and 10.9 M
vertices), ico3, grid512_shuffled / _reordered / _morton (vertex
numbering), grid512_general (dense coefficient matrices), serve (the Poisson
trace through lf_server: p50/p99 job latency), grid512_lloyd (Lloyd-like
rounds and the dual mesh) and dt_sweep (the time step study).
"""
import argparse
import contextlib
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "field nnz-updates/s and HBM GB/s (% of peak) vs plain; p50/p99 job latency"
UNIT = "nnz-updates/s"

def _general_coefs(n):
    """Dense coefficient matrices for n layers: the class values of the default
    parameters (base layer n - 1) plus a seeded perturbation of +-0.025 (stream 31)."""
    cell = np.arange(n) < n - 1
    both = np.outer(cell, cell)
    W = np.where(both, 0.2, 0.0)
    A = np.full((n, n), 0.04)
    E = np.zeros((n, n))
    E[cell, n - 1] = 0.5
    E[n - 1, cell] = -0.5
    out = []
    for t, M in enumerate((W, A, E)):
        np.fill_diagonal(M, 0.0)
        u = synth.uniform01(31, np.arange(t * n * n, (t + 1) * n * n, dtype=np.uint64)).reshape(n, n)
        out.append((M + 0.05 * (u - 0.5)).astype(np.float32))
    return out


def _reordered(m, method="rcm"):
    from paper_1804_09152_gb300.ordering import locality_order
    V, F, _ = locality_order(m.V, m.F, method)
    return synth.Mesh(V, F)


WORKLOADS = {
    "grid512": dict(desc="planar grid 512x512, alternating diagonals, jitter U(-0.2,0.2) (stream 2), "
                         "1024 seeds (stream 3), FP32 field, 2000 time steps",
                    mesh=lambda: synth.planar_grid(512, jitter=0.2, seed=2), k=1024, seed_stream=3,
                    steps=2000, dtype="f32"),
    "torus1024": dict(desc="noisy torus R=1 r=0.35 on a 1024x1024 grid, 4-octave value noise amp 0.02 "
                           "(stream 4), 8192 seeds (stream 5), FP32 field, 3000 time steps",
                      mesh=lambda: synth.noisy_torus(1024), k=8192, seed_stream=5, steps=3000, dtype="f32"),
    "torus3300": dict(desc="noisy torus R=1 r=0.35 on a 3300x3300 grid (10,890,000 vertices, 21.8 M triangles: "
                           "the size of the paper's largest model), value noise as torus1024, 10000 seeds "
                           "(stream 5), FP32 field, 2000 time steps",
                      mesh=lambda: synth.noisy_torus(3300), k=10000, seed_stream=5, steps=2000, dtype="f32"),
    "grid512_shuffled": dict(desc="the grid512 mesh with its vertices renumbered by a random permutation "
                                  "(stream 21), 1024 seeds (stream 3), FP32 field, 2000 time steps",
                             mesh=lambda: synth.shuffled(synth.planar_grid(512, jitter=0.2, seed=2)), k=1024,
                             seed_stream=3, steps=2000, dtype="f32"),
    "grid512_reordered": dict(desc="grid512_shuffled renumbered by reverse Cuthill-McKee (ordering.locality_order), "
                                   "1024 seeds (stream 3), FP32 field, 2000 time steps",
                              mesh=lambda: _reordered(synth.shuffled(synth.planar_grid(512, jitter=0.2, seed=2))),
                              k=1024, seed_stream=3, steps=2000, dtype="f32"),
    "grid512_morton": dict(desc="grid512_shuffled renumbered along a Morton curve of the positions, 1024 seeds "
                                "(stream 3), FP32 field, 2000 time steps",
                           mesh=lambda: _reordered(synth.shuffled(synth.planar_grid(512, jitter=0.2, seed=2)), "morton"),
                           k=1024, seed_stream=3, steps=2000, dtype="f32"),
    "grid512_general": dict(desc="grid512 with dense general coefficient matrices (the class values perturbed "
                                 "by +-0.025, stream 31; 1025 x 1025 each), 1024 seeds (stream 3), FP32 field, "
                                 "2000 time steps",
                            mesh=lambda: synth.planar_grid(512, jitter=0.2, seed=2), k=1024, seed_stream=3,
                            steps=2000, dtype="f32", coefs=_general_coefs),
    "ico3": dict(desc="icosphere level 3 (642 vertices), 16 seeds (stream 1), FP32 field, 300 time steps",
                 mesh=lambda: synth.icosphere(3), k=16, seed_stream=1, steps=300, dtype="f32"),
}

# Counters of the step kernel from ncu captures (DRAM bytes and warp
# instructions; steady state), valid only for the workload and the kernel
# source they were taken on.
# DRAM read + write bytes and warp instructions of the step kernel, from ncu
# captures of the committed profile commands; keyed by workload, then by the
# schedule every job ran under; void once the kernel source changes (the line
# then reports null traffic, with these figures beside it as an earlier
# source's)
NCU_COUNTERS = {"kernel_sha": "b0b64229b4bbf4bf",
                # launches 1001-1003 of the job (steps ~1000 of 2000)
                "grid512": {"ctas4": {"bytes_per_launch": 17872299, "warp_instructions_per_launch": 11770155},
                            "hot": {"bytes_per_launch": 17887403, "warp_instructions_per_launch": 13148319}},
                # one batch step (FP32 launch + BF16 launch, steps ~490-515 of 1000)
                "batch64": {"hot": {"bytes_per_step": 955717952, "warp_instructions_per_step": 495440220},
                            "lean": {"bytes_per_step": 955072192, "warp_instructions_per_step": 486605608}}}
SM_COUNT, SUBPARTITIONS = 152, 4          # GB300: 152 SMs, 4 schedulers each issuing one warp instruction a cycle
L2_FLUSH_BYTES = 512 << 20


def kernel_sha():
    """Hash of the step kernel's source code with comments and blank lines left
    out, so that the recorded counters survive edits to comments only."""
    import re
    p = os.path.join(ROOT, "paper_1804_09152_gb300", "csrc", "lf_kernels.cu")
    src = re.sub(r"/\*.*?\*/", "", open(p).read(), flags=re.S)
    lines = [re.sub(r"//.*$", "", l).rstrip() for l in src.splitlines()]
    code = "\n".join(l for l in lines if l.strip())
    return hashlib.sha256(code.encode()).hexdigest()[:16]


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


@contextlib.contextmanager
def profiled():
    """The timed region as the profiler's capture range (cudaProfilerStart /
    Stop; no effect without a profiler attached)."""
    import torch
    torch.cuda.profiler.start()
    try:
        yield
    finally:
        torch.cuda.profiler.stop()


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def aggregate(dist, seconds, units, device):
    """Whole-job figures over all ranks: the slowest rank's time and the units
    every rank processed (independent jobs per rank, so no other exchange)."""
    if dist is None:
        return seconds, float(units)
    import torch
    t = torch.tensor([float(seconds)], device=device, dtype=torch.float64)
    u = torch.tensor([float(units)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


ORACLE_SAMPLE_SECONDS = 20.0              # bound on one oracle sample (large meshes take fewer steps)
TUNE_AT, TUNE_TRIAL = 100, 32             # batch autotuning: steps before the trials, steps per trial


def host_cores():
    """Cores the threaded oracle runs on (it uses every online core)."""
    return os.cpu_count() or 1


class OracleSample:
    """The FP64 oracle on a bounded sample of a workload's jobs.

    ``jobs`` is a list of (mesh, seeds, coefficient matrices or None).  The
    operators are built once, before any timing; ``run`` then advances every
    job from its seeds by ``n_steps`` time steps (or until ``seconds`` have
    passed) and returns (skeleton entries, seconds, steps taken per job).
    threads = 0 runs each step on every core (orc_step_threads, the same
    arithmetic as the single-thread step), 1 the literal single-thread step.
    """

    def __init__(self, oracle, jobs):
        self.oracle = oracle
        self.jobs = []
        for m, seeds, mats in jobs:
            L = oracle.cotan_laplacian(m.V, m.F)
            mats = [M.astype(np.float64) for M in mats] if mats is not None else (None, None, None)
            self.jobs.append((m.n_v, L, np.asarray(seeds), mats))

    def run(self, n_steps, seconds=ORACLE_SAMPLE_SECONDS, threads=0):
        units, done = 0, []
        t = 0.0
        for n_v, L, seeds, mats in self.jobs:
            F = self.oracle.seed(n_v, seeds)
            k = 0
            while k < n_steps and t < seconds:
                t0 = time.perf_counter()
                F, sk = self.oracle.step(L, F, W=mats[0], A=mats[1], E=mats[2], threads=threads)
                t += time.perf_counter() - t0
                units += sk
                k += 1
            done.append(k)
            if t >= seconds:
                break
        return units, t, done


def oracle_sample(jobs):
    """The one place the benchmark reaches the oracle: its CPU-baseline and
    reference legs."""
    import oracle
    return OracleSample(oracle, jobs)


def single_mesh_jobs(wl):
    m = wl["mesh"]()
    mats = wl["coefs"](wl["k"] + 1) if wl.get("coefs") else None
    return [(m, synth.sample_seeds(m.n_v, wl["k"], wl["seed_stream"]), mats)]


# Vertex order of the batch's meshes as given to the library: "generated"
# (the generators' own: subdivision order for icospheres, scan order for
# tori) or "locality" (renumbered by paper_1804_09152_gb300.ordering, as a
# caller does with a scattered mesh: a Morton curve for icospheres, reverse
# Cuthill-McKee for tori).
BATCH_ORDER = {"ico": "morton", "torus": "rcm"}


def batch_jobs(specs=None, order="generated"):
    specs = specs or synth.batch_mix()
    cache, jobs = {}, []
    for sp in specs:
        key = (sp.kind, sp.size)
        if key not in cache:
            m = synth.make_mesh(sp)
            if order == "locality" and sp.kind in BATCH_ORDER:
                from paper_1804_09152_gb300.ordering import locality_order
                V, F, _ = locality_order(m.V, m.F, BATCH_ORDER[sp.kind])
                m = synth.Mesh(V, F)
            cache[key] = m
        m = cache[key]
        jobs.append((m, synth.sample_seeds(m.n_v, min(sp.k, m.n_v // 4), sp.seed_stream), None))
    return jobs


def cpu_baseline_line(sampler, n_steps, what, seconds=ORACLE_SAMPLE_SECONDS):
    """The cpu_baseline object: the threaded oracle on every core, with a
    short single-thread figure beside it for scale."""
    units, dt, done = sampler.run(n_steps, seconds, threads=0)
    u1, dt1, done1 = sampler.run(min(n_steps, 2), min(seconds, 5.0), threads=1)
    return {"value": units / dt, "unit": UNIT, "cores": host_cores(), "kind": "oracle",
            "sample": f"{what}: the first {max(done)} time steps of {len(done)} job(s) from their seeds "
                      f"({sum(done)} job-steps, {dt:.1f} s, literal Algorithm 1 in FP64 over vertex ranges "
                      f"on {host_cores()} threads)",
            "single_thread": {"value": u1 / dt1, "unit": UNIT, "cores": 1,
                              "sample": f"the first {max(done1)} steps of {len(done1)} job(s), {dt1:.1f} s"}}


def run_reference(args, jobs, config, n_steps):
    """The oracle arm: each bench step advances the bounded sample of the
    workload's jobs on every host core.  Rank 0 only."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    sampler = oracle_sample(jobs)
    vals = []
    for i in range(args.warmup + args.steps):
        units, dt, done = sampler.run(n_steps, ORACLE_SAMPLE_SECONDS, threads=0)
        if i >= args.warmup:
            vals.append((units, dt, done))
    units = sum(v[0] for v in vals)
    secs = sum(v[1] for v in vals)
    value = units / secs
    done = vals[0][2]
    sample = (f"per bench step: the first {max(done)} time steps of {len(done)} job(s) from their seeds, "
              f"FP64 oracle on {host_cores()} threads")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / len(vals),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": config,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": host_cores(), "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(args, wl):
    import torch
    import paper_1804_09152_gb300 as pkg
    pkg.build()
    from paper_1804_09152_gb300 import _lib as lf

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    m = wl["mesh"]()
    seeds = synth.sample_seeds(m.n_v, wl["k"], wl["seed_stream"])
    T = wl["steps"]
    stream = torch.cuda.Stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    with torch.cuda.stream(stream):
        dev = lf.torch_device(stream)
        mesh = lf.Mesh(m.V, m.F, device=dev, field_dtype=wl["dtype"])
        if args.schedule != "auto":
            mesh.set_schedule(args.schedule)
        sched = {v: k for k, v in lf.SCHEDULES.items()}[mesh.schedule]
        coefs = wl["coefs"](wl["k"] + 1) if wl.get("coefs") else None
        if coefs is not None:
            mesh.seed(seeds)
            mesh.set_coefficients(*coefs)          # kept across the re-seeding of every job

        def job():
            mesh.seed(seeds)
            e1 = torch.cuda.Event(enable_timing=True)
            e2 = torch.cuda.Event(enable_timing=True)
            e1.record(stream)
            mesh.step(T)
            e2.record(stream)
            lab = mesh.labels()
            return e1, e2, lab

        for _ in range(args.warmup):
            job()
        stats0 = mesh.stats()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        job_ms, step_ms, units, io, retries = [], [], 0, 0, 0
        wall0 = time.perf_counter()
        with ClockSampler(local) as clk, profiled():
            for _ in range(args.steps):
                flush.zero_()                          # evict L2 between jobs
                torch.cuda.synchronize()
                s0 = mesh.stats()
                e0 = torch.cuda.Event(enable_timing=True)
                e3 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                e1, e2, lab = job()
                e3.record(stream)
                e3.synchronize()
                s1 = mesh.stats()
                job_ms.append(e0.elapsed_time(e3))
                step_ms.append(e1.elapsed_time(e2))
                units += s1["skeleton_total"]
                io += s1["nnz_io_total"]
                retries += s1["retries"]
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        wall = time.perf_counter() - wall0
        st = mesh.stats()

    clk_summary = clk.summary()
    t_job = sum(job_ms) / 1e3
    t_all, units_all = aggregate(dist, t_job, units, "cuda")
    value = units_all / t_all

    # roofline of the step kernel: algorithmic bytes (ideal reuse) per launch
    vb = st["value_bytes"]
    launches = args.steps * T
    bytes_L = 4 * (m.n_v + 1) + 8 * st["operator_nnz"]
    bytes_total = launches * (bytes_L + 2 * 4 * (m.n_v + 1)) + (2 + vb) * io
    t_step = sum(step_ms) / 1e3
    achieved = bytes_total / t_step / 1e9
    peak, peak_kind = measured_peaks()
    counters = None
    if NCU_COUNTERS["kernel_sha"] == kernel_sha() and wl["dtype"] == "f32" and wl.get("coefs") is None:
        counters = NCU_COUNTERS.get(args.workload, {}).get(sched)
    traffic = counters["bytes_per_launch"] if counters else None
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "peak_kind": peak_kind,
                "algorithmic_bytes_per_launch": bytes_total / launches,
                "us_per_launch": 1e6 * t_step / launches}
    stale = NCU_COUNTERS.get(args.workload, {}).get(sched) if NCU_COUNTERS["kernel_sha"] != kernel_sha() else None
    if stale and wl["dtype"] == "f32" and wl.get("coefs") is None:
        # counters of an earlier kernel source: stated beside the null, not as the traffic
        roofline["traffic_earlier_source"] = {"bytes_per_launch": stale["bytes_per_launch"],
                                              "kernel_sha": NCU_COUNTERS["kernel_sha"], "current_sha": kernel_sha()}
    if counters:
        roofline["traffic_measured_under"] = f"schedule {sched}"
        # the bound that binds: instruction issue (ncu's warp-instruction count
        # per launch over the event-timed launch, against one warp instruction
        # per scheduler and cycle at the SM clock sampled during the run)
        mhz = clk_summary.get("sm_mhz") or clk_summary.get("sm_max_mhz") or 2070.0
        peak_issue = SM_COUNT * SUBPARTITIONS * mhz * 1e6
        issued = counters["warp_instructions_per_launch"] / (t_step / launches)
        roofline["issue"] = {"achieved": issued / 1e12, "peak": peak_issue / 1e12, "unit": "T warp-instr/s",
                             "frac": issued / peak_issue,
                             "warp_instructions_per_launch": counters["warp_instructions_per_launch"]}

    # end to end through the C ABI from host buffers: create (mesh upload and
    # device operator build), seed, steps, labels back to the host, destroy
    e2e_units, e2e_t = 0, 0.0
    n_e2e = max(1, min(args.steps, 3))
    # the job's inputs in pinned host memory, as a serving process holds them
    V_h = torch.from_numpy(np.ascontiguousarray(m.V)).pin_memory().numpy()
    F_h = torch.from_numpy(np.ascontiguousarray(m.F)).pin_memory().numpy()
    with torch.cuda.stream(stream):
        for _ in range(n_e2e):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            mm = lf.Mesh(V_h, F_h, device=lf.torch_device(stream), field_dtype=wl["dtype"])
            mm.seed(seeds)
            if coefs is not None:
                mm.set_coefficients(*coefs)
            mm.step(T)
            lab = mm.labels()
            s = mm.stats()
            mm.close()
            torch.cuda.synchronize()
            e2e_t += time.perf_counter() - t0
            e2e_units += s["skeleton_total"]
    h2d = 24 * m.n_v + 12 * m.n_f + 4 * wl["k"]          # vertices, faces, seeds (the operator is built on the device)
    if coefs is not None:
        h2d += sum(M.nbytes for M in coefs)
    d2h = 4 * m.n_v

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": statistics.mean(job_ms), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": wl["dtype"], "data": "synthetic",
        "config": {"workload": args.workload, "desc": wl["desc"], "n_v": m.n_v, "n_f": m.n_f,
                   "seeds": wl["k"], "time_steps_per_job": T, "l2": "flushed between jobs (512 MiB write)",
                   "working_set_bytes": int(bytes_L + 2 * (4 * (m.n_v + 1) + (2 + vb) * st["capacity"])),
                   "schedule": sched,
                   "lloyd_and_dual": "not part of this line"},
        "latency_ms": {"p50": float(np.percentile(job_ms, 50)), "p99": float(np.percentile(job_ms, 99))},
        "roofline": roofline,
        "e2e": {"value": e2e_units / e2e_t, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "jobs": n_e2e},
        "gpu_launches": args.steps * (T + 4) + retries,   # seed (fill, scatter, head records), steps, labels
        "clocks": clk_summary,
        "wall_s": wall,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_line(oracle_sample(single_mesh_jobs(wl)), args.cpu_sample_steps,
                                                 f"{args.workload}, {T} time steps per job")
    mesh.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def _job_bytes(st, n_v):
    """Algorithmic bytes of one step of one job, without the field traffic."""
    return 4 * (n_v + 1) + 8 * st["operator_nnz"] + 2 * 4 * (n_v + 1)


def run_batch(args):
    """Batching form, the default line: 64 mixed jobs (icosphere / noisy torus,
    10k-600k vertices, 32-2048 seeds, FP32 / BF16, 1000 steps) advanced
    together by lf_step_batch, against the same jobs stepped one at a time
    with lf_step.  Under torchrun every rank runs the whole mix on its own GPU
    (independent jobs: weak scaling, no data-path collective)."""
    import torch
    import paper_1804_09152_gb300 as pkg
    pkg.build()
    from paper_1804_09152_gb300 import _lib as lf

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    specs = synth.batch_mix()
    T = specs[0].steps
    stream = torch.cuda.Stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    jobs = batch_jobs(specs, args.order)
    geo = [m for m, _, _ in jobs]
    seeds = [sd for _, sd, _ in jobs]
    with torch.cuda.stream(stream):
        dev = lf.torch_device(stream)
        meshes = [lf.Mesh(m.V, m.F, device=dev, field_dtype=sp.dtype) for m, sp in zip(geo, specs)]

        def seed_all():
            for mesh, sd in zip(meshes, seeds):
                mesh.seed(sd)

        def timed(fn):
            flush.zero_()                      # evict L2 before every timed batch
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            return e0.elapsed_time(e1) / 1e3

        # the autotuner: per job, after TUNE_AT steps from its seeds (past the
        # first transient), time both schedules on the job alone and keep the
        # faster (lf_tune); untimed, reported as tune_s
        torch.cuda.synchronize()
        t_tune = time.perf_counter()
        if args.schedule == "auto":
            for mesh, sd in zip(meshes, seeds):
                mesh.seed(sd)
                mesh.step(args.tune_at)
                mesh.tune(TUNE_TRIAL)
        else:
            for mesh in meshes:
                mesh.set_schedule(args.schedule)
        torch.cuda.synchronize()
        t_tune = time.perf_counter() - t_tune
        tuned = [mesh.schedule for mesh in meshes]
        for _ in range(args.warmup):
            seed_all()
            lf.lf_step_batch(meshes, T)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        times, units, io, retries = [], 0, 0, 0
        with ClockSampler(local) as clk, profiled():
            for _ in range(args.steps):
                seed_all()
                times.append(timed(lambda: lf.lf_step_batch(meshes, T)))
                sts = [mesh.stats() for mesh in meshes]
                units += sum(s["skeleton_total"] for s in sts)
                io += sum(s["nnz_io_total"] * (2 + s["value_bytes"]) for s in sts)
                retries += sum(s["retries"] for s in sts)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        # the same batch under one fixed schedule for every job
        fixed, fixed_s = {}, {}
        for name in (() if args.timed_only else ("ctas4", "ctas5", "ctas3", "hot", "lean")):
            for mesh in meshes:
                mesh.set_schedule(name)
            seed_all()
            lf.lf_step_batch(meshes, T)            # graphs for this grouping
            seed_all()
            t_fixed = timed(lambda: lf.lf_step_batch(meshes, T))
            fixed[name] = sum(mesh.stats()["skeleton_total"] for mesh in meshes) / t_fixed
            fixed_s[name] = t_fixed
        for mesh, sc in zip(meshes, tuned):
            mesh.set_schedule(sc)
        t_plain = units_plain = t_e2e = e2e_units = None
        if not args.timed_only:
            # the same jobs one at a time (each under its tuned schedule)
            seed_all()
            t_plain = timed(lambda: [mesh.step(T) for mesh in meshes])
            units_plain = sum(mesh.stats()["skeleton_total"] for mesh in meshes)
            # end to end through the C ABI from pinned host buffers: create (mesh
            # upload, device operator build), seed, the batch, labels to the host
            pinned = [(torch.from_numpy(np.ascontiguousarray(m.V)).pin_memory().numpy(),
                       torch.from_numpy(np.ascontiguousarray(m.F)).pin_memory().numpy()) for m in geo]
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            fresh = [lf.Mesh(V, F, device=dev, field_dtype=sp.dtype) for (V, F), sp in zip(pinned, specs)]
            for mesh, sd, sc in zip(fresh, seeds, tuned):
                mesh.set_schedule(sc)                   # the tuned schedule, as a serving process keeps it
                mesh.seed(sd)
            lf.lf_step_batch(fresh, T)
            e2e_units = 0
            for mesh in fresh:
                mesh.labels()
                e2e_units += mesh.stats()["skeleton_total"]
                mesh.close()
            torch.cuda.synchronize()
            t_e2e = time.perf_counter() - t0
        sts = [mesh.stats() for mesh in meshes]
    secs = sum(times)
    t_all, units_all = aggregate(dist, secs, units, "cuda")
    value = units_all / t_all
    # roofline: algorithmic bytes of every job's step (operator, row arrays,
    # field in and out) over the event-timed steps; one step is one launch
    # per storage type over all the jobs of that type
    launches = args.steps * T
    bytes_step = sum(_job_bytes(s, m.n_v) for s, m in zip(sts, geo))
    bytes_total = launches * bytes_step + io
    achieved = bytes_total / secs / 1e9
    peak, peak_kind = measured_peaks()
    # DRAM traffic and instructions: captured with every job under one
    # schedule; the line takes the schedule most jobs run under here
    main = max(lf.SCHEDULES, key=lambda k: tuned.count(lf.SCHEDULES[k]))
    counters = None
    if NCU_COUNTERS["kernel_sha"] == kernel_sha():
        counters = NCU_COUNTERS["batch64"].get(main)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": counters["bytes_per_step"] if counters else None, "peak_kind": peak_kind,
                "algorithmic_bytes_per_step": bytes_total / launches, "us_per_step": 1e6 * secs / launches,
                "launches_per_step": len({(sp.dtype, sc) for sp, sc in zip(specs, tuned)})}
    clk_summary = clk.summary()
    stale = NCU_COUNTERS["batch64"].get(main) if NCU_COUNTERS["kernel_sha"] != kernel_sha() else None
    if stale:
        # counters of an earlier kernel source: stated beside the null, not as the traffic
        roofline["traffic_earlier_source"] = {"bytes_per_step": stale["bytes_per_step"], "under": f"every job on {main}",
                                              "kernel_sha": NCU_COUNTERS["kernel_sha"], "current_sha": kernel_sha()}
    if counters:
        roofline["traffic_measured_under"] = f"every job on {main} ({tuned.count(lf.SCHEDULES[main])} of " \
                                             f"{len(tuned)} jobs here)"
        if main in fixed_s:
            # instruction issue of that batch: ncu's warp instructions per step
            # over its event-timed step, against one warp instruction per
            # scheduler and cycle at the SM clock sampled during the run
            mhz = clk_summary.get("sm_mhz") or clk_summary.get("sm_max_mhz") or 2070.0
            peak_issue = SM_COUNT * SUBPARTITIONS * mhz * 1e6
            issued = counters["warp_instructions_per_step"] / (fixed_s[main] / T)
            roofline["issue"] = {"achieved": issued / 1e12, "peak": peak_issue / 1e12, "unit": "T warp-instr/s",
                                 "frac": issued / peak_issue, "under": f"every job on {main}",
                                 "warp_instructions_per_step": counters["warp_instructions_per_step"]}
    n_v_total = sum(m.n_v for m in geo)
    config = {"workload": "batch64", "jobs": len(specs), "n_v_total": n_v_total,
              "time_steps_per_job": T, "bf16_jobs": sum(sp.dtype == "bf16" for sp in specs),
              "desc": "64 jobs: icosphere level 4-8 or noisy torus (p=1/2), n_v log-uniform 10k-600k, "
                      "k log-uniform 32-2048, FP32 or BF16 storage with FP32 arithmetic (p=1/2), "
                      "1000 steps (stream 6); a bench step is the whole batch",
              "l2": "flushed before every timed batch (512 MiB write); the batch working set exceeds L2",
              "vertex_order": args.order if args.order == "generated" else
              "locality: icospheres along a Morton curve, tori by reverse Cuthill-McKee (ordering.locality_order)"}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * t_all / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic", "config": config,
        "latency_ms": {"p50": 1e3 * float(np.percentile(times, 50)), "p99": 1e3 * float(np.percentile(times, 99)),
                       "what": "one batch of 64 jobs, seeds to 1000 steps"},
        "vs_plain": None if t_plain is None else
        {"value": units_plain / t_plain, "unit": UNIT, "speedup": (units / secs) / (units_plain / t_plain),
         "desc": "the same jobs stepped one after another with lf_step on this GPU"},
        "schedules": {("tuned" if args.schedule == "auto" else args.schedule): units / secs,
                      **{f"all_{k}": v for k, v in fixed.items()}, "unit": UNIT,
                      "jobs": {k: tuned.count(v) for k, v in lf.SCHEDULES.items()}, "tune_s": t_tune,
                      "desc": f"per job, lf_tune after {args.tune_at} steps ({TUNE_TRIAL} steps per schedule and round, "
                              "two rounds) picks the step kernel's register allocation for 4, 5 or 3 CTAs per SM, "
                              "the lean register-tier path with the full step for the tiles outside it, or the lean gather with "
                              "the other tiers per vertex (same bits); the "
                              "batch under the tuned schedules against every job under one fixed schedule"},
        "roofline": roofline,
        "e2e": None if t_e2e is None else
        {"value": e2e_units / t_e2e, "unit": UNIT,
         "h2d_bytes_per_step": int(sum(24 * m.n_v + 12 * m.n_f + 4 * len(sd) for m, sd in zip(geo, seeds))),
         "d2h_bytes_per_step": int(4 * n_v_total), "jobs": len(specs)},
        "gpu_launches": launches * roofline["launches_per_step"] + retries,
        "clocks": clk_summary,
    }
    for mesh in meshes:
        mesh.close()
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_line(oracle_sample(jobs), args.cpu_sample_steps,
                                                 "batch64, 1000 time steps per job", seconds=15.0)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def cell_area_stats(m, labels, k):
    """Areas of the cells of a labelling (a vertex carries a third of the area
    of each face around it): coefficient of variation and a histogram of
    area / mean area."""
    P = m.V[m.F]
    fa = 0.5 * np.linalg.norm(np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0]), axis=1)
    va = np.zeros(m.n_v)
    for c in range(3):
        np.add.at(va, m.F[:, c], fa / 3.0)
    cov = labels >= 0
    area = np.bincount(labels[cov], weights=va[cov], minlength=k)
    rel = area / area.mean()
    edges = [0.0, 0.25, 0.5, 0.75, 1.0, 1.25, 1.5, 1.75, 2.0, np.inf]
    hist, _ = np.histogram(rel, bins=edges)
    return {"cv": float(area.std() / area.mean()), "min_rel": float(rel.min()), "max_rel": float(rel.max()),
            "hist_edges": [e if np.isfinite(e) else "inf" for e in edges], "hist": hist.tolist(),
            "empty_cells": int((area == 0).sum()), "base_vertices": int((~cov).sum())}


def dual_quality(V, tris):
    """Triangle quality of a dual mesh as the paper's table of extraction
    metrics reports it: 2 r_in / r_circ (1 for an equilateral triangle; mean
    and minimum), the mean and minimum of the smallest angle per triangle,
    and the share of angles below 30 degrees."""
    P = np.asarray(V)[np.asarray(tris)]
    a = np.linalg.norm(P[:, 1] - P[:, 2], axis=1)
    b = np.linalg.norm(P[:, 2] - P[:, 0], axis=1)
    c = np.linalg.norm(P[:, 0] - P[:, 1], axis=1)
    area = 0.5 * np.linalg.norm(np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0]), axis=1)
    q = 2.0 * (2.0 * area / (a + b + c)) / (a * b * c / (4.0 * area))
    cos = np.stack([(b * b + c * c - a * a) / (2 * b * c), (c * c + a * a - b * b) / (2 * c * a),
                    (a * a + b * b - c * c) / (2 * a * b)], 1)
    ang = np.degrees(np.arccos(np.clip(cos, -1.0, 1.0)))
    return {"triangles": int(len(tris)), "mean_quality": float(q.mean()), "min_quality": float(q.min()),
            "mean_min_angle": float(ang.min(1).mean()), "min_angle": float(ang.min()),
            "angles_below_30_pct": float(100.0 * (ang < 30.0).mean())}


def run_lloyd(args):
    """C2 with the paper's full pipeline (Sec. 5): 2000 steps, then Lloyd-like
    rounds (seed update + 2000 steps each), then the dual mesh (Sec. 5.2)."""
    import torch
    import paper_1804_09152_gb300 as pkg
    pkg.build()
    from paper_1804_09152_gb300 import _lib as lf

    wl = WORKLOADS["grid512"]
    m = wl["mesh"]()
    seeds = synth.sample_seeds(m.n_v, wl["k"], wl["seed_stream"])
    T, R = wl["steps"], args.lloyd_rounds
    stream = torch.cuda.Stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    with torch.cuda.stream(stream):
        mesh = lf.Mesh(m.V, m.F, device=lf.torch_device(stream))

        def ev():
            e = torch.cuda.Event(enable_timing=True)
            e.record(stream)
            return e

        def pipeline():
            mesh.seed(seeds)
            e0 = ev()
            mesh.step(T)
            units = mesh.stats()["skeleton_total"]
            upd_ms = 0.0
            for _ in range(R):
                a = ev()
                mesh.lloyd(1, 0)                  # the seed update alone
                b = ev()
                mesh.step(T)
                b.synchronize()
                upd_ms += a.elapsed_time(b)
                units += mesh.stats()["skeleton_total"]
            c = ev()
            tri = mesh.extract_dual()
            d = ev()
            d.synchronize()
            return e0.elapsed_time(d), upd_ms / max(R, 1), c.elapsed_time(d), units, len(tri)

        for _ in range(args.warmup):
            pipeline()
        res = []
        with ClockSampler(torch.cuda.current_device()) as clk:
            for _ in range(args.steps):
                flush.zero_()
                torch.cuda.synchronize()
                res.append(pipeline())
        # cell areas and dual-mesh quality before, after one and after all
        # rounds (untimed run of the same pipeline)
        mesh.seed(seeds)
        mesh.step(T)
        areas = [cell_area_stats(m, mesh.labels(), wl["k"])]
        quality = {"0": dual_quality(m.V, mesh.extract_dual())}
        for r in range(R):
            mesh.lloyd(1, T)
            if r == 0:
                quality["1"] = dual_quality(m.V, mesh.extract_dual())
        areas.append(cell_area_stats(m, mesh.labels(), wl["k"]))
        quality[str(R)] = dual_quality(m.V, mesh.extract_dual())
        mesh.close()
    total_ms = sum(r[0] for r in res)
    units = sum(r[3] for r in res)
    line = {
        "metric": METRIC, "value": units / (total_ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / len(res), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "grid512_lloyd", "desc": wl["desc"] + f", then {R} Lloyd-like rounds of {T} steps "
                   "and the dual mesh", "lloyd_rounds": R, "time_steps_per_round": T,
                   "l2": "flushed before each pipeline (512 MiB write)"},
        "lloyd_update_ms": statistics.mean(r[1] for r in res),
        "dual_extraction_ms": statistics.mean(r[2] for r in res),
        "dual_triangles": res[-1][4],
        "cell_areas": {"before_lloyd": areas[0], f"after_{R}_rounds": areas[1]},
        "dual_quality_by_rounds": quality,
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)


def run_dt_sweep(args):
    """The Δt study of Sec. 6 on synthetic irregular meshes: the same seeds at
    Δt = 0.1, 1, 5 and 10 for the same simulated time (300 units), labels
    read every unit of simulated time; agreement of the final labels with
    those at Δt = 0.1 and the step count after which no label changes."""
    import torch
    import paper_1804_09152_gb300 as pkg
    pkg.build()
    from paper_1804_09152_gb300 import study

    meshes = {"torus256": lambda: synth.noisy_torus(256), "ico6": lambda: synth.icosphere(6),
              "grid256": lambda: synth.planar_grid(256, jitter=0.2, seed=2)}
    dts = (0.1, 1.0, 5.0, 10.0)
    k, horizon = 256, 300.0
    res, units, total_ms = {}, 0, 0.0
    with ClockSampler(torch.cuda.current_device()) as clk:
        for name, fac in meshes.items():
            m = fac()
            r = study.dt_sweep(m.V, m.F, synth.sample_seeds(m.n_v, k, 11), dts, horizon=horizon)
            res[name] = {str(dt): {key: v for key, v in x.items() if key != "labels"} for dt, x in r.items()}
            res[name]["n_v"] = m.n_v
            units += sum(x["skeleton_total"] for x in r.values())
            total_ms += sum(x["ms"] for x in r.values())
    line = {
        "metric": METRIC, "value": units / (total_ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": 1, "warmup": 0,
        "ms_per_step": total_ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": "dt_sweep", "desc": f"noisy torus 256^2, icosphere level 6, jittered grid 256^2; "
                   f"{k} seeds (stream 11); dt in {list(dts)}, {horizon:g} units of simulated time each, "
                   "labels read every unit", "timing": "host wall clock of each run, label reads included"},
        "study": res,
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)


def run_serve(args):
    """Serving form: the Poisson trace (200 jobs/s by default, 2000 jobs or 60 s;
    n_v log-normal in [5k, 2M]; icosphere / torus / grid; 16-8192 seeds;
    500-3000 steps; half the jobs with 5 Lloyd-like rounds and the dual mesh)
    submitted at its arrival times to an lf_server with a 150 GB budget.
    --serve-rate sets another arrival rate (the same jobs, arrivals scaled),
    --serve-jobs a prefix."""
    import torch
    import paper_1804_09152_gb300 as pkg
    pkg.build()
    from paper_1804_09152_gb300 import _lib as lf

    trace = synth.serve_trace(rate=args.serve_rate)[: args.serve_jobs]
    cache = {}
    for sp in trace:
        if (sp.kind, sp.size) not in cache:
            cache[(sp.kind, sp.size)] = synth.make_mesh(sp)
    seeds = [synth.sample_seeds(cache[(sp.kind, sp.size)].n_v, sp.k, sp.seed_stream) for sp in trace]
    torch.cuda.synchronize()
    with ClockSampler(torch.cuda.current_device()) as clk:
        with lf.Server(**({"chunk_steps": args.chunk_steps} if args.chunk_steps else {})) as srv:
            t0 = time.monotonic_ns()
            ids = []
            for sp, sd in zip(trace, seeds):
                due = t0 + int(sp.arrival * 1e9)
                while time.monotonic_ns() < due:
                    time.sleep(min(1e-3, max(0.0, (due - time.monotonic_ns()) / 1e9)))
                m = cache[(sp.kind, sp.size)]
                ids.append((srv.submit(m.V, m.F, sd, sp.steps, arrival_ns=due, lloyd_rounds=sp.lloyd_rounds,
                                       extract_dual=sp.dual), m.n_v))
            assert srv.drain(3600.0) == lf.LF_OK
            t_end = time.monotonic_ns()
            lat, units = [], 0
            for jid, n_v in ids:
                st, info, _ = srv.wait(jid, 0.0, release=True)
                assert st == lf.LF_OK, st
                lat.append((info["finish_ns"] - info["arrival_ns"]) / 1e6)
                units += info["skeleton_total"]
            sst = srv.stats()
    wall = (t_end - t0) / 1e9
    # the same jobs one at a time through lf_step (no arrivals: back to back);
    # the first --plain-jobs of them (the throughput of a prefix)
    t1 = time.perf_counter()
    units_plain = 0
    n_plain = min(len(trace), args.plain_jobs)
    for sp, sd in zip(trace[:n_plain], seeds[:n_plain]):
        m = cache[(sp.kind, sp.size)]
        with lf.Mesh(m.V, m.F) as mesh:
            mesh.seed(sd)
            mesh.step(sp.steps)
            units_plain += mesh.stats()["skeleton_total"]
            for _ in range(sp.lloyd_rounds):
                mesh.lloyd(1, sp.steps)
                units_plain += mesh.stats()["skeleton_total"]
            if sp.dual:
                mesh.extract_dual()
            mesh.labels()
    t_plain = time.perf_counter() - t1
    line = {
        "metric": METRIC, "value": units / wall, "unit": UNIT, "n_gpus": 1, "steps": len(trace), "warmup": 0,
        "ms_per_step": 1e3 * wall / len(trace), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": "serve", "jobs": len(trace), "arrival_rate_per_s": args.serve_rate,
                   "last_arrival_s": trace[-1].arrival, "hbm_budget_bytes": 150_000_000_000,
                   "lloyd_and_dual_jobs": sum(sp.lloyd_rounds > 0 for sp in trace),
                   "desc": "the Poisson trace (stream 7): n_v log-normal in [5k, 2M], icosphere / "
                           "torus / grid, k log-uniform 16-8192, steps U{500..3000}; half the jobs (stream 8) add 5 "
                           "Lloyd-like rounds and the dual mesh; a step of this line is one job"},
        "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))},
        "jobs_per_s": len(trace) / wall,
        "vs_plain": {"value": units_plain / t_plain, "unit": UNIT, "speedup": (units / wall) / (units_plain / t_plain),
                     "desc": f"the first {n_plain} jobs back to back, one at a time, lf_create_mesh to lf_labels"},
        "server": {"peak_running": sst["peak_running"], "peak_bytes": sst["peak_bytes"], "batches": sst["batches"],
                   "busy_s": sst["busy_ns"] / 1e9},
        "e2e": {"value": units / wall, "unit": UNIT, "h2d_bytes_per_step": None, "d2h_bytes_per_step": None},
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=list(WORKLOADS) + ["batch64", "serve", "grid512_lloyd", "dt_sweep"],
                    default="batch64")
    ap.add_argument("--lloyd-rounds", type=int, default=10)
    ap.add_argument("--dtype", choices=["f32", "bf16", "f16"], default=None,
                    help="storage type of the field values (mesh workloads; default: the workload's)")
    ap.add_argument("--serve-jobs", type=int, default=2000, help="serve: jobs of the trace (it also ends at 60 s)")
    ap.add_argument("--serve-rate", type=float, default=200.0, help="serve: mean arrivals per second")
    ap.add_argument("--plain-jobs", type=int, default=300, help="serve: jobs of the one-at-a-time comparison")
    ap.add_argument("--chunk-steps", type=int, default=0, help="serve: steps between admission rounds (0: default)")
    ap.add_argument("--cpu-sample-steps", type=int, default=None,
                    help="time steps per job of the CPU-baseline sample (default: 200, 60 for batch64)")
    ap.add_argument("--ref-sample-steps", type=int, default=None,
                    help="time steps per job of one reference-arm step (default: 40, 3 for batch64)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--order", choices=["generated", "locality"], default="generated",
                    help="batch64: the meshes' vertex numbering (locality: renumbered before lf_create_mesh)")
    ap.add_argument("--tune-at", type=int, default=TUNE_AT,
                    help="batch64: steps from the seeds before lf_tune's trials")
    ap.add_argument("--timed-only", action="store_true",
                    help="batch64: time the batch only, without the fixed-schedule, one-at-a-time and end-to-end "
                         "runs (the command the profiles capture)")
    ap.add_argument("--schedule", choices=["auto", "ctas4", "ctas5", "ctas3", "hot", "lean"], default="auto",
                    help="the step-kernel schedule of every job (auto: lf_tune per job in batch64, the "
                         "default schedule ctas4 on the single-mesh workloads)")
    args = ap.parse_args()
    batch = args.workload == "batch64"
    if args.cpu_sample_steps is None:
        args.cpu_sample_steps = 60 if batch else 200
    if args.ref_sample_steps is None:
        args.ref_sample_steps = 3 if batch else 40
    if args.impl == "reference" and batch:
        if int(os.environ.get("RANK", "0")) != 0:
            return None
        specs = synth.batch_mix()
        config = {"workload": "batch64", "jobs": len(specs), "time_steps_per_job": specs[0].steps,
                  "desc": "64 jobs: icosphere level 4-8 or noisy torus (p=1/2), n_v log-uniform 10k-600k, "
                          "k log-uniform 32-2048, 1000 steps (stream 6); the oracle computes in FP64"}
        return run_reference(args, batch_jobs(specs, args.order), config, args.ref_sample_steps)
    if args.impl == "reference" and args.workload not in WORKLOADS:
        if int(os.environ.get("RANK", "0")) == 0:
            print(json.dumps({"impl": "reference", "unavailable": f"the oracle arm times the batch and the "
                              f"single-mesh workloads; {args.workload} is a composite of them"}), flush=True)
        return None
    if batch:
        return run_batch(args)
    if args.workload == "serve":
        return run_serve(args)
    if args.workload == "grid512_lloyd":
        return run_lloyd(args)
    if args.workload == "dt_sweep":
        return run_dt_sweep(args)
    wl = dict(WORKLOADS[args.workload])
    if args.dtype:
        wl["dtype"] = args.dtype
        wl["desc"] = wl["desc"].replace("FP32 field", f"{args.dtype.upper()} field storage, FP32 arithmetic")
    if args.impl == "reference":
        run_reference(args, single_mesh_jobs(wl), {"workload": args.workload, "desc": wl["desc"]},
                      args.ref_sample_steps)
    else:
        run_ours(args, wl)


if __name__ == "__main__":
    main()
