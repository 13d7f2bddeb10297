#!/usr/bin/env python
"""Benchmark of the adaptive-multigrid Wilson-Dirac solve on one B300.

One step is one whole job on the 16^3x32 workload (epsilon = 0.6 random SU(3) field, three
masses at which lambda_min(D^dag D) is 1e-3, 1e-4, 1e-5 of its free-field value, 12 point
sources): load the gauge field, run the adaptive setup (2 levels, 4^4 blocks, N = 24,
200 relaxation steps, 2 passes) at the lightest mass, then solve the 12 right-hand sides to a
true FP64 residual of 1e-10 at each of the three masses (red/black outer GCR(8), FP32 cycle and
Krylov vectors, FP64 reliable updates, all right-hand sides of a mass batched).  `value` is the device time of one step (the
time-to-solution of the job, setup included); the same job in all-FP64 with one
right-hand side at a time is timed once for comparison ("plain_fp64").

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl wmg|reference]

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle instead.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402

METRIC = "MG-GCR time-to-solution @1e-10 vs plain; dslash GB/s; p50/p99 solve latency"
WORKLOADS = {
    "16x16x16x32": dict(dims=(16, 16, 16, 32), eps=0.6, gauge_seed=11, nvec=24, block=(4, 4, 4, 4), nrhs=12,
                        masses_file=os.path.join(ROOT, "tests", "golden", "masses_16x16x16x32_eps0.6.json")),
}
# The larger workloads (a line for the design notes, not the benchmark's job): 3 levels, Gaussian
# right-hand sides, a hand-chosen mass near the field's critical region (no oracle mass search was
# run on these volumes); the 48^3x96 one with FP16 null vectors and its device footprint.
LARGE = {
    "24x24x24x48": dict(dims=(24, 24, 24, 48), eps=0.7, gauge_seed=31, nvec=[24, 32],
                        block=[(4, 4, 4, 4), (2, 2, 2, 2)], nrhs=12, mass=-1.2, prec_nullvec=1, gcr_restart=16),
    # FGCR(8) on the red/black system: its FP32 basis (2 x restart half-lattice vectors per rhs)
    # is a quarter of FGCR(16) on the whole lattice
    "48x48x48x96": dict(dims=(48, 48, 48, 96), eps=0.7, gauge_seed=51, nvec=[24, 32],
                        block=[(4, 4, 4, 4), (2, 2, 2, 2)], nrhs=4, mass=-1.2, prec_nullvec=2, gcr_restart=8),
}
# outer iterations per mass the GPU arm measures on this job (mean over the 12 point sources), used
# by --impl reference, which runs without a GPU, to scale its sample to the whole job
REFERENCE_ITERS = {"16x16x16x32": [37.0, 43.9, 49.3]}
REFERENCE_CG = {"16x16x16x32": [9.1, 23.4, 43.0]}  # coarsest CG iterations per cycle, the same source
# DRAM traffic per launch group of a class from one ncu capture (dram__bytes_read.sum +
# dram__bytes_write.sum), taken with the committed command of the named profile; a group of the coarse
# class is one application of the coarsest Schur complement (its odd-site and even-site passes).
# "changed": the kernel changed after the capture, so the line reports no traffic (the last
# capture's figure is kept beside it) until the capture is taken again.
TRAFFIC = {"coarse": {"bytes_per_launch": 46.1e6, "profile": "profiles/coarse_schur_16x16x16x32_nrhs12.md"}}
GAUGE_REALS = 12  # reals per link of the FP32 fine operator in the job (wmg_set_gauge_compression)
PROF_CLASSES = ("dslash_sloppy", "dslash_fp64", "coarse", "restrict", "prolong", "blas", "setup", "cgnr",
                "blas_coarse")


# Used only while the oracle's mass file does not exist yet: masses near the critical mass of
# this field, chosen by hand; the JSON line then says so ("masses_source").
PROVISIONAL_MASSES = {"16x16x16x32": [-1.0, -1.1, -1.2]}


def load_masses(w, override, name):
    """(masses heaviest first, source)."""
    if override:
        return sorted((float(m) for m in override.split(",")), reverse=True), "command line"
    try:
        with open(w["masses_file"]) as f:
            rec = json.load(f)
    except OSError:
        return PROVISIONAL_MASSES[name], "provisional (the oracle mass file is missing)"
    return sorted(rec["masses"].values(), reverse=True), "oracle " + os.path.relpath(w["masses_file"], ROOT)


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0}, "fallback"


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={index}", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        self.p.wait()
        self.f.seek(0)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------------------------------
# CPU oracle (reference arm and cpu_baseline): the FP64 oracle as it stands, timed on this host
# ------------------------------------------------------------------------------------------
def _threads(n):
    """Limit the oracle to n host threads: the OpenMP pool of its C operator and, where
    threadpoolctl is installed, numpy's BLAS pools (the oracle's numpy work is mostly elementwise)."""
    import contextlib
    import ctypes
    try:
        ctypes.CDLL("libgomp.so.1").omp_set_num_threads(int(n))
    except OSError:
        pass
    try:
        from threadpoolctl import threadpool_limits
    except ImportError:
        return contextlib.nullcontext()
    return threadpool_limits(limits=int(n))


class OracleJob:
    """A bounded sample of the job run with the oracle's own code on the workload's shapes.

    The oracle builds its own two-level hierarchy for the field (Gaussian starts, Gram-Schmidt,
    Galerkin product; both timed, they are one setup rebuild).  Then, timed: MR relaxation steps
    on D psi = 0 (the setup's first pass) and outer flexible-GCR iterations of one point source
    with the oracle's cycle (MR nu = 4, even-odd coarsest CG to the GPU arm's coarse tolerance)
    at each mass.  The job estimate scales these by the counts of the job: relaxation steps x N,
    setup passes x rebuilds, (passes - 1) x N cycle applications, and right-hand sides x the outer
    iterations the GPU arm measured at each mass in the same run."""

    def __init__(self, w, masses, coarse_tol, log=None):
        from oracle import mg
        self.w, self.masses, self.coarse_tol = w, list(masses), coarse_tol
        dims, N, blk = w["dims"], w["nvec"], w["block"]
        self.U = synth.gauge_field(dims, w["eps"], w["gauge_seed"])
        self.starts = synth.setup_starts(dims, N, 5)
        self.b = synth.point_sources(dims, 1)[0]
        t0 = time.perf_counter()
        self.P = mg.block_orthonormalise(self.starts, blk)
        self.t_gs = time.perf_counter() - t0
        t0 = time.perf_counter()
        self.Ac = mg.galerkin(mg.WilsonOp(self.U, self.masses[-1]), self.P, blk)
        self.t_gal = time.perf_counter() - t0
        self.cores = os.cpu_count()

    def time_relax(self, steps):
        from oracle import mg, solvers
        op = mg.WilsonOp(self.U, self.masses[-1])
        s = self.starts[0]
        t0 = time.perf_counter()
        solvers.mr(op.apply, np.zeros_like(s), s, steps)
        return (time.perf_counter() - t0) / steps

    def time_iterations(self, m, k):
        """Seconds per outer iteration at mass m (k iterations of the oracle's flexible GCR, its
        closing true residual included) and the mean coarsest-CG iterations per cycle."""
        from oracle import mg, solvers
        op = mg.WilsonOp(self.U, m)
        prm = solvers.CycleParams(nu=4, coarse_tol=self.coarse_tol, coarse_maxit=2000, coarse_eo=True)
        H = solvers.Hierarchy([op, self.Ac.shifted(m - self.masses[-1])], [self.P], [self.w["block"]], prm)
        t0 = time.perf_counter()
        solvers.fgcr(op.apply, lambda r: solvers.cycle(H, 0, r), self.b, 1e-10, 16, max_iter=k)
        return (time.perf_counter() - t0) / k, float(np.mean(H.coarse_iters)) if H.coarse_iters else 0.0

    def time_coarse_cg(self, m, k=10):
        """Seconds per iteration of the oracle's even-odd coarsest CG at mass m (k iterations
        against one, the difference per iteration; no convergence test is met)."""
        from oracle import eo
        A = self.Ac.shifted(m - self.masses[-1])
        b = synth.coarse_starts(A.dims, A.n, 1, 7)[0]
        t0 = time.perf_counter()
        eo.cgnr_eo(A, b, 1e-30, 1)
        t1 = time.perf_counter()
        eo.cgnr_eo(A, b, 1e-30, k + 1)
        t2 = time.perf_counter()
        return ((t2 - t1) - (t1 - t0)) / k

    def estimate(self, t_mr, t_iter, iters, prm):
        """Job seconds: setup (relaxation, rebuilds, improvement cycles) + the solves."""
        N, nrhs = self.w["nvec"], self.w["nrhs"]
        setup = N * prm["setup_relax"] * t_mr + prm["setup_passes"] * (self.t_gs + self.t_gal) \
            + (prm["setup_passes"] - 1) * N * t_iter[-1]
        return setup + sum(nrhs * it * t for it, t in zip(iters, t_iter))


def cpu_baseline_sample(w, masses, iters, cg_per_cycle, prm, k=1):
    """The oracle's sample at all cores and the lightest mass again on one thread.  The coarsest
    solve is charged at the GPU arm's CG iterations per cycle (cg_per_cycle, per mass): the
    oracle's iteration time has its own coarsest CG iterations replaced by those, each at the
    oracle's measured time per CG iteration."""
    job = OracleJob(w, masses, prm["coarse_tol"])
    with _threads(job.cores):
        t_mr = job.time_relax(2)
        timed = [job.time_iterations(m, k) for m in masses]
        t_cg = [job.time_coarse_cg(m) for m in masses]
    t_iter = [t + (g - c) * tc for (t, c), g, tc in zip(timed, cg_per_cycle, t_cg)]
    est = job.estimate(t_mr, t_iter, iters, prm)
    with _threads(1):
        t1, c1 = job.time_iterations(masses[-1], k)
        tc1 = job.time_coarse_cg(masses[-1])
    t1 = t1 + (cg_per_cycle[-1] - c1) * tc1
    out = {"value": est, "unit": "s", "cores": job.cores, "kind": "oracle",
           "sample": (f"FP64 oracle on this host ({job.cores} threads): its own 2-level hierarchy for the 16^3x32 "
                      f"field (Gram-Schmidt {job.t_gs:.1f} s, Galerkin {job.t_gal:.1f} s, timed), 2 MR relaxation "
                      f"steps ({t_mr:.3f} s each) and {k} outer FGCR iteration(s) of one point source at each mass "
                      f"({', '.join(f'{t:.2f}' for t, _ in timed)} s per iteration with "
                      f"{', '.join(f'{c:.0f}' for _, c in timed)} coarsest CG iterations per cycle on the oracle's "
                      f"hierarchy; {', '.join(f'{1e3 * t:.1f}' for t in t_cg)} ms per coarsest CG iteration, charged at "
                      f"the GPU arm's {', '.join(f'{g:.0f}' for g in cg_per_cycle)} per cycle: "
                      f"{', '.join(f'{t:.2f}' for t in t_iter)} s per outer iteration), "
                      f"scaled to the job by its counts: N x {prm['setup_relax']} relaxation steps, "
                      f"{prm['setup_passes']} rebuilds, {prm['setup_passes'] - 1} x N setup cycles, 12 right-hand "
                      f"sides x the GPU arm's outer iterations per mass {[round(i, 1) for i in iters]}"),
           "per_iteration_s": t_iter, "coarse_cg_iteration_s": t_cg, "one_thread": {
               "iteration_s_lightest_mass": t1,
               "value": est * t1 / t_iter[-1],
               "note": "the job estimate scaled by the one-thread / all-thread time of an outer iteration at the "
                       "lightest mass (the rebuild times were taken with all threads)"}}
    return out


def run_reference(args, w):
    """--impl reference: the oracle, each step one timed outer iteration at one of the masses (in
    turn), the value the job estimate from that step (see OracleJob)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    masses, _ = load_masses(w, args.masses, args.workload)
    prm = dict(setup_relax=200, setup_passes=2, coarse_tol=0.1)
    iters, cg = REFERENCE_ITERS[args.workload], REFERENCE_CG[args.workload]
    job = OracleJob(w, masses, prm["coarse_tol"])
    t_mr = job.time_relax(2)
    t_cg = {m: job.time_coarse_cg(m) for m in masses}

    def one(m):
        t, c = job.time_iterations(m, 1)
        return t + (cg[masses.index(m)] - c) * t_cg[m]

    base = {m: one(m) for m in masses}
    vals, walls = [], []
    for i in range(args.warmup + args.steps):
        m = masses[i % len(masses)]
        t0 = time.perf_counter()
        base[m] = one(m)
        wall = time.perf_counter() - t0
        if i >= args.warmup:
            vals.append(job.estimate(t_mr, [base[x] for x in masses], iters, prm))
            walls.append(wall)
    v = statistics.mean(vals)
    sample = (f"FP64 oracle ({job.cores} threads): its own hierarchy for the field (Gram-Schmidt {job.t_gs:.1f} s, "
              f"Galerkin {job.t_gal:.1f} s), 2 MR relaxation steps, then per step one outer FGCR iteration of one "
              f"point source at one of the masses in turn (the step's wall time is ms_per_step); value = the job "
              f"estimate from the latest iteration time at each mass (its coarsest CG charged at the GPU arm's {cg} "
              f"CG iterations per cycle, at the oracle's measured time per CG iteration) x 12 right-hand sides x "
              f"the GPU arm's outer iterations {iters}, plus the setup's relaxation, rebuilds and cycles")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "s", "higher_is_better": False,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": statistics.mean(walls) * 1e3, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": args.workload},
        "cpu_baseline": {"value": v, "unit": "s", "cores": job.cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


# ------------------------------------------------------------------------------------------
# GPU arm
# ------------------------------------------------------------------------------------------
def run_gpu(args, w):
    import torch

    from paper_0912_2186_b300 import build, wmg
    build.build()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    masses, masses_source = load_masses(w, args.masses, args.workload)
    m_light = masses[-1]
    dims, nrhs = w["dims"], w["nrhs"]
    V = int(np.prod(dims))
    U = synth.gauge_field(dims, w["eps"], w["gauge_seed"])
    b = synth.point_sources(dims, nrhs)
    U_dev = torch.from_numpy(U).cuda()
    b_dev = torch.from_numpy(b).cuda()
    x_dev = torch.zeros_like(b_dev)
    ctx = wmg.Context(dims)
    ctx.set_gauge_compression(GAUGE_REALS)
    # setup: 200 relaxation steps and one improvement pass (measured fastest for this field at
    # unchanged outer iteration counts; the library default is 100 steps and 5 passes); the fine
    # solve red/black preconditioned (Sec. 3: multigrid combined with red/black preconditioning);
    # FP64 reliable updates after the iterated residual fell by 1e-5 (library default 1e-4: one
    # FP64 true residual fewer per solve here, at 0.1 more outer iterations); the outer solver is
    # GCR(8), as in Sec. 3 (library default 16)
    params = wmg.default_params(nvec=[w["nvec"]], block=[w["block"]], prec_sloppy=wmg.PREC_SINGLE,
                                seed=1000 + rank, max_iter=20000, setup_relax=200, setup_passes=2, fine_eo=1,
                                reliable_delta=1e-5, gcr_restart=8)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    record = {"iters": [], "true_resid": [], "phases": []}
    # host buffers of the end-to-end measurement: pinned, allocated once
    U_host = torch.from_numpy(U).pin_memory().numpy()
    b_host = torch.from_numpy(b).pin_memory().numpy()
    x_host = torch.zeros(b.shape, dtype=torch.complex128).pin_memory().numpy()

    def step(host=False):
        t0 = time.perf_counter()
        if host:
            ctx.load_gauge(U_host)
        else:
            ctx.load_gauge(U_dev)
        ctx.set_mass(m_light)
        ctx.setup(params)
        ph = {"setup_s": time.perf_counter() - t0, "solve_s": []}
        for m in masses:
            t1 = time.perf_counter()
            ctx.set_mass(m)
            if host:
                st, info = ctx.solve(b_host, x_host, nrhs)
            else:
                st, info = ctx.solve(b_dev, x_dev, nrhs)
            if st != wmg.OK:
                raise RuntimeError(f"solve at m={m} did not converge: {info}")
            ph["solve_s"].append(time.perf_counter() - t1)
            record["iters"].append([i["iters"] for i in info])
            record["true_resid"].append(max(i["true_resid"] for i in info))
        record["phases"].append(ph)

    def barrier():
        if dist:
            dist.barrier()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    # timed region: device time of each step (CUDA events on the legacy stream the library uses)
    record["iters"].clear()
    record["true_resid"].clear()
    record["phases"].clear()
    clocks = Clocks(local)
    times = []
    l0 = wmg.launch_count()
    torch.cuda.nvtx.range_push("timed")  # lets a profiler restrict itself to the timed steps
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        step()
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
    torch.cuda.nvtx.range_pop()
    launches = (wmg.launch_count() - l0) // max(args.steps, 1)
    clk = clocks.stop()
    t_step = statistics.mean(times)
    if dist:
        tt = torch.tensor([t_step], device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_step = float(tt.item())
    iters = record["iters"]
    resid = max(record["true_resid"])
    phases = {"setup_s": statistics.mean(p["setup_s"] for p in record["phases"]),
              "solve_s_per_mass": [statistics.mean(p["solve_s"][i] for p in record["phases"])
                                   for i in range(len(masses))]}

    # end to end through the host-buffer entry points
    e2e = []
    for _ in range(max(1, min(args.steps, 2))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        step(host=True)
        torch.cuda.synchronize()
        e2e.append(time.perf_counter() - t0)
    h2d = U.nbytes + len(masses) * b.nbytes
    d2h = len(masses) * b.nbytes

    # instrumented step, phase by phase (setup, then each mass): per-class kernel time, algorithmic
    # bytes and launches, and the coarsest CG iterations per cycle at each mass (two Schur-complement
    # applications per CG iteration, one cycle per restriction)
    prof, cg_per_cycle = None, []

    def add(tot, part):
        if tot is None:
            return part
        return {k: {f: tot[k][f] + part[k][f] for f in part[k]} for k in part}

    ctx.load_gauge(U_dev)
    ctx.set_mass(m_light)
    ctx.profile(True)
    ctx.setup(params)
    prof = add(prof, ctx.profile_get())
    for m in masses:
        ctx.set_mass(m)
        ctx.profile(True)
        ctx.solve(b_dev, x_dev, nrhs)
        part = ctx.profile_get()
        prof = add(prof, part)
        cg_per_cycle.append(part["coarse"]["launches"] / max(2 * part["restrict"]["launches"], 1))
    ctx.profile(False)
    # the dominant class: the largest share of kernel time among the classes with accounted bytes
    hot = max((k for k in PROF_CLASSES if prof[k]["bytes"] > 0), key=lambda k: prof[k]["ms"])
    peaks, src = measured_peaks()
    achieved = prof[hot]["bytes"] / (prof[hot]["ms"] * 1e-3) / 1e9 if prof[hot]["ms"] > 0 else 0.0
    tr = TRAFFIC.get(hot)
    roof = {"bound": "hbm", "kernel": hot, "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": achieved / peaks["hbm_gbs"],
            "traffic": tr["bytes_per_launch"] if tr and not tr.get("changed") else None,
            "traffic_profile": tr["profile"] if tr else None,
            "traffic_last_capture": tr["bytes_per_launch"] if tr and tr.get("changed") else None,
            "traffic_note": ("kernel changed since the capture: " + tr["changed"]) if tr and tr.get("changed") else None,
            "bytes_per_launch": prof[hot]["bytes"] / max(prof[hot]["launches"], 1), "peak_source": src,
            "launches": prof[hot]["launches"], "ms_per_launch": prof[hot]["ms"] / max(prof[hot]["launches"], 1)}
    total_ms = sum(prof[k]["ms"] for k in PROF_CLASSES)
    breakdown = {k: {"ms": round(prof[k]["ms"], 3), "share": round(prof[k]["ms"] / total_ms, 4) if total_ms else 0,
                     "GB_s": round(prof[k]["bytes"] / (prof[k]["ms"] * 1e6), 1) if prof[k]["ms"] > 0 else None}
                 for k in PROF_CLASSES}
    # the FP64 dslash (true residuals) is bound by the FP64 ALU on this part: 1368 flop per
    # site and right-hand side against the probed FP64 FMA peak
    alu = wmg.probe_alu_peaks() if rank == 0 else None
    if alu and prof["dslash_fp64"]["ms"] > 0:
        gf = 1368.0 * V * prof["dslash_fp64"]["units"] / (prof["dslash_fp64"]["ms"] * 1e-3) / 1e9
        breakdown["dslash_fp64"].update({"GFLOP_s": round(gf, 1), "bound": "fp64 alu",
                                         "frac_of_probed_fp64": round(gf / (alu["fp64_tflops"] * 1e3), 3)})

    # isolated dslash throughput (FP32, 12 right-hand sides and 1; 12-real links, then 8- and 18-real)
    dsl = {}
    for gc, nr in ((12, 1), (12, nrhs), (8, 1), (8, nrhs), (18, 1), (18, nrhs)):
        ctx.set_gauge_compression(gc)
        xin = torch.zeros(nr * 12 * V, dtype=torch.complex64, device="cuda")
        xout = torch.zeros_like(xin)
        ctx.pack(wmg.PREC_SINGLE, b_dev[:nr].contiguous(), xin, nr)
        for _ in range(3):
            ctx.apply_D(wmg.PREC_SINGLE, xin, xout, nr)
        reps = 50
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        flush.zero_()
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            ctx.apply_D(wmg.PREC_SINGLE, xin, xout, nr)
        e1.record()
        torch.cuda.synchronize()
        sec = e0.elapsed_time(e1) / 1e3 / reps
        by = V * 4 * gc * 4 + nr * V * 48 * 4
        dsl[f"nrhs{nr}" + ("" if gc == 12 else f"_{gc}real")] = {"us": sec * 1e6, "GB_s": by / sec / 1e9,
                                                                 "GFLOP_s": 1368 * V * nr / sec / 1e9}
    # one job step each with the 8-real and the 18-real links in the FP32 operator
    step_links = {}
    for gc in (8, 18):
        ctx.set_gauge_compression(gc)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        step()
        e1.record()
        torch.cuda.synchronize()
        step_links[gc] = e0.elapsed_time(e1) / 1e3
    ctx.set_gauge_compression(GAUGE_REALS)
    # one job step without red/black preconditioning (the whole-lattice outer solve, fine_eo = 0)
    params.fine_eo = 0
    n_it = len(record["iters"])
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    step()
    e1.record()
    torch.cuda.synchronize()
    step_eo = {"s": e0.elapsed_time(e1) / 1e3,
               "iters_per_mass": [float(np.mean(i)) for i in record["iters"][n_it:n_it + len(masses)]],
               "max_true_resid": max(record["true_resid"][n_it:])}
    params.fine_eo = 1

    # plain comparison: the same job in all-FP64, one right-hand side at a time
    plain = None
    if not args.no_plain:
        pp = wmg.default_params(nvec=[w["nvec"]], block=[w["block"]], prec_sloppy=wmg.PREC_DOUBLE, seed=1000 + rank,
                                max_iter=20000, setup_relax=200, setup_passes=2, gcr_restart=8)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        ctx.load_gauge(U_dev)
        ctx.set_mass(m_light)
        ctx.setup(pp)
        pit = []
        for m in masses:
            ctx.set_mass(m)
            for r in range(nrhs):
                st, info = ctx.solve(b_dev[r:r + 1].contiguous(), x_dev[r:r + 1], 1)
                pit.append(info[0]["iters"])
        e1.record()
        torch.cuda.synchronize()
        plain = {"s": e0.elapsed_time(e1) / 1e3, "iters_mean": float(np.mean(pit)), "prec": "f64", "nrhs_per_solve": 1}

    # unpreconditioned baselines on the same kernels (FP64, one point source per mass): outer
    # iterations and seconds of plain restarted GCR(16) and of CG on the normal equations, beside
    # MG-GCR's, to show the critical slowing down the multigrid preconditioner removes
    baselines = None
    if not args.no_plain:
        ctx.load_gauge(U_dev)
        baselines = {"gcr16_fp64": [], "cgnr_fp64": []}
        b1 = b_dev[:1].contiguous()
        x1 = torch.zeros_like(b1)
        for m in masses:
            ctx.set_mass(m)
            for key, f in (("gcr16_fp64", lambda: ctx.solve(b1, x1, 1, plain=True)),
                           ("cgnr_fp64", lambda: ctx.solve_cgnr(b1, x1, 1, maxit=40000))):
                x1.zero_()
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                st, info = f()
                torch.cuda.synchronize()
                baselines[key].append({"mass": m, "iters": info[0]["iters"], "s": time.perf_counter() - t0,
                                       "converged": bool(info[0]["converged"]),
                                       "true_resid": info[0]["true_resid"]})

    serving = None
    if rank == 0 and not args.no_serving:
        ctx.close()
        torch.cuda.empty_cache()
        serving = run_serving(wmg, masses, masses_source)
    iters_mean = [float(np.mean(i)) for i in iters[:len(masses)]]
    # the oracle's timed sample, after every GPU measurement (nothing else runs meanwhile)
    cpu = None
    if rank == 0 and not args.no_cpu:
        cpu = cpu_baseline_sample(w, masses, iters_mean, cg_per_cycle, dict(setup_relax=params.setup_relax,
                                                              setup_passes=params.setup_passes,
                                                              coarse_tol=params.coarse_tol))
    if rank != 0:
        return
    out = {
        "metric": METRIC, "value": t_step, "unit": "s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t_step * 1e3, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": args.workload, "lattice": "x".join(map(str, dims)), "epsilon": w["eps"],
                   "masses": masses, "masses_source": masses_source, "rhs": f"{nrhs} point sources", "levels": 2, "block": "4^4", "nvec": w["nvec"],
                   "setup_passes": params.setup_passes, "setup_relax": params.setup_relax,
                   "coarse_tol": params.coarse_tol, "fine": "red/black (even-site Schur complement)",
                   "smoother": "MR nu=4 FP32", "outer": "FGCR(16) FP64 reliable",
                   "l2": "flushed (256 MB write) between timed steps", "parallelism": "replicas" if world > 1 else "1 GPU"},
        "solves_per_s": world * len(masses) * nrhs / t_step,
        "iters_per_mass": iters_mean,
        "iters_growth": max(iters_mean) / min(iters_mean),
        "coarse_cg_per_cycle": cg_per_cycle,
        "phases": phases,
        "max_true_resid": resid,
        "plain_fp64": plain,
        "speedup_vs_plain": (plain["s"] / t_step) if plain else None,
        "unpreconditioned_fp64": baselines,
        "dslash_fp32_isolated": dsl,
        "step_s_8real_links": step_links[8],
        "step_s_18real_links": step_links[18],
        "step_whole_lattice": step_eo,
        "kernel_breakdown": breakdown,
        "roofline": roof,
        "gpu_launches": int(launches),
        "e2e": {"value": statistics.mean(e2e), "unit": "s", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h), "host_memory": "pinned"},
        "cpu_baseline": cpu,
        "alu_peaks": alu,
        "serving": serving,
        "clocks": clk,
    }
    print(json.dumps(out))
    if dist:
        dist.destroy_process_group()


# ------------------------------------------------------------------------------------------
# serving: 200 seeded Poisson arrivals over three resident fields (continuous batching)
# ------------------------------------------------------------------------------------------
SERVING_FIELDS = [
    dict(dims=(8, 8, 8, 8), eps=0.4, gauge_seed=21, nvec=[8], block=[(4, 4, 4, 4)], masses=[0.05]),
    dict(dims=(16, 16, 16, 32), eps=0.6, gauge_seed=11, nvec=[24], block=[(4, 4, 4, 4)], masses=None),
    dict(dims=(24, 24, 24, 48), eps=0.7, gauge_seed=31, nvec=[24, 32], block=[(4, 4, 4, 4), (2, 2, 2, 2)],
         masses=[-1.15, -1.2, -1.25]),
]


def run_serving(wmg, masses16, masses_source, nreq=200, seed=2009, slots=12):
    import threading
    fields = []
    srv = wmg.Server(hbm_budget_bytes=240 << 30)
    for f in SERVING_FIELDS:
        ms = f["masses"] or masses16
        U = synth.gauge_field(f["dims"], f["eps"], f["gauge_seed"])
        ctx = wmg.Context(f["dims"])
        ctx.load_gauge(U)
        ctx.set_mass(ms[-1])  # the hierarchy is built at the field's lightest mass
        p = wmg.default_params(nlevels=len(f["nvec"]) + 1, nvec=f["nvec"], block=f["block"],
                               prec_sloppy=wmg.PREC_SINGLE)
        ctx.setup(p)
        fid = srv.add_field(ctx, slots)
        fields.append((fid, f["dims"], ms))
    rng = np.random.default_rng(seed)
    reqs = []
    for i in range(nreq):
        fi = int(rng.integers(0, len(fields)))
        fid, dims, ms = fields[fi]
        reqs.append((fid, float(ms[int(rng.integers(0, len(ms)))]), synth.gaussian_spinors(dims, int(rng.integers(1, 13)),
                                                                                        10_000 + i)))
    # capacity: the first 12 requests back to back
    t0 = time.perf_counter()
    warm = []
    for fid, m, b in reqs[:12]:
        x = np.zeros_like(b)
        warm.append(srv.submit(fid, m, b, x))
    for t in warm:
        srv.wait(t)
    cap_rhs = sum(b.shape[0] for _, _, b in reqs[:12]) / (time.perf_counter() - t0)
    mean_rhs = np.mean([b.shape[0] for _, _, b in reqs])
    rate = 0.75 * cap_rhs / mean_rhs                     # requests per second
    gaps = rng.exponential(1.0 / rate, size=nreq)
    xs = [np.zeros_like(b) for _, _, b in reqs]
    tickets = [None] * nreq

    def producer():
        for i, (fid, m, b) in enumerate(reqs):
            time.sleep(float(gaps[i]))
            tickets[i] = srv.submit(fid, m, b, xs[i])

    t0 = time.perf_counter()
    th = threading.Thread(target=producer)
    th.start()
    th.join()
    lat, worst, ok = [], 0.0, True
    for i, t in enumerate(tickets):
        st, info, l = srv.wait(t)
        ok = ok and st == wmg.OK
        lat.append(l)
        worst = max(worst, max(x["true_resid"] for x in info))
    wall = time.perf_counter() - t0
    srv.close()
    nrhs_total = sum(b.shape[0] for _, _, b in reqs)
    return {"requests": nreq, "rhs": int(nrhs_total), "arrival_rate_per_s": rate, "wall_s": wall,
            "p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
            "solves_per_s": nrhs_total / wall, "all_converged": ok, "max_true_resid": worst,
            "slots_per_field": slots,
            "fields": ["8^4 eps0.4 N8", "16^3x32 eps0.6 N24 (" + masses_source + " masses)",
                       "24^3x48 eps0.7 3-level N24/32 (hand-chosen masses)"]}


def run_probe(args, w):
    """--probe: the hot kernels of the job on the 16^3x32 workload inside the NVTX range "probe",
    for ncu captures (ncu --nvtx --nvtx-include "probe/") and quick CUDA-event timing.  The hierarchy
    is built first (the job's setup at the lightest mass); inside the range each of the FP32 fine
    dslash, restrict, prolong, the tensor-core coarse stencil and the even-odd Schur complement of
    the coarse operator runs --probe-reps times on 12 right-hand sides, then (--probe-solve) the 12
    point sources are solved once at --probe-mass (default the heaviest of the job's masses), with
    the benchmark's setup and solver parameters."""
    import torch

    from paper_0912_2186_b300 import build, wmg
    build.build()
    masses, _ = load_masses(w, args.masses, args.workload)
    dims, nr = w["dims"], w["nrhs"]
    V = int(np.prod(dims))
    # the library launches on this stream, so that CUDA graphs captured on it replay its kernels
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    ctx = wmg.Context(dims, stream=stream.cuda_stream)
    ctx.load_gauge(torch.from_numpy(synth.gauge_field(dims, w["eps"], w["gauge_seed"])).cuda())
    ctx.set_gauge_compression(args.probe_gauge)
    ctx.set_mass(masses[-1])
    ctx.setup(wmg.default_params(nvec=[w["nvec"]], block=[w["block"]], prec_sloppy=wmg.PREC_SINGLE, setup_relax=200,
                                 setup_passes=2, fine_eo=1, reliable_delta=1e-5, gcr_restart=8))
    m = args.probe_mass if args.probe_mass is not None else masses[0]
    ctx.set_mass(m)
    nc, n = ctx.level_info(1)
    g = torch.Generator(device="cuda").manual_seed(7)
    fi = torch.randn(nr * 12 * V, dtype=torch.complex64, device="cuda", generator=g)
    fo = torch.zeros_like(fi)
    ci = torch.randn(nr * nc * n, dtype=torch.complex64, device="cuda", generator=g)
    co = torch.zeros_like(ci)
    b = torch.from_numpy(synth.point_sources(dims, nr)).cuda()
    x = torch.zeros_like(b)
    ops = {
        "dslash": lambda: ctx.apply_D(wmg.PREC_SINGLE, fi, fo, nr),
        "restrict": lambda: ctx.restrict(0, wmg.PREC_SINGLE, fi, co, nr),
        "prolong": lambda: ctx.prolong(0, wmg.PREC_SINGLE, ci, fo, nr),
        "coarse": lambda: ctx.apply_coarse(1, wmg.PREC_HALF, ci, co, nr),
        "schur": lambda: ctx.apply_coarse_schur(1, wmg.PREC_HALF, ci, co, nr),
    }
    for f in ops.values():
        f()
    if args.probe_solve:
        ctx.solve(b, x, nr)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("probe")
    for f in ops.values():
        for _ in range(args.probe_reps):
            f()
    if args.probe_solve:
        ctx.solve(b, x, nr)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    # device time per call: 20 calls captured in a CUDA graph, replayed 5 times between events on
    # the library's stream (a host loop of short calls would time the host's issue rate instead)
    res = {"mass": m}
    for k, f in ops.items():
        gr = torch.cuda.CUDAGraph()
        with torch.cuda.graph(gr, stream=stream, capture_error_mode="thread_local"):
            for _ in range(20):
                f()
        gr.replay()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(5):
            gr.replay()
        e1.record(stream)
        torch.cuda.synchronize()
        res[k + "_us_per_call"] = e0.elapsed_time(e1) * 1e3 / 100
    print(json.dumps(res))
    ctx.close()


def run_large(args):
    """One setup and one batched solve on a larger workload: 3 levels (4^4 then 2^4 blocks, N = 24 and
    32), FP16 smoother storage, tensor-core coarse stencils (autotuned), Gaussian right-hand sides;
    time-to-solution (setup and solve), iterations, the library's FP64 true residuals, one of them
    checked with the oracle's C operator, the isolated dslash and the device footprint."""
    import torch

    from paper_0912_2186_b300 import build, wmg
    build.build()
    w = LARGE[args.large]
    dims, nrhs, m = w["dims"], w["nrhs"], w["mass"]
    V = int(np.prod(dims))
    U = synth.gauge_field(dims, w["eps"], w["gauge_seed"])
    b = synth.gaussian_spinors(dims, nrhs, w["gauge_seed"] + 1)
    ctx = wmg.Context(dims)
    ctx.load_gauge(torch.from_numpy(U).cuda())
    ctx.set_mass(m)
    p = wmg.default_params(nlevels=3, block=w["block"], nvec=w["nvec"], prec_sloppy=wmg.PREC_SINGLE,
                           prec_smoother=wmg.PREC_HALF, prec_nullvec=w["prec_nullvec"], coarse_tc=3,
                           fine_eo=args.large_eo, gcr_restart=w["gcr_restart"])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ctx.setup(p)
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t0
    bytes_setup = ctx.device_bytes()
    bd = torch.from_numpy(b).cuda()
    x = torch.zeros_like(bd)
    ctx.solve(bd, x, nrhs)  # warm: workspaces and graphs
    x.zero_()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st, info = ctx.solve(bd, x, nrhs)
    torch.cuda.synchronize()
    t_solve = time.perf_counter() - t0
    from oracle import cref
    x0 = x[0].cpu().numpy()
    ores = float(np.linalg.norm(b[0] - cref.apply_D(U, x0, m)) / np.linalg.norm(b[0]))
    impl = [ctx.coarse_impl(lv) for lv in (1, 2)]
    xin = torch.zeros(nrhs * 12 * V, dtype=torch.complex64, device="cuda")
    xout = torch.zeros_like(xin)
    for _ in range(3):
        ctx.apply_D(wmg.PREC_SINGLE, xin, xout, nrhs)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(20):
        ctx.apply_D(wmg.PREC_SINGLE, xin, xout, nrhs)
    e1.record()
    torch.cuda.synchronize()
    sec = e0.elapsed_time(e1) / 1e3 / 20
    peaks, _ = measured_peaks()
    by = V * 48 * 4 + nrhs * V * 48 * 4
    print(json.dumps({
        "workload": args.large, "mass": m, "mass_source": "hand-chosen", "nrhs": nrhs,
        "fine_eo": args.large_eo, "gcr_restart": w["gcr_restart"], "setup_s": t_setup,
        "solve_s": t_solve, "iters": [i["iters"] for i in info], "max_true_resid": max(i["true_resid"] for i in info),
        "oracle_resid_rhs0": ores, "status": int(st), "coarse_impl_and_tuner_ms": impl,
        "device_bytes_after_setup": bytes_setup, "device_bytes_after_solve": ctx.device_bytes(),
        "dslash_fp32": {"nrhs": nrhs, "us": sec * 1e6, "GB_s": by / sec / 1e9, "frac_hbm": by / sec / 1e9 / peaks["hbm_gbs"]},
    }))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="wmg", choices=["wmg", "reference"])
    ap.add_argument("--workload", default="16x16x16x32", choices=sorted(WORKLOADS))
    ap.add_argument("--masses", default=None, help="comma-separated masses (default: the oracle's)")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--probe", action="store_true", help="run the hot kernels in an NVTX range (profiling)")
    ap.add_argument("--probe-reps", type=int, default=2)
    ap.add_argument("--probe-gauge", type=int, default=12, choices=(8, 12, 18),
                    help="reals per link of the FP32 fine operator in --probe")
    ap.add_argument("--probe-mass", type=float, default=None)
    ap.add_argument("--large-eo", type=int, default=1, choices=(0, 1),
                    help="red/black outer solve in --large (fine_eo)")
    ap.add_argument("--probe-solve", action="store_true")
    ap.add_argument("--large", default=None, choices=sorted(LARGE),
                    help="one setup and solve on a larger workload (a line for the design notes)")
    args = ap.parse_args()
    w = WORKLOADS[args.workload]
    if args.large:
        run_large(args)
    elif args.probe:
        run_probe(args, w)
    elif args.impl == "reference":
        run_reference(args, w)
    else:
        run_gpu(args, w)


if __name__ == "__main__":
    main()
