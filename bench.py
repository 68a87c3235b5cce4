#!/usr/bin/env python
"""Throughput benchmark of the dynamical-core hot path on one GB300 (or N replicas).

One benchmark step = one dycore step (nsub predictor-corrector substeps with the
vertically implicit column solve, then Smagorinsky diffusion) followed by the
global mass integral, on a synthetic analytic state resident in HBM. Metric:
cell-level updates per second = cells x levels x substeps / time.

The headline ("value") is the R2B6 grid (327,680 cells, 491,520 edges) with 90
levels on a stretched height coordinate to 75 km, FP64, balanced 35 m/s jet with a
1 m/s Gaussian bump, dt = 90 s in 5 substeps, timed over --steps steps after
--warmup steps. The same JSON line carries the other workloads of the method, each
measured from its own freshly initialised state with its own fixed number of steps
(independent of --steps): the mixed-precision form of the headline workload, one
transported tracer, the divergence-damping and background-diffusion options,
terrain-following levels, R2B8/90 in FP64 and mixed precision with the mixed form's
error, R2B9/60 mixed, and the 64-member batched ensemble against sequential members;
plus the FP64 instruction rate measured on the device, the end-to-end rate through
the C ABI with host buffers, and the FP64 CPU oracle on the host cores (one core and
all cores).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gpu|reference]
                  [--workload r2b6-fp64|r2b8-mixed|r2b9-mixed|ensemble] [--quick]
  python bench.py --profile-step BISECTIONS NLEV PRECISION [NSTEPS [NTRACERS [TOPO_M]]]

--quick skips the R2B8, R2B9 and ensemble measurements. --profile-step runs one small
workload for kernel profilers (ncu) and prints nothing else. Under torchrun (N > 1)
every rank advances its own replica (no data exchange: "scaling": "weak"); rank 0
prints the JSON line with the max time over ranks. --impl reference times the FP64
CPU oracle on the host cores instead (rank 0 only).
"""
import argparse
import json
import multiprocessing
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2511_02021_gb300 import workloads as WL  # noqa: E402

METRIC = "cell-level updates/s per dycore substep, % HBM roofline; mixed vs FP64"
UNIT = "cell-level updates/s"
WORKLOADS = {"r2b6-fp64": WL.R2B6_JET, "r2b8-mixed": WL.R2B8_JET_MIXED, "r2b9-mixed": WL.R2B9_JET_MIXED,
             "ensemble": None}
PROG = ("vn", "w", "rho", "theta_v", "exner")
EPS32 = 2.0 ** -23
GRAV = 9.80665


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


# FP64 instruction rate of the GB300 from its unit counts and clock: 152 SMs x 2 FP64
# operations per SM per cycle (a fused multiply-add is one) x 2.07 GHz. The roofline divides
# by the rate measured on the device (icon_probe_fp64_rate); this derived figure is reported
# beside it.
FP64_INSTR_DERIVED = 152 * 2 * 2.07e9
# FP64 instructions per cell-level of one launch of the FP64 column solve (rows + Thomas +
# update), averaged over predictor and corrector, as ncu counts them executed at R2B5/90
# (sm__thread_inst_executed_pipe_fp64_pred_on.sum over cell-levels): predictor 47.9 + 8.9 +
# 14.0 = 70.8 (it forms and factors the tridiagonal matrix of S^n), corrector 37.9 + 3.9 +
# 17.0 = 58.8 (it substitutes with the predictor's factors).
COLUMN_FP64_OPS = 64.8
# FP64 instructions per cell-level of the mixed column, one launch averaged over the
# predictor and the corrector (the corrector's kernels include the FP64 divergence of the
# FP32 mass fluxes): see MX_OPS below, set from the kernels the state runs
MX_OPS = {"stored": 36, "recompute": 56}
# FP64 instructions per cell-level of the tracer transport of one tracer
TRACER_FP64_OPS = 77
# DRAM bytes per launch of a kernel kind measured by ncu on the current kernels (absent where
# the kernel changed after the counters were taken), mean of the predictor and corrector
# launches. Captured at R2B5/90 (the full sizes hold too much memory for a multi-pass capture)
# and scaled by cell-levels: every column does the same work, so the traffic grows in
# proportion. FP64 column 2.407 GB per launch at R2B5/90; lean mixed column 1.081 GB (its
# default shape, 9 blocks per SM in both stages).
NCU_TRAFFIC = {
    ("R2B6-L90-jet-fp64", "column_solve"): 2.407e9 * 4,
    ("R2B6-L90-jet-fp64", "mx_lean_column"): 1.081e9 * 4,
    ("R2B8-L90-jet-mixed", "mx_lean_column"): 1.081e9 * 64,
    ("R2B9-L60-jet-mixed", "mx_lean_column"): 1.081e9 * 256 * 60 / 90,
}


def max_over_ranks(ms, device):
    """The slowest rank's time: every rank passes its own and receives the maximum."""
    import torch
    import torch.distributed as td
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    td.all_reduce(t, op=td.ReduceOp.MAX)
    return float(t.item())


def job_value(units_per_rank, world, ms):
    """Whole-job throughput: the units all ranks processed (the same on every rank)
    over the slowest rank's time in milliseconds."""
    return world * units_per_rank / (ms * 1e-3)


# algorithmic bytes per cell-level-substep of the whole step: the state read and written by
# the two stages (5 volumes of vn, w, rho, theta_v, pi), the FP64 accumulators and the
# diffusion spread over the substeps
STEP_BYTES = {0: 271.0, 1: 239.0}


def step_hbm_roofline(value, precision, hbm_peak):
    """The whole step against the HBM roofline by its algorithmic bytes (the metric's
    '% HBM roofline'; the dominant kernel's own bound is in "roofline")."""
    b = STEP_BYTES[precision]
    return {"algorithmic_bytes_per_unit": b, "achieved_gbs": value * b / 1e9, "peak_gbs": hbm_peak,
            "frac": value * b / 1e9 / hbm_peak, "peak_source": "measured copy (MEASURED_PEAKS.json)"}


def counts_of(bisections):
    L = bisections + 1
    return 20 * 4 ** L, 30 * 4 ** L, 10 * 4 ** L + 2


def counts(wl):
    return counts_of(wl.bisections)


def kernel_model(kind, wl, mx_ops):
    """(algorithmic bytes, FP64 instructions) of ONE launch of a kernel kind, averaged over
    predictor and corrector launches: every input and output array element read or written
    once (8 B in FP64, 4 B in FP32), and the FP64 instructions of the expressions as written."""
    nc, ne, nv = counts(wl)
    N = wl.nlev
    H = N + 1
    b = 8.0
    table = {
        "vertex_curl_wmean": (b * (ne * N + nc * H + nv * N + nv * H), nv * N * 6 + nv * H * 7),
        "edge_vt_ke": (b * 3 * ne * N, ne * N * 8),
        "cell_ke": (b * (ne + nc) * N, nc * N * 3),
        "edge_tendency_flux": (b * (ne * N * 6.5 + nc * N * 4 + nv * N + nc * H + nv * H + ne * H),
                               ne * N * 22 + ne * H * 11),
        "column_solve": (b * (nc * N * 8 + ne * N * 2 + ne * H + nc * H * 2.5), nc * N * COLUMN_FP64_OPS),
        "diff_vertex": (b * (ne * N + 4 * nv * N), nv * N * 25),
        "diff_div": (b * (ne + nc) * N, nc * N * 7),
        "diff_edge": (b * (ne * N * 4 + nv * N * 5 + nc * N * 2), ne * N * 45),
        "diff_theta": (b * (ne * N + 4 * nc * N), nc * N * 12),
        "global_mass": (b * nc * N, nc * N * 2),
        "mx_vertex": (4.0 * (ne * N + nc * H + nv * N + nv * H), 0),
        "mx_edge_diag": (4.0 * 3 * ne * N, 0),
        "mx_cell_ke": (4.0 * (ne + nc) * N, 0),
        "mx_edge_tendency_flux": (4.0 * (ne * N * 6.5 + ne * H + nc * N * 4 + nv * N + nc * H + nv * H)
                                  + 8.0 * ne * N, ne * N * 1.0),
        "mx_column_solve": (nc * N * 98.0, nc * N * mx_ops),
        # lean column, one launch averaged over predictor and corrector: FP64 S^n read in both
        # sweeps (64 B), gathered inputs, right-hand-side base, elimination scratch, FP32 shadows,
        # and the corrector's FP64 updates and vertical flux (154 B); 11 FP64 instructions
        "mx_lean_column": (nc * N * 154.0, nc * N * 11.0),
        # its gather: three edges' FP32 fluxes and w-advection terms (each edge read for its two
        # cells once), the stage w rows, level-major outputs (40 B); the corrector's FP64
        # divergence (3 per cell-level, 1.5 averaged)
        "mx_lean_gather": (nc * N * 40.0, nc * N * 1.5),
        "mx_column_prep": (4.0 * (3 * ne * N + ne * H + nc * H * 3) + 8.0 * (nc * N * 3 + nc * H), nc * N * 3),
        "mx_diff_vertex": (4.0 * (2 * ne * N + 4 * nv * N + nc * N), 0),
        "mx_diff_edge": (4.0 * (ne * N * 4 + nv * N * 3 + nc * N * 2), 0),
        "mx_diff_theta": (4.0 * ne * N + 40.0 * nc * N, nc * N * 6),
    }
    return table.get(kind)


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi sampled every 200 ms during a timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.path = tempfile.mktemp(suffix=".csv")
        self.f = open(self.path, "w")
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None
        time.sleep(0.4)

    def stop(self):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()
        self.f.close()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9:
                rows.append(f)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------- the oracle on the host cores
class OracleSampler:
    """The oracle on the workload's grid and initial state (built once, untimed); each
    sample times one substep (predictor + corrector) continuing from the last one."""

    def __init__(self, wl):
        import oracle as O
        from oracle import dycore as OD
        self.OD, self.wl = OD, wl
        self.g = O.build_grid(2, wl.bisections)
        self.v = O.vertical_grid(wl.nlev)
        self.s = O.init_state(self.g, self.v, wl.seed, wl.case, noise_K=(wl.noise_K if wl.noise_K >= 0 else None))

    def sample(self):
        g, v, wl = self.g, self.v, self.wl
        acc = {"mflx": np.zeros((g.ne, v.N)), "wflx": np.zeros((g.nc, v.N + 1))}
        t0 = time.perf_counter()
        self.s = self.OD.substep(g, v, self.s, wl.dt / wl.nsub, wl.nsub, acc)
        return time.perf_counter() - t0


SAMPLE_DESC = "one substep (predictor + corrector) of %s per replica, init excluded"
_replica = None


def _replica_init(wl):
    global _replica
    os.environ["OMP_NUM_THREADS"] = "1"
    _replica = OracleSampler(wl)


def _replica_sample(_):
    return _replica.sample()


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def mem_available_gb():
    try:
        for line in open("/proc/meminfo"):
            if line.startswith("MemAvailable:"):
                return int(line.split()[1]) / 1e6
    except OSError:
        pass
    return 8.0


# host memory of one R2B6/90 oracle replica during a substep (grid, state, temporaries; 11.7 GB
# peak resident measured)
REPLICA_GB = 12.0


class OracleReplicas:
    """P replicas of the oracle on P host processes (one core each, started with spawn);
    one sample = one concurrent substep on every replica, timed on the wall clock."""

    def __init__(self, wl, procs):
        self.procs = procs
        ctx = multiprocessing.get_context("spawn")
        self.pool = ctx.Pool(procs, initializer=_replica_init, initargs=(wl,))
        self.pool.map(_replica_sample, range(procs))           # builds every replica (untimed)

    def sample(self):
        t0 = time.perf_counter()
        self.pool.map(_replica_sample, range(self.procs), chunksize=1)
        return time.perf_counter() - t0

    def close(self):
        self.pool.terminate()
        self.pool.join()


def replica_count():
    return max(1, min(host_cores(), int(mem_available_gb() * 0.5 / REPLICA_GB)))


def gpu_config(wl, world=1):
    nc, ne, _ = counts(wl)
    return {"workload": wl.name, "grid": "R2B%d" % wl.bisections, "cells": nc, "edges": ne, "levels": wl.nlev,
            "dt": wl.dt, "nsub": wl.nsub, "precision": "fp64" if wl.precision == 0 else "mixed",
            "parallelism": "replicas" if world > 1 else "single",
            "l2": "inputs larger than L2 (state %.2f GB)" % ((ne * wl.nlev + 4 * nc * wl.nlev) * 8 / 1e9)}


REFERENCE_BUDGET_S = 150.0


def run_reference(args, wl, rank):
    """The reference arm: the FP64 oracle on the host cores, one replica per usable core,
    each step one concurrent substep of the workload on every replica (the unit is the
    same cell-level update per substep as the GPU arm's; the GPU step adds one diffusion
    per 5 substeps)."""
    if rank != 0:
        return
    procs = replica_count()
    reps = OracleReplicas(wl, procs)
    vals = []
    try:
        # one sample is a whole substep of the workload on every replica (about 20-30 s of
        # host time); after one untimed warm-up sample, the arm times as many of the
        # requested steps as fit in REFERENCE_BUDGET_S, so that the run ends within a few
        # minutes, and reports the count it timed
        t_warm = reps.sample()
        n = max(1, min(args.steps, int(REFERENCE_BUDGET_S / max(t_warm, 1e-3))))
        for _ in range(n):
            vals.append(reps.sample())
    finally:
        reps.close()
    t = sum(vals) / len(vals)
    nc, _, _ = counts(wl)
    value = procs * nc * wl.nlev / t
    cfg = gpu_config(wl)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": len(vals), "warmup": 1, "steps_requested": args.steps, "warmup_requested": args.warmup,
            "ms_per_step": t * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": cfg,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": procs, "kind": "oracle",
                             "sample": SAMPLE_DESC % wl.name + "; each step = one concurrent substep on every "
                                       "replica", "cpu": cpu_model(), "host_cores": host_cores()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cpu_baseline(wl):
    """The oracle on one host core and on all usable cores (concurrent replicas)."""
    nc, _, _ = counts(wl)
    one = OracleSampler(wl)
    t1 = one.sample()
    del one
    procs = replica_count()
    reps = OracleReplicas(wl, procs)
    try:
        tp = reps.sample()
    finally:
        reps.close()
    return {"value": procs * nc * wl.nlev / tp, "unit": UNIT, "cores": procs, "kind": "oracle",
            "sample": SAMPLE_DESC % wl.name, "seconds": tp, "cpu": cpu_model(), "host_cores": host_cores(),
            "one_core": {"value": nc * wl.nlev / t1, "unit": UNIT, "cores": 1, "seconds": t1}}


# ---------------------------------------------------------------- GPU helpers
class Gpu:
    """The library bound to one device: PyTorch's allocator and a dedicated stream."""

    def __init__(self, local_rank, probe=True):
        import torch
        self.torch = torch
        torch.cuda.set_device(local_rank)
        from paper_2511_02021_gb300 import build as B
        B.build()
        import paper_2511_02021_gb300 as P
        from paper_2511_02021_gb300 import capi as C
        self.C = C
        P.use_torch_allocator(local_rank)
        self.stream = torch.cuda.Stream()
        torch.cuda.set_stream(self.stream)
        P.bind_torch_stream(self.stream)
        self.local_rank = local_rank
        self.names = [C.icon_kernel_kind_name(k) for k in range(C.ICON_KIND_COUNT)]
        fma, add = C.icon_probe_fp64_rate() if probe else (FP64_INSTR_DERIVED, FP64_INSTR_DERIVED)
        self.fp64_peak = fma
        self.fp64_probe = {"fma_per_s": fma, "add_per_s": add, "derived_per_s": FP64_INSTR_DERIVED,
                           "how": "icon_probe_fp64_rate: 16 x 256 threads per SM, 8 independent FP64 FMA "
                                  "(or ADD) chains per thread, best of 5 launches, CUDA events"}

    def events(self):
        E = self.torch.cuda.Event
        return E(enable_timing=True), E(enable_timing=True)

    def free_cache(self):
        self.torch.cuda.synchronize()
        self.torch.cuda.empty_cache()

    def timed(self, fn):
        """ms of fn() on the bound stream (CUDA events, synchronised on both sides)."""
        self.torch.cuda.synchronize()
        e0, e1 = self.events()
        e0.record(self.stream)
        fn()
        e1.record(self.stream)
        self.torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    def kinds(self, st, dt, nsub):
        """{kind: (ms per step, launches per step)} from two eager steps with CUDA events
        around every launch."""
        kms, kn = None, None
        for _ in range(2):
            kms, kn = self.C.icon_dycore_step_profile(st, dt, nsub, kms, kn)
        return {self.names[k]: (kms[k] / 2, kn[k] / 2) for k in range(self.C.ICON_KIND_COUNT) if kn[k] > 0}


def dominant_roofline(gpu, wl, kinds, hbm_peak, mx_ops, traffic_key=None):
    """The roofline of the kernel kind with the largest share of the step: its
    algorithmic bytes and FP64 instructions per launch over its mean launch time, against
    the measured HBM copy rate and the measured FP64 instruction rate; the bound is the
    larger fraction."""
    top = max(kinds.items(), key=lambda kv: kv[1][0])
    name, (ms_step, n_step) = top
    avg = ms_step / n_step
    model = kernel_model(name, wl, mx_ops)
    if model is None:
        return {"kernel": name, "launch_ms": avg, "launches_per_step": n_step}
    gbs = model[0] / (avg * 1e-3) / 1e9
    fops = model[1] / (avg * 1e-3)
    hbm = {"achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak,
           "peak_source": "measured copy (MEASURED_PEAKS.json)"}
    alu = {"achieved": fops / 1e9, "peak": gpu.fp64_peak / 1e9, "unit": "G FP64 instr/s",
           "frac": fops / gpu.fp64_peak, "peak_source": "measured (icon_probe_fp64_rate, FMA)",
           "derived_peak": FP64_INSTR_DERIVED / 1e9, "frac_of_derived": fops / FP64_INSTR_DERIVED}
    traffic = NCU_TRAFFIC.get((traffic_key or wl.name, name))
    if alu["frac"] > hbm["frac"]:
        roof = dict(alu, kernel=name, bound="alu", traffic=traffic, hbm=hbm)
    else:
        roof = dict(hbm, kernel=name, bound="hbm", traffic=traffic, fp64=alu)
    roof.update(launch_ms=avg, launches_per_step=n_step, fp64_instr_per_cell_level=model[1] / (counts(wl)[0] * wl.nlev))
    return roof


def measure(gpu, grid, wl, precision, steps, warmup, clocks=False, rank=0, world=1, options=(), ntracers=0,
            topo=None, seed=None):
    """Time `steps` steps (+ the mass integral) of a fresh state of the workload; returns
    the measurements. The state is freed afterwards."""
    C = gpu.C
    nc, ne, nv = counts(wl)
    N = wl.nlev
    kw = {}
    if topo:
        kw = {"topo_height_m": topo[0], "topo_radius_m": topo[1]}
    st = C.icon_state_init_ex(grid, wl.seed + rank if seed is None else seed, wl.case, noise_K=wl.noise_K,
                              precision=precision, **kw)
    try:
        for opt, val in options:
            C.icon_state_set_option(st, opt, val)
        if ntracers:
            C.icon_state_add_tracers(st, ntracers)
            xc = C.icon_grid_copy_table(grid, "x_c")
            for t in range(ntracers):
                C.icon_state_set_tracer(st, grid, N, t, np.repeat(1.0 + 0.5 * xc[:, 2:3], N, axis=1))
        m0 = C.icon_global_mass(st)
        for _ in range(warmup):
            C.icon_dycore_step(st, wl.dt, wl.nsub)
        kps = C.icon_state_step_kernels(st, wl.dt, wl.nsub) + 2      # + the mass integral's two
        mass_host = gpu.torch.empty(1, dtype=gpu.torch.float64, pin_memory=True)
        clk = ClockSampler(gpu.local_rank) if (clocks and rank == 0) else None
        if world > 1:
            import torch.distributed as td
            td.barrier()

        def run():
            for _ in range(steps):
                C.icon_dycore_step_async(st, wl.dt, wl.nsub)
                C.icon_global_mass_async(st, mass_host.data_ptr())
        ms = gpu.timed(run)
        if world > 1:
            import torch.distributed as td
            td.barrier()
            ms = max_over_ranks(ms, "cuda")
        clk = clk.stop() if clk else None
        C.icon_state_status(st)                                   # raises on non-finite values
        m1 = float(mass_host[0])
        kinds = gpu.kinds(st, wl.dt, wl.nsub)
        stored = "mx_column_prep" in kinds
        return {"value": job_value(nc * N * wl.nsub * steps, world, ms), "ms_per_step": ms / steps,
                "steps": steps, "warmup": warmup, "gpu_launches": kps * steps, "clocks": clk,
                "mass_rel_drift": abs(m1 - m0) / m0, "kinds": kinds,
                "mx_ops": MX_OPS["stored" if stored else "recompute"]}
    finally:
        C.icon_state_free(st)


def breakdown(kinds):
    tot = sum(v[0] for v in kinds.values())
    return {k: {"ms_per_step": round(v[0], 4), "share": round(v[0] / tot, 4)}
            for k, v in sorted(kinds.items(), key=lambda kv: -kv[1][0])}


def mixed_errors(gpu, grid, wl, seed=77):
    """Error of one mixed step against one FP64 step from the same initial state: rel L2 of
    vn, rho, theta_v, exner, and the RMS difference of w against the mixed bound."""
    C = gpu.C
    N = wl.nlev
    a = C.icon_state_init_ex(grid, seed, wl.case, noise_K=wl.noise_K, precision=0)
    try:
        C.icon_dycore_step(a, wl.dt, wl.nsub)
        ref = {f: C.icon_state_copy_field(a, grid, N, f) for f in ("vn", "rho", "theta_v", "exner", "w")}
    finally:
        C.icon_state_free(a)
    gpu.free_cache()
    b = C.icon_state_init_ex(grid, seed, wl.case, noise_K=wl.noise_K, precision=1)
    err = {}
    try:
        C.icon_dycore_step(b, wl.dt, wl.nsub)
        for f, x in ref.items():
            y = C.icon_state_copy_field(b, grid, N, f)
            if f == "w":
                err["w_rms"] = float(np.sqrt(np.mean((y - x) ** 2)))
            else:
                err[f] = float(np.linalg.norm(y - x) / np.linalg.norm(x))
            del y
    finally:
        C.icon_state_free(b)
    err["w_bound_mixed"] = 10.0 * EPS32 * GRAV * wl.dt        # 10 eps32 g dtau per substep, 1 step
    err["wind_bound"] = 1e-5
    return err


def e2e_rate(gpu, grid, wl, steps):
    """End to end through the C ABI with host buffers: every step copies the prognostic state
    from pinned host memory to the device, steps, integrates the mass and copies the state
    back (wall clock around the whole loop)."""
    C = gpu.C
    nc, ne, _ = counts(wl)
    N = wl.nlev
    st = C.icon_state_init_ex(grid, wl.seed, wl.case, noise_K=wl.noise_K, precision=wl.precision)
    try:
        host = {}
        for f in PROG:
            shape = (ne if f == "vn" else nc, N + 1 if f == "w" else N)
            host[f] = gpu.torch.empty(shape, dtype=gpu.torch.float64, pin_memory=True).numpy()
            C.icon_state_copy_field(st, grid, N, f, host[f])
        C.icon_dycore_step(st, wl.dt, wl.nsub)                     # records the graph
        h2d = sum(a.nbytes for a in host.values())
        gpu.torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(steps):
            for f in PROG:
                C.icon_state_set_field(st, grid, N, f, host[f])
            C.icon_dycore_step(st, wl.dt, wl.nsub)
            C.icon_global_mass(st)
            for f in PROG:
                C.icon_state_copy_field(st, grid, N, f, host[f])
        e2e_s = (time.perf_counter() - t0) / steps
    finally:
        C.icon_state_free(st)
    # the host link on its own: one pinned buffer of the state's size copied to the device and
    # back with plain copies (CUDA events), the floor of the end-to-end transfers
    torch = gpu.torch
    hb = torch.empty(h2d // 8, dtype=torch.float64, pin_memory=True)
    db = torch.empty(h2d // 8, dtype=torch.float64, device="cuda")
    db.copy_(hb, non_blocking=True)
    t_h2d = gpu.timed(lambda: db.copy_(hb, non_blocking=True))
    t_d2h = gpu.timed(lambda: hb.copy_(db, non_blocking=True))
    del hb, db
    return {"value": nc * N * wl.nsub / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": h2d + 8, "steps": steps, "ms_per_step": e2e_s * 1e3,
            "host_link": {"h2d_gbs": h2d / (t_h2d * 1e-3) / 1e9, "d2h_gbs": h2d / (t_d2h * 1e-3) / 1e9,
                          "how": "one pinned buffer of the state's size, torch copy_, CUDA events"}}


def leg(fn, *a, **k):
    """A leg of the JSON line: its measurements, or the reason it could not run."""
    C = sys.modules.get("paper_2511_02021_gb300.capi")
    try:
        return fn(*a, **k)
    except Exception as exc:          # a leg that cannot run (memory, a non-finite state) is reported
        if C is not None and isinstance(exc, C.IconError):
            return {"skipped": str(exc)}
        raise


# ---------------------------------------------------------------- GPU arm: the default line
def run_gpu(args, wl, rank, world, local_rank):
    gpu = Gpu(local_rank)
    C = gpu.C
    nc, ne, nv = counts(wl)
    N = wl.nlev
    hbm_peak, _ = peaks()
    gpu.torch.cuda.synchronize()
    t0 = time.perf_counter()
    grid = C.icon_grid_build(2, wl.bisections, N)
    setup = {"grid_build_ms": (time.perf_counter() - t0) * 1e3}
    t0 = time.perf_counter()
    C.icon_state_free(C.icon_state_init_ex(grid, wl.seed, wl.case, noise_K=wl.noise_K, precision=wl.precision))
    setup["state_init_ms"] = (time.perf_counter() - t0) * 1e3

    head = measure(gpu, grid, wl, wl.precision, args.steps, args.warmup, clocks=True, rank=rank, world=world)
    roof = dominant_roofline(gpu, wl, head["kinds"], hbm_peak, head["mx_ops"])
    roof["kernel_ms_per_step_sum"] = sum(v[0] for v in head["kinds"].values())
    roof["timed_ms_per_step"] = head["ms_per_step"]
    line = {"metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if wl.precision == 0 else "f32+f64",
            "data": "synthetic (analytic balanced jet, resident in HBM)", "config": gpu_config(wl, world),
            "gpu_launches": head["gpu_launches"], "roofline": roof,
            "hbm_roofline": step_hbm_roofline(head["value"], wl.precision, hbm_peak),
            "kernels": breakdown(head["kinds"]), "clocks": head["clocks"], "mass_rel_drift": head["mass_rel_drift"],
            "setup": setup, "fp64_peak": gpu.fp64_probe}
    line["e2e"] = leg(e2e_rate, gpu, grid, wl, max(1, min(args.steps, 5)))
    steps = wl.nsteps

    def variant(precision, **kw):
        r = measure(gpu, grid, wl, precision, steps, 2, clocks=True, rank=rank, world=world, **kw)
        out = {"value": r["value"], "unit": UNIT, "ms_per_step": r["ms_per_step"], "steps": steps,
               "gpu_launches": r["gpu_launches"], "mass_rel_drift": r["mass_rel_drift"], "clocks": r["clocks"],
               "kernels": breakdown(r["kinds"])}
        return out, r

    if wl.precision == 0 and not args.no_mixed:
        def mixed_leg():
            out, r = variant(1)
            out["roofline"] = dominant_roofline(gpu, wl, r["kinds"], hbm_peak, r["mx_ops"])
            out["hbm_roofline"] = step_hbm_roofline(r["value"], 1, hbm_peak)
            out["speedup_vs_fp64"] = r["value"] / head["value"]
            out["rel_l2_vs_fp64_after_1_step"] = mixed_errors(gpu, grid, wl)
            return out
        line["mixed"] = leg(mixed_leg)
    if not args.no_tracer:
        def tracer_leg():
            out, r = variant(wl.precision, ntracers=1)
            t_ms = r["kinds"]["tracer_transport"][0]
            ops = nc * N * TRACER_FP64_OPS
            out.update(tracers=1, ms_per_step_without=head["ms_per_step"], tracer_kernels_ms_per_step=t_ms,
                       roofline={"bound": "alu", "achieved": ops / (t_ms * 1e-3) / 1e9, "peak": gpu.fp64_peak / 1e9,
                                 "unit": "G FP64 instr/s", "frac": ops / (t_ms * 1e-3) / gpu.fp64_peak,
                                 "traffic": None, "peak_source": "measured (icon_probe_fp64_rate, FMA)"})
            return out
        line["tracer"] = leg(tracer_leg)

        def dd_leg():
            # the damping is part of the step (c4 = 0.0025); its cost against the undamped step,
            # and the fourth-order background diffusion on top of the default step
            out, r = variant(wl.precision, options=((C.ICON_OPT_DIVDAMP4, 0.0),))
            dd = head["kinds"].get("divergence_damping", (0.0, 0))[0]
            out = {"c4": 0.0025, "ms_per_step_with_it": head["ms_per_step"], "kernels_ms_per_step": dd,
                   "undamped": out}
            both, r2 = variant(wl.precision, options=((C.ICON_OPT_DIFF4, 0.005),))
            out["background_diffusion"] = {"c": 0.005, "ms_per_step_with_both": both["ms_per_step"],
                                           "kernels_ms_per_step": r2["kinds"]["background_diffusion"][0]}
            return out
        line["divergence_damping"] = leg(dd_leg)
        if wl.precision == 0:
            def topo_leg():
                out, r = variant(0, topo=(1500.0, 800e3))
                out.update(height_m=1500.0, radius_m=800e3, ms_per_step_flat=head["ms_per_step"])
                out["mixed"], _ = variant(1, topo=(1500.0, 800e3))
                return out
            line["topography"] = leg(topo_leg)
    C.icon_grid_free(grid)
    gpu.free_cache()

    if not args.quick and wl.name == WL.R2B6_JET.name:
        line["r2b8_l90"] = leg(large_leg, gpu, WL.R2B8_JET_MIXED, hbm_peak, rank, world, compare_fp64=True)
        gpu.free_cache()
        line["r2b9_l60_mixed"] = leg(large_leg, gpu, WL.R2B9_JET_MIXED, hbm_peak, rank, world, compare_fp64=False)
        gpu.free_cache()
        line["ensemble"] = leg(ensemble_leg, gpu, hbm_peak, rank, world, WL.ENSEMBLE["nsteps"], 2)
        gpu.free_cache()
    line["device_memory_gb"] = {"peak_allocated": round(gpu.torch.cuda.max_memory_allocated() / 1e9, 2),
                                "total": round(gpu.torch.cuda.get_device_properties(0).total_memory / 1e9, 2)}
    if rank != 0:
        return
    line["cpu_baseline"] = None
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(wl)
    print(json.dumps(line), flush=True)


def large_leg(gpu, wl, hbm_peak, rank, world, compare_fp64):
    """One of the large configurations from fresh states: the mixed form (and the FP64 form
    with the mixed form's error against it when asked), each with clocks and roofline."""
    C = gpu.C
    nc, ne, _ = counts(wl)
    t0 = time.perf_counter()
    grid = C.icon_grid_build(2, wl.bisections, wl.nlev)
    out = {"config": gpu_config(wl, world), "grid_build_ms": (time.perf_counter() - t0) * 1e3}
    try:
        r = measure(gpu, grid, wl, 1, wl.nsteps, 1, clocks=True, rank=rank, world=world)
        mixed = {"value": r["value"], "unit": UNIT, "ms_per_step": r["ms_per_step"], "steps": wl.nsteps,
                 "gpu_launches": r["gpu_launches"], "mass_rel_drift": r["mass_rel_drift"], "clocks": r["clocks"],
                 "roofline": dominant_roofline(gpu, wl, r["kinds"], hbm_peak, r["mx_ops"]),
                 "hbm_roofline": step_hbm_roofline(r["value"], 1, hbm_peak), "kernels": breakdown(r["kinds"])}
        out["mixed"] = mixed
        gpu.free_cache()
        if compare_fp64:
            r64 = measure(gpu, grid, wl, 0, wl.nsteps, 1, clocks=True, rank=rank, world=world)
            out["fp64"] = {"value": r64["value"], "unit": UNIT, "ms_per_step": r64["ms_per_step"],
                           "steps": wl.nsteps, "gpu_launches": r64["gpu_launches"],
                           "mass_rel_drift": r64["mass_rel_drift"], "clocks": r64["clocks"],
                           "roofline": dominant_roofline(gpu, wl, r64["kinds"], hbm_peak, r64["mx_ops"]),
                           "hbm_roofline": step_hbm_roofline(r64["value"], 0, hbm_peak),
                           "kernels": breakdown(r64["kinds"])}
            mixed["speedup_vs_fp64"] = r["value"] / r64["value"]
            gpu.free_cache()
            mixed["error_vs_fp64_after_1_step"] = mixed_errors(gpu, grid, wl)
        else:
            # simulated days per wall-clock day of the dycore alone, from the timed steps; the
            # step's stability over a simulated day is shown by the one-day runs of the tests
            mixed["simulated_days_per_day"] = wl.dt / (r["ms_per_step"] * 1e-3)
    finally:
        C.icon_grid_free(grid)
    return out


def ensemble_leg(gpu, hbm_peak, rank, world, steps, warmup):
    """64 members (32 on R2B4 with dt 360 s, 32 on R2B5 with dt 180 s), 60 levels, mixed
    precision, member perturbations from seed 3: one persistent cooperative launch per
    step for all members, against the same members stepped one after another (each
    from its own recorded graph)."""
    C = gpu.C
    E = WL.ENSEMBLE
    N, nsub = E["nlev"], E["nsub"]
    grids = {4: C.icon_grid_build(2, 4, N), 5: C.icon_grid_build(2, 5, N)}
    spec = [(4, E["dt_b4"])] * E["members_b4"] + [(5, E["dt_b5"])] * E["members_b5"]
    cells = sum(counts_of(b)[0] for b, _ in spec)
    dts = [dt for _, dt in spec]
    dist = world > 1

    def make_states():
        return [C.icon_state_init_ex(grids[b], E["seed"] + 1000 * rank, C.ICON_CASE_MEMBER, precision=1, member=m)
                for m, (b, _) in enumerate(spec)]

    def timed(fn):
        if dist:
            import torch.distributed as td
            td.barrier()
        ms = gpu.timed(fn)
        if dist:
            td.barrier()
            ms = max_over_ranks(ms, "cuda")
        return ms

    try:
        sts = make_states()
        ens = C.icon_ensemble_create(sts)
        try:
            C.icon_ensemble_step(ens, dts, nsub, warmup)
            clk = ClockSampler(gpu.local_rank) if rank == 0 else None
            arr = (C.ctypes.c_double * len(dts))(*dts)
            ms_b = timed(lambda: C._check(C._lib.icon_ensemble_step(ens, arr, nsub, steps)))
            clk = clk.stop() if clk else None
            # after the timed region: one step with the phase timer (block 0 stamps the
            # global timer at every grid barrier), the breakdown of the persistent launch
            pms, pcnt = C.icon_ensemble_step_profile(ens, dts, nsub)
            phases = {C.icon_ensemble_phase_name(k): {"ms_per_step": round(float(pms[k]), 3),
                                                      "barriers_per_step": int(pcnt[k])}
                      for k in range(C.ICON_ENS_PHASE_COUNT) if pcnt[k]}
        finally:
            C.icon_ensemble_free(ens)
            for st in sts:
                C.icon_state_free(st)
        sts = make_states()
        try:
            for st, dt in zip(sts, dts):
                for _ in range(warmup):
                    C.icon_dycore_step(st, dt, nsub)

            def seq():
                for _ in range(steps):
                    for st, dt in zip(sts, dts):
                        C.icon_dycore_step_async(st, dt, nsub)
            ms_s = timed(seq)
            for st in sts:
                C.icon_state_status(st)
            launches_seq = sum(C.icon_state_step_kernels(st, dt, nsub) for st, dt in zip(sts, dts))
        finally:
            for st in sts:
                C.icon_state_free(st)
    finally:
        for g in grids.values():
            C.icon_grid_free(g)
    value_b = job_value(cells * N * nsub * steps, world, ms_b)
    value_s = job_value(cells * N * nsub * steps, world, ms_s)
    t_launch = ms_b / steps * 1e-3
    alg_bytes = 239.0 * cells * N * nsub
    alg_ops = (2 * MX_OPS["stored"] + 2.0) * cells * N * nsub
    hbm_frac = alg_bytes / t_launch / 1e9 / hbm_peak
    alu_frac = alg_ops / t_launch / gpu.fp64_peak
    roof = {"kernel": "ensemble_persistent", "bound": "alu" if alu_frac > hbm_frac else "hbm",
            "achieved": alg_ops / t_launch / 1e9 if alu_frac > hbm_frac else alg_bytes / t_launch / 1e9,
            "peak": gpu.fp64_peak / 1e9 if alu_frac > hbm_frac else hbm_peak,
            "unit": "G FP64 instr/s" if alu_frac > hbm_frac else "GB/s",
            "frac": max(alu_frac, hbm_frac), "traffic": None, "hbm_frac": hbm_frac, "fp64_frac": alu_frac,
            "launch_ms": ms_b / steps, "launches_per_step": 1}
    return {"workload": "ensemble-32xR2B4+32xR2B5-L60-mixed", "members": len(spec), "cells": cells, "levels": N,
            "nsub": nsub, "dt": {"R2B4": E["dt_b4"], "R2B5": E["dt_b5"]}, "steps": steps,
            "value": value_b, "unit": UNIT, "ms_per_step": ms_b / steps, "gpu_launches": 2 * steps,
            "roofline": roof, "clocks": clk, "hbm_roofline": step_hbm_roofline(value_b, 1, hbm_peak),
            "sequential": {"value": value_s, "unit": UNIT, "ms_per_step": ms_s / steps,
                           "gpu_launches_per_step": launches_seq},
            "batched_speedup_vs_sequential": value_b / value_s,
            "phases": phases}


def run_single(args, wl, rank, world, local_rank):
    """One of the large workloads alone (--workload r2b8-mixed | r2b9-mixed | ensemble)."""
    gpu = Gpu(local_rank)
    hbm_peak, _ = peaks()
    if wl is None:
        res = ensemble_leg(gpu, hbm_peak, rank, world, args.steps, args.warmup)
        value, ms, clk, launches = res["value"], res["ms_per_step"], res["clocks"], res["gpu_launches"]
        cfg = {"workload": res["workload"], "members": res["members"], "cells": res["cells"], "levels": res["levels"],
               "nsub": res["nsub"], "dt": res["dt"], "l2": "inputs larger than L2 (64 member states)"}
        roof = res["roofline"]
    else:
        res = large_leg(gpu, wl, hbm_peak, rank, world, compare_fp64=not args.no_mixed and wl.bisections <= 8)
        m = res["mixed"]
        value, ms, clk, launches, roof = m["value"], m["ms_per_step"], m["clocks"], m["gpu_launches"], m["roofline"]
        cfg = res["config"]
    if rank != 0:
        return
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": res.get("steps", args.steps),
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic (analytic balanced jet, resident in HBM)",
            "config": cfg, "gpu_launches": launches, "roofline": roof, "clocks": clk, "detail": res,
            "fp64_peak": gpu.fp64_probe, "cpu_baseline": None, "e2e": None}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- profiling mode
def profile_step(argv):
    """One small workload for kernel profilers: BISECTIONS NLEV PRECISION [NSTEPS [NTRACERS
    [TOPO_M]]]: the jet with 0.1 K noise on R2B<BISECTIONS> with NLEV levels (over a Gaussian
    mountain of TOPO_M metres, radius 800 km, when TOPO_M > 0), NTRACERS tracers, NSTEPS steps
    of 180 s in 5 substeps."""
    bis, nlev, prec = int(argv[0]), int(argv[1]), int(argv[2])
    nsteps = int(argv[3]) if len(argv) > 3 else 1
    ntr = int(argv[4]) if len(argv) > 4 else 0
    topo = float(argv[5]) if len(argv) > 5 else 0.0
    gpu = Gpu(0, probe=False)
    C = gpu.C
    g = C.icon_grid_build(2, bis, nlev)
    s = C.icon_state_init_ex(g, 2, C.ICON_CASE_JET, noise_K=0.1, precision=prec, topo_height_m=topo,
                             topo_radius_m=800e3 if topo > 0 else 0.0)
    if ntr:
        C.icon_state_add_tracers(s, ntr)
        xc = C.icon_grid_copy_table(g, "x_c")
        for t in range(ntr):
            C.icon_state_set_tracer(s, g, nlev, t, np.repeat(1.0 + 0.5 * xc[:, 2:3], nlev, axis=1))
    for _ in range(nsteps):
        C.icon_dycore_step(s, 180.0, 5)
    C.icon_state_free(s)
    C.icon_grid_free(g)
    print("ok")


def main():
    if len(sys.argv) > 1 and sys.argv[1] == "--profile-step":
        profile_step(sys.argv[2:])
        return
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gpu", "reference"], default="gpu")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="r2b6-fp64")
    ap.add_argument("--quick", action="store_true", help="skip the R2B8, R2B9 and ensemble measurements")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mixed", action="store_true", help="skip the mixed-precision variant of an FP64 workload")
    ap.add_argument("--no-tracer", action="store_true",
                    help="skip the tracer, option and terrain measurements")
    args = ap.parse_args()
    wl = WORKLOADS[args.workload]
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, wl if wl is not None else WL.R2B6_JET, rank)
        return
    if world > 1:
        import torch
        import torch.distributed as td
        torch.cuda.set_device(local_rank)
        td.init_process_group("nccl")
    if wl is WL.R2B6_JET:
        run_gpu(args, wl, rank, world, local_rank)
    else:
        run_single(args, wl, rank, world, local_rank)
    if world > 1:
        import torch.distributed as td
        td.destroy_process_group()


if __name__ == "__main__":
    main()
