#!/usr/bin/env python
"""Throughput benchmark of the dynamical-core hot path on one GB300 (or N replicas).

One benchmark step = one dycore step (nsub predictor-corrector substeps with the
vertically implicit column solve, then Smagorinsky diffusion) followed by the
global mass integral, on a synthetic analytic state resident in HBM. Metric:
cell-level updates per second = cells x levels x substeps / time.

Default workload: the R2B6 grid (327,680 cells, 491,520 edges) with 90 levels on
a stretched height coordinate to 75 km, FP64, balanced 35 m/s jet with a 1 m/s
Gaussian bump, dt = 90 s in 5 substeps, 10 steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gpu|reference]
                  [--workload r2b6-fp64|r2b8-mixed|r2b9-mixed]

Under torchrun (N > 1) every rank advances its own replica (no data exchange:
"scaling": "weak"); rank 0 prints the JSON line with the max time over ranks.
--impl reference times the FP64 CPU oracle on the host cores instead (rank 0 only).
"""
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

from paper_2511_02021_gb300 import workloads as WL  # noqa: E402

METRIC = "cell-level updates/s per dycore substep, % HBM roofline; mixed vs FP64"
UNIT = "cell-level updates/s"
WORKLOADS = {"r2b6-fp64": WL.R2B6_JET, "r2b8-mixed": WL.R2B8_JET_MIXED, "r2b9-mixed": WL.R2B9_JET_MIXED,
             "ensemble": None}
PROG = ("vn", "w", "rho", "theta_v", "exner")


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


# Peak FP64 instruction rate of the GB300, from its unit counts and clock: 152 SMs x 2 FP64
# operations per SM per cycle (a fused multiply-add is one) x 2.07 GHz = 629 G/s; NVIDIA's
# nominal 1.25 TFLOP/s counts an FMA as two. ncu's "FP64 pipe active" percentages are
# relative to the same rate. An FMA/ADD throughput probe of this machine sustained 505 G/s.
FP64_INSTR_PEAK = 152 * 2 * 2.07e9
# FP64 instructions per cell-level of one launch of the column solves (a fused multiply-add
# is one, the Newton-Raphson reciprocal three), averaged over predictor and corrector,
# counted from the kernel source and checked against ncu's executed counts
# (profiles/ncu_fp64_column_edge_r2b6_l90.md, profiles/ncu_mixed_column_stencils_r2b6_l90.md).
# FP64 step: rows kernel 28 (explicit predictors, linearised state equation) + 5 (half-level
# interpolants) + 23 (w predictor and tridiagonal row), Thomas 9, update 11 (corrector 15);
# executed 70.8 (predictor) and 75.8 (corrector).
COLUMN_FP64_OPS = 73
# mixed step with stored factors: predictor 42 (one downward sweep forming and factoring
# the rows, 39; the upward back substitution and damping, 3, with the provisional state's
# FP32 shadows formed in FP32), corrector 28 (right-hand side, substitution, FP64 updates,
# vertical mass flux); executed 42.7 and 29.9.
MX_COLUMN_FP64_OPS = 36
# mixed step recomputing the factors in both stages (when the stored factors would exceed a
# quarter of the device memory): executed 47.5 (predictor) and 64.5 (corrector).
MX_COLUMN_RECOMPUTE_FP64_OPS = 56
# FP64 instructions per cell-level of the tracer transport of one tracer: cell kernel
# (least-squares gradient 12, vertical slope, departure point and flux 12), edge kernel
# (27 per edge-level, 1.5 edges per cell), update (12); executed (ncu, R2B6/90): 24.2,
# 41.0 and 12.0 (profiles/ncu_tracer_r2b6_l90.md).
TRACER_FP64_OPS = 77
# DRAM bytes (read + write) per launch of the dominant kernel kind, from ncu captures of the
# current kernels (mean of predictor and corrector; same files): FP64 column at R2B6/90
# measured; mixed column at R2B6/90 measured and scaled by cells to R2B8/90; recomputing
# mixed column measured at R2B5/60 and scaled by cells to R2B9/60.
NCU_TRAFFIC = {
    ("R2B6-L90-jet-fp64", "column_solve"): 10.60e9,
    ("R2B6-L90-jet-fp64", "mx_column_solve"): 7.82e9,
    ("R2B8-L90-jet-mixed", "mx_column_solve"): 7.82e9 * 16,
    ("R2B9-L60-jet-mixed", "mx_column_solve"): 1.627e9 * 256,
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
            "frac": value * b / 1e9 / hbm_peak}


def counts(wl):
    L = wl.bisections + 1
    nc, ne, nv = 20 * 4 ** L, 30 * 4 ** L, 10 * 4 ** L + 2
    return nc, ne, nv


def kernel_model(kind, wl, stored_factors=True):
    """(algorithmic bytes, FP64 arithmetic ops) of ONE launch of a kernel kind, averaged
    over predictor and corrector launches: every input and output array element read
    or written once (8 B in FP64), and the FP64 operations of the expressions as
    written (a division counted as one operation)."""
    nc, ne, nv = counts(wl)
    N = wl.nlev
    H = N + 1
    b = 8.0
    table = {
        "vertex_curl_wmean": (b * (ne * N + nc * H + nv * N + nv * H), nv * N * 6 + nv * H * 7),
        "edge_vt_ke": (b * 3 * ne * N, ne * N * 8),
        "cell_ke": (b * (ne + nc) * N, nc * N * 3),
        "edge_tendency_flux": (b * (ne * N * 6.5 + nc * N * 4 + nv * N + nc * H + nv * H + ne * H),
                               ne * N * 23 + ne * H * 11),
        "column_solve": (b * (nc * N * 8 + ne * N * 2 + ne * H + nc * H * 2.5), nc * N * COLUMN_FP64_OPS),
        "diff_vertex": (b * (ne * N + 4 * nv * N), nv * N * 25),
        "diff_div": (b * (ne + nc) * N, nc * N * 7),
        "diff_edge": (b * (ne * N * 4 + nv * N * 5 + nc * N * 2), ne * N * 45),
        "diff_theta": (b * (ne * N + 4 * nc * N), nc * N * 12),
        "global_mass": (b * nc * N, nc * N * 2),
        # mixed precision: FP32 stencil arrays (4 B), FP64 level-major prognostics (8 B)
        "mx_vertex": (4.0 * (ne * N + nc * H + nv * N + nv * H), 0),
        "mx_edge_diag": (4.0 * 3 * ne * N, 0),
        "mx_cell_ke": (4.0 * (ne + nc) * N, 0),
        "mx_edge_tendency_flux": (4.0 * (ne * N * 6.5 + ne * H + nc * N * 4 + nv * N + nc * H + nv * H)
                                  + 8.0 * ne * N, ne * N * 1.0),
        "mx_column_solve": (nc * N * 98.0, nc * N * (MX_COLUMN_FP64_OPS if stored_factors
                                                     else MX_COLUMN_RECOMPUTE_FP64_OPS)),
        "mx_column_prep": (4.0 * (3 * ne * N + ne * H + nc * H * 3) + 8.0 * (nc * N * 3 + nc * H), nc * N * 3),
        "mx_diff_vertex": (4.0 * (2 * ne * N + 4 * nv * N + nc * N), 0),
        "mx_diff_edge": (4.0 * (ne * N * 4 + nv * N * 3 + nc * N * 2), 0),
        "mx_diff_theta": (4.0 * ne * N + 40.0 * nc * N, nc * N * 6),
    }
    return table.get(kind)


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi sampled every 200 ms during the timed region."""
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


# ---------------------------------------------------------------- reference arm (oracle on host cores)
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
        el = time.perf_counter() - t0
        return g.nc * v.N / el, el, "one substep (predictor + corrector) of %s, init excluded" % wl.name


def run_reference(args, wl, rank):
    if rank != 0:
        return
    # the oracle is plain numpy: its array operations run on one host core
    vals = []
    smp = OracleSampler(wl)
    for i in range(args.warmup + args.steps):
        v, el, desc = smp.sample()
        if i >= args.warmup:
            vals.append(el)
    t = sum(vals) / len(vals)
    nc, _, _ = counts(wl)
    value = nc * wl.nlev / t
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl.name, "cells": nc, "levels": wl.nlev, "dt": wl.dt, "nsub": wl.nsub,
                       "sample": "each step = one substep of the workload"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- GPU arm
def run_gpu(args, wl, rank, world, local_rank):
    import torch
    torch.cuda.set_device(local_rank)
    from paper_2511_02021_gb300 import build as B
    B.build()
    import paper_2511_02021_gb300 as P
    from paper_2511_02021_gb300 import capi as C
    P.use_torch_allocator(local_rank)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    P.bind_torch_stream(stream)
    dist = world > 1
    if dist:
        import torch.distributed as td

    nc, ne, nv = counts(wl)
    N = wl.nlev
    # one-time setup, wall clock (untimed by the step metric): grid build (connectivity,
    # geometry, weights on the device) and the initial state of the measured precision
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    grid = C.icon_grid_build(2, wl.bisections, N)
    setup = {"grid_build_ms": (time.perf_counter() - t0) * 1e3}
    t0 = time.perf_counter()
    C.icon_state_free(C.icon_state_init_ex(grid, wl.seed, wl.case, noise_K=wl.noise_K, precision=wl.precision))
    setup["state_init_ms"] = (time.perf_counter() - t0) * 1e3
    hbm_peak, peak_src = peaks()

    def measure(precision, sample_clocks):
        """Time K steps (+ mass) of one precision; returns the state and the measurements."""
        st = C.icon_state_init_ex(grid, wl.seed + rank, wl.case, noise_K=wl.noise_K, precision=precision)
        m0 = C.icon_global_mass(st)
        for _ in range(args.warmup):
            C.icon_dycore_step(st, wl.dt, wl.nsub)
        kps = C.icon_state_step_kernels(st, wl.dt, wl.nsub) + 2      # + the mass integral
        mass_host = torch.empty(1, dtype=torch.float64, pin_memory=True)
        clocks = ClockSampler(local_rank) if (rank == 0 and sample_clocks) else None
        time.sleep(0.4)
        if dist:
            td.barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            C.icon_dycore_step_async(st, wl.dt, wl.nsub)
            C.icon_global_mass_async(st, mass_host.data_ptr())
        e1.record(stream)
        torch.cuda.synchronize()
        if dist:
            td.barrier()
        ms = e0.elapsed_time(e1)
        clk = clocks.stop() if clocks else None
        C.icon_state_status(st)                               # raises on non-finite values
        m1 = float(mass_host[0])
        if dist:
            ms = max_over_ranks(ms, "cuda")
        value = job_value(nc * N * wl.nsub * args.steps, world, ms)
        # per-kernel durations, measured live with CUDA events around every launch
        kms, kn = None, None
        for _ in range(2):
            kms, kn = C.icon_dycore_step_profile(st, wl.dt, wl.nsub, kms, kn)
        rows = []
        # the mixed column with stored factors is the one that launches the gather kernel
        names = [C.icon_kernel_kind_name(k) for k in range(C.ICON_KIND_COUNT)]
        stored = kn[names.index("mx_column_prep")] > 0
        for k in range(C.ICON_KIND_COUNT):
            if kn[k] == 0:
                continue
            name = names[k]
            avg = kms[k] / kn[k]
            model = kernel_model(name, wl, stored)
            gbs = model[0] / (avg * 1e-3) / 1e9 if model else None
            fops = model[1] / (avg * 1e-3) if model else None
            rows.append((kms[k] / 2, name, avg, int(kn[k] // 2), gbs, fops))
        rows.sort(reverse=True)
        top = rows[0]
        hbm_frac = top[4] / hbm_peak if top[4] else None
        alu_frac = top[5] / FP64_INSTR_PEAK if top[5] else None
        if alu_frac is not None and hbm_frac is not None and alu_frac > hbm_frac:
            roof = {"kernel": top[1], "bound": "alu", "achieved": top[5] / 1e9, "peak": FP64_INSTR_PEAK / 1e9,
                    "unit": "G FP64 instr/s", "frac": alu_frac, "traffic": NCU_TRAFFIC.get((wl.name, top[1])),
                    "peak_source": "derived: 152 SMs x 2 FP64/cycle x 2.07 GHz",
                    "hbm": {"achieved": top[4], "peak": hbm_peak, "unit": "GB/s", "frac": hbm_frac,
                            "peak_source": peak_src},
                    "launch_ms": top[2], "launches_per_step": top[3]}
        else:
            roof = {"kernel": top[1], "bound": "hbm", "achieved": top[4], "peak": hbm_peak, "unit": "GB/s",
                    "frac": hbm_frac, "traffic": NCU_TRAFFIC.get((wl.name, top[1])), "peak_source": peak_src,
                    "launch_ms": top[2],
                    "launches_per_step": top[3],
                    "fp64": {"achieved": (top[5] or 0) / 1e9, "peak": FP64_INSTR_PEAK / 1e9,
                             "unit": "G FP64 instr/s", "frac": alu_frac}}
        tot = sum(x[0] for x in rows)
        breakdown = {r[1]: {"ms_per_step": round(r[0], 4), "share": round(r[0] / tot, 4)} for r in rows}
        # the per-kind durations come from two eager steps right after the timed region, on the
        # same stream: their sum against the timed step says how much time lies between kernels
        roof["kernel_ms_per_step_sum"] = tot
        roof["timed_ms_per_step"] = ms / args.steps
        return st, {"value": value, "ms": ms, "kps": kps, "roof": roof, "breakdown": breakdown, "clocks": clk,
                    "mass_rel_drift": abs(m1 - m0) / m0}

    st, res = measure(wl.precision, True)
    value, ms, roof, breakdown, clk = res["value"], res["ms"], res["roof"], res["breakdown"], res["clocks"]
    kernels_per_step = res["kps"]

    # mixed vs FP64 on the same workload: throughput, and the error of one mixed step
    other = None
    if wl.precision == 0 and not args.no_mixed:
        st_m, res_m = measure(1, False)
        C.icon_state_free(st_m)
        a = C.icon_state_init_ex(grid, 77, wl.case, noise_K=wl.noise_K, precision=0)
        b = C.icon_state_init_ex(grid, 77, wl.case, noise_K=wl.noise_K, precision=1)
        C.icon_dycore_step(a, wl.dt, wl.nsub)
        C.icon_dycore_step(b, wl.dt, wl.nsub)
        err = {}
        for f in ("vn", "rho", "theta_v", "exner", "w"):
            x = C.icon_state_copy_field(a, grid, N, f)
            y = C.icon_state_copy_field(b, grid, N, f)
            err[f] = float(np.linalg.norm(y - x) / np.linalg.norm(x))
        C.icon_state_free(a)
        C.icon_state_free(b)
        other = {"precision": "mixed (FP32 stencils, FP64 column solve and prognostics)",
                 "value": res_m["value"], "unit": UNIT, "ms_per_step": res_m["ms"] / args.steps,
                 "speedup_vs_fp64": res_m["value"] / value, "rel_l2_vs_fp64_after_1_step": err,
                 "mass_rel_drift": res_m["mass_rel_drift"], "roofline": res_m["roof"],
                 "kernels": res_m["breakdown"], "gpu_launches": res_m["kps"] * args.steps,
                 "hbm_roofline": step_hbm_roofline(res_m["value"], 1, hbm_peak)}
    m_drift = res["mass_rel_drift"]
    err_vs_fp64 = None
    if wl.precision == 1 and not args.no_mixed:
        # error of one mixed step against one FP64 step from the same state (wind)
        C.icon_state_free(st)
        st = None
        try:
            a = C.icon_state_init_ex(grid, 77, wl.case, noise_K=wl.noise_K, precision=0)
        except C.IconError as ex:
            a = None
            err_vs_fp64 = {"skipped": "an FP64 state of this grid does not fit in device memory (%s)" % ex}
        if a is not None:
            C.icon_dycore_step(a, wl.dt, wl.nsub)
            ref = {f: C.icon_state_copy_field(a, grid, N, f) for f in ("vn", "exner")}
            C.icon_state_free(a)
            b = C.icon_state_init_ex(grid, 77, wl.case, noise_K=wl.noise_K, precision=1)
            C.icon_dycore_step(b, wl.dt, wl.nsub)
            err_vs_fp64 = {}
            for f, x in ref.items():
                y = C.icon_state_copy_field(b, grid, N, f)
                err_vs_fp64[f] = float(np.linalg.norm(y - x) / np.linalg.norm(x))
                del y
            del ref
            st = b
        else:
            st = C.icon_state_init_ex(grid, wl.seed, wl.case, noise_K=wl.noise_K, precision=wl.precision)

    # end to end through the C ABI with host buffers: h2d of the prognostic state,
    # the step, the mass integral and d2h of the updated state, every step
    host = {}
    for f in PROG:
        shape = (ne if f == "vn" else nc, N + 1 if f == "w" else N)
        host[f] = torch.empty(shape, dtype=torch.float64, pin_memory=True).numpy()
        C.icon_state_copy_field(st, grid, N, f, host[f])
    h2d = sum(a.nbytes for a in host.values())
    e2e_steps = max(1, min(args.steps, 3))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        for f in PROG:
            C.icon_state_set_field(st, grid, N, f, host[f])
        C.icon_dycore_step(st, wl.dt, wl.nsub)
        C.icon_global_mass(st)
        for f in PROG:
            C.icon_state_copy_field(st, grid, N, f, host[f])
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    e2e = {"value": nc * N * wl.nsub / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d,
           "d2h_bytes_per_step": h2d + 8}

    # tracer transport (one tracer, same workload and precision), on the state the
    # end-to-end loop used: its kernel time per step from the profiled eager steps, and
    # the step time with it from timed graph replays
    tracer = None
    if not args.no_tracer:
        try:
            C.icon_state_add_tracers(st, 1)
            xc = C.icon_grid_copy_table(grid, "x_c")
            C.icon_state_set_tracer(st, grid, N, 0, np.repeat(1.0 + 0.5 * xc[:, 2:3], N, axis=1))
            for _ in range(args.warmup):
                C.icon_dycore_step(st, wl.dt, wl.nsub)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(args.steps):
                C.icon_dycore_step_async(st, wl.dt, wl.nsub)
            e1.record(stream)
            torch.cuda.synchronize()
            C.icon_state_status(st)
            ms_t = e0.elapsed_time(e1) / args.steps
            kms, kn = None, None
            for _ in range(2):
                kms, kn = C.icon_dycore_step_profile(st, wl.dt, wl.nsub, kms, kn)
            names = [C.icon_kernel_kind_name(k) for k in range(C.ICON_KIND_COUNT)]
            t_ms = kms[names.index("tracer_transport")] / 2
            ops = nc * N * TRACER_FP64_OPS
            tracer = {"tracers": 1, "ms_per_step_with_tracer": ms_t, "ms_per_step_without": ms / args.steps,
                      "tracer_kernels_ms_per_step": t_ms,
                      "roofline": {"bound": "alu", "achieved": ops / (t_ms * 1e-3) / 1e9,
                                   "peak": FP64_INSTR_PEAK / 1e9, "unit": "G FP64 instr/s",
                                   "frac": ops / (t_ms * 1e-3) / FP64_INSTR_PEAK, "traffic": None}}
        except C.IconError as exc:
            tracer = {"skipped": str(exc)}
    # the divergence-damping option (c4 = 0.004) on the same state: step time with it, and
    # its kernels' time per step from the profiled eager steps
    divdamp = None
    if not args.no_tracer:
        try:
            C.icon_state_set_option(st, C.ICON_OPT_DIVDAMP4, 0.004)
            for _ in range(args.warmup):
                C.icon_dycore_step(st, wl.dt, wl.nsub)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(args.steps):
                C.icon_dycore_step_async(st, wl.dt, wl.nsub)
            e1.record(stream)
            torch.cuda.synchronize()
            C.icon_state_status(st)
            ms_d = e0.elapsed_time(e1) / args.steps
            kms, kn = None, None
            for _ in range(2):
                kms, kn = C.icon_dycore_step_profile(st, wl.dt, wl.nsub, kms, kn)
            names = [C.icon_kernel_kind_name(k) for k in range(C.ICON_KIND_COUNT)]
            divdamp = {"c4": 0.004, "ms_per_step_with_it": ms_d,
                       "kernels_ms_per_step": kms[names.index("divergence_damping")] / 2,
                       "note": "on the state of the tracer measurement (one tracer transported)"}
            # and the fourth-order background diffusion on top (c = 0.005)
            C.icon_state_set_option(st, C.ICON_OPT_DIFF4, 0.005)
            for _ in range(args.warmup):
                C.icon_dycore_step(st, wl.dt, wl.nsub)
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(args.steps):
                C.icon_dycore_step_async(st, wl.dt, wl.nsub)
            e1.record(stream)
            torch.cuda.synchronize()
            C.icon_state_status(st)
            kms, kn = None, None
            for _ in range(2):
                kms, kn = C.icon_dycore_step_profile(st, wl.dt, wl.nsub, kms, kn)
            divdamp["background_diffusion"] = {
                "c": 0.005, "ms_per_step_with_both": e0.elapsed_time(e1) / args.steps,
                "kernels_ms_per_step": kms[names.index("background_diffusion")] / 2}
        except C.IconError as exc:
            divdamp = {"skipped": str(exc)}

    C.icon_state_free(st)
    # the same workload on terrain-following levels over a Gaussian mountain (1500 m,
    # e-folding radius 800 km at 90E 30N; FP64 form only): timed graph replays, the kernel
    # time per kind from two profiled eager steps, and the mass drift
    topo = None
    if not args.no_tracer and wl.precision == 0:
        try:
            st = C.icon_state_init_ex(grid, wl.seed, wl.case, noise_K=wl.noise_K, topo_height_m=1500.0,
                                      topo_radius_m=800e3)
            try:
                tm0 = C.icon_global_mass(st)
                for _ in range(args.warmup):
                    C.icon_dycore_step(st, wl.dt, wl.nsub)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(args.steps):
                    C.icon_dycore_step_async(st, wl.dt, wl.nsub)
                e1.record(stream)
                torch.cuda.synchronize()
                C.icon_state_status(st)
                ms_topo = e0.elapsed_time(e1) / args.steps
                kms, kn = None, None
                for _ in range(2):
                    kms, kn = C.icon_dycore_step_profile(st, wl.dt, wl.nsub, kms, kn)
                names = [C.icon_kernel_kind_name(k) for k in range(C.ICON_KIND_COUNT)]
                tm1 = C.icon_global_mass(st)
                topo = {"height_m": 1500.0, "radius_m": 800e3, "value": nc * N * wl.nsub / (ms_topo * 1e-3),
                        "unit": UNIT, "ms_per_step": ms_topo, "ms_per_step_flat": ms / args.steps,
                        "kernels_ms_per_step": {n: round(kms[i] / 2, 4) for i, n in enumerate(names)
                                                if n and kn[i] > 0},
                        "mass_rel_drift": abs(tm1 - tm0) / tm0}
            finally:
                C.icon_state_free(st)
            # the mixed form on the same levels (its column recomputes its factors there)
            st = C.icon_state_init_ex(grid, wl.seed, wl.case, noise_K=wl.noise_K, precision=1,
                                      topo_height_m=1500.0, topo_radius_m=800e3)
            try:
                for _ in range(args.warmup):
                    C.icon_dycore_step(st, wl.dt, wl.nsub)
                torch.cuda.synchronize()
                e0.record(stream)
                for _ in range(args.steps):
                    C.icon_dycore_step_async(st, wl.dt, wl.nsub)
                e1.record(stream)
                torch.cuda.synchronize()
                C.icon_state_status(st)
                ms_tm = e0.elapsed_time(e1) / args.steps
                kms, kn = None, None
                for _ in range(2):
                    kms, kn = C.icon_dycore_step_profile(st, wl.dt, wl.nsub, kms, kn)
                topo["mixed"] = {"value": nc * N * wl.nsub / (ms_tm * 1e-3), "unit": UNIT, "ms_per_step": ms_tm,
                                 "kernels_ms_per_step": {n: round(kms[i] / 2, 4) for i, n in enumerate(names)
                                                         if n and kn[i] > 0}}
            finally:
                C.icon_state_free(st)
        except C.IconError as exc:
            topo = {"skipped": str(exc)}
    C.icon_grid_free(grid)
    if rank != 0:
        return
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        v, el, desc = OracleSampler(wl).sample()
        cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc, "seconds": el}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if wl.precision == 0 else "f32+f64",
            "data": "synthetic (analytic balanced jet, resident in HBM)",
            "config": {"workload": wl.name, "grid": "R2B%d" % wl.bisections, "cells": nc, "edges": ne,
                       "levels": N, "dt": wl.dt, "nsub": wl.nsub, "precision": "fp64" if wl.precision == 0
                       else "mixed", "parallelism": "replicas" if world > 1 else "single",
                       "l2": "inputs larger than L2 (state %.2f GB)" % ((ne * N + 4 * nc * N) * 8 / 1e9)},
            "gpu_launches": kernels_per_step * args.steps, "roofline": roof,
            "hbm_roofline": step_hbm_roofline(value, wl.precision, hbm_peak), "kernels": breakdown,
            "clocks": clk, "e2e": e2e, "cpu_baseline": cpu, "mass_rel_drift": m_drift, "mixed": other,
            "rel_l2_vs_fp64_after_1_step": err_vs_fp64, "tracer": tracer, "divergence_damping": divdamp,
            "topography": topo, "setup": setup,
            "simulated_days_per_day": wl.dt / (ms / args.steps * 1e-3),
            "device_memory_gb": {"peak_allocated": round(torch.cuda.max_memory_allocated() / 1e9, 2),
                                 "total": round(torch.cuda.get_device_properties(0).total_memory / 1e9, 2)}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- ensemble workload
def run_ensemble(args, rank, world, local_rank):
    """64 members (32 on R2B4 with dt 360 s, 32 on R2B5 with dt 180 s), 60 levels, mixed
    precision, member perturbations from seed 3: one persistent cooperative launch per
    step for all members, against the same members stepped one after another (each
    from its own recorded graph)."""
    import torch
    torch.cuda.set_device(local_rank)
    from paper_2511_02021_gb300 import build as B
    B.build()
    import paper_2511_02021_gb300 as P
    from paper_2511_02021_gb300 import capi as C
    P.use_torch_allocator(local_rank)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    P.bind_torch_stream(stream)
    dist = world > 1
    if dist:
        import torch.distributed as td
    E = WL.ENSEMBLE
    N, nsub = E["nlev"], E["nsub"]
    grids = {4: C.icon_grid_build(2, 4, N), 5: C.icon_grid_build(2, 5, N)}
    spec = [(4, E["dt_b4"])] * E["members_b4"] + [(5, E["dt_b5"])] * E["members_b5"]

    def make_states():
        return [C.icon_state_init_ex(grids[b], E["seed"] + 1000 * rank, C.ICON_CASE_MEMBER, precision=1, member=m)
                for m, (b, _) in enumerate(spec)]

    cells = sum(20 * 4 ** (b + 1) for b, _ in spec)
    dts = [dt for _, dt in spec]

    def timed(fn, steps):
        if dist:
            td.barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        if dist:
            td.barrier()
        ms = e0.elapsed_time(e1)
        if dist:
            ms = max_over_ranks(ms, "cuda")
        return ms

    # batched: one persistent launch per step
    sts = make_states()
    ens = C.icon_ensemble_create(sts)
    C.icon_ensemble_step(ens, dts, nsub, args.warmup)
    clocks = ClockSampler(local_rank) if rank == 0 else None
    time.sleep(0.4)
    ms_b = timed(lambda k: C._check(C._lib.icon_ensemble_step(ens, (C.ctypes.c_double * len(dts))(*dts), nsub, k)),
                 args.steps)
    clk = clocks.stop() if clocks else None
    kms, kn = np.zeros(C.ICON_KIND_COUNT), np.zeros(C.ICON_KIND_COUNT, dtype=np.int32)
    value_b = job_value(cells * N * nsub * args.steps, world, ms_b)
    C.icon_ensemble_free(ens)
    for st in sts:
        C.icon_state_free(st)

    # sequential: every member from its own graph, one after another
    sts = make_states()
    for st, dt in zip(sts, dts):
        for _ in range(args.warmup):
            C.icon_dycore_step(st, dt, nsub)

    def seq(k):
        for _ in range(k):
            for st, dt in zip(sts, dts):
                C.icon_dycore_step_async(st, dt, nsub)
    ms_s = timed(seq, args.steps)
    for st in sts:
        C.icon_state_status(st)
    value_s = job_value(cells * N * nsub * args.steps, world, ms_s)
    launches_seq = sum(C.icon_state_step_kernels(st, dt, nsub) for st, dt in zip(sts, dts))
    for st in sts:
        C.icon_state_free(st)
    for g in grids.values():
        C.icon_grid_free(g)
    if rank != 0:
        return
    hbm_peak, peak_src = peaks()
    # algorithmic model of one persistent launch (one step of every member)
    alg_bytes = 239.0 * cells * N * nsub
    alg_flops = (2 * MX_COLUMN_FP64_OPS + 2.0) * cells * N * nsub
    t_launch = ms_b / args.steps * 1e-3
    hbm_frac = alg_bytes / t_launch / 1e9 / hbm_peak
    alu_frac = alg_flops / t_launch / FP64_INSTR_PEAK
    roof = {"kernel": "ensemble_persistent", "bound": "alu" if alu_frac > hbm_frac else "hbm",
            "achieved": alg_flops / t_launch / 1e9 if alu_frac > hbm_frac else alg_bytes / t_launch / 1e9,
            "peak": FP64_INSTR_PEAK / 1e9 if alu_frac > hbm_frac else hbm_peak,
            "unit": "G FP64 instr/s" if alu_frac > hbm_frac else "GB/s",
            "frac": max(alu_frac, hbm_frac), "traffic": None,
            "hbm_frac": hbm_frac, "fp64_frac": alu_frac, "launch_ms": ms_b / args.steps, "launches_per_step": 1}
    line = {"metric": METRIC, "value": value_b, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_b / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic (64 perturbed jet members)",
            "config": {"workload": "ensemble-32xR2B4+32xR2B5-L60-mixed", "members": len(spec), "cells": cells,
                       "levels": N, "nsub": nsub, "dt": {"R2B4": E["dt_b4"], "R2B5": E["dt_b5"]},
                       "l2": "inputs larger than L2 (64 member states)"},
            "gpu_launches": 2 * args.steps, "roofline": roof, "clocks": clk,
            "hbm_roofline": step_hbm_roofline(value_b, 1, hbm_peak),
            "sequential": {"value": value_s, "unit": UNIT, "ms_per_step": ms_s / args.steps,
                           "gpu_launches_per_step": launches_seq},
            "batched_speedup_vs_sequential": value_b / value_s}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gpu", "reference"], default="gpu")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="r2b6-fp64")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mixed", action="store_true", help="skip the mixed-precision variant of an FP64 workload")
    ap.add_argument("--no-tracer", action="store_true",
                    help="skip the tracer-transport and divergence-damping measurements")
    args = ap.parse_args()
    wl = WORKLOADS[args.workload]
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if wl is None and args.impl == "reference":
        wl = WL.Workload("ensemble member R2B5-L60", 5, 60, 3, 3, -1.0, 180.0, 5, 1, 1)
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, wl, rank)
        return
    if world > 1:
        import torch
        import torch.distributed as td
        torch.cuda.set_device(local_rank)
        td.init_process_group("nccl")
    if wl is None:
        run_ensemble(args, rank, world, local_rank)
    else:
        run_gpu(args, wl, rank, world, local_rank)
    if world > 1:
        import torch.distributed as td
        td.destroy_process_group()


if __name__ == "__main__":
    main()
