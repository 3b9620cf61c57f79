"""Benchmark of the online nested polarized-traces solve.

One step = one hz_solve of the whole batch (Newton potentials, FGMRES on the
polarized traces with the Gauss-Seidel sweeps, volume reconstruction, FP64
residual refinement to 1e-8), i.e. every row of the hot path.

Default workload (the largest single-GPU configuration): a layered medium
with two dip-slip faults (c from 1.5 to 5.5 with depth), 2000 x 4000
interior + 30-point PML, 8 points per wavelength at c = 1.5, L = 40 layers x
C = 20 cells, 16 point sources on the first interior row, mixed precision
(complex FP32 operators, FP64 Arnoldi and residual).  The same line carries
the 1024 x 1024 smooth random workload (L = C = 16, 64 sources) as
`secondary` and the plain FP64 form of the default workload as `fp64`.

Metric: RHS*Mdof/s = B * n_x * n_z / 1e6 / (seconds per step), whole job.
Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import hz_inputs as I  # noqa: E402

WORKLOADS = {
    # name: (n, n_pml, L, C, B, ppw, seed)
    "smooth1024": dict(n=1024, n_pml=20, L=16, C=16, B=64, ppw=10.0, seed=2),
    "smooth512": dict(n=512, n_pml=20, L=8, C=8, B=32, ppw=10.0, seed=5),
    "smooth256": dict(n=256, n_pml=16, L=8, C=4, B=16, ppw=10.0, seed=2),
    # same per-launch shapes as smooth1024 (64-row layers, 64-column cells, 20-point PML, 64 sources)
    "smooth256_shape1024": dict(n=256, n_pml=20, L=4, C=4, B=64, ppw=10.0, seed=2),
    # a 1024-wide, 256-deep strip: every launch has the shape of the 1024x1024 workload (16 cells per layer)
    "strip1024x256": dict(n=1024, n_z=256, n_pml=20, L=4, C=16, B=64, ppw=10.0, seed=2),
    # three frequencies (6, 8, 10 ppw) of one 512x512 smooth random medium, uneven layers and cells
    # (24-64 points), 256 sources each, solved as one group (one context and stream per frequency)
    "multifreq512": dict(n=512, n_pml=20, B=256, ppws=(6.0, 8.0, 10.0), seed=4, part_seed=40),
    # layered medium with faults, 2000 wide x 4000 deep + 30 PML, L=40 x C=20, 16 sources, 8 ppw at c=1.5
    "layered2000x4000": dict(n=2000, n_z=4000, n_pml=30, L=40, C=20, B=16, ppw=8.0, seed=3, layered=True),
    # the decomposition of the paper's runtime figure (L = 9 layers x L_c = 3 cells), smooth random medium
    "smooth384_9x3": dict(n=384, n_pml=20, L=9, C=3, B=16, ppw=10.0, seed=6),
    # the same generator at 2000 x 400 (4 layers): every launch has the shape of the 2000 x 4000 workload
    "layered2000x400": dict(n=2000, n_z=400, n_pml=30, L=4, C=20, B=16, ppw=8.0, seed=3, layered=True),
}
DEFAULT_WORKLOAD = "layered2000x4000"
SECONDARY_WORKLOAD = "smooth1024"
METRIC = "RHS*Mdof/s, nested polarized-traces solve at 1e-8 residual; % HBM roofline"
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum, one ncu capture of
# launches with the per-launch shapes of a workload) divided by the algorithmic
# bytes of the same launches; the live traffic estimate of a launch is this
# ratio times its algorithmic bytes (traffic grows with the steps, layers and
# cells a launch processes).  Keyed by (kernel class, workload whose launch
# shapes were captured); a class without a capture of its current kernel
# reports traffic null.
# ncu DRAM bytes (read + write) over algorithmic bytes of a kernel class, from one capture of
# its current kernel.  The traffic per launch reported beside the roofline is this ratio times
# the live algorithmic bytes per launch.  The 2000 x 400 layered shape has the cells of the
# 2000 x 4000 one (160 x 160 cell boxes, 16 right-hand sides), so its ratio stands for both.
_CELL_RATIO = (0.987, "ncu DRAM bytes of one cell-solve launch (80 cells of 160 x 160, 16 right-hand sides)"
                      " of the 2000 x 400 layered shape over its algorithmic bytes")
DRAM_PER_ALGO = {
    ("cell_chain", "layered2000x4000", "simt"): _CELL_RATIO,
    ("cell_chain", "layered2000x400", "simt"): _CELL_RATIO,
}
UNIT = "RHS*Mdof/s"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class Clocks:
    """nvidia-smi sampler running during the timed region."""

    def __init__(self, index=0):
        self.index = index
        self.samples = []
        self.proc = None

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap,utilization.gpu")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 8:
                self.samples.append(parts)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return float("nan")
        util = [num(s[7]) for s in self.samples]
        load = [s for s, u in zip(self.samples, util) if u >= 50] or self.samples
        sm = sorted(num(s[0]) for s in load)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in load for i in range(4) if s[3 + i].lower().startswith("active")})
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": num(load[0][1]), "reasons": reasons,
                "samples": len(self.samples)}


def reduce_max(value, world):
    """Max of a scalar over all ranks (the step time of the slowest replica)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as tdist
    dev = "cuda" if tdist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world, B, mdof, ms_per_step):
    """Whole-job RHS*Mdof/s: every replica solves its own batch of B sources."""
    return world * B * mdof / (ms_per_step / 1e3)


def make_problems(wl):
    """[(problem, sources)] of a workload: one entry, or one per frequency."""
    if "ppws" in wl:
        probs = I.uneven_multifreq(n=wl["n"], n_pml=wl["n_pml"], seed=wl["seed"], part_seed=wl["part_seed"],
                                   ppw_list=wl["ppws"])
        return [(pb, I.point_sources_row(pb.n_x, pb.n_z, pb.n_pml, pb.h, wl["B"])) for pb in probs]
    return [make_problem(wl)]


def describe(wl, pbs, B, precision):
    pb = pbs[0]
    if "ppws" in wl:
        return (f"smooth random c in [1.5,4.5] corr 20h, {pb.n_x}x{pb.n_z}+{pb.n_pml} PML, "
                f"{len(pbs)} frequencies ({'/'.join(f'{v:g}' for v in wl['ppws'])} ppw) solved as one group, "
                f"uneven layers/cells 24-64 pts (L={pb.L} x C={pb.C}), {B} point sources row 1 per frequency, "
                f"{precision}")
    medium = ("layered medium with two dip-slip faults, c in [1.5,5.5]" if wl.get("layered")
              else "smooth random c in [1.5,4.5] corr 20h")
    return (f"{medium}, {pb.n_x}x{pb.n_z}+{pb.n_pml} PML, {wl['ppw']:g} ppw, "
            f"L={pb.L} x C={pb.C}, {B} point sources row 1, {precision}")


def make_problem(wl):
    if wl.get("layered"):
        pb = I.layered_faulted(n_x=wl["n"], n_z=wl["n_z"], n_pml=wl["n_pml"], L=wl["L"], C=wl["C"], seed=wl["seed"],
                               ppw=wl["ppw"])
        return pb, I.point_sources_row(pb.n_x, pb.n_z, pb.n_pml, pb.h, wl["B"])
    pb = I.smooth_random(wl["n"], n_pml=wl["n_pml"], L=wl["L"], C=wl["C"], seed=wl["seed"], ppw=wl["ppw"],
                         n_z=wl.get("n_z"))
    f = I.point_sources_row(pb.n_x, pb.n_z, pb.n_pml, pb.h, wl["B"])
    return pb, f


# ------------------------------------------------------------ GPU arm ---
CLASS_NAMES = ["cell_chain", "inner_chain", "batched_fes_gemm"]


def widest_cell(pb):
    """Columns of the widest cell box (interior columns + the PML on both sides)."""
    cols = pb.cell_cols if pb.cell_cols is not None else [-(-pb.n_x // pb.C)]
    return max(cols) + 2 * pb.n_pml


def roofline(kt_ms, kt_n, kt_b, kt_f, ms, steps, mixed, tensor_cores, workload):
    """tensor_cores: the cell solves run on the tensor cores (mixed precision, cells of at
    most 128 columns); otherwise on the FP32 / FP64 pipes."""
    """Roofline of the kernel class with the largest device time, against the roof
    it is closer to, plus every class's algorithmic rates against both roofs."""
    top = int(np.argmax(kt_ms))
    peaks, src = _peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    # FP32 SIMT peak from unit counts and the maximum SM clock: 152 SMs x 128 FMA lanes x 2 flops
    alu_peak = 152 * 128 * 2 * sm_max * 1e6 / 1e12 if mixed else 1.25
    hbm = float(peaks.get("hbm_gbs", 6800.0))

    def rates(i):
        if kt_ms[i] <= 0:
            return 0.0, 0.0
        return kt_b[i] / (kt_ms[i] / 1e3) / 1e9, kt_f[i] / (kt_ms[i] / 1e3) / 1e12
    gbs, tfl = rates(top)
    if gbs / hbm >= tfl / alu_peak:
        roof = {"bound": "hbm", "achieved": round(gbs, 1), "peak": hbm, "unit": "GB/s", "frac": round(gbs / hbm, 4)}
    else:
        roof = {"bound": "alu", "achieved": round(tfl, 3), "peak": round(alu_peak, 2), "unit": "TFLOP/s",
                "frac": round(tfl / alu_peak, 4)}
    traffic, traffic_src = None, None
    key = (CLASS_NAMES[top], workload, "tc" if (mixed and tensor_cores) else "simt" if mixed else "fp64")
    if key in DRAM_PER_ALGO and kt_n[top] > 0:
        ratio, traffic_src = DRAM_PER_ALGO[key]
        traffic = round(float(ratio * kt_b[top] / kt_n[top]))
    roof.update({
        "kernel": CLASS_NAMES[top], "traffic": traffic, "traffic_source": traffic_src,
        "peak_source": (("derived from unit counts: 152 SMs x 128 FP32 lanes x 2 flops x the max SM clock"
                         " (" + src + "); a register-only FMA loop measured 73.3 TFLOP/s")
                        if mixed else "FP64 DFMA, a register-only loop measured 1.255 TFLOP/s")
        if roof["bound"] == "alu" else src + " copy GB/s",
        "launches": int(kt_n[top]), "avg_ms": round(float(kt_ms[top] / max(kt_n[top], 1)), 4),
        "share_of_step": round(float(kt_ms[top] / (ms * steps)), 3),
        "classes": {n: {"ms_per_step": round(float(kt_ms[i] / steps), 3),
                        "launches_per_step": round(float(kt_n[i] / steps), 1),
                        "gb_s": round(rates(i)[0], 1), "tflop_s": round(rates(i)[1], 3),
                        "frac_hbm": round(rates(i)[0] / hbm, 4), "frac_alu": round(rates(i)[1] / alu_peak, 4)}
                    for i, n in enumerate(CLASS_NAMES)}})
    if mixed and tensor_cores and kt_ms[0] > 0:
        # the cell solves run on the tensor cores: 3 TF32 products per real product, against
        # the TF32 rate measured by an MMA-rate probe (1286 TFLOP/s at N >= 128)
        roof["classes"]["cell_chain"]["frac_tensor_3xtf32"] = round(rates(0)[1] / (1286.0 / 3), 4)
    return roof


def measure(args, workload, precision, steps, warmup, world, e2e=False, measure_update=False):
    """Factor one workload, time `steps` solves after `warmup` untimed ones (CUDA events on the
    solver's stream, barrier + synchronize on both sides, max over ranks) and return its record."""
    import torch

    from paper_1510_01831_gb300 import hz

    wl = dict(WORKLOADS[workload])
    if args.B:
        wl["B"] = args.B
    items = make_problems(wl)
    pbs = [pb for pb, _ in items]
    B = items[0][1].shape[0]
    mixed = precision == "mixed"
    prec = hz.HZ_MIXED if mixed else hz.HZ_FP64
    tc = 0 if args.no_tensor_cores else (2 if args.tc_gemm else 1)
    streams = [torch.cuda.Stream() for _ in items]
    ctxs = []
    t0 = time.time()
    for (pb, _), stream in zip(items, streams):
        kw = {}
        if pb.layer_rows is not None:
            kw = dict(layer_rows=pb.layer_rows, cell_cols=pb.cell_cols)
        ctx = hz.Context(pb.m, pb.n_x, pb.n_z, pb.omega, pb.h, pb.n_pml, pb.L, pb.C, precision=prec,
                         device_ptrs=True, stream=stream.cuda_stream, time_kernels=True, refine_tol=1e-8,
                         tensor_cores=tc, krylov=1 if args.krylov == "bicgstab" else 0,
                         precond={"gs": hz.HZ_PGS, "jacobi": hz.HZ_PJAC}[args.precond],
                         inner=hz.HZ_INNER_NESTED if args.inner == "nested" else hz.HZ_INNER_LU,
                         inner_tol=args.inner_tol, compress=args.compress,
                         autotune=args.autotune, tol=args.tol, rhs_lanes=args.rhs_lanes, **kw)
        ctx.hz_factor()
        ctxs.append(ctx)
    t_factor = time.time() - t0
    f_dev = [torch.from_numpy(f).to("cuda") for _, f in items]
    u_dev = [torch.empty_like(x) for x in f_dev]

    def step(fs, us):
        if len(ctxs) == 1:
            _, st = ctxs[0].hz_solve(fs[0], us[0])
            return [st]
        _, sts = hz.hz_solve_group(ctxs, fs, us)
        return sts

    torch.cuda.synchronize()
    for _ in range(warmup):
        step(f_dev, u_dev)
    if world > 1:
        import torch.distributed as tdist
        tdist.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def region(kernel_events):
        # every member stream has finished when a step returns, so events on the first stream
        # bracket all of them
        for c in ctxs:
            c.hz_set_time_kernels(kernel_events)
        if world > 1:
            import torch.distributed as tdist
            tdist.barrier()
        torch.cuda.synchronize()
        sts = []  # one list of member stats per step
        ev0.record(streams[0])
        for _ in range(steps):
            sts.append([st.as_dict() for st in step(f_dev, u_dev)])
        ev1.record(streams[0])
        torch.cuda.synchronize()
        if world > 1:
            import torch.distributed as tdist
            tdist.barrier()
        return reduce_max(ev0.elapsed_time(ev1) / steps, world), sts

    # the timed region runs without per-launch events (consecutive launches may overlap their
    # prologues); the same steps are then run again with an event pair around every launch,
    # which gives the per-class kernel times of the roofline
    with Clocks(int(os.environ.get("LOCAL_RANK", 0))) as clk:
        ms, stats = region(False)
        ms_ev, stats_ev = region(True)
    for c in ctxs:
        c.hz_set_time_kernels(False)
    mdof = sum(pb.n_x * pb.n_z for pb in pbs) / 1e6
    flat = [m for st in stats for m in st]
    flat_ev = [m for st in stats_ev for m in st]
    kt_ms = np.sum([s["kt_ms"] for s in flat_ev], axis=0)
    kt_n = np.sum([s["kt_launches"] for s in flat_ev], axis=0)
    kt_b = np.sum([s["kt_bytes"] for s in flat_ev], axis=0)
    kt_f = np.sum([s["kt_flops"] for s in flat_ev], axis=0)
    last = stats[-1]
    solve = [{"iterations": m["iterations"], "refinements": m["refinements"], "resid": m["resid"],
              "gmres_resid": m["gmres_resid"], "inner_iterations": m["inner_iterations"],
              "compress_rank": m["compress_rank"],
              "phase_ms": {k: round(m[k], 2) for k in ("t_local_ms", "t_gmres_ms", "t_recon_ms", "t_resid_ms",
                                                       "t_total_ms")}} for m in last]
    solve[0]["t_factor_s"] = round(t_factor, 2)
    out = {"workload": f"{workload}: " + describe(wl, pbs, B, precision),
           "value": round(job_throughput(world, B, mdof, ms), 3), "unit": UNIT, "ms_per_step": round(ms, 3),
           "steps": steps, "warmup": warmup, "B": B, "n_x": pbs[0].n_x, "n_z": pbs[0].n_z, "L": pbs[0].L,
           "C": pbs[0].C, "frequencies": len(pbs),
           "gpu_launches": int(sum(m["gpu_launches"] for m in flat)),
           "solve": solve[0] if len(solve) == 1 else solve,
           "ms_per_step_with_kernel_events": round(ms_ev, 3),
           "roofline": roofline(kt_ms, kt_n, kt_b, kt_f, ms_ev, steps, mixed,
                                tc > 0 and max(widest_cell(pb) for pb in pbs) <= 128, workload),
           "clocks": clk.summary()}
    if e2e:
        # end-to-end through the same entry point with pinned host buffers: the copies of the
        # sources in and the fields out are inside the timed region
        f_host = [torch.from_numpy(f).pin_memory() for _, f in items]
        u_host = [torch.empty_like(x).pin_memory() for x in f_host]
        for c in ctxs:
            c.hz_set_device_ptrs(False)
        fh, uh = [x.numpy() for x in f_host], [x.numpy() for x in u_host]
        step(fh, uh)
        torch.cuda.synchronize()
        e_steps = max(1, min(steps, 3))
        t1 = time.perf_counter()
        for _ in range(e_steps):
            step(fh, uh)
        torch.cuda.synchronize()
        e_ms = reduce_max((time.perf_counter() - t1) * 1e3 / e_steps, world)
        for c in ctxs:
            c.hz_set_device_ptrs(True)
        nbytes = sum(f.nbytes for _, f in items)
        out["e2e"] = {"value": round(job_throughput(world, B, mdof, e_ms), 3), "unit": UNIT,
                      "h2d_bytes_per_step": int(nbytes), "d2h_bytes_per_step": int(nbytes)}
    if measure_update:
        # local model update outside the timed region: a patch of the medium inside one
        # cell of the middle layer changes; only that layer is re-factored
        pb0, ctx0 = pbs[0], ctxs[0]
        rows = pb0.layer_rows if pb0.layer_rows is not None else [pb0.n_z // pb0.L] * pb0.L
        z0 = pb0.n_pml + sum(rows[:pb0.L // 2]) + rows[pb0.L // 2] // 4
        x0 = pb0.n_pml + pb0.n_x // (2 * pb0.C)
        m1 = pb0.m.copy()
        m1[z0:z0 + 8, x0:x0 + 8] *= 1.05
        torch.cuda.synchronize()
        t1 = time.time()
        nlay = ctx0.hz_update_model(m1)
        out["local_update"] = {"layers_refactored": nlay, "layers": pb0.L, "t_update_s": round(time.time() - t1, 3),
                               "t_factor_s": round(t_factor / len(ctxs), 3), "patch": "8 x 8 points, m x 1.05"}
    for c in ctxs:
        c.close()
    del f_dev, u_dev
    torch.cuda.empty_cache()
    return out


def run_ours(args, rank, world):
    import torch

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
    main_ = measure(args, args.workload, args.precision, args.steps, args.warmup, world, e2e=not args.no_e2e,
                    measure_update=args.measure_update)
    out = {
        "metric": METRIC, "value": main_["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": main_["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "c64+f64" if args.precision == "mixed" else "c128", "data": "synthetic",
        "config": {"workload": main_["workload"], "B": main_["B"], "n_x": main_["n_x"], "n_z": main_["n_z"],
                   "L": main_["L"], "C": main_["C"], "precision": args.precision,
                   "frequencies": main_["frequencies"], "krylov": args.krylov, "precond": args.precond,
                   "inner": args.inner,
                   "compress": args.compress if args.compress >= 0 else (1e-8 if args.precision == "mixed" else 0.0),
                   "autotune": args.autotune, "rhs_lanes": args.rhs_lanes,
                   "tensor_cores": "off" if args.no_tensor_cores else
                   ("cell solves + batched products" if args.tc_gemm else "cell solves"),
                   "l2": "inputs and operators larger than L2 (no flush needed)", "parallelism": "replicas"},
        "gpu_launches": main_["gpu_launches"],
        "solve": main_["solve"],
        "roofline": dict(main_["roofline"], events_region={
            "ms_per_step": main_["ms_per_step_with_kernel_events"],
            "what": "the same steps run again right after the timed region, with an event pair around every "
                    "launch on the solver's stream; kernel times and shares come from this run"}),
        "e2e": main_.get("e2e"),
        "clocks": main_["clocks"],
    }
    if "local_update" in main_:
        out["local_update"] = main_["local_update"]
    if not args.no_extra:
        if args.workload != SECONDARY_WORKLOAD:
            sec = measure(args, SECONDARY_WORKLOAD, args.precision, args.steps, args.warmup, world)
            out["secondary"] = {k: sec[k] for k in ("workload", "value", "unit", "ms_per_step", "steps", "warmup",
                                                    "gpu_launches", "solve", "roofline", "clocks")}
        if args.precision == "mixed":
            # the plain FP64 form of the same workload, for "mixed beats FP64 at equal final residual"
            k = max(1, min(args.steps, 2))
            f64 = measure(args, args.workload, "fp64", k, 1, world)
            out["fp64"] = {k_: f64[k_] for k_ in ("workload", "value", "unit", "ms_per_step", "steps", "warmup",
                                                  "solve", "clocks")}
            out["fp64"]["mixed_over_fp64"] = round(out["value"] / f64["value"], 2) if f64["value"] else None
    return out


# ------------------------------------------------- oracle (CPU) timing ---
ORACLE_ROWS = 12


def oracle_sample(wl, rows=ORACLE_ROWS):
    """Time the CPU oracle on a bounded sample of the workload: the row-block
    elimination (block-tridiagonal over grid rows, LAPACK-pivoted Schur blocks)
    of the leading `rows` grid rows of the full-width operator, factor plus the
    forward and backward substitution of all B sources.  Every row of the
    elimination costs the same (one NX x NX Schur block), so the time scales by
    rows to the whole grid.  A multi-frequency workload times one sample per
    frequency."""
    import oracle as O
    t_full = t_fac = t_sol = 0.0
    work = 0.0
    for pb, f in make_problems(wl):
        # the top strip of the medium (its own bottom PML) holds the sampled rows; the
        # rows eliminated cost what the same rows of the whole grid cost
        p = pb.n_pml
        nz_s = max(1, rows - 2 * p + 1)
        strip = O.Box(np.ascontiguousarray(pb.m[:nz_s + 2 * p]), pb.n_x, nz_s, p, pb.omega, pb.h,
                      O.default_pml_C(pb.m))
        fs = np.ascontiguousarray(f[:, :nz_s + 2 * p])
        t0 = time.perf_counter()
        fac = strip.factor_rows(rows=rows)
        t1 = time.perf_counter()
        fac.solve(fs)
        t2 = time.perf_counter()
        scale = (pb.n_z + 2 * p) / fac.NZ
        t_full += (t2 - t0) * scale
        t_fac += t1 - t0
        t_sol += t2 - t1
        work += f.shape[0] * pb.n_x * pb.n_z / 1e6
    return work / t_full, {"factor_s": round(t_fac, 3), "solve_s": round(t_sol, 3), "rows": rows,
                           "scale": round(scale, 2), "work": work, "sample_s": round(t_fac + t_sol, 3)}


def _sample_text(det, B):
    return (f"row-block elimination of the leading {det['rows']} grid rows of the full-width operator (on the "
            f"top strip of the medium) "
            f"(factor + forward/backward substitution of {B} sources), time scaled x{det['scale']:.1f} to the "
            f"whole grid")


def oracle_single_thread(workload, B):
    """The same sample with the BLAS limited to one thread (a child process, so the
    thread count is fixed before numpy loads)."""
    env = dict(os.environ, OPENBLAS_NUM_THREADS="1", OMP_NUM_THREADS="1", MKL_NUM_THREADS="1")
    cmd = [sys.executable, os.path.abspath(__file__), "--oracle-sample", "--workload", workload, "--B", str(B)]
    try:
        r = subprocess.run(cmd, env=env, capture_output=True, text=True, timeout=300)
        return json.loads(r.stdout.strip().splitlines()[-1])
    except Exception as e:  # reported, never fatal for the GPU line
        return {"error": str(e)[:200]}


def cpu_baseline(workload, B):
    wl = dict(WORKLOADS[workload])
    wl["B"] = B
    v, det = oracle_sample(wl)
    one = oracle_single_thread(workload, B)
    return {"value": round(v, 5), "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": _sample_text(det, B) + f"; measured sample time {det['sample_s']} s",
            "single_thread": one}


def run_reference(args, rank, world):
    wl = dict(WORKLOADS[args.workload])
    if args.B:
        wl["B"] = args.B
    cores = os.cpu_count()
    vals, samples = [], []
    det = None
    for _ in range(args.warmup + args.steps):
        v, det = oracle_sample(wl)
        vals.append(v)
        samples.append(det["sample_s"])
    v = float(np.mean(vals[args.warmup:]))
    sample_ms = float(np.mean(samples[args.warmup:])) * 1e3
    ms = det["work"] / v * 1e3
    return {"impl": "reference", "metric": METRIC, "value": round(v, 5), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 1),
            "ms_per_step_is": f"extrapolated: the measured sample ({round(sample_ms, 1)} ms per step) x{det['scale']}",
            "sample_ms_per_step": round(sample_ms, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c128", "data": "synthetic",
            "config": {"workload": args.workload, "B": wl["B"]},
            "cpu_baseline": {"value": round(v, 5), "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": _sample_text(det, wl["B"])},
            "e2e": {"value": round(v, 5), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--precond", default="gs", choices=["gs", "jacobi"], help="outer preconditioner")
    ap.add_argument("--B", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the secondary workload and the FP64 form")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end (host buffer) measurement")
    ap.add_argument("--no-tensor-cores", action="store_true", help="mixed precision: cell solves on the SIMT pipes")
    ap.add_argument("--measure-update", action="store_true",
                    help="after the timed steps, time a local model update of one patch (reported, not timed)")
    ap.add_argument("--rhs-lanes", type=int, default=1,
                    help="solve the right-hand sides as this many groups in lockstep on separate streams")
    ap.add_argument("--tc-gemm", action="store_true",
                    help="mixed precision: batched F/E/S/W products with long K on the tensor cores too")
    ap.add_argument("--krylov", default="gmres", choices=["gmres", "bicgstab"], help="outer Krylov method")
    ap.add_argument("--inner", default="lu", choices=["lu", "nested"],
                    help="local solver of the layers: exact inner block LU or inner nested polarized traces")
    ap.add_argument("--inner-tol", type=float, default=0.0, help="nested inner level: preconditioner inner tolerance")
    ap.add_argument("--compress", type=float, default=-1.0,
                    help="compressed-block LU tolerance for the inner factors (0: dense; < 0: library default, "
                         "1e-8 in mixed precision)")
    ap.add_argument("--autotune", action="store_true", help="time the sweep launch configurations during warm-up")
    ap.add_argument("--tol", type=float, default=0.0, help="GMRES tolerance of the first pass (0: library default)")
    ap.add_argument("--oracle-sample", action="store_true", help=argparse.SUPPRESS)
    args = ap.parse_args()
    if args.oracle_sample:  # child process of oracle_single_thread
        wl = dict(WORKLOADS[args.workload])
        if args.B:
            wl["B"] = args.B
        v, det = oracle_sample(wl, rows=2)
        print(json.dumps({"value": round(v, 6), "unit": UNIT, "cores": 1, "sample": _sample_text(det, wl["B"]),
                          "sample_s": det["sample_s"]}))
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.gpus != world:
        print(f"bench.py: --gpus {args.gpus} but WORLD_SIZE={world}; launch one process per GPU with "
              f"torch.distributed.run --nproc-per-node {args.gpus}", file=sys.stderr)
        sys.exit(2)
    if args.impl == "reference":
        # the CPU oracle runs once, on rank 0; the other ranks exit without work
        if rank == 0:
            print(json.dumps(run_reference(args, rank, world)), flush=True)
        return
    if world > 1:
        import torch
        import torch.distributed as tdist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        tdist.init_process_group("nccl")
    out = run_ours(args, rank, world)
    if rank == 0:
        if not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline(args.workload, out["config"]["B"])
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as tdist
        tdist.destroy_process_group()


if __name__ == "__main__":
    main()
