"""Benchmark of the online nested polarized-traces solve.

One step = one hz_solve of the whole batch (Newton potentials, FGMRES on the
polarized traces with the Gauss-Seidel sweeps, volume reconstruction, FP64
residual refinement to 1e-8), i.e. every row of the hot path.

Default workload: smooth random medium (c in [1.5, 4.5], correlation length
20h), 1024 x 1024 interior + 20-point PML, 10 points per wavelength at
c_min, L = 16 layers x C = 16 cells, 64 point sources on the first interior
row, mixed precision (complex FP32 operators, FP64 Arnoldi and residual).

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
}
METRIC = "RHS*Mdof/s, nested polarized-traces solve at 1e-8 residual; % HBM roofline"
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum, one ncu capture of
# launches with the per-launch shapes of the 1024x1024 workload) divided by the
# algorithmic bytes of the same launches; the live traffic estimate of a launch
# is this ratio times its algorithmic bytes (traffic grows with the steps,
# layers and cells a launch processes)
DRAM_PER_ALGO = {
    "inner_chain": (0.65, "profiles/k_inner_sweep_smooth256_shape1024.md"),
    "cell_chain": (0.742, "profiles/k_cell_chain_smooth256_shape1024.md"),
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
def run_ours(args, rank, world):
    import torch

    from paper_1510_01831_gb300 import hz

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
    wl = dict(WORKLOADS[args.workload])
    if args.B:
        wl["B"] = args.B
    items = make_problems(wl)
    pbs = [pb for pb, _ in items]
    B = items[0][1].shape[0]
    prec = hz.HZ_MIXED if args.precision == "mixed" else hz.HZ_FP64
    streams = [torch.cuda.Stream() for _ in items]
    ctxs = []
    t0 = time.time()
    for (pb, _), stream in zip(items, streams):
        kw = {}
        if pb.layer_rows is not None:
            kw = dict(layer_rows=pb.layer_rows, cell_cols=pb.cell_cols)
        ctx = hz.Context(pb.m, pb.n_x, pb.n_z, pb.omega, pb.h, pb.n_pml, pb.L, pb.C, precision=prec,
                         device_ptrs=True, stream=stream.cuda_stream, time_kernels=True, refine_tol=1e-8,
                         tensor_cores=0 if args.no_tensor_cores else (2 if args.tc_gemm else 1), krylov=1 if args.krylov == "bicgstab" else 0,
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
    for _ in range(args.warmup):
        step(f_dev, u_dev)
    dist = world > 1
    if dist:
        import torch.distributed as tdist
        tdist.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stats = []  # one list of member stats per step
    # every member stream has finished when a step returns, so events on the first stream bracket all of them
    with Clocks(int(os.environ.get("LOCAL_RANK", 0))) as clk:
        ev0.record(streams[0])
        for _ in range(args.steps):
            stats.append([st.as_dict() for st in step(f_dev, u_dev)])
        ev1.record(streams[0])
        torch.cuda.synchronize()
    ms = reduce_max(ev0.elapsed_time(ev1) / args.steps, world)
    mdof = sum(pb.n_x * pb.n_z for pb in pbs) / 1e6
    value = job_throughput(world, B, mdof, ms)
    # end-to-end through the same entry point with pinned host buffers
    f_host = [torch.from_numpy(f).pin_memory() for _, f in items]
    u_host = [torch.empty_like(x).pin_memory() for x in f_host]
    for c in ctxs:
        c.hz_set_device_ptrs(False)
    fh, uh = [x.numpy() for x in f_host], [x.numpy() for x in u_host]
    step(fh, uh)
    torch.cuda.synchronize()
    e_steps = max(1, min(args.steps, 3))
    t0 = time.perf_counter()
    for _ in range(e_steps):
        step(fh, uh)
    torch.cuda.synchronize()
    e_ms = (time.perf_counter() - t0) * 1e3 / e_steps
    for c in ctxs:
        c.hz_set_device_ptrs(True)
    flat = [m for st in stats for m in st]
    # kernel-class timings over the timed region
    kt_ms = np.sum([s["kt_ms"] for s in flat], axis=0)
    kt_n = np.sum([s["kt_launches"] for s in flat], axis=0)
    kt_b = np.sum([s["kt_bytes"] for s in flat], axis=0)
    kt_f = np.sum([s["kt_flops"] for s in flat], axis=0)
    names = ["cell_chain", "inner_chain", "batched_fes_gemm"]
    top = int(np.argmax(kt_ms))
    peaks, src = _peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    # FP32 SIMT peak from unit counts and the maximum SM clock: 152 SMs x 128 FMA lanes x 2 flops
    alu_peak = 152 * 128 * 2 * sm_max * 1e6 / 1e12 if prec == hz.HZ_MIXED else 1.25
    gbs = kt_b[top] / (kt_ms[top] / 1e3) / 1e9 if kt_ms[top] > 0 else 0.0
    tfl = kt_f[top] / (kt_ms[top] / 1e3) / 1e12 if kt_ms[top] > 0 else 0.0
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    # the kernel is bound by whichever roof it is closer to
    if gbs / hbm >= tfl / alu_peak:
        roof = {"bound": "hbm", "achieved": round(gbs, 1), "peak": hbm, "unit": "GB/s",
                "frac": round(gbs / hbm, 4)}
    else:
        roof = {"bound": "alu", "achieved": round(tfl, 3), "peak": round(alu_peak, 2), "unit": "TFLOP/s",
                "frac": round(tfl / alu_peak, 4)}
    traffic, traffic_src = None, None
    if names[top] in DRAM_PER_ALGO and kt_n[top] > 0 and (names[top] != "cell_chain" or args.no_tensor_cores):
        ratio, traffic_src = DRAM_PER_ALGO[names[top]]
        traffic = round(float(ratio * kt_b[top] / kt_n[top]))
    roof.update({"kernel": names[top], "traffic": traffic, "traffic_source": traffic_src,
                 "peak_source": (("derived from unit counts: 152 SMs x 128 FP32 lanes x 2 flops x the max SM clock"
                                  " (" + src + "); a register-only FMA loop measured 73.3 TFLOP/s")
                                 if prec == hz.HZ_MIXED else "FP64 DFMA, a register-only loop measured 1.255 TFLOP/s")
                                if roof["bound"] == "alu" else src + " copy GB/s",
                 "launches": int(kt_n[top]), "avg_ms": round(float(kt_ms[top] / max(kt_n[top], 1)), 4),
                 "share_of_step": round(float(kt_ms[top] / (ms * args.steps)), 3),
                 "classes_ms_per_step": {n: round(float(v / args.steps), 3) for n, v in zip(names, kt_ms)},
                 # every timed class: algorithmic rates over its own event time, against both roofs
                 "classes": {n: {"ms_per_step": round(float(kt_ms[i] / args.steps), 3),
                                 "launches_per_step": round(float(kt_n[i] / args.steps), 1),
                                 "gb_s": round(float(kt_b[i] / (kt_ms[i] / 1e3) / 1e9), 1) if kt_ms[i] > 0 else 0.0,
                                 "tflop_s": round(float(kt_f[i] / (kt_ms[i] / 1e3) / 1e12), 3) if kt_ms[i] > 0 else 0.0,
                                 "frac_hbm": round(float(kt_b[i] / (kt_ms[i] / 1e3) / 1e9 / hbm), 4) if kt_ms[i] > 0 else 0.0,
                                 "frac_alu": round(float(kt_f[i] / (kt_ms[i] / 1e3) / 1e12 / alu_peak), 4)
                                 if kt_ms[i] > 0 else 0.0}
                             for i, n in enumerate(names)}})
    if prec == hz.HZ_MIXED and not args.no_tensor_cores and kt_ms[0] > 0:
        # the cell solves run on the tensor cores: 3 TF32 products per real product, against
        # the TF32 rate measured by an MMA-rate probe (1286 TFLOP/s at N >= 128)
        roof["classes"]["cell_chain"]["frac_tensor_3xtf32"] = round(float(kt_f[0] / (kt_ms[0] / 1e3) / 1e12 /
                                                                          (1286.0 / 3)), 4)
    last = stats[-1]
    pb = pbs[0]
    nbytes = sum(f.nbytes for _, f in items)
    solve = [{"iterations": m["iterations"], "refinements": m["refinements"], "resid": m["resid"],
              "gmres_resid": m["gmres_resid"],
              "phase_ms": {k: round(m[k], 2) for k in ("t_local_ms", "t_gmres_ms", "t_recon_ms", "t_resid_ms",
                                                       "t_total_ms")}} for m in last]
    solve[0]["t_factor_s"] = round(t_factor, 2)
    out = {
        "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "c64+f64" if prec == hz.HZ_MIXED else "c128", "data": "synthetic",
        "config": {"workload": f"{args.workload}: " + describe(wl, pbs, B, args.precision),
                   "B": B, "n_x": pb.n_x, "n_z": pb.n_z, "L": pb.L, "C": pb.C, "precision": args.precision,
                   "frequencies": len(pbs), "krylov": args.krylov, "autotune": args.autotune,
                   "rhs_lanes": args.rhs_lanes, "tensor_cores": "off" if args.no_tensor_cores else
                   ("cell solves + batched products" if args.tc_gemm else "cell solves"),
                   "l2": "inputs and operators larger than L2 (no flush needed)", "parallelism": "replicas"},
        "gpu_launches": int(sum(m["gpu_launches"] for m in flat)),
        "solve": solve[0] if len(solve) == 1 else solve,
        "roofline": roof,
        "e2e": {"value": round(world * B * mdof / (e_ms / 1e3), 3), "unit": UNIT,
                "h2d_bytes_per_step": int(nbytes), "d2h_bytes_per_step": int(nbytes)},
        "clocks": clk.summary(),
    }
    if args.measure_update:
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
        t_upd = time.time() - t1
        out["local_update"] = {"layers_refactored": nlay, "layers": pb0.L, "t_update_s": round(t_upd, 3),
                               "t_factor_s": round(t_factor / len(ctxs), 3), "patch": "8 x 8 points, m x 1.05"}
    for c in ctxs:
        c.close()
    return out


# ------------------------------------------------- oracle (CPU) timing ---
def oracle_sample(wl, rows=4, nthreads=None):
    """Time the CPU oracle (banded LU) on a full-width strip of the workload's
    medium and scale to the full grid: with x-fastest ordering the band width
    is the full extended width, so the cost per grid row is the same as for
    the full problem.  A multi-frequency workload times one strip per
    frequency."""
    import oracle as O
    t_full = t_fac = t_sol = 0.0
    work = 0.0
    for pb, f in make_problems(wl):
        p = pb.n_pml
        NZs = rows + 2 * p
        m = np.ascontiguousarray(pb.m[:NZs, :])
        fs = np.ascontiguousarray(f[:, :NZs, :])
        box = O.Box(m, pb.n_x, rows, p, pb.omega, pb.h, O.default_pml_C(pb.m))
        t0 = time.perf_counter()
        fac = box.factor(order=1)
        t1 = time.perf_counter()
        fac.solve(fs)
        t2 = time.perf_counter()
        scale = (pb.n_z + 2 * p) / NZs
        t_full += (t2 - t0) * scale
        t_fac += t1 - t0
        t_sol += t2 - t1
        work += f.shape[0] * pb.n_x * pb.n_z / 1e6
    value = work / t_full
    return value, {"factor_s": round(t_fac, 2), "solve_s": round(t_sol, 2), "rows": rows, "scale": scale,
                   "work": work}


def run_reference(args, rank, world):
    wl = dict(WORKLOADS[args.workload])
    if args.B:
        wl["B"] = args.B
    cores = os.cpu_count()
    steps = []
    det = None
    for _ in range(args.warmup + args.steps):
        v, det = oracle_sample(wl)
        steps.append(v)
    v = float(np.mean(steps[args.warmup:]))
    ms = det["work"] / v * 1e3
    sample = (f"banded LU (x-fastest, band = full extended width) of a {det['rows']}-row full-width strip of the "
              f"workload, factor + {wl['B']} solves, time scaled by {det['scale']:.1f} to the full grid")
    return {"impl": "reference", "metric": METRIC, "value": round(v, 5), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c128", "data": "synthetic",
            "config": {"workload": args.workload, "B": wl["B"]},
            "cpu_baseline": {"value": round(v, 5), "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": round(v, 5), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="smooth1024", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--B", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-tensor-cores", action="store_true", help="mixed precision: cell solves on the SIMT pipes")
    ap.add_argument("--measure-update", action="store_true",
                    help="after the timed steps, time a local model update of one patch (reported, not timed)")
    ap.add_argument("--rhs-lanes", type=int, default=1,
                    help="solve the right-hand sides as this many groups in lockstep on separate streams")
    ap.add_argument("--tc-gemm", action="store_true",
                    help="mixed precision: batched F/E/S/W products with long K on the tensor cores too")
    ap.add_argument("--krylov", default="gmres", choices=["gmres", "bicgstab"], help="outer Krylov method")
    ap.add_argument("--autotune", action="store_true", help="time the sweep launch configurations during warm-up")
    ap.add_argument("--tol", type=float, default=0.0, help="GMRES tolerance of the first pass (0: library default)")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1 and args.impl == "ours":
        import torch
        import torch.distributed as tdist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        tdist.init_process_group("nccl")
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args, rank, world)), flush=True)
        return
    out = run_ours(args, rank, world)
    if rank == 0:
        if not args.no_cpu_baseline:
            wl = dict(WORKLOADS[args.workload])
            if args.B:
                wl["B"] = args.B
            v, det = oracle_sample(wl)
            out["cpu_baseline"] = {"value": round(v, 5), "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                                   "sample": f"{det['rows']}-row full-width strip, band LU factor + solves, "
                                             f"scaled x{det['scale']:.1f} to the full grid"}
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as tdist
        tdist.destroy_process_group()


if __name__ == "__main__":
    main()
