#!/usr/bin/env python
"""Throughput of the third-order DUGKS (T3S3) step on GB300.

Metric: G cell-velocity updates/s (cells x velocities x steps / device time)
of the full T3S3 step (Sec. 2.1.3 of arXiv:1709.05458) on the lid-driven
cavity workload ``cavity256``: 256^2 cells, D2Q9 Gauss-Hermite, Re = 1000,
lid Ma = 0.1, bounce-back/moving walls, FP64.  One bench step = one T3S3
time step of the whole grid; the L2 cache is flushed (a 256 MiB write)
before every timed step, and each step is timed with CUDA events on the
solver's stream.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload W] [--storage fp64|fp32|bf16|f64dw] [--scheme t3s3|t2s3|t2s2]

``--impl reference`` times the CPU oracle (plain FP64 numpy restatement of
the paper) on the host cores on the same workload; N > 1 runs independent
replicas (one per rank, no data-path collective).  Other workloads:
``cavityN`` (N^2 D2Q9 cavity), ``rarefied128_kn{0.1,1,10}_nv64`` (Newton-Cotes
64 x 64, diffuse walls), ``batched64`` (64 uneven instances in one CUDA
graph per step), ``adjoint128`` (the checkpointed gradient of the 128^2
cavity).  The default line also reports the FP32, BF16 and double-word
forms of the same workload (``forms``).
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = "cavity256"
L2_FLUSH_BYTES = 256 << 20

# Algorithmic FP64 flops (FMA = 2) per unit of each kernel, from the
# arithmetic of the method (counted in the design notes): per cell-velocity
# for cell/update kernels, per face-velocity for face kernels.
FLOPS_PER_UNIT = {
    "cell_stage1": 17, "cell_stage2": 17,
    "face_x_stage1": 34, "face_y_stage1": 34, "face_x_stage2": 34, "face_y_stage2": 34,
    "update_stage1": 17, "update_stage2": 21,
    # fused D2Q9 kernels, per cell-velocity: two faces (2 x 22.0: the 70
    # non-zero stencil products of the nine velocities, face moments, one
    # reciprocal, the equilibrium polynomials and f-bar -> f of the six
    # velocities that cross the face) plus the cell part (stage 1: L*, f~',
    # moments, feq', dt Omega', g2, X = 25.9; stage 2: L**, f^, moments, feq,
    # g1 = 13.8)
    "d2q9_stage1": 69.9, "d2q9_stage2": 57.8,
    # T2 schemes on the generic kernels (counted as the T3S3 generic ones)
    "t2_cell": 17, "t2_face_x": 34, "t2_face_y": 34, "t2_update": 19,
}
SCHEMES = {"t3s3": 0, "t2s3": 1, "t2s2": 2}
PATHS = {"auto": 0, "generic": 1, "reference": 2}
# The same kernels in FP64 (dugks_generic_mixed.cu with FP64 storage): all
# their arithmetic is FP64 -- cell: moment sums 5 + g = a f + b W P(xi) with
# P quadratic (5 FMAs) 14; face: 9-point stencil 18 + moment sums 5;
# updates: the cubic equilibrium term W S(xi) (10 FMAs + 1) + face
# differences 6 + the stage maps 9 (stage 1) / 3 (stage 2).
FLOPS_PER_UNIT_GDEV_FP64 = {
    "gdev_cell": 19, "gdev_face_x": 23, "gdev_face_y": 23,
    "gdev_update_stage1": 36, "gdev_update_stage2": 30,
}
# On a tensor velocity grid (Newton-Cotes n x n with n a multiple of 16) the
# 16 velocities a thread takes share xi_x: P and S reduce, once per thread,
# to polynomials in xi_y (2 and 3 FMAs per velocity).
FLOPS_PER_UNIT_GDEV_FP64_TGRID = {
    "gdev_cell": 13, "gdev_update_stage1": 22, "gdev_update_stage2": 16,
}
# The deviation forms (FP32 / BF16 per-cell arrays; face values FP32 in
# both) against HBM: algorithmic bytes per cell- or face-velocity.
HBM_BYTES_PER_UNIT = {
    # moments: read d; g pass: read d, write g
    "gdev_cell": {"fp32": 12, "bf16": 6},
    # face pass: read g, write the face value f-bar (FP32)
    "gdev_face_x": {"fp32": 8, "bf16": 6}, "gdev_face_y": {"fp32": 8, "bf16": 6},
    # read f^, g1, x and y faces; write f~', acc
    "gdev_update_stage1": {"fp32": 24, "bf16": 16},
    # read f~', acc, x and y faces; write f^
    "gdev_update_stage2": {"fp32": 20, "bf16": 14},
    # fused D2Q9 stage kernels: read g and the cell's own array, write two arrays
    "d2q9m_stage1": {"fp32": 16, "bf16": 8}, "d2q9m_stage2": {"fp32": 16, "bf16": 8},
    # the same in double-word arithmetic on FP64 arrays
    "d2q9dw_stage1": {"f64dw": 32}, "d2q9dw_stage2": {"f64dw": 32},
    # class-moment generic path (deviation forms): the sums pass reads the
    # stage source once; update 1 reads f^ and writes f~'; update 2 reads
    # f~' and f^ and writes f^ (per cell-velocity; halo re-reads and the
    # O(cells) finaliser data are not counted)
    "gnc_sums": {"fp32": 4, "bf16": 2},
    "gnc_update_stage1": {"fp32": 8, "bf16": 4},
    "gnc_update_stage2": {"fp32": 12, "bf16": 6},
}
# Algorithmic DRAM bytes per unit (FP64 values each kernel must read/write once).
BYTES_PER_UNIT = {
    "cell_stage1": 16, "cell_stage2": 16,              # read f, write g
    "face_x_stage1": 16, "face_y_stage1": 16,          # read g (upwind), write f_b
    "face_x_stage2": 16, "face_y_stage2": 16,
    "update_stage1": 48,                               # read f^, g, 2 faces; write f~', acc (per cell: 6 values)
    "update_stage2": 40,                               # read f~', acc, 2 faces; write f^
    # fused D2Q9 stage kernels (FP64 arrays, both arithmetic forms): read g
    # and the cell's own array, write two arrays, one density per cell
    "d2q9_stage1": 32 + 8 / 9, "d2q9_stage2": 32 + 8 / 9,
    "d2q9dw_stage1": 32 + 8 / 9, "d2q9dw_stage2": 32 + 8 / 9,
    # optimised generic kernels with FP64 storage: cell = moments (read f) +
    # g pass (read f, write g); face = read g, write f-bar
    "gdev_cell": 24, "gdev_face_x": 16, "gdev_face_y": 16,
    "gdev_update_stage1": 48, "gdev_update_stage2": 40,
}


# DRAM bytes (read + write) per unit measured by ncu for the kernels named,
# from a capture of the 1024^2 D2Q9 cavity (scaled to a launch by the units
# it processes); kept only while the kernel is unchanged.
TRAFFIC_BYTES_PER_UNIT = {
    "d2q9_stage1": (151.364352e6 + 110.542336e6) / (1024 * 1024 * 9),
    "d2q9_stage2": (151.349504e6 + 114.771968e6) / (1024 * 1024 * 9),
    # the double-word instantiation, same capture
    "d2q9dw_stage1": (151.452672e6 + 109.881856e6) / (1024 * 1024 * 9),
    "d2q9dw_stage2": (151.430400e6 + 114.004992e6) / (1024 * 1024 * 9),
}


def kernel_launch_units(name, nv, nx, ny):
    """Units one launch of the named kernel processes: face-velocities for
    the generic face kernels, cell-velocities for every other kernel."""
    face = name.replace("gdev_", "")[:6]
    return {"face_x": nv * ny * (nx + 1), "face_y": nv * (ny + 1) * nx}.get(face, nv * nx * ny)


def hbm_view(prof, label, nv, nx, ny, peak_gbs):
    """A form's dominant kernel (largest device time among those with an
    algorithmic byte count for the form) against HBM: bytes per unit x
    units per launch / mean launch time, and that over the copy bandwidth.
    prof: kernel name -> (launches, total ms).  None if no kernel counts."""
    cand = [(k, v) for k, v in prof.items()
            if label in HBM_BYTES_PER_UNIT.get(k, {}) and v[0] > 0 and v[1] > 0]
    if not cand:
        return None
    name, (nl, kms) = max(cand, key=lambda kv: kv[1][1])
    bpu = HBM_BYTES_PER_UNIT[name][label]
    gbs = bpu * kernel_launch_units(name, nv, nx, ny) / (kms * 1e-3 / nl) / 1e9
    return {"kernel": name, "achieved_gbs": gbs, "frac": gbs / peak_gbs, "bytes_per_unit": bpu}


# Stated accuracy of each storage form against FP64 over the workloads' full
# lengths (bounds asserted by tests/test_gpu_forms_long.py, measured values
# from those runs on GB300): the metric's "at stated L2 error".
STATED_BOUNDS = {
    "cavity256": {
        "fp32": {"steps": 20000, "E_u_bound": 2e-3, "E_u_measured": 4.4e-4},
        "bf16": {"steps": 20000, "E_u_bound": 0.6, "E_u_measured": 0.281},
        "f64dw": {"steps": 20000, "E_u_bound": 2e-10, "E_u_measured": 3.6e-11},
    },
    "rarefied128_kn1_nv64": {
        "fp32": {"steps": 500, "E_u_bound": 2e-7, "E_u_measured": 4.9e-8},
        "bf16": {"steps": 500, "E_u_bound": 0.3, "E_u_measured": 0.083},
    },
}


def alu_peaks(P, stream, clocks_index=None):
    """FMA-throughput microbenchmark (dugks_alu_peak) on this GPU: FP64 DFMA,
    FP32 FFMA and packed FP32 pairs; best of several launches of ~10-20 ms,
    with the SM clock sampled during them.  TFLOP/s at the clocks seen, and
    the same per SM per clock (flops / (SMs x MHz)), which does not depend
    on the clock."""
    import torch
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    bps = 4
    out = torch.empty(sms * bps * 256, dtype=torch.float64, device="cuda")
    clk = Clocks(clocks_index) if clocks_index is not None else None
    if clk:
        clk.start()
        time.sleep(0.3)
    res = {}
    for name, kind, iters, reps in (("fp64", P.ALU_FP64, 500, 6), ("fp32", P.ALU_FP32, 30000, 4),
                                    ("fp32x2", P.ALU_FP32X2, 30000, 4)):
        best = None
        for _ in range(reps):
            fl, ms = P.dugks_alu_peak(kind, iters, bps, out, stream)
            r = fl / (ms * 1e-3) / 1e12
            best = r if best is None or r > best else best
        res[name] = best
    c = clk.stop() if clk else None
    mhz = (c or {}).get("sm_mhz")
    d = {"unit": "TFLOP/s", "sms": sms, "fp64_tflops": res["fp64"], "fp32_tflops": res["fp32"],
         "fp32x2_tflops": res["fp32x2"], "sm_mhz_median": mhz,
         "how": "dugks_alu_peak: SMs x 4 blocks x 256 threads, 8 FMA chains per thread, "
                "best of 4-6 launches (CUDA events)"}
    if mhz:
        d["fp64_flop_per_sm_per_clk"] = res["fp64"] * 1e12 / (sms * mhz * 1e6)
        d["fp32_flop_per_sm_per_clk"] = res["fp32"] * 1e12 / (sms * mhz * 1e6)
    if c:
        d["clocks"] = c
    return d


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f)
    return {}


class Clocks:
    """nvidia-smi sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def reduce_max(vals, world):
    """Max over the ranks of a list of floats (the timing rule: the slowest
    rank's time); one rank returns the list unchanged."""
    vals = [float(v) for v in vals]
    if world == 1:
        return vals
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor(vals, dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.cpu()]


def whole_job_rate(units_per_rank, steps, world, seconds):
    """G updates/s of the whole job: every rank advances its own replica of
    units_per_rank cell-velocities per step (weak scaling)."""
    return units_per_rank * steps * world / seconds / 1e9


def make_solver(P, PV, WL, stream, storage=0, scheme="t3s3", path=0):
    c = WL.config(WORKLOAD)
    if c.get("vel") == "nc":
        xi, W, RT = PV.newton_cotes(c["nv1"], c["RT"])
    else:
        xi, W, RT = PV.d2q9(c["RT"])
    n = c["nx"]
    s = P.Solver(n, n, 1.0 / n, 1.0 / n, xi, W, RT, c["tau"], c["dt"], c["bc"], stream=stream,
                 storage=storage, scheme=SCHEMES[scheme], path=path)
    s.set_equilibrium(*WL.rest_fields(n, n))
    return s, c, len(W)


def cpu_oracle_rate(steps, budget_s=20.0, workload=None):
    """The oracle as it stands on one host core: T3S3 steps of the full
    cavity256 grid from rest.  Returns (updates/s, steps run, seconds, 1)."""
    os.environ["OMP_NUM_THREADS"] = "1"
    os.environ["OPENBLAS_NUM_THREADS"] = "1"
    from oracle import dugks_oracle as O
    from oracle import velocity_sets as OV
    import workloads as WL
    c = WL.config(workload or WORKLOAD)
    xi, W, RT = OV.d2q9(c["RT"])
    n = c["nx"]
    s = O.Setup(n, n, 1.0 / n, 1.0 / n, xi, W, RT, c["tau"], c["dt"], c["bc"])
    f = O.equilibrium_state(*WL.rest_fields(n, n), s)
    f = O.t3s3_step(f, s)                       # first step: allocation warm-up
    t0 = time.perf_counter()
    done = 0
    while done < steps:
        f = O.t3s3_step(f, s)
        done += 1
        if budget_s is not None and time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    return n * n * len(W) * done / dt, done, dt, 1


def _oracle_worker(args):
    steps, budget, workload = args
    return cpu_oracle_rate(steps, budget, workload)


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.processor() or platform.machine()


def cpu_oracle_all_cores(steps, budget_s):
    """The oracle on every host core at once: one single-threaded worker per
    core (spawned processes, never forked from this CUDA process), each
    advancing its own copy of the workload for the same time budget.  The
    aggregate rate is the sum of the workers' rates.  Returns (updates/s,
    total steps, seconds, cores, per-worker rates)."""
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    os.environ["OMP_NUM_THREADS"] = "1"
    os.environ["OPENBLAS_NUM_THREADS"] = "1"
    ctx = mp.get_context("spawn")
    t0 = time.perf_counter()
    with ctx.Pool(cores) as pool:
        res = pool.map(_oracle_worker, [(steps, budget_s, WORKLOAD)] * cores)
    secs = time.perf_counter() - t0
    return sum(r[0] for r in res), sum(r[1] for r in res), secs, cores, [r[0] for r in res]


def run_reference(args):
    world, rank, _ = dist_setup()
    if rank != 0:
        return 0
    import workloads as WL
    c = WL.config(WORKLOAD)
    for _ in range(args.warmup):
        cpu_oracle_rate(1, None)
    # every timed step: one full T3S3 step of the workload on every host core
    # (one spawned single-threaded process per core)
    rate, done, secs, cores, _ = cpu_oracle_all_cores(args.steps, None)
    done //= cores
    units = c["nx"] * c["ny"] * 9
    val = rate / 1e9
    line = {
        "impl": "reference", "metric": "G cell-velocity updates/s (T3S3 step)",
        "value": val, "unit": "G updates/s", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * units * cores / rate, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "cells": f"{c['nx']}x{c['ny']}", "velocities": "D2Q9",
                   "bc": "bounce-back, moving lid", "units_per_step": units},
        "cpu_baseline": {"value": val, "unit": "G updates/s", "cores": cores, "kind": "oracle",
                         "cpu_model": cpu_model(),
                         "sample": (f"{done} full T3S3 steps of {WORKLOAD} from rest on each of "
                                    f"{cores} host cores (numpy FP64 oracle, one process per core)")},
        "e2e": {"value": val, "unit": "G updates/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def timed_steps(P, solver, stream, flush, steps):
    """K T3S3 steps, each after an L2 flush, each timed with CUDA events on
    the solver's stream.  Returns (total ms, per-kernel profile)."""
    import torch
    P.dugks_profile(solver.ctx, True)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(steps)]
    with torch.cuda.stream(stream):
        for a, b in evs:
            flush.fill_(1.0)
            a.record(stream)
            solver.step(1)
            b.record(stream)
    torch.cuda.synchronize()
    prof = P.dugks_profile_read(solver.ctx)
    P.dugks_profile(solver.ctx, False)
    return sum(a.elapsed_time(b) for a, b in evs), prof


def batched_measure(P, PV, WL, stream, steps, warmup, world=1, individual=True, storage=0):
    """The batched workload: 64 seeded uneven instances advanced together
    (one persistent launch per stage for the D2Q9 ones, one CUDA graph per
    bench step); per step: sum of cells x velocities over all instances.
    Also times the same instances stepped one by one (each context's own
    launches, no graph) for the gain of batching.  Returns a dict."""
    import torch
    insts = WL.config("batched64")["instances"]
    sols, units, tuned = [], 0, {}
    for it in insts:
        N = it["N"]
        if it["vel"] == "d2q9":
            xi, W, RT = PV.d2q9(it["RT"])
        else:
            xi, W, RT = PV.newton_cotes(it["nv1"], it["RT"])
        if it["kind"] == "tgv":
            bc = [(P.PERIODIC, 0, 0)] * 4
        else:
            kw = P.BOUNCEBACK if it["vel"] == "d2q9" else P.DIFFUSE
            bc = [(kw, 0, 0)] * 3 + [(kw, it["U"], 0)]
        s = P.Solver(N, N, 1.0 / N, 1.0 / N, xi, W, RT, it["tau"], it["dt"], bc, stream=stream,
                     storage=storage)
        if it["kind"] == "tgv":
            s.set_equilibrium(*WL.tgv_fields(N, N, it["U"] * 2 * 3.141592653589793, RT))
        else:
            s.set_equilibrium(*WL.rest_fields(N, N))
        if it["vel"] == "d2q9":
            tuned[id(s)] = P.dugks_autotune(s.ctx, trials=2)
        sols.append(s)
        units += N * N * len(W)
    batch = P.Batch(sols)
    batch_ty = batch.autotune(2)              # tile height of the persistent D2Q9 launch
    for _ in range(max(warmup, 0)):
        batch.step(1)
    torch.cuda.synchronize()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(steps)]
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    with torch.cuda.stream(stream):
        for a, b in evs:
            flush.fill_(1.0)
            a.record(stream)
            batch.step(1)
            b.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ms = sum(a.elapsed_time(b) for a, b in evs)
    ind_ms = None
    if individual:
        # the same contexts stepped one after another with their own launches
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(steps)]
        with torch.cuda.stream(stream):
            for a, b in evs:
                flush.fill_(1.0)
                a.record(stream)
                for sv in sols:
                    sv.step(1)
                b.record(stream)
        torch.cuda.synchronize()
        ind_ms = sum(a.elapsed_time(b) for a, b in evs)
    ok = all(sv.check() == P.DUGKS_OK for sv in sols)
    n_d2q9 = sum(1 for it in insts if it["vel"] == "d2q9")
    d2q9_units = sum(it["N"] ** 2 * 9 for it in insts if it["vel"] == "d2q9")
    batch.close()
    for sv in sols:
        sv.close()
    out = {"ms": ms, "units": units, "steps": steps, "instances": len(insts),
           "d2q9_instances": n_d2q9, "d2q9_units_per_step": d2q9_units,
           "tile_heights": sorted(set(tuned.values())), "batch_tile_height": batch_ty,
           "stable": ok}
    if ind_ms is not None:
        out["individual_ms"] = ind_ms
    return out


def run_batched(args):
    """``--workload batched64``: the batched measurement as the headline line."""
    import torch
    import paper_1709_05458_gb300 as P
    from paper_1709_05458_gb300 import velocity_sets as PV
    import workloads as WL

    world, rank, local = dist_setup()
    if world > 1:                                 # one replica of the batch per rank
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    stream = torch.cuda.Stream()
    P.load()
    st = {"fp64": 0, "fp32": 1, "bf16": 2}[args.storage]
    m = batched_measure(P, PV, WL, stream, args.steps, args.warmup, world, storage=st)
    ms, = reduce_max([m["ms"]], world)
    if rank != 0:
        return 0
    units = m["units"]
    line = {
        "metric": "G cell-velocity updates/s (T3S3 step, batched instances)",
        "value": whole_job_rate(units, args.steps, world, ms * 1e-3), "unit": "G updates/s",
        "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp64": "f64", "fp32": "f32 (f32 deviation storage)",
                  "bf16": "f32 (bf16 deviation storage)"}[args.storage],
        "data": "synthetic",
        "config": {"workload": "batched64", "instances": m["instances"],
                   "d2q9_instances": m["d2q9_instances"],
                   "units_per_step": units, "d2q9_units_per_step": m["d2q9_units_per_step"],
                   "graph": "one CUDA graph per bench step",
                   "parallelism": f"replicas{world}" if world > 1 else "single",
                   "tile_heights": m["tile_heights"],
                   "batch_tile_height": m["batch_tile_height"],
                   "l2": "flushed (256 MiB write) before every timed step"},
        "individual": {"ms_per_step": m["individual_ms"] / args.steps,
                       "value": units * args.steps / (m["individual_ms"] * 1e-3) / 1e9},
        "stable": m["stable"],
    }
    print(json.dumps(line))
    return 0


def workload_measure(P, PV, WL, stream, flush, steps, warmup, storage, label,
                     workload="rarefied128_kn1_nv64"):
    """Another workload (default rarefied128: 128^2 cells, 64 x 64
    Newton-Cotes, Kn 1, diffuse walls) in one storage form: device-timed
    steps, the dominant kernel against HBM and the whole step against the
    algorithmic bytes of one read and one write of the stored state per
    update."""
    saved = globals()["WORKLOAD"]
    globals()["WORKLOAD"] = workload
    try:
        s, c, nv = make_solver(P, PV, WL, stream, storage=storage)
    finally:
        globals()["WORKLOAD"] = saved
    units = c["nx"] * c["ny"] * nv
    for _ in range(max(warmup, 0)):
        s.step(1)
    ms, prof = timed_steps(P, s, stream, flush, steps)
    ok = s.check() == P.DUGKS_OK
    try:                                          # fused D2Q9 kernels only
        tile_height = P.dugks_tile_height(s.ctx)
    except Exception:
        tile_height = None
    s.close()
    peak = measured_peaks().get("hbm_gbs", 6800.0)
    sbytes = {"fp32": 4, "bf16": 2, "fp64": 8}[label]
    step_s = ms * 1e-3 / steps
    return {"workload": workload, "storage": label,
            "value": units / step_s / 1e9, "unit": "G updates/s", "ms_per_step": step_s * 1e3,
            "steps": steps, "units_per_step": units,
            "step_hbm": {"bytes_per_update": 2 * sbytes,
                         "achieved_gbs": 2 * sbytes * units / step_s / 1e9,
                         "frac": 2 * sbytes * units / step_s / 1e9 / peak,
                         "basis": "one read and one write of the stored state per update"},
            "hbm": hbm_view(prof, label, nv, c["nx"], c["ny"], peak),
            "stated_bound": STATED_BOUNDS.get(workload, {}).get(label),
            **({"tile_height": tile_height} if tile_height else {}),
            "kernels": {k: {"launches": v[0], "ms": round(v[1], 4)} for k, v in prof.items() if v[0]},
            "stable": ok}


def run_adjoint(args):
    """The gradient workload (cavity 128^2 D2Q9 FP64, Re 1000, lid Ma 0.1,
    CFL 0.25, checkpoints every 100 steps): one dugks_adjoint_run over K
    forward steps -- the checkpointed forward sweep, then per segment the
    recomputed forward states and the reverse steps -- timed with CUDA events
    on the solver's stream; value = cells x velocities x K / time.  The
    forward-only rate of the same solver is reported beside it."""
    import numpy as np
    import torch
    import paper_1709_05458_gb300 as P
    from paper_1709_05458_gb300 import velocity_sets as PV
    import workloads as WL

    world, rank, local = dist_setup()
    if rank != 0:
        return 0
    torch.cuda.set_device(local)
    stream = torch.cuda.Stream()
    P.load()
    n = 128
    c = WL.config("cavity128")
    xi, W, RT = PV.d2q9(c["RT"])
    dt = 0.5 * c["dt"]
    s = P.Solver(n, n, 1.0 / n, 1.0 / n, xi, W, RT, c["tau"], dt, c["bc"], stream=stream)
    s.set_equilibrium(*WL.rest_fields(n, n))
    units = n * n * len(W)
    every = 100
    with torch.cuda.stream(stream):
        f0 = torch.empty((len(W), n, n), dtype=torch.float64, device="cuda")
        P.dugks_get_state(s.ctx, f0)
        lam = torch.ones_like(f0)
        lam0 = torch.empty_like(f0)
        for _ in range(max(args.warmup, 0)):
            P.dugks_adjoint_run(s.ctx, f0, every, every, lam, lam0)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        P.dugks_adjoint_run(s.ctx, f0, args.steps, every, lam, lam0)
        b.record(stream)
        b.synchronize()
        ms = a.elapsed_time(b)
        P.dugks_set_state(s.ctx, f0)
        fa, fb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        fa.record(stream)
        s.step(args.steps)
        fb.record(stream)
        fb.synchronize()
        fms = fa.elapsed_time(fb)
    ok = bool(torch.isfinite(lam0).all()) and s.check() == P.DUGKS_OK
    line = {
        "metric": "G cell-velocity updates/s (T3S3 gradient: checkpointed forward + reverse)",
        "value": units * args.steps / (ms * 1e-3) / 1e9, "unit": "G updates/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "adjoint128", "cells": f"{n}x{n}", "velocities": "D2Q9",
                   "bc": "bounce-back walls, moving lid", "checkpoint_every": every,
                   "units_per_step": units, "l2": "not flushed (one call covers all steps)"},
        "forward_only": {"value": units * args.steps / (fms * 1e-3) / 1e9,
                         "ms_per_step": fms / args.steps},
        "stable": ok,
    }
    print(json.dumps(line))
    s.close()
    return 0


def run_ours(args):
    import numpy as np
    import torch
    import paper_1709_05458_gb300 as P
    from paper_1709_05458_gb300 import velocity_sets as PV
    import workloads as WL

    world, rank, local = dist_setup()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev_index = torch.cuda.current_device()
    stream = torch.cuda.Stream()
    P.load()
    main_storage = {"fp64": P.FP64, "fp32": P.G_FP32, "bf16": P.G_BF16,
                    "f64dw": P.F64_DW}[args.storage]
    solver, c, nv = make_solver(P, PV, WL, stream, storage=main_storage, scheme=args.scheme,
                                path=PATHS[args.path])
    units = c["nx"] * c["ny"] * nv
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    # warm-up
    for _ in range(max(args.warmup, 0)):
        solver.step(1)
    solver.synchronize()
    assert solver.check() == P.DUGKS_OK, "warm-up produced an unstable state"

    # device-timed region (FP64 form)
    clocks = Clocks(dev_index) if rank == 0 else None
    if clocks:
        clocks.start()
        time.sleep(0.3)
    barrier()
    torch.cuda.synchronize()
    t_wall = time.perf_counter()
    ms, prof = timed_steps(P, solver, stream, flush, args.steps)
    barrier()
    t_wall = time.perf_counter() - t_wall
    clk = clocks.stop() if clocks else None
    ok = solver.check() == P.DUGKS_OK
    _, u64, v64 = solver.moments()

    # end to end through the C ABI with host buffers: upload f^ from pinned
    # host memory, one step, read the moments back, every step
    f_host = torch.empty((nv, c["ny"], c["nx"]), dtype=torch.float64).pin_memory()
    # rho, ux, uy as the three planes of one pinned buffer: one read-back copy
    mom_host = torch.empty((3, c["ny"], c["nx"]), dtype=torch.float64).pin_memory()
    P.dugks_get_state(solver.ctx, f_host.numpy())
    fh = f_host.numpy()
    mh = list(mom_host.numpy())
    for _ in range(0 if args.no_e2e else 2):
        P.dugks_set_state(solver.ctx, fh)
        solver.step(1)
        P.dugks_moments(solver.ctx, *mh)
    e2e_steps = 0 if args.no_e2e else max(1, min(args.steps, 200))
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        P.dugks_set_state(solver.ctx, fh)
        solver.step(1)
        P.dugks_moments(solver.ctx, *mh)
    torch.cuda.synchronize()
    barrier()
    e2e_s = time.perf_counter() - t0

    # the FP32 and BF16 deviation-storage forms on the same workload and
    # protocol; E(u) against the FP64 run after the same W + K steps
    forms = {}
    if not args.no_forms and args.storage == "fp64" and args.scheme == "t3s3":
        extra = (("f64dw", P.F64_DW),) if c.get("vel") != "nc" else ()
        for label, st in (("fp32", P.G_FP32), ("bf16", P.G_BF16)) + extra:
            s2, _, _ = make_solver(P, PV, WL, stream, storage=st)
            for _ in range(max(args.warmup, 0)):
                s2.step(1)
            fms, fprof = timed_steps(P, s2, stream, flush, args.steps)
            _, u2, v2 = s2.moments()
            num = np.sqrt(((u2 - u64) ** 2 + (v2 - v64) ** 2).sum())
            den = np.sqrt((u64 ** 2 + v64 ** 2).sum())
            forms[label] = {"value": units * args.steps * world / (fms * 1e-3) / 1e9,
                            "ms_per_step": fms / args.steps,
                            "E_u_vs_fp64_after_bench_steps": float(num / den),
                            "stated_bound": STATED_BOUNDS.get(WORKLOAD, {}).get(label),
                            "hbm": hbm_view(fprof, label, nv, c["nx"], c["ny"],
                                            measured_peaks().get("hbm_gbs", 6800.0)),
                            "kernels": {k: {"launches": v[0], "ms": round(v[1], 4)}
                                        for k, v in fprof.items() if v[0]}}
            s2.close()

    # the ALU peaks of this GPU (the FP64 form's roofline denominator)
    peaks = alu_peaks(P, stream, dev_index if rank == 0 else None)

    # the rarefied (Newton-Cotes) and batched workloads beside the headline
    extra = {}
    if not args.no_extra and WORKLOAD == "cavity256":
        extra["rarefied128_fp32"] = workload_measure(P, PV, WL, stream, flush, 20, 3, P.G_FP32,
                                                     "fp32")
        extra["cavity1024_fp32"] = workload_measure(P, PV, WL, stream, flush, 50, 3, P.G_FP32,
                                                    "fp32", workload="cavity1024")
        for key, st in (("batched64", P.FP64), ("batched64_fp32", P.G_FP32)):
            b = batched_measure(P, PV, WL, stream, 3, 2, world, storage=st)
            extra[key] = {
                "value": b["units"] * b["steps"] / (b["ms"] * 1e-3) / 1e9, "unit": "G updates/s",
                "ms_per_step": b["ms"] / b["steps"], "steps": b["steps"],
                "storage": {P.FP64: "fp64", P.G_FP32: "fp32"}[st],
                "units_per_step": b["units"], "instances": b["instances"],
                "d2q9_instances": b["d2q9_instances"], "tile_heights": b["tile_heights"],
                "batch_tile_height": b["batch_tile_height"],
                "individual": {"ms_per_step": b["individual_ms"] / b["steps"],
                               "value": b["units"] * b["steps"] / (b["individual_ms"] * 1e-3) / 1e9},
                "graph": "one CUDA graph per step", "stable": b["stable"]}

    ms, e2e_s = reduce_max([ms, e2e_s], world)
    if rank != 0:
        return 0

    value = whole_job_rate(units, args.steps, world, ms * 1e-3)
    e2e = whole_job_rate(units, e2e_steps, world, e2e_s) if e2e_steps else None

    # roofline of the dominant kernel (largest share of device time)
    flops_per_unit = dict(FLOPS_PER_UNIT)
    hbm_per_unit = dict(HBM_BYTES_PER_UNIT)
    if args.storage == "fp64":
        flops_per_unit.update(FLOPS_PER_UNIT_GDEV_FP64)
        if c.get("vel") == "nc" and c["nv1"] % 16 == 0:
            flops_per_unit.update(FLOPS_PER_UNIT_GDEV_FP64_TGRID)
        hbm_per_unit = {}
    else:
        for k in hbm_per_unit:
            flops_per_unit.pop(k, None)
    name, (nl, kms) = max(((k, v) for k, v in prof.items()
                           if (k in flops_per_unit or k in hbm_per_unit)
                           and v[0] > 0 and v[1] > 0),
                          key=lambda kv: kv[1][1])
    nx, ny = c["nx"], c["ny"]
    per_launch_units = kernel_launch_units(name, nv, nx, ny)
    # gdev face and cell entries cover both stages: two launches per step
    avg_s = kms * 1e-3 / max(nl, 1)
    if name in hbm_per_unit:
        bound, unit = "hbm", "GB/s"
        achieved = hbm_per_unit[name][args.storage] * per_launch_units / avg_s / 1e9
        peak = measured_peaks().get("hbm_gbs", 6800.0)
        peak_source = ("measured copy bandwidth" if "hbm_gbs" in measured_peaks()
                       else "fallback 6.8 TB/s")
    else:
        bound, unit = "alu", "TFLOP/s"
        achieved = flops_per_unit[name] * per_launch_units / avg_s / 1e12
        peak = peaks["fp64_tflops"]
        peak_source = (f"measured: FP64 DFMA microbenchmark on this GPU ({peaks['sms']} SMs, "
                       f"median SM clock {peaks['sm_mhz_median']} MHz)")
    # the same kernel against HBM (the metric's "% HBM peak"), from its
    # algorithmic bytes, where the bound above is the FP64 pipe
    hbm_extra = {}
    if bound == "alu" and name in BYTES_PER_UNIT:
        hbm_gbs = BYTES_PER_UNIT[name] * per_launch_units / avg_s / 1e9
        hbm_peak = measured_peaks().get("hbm_gbs", 6800.0)
        hbm_extra = {"hbm_achieved_gbs": hbm_gbs, "hbm_frac": hbm_gbs / hbm_peak,
                     "hbm_bytes_per_unit": BYTES_PER_UNIT[name]}
    launches = sum(v[0] for k, v in prof.items())
    try:                                         # fused D2Q9 kernels only
        tile_height = P.dugks_tile_height(solver.ctx)
    except Exception:
        tile_height = None
    line = {
        "metric": "G cell-velocity updates/s (T3S3 step)", "value": value,
        "unit": "G updates/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None,
        "dtype": {"fp64": "f64", "fp32": "f32 (f32 deviation storage)",
                  "bf16": "f32 (bf16 deviation storage)",
                  "f64dw": "f32 pairs (f64 storage, double-word arithmetic)"}[args.storage],
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "cells": f"{nx}x{ny}", "scheme": args.scheme.upper(),
                   "velocities": ("D2Q9" if c.get("vel") != "nc"
                                  else f"Newton-Cotes {c['nv1']}x{c['nv1']}"),
                   "bc": ("bounce-back walls, moving lid" if c.get("vel") != "nc"
                          else "diffuse walls, moving lid"),
                   **({"Re": 1000, "Ma": 0.1} if c.get("vel") != "nc" else {"Kn": c.get("Kn")}),
                   "units_per_step": units, "l2": "flushed (256 MiB write) before every timed step",
                   "parallelism": f"replicas{world}" if world > 1 else "single",
                   **({"tile_height": tile_height} if tile_height else {}),
                   **({"kernel_path": args.path} if args.path != "auto" else {})},
        "roofline": {"bound": bound, "kernel": name, "achieved": achieved, "peak": peak,
                     "unit": unit, "frac": achieved / peak,
                     "traffic": (TRAFFIC_BYTES_PER_UNIT[name] * per_launch_units
                                 if name in TRAFFIC_BYTES_PER_UNIT else None),
                     "peak_source": peak_source,
                     "kernel_ms_per_launch": avg_s * 1e3,
                     "kernel_share": kms / sum(v[1] for v in prof.values()),
                     **hbm_extra},
        "kernels": {k: {"launches": v[0], "ms": round(v[1], 4)} for k, v in prof.items() if v[0]},
        "e2e": {"value": e2e, "unit": "G updates/s",
                "h2d_bytes_per_step": int(fh.nbytes), "d2h_bytes_per_step": int(sum(m.nbytes for m in mh))},
        "gpu_launches": int(launches), "stable": ok, "wall_s": t_wall,
    }
    line["alu_peaks"] = peaks
    if forms:
        line["forms"] = forms
    line.update(extra)
    if clk:
        line["clocks"] = clk
    if not args.no_cpu_baseline and world == 1:
        r1, d1, t1, _ = cpu_oracle_rate(10_000, budget_s=min(args.cpu_budget, 8.0))
        rate, done, secs, cores, per = cpu_oracle_all_cores(10_000, args.cpu_budget)
        line["cpu_baseline"] = {
            "value": rate / 1e9, "unit": "G updates/s", "cores": cores, "kind": "oracle",
            "cpu_model": cpu_model(),
            "sample": (f"{cores} spawned single-threaded processes, each running full T3S3 "
                       f"steps of {WORKLOAD} from rest for {args.cpu_budget:.0f} s "
                       f"({done} steps in all); rate = sum of the processes' rates"),
            "single_core": {"value": r1 / 1e9, "steps": d1, "seconds": round(t1, 2)},
            "per_process_min_max": [min(per) / 1e9, max(per) / 1e9]}
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--workload", default=WORKLOAD,
                    help="cavityN (N^2 D2Q9 cavity); the default is the reported workload")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--path", default="auto", choices=list(PATHS),
                    help="kernel path of dugks_init_ex (auto: fused D2Q9 or optimised "
                         "generic; generic: optimised generic for every set; reference: the "
                         "FP64 kernels that also run the T2 schemes)")
    ap.add_argument("--scheme", default="t3s3", choices=list(SCHEMES),
                    help="time scheme (T2S3/T2S2: the second-order comparison schemes, "
                         "generic FP64 kernels; the step they time is a T2 step)")
    ap.add_argument("--storage", default="fp64", choices=["fp64", "fp32", "bf16", "f64dw"],
                    help="storage form of the measured line (default FP64)")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the FP32/BF16 deviation-storage forms")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the rarefied128 FP32 and batched64 sub-lines")
    args = ap.parse_args()
    globals()["WORKLOAD"] = args.workload
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched64":
        return run_batched(args)
    if args.workload == "adjoint128":
        return run_adjoint(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
