#!/usr/bin/env python3
"""Benchmark of the batched PSATD push on one GB300.

Workload (default): the 'local' decomposition of a 512^3 periodic domain into
8x8x8 sub-domains of 64^3 cells, each padded with 16 guard cells per face
(512 FFT boxes of 96^3), stencil order p = 32, FP32 fields with FP64-generated
tables, vacuum, Gaussian laser pulse (lambda = 16, waist 32, duration 20
cells) travelling along +x, dt = 0.9.  One step = S1 forward FFT of E, B on
every box, S2 k-space update, S3 inverse FFT, S4 guard exchange.

Metric: interior cell-steps per second (512^3 interior cells per step).
Inputs (10.9 GB of fields) are far larger than L2, so no flush is needed.

``--impl reference`` times the FP64 CPU oracle on a bounded sample of the
same workload on the host cores instead.

Multi-GPU: the push shards into independent replicas (one plan per GPU, no
data-path collective); ``value`` is the sum over ranks.
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

METRIC = "PSATD cell-steps/s, FP32-batched vs FP64-plain at stated L2 err; % HBM roofline"
UNIT = "cell-steps/s"
FALLBACK_HBM = 6800.0

WORKLOADS = {
    # name: (layout builder args, dt, p)
    "local_512": dict(kind="local", global_n=(512, 512, 512), nsub=(8, 8, 8), ng=16, p=32, dt=0.9, steps=400),
    # small case of the same kernels (8 boxes of 96^3) for detailed profiles
    "local_128": dict(kind="local", global_n=(128, 128, 128), nsub=(2, 2, 2), ng=16, p=32, dt=0.9),
    "hybrid_1024": dict(kind="hybrid", global_n=(1024, 256, 256), nsub=(4, 1, 1), ng=64, p=64, dt=0.9,
                        steps=200),
    "local_1024": dict(kind="local", global_n=(1024, 256, 256), nsub=(16, 4, 4), ng=64, p=64, dt=0.9,
                       steps=200),
    # the other synthetic configurations (seeded inputs from inputs.make_workload);
    # their lines add the error against the analytic solution or the FP64 GPU push
    "plane_waves_32": dict(kind="config", precision=64),
    "sources_128": dict(kind="config", precision=32),
    "uneven_300": dict(kind="config", precision=32),
}


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("gpu", "reference"), default="gpu")
    ap.add_argument("--workload", default="local_512", choices=sorted(WORKLOADS))
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--precision", type=int, choices=(32, 64), default=None,
                    help="override the precision of a configuration workload")
    ap.add_argument("--pencil", action="store_true",
                    help="run the boxes the plane kernels would take on the pencil kernels")
    ap.add_argument("--autotune", action="store_true",
                    help="choose the kernel family and launch knobs by measurement (cached per layout)")
    ap.add_argument("--no-errors", action="store_true",
                    help="skip the error check against the reference (the configuration's full step count)")
    return ap.parse_args(argv)


# ----------------------------------------------------------------------------
# distributed plumbing (replicas only)
# ----------------------------------------------------------------------------

def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")),
            int(os.environ.get("WORLD_SIZE", "1")))


def dist_init(backend):
    import torch.distributed as dist
    rank, local, world = dist_env()
    if world > 1 and not dist.is_initialized():
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        os.environ.setdefault("MASTER_PORT", "29511")
        dist.init_process_group(backend, rank=rank, world_size=world)
    return rank, local, world


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


def reduce_max(x: float, device=None) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def total_units(per_rank: float, world: int) -> float:
    """Weak scaling: every rank processes the same workload."""
    return per_rank * world


# ----------------------------------------------------------------------------
# helpers
# ----------------------------------------------------------------------------

def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    except Exception:
        return FALLBACK_HBM, "fallback 6.8 TB/s (no MEASURED_PEAKS.json)"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = []
        with open(self.path) as fh:
            for line in fh:
                p = [x.strip() for x in line.split(",")]
                if len(p) >= 9:
                    rows.append(p)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        top = max(sm) if sm else 0
        under = [s for s in sm if s >= 0.5 * top] or sm
        return {"sm_mhz": statistics.median(under) if under else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows),
                "power_w_max": max((float(r[3]) for r in rows if _isnum(r[3])), default=None)}


def _isnum(s):
    try:
        float(s)
        return True
    except ValueError:
        return False


def build_layout(name):
    from paper_1812_07357_gb300 import inputs as I
    w = WORKLOADS[name]
    if w["kind"] == "local":
        return I.local_layout(w["global_n"], w["nsub"], w["ng"], w["p"])
    return I.hybrid_layout(w["global_n"], w["nsub"], w["ng"], w["p"])


def workload_config(name, lay, w, world):
    """The ``config`` object of a line: the workload alone (both arms)."""
    return {"workload": name, "decomposition": lay.kind,
            "global_n": list(lay.global_n), "boxes": len(lay.boxes),
            "box_n": list(lay.boxes[0].n), "ng": lay.boxes[0].ng_lo[0],
            "order_p": lay.boxes[0].p, "dt": w["dt"], "tables": "f64-generated",
            "interior_cells": lay.interior_cells, "padded_cells": lay.cells,
            "l2": "inputs larger than L2 (%.1f GB of fields)" % (6 * lay.cells * 4 / 1e9),
            "parallelism": "replicas" if world > 1 else "1 GPU"}


def kernel_bytes(layout, s=4, fin=6, fout=6, fused=True, guard_frac=1.0):
    """Compulsory bytes of one launch of every kernel kind (each kernel reads
    its inputs once and writes its outputs once).  Kinds: forward x(+y),
    generic y forward, z + update, generic y inverse, inverse (y+)x, exchange.
    On the fast path the y passes are fused into the x kernels, so kinds 0 and
    4 carry the plane kernels' bytes and kinds 1 and 3 do not launch; its z
    kernel stores the interior z planes only, and with `fused` the inverse
    plane kernel also writes the guard cells its plane feeds (the exchange
    kind then does not launch) -- in the fraction `guard_frac` of its launches
    (the deferred exchange stores them in the last step of a push only; the
    forward pass reads every padded cell either way)."""
    C = sum(b.cells for b in layout.boxes)
    M = sum((b.n[0] // 2 + 1) * b.n[1] * b.n[2] for b in layout.boxes)
    Mz = sum((b.n[0] // 2 + 1) * b.n[1] * b.interior[2] for b in layout.boxes)
    Mr = sum((b.n[0] // 2 + 1) * b.interior[1] * b.interior[2] for b in layout.boxes)
    I_ = layout.interior_cells
    G = layout.guard_cells
    c = 2 * s
    return {"generic": [fin * (C * s + M * c),          # k_fwd_x: real in, half spectrum out
                        fin * 2 * M * c,                # k_col forward along y (in place)
                        (fin + fout) * M * c,           # k_z_update
                        fout * 2 * Mz * c,              # k_col inverse along y (interior z)
                        fout * (Mr * c + I_ * s),       # k_inv_x (interior rows, cells)
                        fout * 2 * G * s],              # k_exchange: read interior, write guard
            "fast": [fin * (C * s + M * c),             # plane forward: real plane in, spectrum out
                     0,
                     fin * M * c + fout * Mz * c,       # z kernel: all planes in, interior z out
                     0,
                     fout * (Mz * c + I_ * s + (guard_frac * G * s if fused else 0)),   # plane inverse
                     fout * 2 * G * s]}


def step_algorithmic_bytes(layout, s=4, fin=6, fout=6):
    """Minimal bytes of one step: every padded cell of every field read once
    and written once, plus one write per guard cell and output field."""
    return fin * layout.cells * s + fout * layout.cells * s + fout * layout.guard_cells * s


# ----------------------------------------------------------------------------
# GPU arm
# ----------------------------------------------------------------------------

def run_config(args):
    """One of the other synthetic configurations on one GPU: the config's own
    step count is pushed once from the seeded initial state and compared with
    its reference (32^3 plane waves: the analytic solution; with sources: the
    library's FP64 push of the same inputs -- for a single periodic box one
    step of the whole interval, equal to the stepped result for a
    time-constant current; the FP64 GPU pushes are held to the oracle by the
    tests); then K steps are timed as one multi-step push (replayed CUDA
    graph) after W warm-up steps."""
    import numpy as np
    import torch
    from paper_1812_07357_gb300 import _abi as A
    from paper_1812_07357_gb300 import build as B
    from paper_1812_07357_gb300 import inputs as I
    from paper_1812_07357_gb300.solver import Plan

    B.build()
    A.load()
    w = I.make_workload(args.workload)
    prec = args.precision or WORKLOADS[args.workload]["precision"]
    lay = w.layout
    fields = w.fields
    src = w.src
    if prec == 32:
        fields = {k: I.round_to(v, np.float32) for k, v in fields.items()}
        src = {k: I.round_to(v, np.float32) for k, v in src.items()}
    # the source workloads keep J constant in time: its spectrum is computed once per push call
    tune = None
    if args.autotune:
        from paper_1812_07357_gb300 import autotune as AT
        tune = AT.tune(lay, w.h, w.dt, precision=prec, sources=w.sources, c=w.c, eps0=w.eps0,
                       j_constant=w.sources != "vacuum")
        plan = Plan(lay, w.h, w.dt, c=w.c, eps0=w.eps0, precision=prec, sources=w.sources,
                    j_constant=w.sources != "vacuum", tuning=tune["tuning"] or None,
                    **AT.family_kwargs(tune["family"]))
    else:
        plan = Plan(lay, w.h, w.dt, c=w.c, eps0=w.eps0, precision=prec, sources=w.sources, pencil=args.pencil,
                    j_constant=w.sources != "vacuum")
    errors = None
    if not args.no_errors:
        df = plan.pack_fields(fields)
        ds = plan.pack_fields(src) if w.sources != "vacuum" else None
        plan.push(df, ds, w.steps)
        plan.sync()
        got = plan.unpack_fields(df)
        if w.sources == "rho":
            got["rho"] = plan.unpack(ds["rho"])
        ref64 = None
        if w.sources != "vacuum":
            # the FP64 GPU push of the same (FP32-rounded) inputs: a single
            # periodic box in one step of the whole interval; self-periodic
            # boxes (guards refilled from their own interiors every step) in
            # the config's steps
            one = lay.kind == "global"
            p64 = Plan(lay, w.h, w.dt * (w.steps if one else 1), c=w.c, eps0=w.eps0, precision=64,
                       sources=w.sources, j_constant=True)
            d64 = p64.pack_fields(fields)
            s64 = p64.pack_fields(src)
            p64.push(d64, s64, 1 if one else w.steps)
            p64.sync()
            ref64 = p64.unpack_fields(d64)
            if w.sources == "rho":
                ref64["rho"] = p64.unpack(s64["rho"])
            p64.close()
        errors = _config_errors(args.workload, w, lay, got, I, ref64)
    df = plan.pack_fields(fields)
    ds = plan.pack_fields(src) if w.sources != "vacuum" else None
    plan.push(df, ds, args.warmup)
    plan.sync()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(plan.stream):
        e0.record(plan.stream)
        plan.push(df, ds, args.steps)
        e1.record(plan.stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    launches = plan.last_launch_count()
    # per-kernel split from a few more steps with launch-level events (no graph)
    A.psatd_plan_set_timing(plan.handle, True)
    A.psatd_plan_kernel_times(plan.handle)
    plan.push(df, ds, 3)
    plan.sync()
    kms, kn = A.psatd_plan_kernel_times(plan.handle)
    A.psatd_plan_set_timing(plan.handle, False)
    kernels = {A.KERNEL_NAMES[i]: {"launches": kn[i], "ms_per_step": kms[i] / 3} for i in range(len(kms)) if kn[i]}
    plan.close()
    fin, fout = {"vacuum": (6, 6), "J": (9, 6), "rho": (10, 7)}[w.sources]
    s = prec // 8
    sab = step_algorithmic_bytes(lay, s=s, fin=fin, fout=fout)
    step_ms = ms / args.steps
    peak, peak_src = measured_peaks()
    out = {"metric": METRIC, "value": lay.interior_cells * args.steps / (ms / 1e3), "unit": UNIT, "n_gpus": 1,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f%d" % prec, "data": "synthetic",
           "config": {"workload": args.workload, "decomposition": lay.kind, "boxes": len(lay.boxes),
                      "interior_cells": lay.interior_cells, "padded_cells": lay.cells, "form": w.sources,
                      "config_steps": w.steps, "dt": w.dt, "launch": "one multi-step push (CUDA graph)"},
           "step_roofline": {"bound": "hbm", "algorithmic_bytes_per_step": sab,
                             "achieved": sab / (step_ms / 1e3) / 1e9, "peak": peak, "unit": "GB/s",
                             "frac": sab / (step_ms / 1e3) / 1e9 / peak, "peak_source": peak_src},
           "gpu_launches": launches, "kernels": kernels, "errors": errors,
           "tuning": {"family": tune["family"], "knobs": tune["tuning"], "cached": tune["cached"],
                      "trials": len(tune["trials"])} if tune else None}
    print(json.dumps(out), flush=True)


def _config_errors(name, w, lay, got, I, ref64=None):
    """Relative L2 and max-norm errors per field vector over interior cells."""
    import numpy as np
    if ref64 is not None:
        ref = ref64
        ref_name = ("FP64 GPU push of the same inputs, one step of %d dt" % w.steps if lay.kind == "global"
                    else "FP64 GPU push of the same inputs, %d steps" % w.steps)
    elif name == "plane_waves_32":
        n = lay.global_n
        waves = I.plane_wave_set(seed=1, mmax=min(6, n[0] // 2 - 2))
        f = I.plane_wave_fields(waves, n, w.h, w.c, w.dt * w.steps)
        ref = {k: I.scatter_global(v, lay) for k, v in f.items()}
        ref_name = "analytic solution at t = %g" % (w.dt * w.steps)
    else:
        raise KeyError(name)
    out = {"reference": ref_name}
    groups = {"E": ("Ex", "Ey", "Ez"), "B": ("Bx", "By", "Bz")}
    if "rho" in got:
        groups["rho"] = ("rho",)
    inner = lambda b: tuple(slice(b.ng_lo[d], b.n[d] - b.ng_hi[d]) for d in (2, 1, 0))
    for g, comps in groups.items():
        d2 = r2 = dm = rm = 0.0
        for k in comps:
            for b, x, y in zip(lay.boxes, got[k], ref[k]):
                xi, yi = x[inner(b)], y[inner(b)]
                d2 += float(np.sum((xi - yi) ** 2))
                r2 += float(np.sum(yi ** 2))
                dm = max(dm, float(np.abs(xi - yi).max()))
                rm = max(rm, float(np.abs(yi).max()))
        out[g] = {"rel_l2": (d2 / r2) ** 0.5 if r2 > 0 else d2 ** 0.5, "max_norm": dm / rm if rm > 0 else dm}
    return out


def run_gpu(args):
    import torch
    rank, local, world = dist_init("nccl" if int(os.environ.get("WORLD_SIZE", "1")) > 1 else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_1812_07357_gb300 import _abi as A
    from paper_1812_07357_gb300 import build as B
    from paper_1812_07357_gb300 import inputs as I
    from paper_1812_07357_gb300.solver import Plan

    if rank == 0 or world == 1:
        B.build()
    barrier()
    A.load()
    lay = build_layout(args.workload)
    w = WORKLOADS[args.workload]
    h = (1.0, 1.0, 1.0)
    tune = None
    if args.autotune:
        from paper_1812_07357_gb300 import autotune as AT
        tune = AT.tune(lay, h, w["dt"], precision=32, sources="vacuum")
        plan = Plan(lay, h, w["dt"], precision=32, sources="vacuum", tuning=tune["tuning"] or None,
                    **AT.family_kwargs(tune["family"]))
    else:
        plan = Plan(lay, h, w["dt"], precision=32, sources="vacuum", pencil=args.pencil)
    fac = I.laser_box_factors(lay, h)
    fields = {k: plan.pack_separable(fac[k]) for k in I.COMPONENTS}
    plan.guard_exchange(fields)
    plan.sync()
    stream = plan.stream

    plan.push(fields, None, args.warmup)
    plan.sync()

    clocks = ClockSampler(local).start() if rank == 0 else None
    barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    # the K timed steps are one push, launched as the product runs it (one
    # replayed CUDA graph per step variant; with the deferred exchange each
    # step's guard exchange is done by the next step's forward gather and the
    # last step stores the guards)
    with torch.cuda.stream(stream):
        e0.record(stream)
        plan.push(fields, None, args.steps)
        e1.record(stream)
    launches = plan.last_launch_count()
    torch.cuda.synchronize()
    barrier()
    ms = e0.elapsed_time(e1)
    ms_max = reduce_max(ms, dev if world > 1 else None)
    # per-kernel device times: a second push of the same K steps with CUDA
    # events recorded around every launch on the plan's stream (direct
    # launches; the kernels are the same as in the graph)
    A.psatd_plan_set_timing(plan.handle, True)
    A.psatd_plan_kernel_times(plan.handle)
    plan.push(fields, None, args.steps)
    kms, kn = A.psatd_plan_kernel_times(plan.handle)
    A.psatd_plan_set_timing(plan.handle, False)
    clk = clocks.stop() if clocks else None

    interior = lay.interior_cells
    value = total_units(interior * args.steps, world) / (ms_max / 1e3)
    peak, peak_src = measured_peaks()
    gfrac = 1.0 / args.steps if plan.deferred_exchange else 1.0
    kb = kernel_bytes(lay, fused=kn[5] == 0, guard_frac=gfrac)["fast" if plan.fast_boxes == len(lay.boxes) else "generic"]
    avg = [kms[i] / kn[i] if kn[i] else 0.0 for i in range(len(kms))]
    dom = max(range(len(avg)), key=lambda i: avg[i])
    ach = kb[dom] / (avg[dom] / 1e3) / 1e9
    step_ms = ms_max / args.steps
    sab = step_algorithmic_bytes(lay)
    traffic = _ncu_traffic(A.KERNEL_NAMES[dom], args.workload)

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": workload_config(args.workload, lay, w, world),
        "plan": {"fast_boxes": plan.fast_boxes,
                 "guard_exchange": "deferred into the next step's forward gather; guards stored by the last step"
                                   if plan.deferred_exchange else "stored every step"},
        "roofline": {"bound": "hbm", "kernel": A.KERNEL_NAMES[dom], "achieved": ach,
                     "peak": peak, "unit": "GB/s", "frac": ach / peak, "traffic": traffic,
                     "algorithmic_bytes_per_launch": kb[dom], "avg_launch_ms": avg[dom],
                     "peak_source": peak_src,
                     "step_frac": sab / (step_ms / 1e3) / 1e9 / peak},
        "step_roofline": {"algorithmic_bytes_per_step": sab,
                          "achieved": sab / (step_ms / 1e3) / 1e9, "peak": peak, "unit": "GB/s",
                          "frac": sab / (step_ms / 1e3) / 1e9 / peak, "peak_source": peak_src},
        "kernels": {A.KERNEL_NAMES[i]: {"launches": kn[i], "total_ms": kms[i], "avg_ms": avg[i],
                                        "bytes_per_launch": kb[i],
                                        "gbps": (kb[i] / (avg[i] / 1e3) / 1e9) if avg[i] else None,
                                        "frac": (kb[i] / (avg[i] / 1e3) / 1e9 / peak) if avg[i] else None}
                    for i in range(len(kms))},
        "kernel_timing": "second push of the same K steps, CUDA events around every launch on the plan's stream",
        "gpu_launches": launches,
        "tuning": {"family": tune["family"], "knobs": tune["tuning"], "cached": tune["cached"],
                   "trials": len(tune["trials"])} if tune else None,
        "clocks": clk,
        "memory": dict(zip(("field_bytes", "workspace_bytes"), A.psatd_plan_memory(plan.handle))),
    }
    if not args.no_e2e:
        out["e2e"] = run_e2e(plan, fields, args, lay, world)
    if not args.no_errors and w.get("steps"):
        # the headline's stated error: the configuration's full step count
        # from the initial laser, against the global single-box FP64 result
        out["errors"] = global_reference_errors(lay, w, w["steps"], plan=plan)
    if rank == 0 and world == 1 and not args.no_fp64:
        out["fp64_plain"] = run_fp64_plain(lay, w, fac)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = oracle_sample(lay, w, fac, target_s=12.0)
    plan.close()
    if rank == 0:
        print(json.dumps(out), flush=True)


def global_reference_errors(lay, w, steps, plan=None, fields=None, pencil=False):
    """Error of the FP32 batched push of a local or hybrid workload after the
    configuration's `steps` against the global single-box FP64 solution of the
    same domain (paper Sec. 1.3: the guard truncation error is what the local
    decomposition trades for its independent FFTs).

    The reference is one step of steps * dt on one periodic box of the whole
    domain, FP64, on the library's generic kernels: the update is the exact
    solution of every mode in vacuum, so one step of n dt equals n steps of dt
    (the semigroup property, a pin of the oracle; the generic FP64 kernels at
    these lengths are held to the oracle by the GPU tests).  Both runs start
    from the laser rounded to FP32.  Relative L2 and max-norm per field
    vector over every interior cell of every box, computed on the GPU."""
    import torch
    from paper_1812_07357_gb300 import inputs as I
    from paper_1812_07357_gb300.solver import Plan
    h = (1.0, 1.0, 1.0)
    own = plan is None
    if own:
        plan = Plan(lay, h, w["dt"], precision=32, sources="vacuum", pencil=pencil)
    fac = I.laser_box_factors(lay, h)
    fields = {k: plan.pack_separable(fac[k]) for k in I.COMPONENTS}
    plan.guard_exchange(fields)
    t0 = time.perf_counter()
    plan.push(fields, None, steps)
    plan.sync()
    t_local = time.perf_counter() - t0
    glay = I.global_layout(lay.global_n, lay.boxes[0].p)
    gplan = Plan(glay, h, w["dt"] * steps, precision=64, sources="vacuum")
    gfac = I.laser_box_factors(glay, h)
    gf = {k: gplan.pack_separable(gfac[k]).float().double() for k in I.COMPONENTS}
    gplan.push(gf, None, 1)
    gplan.sync()
    gn = lay.global_n
    groups = {"E": ("Ex", "Ey", "Ez"), "B": ("Bx", "By", "Bz")}
    out = {"reference": "global single-box %dx%dx%d FP64, one step of %d dt (GPU generic kernels)"
                        % (gn[0], gn[1], gn[2], steps), "steps": steps, "push_s": t_local}
    for g, comps in groups.items():
        num = den = 0.0
        dmax = rmax = 0.0
        for k in comps:
            G = gf[k].view(gn[2], gn[1], gn[0])
            L = fields[k]
            for (off, n), b in zip(plan.offsets, lay.boxes):
                a = L[off:off + n].view(b.n[2], b.n[1], b.n[0])
                lo, m = b.ng_lo, b.interior
                ai = a[lo[2]:lo[2] + m[2], lo[1]:lo[1] + m[1], lo[0]:lo[0] + m[0]].double()
                o = b.origin
                r = G[o[2]:o[2] + m[2], o[1]:o[1] + m[1], o[0]:o[0] + m[0]]
                d = ai - r
                num += float((d * d).sum())
                den += float((r * r).sum())
                dmax = max(dmax, float(d.abs().max()))
                rmax = max(rmax, float(r.abs().max()))
        out[g] = {"rel_l2": (num / den) ** 0.5 if den > 0 else num ** 0.5,
                  "max_norm": dmax / rmax if rmax > 0 else dmax}
    gplan.close()
    del gf
    if own:
        plan.close()
    del fields
    torch.cuda.empty_cache()
    return out


def _global_host_fields(lay):
    """The workload's initial fields as whole-domain page-locked host arrays
    (the laser's separable factors multiplied out on the GPU, then copied)."""
    import torch
    from paper_1812_07357_gb300 import inputs as I
    glay = I.global_layout(lay.global_n, lay.boxes[0].p)
    fac = I.laser_box_factors(glay, (1.0,) * 3)
    gn = lay.global_n
    out = {}
    for k in I.COMPONENTS:
        if fac[k] is None:
            t = torch.zeros(gn[0] * gn[1] * gn[2], dtype=torch.float32)
        else:
            fz, fy, fx, d = fac[k][0]
            z, y, x = (torch.from_numpy(v).cuda() for v in (fz, fy, fx))
            t = ((z.view(-1, 1, 1) * y.view(1, -1, 1) * x.view(1, 1, -1)) / d).float().reshape(-1).cpu()
        out[k] = t.pin_memory()
    return out


def host_link_rates(nbytes=1 << 30):
    """Copy rates between page-locked host memory and the device: one
    cudaMemcpyAsync of nbytes each way (torch's copy of a pinned tensor),
    best of 3 after one warm-up.  No host path can copy faster."""
    import torch
    h = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
    d = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    s = torch.cuda.Stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    out = {}
    for name, dst, src in (("h2d_gbs", d, h), ("d2h_gbs", h, d)):
        best = float("inf")
        for r in range(4):
            with torch.cuda.stream(s):
                e0.record(s)
                dst.copy_(src, non_blocking=True)
                e1.record(s)
            s.synchronize()
            if r > 0:
                best = min(best, e0.elapsed_time(e1))
        out[name] = nbytes / (best * 1e6)
    del h, d
    return out


def run_e2e(plan, fields, args, lay, world):
    """Same metric end to end through the C ABI with HOST buffers: every step
    copies the six field components of the whole domain from page-locked host
    memory to the device, scatters them into the padded boxes, pushes one
    step, gathers the box interiors back and copies the domain to the host
    (psatd_push_host_global); the copies are inside the timed region.  Also
    timed: the other host copy mode, and the host path that keeps the padded
    boxes on the host (psatd_push_host, 3.4x the bytes)."""
    import torch
    from paper_1812_07357_gb300 import _abi as A
    stream = plan.stream
    host = _global_host_fields(lay)
    plan.push_host_global(host, host, None, 1)   # first call allocates the staging buffers
    torch.cuda.synchronize()
    nb = sum(v.numel() * v.element_size() for v in host.values())

    def timed_steps(fn, buf):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            e0.record(stream)
            for _ in range(args.e2e_steps):
                fn(buf, buf, None, 1)
            e1.record(stream)
        torch.cuda.synchronize()
        return reduce_max(e0.elapsed_time(e1), torch.device("cuda", torch.cuda.current_device())
                          if world > 1 else None)

    link = host_link_rates()
    rate = lambda ms: total_units(lay.interior_cells * args.e2e_steps, world) / (ms / 1e3)
    names = {1: "copy kernel through the host buffers' device mapping", 0: "copy engines"}
    mode = A.psatd_plan_tuning(plan.handle, A.PSATD_TUNE_HOST_COPY)
    ms = timed_steps(plan.push_host_global, host)          # the plan's default copy mode
    A.psatd_plan_tune(plan.handle, A.PSATD_TUNE_HOST_COPY, 1 - mode)
    ms_other = timed_steps(plan.push_host_global, host)
    A.psatd_plan_tune(plan.handle, A.PSATD_TUNE_HOST_COPY, mode)
    del host
    boxes = {k: torch.empty(v.shape, dtype=v.dtype, pin_memory=True) for k, v in fields.items()}
    for k in boxes:
        boxes[k].copy_(fields[k])
    plan.push_host(boxes, boxes, None, 1)
    torch.cuda.synchronize()
    ms_boxes = timed_steps(plan.push_host, boxes)
    nbb = sum(v.numel() * v.element_size() for v in boxes.values())
    return {"value": rate(ms), "unit": UNIT, "h2d_bytes_per_step": nb, "d2h_bytes_per_step": nb,
            "steps": args.e2e_steps, "ms_per_step": ms / args.e2e_steps,
            "api": "psatd_push_host_global (whole-domain host arrays), " + names[mode],
            "other_copy_mode": {"copies": names[1 - mode], "ms_per_step": ms_other / args.e2e_steps,
                                "value": rate(ms_other)},
            "padded_boxes_on_host": {"api": "psatd_push_host, " + names[mode], "ms_per_step": ms_boxes / args.e2e_steps,
                                     "value": rate(ms_boxes), "h2d_bytes_per_step": nbb, "d2h_bytes_per_step": nbb},
            "host_link": {"h2d_gbs": link["h2d_gbs"], "d2h_gbs": link["d2h_gbs"],
                          "copy_ms_per_step": nb / (link["h2d_gbs"] * 1e6) + nb / (link["d2h_gbs"] * 1e6),
                          "what": "1 GiB cudaMemcpyAsync each way from page-locked memory; every input copy of "
                                  "a step precedes its z pass and every result copy follows it, so "
                                  "copy_ms_per_step plus the z pass bounds ms_per_step from below"}}


def run_fp64_plain(lay, w, fac, nsteps=2):
    """Plain FP64 GPU push: the same kernels in double, one box per push call
    (no batching), over every box of the workload.  All boxes share one shape,
    so one single-box plan (self-periodic box, direct launches) pushes each
    box's own field buffers in turn; the timed region covers all boxes."""
    import torch
    from paper_1812_07357_gb300 import inputs as I
    from paper_1812_07357_gb300.solver import Plan
    box = lay.boxes[0]
    assert all(b.n == box.n and b.p == box.p for b in lay.boxes)
    sub = I.Layout("independent", (0, 0, 0), (1, 1, 1), [box])
    plan = Plan(sub, (1.0,) * 3, w["dt"], precision=64, sources="vacuum", no_graph=True)
    per_box = []
    for b in range(len(lay.boxes)):
        per_box.append({k: plan.pack_separable([fac[k][b]] if fac[k] is not None else None)
                        for k in I.COMPONENTS})
    plan.push(per_box[0], None, 1)
    plan.sync()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(plan.stream):
        e0.record(plan.stream)
        for f in per_box:
            plan.push(f, None, nsteps)
        e1.record(plan.stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    cells = sum(b.interior_cells for b in lay.boxes) * nsteps
    plan.close()
    del per_box
    torch.cuda.empty_cache()
    return {"value": cells / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / nsteps,
            "sample": f"all {len(lay.boxes)} boxes x {nsteps} steps, FP64, one box per push call "
                      "(unbatched, direct launches); guard exchange of a self-periodic box"}


def oracle_sample(lay, w, fac, target_s=12.0, max_boxes=64):
    """The FP64 oracle (as it stands) on a bounded sample: S1-S3 of whole
    boxes for one step, on the host cores."""
    import numpy as np
    from oracle import psatd_oracle as O
    from paper_1812_07357_gb300 import inputs as I
    boxes = []
    t0 = time.perf_counter()
    done = 0
    cells = 0
    while done < max_boxes and (done == 0 or (time.perf_counter() - t0) < target_s):
        b = done
        box = lay.boxes[b]
        f = {}
        for k in I.COMPONENTS:
            if fac[k] is None:
                f[k] = np.zeros(box.shape)
            else:
                fz, fy, fx, d = fac[k][b]
                f[k] = (fz[:, None, None] * fy[None, :, None] * fx[None, None, :]) / d
        f = I.round_to(f, np.float32)
        O.push_box(f, None, (1.0,) * 3, box.p, w["dt"], form="vacuum")
        done += 1
        cells += box.interior_cells
    dt = time.perf_counter() - t0
    return {"value": cells / dt, "unit": UNIT, "cores": O.threads(), "kind": "oracle",
            "sample": f"{done} of {len(lay.boxes)} boxes x 1 step (S1-S3 per box, FP64 C++ oracle "
                      f"with its own FFT, OpenMP), {dt:.1f} s"}


def kernel_source_digest():
    """SHA-256 over the CUDA/C++ sources of the library (sorted by name): a
    committed ncu traffic figure counts only for the sources it was taken on."""
    import hashlib
    d = os.path.join(ROOT, "paper_1812_07357_gb300", "csrc")
    h = hashlib.sha256()
    for name in sorted(os.listdir(d)):
        if name.endswith((".cu", ".cuh", ".h", ".cpp")):
            h.update(name.encode())
            with open(os.path.join(d, name), "rb") as fh:
                h.update(fh.read())
    return h.hexdigest()


def _ncu_traffic(kernel_name, workload):
    """Per-launch DRAM bytes of the dominant kernel from a committed ncu
    summary (profiles/<kernel>_<workload>.json), if one exists for the
    current kernel sources; else None."""
    base = kernel_name.split("(")[0]
    p = os.path.join(ROOT, "profiles", f"{base}_{workload}.json")
    try:
        with open(p) as fh:
            d = json.load(fh)
        if d.get("source_sha256") != kernel_source_digest():
            return None
        return d.get("dram_bytes_per_launch")
    except Exception:
        return None


# ----------------------------------------------------------------------------
# reference arm: the FP64 oracle on the host cores
# ----------------------------------------------------------------------------

def run_reference(args):
    rank, _, world = dist_env()
    if rank != 0:
        return
    from paper_1812_07357_gb300 import inputs as I
    lay = build_layout(args.workload)
    w = WORKLOADS[args.workload]
    fac = I.laser_box_factors(lay, (1.0,) * 3)
    for _ in range(args.warmup):
        oracle_sample(lay, w, fac, target_s=0.0, max_boxes=1)
    t0 = time.perf_counter()
    vals = []
    for _ in range(args.steps):
        r = oracle_sample(lay, w, fac, target_s=0.0, max_boxes=1)
        vals.append(r)
    dt = time.perf_counter() - t0
    cells = lay.boxes[0].interior_cells * args.steps
    value = cells / dt
    cb = {"value": value, "unit": UNIT, "cores": vals[0]["cores"], "kind": "oracle",
          "sample": f"1 of {len(lay.boxes)} boxes per step (S1-S3 of one box, FP64 C++ oracle, "
                    f"{vals[0]['cores']} OpenMP threads)"}
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "impl": "reference",
           "config": workload_config(args.workload, lay, w, world),
           "cpu_baseline": cb,
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main(argv=None):
    args = parse(argv)
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif WORKLOADS[args.workload]["kind"] == "config":
        run_config(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
