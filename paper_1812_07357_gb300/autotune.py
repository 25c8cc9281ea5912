"""Autotuner: per layout (its box sizes, guard widths and stencil orders,
precision and equation form) choose the kernel family and the launch
parameters of a plan by measuring candidate plans on the GPU, and keep the
choice in a JSON cache so that the next plan of the same layout starts tuned.

The paper tunes its hybrid groups by experiment (Sec. 2.4.3: the best number
of ranks per group depends on the machine and the problem size) and leaves
the automation for later.  Here the per-box work of one GPU is what is
tuned:

* kernel family (``PSATD_*_KERNELS``): plane kernels, pencil kernels or
  generic kernels, for the boxes each family takes;
* ``reg_planes``: the register plane kernels for the FP32 boxes whose plane
  shape has them, or the family those boxes take without them;
* ``z_tile``: mx columns per z tile of the plane and pencil families (more,
  smaller CTAs for small boxes);
* ``pencil_rows_kb``: pencil batching -- the shared memory, hence the number
  of x rows, of one pencil CTA;
* ``z_prefetch``: the register z kernel's L2 prefetch distance;
* ``pencil_reg_z``: the register z kernel or the shared-memory one for the z
  pass of pencil boxes whose z length has both;
* ``z_one_launch``: those boxes' z pass in one persistent launch for every z
  length, or one launch per length.

The FFT radix order of every length is fixed at build time (two-pass
factorisations and prime-factor codelets per length), so it is not searched.

Search: one stage per parameter (family first, then every knob the chosen
family uses), each stage keeping the fastest; every trial is recorded.  The
cache key includes the device name.
"""
from __future__ import annotations

import hashlib
import json
import os
from typing import Callable, Dict, List, Optional, Tuple

from . import _abi as A

FAMILIES = ("default", "plane", "pencil", "generic")
KNOB_VALUES = {
    "reg_planes": (1, 0),
    "pencil_reg_z": (1, 0),
    "z_one_launch": (0, 1),
    "z_tile": {32: (8, 4, 2), 64: (4, 2)},
    "pencil_rows_kb": (16, 32, 64, 128),
    "z_prefetch": (0, 64, 152),
}


def default_cache() -> str:
    return os.environ.get("PSATD_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "psatd", "autotune.json"))


def signature(layout, precision: int, sources: str, nodal: bool = False, device: str = "") -> str:
    """Key of a tuning problem: the decomposition kind, the multiset of boxes
    (sizes, guards, orders), precision, form, variant and device."""
    boxes = sorted((tuple(b.n), tuple(b.ng_lo), tuple(b.ng_hi), int(b.p)) for b in layout.boxes)
    text = json.dumps([layout.kind, list(layout.global_n), list(layout.periodic), boxes, int(precision), sources,
                       bool(nodal), device])
    return hashlib.sha1(text.encode()).hexdigest()


def family_kwargs(family: str) -> Dict[str, bool]:
    return {"default": {}, "plane": {"plane": True}, "pencil": {"pencil": True},
            "generic": {"generic": True}}[family]


def search(measure: Callable[[str, Dict[str, int]], Tuple[float, Dict[str, int]]], precision: int):
    """Stage-wise search.  measure(family, tuning) -> (ms per step, the knobs
    the resulting plan uses with their values).  Returns (best family, best
    tuning, best ms, trials)."""
    trials = []

    def run(fam, tun):
        ms, used = measure(fam, tun)
        trials.append({"family": fam, "tuning": dict(tun), "ms_per_step": ms, "uses": sorted(used)})
        return ms, used

    best = None
    for fam in FAMILIES:
        ms, used = run(fam, {})
        if best is None or ms < best[2]:
            best = (fam, {}, ms, used)
    fam, tun, ms, used = best
    for knob in ("reg_planes", "pencil_reg_z", "z_one_launch", "z_tile", "pencil_rows_kb", "z_prefetch"):
        if knob not in used:                    # not used by the best plan so far
            continue
        values = KNOB_VALUES[knob][precision] if isinstance(KNOB_VALUES[knob], dict) else KNOB_VALUES[knob]
        for v in values:
            if used.get(knob) == v:
                continue                        # the best plan's own value: already measured
            t = dict(tun, **{knob: v})
            m, u = run(fam, t)
            if m < ms:
                tun, ms, used = t, m, u
    # keep only the knobs the chosen plan uses
    tun = {k: v for k, v in tun.items() if k in used}
    return fam, tun, ms, trials


def _load(path):
    try:
        with open(path) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def _store(path, data):
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    tmp = path + ".%d.tmp" % os.getpid()
    with open(tmp, "w") as fh:
        json.dump(data, fh, indent=1, sort_keys=True)
    os.replace(tmp, path)


def gpu_measure(layout, h, dt, *, precision=32, sources="vacuum", nodal=False, steps=3, warmup=2, c=1.0,
                eps0=1.0, j_constant=False):
    """A measure() for search(): builds each candidate plan, pushes `warmup`
    steps, then times `steps` steps (one push, CUDA events on the plan's
    stream) on zero fields (the kernels' time does not depend on the
    values)."""
    import torch
    from .solver import Plan

    def measure(family, tuning):
        plan = Plan(layout, h, dt, c=c, eps0=eps0, precision=precision, sources=sources, nodal=nodal,
                    j_constant=j_constant, tuning=tuning or None, **family_kwargs(family))
        try:
            f = {k: plan.empty() for k in ("Ex", "Ey", "Ez", "Bx", "By", "Bz")}
            s = None
            if sources != "vacuum":
                s = {k: plan.empty() for k in ("Jx", "Jy", "Jz")}
                s["rho"] = plan.empty() if sources == "rho" else None
            plan.push(f, s, warmup)
            plan.sync()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(plan.stream):
                e0.record(plan.stream)
                plan.push(f, s, steps)
                e1.record(plan.stream)
            torch.cuda.synchronize()
            return e0.elapsed_time(e1) / steps, plan.tuning()
        finally:
            plan.close()

    return measure


def tune(layout, h, dt, *, precision=32, sources="vacuum", nodal=False, cache: Optional[str] = None,
         measure: Optional[Callable] = None, device: Optional[str] = None, **measure_kw) -> Dict:
    """The tuned choice for a layout: from the cache, else measured (and
    stored).  Returns {"family", "tuning", "ms_per_step", "trials",
    "cached"}."""
    if device is None:
        import torch
        device = torch.cuda.get_device_name() if torch.cuda.is_available() else "cpu"
    key = signature(layout, precision, sources, nodal, device)
    path = cache or default_cache()
    data = _load(path)
    if key in data:
        return dict(data[key], cached=True)
    if measure is None:
        measure = gpu_measure(layout, h, dt, precision=precision, sources=sources, nodal=nodal, **measure_kw)
    fam, tun, ms, trials = search(measure, precision)
    entry = {"family": fam, "tuning": tun, "ms_per_step": ms, "trials": trials, "device": device,
             "boxes": len(layout.boxes)}
    data = _load(path)
    data[key] = entry
    _store(path, data)
    return dict(entry, cached=False)


def tuned_plan(layout, h, dt, *, precision=32, sources="vacuum", nodal=False, cache=None, **plan_kw):
    """A Plan with the tuned family and knobs of its layout (tuning it first
    when the cache has no entry)."""
    from .solver import Plan
    choice = tune(layout, h, dt, precision=precision, sources=sources, nodal=nodal, cache=cache,
                  c=plan_kw.get("c", 1.0), eps0=plan_kw.get("eps0", 1.0),
                  j_constant=plan_kw.get("j_constant", False))
    kw = dict(plan_kw)
    kw.update(family_kwargs(choice["family"]))
    return Plan(layout, h, dt, precision=precision, sources=sources, nodal=nodal,
                tuning=choice["tuning"] or None, **kw)
