"""Group-size chooser for the hybrid decomposition on one GPU.

The paper (Sec. 2.4.1 - 2.4.3) picks the number of sub-domains per hybrid
group from a model of the FFT time fitted to measurements -- on its clusters
T_FFT = alpha n^3 log n / n_proc + beta n^3 / n_proc^(4/5), a compute term and
a network-transposition term -- and notes that the best group size lies
between the local solver (one sub-domain per group) and the global one.

On one GB300 there is no network: every group is one batched FFT box, and a
step costs, per box of N padded cells, a compute term in N log N and a
memory-traffic term in N, plus the guard exchange (cells G).  The chooser

* enumerates the candidate decompositions of nsub sub-domains with n_g guard
  cells: the local one and every hybrid grouping (m_d sub-domains merged per
  group along axis d, m_d dividing nsub_d; guards only on split axes), keeping
  those whose box sizes are valid FFT boxes;
* gives each one's memory (plan workspace and the caller's field buffers, from
  the plan) and, optionally, its measured time per step;
* fits T = a * sum_b N_b log2 N_b + b * sum_b N_b + c * G to the measured
  candidates by least squares (the analogue of the paper's alpha, beta fit);
* returns the fastest candidate within a memory budget.
"""
from __future__ import annotations

import dataclasses
import itertools
import math
from typing import List, Optional, Sequence

import numpy as np

from . import inputs as I

MAX_N = (1024, 512, 512)


@dataclasses.dataclass
class Candidate:
    name: str                        # "local" or "hybrid m0xm1xm2"
    merge: tuple                     # sub-domains per group along x, y, z
    layout: I.Layout
    padded_cells: int
    guard_cells: int
    nlogn: float                     # sum over boxes of N log2 N
    memory_bytes: Optional[int] = None
    ms_per_step: Optional[float] = None
    model_ms: Optional[float] = None


def _five_smooth(n: int) -> bool:
    for f in (2, 3, 5):
        while n % f == 0:
            n //= f
    return n == 1


def valid_box(n) -> bool:
    return all(v % 2 == 0 and _five_smooth(v) and 4 <= v <= MAX_N[d] for d, v in enumerate(n))


def candidates(global_n: Sequence[int], nsub: Sequence[int], ng: int, p: int,
               periodic=(1, 1, 1)) -> List[Candidate]:
    """The local decomposition and every hybrid grouping of its sub-domains."""
    out = []
    divisors = [[m for m in range(1, s + 1) if s % m == 0] for s in nsub]
    for merge in itertools.product(*divisors):
        groups = tuple(nsub[d] // merge[d] for d in range(3))
        if merge == (1, 1, 1):
            lay = I.local_layout(global_n, nsub, ng, p, periodic=periodic)
            name = "local"
        else:
            lay = I.hybrid_layout(global_n, groups, ng, p, periodic=periodic)
            name = "hybrid %dx%dx%d" % merge
        if not all(valid_box(b.n) for b in lay.boxes):
            continue
        cells = [b.cells for b in lay.boxes]
        out.append(Candidate(name, tuple(merge), lay, sum(cells), lay.guard_cells,
                             float(sum(c * math.log2(c) for c in cells))))
    return out


def measure(c: Candidate, h=(1.0, 1.0, 1.0), dt=0.9, precision=32, steps=3, warmup=2):
    """Time `steps` pushes of the candidate (after `warmup`) on zero fields;
    record the plan's memory.  Needs a CUDA device."""
    import torch
    from .solver import Plan
    plan = Plan(c.layout, h, dt, precision=precision, sources="vacuum")
    try:
        fields = {k: plan.empty() for k in I.COMPONENTS}
        plan.push(fields, None, warmup)
        plan.sync()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(plan.stream):
            e0.record(plan.stream)
            plan.push(fields, None, steps)
            e1.record(plan.stream)
        torch.cuda.synchronize()
        c.ms_per_step = e0.elapsed_time(e1) / steps
        c.memory_bytes = int(plan.workspace_bytes + 6 * plan.field_elems * (4 if precision == 32 else 8))
    finally:
        plan.close()
    return c


def fit(cands: Sequence[Candidate]):
    """Least-squares (a, b, c) of T = a sum N log2 N + b sum N + c G over the
    measured candidates (non-negative coefficients are not enforced)."""
    m = [c for c in cands if c.ms_per_step is not None]
    if len(m) < 3:
        raise ValueError("need at least three measured candidates")
    A = np.array([[c.nlogn, c.padded_cells, c.guard_cells] for c in m], dtype=np.float64)
    t = np.array([c.ms_per_step for c in m])
    scale = A.max(axis=0)
    scale[scale == 0] = 1.0
    coef, *_ = np.linalg.lstsq(A / scale, t, rcond=None)
    coef = coef / scale
    for c in cands:
        c.model_ms = float(np.dot(coef, [c.nlogn, c.padded_cells, c.guard_cells]))
    return coef


def choose(global_n, nsub, ng, p, budget_bytes: Optional[int] = None, precision=32, periodic=(1, 1, 1),
           run=True, **measure_kw):
    """Best candidate (fastest measured time, else smallest padded volume)
    within the memory budget, and the whole sorted report."""
    cands = candidates(global_n, nsub, ng, p, periodic)
    if run:
        for c in cands:
            measure(c, precision=precision, **measure_kw)
        if len(cands) >= 3:
            fit(cands)
    ok = [c for c in cands if budget_bytes is None or c.memory_bytes is None or c.memory_bytes <= budget_bytes]
    if not ok:
        raise ValueError("no candidate fits the memory budget")
    key = (lambda c: c.ms_per_step) if run else (lambda c: c.padded_cells)
    ok.sort(key=key)
    return ok[0], sorted(cands, key=key)
