"""Parity at the benchmark's full size and launch configuration.

The 512^3 periodic domain as 8 x 8 x 8 local sub-domains of 64^3 (512 FFT
boxes of 96^3, n_g = 16, p = 32, FP32, laser pulse), pushed by the same plan
the benchmark times (register-resident plane and z kernels, deferred guard
exchange: the first step reads the caller's guards, the middle steps gather
them from their owners' interiors, the last step stores them).  The oracle
cannot push 512 boxes in seconds, so:

* one step, sampled boxes: the interior of a box after one step depends only
  on that box's own padded data, so the oracle's one-box step of the box's
  FP32-rounded input must match the GPU interior;
* three steps (first, middle and last step variants), the strongest box: its
  interior after step 3 depends on the 27 boxes around it after step 2, and
  those on the 125 boxes around it after step 1.  The oracle pushes exactly
  that cone of boxes, each padded input assembled from the previous step's
  interiors of its owners (the guard exchange of Fig. 1, step (ii)), starting
  from the FP64 laser sampled at the boxes' global positions;
* the guard exchange at full size: after the 3-step push every cell of a
  sampled box, guards included, must equal the owning interior cell of the
  periodic global array, bit for bit (assembled from the 27 boxes around it).
"""
import itertools

import numpy as np
import pytest

from oracle import psatd_oracle as O
from paper_1812_07357_gb300 import inputs as I
from _parity import assert_fields

pytestmark = pytest.mark.gpu

GLOBAL_N, NSUB, NG, P, DT = (512, 512, 512), (8, 8, 8), 16, 32, 0.9
INNER = 64
H = (1.0, 1.0, 1.0)


def _push(nsteps):
    from paper_1812_07357_gb300.solver import Plan
    lay = I.local_layout(GLOBAL_N, NSUB, NG, P)
    plan = Plan(lay, H, DT, precision=32, sources="vacuum")
    assert plan.fast_boxes == len(lay.boxes) and plan.deferred_exchange
    fac = I.laser_box_factors(lay, H)
    fields = {k: plan.pack_separable(fac[k]) for k in I.COMPONENTS}
    plan.guard_exchange(fields)
    plan.push(fields, None, nsteps)
    plan.sync()
    return lay, plan, fac, fields


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1812_07357_gb300 import build
    build.build()
    return torch


def _box_input(lay, fac, b):
    box = lay.boxes[b]
    out = {}
    for k in O.COMPS:
        if fac[k] is None:
            out[k] = np.zeros(box.shape)
        else:
            fz, fy, fx, d = fac[k][b]
            out[k] = (fz[:, None, None] * fy[None, :, None] * fx[None, None, :]) / d
    return I.round_to(out, np.float32)


def _box_output(plan, fields, b):
    off, n = plan.offsets[b]
    shp = plan.layout.boxes[b].shape
    return {k: fields[k][off:off + n].view(*shp).cpu().numpy().astype(np.float64) for k in O.COMPS}


def _strongest_boxes(lay, fac, count):
    amp = []
    for b in range(len(lay.boxes)):
        fz, fy, fx, d = fac["Ey"][b]
        amp.append(float(np.abs(fz).max() * np.abs(fy).max() * np.abs(fx).max() / abs(d)))
    return list(np.argsort(amp)[::-1][:count])


def _one_box_layout(box):
    return I.Layout("independent", (0, 0, 0), (1, 1, 1), [box])


def _check_interior(box, got, ref, what):
    lay1 = _one_box_layout(box)
    assert_fields(lay1, {k: [got[k]] for k in O.COMPS}, {k: [ref[k]] for k in O.COMPS}, O.COMPS, 32, what=what)


def test_one_step_sampled_boxes_match_oracle(env):
    lay, plan, fac, fields = _push(1)
    for b in _strongest_boxes(lay, fac, 2) + [0, len(lay.boxes) - 1]:
        box = lay.boxes[b]
        ref = O.push_box(_box_input(lay, fac, b), None, H, box.p, DT, form="vacuum")
        got = _box_output(plan, fields, b)
        sl = O._interior_slices(box)
        if max(float(np.abs(ref[k][sl]).max()) for k in O.COMPS) > 0:
            _check_interior(box, got, ref, f"box {b}, 1 step")
        else:      # the laser underflows to 0 in FP32 there: the interior stays 0
            assert all(not np.any(got[k][sl]) for k in O.COMPS), b
    plan.close()


def _cone_reference(lay, fac, b, nsteps):
    """Interior of box b after nsteps local-decomposition steps, from the
    oracle pushing only the boxes it depends on."""
    index = {tuple(bx.origin): i for i, bx in enumerate(lay.boxes)}
    c0 = lay.boxes[b].origin

    def box_at(d):
        return index[tuple((c0[a] + d[a] * INNER) % GLOBAL_N[a] for a in range(3))]

    lo, hi = NG, NG + INNER
    R = nsteps - 1
    cur = {}
    for d in itertools.product(range(-R, R + 1), repeat=3):
        i = box_at(d)
        out = O.push_box(_box_input(lay, fac, i), None, H, P, DT, form="vacuum")
        cur[d] = {k: out[k][lo:hi, lo:hi, lo:hi] for k in O.COMPS}
    # padded-box slices owned by the neighbour at offset -1, 0, +1 (one axis)
    dst = {-1: slice(0, NG), 0: slice(NG, NG + INNER), 1: slice(NG + INNER, 2 * NG + INNER)}
    src = {-1: slice(INNER - NG, INNER), 0: slice(0, INNER), 1: slice(0, NG)}
    for step in range(2, nsteps + 1):
        r = nsteps - step
        nxt = {}
        for d in itertools.product(range(-r, r + 1), repeat=3):
            inp = {k: np.empty((INNER + 2 * NG,) * 3) for k in O.COMPS}
            for dd in itertools.product((-1, 0, 1), repeat=3):      # (x, y, z) offsets
                owner = cur[tuple(d[a] + dd[a] for a in range(3))]
                for k in O.COMPS:
                    inp[k][dst[dd[2]], dst[dd[1]], dst[dd[0]]] = owner[k][src[dd[2]], src[dd[1]], src[dd[0]]]
            out = O.push_box(inp, None, H, P, DT, form="vacuum")
            nxt[d] = {k: out[k][lo:hi, lo:hi, lo:hi] for k in O.COMPS}
        cur = nxt
    return cur[(0, 0, 0)]


@pytest.fixture(scope="module")
def pushed3(env):
    lay, plan, fac, fields = _push(3)
    yield lay, plan, fac, fields
    plan.close()


def test_three_steps_strongest_box_matches_oracle_cone(pushed3):
    lay, plan, fac, fields = pushed3
    b = _strongest_boxes(lay, fac, 1)[0]
    ref = _cone_reference(lay, fac, b, 3)
    got = _box_output(plan, fields, b)
    lo, hi = NG, NG + INNER
    box = lay.boxes[b]
    gi = {k: got[k][lo:hi, lo:hi, lo:hi] for k in O.COMPS}
    inner = I.Box((INNER,) * 3, (0,) * 3, (0,) * 3, (0, 0, 0), P)
    _check_interior(inner, gi, ref, f"box {b} ({box.origin}), 3 steps")


def test_guards_equal_owning_interior_cells(pushed3):
    lay, plan, fac, fields = pushed3
    index = {tuple(bx.origin): i for i, bx in enumerate(lay.boxes)}
    for b in _strongest_boxes(lay, fac, 1) + [0]:
        box = lay.boxes[b]
        org = box.origin
        got = _box_output(plan, fields, b)
        # the periodic global array on the 3 x 3 x 3 sub-domains around b
        patch = {k: np.empty((3 * INNER,) * 3) for k in O.COMPS}
        for dz in range(3):
            for dy in range(3):
                for dx in range(3):
                    o = tuple((org[d] + (dd - 1) * INNER) % GLOBAL_N[d] for d, dd in zip(range(3), (dx, dy, dz)))
                    nb = index[o]
                    src = _box_output(plan, fields, nb)
                    sl = O._interior_slices(lay.boxes[nb])
                    for k in O.COMPS:
                        patch[k][dz * INNER:(dz + 1) * INNER, dy * INNER:(dy + 1) * INNER,
                                 dx * INNER:(dx + 1) * INNER] = src[k][sl]
        lo = INNER - NG
        for k in O.COMPS:
            want = patch[k][lo:lo + box.n[2], lo:lo + box.n[1], lo:lo + box.n[0]]
            assert np.array_equal(got[k], want), (b, k)
