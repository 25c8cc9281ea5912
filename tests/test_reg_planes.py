"""Register plane kernels on every plane shape they take (n0/2 in 24, 30, 40,
48, 60 by n1 in 48, 60, 80, 96, 120; one launch per shape), with the z pass
of batches of several z lengths on the register z kernel, against the FP64
oracle (FP32 bound of test_gpu_parity, per field, relative L2 and max-norm)
and against the pencil kernels; the deferred guard exchange of a batch of
shapes (gather tables in the order of the shape groups) against the eager
one, bit for bit."""
import numpy as np
import pytest

from oracle import psatd_oracle as O
from paper_1812_07357_gb300 import inputs as I
from _parity import assert_fields

pytestmark = pytest.mark.gpu

LENGTHS = (48, 60, 80, 96, 120)


@pytest.fixture(scope="module", autouse=True)
def built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1812_07357_gb300 import build
    build.build()


def _every_shape_layout():
    """25 self-periodic boxes, one per (n0, n1) pair of LENGTHS, z lengths
    cycling through LENGTHS, guard widths 4..8, orders 8, 16, 32, inf."""
    boxes = []
    for i, n0 in enumerate(LENGTHS):
        for j, n1 in enumerate(LENGTHS):
            n2 = LENGTHS[(i + 2 * j) % 5]
            ng = 4 + (i + j) % 5
            boxes.append(I.Box((n0, n1, n2), (ng,) * 3, (ng,) * 3, (0, 0, 0), (8, 16, 32, 0)[(i + j) % 4]))
    return I.Layout("independent", (0, 0, 0), (1, 1, 1), boxes)


def _inputs(lay, form, seed):
    rng = np.random.default_rng(seed)
    src = {}
    if form != "vacuum":
        js = {k: [] for k in ("Jx", "Jy", "Jz")}
        for b in lay.boxes:
            j = I.band_limited_current(b.interior, rng)
            for k in js:
                js[k].append(j[k])
        src = {k: I.round_to(I.scatter_self(v, lay), np.float32) for k, v in js.items()}
        if form == "rho":
            src["rho"] = I.zeros(lay)
    fields = {k: I.round_to(O.exchange(lay, [rng.standard_normal(b.shape) for b in lay.boxes]), np.float32)
              for k in O.COMPS}
    return fields, src


def _push(lay, fields, src, form, nsteps, **plan_kw):
    from paper_1812_07357_gb300.solver import Plan
    plan = Plan(lay, (1.0, 0.9, 1.1), 0.8, precision=32, sources=form, j_constant=form != "vacuum", **plan_kw)
    info = (plan.fast_boxes, plan.pencil_boxes, plan.deferred_exchange, plan.tuning())
    df = plan.pack_fields(fields)
    ds = plan.pack_fields(src) if form != "vacuum" else None
    plan.push(df, ds, nsteps)
    plan.sync()
    got = plan.unpack_fields(df)
    if form == "rho":
        got["rho"] = plan.unpack(ds["rho"])
    plan.close()
    return got, info


def test_every_register_plane_shape_vacuum():
    """All 25 shapes in one plan: 25 plane launches per pass, the z pass over
    five z lengths on the register z kernel; 3 steps against the oracle."""
    lay = _every_shape_layout()
    fields, src = _inputs(lay, "vacuum", 61)
    got, (nfast, npen, deferred, tun) = _push(lay, fields, src, "vacuum", 3)
    assert (nfast, npen) == (25, 0) and deferred
    assert tun.get("reg_planes") == 1 and tun.get("pencil_reg_z") == 1
    ref = O.push(lay, fields, src, 3, (1.0, 0.9, 1.1), 0.8, form="vacuum")
    assert_fields(lay, got, ref, O.COMPS, 32, what="every register plane shape")


@pytest.mark.parametrize("form", ["J", "rho"])
def test_register_planes_with_sources(form):
    """Eight of the shapes with a constant current (J and rho forms): against
    the oracle, and against the pencil kernels on the same boxes."""
    lay = _every_shape_layout()
    lay = I.Layout("independent", (0, 0, 0), (1, 1, 1), lay.boxes[::3])
    fields, src = _inputs(lay, form, 62)
    comps = O.COMPS + (("rho",) if form == "rho" else ())
    ref = O.push(lay, fields, src, 3, (1.0, 0.9, 1.1), 0.8, form=form)
    got, (nfast, npen, _, _) = _push(lay, fields, src, form, 3)
    assert (nfast, npen) == (len(lay.boxes), 0)
    assert_fields(lay, got, ref, comps, 32, what=f"register planes, {form} form")
    pen, (nfast, npen, _, _) = _push(lay, fields, src, form, 3, pencil=True)
    assert (nfast, npen) == (0, len(lay.boxes))
    assert_fields(lay, pen, ref, comps, 32, what=f"pencil kernels, {form} form")
    assert_fields(lay, got, pen, comps, 32, what="register planes vs pencil kernels")


def test_register_planes_one_z_length_several_shapes():
    """Three shapes sharing z length 96: one register z launch (no fixed z
    stride), the shared-memory z kernel with the pencil_reg_z knob off not
    involved; and z pass variants of a mixed-z batch (register z per length,
    in one persistent launch, shared-memory plane z kernel) agree."""
    sizes = [(96, 96, 96), (48, 120, 96), (120, 60, 96)]
    boxes = [I.Box(n, (6,) * 3, (6,) * 3, (0, 0, 0), p) for n, p in zip(sizes, (16, 0, 32))]
    lay = I.Layout("independent", (0, 0, 0), (1, 1, 1), boxes)
    fields, src = _inputs(lay, "vacuum", 63)
    ref = O.push(lay, fields, src, 3, (1.0, 0.9, 1.1), 0.8, form="vacuum")
    got, (nfast, _, _, tun) = _push(lay, fields, src, "vacuum", 3)
    assert nfast == 3 and "pencil_reg_z" not in tun and "z_one_launch" not in tun
    assert_fields(lay, got, ref, O.COMPS, 32, what="one z length")

    sizes = [(96, 48, 60), (48, 120, 80), (120, 60, 48), (60, 80, 120)]
    boxes = [I.Box(n, (4,) * 3, (4,) * 3, (0, 0, 0), p) for n, p in zip(sizes, (16, 0, 32, 8))]
    lay = I.Layout("independent", (0, 0, 0), (1, 1, 1), boxes)
    fields, src = _inputs(lay, "rho", 64)
    comps = O.COMPS + ("rho",)
    ref = O.push(lay, fields, src, 3, (1.0, 0.9, 1.1), 0.8, form="rho")
    outs = []
    for tuning in ({"pencil_reg_z": 1, "z_one_launch": 0}, {"pencil_reg_z": 1, "z_one_launch": 1},
                   {"pencil_reg_z": 0}):
        got, (nfast, _, _, tun) = _push(lay, fields, src, "rho", 3, tuning=tuning)
        assert nfast == 4 and tun.get("pencil_reg_z") == tuning["pencil_reg_z"]
        assert tun.get("z_one_launch", -1) == tuning.get("z_one_launch", -1)
        assert_fields(lay, got, ref, comps, 32, what=f"mixed z lengths, {tuning}")
        outs.append(got)
    for got in outs[1:]:
        assert_fields(lay, outs[0], got, comps, 32, what="z pass variants against each other")


def test_register_planes_mixed_with_pencil_boxes():
    """Register-shape boxes and boxes the register kernels do not take
    (n0/2 = 80, n1 = 24) in one plan: plane and pencil families side by side."""
    sizes = [(60, 96, 48), (160, 24, 48), (80, 48, 96), (64, 64, 64)]
    boxes = [I.Box(n, (4,) * 3, (4,) * 3, (0, 0, 0), p) for n, p in zip(sizes, (8, 16, 0, 32))]
    lay = I.Layout("independent", (0, 0, 0), (1, 1, 1), boxes)
    fields, src = _inputs(lay, "vacuum", 65)
    got, (nfast, npen, _, _) = _push(lay, fields, src, "vacuum", 3)
    assert (nfast, npen) == (2, 2)
    ref = O.push(lay, fields, src, 3, (1.0, 0.9, 1.1), 0.8, form="vacuum")
    assert_fields(lay, got, ref, O.COMPS, 32, what="register planes beside pencil boxes")


def test_register_planes_deferred_equals_eager():
    """The deferred exchange of a batch of shapes (gather tables in the order
    of the shape groups) gives the eager exchange's result bit for bit."""
    lay = _every_shape_layout()
    lay = I.Layout("independent", (0, 0, 0), (1, 1, 1), lay.boxes[1::2])
    fields, src = _inputs(lay, "vacuum", 66)
    a, (_, _, deferred_a, _) = _push(lay, fields, src, "vacuum", 4)
    b, (_, _, deferred_b, _) = _push(lay, fields, src, "vacuum", 4, eager_exchange=True)
    assert deferred_a and not deferred_b
    for k in O.COMPS:
        for x, y in zip(a[k], b[k]):
            assert np.array_equal(x, y), k


# ---------------------------------------------------------------------------
# wide planes (k_plane_*_wide): 128 x 128 and 192 x 192
# ---------------------------------------------------------------------------

def test_wide_planes_local_192_laser():
    """Two local 192^3 boxes (64^3 interior + 64 guards, the local 1024
    workload's box), p = 64, laser, 3 steps: wide plane kernels (2 threads
    per row, 4 per column), the pencil z kernel for z = 192, the deferred
    exchange; against the oracle and against the pencil kernels."""
    lay = I.local_layout((128, 64, 64), (2, 1, 1), 64, 64)
    assert all(b.n == (192, 192, 192) for b in lay.boxes)
    f = I.laser_fields((128, 64, 64), wavelength=8.0, waist=12.0, duration=8.0)
    fields = {k: I.round_to(I.scatter_global(v, lay), np.float32) for k, v in f.items()}
    ref = O.push(lay, fields, {}, 3, (1.0, 0.9, 1.1), 0.8, form="vacuum")
    got, (nfast, npen, deferred, tun) = _push(lay, fields, {}, "vacuum", 3)
    assert (nfast, npen) == (2, 0) and deferred and tun.get("reg_planes") == 1
    assert_fields(lay, got, ref, O.COMPS, 32, what="wide 192 x 192 planes")
    pen, (nfast, npen, _, _) = _push(lay, fields, {}, "vacuum", 3, pencil=True)
    assert (nfast, npen) == (0, 2)
    assert_fields(lay, got, pen, O.COMPS, 32, what="wide planes vs pencil kernels")


@pytest.mark.parametrize("form", ["vacuum", "rho"])
@pytest.mark.parametrize("sizes", [
    # several z lengths: 128, 96, 60, 192
    [(128, 128, 128), (128, 128, 192), (192, 192, 60), (128, 128, 96)],
    # one z length: 96
    [(128, 128, 96), (192, 192, 96)],
], ids=["mixed_z", "z96"])
@pytest.mark.parametrize("reg_z", [1, 0])
def test_wide_planes_with_every_z_route(form, sizes, reg_z):
    """Self-periodic 128 x 128 and 192 x 192 planes with the z pass on each
    of its kernels: the register z kernels (thread pairs for 60 and 96,
    thread quads for 128 and 192; knob pencil_reg_z = 1), or the
    shared-memory plane z kernel (lengths up to 128) and the pencil z kernel
    (192) with the knob at 0; the one-length batch on the register z kernel
    either way.  Against the oracle."""
    boxes = [I.Box(n, (6,) * 3, (6,) * 3, (0, 0, 0), p) for n, p in zip(sizes, (16, 0, 32, 8))]
    lay = I.Layout("independent", (0, 0, 0), (1, 1, 1), boxes)
    fields, src = _inputs(lay, form, 67)
    comps = O.COMPS + (("rho",) if form == "rho" else ())
    ref = O.push(lay, fields, src, 3, (1.0, 0.9, 1.1), 0.8, form=form)
    got, (nfast, npen, deferred, tun) = _push(lay, fields, src, form, 3, tuning={"pencil_reg_z": reg_z})
    assert (nfast, npen) == (len(boxes), 0) and deferred
    assert tun.get("pencil_reg_z", -1) == (reg_z if len(sizes) == 4 else -1)
    assert_fields(lay, got, ref, comps, 32, what=f"wide planes, {sizes}, {form} form, pencil_reg_z {reg_z}")


def test_wide_planes_beside_shared_memory_planes():
    """The plane family forced on a batch with a shape that has no register
    plane kernels (64 x 64 planes: the shared-memory plane kernels, launched
    on their own job range) and one that has (128 x 128): against the
    oracle."""
    sizes = [(64, 64, 64), (128, 128, 64)]
    boxes = [I.Box(n, (4,) * 3, (4,) * 3, (0, 0, 0), p) for n, p in zip(sizes, (16, 32))]
    lay = I.Layout("independent", (0, 0, 0), (1, 1, 1), boxes)
    fields, src = _inputs(lay, "vacuum", 68)
    ref = O.push(lay, fields, src, 3, (1.0, 0.9, 1.1), 0.8, form="vacuum")
    got, (nfast, npen, deferred, _) = _push(lay, fields, src, "vacuum", 3, plane=True)
    assert (nfast, npen) == (2, 0) and not deferred
    assert_fields(lay, got, ref, O.COMPS, 32, what="wide and shared-memory plane kernels in one plan")
