"""Pencil kernels (boxes with two-pass FFT lengths whose planes are too large
for the plane kernels: n0/2 above 64 in FP32 / 48 in FP64, or n1 above 128)
against the FP64 oracle, against the generic kernels, and mixed with plane and
generic boxes in one plan (guard exchange across the three kernel families).
Tolerances as in test_gpu_parity: FP64 <= 1e-12, FP32 <= 2e-5 relative L2."""
import numpy as np
import pytest

from oracle import psatd_oracle as O
from paper_1812_07357_gb300 import inputs as I
from _parity import assert_fields

pytestmark = pytest.mark.gpu

TOL = {64: 1e-12, 32: 2e-5}


@pytest.fixture(scope="module", autouse=True)
def built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1812_07357_gb300 import build
    build.build()


def _run(lay, fields, src, nsteps, h, dt, prec, form, **plan_kw):
    from paper_1812_07357_gb300.solver import Plan
    plan = Plan(lay, h, dt, precision=prec, sources=form, **plan_kw)
    paths = (plan.fast_boxes, plan.pencil_boxes)
    df = plan.pack_fields(fields)
    ds = plan.pack_fields(src) if form != "vacuum" else None
    plan.push(df, ds, nsteps)
    plan.sync()
    out = plan.unpack_fields(df)
    if form == "rho":
        out["rho"] = plan.unpack(ds["rho"])
    plan.close()
    return out, paths


def _check(lay, fields, src, nsteps, h, dt, prec, form, paths, **plan_kw):
    if prec == 32:
        fields = {k: I.round_to(v, np.float32) for k, v in fields.items()}
        src = {k: I.round_to(v, np.float32) for k, v in src.items()}
    got, p = _run(lay, fields, src, nsteps, h, dt, prec, form, **plan_kw)
    assert p == paths, p
    ref = O.push(lay, fields, src, nsteps, h, dt, form=form)
    comps = O.COMPS + (("rho",) if form == "rho" else ())
    assert_fields(lay, got, ref, comps, prec)
    for k in comps:   # guards too (exchange ran)
        for g, r in zip(got[k], ref[k]):
            assert np.abs(g - r).max() <= 50 * TOL[prec] * max(1.0, float(np.abs(r).max())) * nsteps ** 0.5
    return got


@pytest.mark.parametrize("prec", [64, 32])
def test_pencil_independent_long_x_rho(prec):
    """Self-periodic boxes with n0/2 in {80, 96, 128} (pencil in both
    precisions) and short y, z; rho form."""
    sizes = [(160, 24, 32), (192, 30, 40), (256, 32, 24)]
    boxes = [I.Box(n, (4, 4, 4), (4, 4, 4), (0, 0, 0), p) for n, p in zip(sizes, (8, 16, 0))]
    lay = I.Layout("independent", (0, 0, 0), (1, 1, 1), boxes)
    rng = np.random.default_rng(21)
    js = {k: [] for k in ("Jx", "Jy", "Jz")}
    for b in lay.boxes:
        j = I.band_limited_current(b.interior, rng)
        for k in js:
            js[k].append(j[k])
    src = {k: I.scatter_self(v, lay) for k, v in js.items()}
    src["rho"] = I.zeros(lay)
    fields = {k: I.zeros(lay) for k in O.COMPS}
    _check(lay, fields, src, 3, (1.0, 1.0, 1.0), 0.9, prec, "rho", (0, 3))


@pytest.mark.parametrize("prec", [64, 32])
def test_pencil_local_laser(prec):
    """8 local boxes of 192 x 96 x 96 (128 x 32 x 32 interior + 32 guards),
    p = 16, laser, 3 steps: pencil x, y and z passes with the batched exchange."""
    lay = I.local_layout((256, 64, 64), (2, 2, 2), 32, 16)
    assert all(b.n == (192, 96, 96) for b in lay.boxes)
    f = I.laser_fields((256, 64, 64), wavelength=8.0, waist=10.0, duration=8.0)
    fields = {k: I.scatter_global(v, lay) for k, v in f.items()}
    _check(lay, fields, {}, 3, (1.0, 1.0, 1.0), 0.9, prec, "vacuum", (0, 8))


def test_pencil_long_y_jform():
    """n1 = 160 > 128 (pencil along y with a 48-point x), J form, FP32."""
    lay = I.global_layout((48, 160, 24), 8)
    rng = np.random.default_rng(23)
    shp = lay.boxes[0].shape
    src = {k: [rng.standard_normal(shp)] for k in ("Jx", "Jy", "Jz")}
    fields = {k: [rng.standard_normal(shp)] for k in O.COMPS}
    _check(lay, fields, src, 3, (1.0, 0.9, 1.1), 0.8, 32, "J", (0, 1))


def test_pencil_equals_generic_fp32():
    lay = I.local_layout((256, 64, 64), (2, 2, 2), 32, 16)
    f = I.laser_fields((256, 64, 64), wavelength=8.0, waist=10.0, duration=8.0)
    fields = {k: I.round_to(I.scatter_global(v, lay), np.float32) for k, v in f.items()}
    a, pa = _run(lay, fields, {}, 3, (1.0,) * 3, 0.9, 32, "vacuum")
    b, pb = _run(lay, fields, {}, 3, (1.0,) * 3, 0.9, 32, "vacuum", generic=True)
    assert pa == (0, 8) and pb == (0, 0)
    assert O.rel_l2_fields(lay, a, b, O.COMPS) < 2e-6


def test_mixed_plane_pencil_generic_boxes():
    """One plan with a plane box (48^3), a pencil box (160 x 48 x 48) and a
    generic box (50 x 50 x 50: 25 is not a two-pass length), self-periodic,
    FP64, vacuum."""
    boxes = [I.Box((48, 48, 48), (4,) * 3, (4,) * 3, (0, 0, 0), 8),
             I.Box((160, 48, 48), (8,) * 3, (8,) * 3, (0, 0, 0), 16),
             I.Box((50, 50, 50), (5,) * 3, (5,) * 3, (0, 0, 0), 0)]
    lay = I.Layout("independent", (0, 0, 0), (1, 1, 1), boxes)
    rng = np.random.default_rng(25)
    fields = {k: [rng.standard_normal(b.shape) for b in lay.boxes] for k in O.COMPS}
    fields = {k: O.exchange(lay, v) for k, v in fields.items()}
    _check(lay, fields, {}, 3, (1.0, 1.0, 1.0), 0.9, 64, "vacuum", (1, 1), plane=True)


@pytest.mark.parametrize("prec", [64, 32])
def test_pencil_flag_on_plane_boxes(prec):
    """48^3 local boxes on the pencil kernels (PSATD_PENCIL_KERNELS) and on
    the plane kernels (PSATD_PLANE_KERNELS: the register plane kernels in
    FP32): against the oracle and each other."""
    from paper_1812_07357_gb300.solver import Plan
    lay = I.local_layout((64, 64, 64), (2, 2, 2), 8, 16)
    f = I.laser_fields((64, 64, 64), wavelength=8.0, waist=8.0, duration=5.0)
    fields = {k: I.scatter_global(v, lay) for k, v in f.items()}
    if prec == 32:
        fields = {k: I.round_to(v, np.float32) for k, v in fields.items()}
    outs = []
    for pencil in (True, False):
        plan = Plan(lay, (1.0,) * 3, 0.9, precision=prec, sources="vacuum", pencil=pencil, plane=not pencil)
        assert (plan.fast_boxes, plan.pencil_boxes) == ((0, 8) if pencil else (8, 0))
        df = plan.pack_fields(fields)
        plan.push(df, None, 3)
        plan.sync()
        outs.append(plan.unpack_fields(df))
        plan.close()
    ref = O.push(lay, fields, {}, 3, (1.0,) * 3, 0.9, form="vacuum")
    assert_fields(lay, outs[0], ref, O.COMPS, prec)
    assert_fields(lay, outs[0], outs[1], O.COMPS, prec)


def test_default_family_choice():
    """Without a flag: FP32 boxes whose plane shape has register plane kernels
    (n0/2 in 24 .. 60, n1 in 48 .. 120) take the plane kernels, unless the
    reg_planes knob is 0; FP64 boxes and other plane-eligible shapes (64^3:
    n0/2 = 32) take the pencil kernels."""
    from paper_1812_07357_gb300.solver import Plan
    reg = I.local_layout((128, 64, 32), (2, 1, 2), (16, 16, 4), 16)        # 96 x 96 x 24 boxes
    reg48 = I.local_layout((64, 64, 64), (2, 2, 2), 8, 16)                 # 48^3 boxes
    other = I.local_layout((96, 96, 96), (2, 2, 2), 8, 16)                 # 64^3 boxes
    for lay, prec, tun, want in ((reg, 32, None, (4, 0)), (reg, 64, None, (0, 4)), (reg48, 32, None, (8, 0)),
                                 (reg48, 32, {"reg_planes": 0}, (0, 8)), (other, 32, None, (0, 8))):
        plan = Plan(lay, (1.0,) * 3, 0.9, precision=prec, sources="vacuum", tuning=tun)
        assert (plan.fast_boxes, plan.pencil_boxes) == want, (lay.boxes[0].n, prec, tun)
        assert plan.tuning().get("reg_planes", -1) == (-1 if lay is other or prec == 64 else
                                                      (tun or {}).get("reg_planes", 1))
        plan.close()


@pytest.mark.parametrize("prec", [32, 64])
def test_pencil_lengths_of_the_1024_workloads(prec):
    """The FFT lengths of the 1024 x 256 x 256 workloads, each its own kernel
    instance: n0/2 = 192 (hybrid groups, 384 cells along x), and 192 and 256
    along y and z (local 192^3 boxes, hybrid 256 x 256 planes), on
    self-periodic boxes with short other axes; p = 64 and infinite order;
    J form.  In FP64 the pencil z pass stops at 128, so the boxes with z = 192
    and 256 run on the generic kernels there.  In FP32 on the pencil kernels
    (flag), and by default, where the two 48 x 48-plane boxes with z = 192
    and 256 take the register plane kernels with the pencil z kernel."""
    sizes = [(384, 48, 48), (48, 192, 48), (48, 256, 48), (48, 48, 192), (48, 48, 256)]
    boxes = [I.Box(n, (8, 8, 8), (8, 8, 8), (0, 0, 0), p) for n, p in zip(sizes, (64, 0, 64, 0, 64))]
    lay = I.Layout("independent", (0, 0, 0), (1, 1, 1), boxes)
    rng = np.random.default_rng(27)
    fields = {k: O.exchange(lay, [rng.standard_normal(b.shape) for b in lay.boxes]) for k in O.COMPS}
    src = {k: O.exchange(lay, [rng.standard_normal(b.shape) for b in lay.boxes]) for k in ("Jx", "Jy", "Jz")}
    if prec == 32:
        _check(lay, fields, src, 2, (1.0, 1.0, 1.0), 0.9, prec, "J", (0, 5), pencil=True)
        _check(lay, fields, src, 2, (1.0, 1.0, 1.0), 0.9, prec, "J", (2, 3))
    else:
        _check(lay, fields, src, 2, (1.0, 1.0, 1.0), 0.9, prec, "J", (0, 3))


def test_pencil_local_192_boxes_and_hybrid_384_groups():
    """Two local 192^3 boxes (64^3 interior + 64 guards, the local 1024
    workload's box; on the pencil kernels by flag, the default being the wide
    register plane kernels) and four hybrid groups of 384 x 48 x 48 (256 cells
    + 64 guards on the x faces; y, z periodic inside the group), p = 64,
    laser, FP32, 2 steps with the guard exchange."""
    lay = I.local_layout((128, 64, 64), (2, 1, 1), 64, 64)
    assert all(b.n == (192, 192, 192) for b in lay.boxes)
    f = I.laser_fields((128, 64, 64), wavelength=8.0, waist=12.0, duration=8.0)
    _check(lay, {k: I.scatter_global(v, lay) for k, v in f.items()}, {}, 2, (1.0,) * 3, 0.9, 32, "vacuum",
           (0, 2), pencil=True)
    lay = I.hybrid_layout((1024, 48, 48), (4, 1, 1), 64, 64)
    assert all(b.n == (384, 48, 48) for b in lay.boxes)
    f = I.laser_fields((1024, 48, 48), wavelength=16.0, waist=12.0, duration=20.0)
    _check(lay, {k: I.scatter_global(v, lay) for k, v in f.items()}, {}, 2, (1.0,) * 3, 0.9, 32, "vacuum",
           (0, 4))


@pytest.mark.parametrize("form", ["vacuum", "J", "rho"])
def test_pencil_boxes_z_pass_on_register_kernel_and_shared_memory_kernel(form):
    """FP32 pencil boxes with z lengths 48, 60, 80, 96, 120 (the uneven
    batch's), 128 and 192: their z pass runs on the register z kernels
    (thread pairs up to 120, thread quads for 128 and 192), one launch per
    length (default) or, where every length has it, in one persistent launch,
    or on the shared-memory pencil z kernel (tuning knobs); each against the
    oracle, and against each other."""
    from paper_1812_07357_gb300.solver import Plan
    sizes = [(160, 24, 48), (48, 160, 60), (60, 48, 80), (80, 60, 96), (48, 48, 120), (48, 60, 128),
             (60, 48, 192)]
    boxes = [I.Box(n, (4, 4, 4), (4, 4, 4), (0, 0, 0), p) for n, p in zip(sizes, (8, 16, 32, 0, 16, 8, 0))]
    lay = I.Layout("independent", (0, 0, 0), (1, 1, 1), boxes)
    rng = np.random.default_rng(28)
    if form != "vacuum":
        js = {k: [] for k in ("Jx", "Jy", "Jz")}
        for b in lay.boxes:
            j = I.band_limited_current(b.interior, rng)
            for k in js:
                js[k].append(j[k])
        src = {k: I.round_to(I.scatter_self(v, lay), np.float32) for k, v in js.items()}
        if form == "rho":
            src["rho"] = I.zeros(lay)
    else:
        src = {}
    fields = {k: I.round_to(O.exchange(lay, [rng.standard_normal(b.shape) for b in lay.boxes]), np.float32)
              for k in O.COMPS}
    comps = O.COMPS + (("rho",) if form == "rho" else ())
    ref = O.push(lay, fields, src, 3, (1.0,) * 3, 0.9, form=form)
    outs = []
    for tuning in ({"pencil_reg_z": 1, "z_one_launch": 1}, {"pencil_reg_z": 1, "z_one_launch": 0},
                   {"pencil_reg_z": 0}):
        plan = Plan(lay, (1.0,) * 3, 0.9, precision=32, sources=form, pencil=True, j_constant=form != "vacuum",
                    tuning=tuning)
        used = plan.tuning()
        assert plan.pencil_boxes == 7 and used.get("pencil_reg_z") == tuning["pencil_reg_z"]
        assert "z_one_launch" not in used     # 128 and 192 have no persistent multi-length kernel
        df = plan.pack_fields(fields)
        ds = plan.pack_fields(src) if form != "vacuum" else None
        plan.push(df, ds, 3)
        plan.sync()
        got = plan.unpack_fields(df)
        if form == "rho":
            got["rho"] = plan.unpack(ds["rho"])
        plan.close()
        assert_fields(lay, got, ref, comps, 32, what=f"tuning {tuning}")
        outs.append(got)
    for got in outs[1:]:
        assert_fields(lay, outs[0], got, comps, 32, what="z pass variants against each other")
