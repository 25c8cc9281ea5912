"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the
same seeded inputs.

Tolerances: FP64 GPU <= 1e-12 relative L2; FP32 GPU <= 2e-5 relative L2 (the
FP32 run is compared with the oracle fed the FP32-rounded inputs).  The
guard exchange is pure data movement and must be bit-exact.
"""
import numpy as np
import pytest

from oracle import psatd_oracle as O
from paper_1812_07357_gb300 import inputs as I
from _parity import assert_fields

pytestmark = pytest.mark.gpu

TOL = {64: 1e-12, 32: 2e-5}
FFT_TOL = {64: 1e-13, 32: 2e-6}


@pytest.fixture(scope="module", autouse=True)
def built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1812_07357_gb300 import build
    build.build()


def Plan(*a, **k):
    from paper_1812_07357_gb300.solver import Plan as P
    return P(*a, **k)


def rel_l2(a, b):
    num = sum(float(np.sum(np.abs(x - y) ** 2)) for x, y in zip(a, b))
    den = sum(float(np.sum(np.abs(y) ** 2)) for y in b)
    return (num / den) ** 0.5


def run_push(lay, fields, src, nsteps, h, dt, prec, form, **plan_kw):
    plan = Plan(lay, h, dt, precision=prec, sources=form, **plan_kw)
    df = plan.pack_fields(fields)
    ds = plan.pack_fields(src) if form != "vacuum" else None
    plan.push(df, ds, nsteps)
    plan.sync()
    out = plan.unpack_fields(df)
    if form == "rho":
        out["rho"] = plan.unpack(ds["rho"])
    plan.close()
    return out


def check_push(lay, fields, src, nsteps, h, dt, prec, form, tol=None, **plan_kw):
    if prec == 32:
        fields = {k: I.round_to(v, np.float32) for k, v in fields.items()}
        src = {k: I.round_to(v, np.float32) for k, v in src.items()}
    got = run_push(lay, fields, src, nsteps, h, dt, prec, form, **plan_kw)
    ref = O.push(lay, fields, src, nsteps, h, dt, form=form)
    comps = O.COMPS + (("rho",) if form == "rho" else ())
    # every field vector on its own (E, B, rho), relative L2 and max-norm
    errs = assert_fields(lay, got, ref, comps, prec, tol)
    err = max(l2 for l2, _ in errs.values())
    # guards are consistent after the step (exchange ran): whole box compared
    for k in comps:
        for g, r in zip(got[k], ref[k]):
            scale = max(1.0, float(np.abs(r).max()))
            assert np.abs(g - r).max() <= 50 * TOL[prec] * scale * max(1, nsteps) ** 0.5
    return err


# ---------------------------------------------------------------------------
# S1 / S3 alone
# ---------------------------------------------------------------------------

def _fft_layout():
    boxes = [I.Box(n, (0, 0, 0), (0, 0, 0), (0, 0, 0), 0) for n in
             [(8, 8, 8), (12, 10, 6), (96, 48, 20), (30, 18, 50), (4, 4, 4), (160, 8, 6),
              (1024, 4, 4), (6, 512, 4), (4, 6, 512)]]
    return I.Layout("independent", (0, 0, 0), (1, 1, 1), boxes)


@pytest.mark.parametrize("prec", [64, 32])
def test_forward_fft_matches_oracle_fft(prec):
    lay = _fft_layout()
    rng = np.random.default_rng(21)
    arrs = I.round_to([rng.standard_normal(b.shape) for b in lay.boxes], np.float32 if prec == 32 else np.float64)
    plan = Plan(lay, (1.0,) * 3, 0.5, precision=prec)
    spec = plan.forward_fft(plan.pack(arrs))
    plan.sync()
    got = plan.unpack_spectrum(spec)
    for b, a, g in zip(lay.boxes, arrs, got):
        ref = O.fft3(a)[:, :, : b.n[0] // 2 + 1]
        assert rel_l2([g], [ref]) <= FFT_TOL[prec], b.n
    plan.close()


@pytest.mark.parametrize("prec", [64, 32])
def test_inverse_fft_roundtrip(prec):
    lay = _fft_layout()
    rng = np.random.default_rng(22)
    arrs = [rng.standard_normal(b.shape) for b in lay.boxes]
    plan = Plan(lay, (1.0,) * 3, 0.5, precision=prec)
    import torch
    host = np.zeros(plan.spec_elems, np.complex128)
    for (off, n), b, a in zip(plan.spec_offsets, lay.boxes, arrs):
        host[off:off + n] = O.fft3(a)[:, :, : b.n[0] // 2 + 1].ravel()
    spec = torch.from_numpy(host.astype(np.complex64 if prec == 32 else np.complex128)).cuda()
    out = plan.unpack(plan.inverse_fft(spec))
    plan.sync()
    for b, a, g in zip(lay.boxes, arrs, out):
        assert rel_l2([g], [a]) <= FFT_TOL[prec], b.n
    plan.close()


# ---------------------------------------------------------------------------
# guard exchange: bit-exact
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("kind", ["local", "local_open", "hybrid", "independent"])
def test_guard_exchange_bit_exact(prec, kind):
    if kind == "local":
        lay = I.local_layout((48, 32, 32), (3, 2, 2), 4, 8)
    elif kind == "local_open":
        lay = I.local_layout((48, 32, 32), (3, 2, 2), 4, 8, periodic=(0, 1, 0))
    elif kind == "hybrid":
        lay = I.hybrid_layout((96, 24, 20), (4, 1, 1), 6, 8)
    else:
        lay = I.independent_layout(seed=4, nboxes=7, sizes=(16, 20, 24, 30, 32), ngs=(2, 4, 6),
                                   min_interior=8)
    rng = np.random.default_rng(23)
    dt = np.float32 if prec == 32 else np.float64
    f = {k: I.round_to([rng.standard_normal(b.shape) for b in lay.boxes], dt) for k in O.COMPS}
    plan = Plan(lay, (1.0,) * 3, 0.5, precision=prec)
    df = plan.pack_fields(f)
    plan.guard_exchange(df)
    plan.sync()
    got = plan.unpack_fields(df)
    for k in O.COMPS:
        ref = O.exchange(lay, f[k])
        for g, r in zip(got[k], ref):
            assert np.array_equal(g, r)
    plan.close()


# ---------------------------------------------------------------------------
# whole push, each decomposition and equation form
# ---------------------------------------------------------------------------

def test_plane_waves_infinite_order_fp64():
    """32^3 periodic, p = infinity, dt = 0.5, 64 steps (full size): GPU FP64
    vs oracle and vs the analytic solution."""
    w = I.make_workload("plane_waves_32")
    err = check_push(w.layout, w.fields, w.src, w.steps, w.h, w.dt, 64, "vacuum")
    got = run_push(w.layout, w.fields, w.src, w.steps, w.h, w.dt, 64, "vacuum")
    ana = I.plane_wave_fields(I.plane_wave_set(seed=1), (32, 32, 32), w.h, 1.0, w.steps * w.dt)
    assert_fields(w.layout, got, {k: [v] for k, v in ana.items()}, O.COMPS, 64)
    assert err <= 1e-12


@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("form", ["rho", "J"])
def test_sources_global_reduced(prec, form):
    """Sources workload at 32^3 (p = 16, dt = 0.9, filtered J), 20 steps."""
    w = I.make_workload("sources_128", scale=4, steps=20)
    src = dict(w.src)
    if form == "J":
        src.pop("rho")
    check_push(w.layout, w.fields, src, w.steps, w.h, w.dt, prec, form)


@pytest.mark.parametrize("prec", [64, 32])
def test_local_decomposition_reduced(prec):
    """Local layout 2x2x2 boxes of 16^3 + 4 guards, p = 8, laser, 6 steps."""
    lay = I.local_layout((32, 32, 32), (2, 2, 2), 4, 8)
    f = I.laser_fields((32, 32, 32), wavelength=8.0, waist=5.0, duration=4.0)
    fields = {k: I.scatter_global(v, lay) for k, v in f.items()}
    check_push(lay, fields, {}, 6, (1.0,) * 3, 0.9, prec, "vacuum")


@pytest.mark.parametrize("prec", [64, 32])
def test_local_nonperiodic_anisotropic(prec):
    lay = I.local_layout((48, 16, 24), (2, 2, 3), (4, 2, 2), 4, periodic=(0, 1, 1))
    f = I.laser_fields((48, 16, 24), wavelength=6.0, waist=4.0, duration=4.0)
    fields = {k: I.scatter_global(v, lay) for k, v in f.items()}
    check_push(lay, fields, {}, 4, (1.0, 0.8, 1.2), 0.7, prec, "vacuum")


@pytest.mark.parametrize("prec", [64, 32])
def test_hybrid_reduced(prec):
    """Hybrid: 4 groups along x of 16 cells with 4 guards on the x faces."""
    w = I.make_workload("hybrid_1024", scale=16, steps=5)
    check_push(w.layout, w.fields, w.src, w.steps, w.h, w.dt, prec, "vacuum")


@pytest.mark.parametrize("prec", [64, 32])
def test_uneven_independent_reduced(prec):
    """Uneven batch of self-periodic boxes, mixed sizes/guards/orders, rho form."""
    w = I.make_workload("uneven_300", scale=4, steps=5)
    check_push(w.layout, w.fields, w.src, w.steps, w.h, w.dt, prec, "rho")


def test_zero_steps_is_identity():
    lay = I.local_layout((32, 16, 16), (2, 1, 1), 4, 8)
    rng = np.random.default_rng(5)
    f = {k: [rng.standard_normal(b.shape) for b in lay.boxes] for k in O.COMPS}
    got = run_push(lay, f, {}, 0, (1.0,) * 3, 0.5, 64, "vacuum")
    for k in O.COMPS:
        for g, r in zip(got[k], f[k]):
            assert np.array_equal(g, r)


def test_errors_are_reported_not_raised_on_device():
    import torch
    from paper_1812_07357_gb300 import _abi as A
    lay = I.global_layout((16, 16, 16), 8)
    plan = Plan(lay, (1.0,) * 3, 0.5, precision=32, sources="rho")
    f = {k: plan.empty() for k in O.COMPS}
    with pytest.raises(A.PsatdError) as e:
        plan.push(f, None, 1)           # sources missing
    assert e.value.status == A.PSATD_ERR_INVALID_ARG
    s = {k: plan.empty() for k in ("Jx", "Jy", "Jz", "rho")}
    bad = dict(f)
    raw = torch.zeros(plan.field_elems + 4, dtype=torch.float32, device="cuda")
    bad["Ex"] = raw[1:]                 # 4-byte misaligned
    with pytest.raises(A.PsatdError) as e:
        plan.push(bad, s, 1)
    assert e.value.status == A.PSATD_ERR_INVALID_ARG
    with pytest.raises(A.PsatdError):
        plan.push(f, s, -1)
    plan.push(f, s, 1)
    plan.sync()
    plan.close()


# ---------------------------------------------------------------------------
# fast path (two-pass register FFT kernels) on fast box sizes
# ---------------------------------------------------------------------------

def _fast_plan_check(lay, fields, src, nsteps, h, dt, prec, form, expect_fast):
    """The plane kernels (requested explicitly: without the flag, boxes whose
    shape has no register plane kernels run on the pencil kernels); in FP32
    both the register plane kernels, where the shape has them, and the
    shared-memory plane kernels (reg_planes knob 0)."""
    for tuning in ((None, {"reg_planes": 0}) if prec == 32 else (None,)):
        plan = Plan(lay, h, dt, precision=prec, sources=form, plane=True, tuning=tuning)
        assert plan.fast_boxes == expect_fast, (plan.fast_boxes, expect_fast)
        plan.close()
        got = check_push(lay, fields, src, nsteps, h, dt, prec, form, plane=True, tuning=tuning)
    return got


@pytest.mark.parametrize("prec", [64, 32])
def test_fast_local_48(prec):
    """8 local boxes of 48^3 (32^3 + 8 guards), p = 16, laser, 4 steps."""
    lay = I.local_layout((64, 64, 64), (2, 2, 2), 8, 16)
    f = I.laser_fields((64, 64, 64), wavelength=8.0, waist=8.0, duration=5.0)
    fields = {k: I.scatter_global(v, lay) for k, v in f.items()}
    _fast_plan_check(lay, fields, {}, 4, (1.0,) * 3, 0.9, prec, "vacuum", 8)


@pytest.mark.parametrize("prec", [64, 32])
def test_fast_uneven_rho(prec):
    """Self-periodic boxes with fast sizes {48, 60, 80} per axis, rho form."""
    lay = I.independent_layout(seed=11, nboxes=4, sizes=(48, 60, 80), ngs=(4, 8), min_interior=16)
    rng = np.random.default_rng(12)
    js = {k: [] for k in ("Jx", "Jy", "Jz")}
    for b in lay.boxes:
        j = I.band_limited_current(b.interior, rng)
        for k in js:
            js[k].append(j[k])
    src = {k: I.scatter_self(v, lay) for k, v in js.items()}
    src["rho"] = I.zeros(lay)
    fields = {k: I.zeros(lay) for k in O.COMPS}
    _fast_plan_check(lay, fields, src, 3, (1.0,) * 3, 0.9, prec, "rho", 4)


@pytest.mark.parametrize("prec", [64, 32])
def test_fast_global_jform_anisotropic(prec):
    """One 60 x 48 x 80 periodic box (all three lengths fast), J form."""
    lay = I.global_layout((60, 48, 80), 8)
    rng = np.random.default_rng(13)
    src = {k: [rng.standard_normal(lay.boxes[0].shape)] for k in ("Jx", "Jy", "Jz")}
    fields = {k: [rng.standard_normal(lay.boxes[0].shape)] for k in O.COMPS}
    _fast_plan_check(lay, fields, src, 3, (1.0, 0.9, 1.1), 0.8, prec, "J", 1)


def test_fast_equals_generic_fp32():
    """The fast and the generic kernels give the same FP32 push."""
    lay = I.local_layout((64, 128, 64), (2, 2, 1), (8, 16, 0), 32)
    f = I.laser_fields((64, 128, 64), wavelength=8.0, waist=8.0, duration=5.0)
    fields = {k: I.round_to(I.scatter_global(v, lay), np.float32) for k, v in f.items()}
    outs = []
    for generic in (False, True):
        plan = Plan(lay, (1.0,) * 3, 0.9, precision=32, sources="vacuum", generic=generic, plane=not generic)
        assert plan.fast_boxes == (0 if generic else 4)
        df = plan.pack_fields(fields)
        plan.push(df, None, 5)
        plan.sync()
        outs.append(plan.unpack_fields(df))
        plan.close()
    assert O.rel_l2_fields(lay, outs[0], outs[1], O.COMPS) < 2e-6


@pytest.mark.parametrize("prec", [32])
def test_register_planes_local_96(prec):
    """Boxes 96 x 96 x 24 (the 96^2 planes of the benchmark boxes run on the
    register-resident plane kernels), local layout, p = 16, laser, 3 steps;
    against the oracle and against the generic kernels."""
    lay = I.local_layout((128, 64, 32), (2, 1, 2), (16, 16, 4), 16)
    assert all(b.n == (96, 96, 24) for b in lay.boxes)
    f = I.laser_fields((128, 64, 32), wavelength=8.0, waist=10.0, duration=6.0)
    fields = {k: I.round_to(I.scatter_global(v, lay), np.float32) for k, v in f.items()}
    _fast_plan_check(lay, fields, {}, 3, (1.0,) * 3, 0.9, prec, "vacuum", 4)
    outs = []
    for generic in (False, True):
        plan = Plan(lay, (1.0,) * 3, 0.9, precision=32, sources="vacuum", generic=generic)
        df = plan.pack_fields(fields)
        plan.push(df, None, 3)
        plan.sync()
        outs.append(plan.unpack_fields(df))
        plan.close()
    assert O.rel_l2_fields(lay, outs[0], outs[1], O.COMPS) < 2e-6
    for k in O.COMPS:          # guards written by the fused exchange agree too
        for a, b in zip(outs[0][k], outs[1][k]):
            assert np.abs(a - b).max() <= 1e-5 * max(1.0, np.abs(b).max())


@pytest.mark.parametrize("form", ["rho", "J"])
def test_register_z_kernel_sources(form):
    """One 60 x 48 x 96 periodic box, FP32: z length 96 runs on the
    register-resident z kernel (with sources), including the Nyquist tiles."""
    lay = I.global_layout((60, 48, 96), 16)
    rng = np.random.default_rng(41)
    shp = lay.boxes[0].shape
    src = {k: [rng.standard_normal(shp)] for k in ("Jx", "Jy", "Jz")}
    fields = {k: [rng.standard_normal(shp)] for k in O.COMPS}
    if form == "rho":
        src["rho"] = [np.zeros(shp)]
        fields = {k: [np.zeros(shp)] for k in O.COMPS}
    _fast_plan_check(lay, fields, src, 3, (1.0, 1.0, 1.0), 0.9, 32, form, 1)


def test_global_reference_lengths_fp64_long_step():
    """The global single-box FP64 reference of the benchmark's error leg runs
    the generic kernels at lengths 512 (512^3 domain) and 1024, 256 (the
    1024 x 256 x 256 domain), one step of 400 dt (no Courant limit, Sec.
    1.1).  Each length on a self-periodic box with short other axes, against
    the oracle's same step."""
    boxes = [I.Box(n, (0, 0, 0), (0, 0, 0), (0, 0, 0), p) for n, p in
             [((512, 16, 16), 32), ((16, 512, 16), 32), ((16, 16, 512), 32),
              ((1024, 16, 16), 64), ((16, 256, 16), 64), ((16, 16, 256), 0)]]
    lay = I.Layout("independent", (0, 0, 0), (1, 1, 1), boxes)
    rng = np.random.default_rng(29)
    fields = {k: [rng.standard_normal(b.shape) for b in lay.boxes] for k in O.COMPS}
    plan = Plan(lay, (1.0,) * 3, 400 * 0.9, precision=64, sources="vacuum")
    assert (plan.fast_boxes, plan.pencil_boxes) == (0, 0)
    plan.close()
    check_push(lay, fields, {}, 1, (1.0,) * 3, 400 * 0.9, 64, "vacuum")


# ---------------------------------------------------------------------------
# edge cases: the smallest boxes, one-sided guards, the largest box
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("prec", [64, 32])
def test_smallest_boxes_and_one_sided_guards(prec):
    """Self-periodic boxes at the size limits' low end (4 cells on an axis,
    one guard) and with different guard widths on the two faces of an axis,
    J form, 3 steps."""
    boxes = [I.Box((4, 4, 4), (1, 1, 1), (1, 1, 1), (0, 0, 0), 2),
             I.Box((4, 6, 8), (1, 2, 0), (1, 0, 3), (0, 0, 0), 4),
             I.Box((24, 20, 18), (2, 3, 1), (4, 1, 3), (0, 0, 0), 8),
             I.Box((30, 10, 6), (0, 1, 2), (5, 2, 0), (0, 0, 0), 0)]
    lay = I.Layout("independent", (0, 0, 0), (1, 1, 1), boxes)
    rng = np.random.default_rng(33)
    fields = {k: O.exchange(lay, [rng.standard_normal(b.shape) for b in lay.boxes]) for k in O.COMPS}
    src = {k: O.exchange(lay, [rng.standard_normal(b.shape) for b in lay.boxes]) for k in ("Jx", "Jy", "Jz")}
    check_push(lay, fields, src, 3, (1.0, 0.8, 1.2), 0.6, prec, "J")


def test_largest_box_fft_sampled_modes_and_round_trip():
    """The largest box the ABI accepts (1024 x 512 x 512 cells, FP32): the
    forward transform at sampled modes against the DFT summed directly in
    FP64 (separable phases, all 2.7e8 cells), and the inverse of the forward
    transform against the input (a property at any size)."""
    import torch
    n0, n1, n2 = 1024, 512, 512
    lay = I.Layout("independent", (0, 0, 0), (1, 1, 1), [I.Box((n0, n1, n2), (0,) * 3, (0,) * 3, (0, 0, 0), 0)])
    plan = Plan(lay, (1.0,) * 3, 0.5, precision=32)
    gen = torch.Generator(device="cuda").manual_seed(34)
    x = torch.randn(n0 * n1 * n2, generator=gen, device="cuda", dtype=torch.float32)
    spec = plan.forward_fft(x)
    back = plan.inverse_fft(spec.clone())
    plan.sync()
    rel = float((back - x).double().norm() / x.double().norm())
    assert rel <= FFT_TOL[32], rel
    xs = x.view(n2, n1, n0).double().cpu().numpy()
    sv = spec[: (n0 // 2 + 1) * n1 * n2].view(n2, n1, n0 // 2 + 1).cpu().numpy()
    rng = np.random.default_rng(35)
    modes = [(0, 0, 0), (n0 // 2, n1 // 2, n2 // 2), (1, n1 - 1, 3)] + \
            [(int(rng.integers(0, n0 // 2 + 1)), int(rng.integers(0, n1)), int(rng.integers(0, n2))) for _ in range(3)]
    scale = float(np.sqrt(np.sum(xs ** 2)))          # |X(m)| ~ ||x|| for white noise
    for mx, my, mz in modes:
        ex = np.exp(-2j * np.pi * mx * np.arange(n0) / n0)
        ey = np.exp(-2j * np.pi * my * np.arange(n1) / n1)
        ez = np.exp(-2j * np.pi * mz * np.arange(n2) / n2)
        ax = xs @ ex.real + 1j * (xs @ ex.imag)           # no complex copy of the 2 GB array
        want = ez @ (ax @ ey)
        got = complex(sv[mz, my, mx])
        assert abs(got - want) <= FFT_TOL[32] * scale, (mx, my, mz, got, want)
    plan.close()
