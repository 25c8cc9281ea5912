"""PSATD_J_CONSTANT: the current's spectrum is computed once per push call and
reused by every step.  Against the FP64 oracle (which transforms J every
step) on every kernel family, both forms with sources, both precisions."""
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


def _sources(lay, seed, form):
    rng = np.random.default_rng(seed)
    js = {k: [] for k in ("Jx", "Jy", "Jz")}
    for b in lay.boxes:
        j = I.band_limited_current(b.interior, rng)
        for k in js:
            js[k].append(j[k])
    src = {k: I.scatter_self(v, lay) if lay.kind == "independent" else O_exchange(lay, v) for k, v in js.items()}
    if form == "rho":
        src["rho"] = I.zeros(lay)
    return src


def O_exchange(lay, per_box_interior):
    """Embed per-box interior arrays into padded boxes with consistent guards."""
    arrs = []
    for b, a in zip(lay.boxes, per_box_interior):
        full = np.zeros(b.shape)
        full[O._interior_slices(b)] = a
        arrs.append(full)
    return O.exchange(lay, arrs)


def _check(lay, prec, form, nsteps=3, **plan_kw):
    from paper_1812_07357_gb300.solver import Plan
    src = _sources(lay, 31, form)
    rng = np.random.default_rng(32)
    fields = {k: O.exchange(lay, [rng.standard_normal(b.shape) for b in lay.boxes]) for k in O.COMPS}
    if prec == 32:
        fields = {k: I.round_to(v, np.float32) for k, v in fields.items()}
        src = {k: I.round_to(v, np.float32) for k, v in src.items()}
    plan = Plan(lay, (1.0, 1.0, 1.0), 0.9, precision=prec, sources=form, j_constant=True, **plan_kw)
    df = plan.pack_fields(fields)
    ds = plan.pack_fields(src)
    plan.push(df, ds, nsteps)
    plan.sync()
    got = plan.unpack_fields(df)
    if form == "rho":
        got["rho"] = plan.unpack(ds["rho"])
    jgot = {k: plan.unpack(ds[k]) for k in ("Jx", "Jy", "Jz")}
    paths = (plan.fast_boxes, plan.pencil_boxes)
    plan.close()
    ref = O.push(lay, fields, src, nsteps, (1.0, 1.0, 1.0), 0.9, form=form)
    comps = O.COMPS + (("rho",) if form == "rho" else ())
    assert_fields(lay, got, ref, comps, prec)
    for k in ("Jx", "Jy", "Jz"):   # the current is read only
        for a, b in zip(jgot[k], src[k]):
            assert np.array_equal(a, b)
    return paths


@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("form", ["rho", "J"])
def test_jconst_pencil_local(prec, form):
    lay = I.local_layout((64, 64, 64), (2, 2, 2), 8, 16)          # 48^3 boxes on the pencil kernels
    assert _check(lay, prec, form, pencil=True) == (0, 8)


@pytest.mark.parametrize("form", ["rho", "J"])
def test_jconst_plane_kernels(form):
    lay = I.local_layout((64, 64, 64), (2, 2, 2), 8, 16)
    assert _check(lay, 32, form, plane=True) == (8, 0)


@pytest.mark.parametrize("form", ["rho", "J"])
def test_jconst_register_kernels(form):
    lay = I.local_layout((128, 64, 32), (2, 1, 2), (16, 16, 4), 16)   # 96 x 96 x 24: register planes
    assert _check(lay, 32, form) == (4, 0)


def test_jconst_register_z_kernel():
    lay = I.global_layout((60, 48, 96), 16)                          # z length 96: register z kernel
    assert _check(lay, 32, "rho", plane=True) == (1, 0)


def test_jconst_generic_kernels():
    lay = I.local_layout((80, 80, 80), (2, 2, 2), 5, 8)              # 50^3 boxes: generic kernels
    assert _check(lay, 64, "rho") == (0, 0)
