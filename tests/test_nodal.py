"""PSATD_NODAL (collocated variant): the plan generates the centred order-p
symbol and unit phases; every kernel family against the oracle's nodal push."""
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


def _check(lay, prec, form, paths, nsteps=3, **kw):
    from paper_1812_07357_gb300.solver import Plan
    rng = np.random.default_rng(41)
    fields = {k: O.exchange(lay, [rng.standard_normal(b.shape) for b in lay.boxes]) for k in O.COMPS}
    src = {}
    if form != "vacuum":
        src = {k: O.exchange(lay, [rng.standard_normal(b.shape) for b in lay.boxes]) for k in ("Jx", "Jy", "Jz")}
        if form == "rho":
            src["rho"] = I.zeros(lay)
    if prec == 32:
        fields = {k: I.round_to(v, np.float32) for k, v in fields.items()}
        src = {k: I.round_to(v, np.float32) for k, v in src.items()}
    plan = Plan(lay, (1.0, 0.9, 1.1), 0.8, precision=prec, sources=form, nodal=True, **kw)
    assert (plan.fast_boxes, plan.pencil_boxes) == paths
    df = plan.pack_fields(fields)
    ds = plan.pack_fields(src) if form != "vacuum" else None
    plan.push(df, ds, nsteps)
    plan.sync()
    got = plan.unpack_fields(df)
    if form == "rho":
        got["rho"] = plan.unpack(ds["rho"])
    plan.close()
    ref = O.push(lay, fields, src, nsteps, (1.0, 0.9, 1.1), 0.8, form=form, nodal=True)
    comps = O.COMPS + (("rho",) if form == "rho" else ())
    assert_fields(lay, got, ref, comps, prec)


@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("form", ["vacuum", "rho"])
def test_nodal_pencil(prec, form):
    _check(I.local_layout((64, 64, 64), (2, 2, 2), 8, 16), prec, form, (0, 8), pencil=True)


@pytest.mark.parametrize("form", ["vacuum", "J"])
def test_nodal_register_planes(form):
    _check(I.local_layout((128, 64, 32), (2, 1, 2), (16, 16, 4), 16), 32, form, (4, 0))


def test_nodal_plane_kernels():
    _check(I.local_layout((64, 64, 64), (2, 2, 2), 8, 8), 64, "vacuum", (8, 0), plane=True)


def test_nodal_generic_infinite_order():
    _check(I.local_layout((80, 80, 80), (2, 2, 2), 5, 0), 64, "rho", (0, 0))
