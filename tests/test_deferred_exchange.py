"""Deferred guard exchange (paper Fig. 1, step (ii)): on plans whose boxes all
run on the register plane kernels, a step's guard cells are not stored; the
next step's forward pass reads them from the interior cells that own them,
and the last step of a push stores them.  The values read are the ones the
exchange would have stored, so every result is bit-identical to the eager
exchange (PSATD_EAGER_EXCHANGE), guards included."""
import numpy as np
import pytest

from oracle import psatd_oracle as O
from paper_1812_07357_gb300 import inputs as I
from _parity import assert_fields

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1812_07357_gb300 import build
    build.build()


def _layout(periodic=(1, 1, 1)):
    # 96 x 96 x 24 boxes: the register plane shape, guards on all six faces
    lay = I.local_layout((128, 64, 32), (2, 1, 2), (16, 16, 4), 16, periodic=periodic)
    assert all(b.n == (96, 96, 24) for b in lay.boxes)
    return lay


def _laser(lay):
    f = I.laser_fields(lay.global_n, wavelength=8.0, waist=10.0, duration=6.0)
    return {k: I.round_to(I.scatter_global(v, lay), np.float32) for k, v in f.items()}


def _run(lay, fields, src, counts, form="vacuum", **kw):
    from paper_1812_07357_gb300.solver import Plan
    plan = Plan(lay, (1.0, 1.0, 1.0), 0.9, precision=32, sources=form, **kw)
    deferred = plan.deferred_exchange
    df = plan.pack_fields(fields)
    ds = plan.pack_fields(src) if form != "vacuum" else None
    for n in counts:
        plan.push(df, ds, n)
    plan.sync()
    out = plan.unpack_fields(df)
    if form == "rho":
        out["rho"] = plan.unpack(ds["rho"])
    plan.close()
    return out, deferred


def _same(a, b):
    for k in a:
        for x, y in zip(a[k], b[k]):
            assert np.array_equal(x, y), k


@pytest.mark.parametrize("nsteps", [1, 2, 5])
@pytest.mark.parametrize("no_graph", [False, True])
def test_deferred_equals_eager(nsteps, no_graph):
    lay = _layout()
    fields = _laser(lay)
    a, da = _run(lay, fields, {}, [nsteps], no_graph=no_graph)
    b, db = _run(lay, fields, {}, [nsteps], no_graph=no_graph, eager_exchange=True)
    assert da and not db
    _same(a, b)


def test_split_pushes_equal_one_push():
    lay = _layout()
    fields = _laser(lay)
    a, _ = _run(lay, fields, {}, [2, 1, 3])
    b, _ = _run(lay, fields, {}, [6])
    _same(a, b)


def test_open_boundary_against_oracle():
    """Non-periodic x: the guard cells outside the domain have no owner and
    keep their values (read from the box itself)."""
    lay = _layout(periodic=(0, 1, 1))
    fields = _laser(lay)
    a, da = _run(lay, fields, {}, [4])
    b, _ = _run(lay, fields, {}, [4], eager_exchange=True)
    assert da
    _same(a, b)
    ref = O.push(lay, fields, {}, 4, (1.0, 1.0, 1.0), 0.9, form="vacuum")
    assert_fields(lay, a, ref, O.COMPS, 32)


@pytest.mark.parametrize("form,jc", [("rho", False), ("rho", True), ("J", False)])
def test_sources_deferred_equals_eager(form, jc):
    """E, B (and rho) are gathered; J is read as given every step."""
    lay = _layout()
    rng = np.random.default_rng(51)
    js = I.band_limited_current(lay.global_n, rng)
    src = {k: I.round_to(I.scatter_global(v, lay), np.float32) for k, v in js.items()}
    if form == "rho":
        src["rho"] = I.zeros(lay)
    fields = _laser(lay)
    a, da = _run(lay, fields, src, [3], form=form, j_constant=jc)
    b, _ = _run(lay, fields, src, [3], form=form, j_constant=jc, eager_exchange=True)
    assert da
    _same(a, b)


def test_which_plans_defer():
    from paper_1812_07357_gb300.solver import Plan
    lay = _layout()
    for kw, want in (({"generic": True}, False), ({"pencil": True}, True), ({"eager_exchange": True}, False),
                     ({"pencil": True, "eager_exchange": True}, False), ({}, True)):
        plan = Plan(lay, (1.0, 1.0, 1.0), 0.9, precision=32, sources="vacuum", **kw)
        assert plan.deferred_exchange == want, kw
        plan.close()
    plan = Plan(I.global_layout((96, 96, 48), 8), (1.0, 1.0, 1.0), 0.9, precision=32, sources="vacuum")
    assert not plan.deferred_exchange      # no guards
    plan.close()


@pytest.mark.parametrize("prec", [32, 64])
def test_pencil_local_deferred_equals_eager(prec):
    """192 x 96 x 96 local boxes on the pencil kernels: the x-forward pass
    gathers every row's three x bands from their owners."""
    from paper_1812_07357_gb300.solver import Plan
    lay = I.local_layout((256, 64, 64), (2, 2, 2), 32, 16)
    f = I.laser_fields((256, 64, 64), wavelength=8.0, waist=10.0, duration=8.0)
    fields = {k: I.scatter_global(v, lay) for k, v in f.items()}
    if prec == 32:
        fields = {k: I.round_to(v, np.float32) for k, v in fields.items()}
    outs = []
    for eager in (False, True):
        plan = Plan(lay, (1.0, 1.0, 1.0), 0.9, precision=prec, sources="vacuum", eager_exchange=eager)
        assert plan.pencil_boxes == 8 and plan.deferred_exchange == (not eager)
        df = plan.pack_fields(fields)
        plan.push(df, None, 4)
        plan.sync()
        outs.append(plan.unpack_fields(df))
        plan.close()
    _same(outs[0], outs[1])
    ref = O.push(lay, fields, {}, 4, (1.0, 1.0, 1.0), 0.9, form="vacuum")
    assert_fields(lay, outs[0], ref, O.COMPS, prec)


def test_pencil_independent_rho_deferred_equals_eager():
    """Self-periodic boxes of different sizes (guards wrap onto the box's own
    interior), rho form, on the pencil kernels."""
    from paper_1812_07357_gb300.solver import Plan
    sizes = [(160, 24, 32), (192, 30, 40), (256, 32, 24)]
    boxes = [I.Box(n, (4, 4, 4), (4, 4, 4), (0, 0, 0), p) for n, p in zip(sizes, (8, 16, 0))]
    lay = I.Layout("independent", (0, 0, 0), (1, 1, 1), boxes)
    rng = np.random.default_rng(53)
    js = {k: [] for k in ("Jx", "Jy", "Jz")}
    for b in lay.boxes:
        j = I.band_limited_current(b.interior, rng)
        for k in js:
            js[k].append(j[k])
    src = {k: I.round_to(I.scatter_self(v, lay), np.float32) for k, v in js.items()}
    src["rho"] = I.zeros(lay)
    fields = {k: I.zeros(lay) for k in O.COMPS}
    a, da = _run(lay, fields, src, [3], form="rho")
    b, _ = _run(lay, fields, src, [3], form="rho", eager_exchange=True)
    assert da
    _same(a, b)


def test_guards_wider_than_neighbours():
    """n_g = 40 on 16-cell interiors: a guard face spans three neighbours, so
    a plane has more than 3 x 3 rectangles (the general rectangle-list
    gather); against the eager exchange (bitwise) and the oracle."""
    lay = I.local_layout((64, 64, 32), (4, 4, 2), (40, 40, 4), 16)
    assert all(b.n == (96, 96, 24) for b in lay.boxes)
    fields = _laser(lay)
    a, da = _run(lay, fields, {}, [3])
    b, _ = _run(lay, fields, {}, [3], eager_exchange=True)
    assert da
    _same(a, b)
    ref = O.push(lay, fields, {}, 3, (1.0, 1.0, 1.0), 0.9, form="vacuum")
    assert_fields(lay, a, ref, O.COMPS, 32)
