"""Multi-step pushes replay one captured step (CUDA graph): the results must be
bit-identical to launching the kernels directly (PSATD_NO_GRAPH), on the fast
and on the generic kernels, on the legacy default stream and on a created
stream, and after the field buffers change (the graph is captured again)."""
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


def _run(lay, fields, src, nsteps, form, prec, no_graph, stream=None, swap=False):
    from paper_1812_07357_gb300.solver import Plan
    plan = Plan(lay, (1.0, 1.0, 1.0), 0.9, precision=prec, sources=form, no_graph=no_graph, stream=stream)
    df = plan.pack_fields(fields)
    ds = plan.pack_fields(src) if form != "vacuum" else None
    plan.push(df, ds, nsteps)
    launches = plan.last_launch_count()
    if swap:   # new buffers holding the same values: a new graph is captured
        df = {k: v.clone() for k, v in df.items()}
        if ds is not None:
            ds = {k: v.clone() for k, v in ds.items()}
        plan.push(df, ds, nsteps)
    plan.sync()
    out = plan.unpack_fields(df)
    if form == "rho":
        out["rho"] = plan.unpack(ds["rho"])
    plan.close()
    return out, launches


def _same(a, b):
    for k in a:
        for x, y in zip(a[k], b[k]):
            assert np.array_equal(x, y), k


@pytest.mark.parametrize("swap", [False, True])
def test_graph_equals_direct_fast_path(swap):
    lay = I.local_layout((96, 96, 96), (2, 2, 2), 24, 16)     # 96^3 boxes: register kernels
    f = I.laser_fields((96, 96, 96), wavelength=8.0, waist=10.0, duration=6.0)
    fields = {k: I.round_to(I.scatter_global(v, lay), np.float32) for k, v in f.items()}
    g, ng = _run(lay, fields, {}, 4, "vacuum", 32, False, swap=swap)
    d, nd = _run(lay, fields, {}, 4, "vacuum", 32, True, swap=swap)
    assert ng == nd > 0
    _same(g, d)


@pytest.mark.parametrize("prec", [64, 32])
def test_graph_equals_direct_generic_rho(prec):
    lay = I.global_layout((30, 18, 50), 8)
    rng = np.random.default_rng(7)
    shp = lay.boxes[0].shape
    fields = {k: [rng.standard_normal(shp)] for k in O.COMPS}
    src = {k: [rng.standard_normal(shp)] for k in ("Jx", "Jy", "Jz", "rho")}
    g, ng = _run(lay, fields, src, 3, "rho", prec, False)
    d, nd = _run(lay, fields, src, 3, "rho", prec, True)
    assert ng == nd > 0
    _same(g, d)


def test_graph_on_a_created_stream():
    import torch
    lay = I.local_layout((64, 64, 64), (2, 2, 1), 8, 8)
    rng = np.random.default_rng(9)
    fields = {k: [rng.standard_normal(b.shape) for b in lay.boxes] for k in O.COMPS}
    fields = {k: O.exchange(lay, v) for k, v in fields.items()}
    s = torch.cuda.Stream()
    g, _ = _run(lay, fields, {}, 3, "vacuum", 64, False, stream=s)
    d, _ = _run(lay, fields, {}, 3, "vacuum", 64, True)
    _same(g, d)
    ref = O.push(lay, fields, {}, 3, (1.0, 1.0, 1.0), 0.9, form="vacuum")
    assert_fields(lay, g, ref, O.COMPS, 64)
