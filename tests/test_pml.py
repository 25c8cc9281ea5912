"""Absorbing layers (the two-step split-field PML; see include/psatd.h) on the
GPU against the oracle's layers: the fields and the stored split parts, per
field vector, FP64 <= 1e-12 and FP32 <= 2e-5 relative L2 (max-norm 10x), on
a global box and on a local decomposition whose edge boxes hold the layers."""
import numpy as np
import pytest

from oracle import psatd_oracle as O
from paper_1812_07357_gb300 import inputs as I
from _parity import TOL, assert_fields

pytestmark = pytest.mark.gpu

PARTS = O.SPLIT


@pytest.fixture(scope="module", autouse=True)
def built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1812_07357_gb300 import build
    build.build()


def _pulse(global_n, x0, tau, lam, waist):
    """E_y, B_z of a Gaussian pulse along +x, sampled at their Yee positions."""
    nx, ny, nz = global_n
    out = {k: np.zeros((nz, ny, nx)) for k in O.COMPS}
    y = (np.arange(ny) + 0.5 - ny / 2)[None, :, None]
    z = (np.arange(nz) - nz / 2)[:, None, None]
    for comp, sx, sz in (("Ey", 0.0, 0.0), ("Bz", 0.5, 0.0)):
        x = (np.arange(nx) + sx)[None, None, :]
        out[comp] = np.exp(-((x - x0) / tau) ** 2 - (y ** 2 + (z + sz) ** 2) / waist ** 2) * np.cos(
            2 * np.pi / lam * (x - x0)) + 0 * z
    return out


def _run(lay, fields, nsteps, dt, prec, pml):
    from paper_1812_07357_gb300.solver import Plan
    plan = Plan(lay, (1.0,) * 3, dt, precision=prec, sources="vacuum", pml=pml)
    assert (plan.fast_boxes, plan.pencil_boxes) == (0, 0)      # generic kernels
    df = plan.pack_fields(fields)
    plan.push(df, None, nsteps)
    plan.sync()
    got = plan.unpack_fields(df)
    parts = plan.pml_parts()
    got.update({k: plan.unpack(v) for k, v in parts.items()})
    plan.close()
    return got


def _pml_boxes(lay, pml):
    idx = []
    for i, b in enumerate(lay.boxes):
        for a in range(3):
            w = pml["width"][a]
            if w and (b.origin[a] < w or b.origin[a] + b.interior[a] > lay.global_n[a] - w):
                idx.append(i)
                break
    return idx


def _check(lay, fields, nsteps, dt, prec, pml):
    if prec == 32:
        fields = {k: I.round_to(v, np.float32) for k, v in fields.items()}
    got = _run(lay, fields, nsteps, dt, prec, pml)
    ref = O.push(lay, fields, {}, nsteps, (1.0,) * 3, dt, pml=pml)
    assert_fields(lay, got, ref, O.COMPS, prec, what="fields with absorbing layers")
    # stored split parts, where the layers are (elsewhere they are not tracked)
    sel = _pml_boxes(lay, pml)
    sub = I.Layout(lay.kind, lay.global_n, lay.periodic, [lay.boxes[i] for i in sel])
    for k in PARTS:
        g = [got[k][i] for i in sel]
        r = [ref[k][i] for i in sel]
        l2, mx = O.rel_errors(sub, g, r)
        scale = max(float(np.abs(x).max()) for x in r)
        assert l2 <= TOL[prec] * 10 or scale == 0.0, (k, l2, mx)


@pytest.mark.parametrize("prec", [64, 32])
def test_pml_global_box_pulse_into_layers(prec):
    """128 x 16 x 16 periodic box, layers of 16 cells on the x faces (s_max
    0.4, order 2), p = 16, a pulse launched towards +x, 70 steps of dt = 0.9
    (the pulse crosses the high-x layer and wraps into the low-x one)."""
    lay = I.global_layout((128, 16, 16), 16)
    f = _pulse((128, 16, 16), x0=80.0, tau=6.0, lam=8.0, waist=5.0)
    pml = dict(width=(16, 0, 0), sigma_max=(0.4, 0.0, 0.0), order=2)
    _check(lay, {k: [v] for k, v in f.items()}, 70, 0.9, prec, pml)


@pytest.mark.parametrize("prec", [64, 32])
def test_pml_local_boxes_all_faces(prec):
    """Local decomposition 4 x 2 x 2 of a 64 x 32 x 32 domain (guards 8,
    p = 8) with layers on every face (widths 8, 6, 6; orders 3), a pulse in
    the middle, 20 steps: edge boxes damp, the exchange runs every step."""
    lay = I.local_layout((64, 32, 32), (4, 2, 2), 8, 8)
    f = _pulse((64, 32, 32), x0=32.0, tau=4.0, lam=6.0, waist=4.0)
    fields = {k: I.scatter_global(v, lay) for k, v in f.items()}
    pml = dict(width=(8, 6, 6), sigma_max=(0.5, 0.4, 0.4), order=3)
    _check(lay, fields, 20, 0.7, prec, pml)


def test_pml_rejects_sources_and_wide_layers():
    from paper_1812_07357_gb300 import _abi as A
    from paper_1812_07357_gb300.solver import Plan
    lay = I.global_layout((32, 16, 16), 8)
    with pytest.raises(A.PsatdError):
        Plan(lay, (1.0,) * 3, 0.5, precision=32, sources="rho", pml=dict(width=(4, 0, 0), sigma_max=(1, 0, 0),
                                                                         order=2))
    with pytest.raises(A.PsatdError):
        Plan(lay, (1.0,) * 3, 0.5, precision=32, sources="vacuum", pml=dict(width=(20, 0, 0),
                                                                            sigma_max=(1, 0, 0), order=2))
