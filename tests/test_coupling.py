"""Dual-grid coupling on the GPU (paper Sec. 2.5.2): the copies G1 -> G2 and
G2 -> G1 are bit-exact against the oracle's coupling, and a dual-grid cycle
(fill the FFT grid from the particle grid, push it, copy the fields back)
matches the oracle running the same cycle."""
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


def _grids(periodic=(1, 1, 1)):
    g2 = I.hybrid_layout((64, 24, 20), (2, 1, 1), 8, 8, periodic=periodic)        # FFT boxes 48 x 24 x 20
    g1 = I.local_layout((64, 24, 20), (4, 3, 2), (1, 2, 1), 8, periodic=periodic)  # particle grid
    return g1, g2


@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("periodic", [(1, 1, 1), (0, 1, 1)])
def test_couple_both_directions_bit_exact(prec, periodic):
    from paper_1812_07357_gb300.solver import Coupling, Plan
    g1, g2 = _grids(periodic)
    rng = np.random.default_rng(8)
    rnd = lambda lay: [I.round_to([rng.standard_normal(b.shape)], np.float32)[0] if prec == 32 else
                       rng.standard_normal(b.shape) for b in lay.boxes]
    a1 = {k: rnd(g1) for k in O.COMPS}
    a2 = {k: rnd(g2) for k in O.COMPS}
    plan = Plan(g2, (1.0, 1.0, 1.0), 0.9, precision=prec, sources="vacuum")
    cp = Coupling(plan, g1)
    d1 = {k: cp.pack(v) for k, v in a1.items()}
    d2 = {k: plan.pack(v) for k, v in a2.items()}
    cp.to_fft(d1, d2)
    plan.sync()
    for k in O.COMPS:
        for g, r in zip(plan.unpack(d2[k]), O.couple(g1, a1[k], g2)):
            assert np.array_equal(g, r), k
    d2 = {k: plan.pack(v) for k, v in a2.items()}
    cp.from_fft(d2, d1)
    plan.sync()
    for k in O.COMPS:
        for g, r in zip(cp.unpack(d1[k]), O.couple(g2, a2[k], g1)):
            assert np.array_equal(g, r), k
    cp.close()
    plan.close()


@pytest.mark.parametrize("prec", [64, 32])
def test_dual_grid_cycle(prec):
    """Three PIC-cycle field steps: G1 -> G2 (FFT boxes with their guards),
    push the FFT grid one step, G2 -> G1."""
    from paper_1812_07357_gb300.solver import Coupling, Plan
    g1, g2 = _grids()
    f = I.laser_fields((64, 24, 20), wavelength=8.0, waist=6.0, duration=6.0)
    a1 = {k: I.scatter_global(v, g1) for k, v in f.items()}
    if prec == 32:
        a1 = {k: I.round_to(v, np.float32) for k, v in a1.items()}
    plan = Plan(g2, (1.0, 1.0, 1.0), 0.9, precision=prec, sources="vacuum")
    cp = Coupling(plan, g1)
    d1 = {k: cp.pack(v) for k, v in a1.items()}
    d2 = {k: plan.empty() for k in O.COMPS}
    ref = a1
    for _ in range(3):
        cp.to_fft(d1, d2)
        plan.push(d2, None, 1)
        cp.from_fft(d2, d1)
        r2 = {k: O.couple(g1, ref[k], g2) for k in O.COMPS}
        r2 = O.push(g2, r2, {}, 1, (1.0, 1.0, 1.0), 0.9, form="vacuum")
        ref = {k: O.couple(g2, r2[k], g1) for k in O.COMPS}
    plan.sync()
    got = {k: cp.unpack(d1[k]) for k in O.COMPS}
    assert_fields(g1, got, ref, O.COMPS, prec)
    cp.close()
    plan.close()
