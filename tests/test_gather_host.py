"""Host logic of the deferred guard exchange (no GPU): for every cell of a
padded plane, the cell the forward pass reads there (psatd_plane_gather)
must be the one whose value the oracle's guard exchange (paper Fig. 1, step
(ii)) stores in that cell.  The expected map comes from the oracle itself:
every box array is filled with a code of (box, cell), the oracle exchanges
the codes, and each padded cell's code names its owner (a zero-filled cell
outside a non-periodic domain is never written by a step, so the pass reads
the cell itself)."""
import numpy as np
import pytest

from oracle import psatd_oracle as O
from paper_1812_07357_gb300 import _abi as A
from paper_1812_07357_gb300 import inputs as I
from paper_1812_07357_gb300.solver import make_desc

SCALE = 10 ** 7          # code = 1 + box * SCALE + cell, exact in FP64


def _expected(lay):
    codes = [1.0 + b * SCALE + np.arange(np.prod(bx.shape), dtype=np.float64).reshape(bx.shape)
             for b, bx in enumerate(lay.boxes)]
    return O.exchange(lay, codes)


def _check_layout(lay, precision=32, planes=None, want_grid=None):
    desc = make_desc(lay, (1.0, 1.0, 1.0), 0.9, precision=precision, sources="vacuum")
    ex = _expected(lay)
    for b, bx in enumerate(lay.boxes):
        n0, n1, n2 = bx.n
        zs = range(n2) if planes is None else [z for z in planes if z < n2]
        for z in zs:
            sb, sc, grid = A.psatd_plane_gather(desc, b, z)
            if want_grid is not None:
                assert grid == want_grid, (b, z)
            code = ex[b][z]                                   # (n1, n0)
            own = (np.arange(n1 * n0).reshape(n1, n0) + z * n1 * n0)
            zero = code == 0
            exp_box = np.where(zero, b, ((code - 1) // SCALE).astype(np.int64))
            exp_cell = np.where(zero, own, ((code - 1) % SCALE).astype(np.int64))
            assert np.array_equal(sb, exp_box), (b, z)
            assert np.array_equal(sc, exp_cell), (b, z)


def test_local_periodic_planes_are_grids():
    lay = I.local_layout((128, 64, 32), (2, 1, 2), (16, 16, 4), 16)
    _check_layout(lay, want_grid=True)


def test_local_open_boundary():
    lay = I.local_layout((128, 64, 32), (2, 2, 2), (16, 8, 4), 8, periodic=(0, 1, 0))
    _check_layout(lay, want_grid=True)


def test_hybrid():
    lay = I.hybrid_layout((96, 48, 40), (2, 1, 1), 8, 8)
    _check_layout(lay, want_grid=True)


def test_independent_self_periodic():
    boxes = [I.Box(n, (g,) * 3, (g,) * 3, (0, 0, 0), 8)
             for n, g in (((48, 40, 32), 8), ((60, 48, 24), 4), ((40, 40, 40), 12))]
    lay = I.Layout("independent", (0, 0, 0), (1, 1, 1), boxes)
    _check_layout(lay, want_grid=True)


def test_guards_wider_than_neighbours_use_rectangle_lists():
    """n_g = 40 on 16-cell interiors: a guard face spans three neighbours."""
    lay = I.local_layout((64, 64, 32), (4, 4, 2), (40, 40, 4), 16)
    _check_layout(lay, planes=[0, 3, 4, 11, 23], want_grid=False)


@pytest.mark.parametrize("precision,want", [(32, False), (64, True)])
def test_16_byte_units(precision, want):
    """Guard width 2: the x bands start at element 2, a 16-byte boundary for
    FP64 only, so only FP64 planes take the grid form; the map is right in
    both."""
    lay = I.local_layout((64, 32, 16), (2, 2, 1), (2, 2, 0), 4)
    _check_layout(lay, precision=precision, want_grid=want)


def test_rejects_bad_arguments():
    lay = I.local_layout((64, 32, 16), (2, 1, 1), (4, 0, 0), 4)
    desc = make_desc(lay, (1.0, 1.0, 1.0), 0.9)
    for box, z in ((-1, 0), (2, 0), (0, 16), (0, -1)):
        with pytest.raises(A.PsatdError):
            A.psatd_plane_gather(desc, box, z)
