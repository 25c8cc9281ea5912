"""Host-side tests of the C ABI (no GPU): the library loads and exports every
symbol declared in include/psatd.h, descriptions are validated, and the
precomputed guard-exchange protocol fills guards exactly like the oracle's
exchange when applied on host arrays."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle import psatd_oracle as O
from paper_1812_07357_gb300 import _abi as A
from paper_1812_07357_gb300 import build as B
from paper_1812_07357_gb300 import inputs as I
from paper_1812_07357_gb300.solver import make_desc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return A.load()


def header_functions():
    txt = open(os.path.join(ROOT, "include", "psatd.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(psatd_\w+)\s*\(", txt)))


def test_exports_every_declared_symbol(lib):
    names = header_functions()
    assert "psatd_push" in names and "psatd_plan_create" in names
    for n in names:
        assert hasattr(lib, n), n
        assert n in A._SIGS, f"binding lacks {n}"


def test_status_strings(lib):
    for s in range(8):
        assert A.psatd_status_string(s)
    assert A.psatd_status_string(0) == "ok"


def _desc(layout, **kw):
    return make_desc(layout, (1.0, 1.0, 1.0), 0.5, **kw)


def test_validate_accepts_workload_layouts(lib):
    for lay in (I.global_layout((32, 32, 32), 0), I.local_layout((64, 64, 64), (4, 4, 4), 8, 16),
                I.hybrid_layout((128, 32, 32), (4, 1, 1), 8, 8), I.independent_layout(nboxes=20)):
        st, msg = A.psatd_plan_validate(_desc(lay))
        assert st == A.PSATD_OK, msg


@pytest.mark.parametrize("case,expected", [
    ("odd", A.PSATD_ERR_UNSUPPORTED_SIZE),
    ("seven", A.PSATD_ERR_UNSUPPORTED_SIZE),
    ("big", A.PSATD_ERR_UNSUPPORTED_SIZE),
    ("guards", A.PSATD_ERR_INVALID_ARG),
    ("order", A.PSATD_ERR_UNSUPPORTED_ORDER),
    ("prec", A.PSATD_ERR_INVALID_ARG),
    ("dt", A.PSATD_ERR_INVALID_ARG),
    ("flags", A.PSATD_ERR_INVALID_ARG),
    ("cover", A.PSATD_ERR_INVALID_ARG),
    ("overlap", A.PSATD_ERR_INVALID_ARG),
])
def test_validate_rejects(lib, case, expected):
    lay = I.local_layout((32, 16, 16), (2, 1, 1), 4, 8)
    kw = {}
    d = _desc(lay)
    b = d._boxes
    if case == "odd":
        b[0].n[0] = 25
    elif case == "seven":
        b[0].n[1] = 28
    elif case == "big":
        b[0].n[2] = 1024
    elif case == "guards":
        b[0].ng_lo[0] = 12
        b[0].ng_hi[0] = 12
    elif case == "order":
        b[1].order_p = 7
    elif case == "prec":
        d.precision = 16
    elif case == "dt":
        d.dt = 0.0
    elif case == "flags":
        d.flags = A.PSATD_VACUUM | A.PSATD_RHO_CONTINUITY
    elif case == "cover":
        d.global_n[0] = 40
    elif case == "overlap":
        b[1].origin[0] = 8
    st, msg = A.psatd_plan_validate(d)
    assert st == expected, msg
    assert msg and msg != "ok"


def test_plan_create_rejects_before_touching_gpu(lib):
    lay = I.global_layout((30, 30, 30), 0)
    d = _desc(lay)
    d._boxes[0].n[0] = 31
    with pytest.raises(A.PsatdError) as e:
        A.psatd_plan_create(d)
    assert e.value.status == A.PSATD_ERR_UNSUPPORTED_SIZE
    assert "31" in A.psatd_last_error()


def _apply_blocks(layout, blocks, arrays):
    out = [a.copy() for a in arrays]
    for bl in blocks:
        ex, ey, ez = bl.ext
        dx, dy, dz = bl.dst_lo
        if bl.src_box < 0:
            out[bl.dst_box][dz:dz + ez, dy:dy + ey, dx:dx + ex] = 0.0
        else:
            sx, sy, sz = bl.src_lo
            out[bl.dst_box][dz:dz + ez, dy:dy + ey, dx:dx + ex] = \
                arrays[bl.src_box][sz:sz + ez, sy:sy + ey, sx:sx + ex]
    return out


@pytest.mark.parametrize("kind", ["local", "local_open", "hybrid", "hybrid_yz", "independent",
                                  "uneven_local"])
def test_exchange_blocks_match_oracle_exchange(lib, kind):
    if kind == "local":
        lay = I.local_layout((24, 16, 16), (3, 2, 2), 4, 8)
    elif kind == "local_open":
        lay = I.local_layout((24, 16, 16), (3, 2, 2), 2, 8, periodic=(0, 1, 0))
    elif kind == "hybrid":
        lay = I.hybrid_layout((48, 12, 10), (4, 1, 1), 6, 8)
    elif kind == "hybrid_yz":
        lay = I.hybrid_layout((20, 24, 24), (1, 2, 3), 2, 8)
    elif kind == "independent":
        lay = I.independent_layout(seed=9, nboxes=5, sizes=(8, 10, 12, 16), ngs=(1, 2, 3),
                                   min_interior=4)
    else:
        # unequal sub-domains, one spanning the whole periodic x extent
        boxes = [I.Box((24, 12, 8), (0, 2, 2), (0, 2, 2), (0, 0, 0), 4),
                 I.Box((24, 16, 8), (0, 2, 2), (0, 2, 2), (0, 8, 0), 4),
                 I.Box((24, 30, 8), (0, 3, 2), (0, 3, 2), (0, 20, 0), 4)]
        lay = I.Layout("local", (24, 44, 4), (1, 1, 1), boxes)
    rng = np.random.default_rng(3)
    arrs = [rng.standard_normal(b.shape) for b in lay.boxes]
    blocks = A.psatd_exchange_blocks(_desc(lay))
    got = _apply_blocks(lay, blocks, arrs)
    ref = O.exchange(lay, arrs)
    for g, r in zip(got, ref):
        assert np.array_equal(g, r)
    # only guard cells are written, only interior cells are read
    for bl in blocks:
        box = lay.boxes[bl.dst_box]
        inside = all(box.ng_lo[d] <= bl.dst_lo[d] and bl.dst_lo[d] + bl.ext[d] <= box.n[d] - box.ng_hi[d]
                     for d in range(3))
        assert not inside
        if bl.src_box >= 0:
            sb = lay.boxes[bl.src_box]
            assert all(sb.ng_lo[d] <= bl.src_lo[d] and bl.src_lo[d] + bl.ext[d] <= sb.n[d] - sb.ng_hi[d]
                       for d in range(3))


def test_exchange_block_count_local_512():
    """Full local workload: 512 boxes x 26 neighbour regions."""
    B.build()
    lay = I.local_layout((512, 512, 512), (8, 8, 8), 16, 32)
    blocks = A.psatd_exchange_blocks(_desc(lay))
    assert len(blocks) == 512 * 26
    vol = sum(b.ext[0] * b.ext[1] * b.ext[2] for b in blocks)
    assert vol == lay.guard_cells


# ---------------------------------------------------------------------------
# dual-grid coupling (host-only block computation)
# ---------------------------------------------------------------------------

def _apply_coupling(blocks, dst_arrays, src_arrays):
    out = [a.copy() for a in dst_arrays]
    for bl in blocks:
        ex, ey, ez = bl.ext
        dx, dy, dz = bl.dst_lo
        if bl.src_box < 0:
            out[bl.dst_box][dz:dz + ez, dy:dy + ey, dx:dx + ex] = 0.0
        else:
            sx, sy, sz = bl.src_lo
            out[bl.dst_box][dz:dz + ez, dy:dy + ey, dx:dx + ex] = \
                src_arrays[bl.src_box][sz:sz + ez, sy:sy + ey, sx:sx + ex]
    return out


@pytest.mark.parametrize("periodic", [(1, 1, 1), (0, 1, 1)])
def test_coupling_blocks_match_oracle(lib, periodic):
    g2 = I.hybrid_layout((32, 12, 10), (2, 1, 1), 4, 8, periodic=periodic)     # FFT grid
    g1 = I.local_layout((32, 12, 10), (4, 3, 2), (1, 2, 1), 4, periodic=periodic)   # particle grid
    rng = np.random.default_rng(5)
    a1 = [rng.standard_normal(b.shape) for b in g1.boxes]
    a2 = [rng.standard_normal(b.shape) for b in g2.boxes]
    d = _desc(g2)
    fwd = A.psatd_coupling_blocks(d, g1.boxes, A.PSATD_G1_TO_G2)
    for g, r in zip(_apply_coupling(fwd, [np.full(b.shape, np.nan) for b in g2.boxes], a1), O.couple(g1, a1, g2)):
        assert np.array_equal(g, r)          # every G2 cell written
    back = A.psatd_coupling_blocks(d, g1.boxes, A.PSATD_G2_TO_G1)
    for g, r in zip(_apply_coupling(back, [np.full(b.shape, np.nan) for b in g1.boxes], a2), O.couple(g2, a2, g1)):
        assert np.array_equal(g, r)
    # sources read interior cells only
    for blocks, src in ((fwd, g1), (back, g2)):
        for bl in blocks:
            if bl.src_box >= 0:
                sb = src.boxes[bl.src_box]
                assert all(sb.ng_lo[k] <= bl.src_lo[k] and bl.src_lo[k] + bl.ext[k] <= sb.n[k] - sb.ng_hi[k]
                           for k in range(3))


def test_coupling_rejects_bad_g1(lib):
    g2 = I.local_layout((16, 16, 16), (2, 2, 2), 4, 4)
    d = _desc(g2)
    gap = I.local_layout((16, 16, 16), (2, 2, 2), 1, 4).boxes[:-1]                       # a hole
    over = list(I.local_layout((16, 16, 16), (2, 2, 2), 1, 4).boxes)
    over[1] = I.Box(over[1].n, over[1].ng_lo, over[1].ng_hi, (4, 0, 0), 4)                 # overlap + hole
    outside = [I.Box((18, 18, 18), (1,) * 3, (1,) * 3, (8, 0, 0), 4)]                      # past the domain
    for boxes in (gap, over, outside):
        with pytest.raises(A.PsatdError) as e:
            A.psatd_coupling_blocks(d, boxes, A.PSATD_G1_TO_G2)
        assert e.value.status == A.PSATD_ERR_INVALID_ARG
    with pytest.raises(A.PsatdError):
        A.psatd_coupling_blocks(d, I.local_layout((16, 16, 16), (2, 2, 2), 1, 4).boxes, 2)
    ind = I.independent_layout(seed=3, nboxes=2, sizes=(8, 10), ngs=(1,), min_interior=4)
    with pytest.raises(A.PsatdError):
        A.psatd_coupling_blocks(_desc(ind), ind.boxes, A.PSATD_G1_TO_G2)


@pytest.mark.parametrize("case", ["ok", "sources", "nodal", "independent", "wide", "sigma", "order"])
def test_validate_absorbing_layers(lib, case):
    lay = I.local_layout((32, 16, 16), (2, 1, 1), 4, 8)
    pml = dict(width=(4, 2, 0), sigma_max=(1.0, 0.5, 0.0), order=2)
    kw = {"sources": "vacuum"}
    if case == "sources":
        kw["sources"] = "J"
    elif case == "nodal":
        kw["nodal"] = True
    elif case == "independent":
        lay = I.independent_layout(nboxes=3)
    elif case == "wide":
        pml["width"] = (17, 0, 0)
    elif case == "sigma":
        pml["sigma_max"] = (-1.0, 0.0, 0.0)
    elif case == "order":
        pml["order"] = 17
    st, msg = A.psatd_plan_validate(_desc(lay, pml=pml, **kw))
    assert (st == A.PSATD_OK) == (case == "ok"), (case, msg)
    if case != "ok":
        assert st == A.PSATD_ERR_INVALID_ARG, msg


def test_validate_rejects_an_empty_plan(lib):
    d = _desc(I.global_layout((16, 16, 16), 8))
    d.num_boxes = 0
    st, msg = A.psatd_plan_validate(d)
    assert st == A.PSATD_ERR_INVALID_ARG and "box" in msg


def test_header_constants_match_the_binding():
    """Every PSATD_* integer constant of include/psatd.h that the ctypes
    binding names has the header's value; every tuning knob is in TUNE_KNOBS."""
    txt = open(os.path.join(ROOT, "include", "psatd.h")).read()
    consts = {k: int(v) for k, v in re.findall(r"^#define\s+(PSATD_\w+)\s+(-?\d+)\s*(?:/\*.*)?$", txt, re.M)}
    named = [k for k in consts if hasattr(A, k)]
    assert len(named) >= 10
    for k in named:
        assert getattr(A, k) == consts[k], k
    knobs = {v for k, v in consts.items() if k.startswith("PSATD_TUNE_")}
    assert knobs == set(A.TUNE_KNOBS.values())


@pytest.mark.parametrize("knob,value", [("reg_planes", 2), ("pencil_reg_z", -1), ("z_one_launch", 3),
                                        ("z_tile", 0), ("pencil_rows_kb", 4)])
def test_validate_rejects_bad_tuning(lib, knob, value):
    lay = I.global_layout((48, 48, 48), 4)
    d = make_desc(lay, (1.0,) * 3, 0.5, tuning={knob: value})
    st, msg = A.psatd_plan_validate(d)
    assert st == A.PSATD_ERR_INVALID_ARG and "tuning knob" in msg, (st, msg)
