"""Autotuner: the stage-wise search and the cache (CPU, with a fake
measurement), and on the GPU a tuned plan that matches the oracle."""
import json

import numpy as np
import pytest

from paper_1812_07357_gb300 import autotune as T
from paper_1812_07357_gb300 import inputs as I


def test_signature_depends_on_boxes_precision_form_and_device():
    a = I.local_layout((64, 64, 64), (2, 2, 2), 8, 16)
    b = I.local_layout((64, 64, 64), (2, 2, 2), 8, 8)
    s = T.signature(a, 32, "vacuum", device="X")
    assert s == T.signature(I.local_layout((64, 64, 64), (2, 2, 2), 8, 16), 32, "vacuum", device="X")
    assert len({s, T.signature(b, 32, "vacuum", device="X"), T.signature(a, 64, "vacuum", device="X"),
                T.signature(a, 32, "rho", device="X"), T.signature(a, 32, "vacuum", device="Y")}) == 5


def test_search_stages_and_cache(tmp_path):
    calls = []

    def measure(family, tuning):
        calls.append((family, dict(tuning)))
        # pencil is fastest; among its knobs z_tile 2 and 32 KiB rows win
        base = {"default": 5.0, "plane": 7.0, "pencil": 4.0, "generic": 9.0}[family]
        ms = base - (0.5 if tuning.get("z_tile") == 2 else 0) - (0.25 if tuning.get("pencil_rows_kb") == 32 else 0)
        used = {"z_tile": tuning.get("z_tile", 8), "pencil_rows_kb": tuning.get("pencil_rows_kb", 64)} \
            if family == "pencil" else {}
        return ms, used

    lay = I.independent_layout(seed=3, nboxes=5, sizes=(48, 60), ngs=(4,), min_interior=16)
    cache = str(tmp_path / "tune.json")
    c = T.tune(lay, (1.0,) * 3, 0.9, cache=cache, measure=measure, device="test")
    assert (c["family"], c["tuning"], c["cached"]) == ("pencil", {"z_tile": 2, "pencil_rows_kb": 32}, False)
    assert c["ms_per_step"] == 3.25
    # four families; z_tile 4 and 2 (8 is the default); rows 16, 32, then 64
    # (no longer the current best's value once 32 won) and 128
    assert len(calls) == 4 + 2 + 4
    again = T.tune(lay, (1.0,) * 3, 0.9, cache=cache, measure=measure, device="test")
    assert again["cached"] and len(calls) == 10
    d = json.load(open(cache))
    assert len(d) == 1 and list(d.values())[0]["family"] == "pencil"


@pytest.mark.gpu
def test_tuned_plan_matches_the_oracle(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from oracle import psatd_oracle as O
    from paper_1812_07357_gb300 import build
    from _parity import assert_fields
    build.build()
    lay = I.independent_layout(seed=11, nboxes=6, sizes=(48, 60, 80), ngs=(4, 8), min_interior=16)
    cache = str(tmp_path / "tune.json")
    c = T.tune(lay, (1.0,) * 3, 0.9, precision=32, sources="rho", cache=cache, j_constant=True)
    assert not c["cached"] and len(c["trials"]) >= 4
    assert c["ms_per_step"] == min(t["ms_per_step"] for t in c["trials"])
    plan = T.tuned_plan(lay, (1.0,) * 3, 0.9, precision=32, sources="rho", cache=cache, j_constant=True)
    assert plan.tuning().items() >= c["tuning"].items()
    rng = np.random.default_rng(12)
    js = {k: [] for k in ("Jx", "Jy", "Jz")}
    for b in lay.boxes:
        j = I.band_limited_current(b.interior, rng)
        for k in js:
            js[k].append(j[k])
    src = {k: I.round_to(I.scatter_self(v, lay), np.float32) for k, v in js.items()}
    src["rho"] = I.zeros(lay)
    fields = {k: I.zeros(lay) for k in O.COMPS}
    df = plan.pack_fields(fields)
    ds = plan.pack_fields(src)
    plan.push(df, ds, 4)
    plan.sync()
    got = plan.unpack_fields(df)
    got["rho"] = plan.unpack(ds["rho"])
    plan.close()
    ref = O.push(lay, fields, src, 4, (1.0,) * 3, 0.9, form="rho")
    assert_fields(lay, got, ref, O.COMPS + ("rho",), 32, what=f"tuned plan {c['family']} {c['tuning']}")


def test_search_skips_and_drops_knobs_the_chosen_plan_does_not_use(tmp_path):
    """A knob that the best plan no longer uses (z_one_launch once
    pencil_reg_z = 0 won) is neither searched nor kept in the result."""
    calls = []

    def measure(family, tuning):
        calls.append((family, dict(tuning)))
        base = {"default": 5.0, "plane": 7.0, "pencil": 6.0, "generic": 9.0}[family]
        reg_z = tuning.get("pencil_reg_z", 1)
        ms = base - (0.5 if reg_z == 0 else 0.0)
        used = {"pencil_reg_z": reg_z}
        if reg_z:
            used["z_one_launch"] = tuning.get("z_one_launch", 0)
        return ms, used

    lay = I.independent_layout(seed=3, nboxes=5, sizes=(48, 60), ngs=(4,), min_interior=16)
    c = T.tune(lay, (1.0,) * 3, 0.9, cache=str(tmp_path / "t.json"), measure=measure, device="test")
    assert (c["family"], c["tuning"], c["ms_per_step"]) == ("default", {"pencil_reg_z": 0}, 4.5)
    assert len(calls) == 4 + 1
    assert not any("z_one_launch" in t for _, t in calls)
