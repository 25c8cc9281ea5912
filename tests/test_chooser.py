"""Group-size chooser: candidate decompositions against the paper's memory
model (eqs. (1), (3)), the least-squares cost fit, and (GPU) a measured
choice."""
import numpy as np
import pytest

from oracle import psatd_oracle as O
from paper_1812_07357_gb300 import chooser as C


def test_candidates_match_memory_model():
    n, n_p, ng = 96, 4, 8
    cands = C.candidates((n, n, n), (n_p,) * 3, ng, 16)
    names = {c.name for c in cands}
    assert "local" in names and "hybrid 2x2x2" in names
    for c in cands:
        if c.merge == (1, 1, 1):
            assert c.padded_cells == O.memory_local(n, n_p, ng)
        m = c.merge[0]
        if c.merge == (m, m, m) and m < n_p:
            assert c.padded_cells == O.memory_hybrid(n, n_p, ng, m)
        assert all(C.valid_box(b.n) for b in c.layout.boxes)
    # every candidate tiles the domain: interiors add up to n^3
    assert all(c.layout.interior_cells == n ** 3 for c in cands)


def test_invalid_boxes_are_skipped():
    # local boxes 22 + 2 x 5 = 32 on every axis (valid); the single group
    # (66 x 22 x 22, periodic, no guards) is not 5-smooth
    cands = C.candidates((66, 22, 22), (3, 1, 1), 5, 8)
    assert [c.name for c in cands] == ["local"]


def test_fit_recovers_model_coefficients():
    cands = C.candidates((128, 64, 64), (4, 2, 2), 8, 16)
    a, b, g = 2e-9, 3e-7, 5e-7
    for c in cands:
        c.ms_per_step = a * c.nlogn + b * c.padded_cells + g * c.guard_cells
    coef = C.fit(cands)
    assert np.allclose(coef, [a, b, g], rtol=1e-6)
    assert all(abs(c.model_ms - c.ms_per_step) <= 1e-9 * c.ms_per_step for c in cands)


def test_choose_without_measurement_takes_smallest_volume():
    best, report = C.choose((96, 96, 96), (4, 4, 4), 8, 16, run=False)
    assert best.padded_cells == min(c.padded_cells for c in report)


@pytest.mark.gpu
def test_choose_measures_and_fits():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    best, report = C.choose((128, 64, 64), (4, 2, 2), 8, 16, steps=2, warmup=1)
    assert all(c.ms_per_step > 0 and c.memory_bytes > 0 for c in report)
    assert best.ms_per_step == min(c.ms_per_step for c in report)
    assert all(c.model_ms is not None for c in report)
    tight = min(c.memory_bytes for c in report)
    best2, _ = C.choose((128, 64, 64), (4, 2, 2), 8, 16, budget_bytes=tight, steps=2, warmup=1)
    assert best2.memory_bytes <= tight
