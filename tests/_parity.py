"""Per-field parity checks shared by the GPU tests.

Every field vector (E, B, and rho where present) is compared on its own
against the FP64 oracle, over interior cells, by two norms:

* relative L2  ||got - ref||_2 / ||ref||_2 <= tol,
* max-norm     max|got - ref| / max|ref|   <= MAX_FACTOR * tol.

tol is 1e-12 for FP64 and 2e-5 for FP32 (the FP32 run is compared with the
oracle fed the FP32-rounded inputs, so input rounding is not charged).  The
max-norm bound: for an error that is spread over the box like rounding noise,
its largest cell is sqrt(2 ln n) ~ 5-6 times its rms over n ~ 1e4-1e7 cells,
while max|ref| >= rms(ref); so max-norm <= ~6 x relative L2, and 10 x tol
leaves room for the cell statistics of small boxes.
"""
import numpy as np

from oracle import psatd_oracle as O
from paper_1812_07357_gb300 import inputs as I

TOL = {64: 1e-12, 32: 2e-5}
MAX_FACTOR = 10.0
GROUPS = {"E": ("Ex", "Ey", "Ez"), "B": ("Bx", "By", "Bz"), "rho": ("rho",)}


def field_errors(lay, got, ref, comps):
    """{field: (relative L2, max-norm)} over the interior cells of every box,
    for each field vector whose components are all in `comps`."""
    out = {}
    for g, cs in GROUPS.items():
        if not all(c in comps for c in cs):
            continue
        rep = I.Layout(lay.kind, lay.global_n, lay.periodic, list(lay.boxes) * len(cs))
        out[g] = O.rel_errors(rep, sum((list(got[c]) for c in cs), []), sum((list(ref[c]) for c in cs), []))
    return out


def assert_fields(lay, got, ref, comps, prec=None, tol=None, what=""):
    """Assert every field vector within its bound; tol may be a number or a
    {field: bound} dict (fields not listed take TOL[prec])."""
    errs = field_errors(lay, got, ref, comps)
    for g, (l2, mx) in errs.items():
        t = tol.get(g, TOL[prec]) if isinstance(tol, dict) else (tol if tol is not None else TOL[prec])
        assert l2 <= t, (what, g, "rel L2", l2, t, errs)
        assert mx <= MAX_FACTOR * t, (what, g, "max-norm", mx, MAX_FACTOR * t, errs)
    return errs


def assert_arrays(a, b, prec=None, tol=None, what=""):
    """Relative L2 and max-norm of two lists of arrays (no layout)."""
    t = tol if tol is not None else TOL[prec]
    num = sum(float(np.sum(np.abs(x - y) ** 2)) for x, y in zip(a, b))
    den = sum(float(np.sum(np.abs(y) ** 2)) for y in b)
    l2 = (num / den) ** 0.5 if den > 0 else num ** 0.5
    dm = max(float(np.abs(x - y).max()) for x, y in zip(a, b))
    rm = max(float(np.abs(y).max()) for y in b)
    mx = dm / rm if rm > 0 else dm
    assert l2 <= t, (what, "rel L2", l2, t)
    assert mx <= MAX_FACTOR * t, (what, "max-norm", mx, MAX_FACTOR * t)
    return l2, mx
