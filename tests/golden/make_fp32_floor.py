"""Write fp32_floor.txt: the FP32 rounding floor of the long source runs.

The oracle's FP32 rounding model (oracle.psatd_oracle.push with precision=32:
the same algorithm in FP32 arithmetic and storage, FP64-generated
coefficients rounded once) is run on the FP32-rounded inputs of each case and
compared, per field vector, with the FP64 oracle.  The GPU parity tests of
these cases bound the FP32 error of each field by max(2e-5, 2 x this floor).

Cases (the seeded workloads of paper_1812_07357_gb300.inputs):
  sources_128   128^3 periodic box, p = 16, rho form, filtered constant J,
                200 steps of dt = 0.9 (FP64 reference: one step of 200 dt,
                exact for a time-constant current)
  uneven_300_4  the 4 smallest boxes of the 300-box uneven batch (self-
                periodic, rho form, band-limited constant J), 100 steps

Run: python tests/golden/make_fp32_floor.py   (about 10 minutes on 8 cores)
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import psatd_oracle as O  # noqa: E402
from paper_1812_07357_gb300 import inputs as I  # noqa: E402

GROUPS = {"E": ("Ex", "Ey", "Ez"), "B": ("Bx", "By", "Bz"), "rho": ("rho",)}


def smallest_boxes(lay, count):
    return sorted(range(len(lay.boxes)), key=lambda i: (lay.boxes[i].cells, i))[:count]


def sub_workload(w, idx):
    lay = I.Layout(w.layout.kind, w.layout.global_n, w.layout.periodic, [w.layout.boxes[i] for i in idx])
    pick = lambda d: {k: [v[i] for i in idx] for k, v in d.items()}
    return lay, pick(w.fields), pick(w.src)


def errors(lay, got, ref):
    out = {}
    for g, comps in GROUPS.items():
        rep = I.Layout(lay.kind, lay.global_n, lay.periodic, list(lay.boxes) * len(comps))
        out[g] = O.rel_errors(rep, sum((list(got[c]) for c in comps), []), sum((list(ref[c]) for c in comps), []))
    return out


def main():
    rows = []
    w = I.make_workload("sources_128")
    f = {k: I.round_to(v, np.float32) for k, v in w.fields.items()}
    s = {k: I.round_to(v, np.float32) for k, v in w.src.items()}
    ref = O.push(w.layout, f, s, 1, w.h, w.dt * w.steps, form="rho")
    got = O.push(w.layout, f, s, w.steps, w.h, w.dt, form="rho", precision=32)
    rows += [("sources_128", g, e) for g, e in errors(w.layout, got, ref).items()]
    w = I.make_workload("uneven_300")
    lay, f, s = sub_workload(w, smallest_boxes(w.layout, 4))
    f = {k: I.round_to(v, np.float32) for k, v in f.items()}
    s = {k: I.round_to(v, np.float32) for k, v in s.items()}
    ref = O.push(lay, f, s, w.steps, w.h, w.dt, form="rho")
    got = O.push(lay, f, s, w.steps, w.h, w.dt, form="rho", precision=32)
    rows += [("uneven_300_4", g, e) for g, e in errors(lay, got, ref).items()]
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "fp32_floor.txt")
    with open(path, "w") as fh:
        fh.write("# FP32 rounding floor per field vector (relative L2, max-norm), written by\n"
                 "# make_fp32_floor.py from the oracle's FP32 rounding model against the FP64 oracle\n"
                 "# case field rel_l2 max_norm\n")
        for case, g, (l2, mx) in rows:
            fh.write(f"{case} {g} {l2:.6e} {mx:.6e}\n")
    print(open(path).read())


if __name__ == "__main__":
    main()
