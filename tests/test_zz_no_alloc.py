"""psatd_push_box_static: the push for callers that may not allocate device
memory (for example code running under a framework that owns every device
allocation).  It keeps its workspace and tables in the library's static
device array instead of cudaMalloc'd plan memory, so its results must equal
those of the ordinary plan-based psatd_push on the same box, and both must
match the FP64 oracle.

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test.
"""
import numpy as np
import pytest

from _parity import assert_fields

pytestmark = pytest.mark.gpu

FP32_TOL = 2e-5   # the FP32 relative-L2 bound used by every GPU parity test
COMPS = ("Ex", "Ey", "Ez", "Bx", "By", "Bz")


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1812_07357_gb300 import build
    build.build()
    from paper_1812_07357_gb300 import _abi as A
    A.load()
    return torch, A


def _rel_l2(a, b):
    return float(((a - b).double().norm() / b.double().norm()).item())


def test_static_push_matches_plan_push_on_two_calls(env):
    torch, A = env
    from paper_1812_07357_gb300 import inputs as I
    from paper_1812_07357_gb300.solver import Plan
    n, p, dx, dt, c = (48, 40, 36), 16, (1.0, 0.9, 1.1), 0.7, 1.0
    rng = np.random.default_rng(31)
    f = {k: rng.standard_normal((n[2], n[1], n[0])).astype(np.float32) for k in COMPS}
    lay = I.global_layout(n, p)
    plan = Plan(lay, dx, dt, c=c, precision=32, sources="vacuum")
    ref = plan.pack_fields({k: [v] for k, v in f.items()})
    got = {k: torch.from_numpy(v.ravel().copy()).cuda() for k, v in f.items()}
    cells = n[0] * n[1] * n[2]
    stream = plan.stream.cuda_stream
    # the FP64 oracle on the same FP32 inputs, 3 and 6 steps: an anchor that
    # does not go through the plan's code path
    from oracle import psatd_oracle as O
    f64 = {k: [v.astype(np.float64)] for k, v in f.items()}
    want = [O.push(lay, f64, {}, 3, dx, dt, c=c), O.push(lay, f64, {}, 6, dx, dt, c=c)]
    for call in range(2):
        plan.push(ref, None, 3)
        A.psatd_push_box_static(n, p, dx, dt, c, Plan.fields_struct(got), 3, stream)
        torch.cuda.synchronize()
        for k in COMPS:
            err = _rel_l2(got[k], ref[k][:cells])
            assert err <= FP32_TOL, (call, k, err)
        out = {k: [got[k].cpu().numpy().astype(np.float64).reshape(n[2], n[1], n[0])] for k in COMPS}
        assert_fields(lay, out, want[call], COMPS, 32, what=f"static push, call {call}")
    plan.close()


def test_static_push_rejects_boxes_beyond_the_scratch(env):
    torch, A = env
    from paper_1812_07357_gb300.solver import Plan
    z = {k: torch.zeros(16, dtype=torch.float32, device="cuda") for k in COMPS}
    with pytest.raises(A.PsatdError) as e:
        A.psatd_push_box_static((160, 160, 160), 8, (1.0,) * 3, 0.5, 1.0, Plan.fields_struct(z), 1)
    assert e.value.status == A.PSATD_ERR_UNSUPPORTED_SIZE
    assert str(A.PSATD_STATIC_SCRATCH_BYTES) in str(e.value)
