"""psatd_push_host: fields in host memory, copied to the plan's device
staging buffers and back inside the call (by the SM copy kernel through the
buffers' device mapping, or by the copy engines).  The result must equal the
device-buffer push bit for bit (same kernels, same data) and match the
oracle; separate in/out host buffers leave the input untouched."""
import numpy as np
import pytest

from oracle import psatd_oracle as O
from paper_1812_07357_gb300 import inputs as I
from _parity import assert_fields

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1812_07357_gb300 import build
    build.build()
    return t


@pytest.mark.parametrize("prec,copy,split,eager", [(32, 1, True, False), (64, 1, True, False), (32, 0, True, False),
                                                  (32, 1, False, False), (32, 1, True, True)])
def test_host_push_equals_device_push_and_oracle(torch, prec, copy, split, eager):
    """split: the first step's forward pass and the last step's inverse pass
    go component by component between the copies (vacuum form); with
    per-kernel timing on, psatd_push runs whole between the copies.  eager:
    the guard exchange after every step (one component at a time after the
    split inverse pass) instead of the deferred one."""
    from paper_1812_07357_gb300 import _abi as A
    from paper_1812_07357_gb300.solver import Plan
    lay = I.local_layout((128, 64, 32), (2, 1, 2), (16, 16, 4), 16)     # register kernels in FP32
    f = I.laser_fields((128, 64, 32), wavelength=8.0, waist=10.0, duration=6.0)
    fields = {k: I.scatter_global(v, lay) for k, v in f.items()}
    if prec == 32:
        fields = {k: I.round_to(v, np.float32) for k, v in fields.items()}
    plan = Plan(lay, (1.0,) * 3, 0.9, precision=prec, sources="vacuum", eager_exchange=eager)
    A.psatd_plan_tune(plan.handle, A.PSATD_TUNE_HOST_COPY, copy)
    assert plan.tuning()["host_copy"] == copy
    dev = plan.pack_fields(fields)
    host_in = {k: v.cpu().pin_memory() for k, v in dev.items()}
    keep = {k: v.clone() for k, v in host_in.items()}
    host_out = {k: torch.empty_like(v).pin_memory() for k, v in host_in.items()}
    if not split:
        A.psatd_plan_set_timing(plan.handle, True)
    plan.push(dev, None, 3)
    plan.push_host(host_in, host_out, None, 3)
    plan.sync()
    torch.cuda.synchronize()
    for k in O.COMPS:
        assert torch.equal(host_out[k], dev[k].cpu()), k
        assert torch.equal(host_in[k], keep[k]), k
    # in place, twice more
    plan.push_host(host_out, None, None, 2)
    torch.cuda.synchronize()
    got = {k: plan.unpack(host_out[k].cuda()) for k in O.COMPS}
    plan.close()
    ref = O.push(lay, fields, {}, 5, (1.0,) * 3, 0.9)
    assert_fields(lay, got, ref, O.COMPS, prec)


@pytest.mark.parametrize("prec,copy,nsteps,split", [(32, 1, 3, True), (64, 1, 3, True), (32, 0, 3, True),
                                                    (32, 1, 1, True), (32, 0, 1, True), (64, 1, 1, True),
                                                    (32, 1, 2, False), (32, 0, 1, False)])
def test_host_global_push_matches_device_push_and_oracle(torch, prec, copy, nsteps, split):
    """Whole-domain host arrays: scattered into the boxes (guards included),
    pushed, interiors gathered back, component by component (split: the
    first step's forward pass and the last step's inverse pass per component
    too; with per-kernel timing on, psatd_push runs whole between the
    scatters and the gathers).  Two calls in place: equal to two device
    pushes of the same boxes bit for bit, and to the oracle."""
    from paper_1812_07357_gb300 import _abi as A
    from paper_1812_07357_gb300.solver import Plan
    g = (128, 64, 32)
    lay = I.local_layout(g, (2, 1, 2), (16, 16, 4), 16)
    f = I.laser_fields(g, wavelength=8.0, waist=10.0, duration=6.0)
    if prec == 32:
        f = {k: I.round_to(v, np.float32) for k, v in f.items()}
    plan = Plan(lay, (1.0,) * 3, 0.9, precision=prec, sources="vacuum")
    A.psatd_plan_tune(plan.handle, A.PSATD_TUNE_HOST_COPY, copy)
    dt_ = torch.float32 if prec == 32 else torch.float64
    host = {k: torch.from_numpy(v.ravel().copy()).to(dt_).pin_memory() for k, v in f.items()}
    boxes = {k: I.scatter_global(v, lay) for k, v in f.items()}
    dev = plan.pack_fields(boxes)
    if not split:
        A.psatd_plan_set_timing(plan.handle, True)
    for _ in range(2):
        plan.push(dev, None, nsteps)
        plan.push_host_global(host, None, None, nsteps)
    torch.cuda.synchronize()
    got_dev = plan.unpack_fields(dev)
    for k in O.COMPS:
        hg = host[k].double().numpy().reshape(g[2], g[1], g[0])
        for b, a in zip(lay.boxes, got_dev[k]):
            o, m = b.origin, b.interior
            assert np.array_equal(hg[o[2]:o[2] + m[2], o[1]:o[1] + m[1], o[0]:o[0] + m[0]],
                                  a[O._interior_slices(b)]), k
    ref = O.push(lay, boxes, {}, 2 * nsteps, (1.0,) * 3, 0.9)
    assert_fields(lay, got_dev, ref, O.COMPS, prec)
    plan.close()
