"""The device work of a group spread over ranks (paper Sec. 2.4.1: the group's
FFT distributed axis by axis over ranks; Sec. 2.6: the spectrum solved in the
transposed layout, two transpositions per step), run for several ranks on one
GPU: each rank is a plan of the group box distributed with
psatd_plan_distribute, its x, y transforms, z transform + update + inverse z
transform and inverse y, x transforms go through the psatd_dist_* calls, and
the two all-to-alls between the ranks' slabs and rows are done by copies on
the device (what NCCL would move between GPUs).  Checked against the oracle's
single-box push of the group, and bit for bit against one rank holding the
whole group (every line and every mode is transformed and updated alone, so
the partition must not change a bit)."""
import numpy as np
import pytest

from oracle import psatd_oracle as O
from paper_1812_07357_gb300 import inputs as I

from _parity import assert_fields

COMPS = ("Ex", "Ey", "Ez", "Bx", "By", "Bz")


def _slot_names(form):
    return COMPS + {"vacuum": (), "J": ("Jx", "Jy", "Jz"), "rho": ("rho", "Jx", "Jy", "Jz")}[form]


def _run_ranks(n, p, h, dt, form, prec, world, full, nsteps):
    """`nsteps` steps of the group on `world` emulated ranks; returns the
    assembled output components {name: (n2, n1, n0)} (numpy)."""
    import torch
    from paper_1812_07357_gb300 import distributed as D
    from paper_1812_07357_gb300.solver import Plan

    lay = I.global_layout(n, p)
    names = _slot_names(form)
    dtype = torch.float64 if prec == 64 else torch.float32
    dev = torch.device("cuda", 0)
    plans = [Plan(lay, h, dt, precision=prec, sources=form) for _ in range(world)]
    ranks = [D.DeviceRank(pl, world, r) for r, pl in enumerate(plans)]
    g = torch.stack([torch.from_numpy(full[k]) for k in names]).to(dev, dtype)   # (F, n2, n1, n0)
    slabs = [g[:, rk.z0:rk.z1].contiguous() for rk in ranks]
    nout = ranks[0].nout
    for _ in range(nsteps):
        specs = [rk.xy_forward(s) for rk, s in zip(ranks, slabs)]
        # all-to-all: rank r receives the rows [y0_r, y1_r) of every slab
        rows = [torch.cat([sp[:, :, rk.y0:rk.y1] for sp in specs], dim=1).contiguous() for rk in ranks]
        rows = [rk.z_update(rw, rk.y0) for rk, rw in zip(ranks, rows)]
        # and back: rank r receives the planes [z0_r, z1_r) of every rank's rows
        specs = [torch.cat([rw[:, rk.z0:rk.z1] for rw in rows], dim=2).contiguous() for rk in ranks]
        outs = [rk.yx_inverse(sp) for rk, sp in zip(ranks, specs)]
        # the next step's slabs: new E, B (rho), the constant current
        slabs = [torch.cat([o, s[nout:]]) if nout < len(names) else o.contiguous() for o, s in zip(outs, slabs)]
    torch.cuda.synchronize()
    got = torch.cat([s[:nout] for s in slabs], dim=1).cpu().numpy()
    for pl in plans:
        pl.close()
    return {k: got[i] for i, k in enumerate(names[:nout])}


def _inputs(n, form, seed):
    n0, n1, n2 = n
    rng = np.random.default_rng(seed)
    full = {k: rng.standard_normal((n2, n1, n0)) for k in _slot_names(form)}
    return full


@pytest.mark.gpu
@pytest.mark.parametrize("world,prec,form,p", [(2, 64, "vacuum", 8), (3, 64, "rho", 16), (3, 64, "J", 0),
                                               (2, 32, "vacuum", 8), (4, 32, "rho", 0)])
def test_distributed_ranks_match_the_oracle(world, prec, form, p):
    n, h, dt, nsteps = (16, 12, 10), (1.0, 0.9, 1.1), 0.7, 3
    full = _inputs(n, form, 91 + world)
    if prec == 32:
        full = {k: v.astype(np.float32).astype(np.float64) for k, v in full.items()}
    got = _run_ranks(n, p, h, dt, form, prec, world, full, nsteps)
    lay = I.global_layout(n, p)
    fields = {k: [full[k]] for k in COMPS}
    src = {k: [full[k]] for k in _slot_names(form)[6:]}
    ref = O.push(lay, fields, src, nsteps, h, dt, form=form)
    comps = tuple(got)
    assert_fields(lay, {k: [got[k]] for k in comps}, {k: [ref[k][0]] for k in comps}, comps, prec=prec,
                  what=f"{world} ranks, {form}, FP{prec}")


@pytest.mark.gpu
@pytest.mark.parametrize("prec", [64, 32])
def test_distributed_ranks_bit_identical_to_one_rank(prec):
    n, h, dt, p = (20, 16, 12), (1.0, 1.0, 1.0), 0.9, 32
    full = _inputs(n, "rho", 7)
    one = _run_ranks(n, p, h, dt, "rho", prec, 1, full, 2)
    for world in (2, 3, 5):
        got = _run_ranks(n, p, h, dt, "rho", prec, world, full, 2)
        for k in one:
            assert np.array_equal(got[k], one[k]), (world, k)


@pytest.mark.gpu
def test_distribute_rejects_what_it_cannot_split():
    from paper_1812_07357_gb300 import _abi as A
    from paper_1812_07357_gb300.solver import Plan
    lay = I.global_layout((16, 12, 10), 8)
    pl = Plan(lay, (1.0, 1.0, 1.0), 0.5, precision=64, sources="vacuum")
    with pytest.raises(A.PsatdError):
        A.psatd_dist_z_update(pl.handle, 0)                  # before psatd_plan_distribute
    with pytest.raises(A.PsatdError):
        A.psatd_plan_distribute(pl.handle, 11, 0)            # more ranks than z planes
    with pytest.raises(A.PsatdError):
        A.psatd_plan_distribute(pl.handle, 2, 2)             # no such rank
    A.psatd_plan_distribute(pl.handle, 3, 2)
    assert A.psatd_dist_bounds(pl.handle) == (7, 10, 8, 12)  # 10 planes: 4 + 3 + 3; 12 rows: 4 each
    with pytest.raises(A.PsatdError):
        A.psatd_plan_distribute(pl.handle, 3, 1)             # already distributed
    pl.close()
    lay2 = I.local_layout((32, 16, 16), (2, 1, 1), 4, 8)
    pl2 = Plan(lay2, (1.0, 1.0, 1.0), 0.5, precision=64, sources="vacuum")
    with pytest.raises(A.PsatdError):
        A.psatd_plan_distribute(pl2.handle, 2, 0)            # two boxes
    pl2.close()


def _free_port():
    import socket
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _process_rank(rank, world, port, out_dir, n, p, h, dt, nsteps):
    """One process per rank: the device work on the GPU through DeviceRank,
    the two all-to-alls of GroupStep over gloo (host copies of the spectrum:
    every process shares the one GPU here, which NCCL does not allow)."""
    import os
    import torch
    import torch.distributed as dist
    from paper_1812_07357_gb300 import distributed as D
    from paper_1812_07357_gb300.solver import Plan
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), OMP_NUM_THREADS="1")
    dist.init_process_group("gloo", rank=rank, world_size=world)
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    plan = Plan(I.global_layout(n, p), h, dt, precision=64, sources="vacuum")
    rk = D.DeviceRank(plan, world, rank)
    step = D.GroupStep(n, world, rank,
                       lambda s: rk.xy_forward(s.to(dev)).cpu(),
                       lambda r, y0: rk.z_update(r.to(dev).contiguous(), y0).cpu(),
                       lambda sp: rk.yx_inverse(sp.to(dev)).cpu())
    full = _inputs(n, "vacuum", 5)
    slab = D.split_components({k: torch.from_numpy(v) for k, v in full.items()}, COMPS, step.t)
    for _ in range(nsteps):
        slab = step(slab)
    np.save(os.path.join(out_dir, f"r{rank}.npy"), slab.numpy())
    np.save(os.path.join(out_dir, f"z{rank}.npy"), np.array(step.t.z_slab + (step.t.transpositions,)))
    plan.close()
    dist.destroy_process_group()


@pytest.mark.gpu
def test_group_step_over_processes_with_device_ranks(tmp_path):
    """GroupStep (the partition and the gloo all-to-alls) driving DeviceRank in
    two processes sharing the GPU, against the oracle's single-box push."""
    import torch.multiprocessing as mp
    world, n, p, h, dt, nsteps = 2, (16, 12, 10), 8, (1.0, 0.9, 1.1), 0.7, 3
    mp.start_processes(_process_rank, args=(world, _free_port(), str(tmp_path), n, p, h, dt, nsteps),
                       nprocs=world, join=True, start_method="spawn")
    n0, n1, n2 = n
    got = np.zeros((6, n2, n1, n0))
    for r in range(world):
        z0, z1, moves = np.load(tmp_path / f"z{r}.npy")
        assert moves == 2 * nsteps
        got[:, z0:z1] = np.load(tmp_path / f"r{r}.npy")
    full = _inputs(n, "vacuum", 5)
    lay = I.global_layout(n, p)
    ref = O.push(lay, {k: [full[k]] for k in COMPS}, {}, nsteps, h, dt)
    assert_fields(lay, {k: [got[i]] for i, k in enumerate(COMPS)}, {k: [ref[k][0]] for k in COMPS}, COMPS,
                  prec=64, what="2 processes")
