"""A hybrid group distributed over gloo ranks on the CPU (paper Sec. 2.4.1
distributed FFT, Sec. 2.6 spectrum kept in the transposed layout): the slab
partition, the two transpositions (bit for bit), and whole steps against the
oracle's single-box push of the group.  The per-rank transforms and the
update are test-side stand-ins (torch FFTs and the oracle's per-mode update)
for the device work; what is under test is the partition and the data
movement of paper_1812_07357_gb300.distributed."""
import json
import os
import socket

import numpy as np
import pytest

from paper_1812_07357_gb300 import distributed as D


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_slab_bounds_cover_and_balance():
    for n, parts in [(8, 2), (10, 3), (96, 7), (5, 5)]:
        b = D.slab_bounds(n, parts)
        assert b[0][0] == 0 and b[-1][1] == n
        assert all(b[i][1] == b[i + 1][0] for i in range(parts - 1))
        sizes = [hi - lo for lo, hi in b]
        assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        D.slab_bounds(3, 4)


def _code(z, y, x):
    return z * 10000.0 + y * 100.0 + x


def _rank_transpose(rank, world, port, out_dir, n):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t = D.SlabTranspose(n, world, rank)
    n0, n1, n2 = n
    hx = n0 // 2 + 1
    z0, z1 = t.z_slab
    z, y, x = torch.meshgrid(torch.arange(z0, z1), torch.arange(n1), torch.arange(hx), indexing="ij")
    spec = torch.complex(_code(z, y, x).double(), -_code(z, y, x).double())
    spec = torch.stack([spec, 2 * spec])                  # two components in one exchange
    rows = t.forward(spec)
    y0, y1 = t.y_rows
    z, y, x = torch.meshgrid(torch.arange(n2), torch.arange(y0, y1), torch.arange(hx), indexing="ij")
    want = torch.complex(_code(z, y, x).double(), -_code(z, y, x).double())
    ok_fwd = bool(torch.equal(rows[0], want) and torch.equal(rows[1], 2 * want))
    back = t.inverse(rows)
    ok_inv = bool(torch.equal(back, spec))
    with open(os.path.join(out_dir, f"t{rank}.json"), "w") as fh:
        json.dump({"fwd": ok_fwd, "inv": ok_inv, "count": t.transpositions}, fh)
    dist.destroy_process_group()


@pytest.mark.parametrize("world,n", [(2, (12, 10, 8)), (3, (16, 10, 8))])
def test_transpositions_move_every_mode_to_its_owner(tmp_path, world, n):
    import torch.multiprocessing as mp
    mp.start_processes(_rank_transpose, args=(world, _free_port(), str(tmp_path), n), nprocs=world, join=True,
                       start_method="spawn")
    for r in range(world):
        d = json.load(open(tmp_path / f"t{r}.json"))
        assert d == {"fwd": True, "inv": True, "count": 2}, (r, d)


# ---------------------------------------------------------------------------
# whole steps of a distributed group against the oracle
# ---------------------------------------------------------------------------

COMPS = ("Ex", "Ey", "Ez", "Bx", "By", "Bz")


def _stand_ins(n, h, p, dt):
    """Per-rank transforms (torch FFTs) and the update (the oracle's per-mode
    update on centred spectra with the global wavenumbers)."""
    import torch
    from oracle import psatd_oracle as O
    n0, n1, n2 = n
    hx = n0 // 2 + 1
    kx = O.axis_wavenumbers(n0, h[0])[:hx]
    ky_all = O.axis_wavenumbers(n1, h[1])
    kz = O.axis_wavenumbers(n2, h[2])

    def xy_forward(slab):
        return torch.fft.rfft2(slab, dim=(-2, -1))

    def z_update(rows, y_lo):
        spec = torch.fft.fft(rows, dim=-3).numpy()
        ny = spec.shape[-2]
        ky = ky_all[y_lo:y_lo + ny]
        KX = O.modified_wavenumber(kx, h[0], p)[None, None, :]
        KY = O.modified_wavenumber(ky, h[1], p)[None, :, None]
        KZ = O.modified_wavenumber(kz, h[2], p)[:, None, None]
        k = (kx[None, None, :], ky[None, :, None], kz[:, None, None])
        ph = {c: np.exp(-1j * sum(k[d] * O.YEE[c][d] * h[d] for d in range(3))) for c in COMPS}
        cen = [spec[i] * ph[c] for i, c in enumerate(COMPS)]
        En, Bn, _ = O.update_modes(tuple(cen[:3]), tuple(cen[3:]), None, None, (KX, KY, KZ), dt)
        out = np.stack([v / ph[c] for v, c in zip(list(En) + list(Bn), COMPS)])
        return torch.fft.ifft(torch.from_numpy(out), dim=-3)

    def yx_inverse(spec):
        return torch.fft.irfft2(spec, s=(n1, n0), dim=(-2, -1))

    return xy_forward, z_update, yx_inverse


def _rank_steps(rank, world, port, out_dir, n, p, nsteps):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), OMP_NUM_THREADS="1")
    dist.init_process_group("gloo", rank=rank, world_size=world)
    h, dt = (1.0, 0.9, 1.1), 0.7
    rng = np.random.default_rng(71)
    n0, n1, n2 = n
    full = {k: torch.from_numpy(rng.standard_normal((n2, n1, n0))) for k in COMPS}   # same on every rank
    step = D.GroupStep(n, world, rank, *_stand_ins(n, h, p, dt))
    slab = D.split_components(full, COMPS, step.t)
    for _ in range(nsteps):
        slab = step(slab)
    np.save(os.path.join(out_dir, f"s{rank}.npy"), slab.numpy())
    with open(os.path.join(out_dir, f"s{rank}.json"), "w") as fh:
        json.dump({"z": list(step.t.z_slab), "transpositions": step.t.transpositions}, fh)
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_distributed_group_steps_match_the_oracle(tmp_path, world):
    import torch.multiprocessing as mp
    from oracle import psatd_oracle as O
    from paper_1812_07357_gb300 import inputs as I
    n, p, nsteps = (12, 10, 9), 8, 3
    mp.start_processes(_rank_steps, args=(world, _free_port(), str(tmp_path), n, p, nsteps), nprocs=world,
                       join=True, start_method="spawn")
    n0, n1, n2 = n
    got = np.zeros((6, n2, n1, n0))
    for r in range(world):
        meta = json.load(open(tmp_path / f"s{r}.json"))
        assert meta["transpositions"] == 2 * nsteps      # two per step: the last one is skipped
        z0, z1 = meta["z"]
        got[:, z0:z1] = np.load(tmp_path / f"s{r}.npy")
    rng = np.random.default_rng(71)
    f0 = {k: [rng.standard_normal((n2, n1, n0))] for k in COMPS}
    lay = I.global_layout(n, p)
    ref = O.push(lay, f0, {}, nsteps, (1.0, 0.9, 1.1), 0.7)
    for i, k in enumerate(COMPS):
        r = ref[k][0]
        assert np.abs(got[i] - r).max() <= 1e-12 * np.abs(r).max(), k
