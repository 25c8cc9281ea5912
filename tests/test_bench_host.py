"""Host-side logic of bench.py on the CPU: the algorithmic byte counts, and
the multi-rank path (replicas, max over ranks, weak-scaling unit count)
with world_size-2 gloo process groups; the reference arm under torchrun
prints one line from rank 0 only."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_step_bytes_of_the_512_local_workload():
    # 452,984,832 padded cells x 48 B + 318,767,104 guard cells x 24 B
    lay = bench.build_layout("local_512")
    assert lay.cells == 452_984_832
    assert lay.guard_cells == 318_767_104
    assert bench.step_algorithmic_bytes(lay) == 29_393_682_432


def test_kernel_bytes_fast_path():
    lay = bench.build_layout("local_128")
    b = lay.boxes[0]
    hx = b.n[0] // 2 + 1
    nb = len(lay.boxes)
    kb = bench.kernel_bytes(lay, fused=True)["fast"]
    assert kb[0] == 6 * nb * (b.cells * 4 + hx * b.n[1] * b.n[2] * 8)
    assert kb[2] == 6 * nb * hx * b.n[1] * (b.n[2] + b.interior[2]) * 8
    assert kb[4] == 6 * nb * (hx * b.n[1] * b.interior[2] * 8 + b.interior_cells * 4) + 6 * lay.guard_cells * 4
    assert kb[1] == kb[3] == 0
    # without the fused exchange the inverse kernel writes no guard cells
    assert bench.kernel_bytes(lay, fused=False)["fast"][4] == kb[4] - 6 * lay.guard_cells * 4
    # deferred exchange timed over a 20-step push: one guard-storing launch in 20
    kd = bench.kernel_bytes(lay, fused=True, guard_frac=1 / 20)["fast"]
    assert kd[4] == pytest.approx(kb[4] - 6 * lay.guard_cells * 4 * 19 / 20)
    assert kd[0] == kb[0] and kd[2] == kb[2]     # the forward pass reads every padded cell either way


def test_inverse_bytes_of_a_middle_step_at_full_size():
    # 6 x (8 x 49 x 96 x 64 x 512 spectrum in + 4 x 512^3 interior out)
    lay = bench.build_layout("local_512")
    assert bench.kernel_bytes(lay, guard_frac=0.0)["fast"][4] == 10_619_977_728


def _rank_main(rank, world, port, out_dir):
    os.environ.update(RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(world),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    r, _, w = bench.dist_init("gloo")
    assert (r, w) == (rank, world)
    bench.barrier()
    mx = bench.reduce_max(10.0 + rank)
    units = bench.total_units(1000.0, w)
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as fh:
        json.dump({"max": mx, "units": units}, fh)
    dist.destroy_process_group()


def test_two_rank_gloo_reduce_max_and_units(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    for r in range(2):
        d = json.load(open(tmp_path / f"r{r}.json"))
        assert d == {"max": 11.0, "units": 2000.0}


def test_reference_arm_under_torchrun_prints_once():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "3", "--workload", "local_128"]
    env = dict(os.environ, PSATD_ORACLE_THREADS="2", OMP_NUM_THREADS="1")
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2
    assert d["cpu_baseline"]["kind"] == "oracle" and d["value"] > 0
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
