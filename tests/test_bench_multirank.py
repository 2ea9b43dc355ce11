"""The N > 1 host path of bench.py on CPU (gloo, world size 2): the max over
ranks of the timed region, the split of the 64-image batch into disjoint
pixel-balanced shares and the gathering of the shares' figures, and the
reference arm under torchrun (rank 0 alone runs and prints one JSON line; the
other rank exits 0 without work)."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
torch = pytest.importorskip("torch")


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        got = bench.reduce_max(1.5 + rank, world, "cpu")
        g = bench.gather_shards((100.0 + 50.0 * rank, 30 + rank, 1e9 * (rank + 1)), world, "cpu")
        with open(os.path.join(out_dir, f"r{rank}.txt"), "w") as f:
            f.write(repr(got))
        with open(os.path.join(out_dir, f"g{rank}.json"), "w") as f:
            f.write(json.dumps(g))
    finally:
        dist.destroy_process_group()


def test_reduce_max_over_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp

    mp.start_processes(_worker, args=(2, free_port(), str(tmp_path)), nprocs=2, start_method="spawn")
    vals = [float(open(tmp_path / f"r{r}.txt").read()) for r in range(2)]
    assert vals == [2.5, 2.5]
    for r in range(2):  # every rank sees the whole batch: slowest time, summed images and work
        g = json.loads(open(tmp_path / f"g{r}.json").read())
        assert g["ms"] == 150.0 and g["images"] == 61
        assert abs(g["images_per_s"] - 61 / 0.15) < 1e-9 and abs(g["value"] - 3e3 / 0.15) < 1e-6


@pytest.mark.parametrize("world", [1, 2, 3, 4, 8])
def test_batch_shards_are_disjoint_and_pixel_balanced(world):
    sys.path.insert(0, ROOT)
    import bench
    from paper_2506_08793_gb300 import scenes

    sizes = scenes.batch_sizes(3000, 64)
    parts = bench.shard(sizes, world)
    assert len(parts) == world
    flat = sorted(k for p in parts for k in p)
    assert flat == list(range(64))  # disjoint, and together the whole batch
    loads = [sum(sizes[k][0] * sizes[k][1] for k in p) for p in parts]
    biggest = max(H * W for H, W in sizes)
    assert max(loads) - min(loads) <= biggest
    assert parts == bench.shard(sizes, world)  # deterministic


def test_reduce_max_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.reduce_max(3.25, 1, "cpu") == 3.25


def test_reference_arm_under_torchrun_two_ranks():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(free_port()), "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "3", "--ref-iters", "1"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"
