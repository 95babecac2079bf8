"""The N > 1 path of bench.py on CPU: independent replicas over a world_size-2
gloo process group (no collective touches the data path; the timing takes the
slowest replica, the value counts every replica's work)."""
import json
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _replica(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # each replica times a different amount; the job takes the slowest
    t = bench.max_over_ranks(1.0 + rank, world, torch.device("cpu"))
    with open(os.path.join(out, f"{rank}.json"), "w") as f:
        json.dump([t, bench.job_value(100.0, world, t), list(bench.dist_env())], f)
    dist.destroy_process_group()


def test_max_over_ranks_and_job_value_on_two_gloo_ranks(tmp_path):
    port = _free_port()
    mp.spawn(_replica, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    for rank in (0, 1):
        with open(tmp_path / f"{rank}.json") as f:
            t, value, env = json.load(f)
        assert t == 2.0                  # the slowest replica's time, on every rank
        assert value == 2 * 100.0 / 2.0  # both replicas' work over that time
        assert env == [rank, 2, rank]


def test_single_process_needs_no_group():
    import bench
    assert bench.max_over_ranks(3.5, 1, None) == 3.5
    assert bench.job_value(10.0, 1, 2.0) == 5.0


def _reference_rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    args = bench.parse(["--impl", "reference", "--steps", "1", "--warmup", "0"])
    res = bench.run_reference(args) if rank != 0 else "skipped"
    with open(os.path.join(out, f"{rank}.json"), "w") as f:
        json.dump(res, f)


def test_reference_arm_runs_on_rank_zero_only(tmp_path):
    """Under torchrun the reference arm's other ranks exit without work."""
    port = _free_port()
    mp.spawn(_reference_rank, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    with open(tmp_path / "1.json") as f:
        assert json.load(f) is None
