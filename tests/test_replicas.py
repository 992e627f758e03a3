"""The replicas-only multi-GPU mode's host logic with two gloo ranks on the CPU: rank
environment, barrier, max-over-ranks timing, whole-job throughput and per-rank problems."""
import json
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist
    from paper_2402_12947_gb300 import inputs, replicas
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, local = replicas.dist_env()
        replicas.barrier(cuda=False)
        # a rank's "timings": the job's time is the slowest rank's
        ms = replicas.max_over_ranks([10.0 + rank, 5.0 - rank])
        value = replicas.job_throughput(1000.0, w, ms[0])
        m = inputs.config_c1(seed=replicas.mesh_seed(1, r))[0]
        b = inputs.uniform_rhs(16, replicas.rhs_seed(2, r))
        replicas.barrier(cuda=False)
        with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
            json.dump({"env": [r, w, local], "ms": ms, "value": value, "coords_sum": float(m.coords.sum()),
                       "b0": float(b[0])}, f)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp
    world, port = 2, _free_port()
    mp.start_processes(_worker, args=(world, port, str(tmp_path)), nprocs=world, join=True, start_method="spawn")
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]
    for r, d in enumerate(res):
        assert d["env"] == [r, world, r]
        assert d["ms"] == [11.0, 5.0]                       # element-wise max over both ranks
        assert d["value"] == pytest.approx(1000.0 * world / 11.0e-3)
    # independent problems: different meshes and right-hand sides per rank
    assert res[0]["coords_sum"] != res[1]["coords_sum"]
    assert res[0]["b0"] != res[1]["b0"]


def test_single_process_defaults(monkeypatch):
    from paper_2402_12947_gb300 import replicas
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert replicas.dist_env() == (0, 1, 0)
    assert replicas.max_over_ranks([3.0, 1.0]) == [3.0, 1.0]
    assert replicas.job_throughput(50.0, 1, 10.0) == pytest.approx(5000.0)
    assert replicas.mesh_seed(2, 0) == 2 and replicas.mesh_seed(2, 3) == 3002
