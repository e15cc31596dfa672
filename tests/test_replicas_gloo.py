"""The benchmark's multi-GPU path (replicas only: tiles are independent, so
each GPU encodes and decodes its own slide with no exchange) on CPU ranks:
two `gloo` processes check the rank seeds, the MAX-over-ranks timing and the
whole-job throughput that `bench.py --gpus N` reports, and the reference
arm's rule that ranks other than 0 do no work."""
import json
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir, ms_by_rank, steps, mp):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        ms = bench.max_over_ranks(ms_by_rank[rank], world, "cpu")
        ms_step, value = bench.replica_throughput(ms, steps, world, mp)
        with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
            json.dump({"ms": ms, "ms_step": ms_step, "value": value, "seed": bench.replica_seed(rank)}, f)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_replicas_report_the_slowest_rank(tmp_path):
    import torch.multiprocessing as mp
    world, steps, mp_per_replica = 2, 4, 1200.0
    ms_by_rank = [31.5, 47.25]   # rank 1 is the slow one
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path), ms_by_rank, steps, mp_per_replica),
             nprocs=world, join=True)
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]
    for r in res:
        # every rank sees the slowest rank's time, and the job's pixels over it
        assert r["ms"] == max(ms_by_rank)
        assert r["ms_step"] == pytest.approx(max(ms_by_rank) / steps)
        assert r["value"] == pytest.approx(world * mp_per_replica / (max(ms_by_rank) / steps / 1e3))
    # weak scaling: each replica has its own slide
    assert res[0]["seed"] != res[1]["seed"]


def test_replica_seeds_give_different_slides():
    sys.path.insert(0, ROOT)
    import bench
    from paper_2005_08713_gb300 import synth
    a = synth.slide(bench.replica_seed(0), 0, 0, 64, 64)
    b = synth.slide(bench.replica_seed(1), 0, 0, 64, 64)
    assert a.shape == b.shape == (64, 64, 3)
    assert not np.array_equal(a, b)
    # rank 0's replica is the single-GPU workload
    assert bench.replica_seed(0) == synth.config_seed(3)


def test_one_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(12.5, 1, "cpu") == 12.5
    ms_step, value = bench.replica_throughput(50.0, 5, 1, 1200.0)
    assert ms_step == 10.0 and value == pytest.approx(120000.0)


def test_reference_arm_runs_on_rank_0_only(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    # rank 1 returns before touching the oracle or the generator: args are never read
    assert bench.run_reference(None) is None
