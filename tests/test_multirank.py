"""The N > 1 path of bench.py on CPU: two gloo ranks, each with its own stream
(weak scaling, no data-path collective); the job's time is the slowest
rank's and its units are every rank's entries, reduced on the host."""
import json
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank,
                            world_size=world)
    try:
        ms = [120.0, 95.5][rank]            # the ranks' own timings
        nnz = [1_000_003, 999_871][rank]    # seed = rank: streams differ in length
        ms_job = bench.over_ranks(ms, world, "max")
        nnz_job = int(bench.over_ranks(nnz, world, "sum"))
        rate = bench.whole_job_rate(nnz_job, 3, ms_job)
        with open(os.path.join(out_dir, "rank%d.json" % rank), "w") as f:
            json.dump({"ms": ms_job, "nnz": nnz_job, "rate": rate}, f)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_time_and_units(tmp_path):
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    res = [json.load(open(tmp_path / ("rank%d.json" % r))) for r in range(world)]
    for r in res:   # every rank agrees
        assert r["ms"] == 120.0
        assert r["nnz"] == 1_000_003 + 999_871
        assert r["rate"] == pytest.approx((1_000_003 + 999_871) * 3 / 0.120)


def test_single_rank_is_identity():
    assert bench.over_ranks(7.5, 1, "max") == 7.5
    assert bench.over_ranks(11, 1, "sum") == 11
    assert bench.whole_job_rate(1000, 2, 500.0) == pytest.approx(4000.0)
