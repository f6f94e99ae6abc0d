"""The N > 1 path of bench.py on CPU: two gloo ranks run the bench's own partition and timing
reduction.  Points are independent, so the path shards with no data-path collective: ranks
must solve disjoint points that together are consecutive blocks of the (k, E) grid, every rank
must end with the slowest rank's time, and the rate counts the points of all ranks."""
import json
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402

P, STEPS, WORLD = 48, 5, 2


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, outdir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        pts = [np.stack(bench.rank_points(s, rank, world, P), axis=1).tolist()
               for s in range(STEPS)]
        ms = 100.0 + 37.5 * rank          # the ranks' own timings differ
        m = bench.max_over_ranks(ms, dist, "cpu")
        rate = bench.aggregate_rate(STEPS, P, world, m)
        with open(os.path.join(outdir, f"rank{rank}.json"), "w") as f:
            json.dump(dict(points=pts, ms=m, rate=rate), f)
    finally:
        dist.destroy_process_group()


@pytest.fixture(scope="module")
def ranks(tmp_path_factory):
    out = tmp_path_factory.mktemp("ranks")
    mp.start_processes(_rank, args=(WORLD, _free_port(), str(out)), nprocs=WORLD,
                       start_method="spawn", join=True)
    res = []
    for r in range(WORLD):
        with open(out / f"rank{r}.json") as f:
            res.append(json.load(f))
    return res


def test_ranks_solve_disjoint_consecutive_points(ranks):
    n_E = bench.WORK["n_E"]
    for s in range(STEPS):
        flat = [k * n_E + e for res in ranks for k, e in res["points"][s]]
        # the step's points over all ranks are one consecutive block of WORLD * P grid points
        assert flat == list(range(s * WORLD * P, (s + 1) * WORLD * P))
        assert len(set(flat)) == WORLD * P


def test_every_rank_gets_the_slowest_time(ranks):
    slowest = 100.0 + 37.5 * (WORLD - 1)
    assert all(res["ms"] == slowest for res in ranks)


def test_rate_counts_all_ranks(ranks):
    expect = STEPS * P * WORLD / (100.0 + 37.5 * (WORLD - 1)) * 1e3
    assert all(abs(res["rate"] - expect) <= 1e-9 * expect for res in ranks)


def test_single_rank_needs_no_collective():
    assert bench.max_over_ranks(12.5, None, "cpu") == 12.5
    k, e = bench.rank_points(0, 0, 1, 4)
    assert (k.tolist(), e.tolist()) == ([0, 0, 0, 0], [0, 1, 2, 3])
