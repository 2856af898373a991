"""The N > 1 path on CPU: world size 2 over gloo.

Under torchrun every rank solves its own seeded video (independent problems,
weak scaling); the only collectives are the two host-side reductions that
turn per-rank timings into the job's figure: the maximum of the per-rank
times and the sum of the per-rank work units.  These tests run exactly those
reductions (`bench.max_over_ranks`, `bench.sum_over_ranks`) on two gloo
ranks, check that the ranks draw different inputs, and that a sharded run of
the oracle gives each rank the same iterate as a lone run of its video.
"""
import json
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                      RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        import oracle
        from paper_1907_02731_gb300 import inputs
        res = {}
        # per-rank timings: (total ms, e2e ms, step ms)
        times = [1.0 + rank, 10.0 - rank, 3.0 + 0.5 * rank]
        res["max"] = bench.max_over_ranks(times, world)
        res["units"] = bench.sum_over_ranks(1000 * (rank + 1), world)
        # each rank's own video: small shape, seed from the rank
        wl = inputs.WORKLOADS["small_16x64x64"]
        seed = inputs.config_seed(wl.config, bench.rank_video_index(rank))
        f, _ = inputs.make_video(4, 16, 16, seed, 1)
        f = f.astype(np.float64)
        sp = oracle.unary(f, wl.p)
        r = oracle.power_iterate(sp, f, f, 5, (1, 2, 2), (1.5, 2.0, 2.0), 1.0)
        x = torch.from_numpy(np.ascontiguousarray(r["x"]))
        gathered = [torch.empty_like(x) for _ in range(world)]
        dist.all_gather(gathered, x)                 # test-side only: collect the shards
        if rank == 0:
            np.save(os.path.join(out_dir, "x_all.npy"), torch.stack(gathered).numpy())
        with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as fh:
            json.dump(res, fh)
        # the reference arm does its work on rank 0 only
        if rank != 0:
            class A:
                warmup, steps, gpus = 1, 1, world
            assert bench.run_reference(A, wl) is None
    finally:
        dist.destroy_process_group()


@pytest.fixture(scope="module")
def two_rank_run(tmp_path_factory):
    out = tmp_path_factory.mktemp("ranks")
    mp.start_processes(_worker, args=(2, _free_port(), str(out)), nprocs=2, join=True,
                       start_method="spawn")
    return out


def test_max_over_ranks(two_rank_run):
    for rank in range(2):
        with open(two_rank_run / f"rank{rank}.json") as fh:
            res = json.load(fh)
        assert res["max"] == [2.0, 10.0, 3.5]          # every rank sees the slowest
        assert res["units"] == 3000.0                  # 1000 + 2000


def test_ranks_solve_their_own_videos(two_rank_run):
    import oracle
    from paper_1907_02731_gb300 import inputs
    import bench
    x_all = np.load(two_rank_run / "x_all.npy")
    wl = inputs.WORKLOADS["small_16x64x64"]
    assert not np.allclose(x_all[0], x_all[1])
    for rank in range(2):
        f, _ = inputs.make_video(4, 16, 16, inputs.config_seed(wl.config, bench.rank_video_index(rank)), 1)
        f = f.astype(np.float64)
        r = oracle.power_iterate(oracle.unary(f, wl.p), f, f, 5, (1, 2, 2), (1.5, 2.0, 2.0), 1.0)
        np.testing.assert_array_equal(x_all[rank], r["x"])


def test_single_rank_reductions_are_identity():
    import bench
    assert bench.max_over_ranks([4.0, 5.0], 1) == [4.0, 5.0]
    assert bench.sum_over_ranks(7, 1) == 7.0
