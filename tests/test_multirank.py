"""The benchmark's multi-rank path on CPU: two gloo ranks (one process each)
run the same setup code as `bench.py --gpus 2` under torchrun, without a GPU.

Environments are independent, so N ranks are N replicas of the per-GPU
workload with no data-path collective; what needs checking is the host side:
rank setup from the launcher's environment, the maximum of the ranks' times,
and that the ranks' environments together are exactly the first N x E
environments of one large batch.
"""
import os
import socket

import numpy as np

from paper_2605_01352_b300 import scene as S


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, envs, q):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(ws), "LOCAL_RANK": str(rank), "CUDA_VISIBLE_DEVICES": ""})
    import torch.distributed as dist

    import bench
    from paper_2605_01352_b300 import scene as Sc
    got_ws, got_rank, _ = bench.dist_setup()
    # each rank reports its own time; the job's time is the slowest rank's
    t_max = bench.allreduce_max(got_ws, 0.25 * (rank + 1))
    sc = bench.rank_scene(Sc, got_rank, envs)
    bench.barrier(got_ws)
    q.put((got_rank, got_ws, dist.get_backend(), t_max, sc.pos.copy(), sc.shape_dims.copy(), sc.body_off.copy()))
    dist.destroy_process_group()


def test_two_gloo_ranks_replicate_the_benchmark_workload():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    ws, envs = 2, 3
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, ws, port, envs, q)) for r in range(ws)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(ws))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[0] for o in out] == [0, 1] and all(o[1] == ws for o in out)
    assert all(o[2] == "gloo" for o in out)
    assert all(o[3] == 0.5 for o in out)          # max over ranks of 0.25, 0.5
    # the two ranks' environments are environments 0..5 of one batch, in order
    whole = S.cfg2(ws * envs)
    pos = np.concatenate([o[4] for o in out], axis=1)
    dims = np.concatenate([o[5] for o in out], axis=1)
    np.testing.assert_array_equal(pos, whole.pos)
    np.testing.assert_array_equal(dims, whole.shape_dims)
    assert all(np.array_equal(o[6], whole.body_off[: envs + 1]) for o in out)


def test_job_throughput_counts_every_rank_over_the_slowest():
    import bench
    assert bench.job_throughput(4, 1024, 200, 0.1) == 4 * 1024 * 200 / 0.1
    assert bench.allreduce_max(1, 0.3) == 0.3
