"""The multi-rank path of bench.py on the CPU: two gloo ranks, as torchrun
would start them. Replicas only: each rank gets its own query pose of the same
scene, the step time is the slowest rank's, and the whole-job value counts
every rank's pixels; nothing else is exchanged."""
import os
import socket

import numpy as np
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import bench
    r, w, local = bench.dist_env()
    dist.init_process_group("gloo", rank=r, world_size=w)
    _, cam, T_ref, T_q = bench.make_workload(r)
    ms = 1.0 + 0.5 * r  # rank 1 is the slower one
    slow = bench.max_over_ranks(ms, w, device="cpu")
    bench.barrier(w)
    P = cam["height"] * cam["width"]
    out[r] = (r, w, local, slow, bench.job_mpix_per_s(w, P, slow), T_q.tolist(), T_ref.tolist())
    dist.destroy_process_group()


def test_two_gloo_ranks_replicas_only():
    world, port = 2, _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
        res = dict(out)
    assert sorted(res) == [0, 1]
    for r in (0, 1):
        rr, w, local, slow, value, Tq, Tref = res[r]
        assert (rr, w, local) == (r, 2, r)
        assert slow == 1.5  # both ranks see the slowest step time
        assert value == 2 * 1920 * 1080 / 1.5e-3 / 1e6
    # the same reference view, a different query pose per rank (independent units)
    np.testing.assert_array_equal(res[0][6], res[1][6])
    assert not np.allclose(res[0][5], res[1][5])
