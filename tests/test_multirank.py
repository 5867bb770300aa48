"""Multi-rank host logic of bench.py on CPU (gloo, world size 2): every rank
renders its own frame of the camera orbit (weak scaling, no data-path
collective) and the job time is the maximum over ranks."""
import os
import socket


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    scenes, desc = bench.workload("bulb_1080p", rank)
    eye = scenes[0]["camera"]["eye"]
    t = bench.max_over_ranks(torch, dist, 1.0 + rank, "cpu")
    batch, _ = bench.workload("batch_mixed", rank)
    dist.barrier()
    q.put((rank, eye, t, desc, len(batch), batch[0]["camera"]["width"]))
    dist.destroy_process_group()


def test_two_ranks_gloo():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, eye0, t0, d0, n0, w0), (r1, eye1, t1, d1, n1, w1) = got
    assert eye0 != eye1 and "frame 10" in d0 and "frame 11" in d1  # own frame per rank
    assert t0 == t1 == 2.0  # max over ranks
    assert n0 == n1 == 64 and (w0, w1) != (None, None)


def test_single_rank_needs_no_process_group():
    import torch

    import bench

    assert bench.max_over_ranks(torch, None, 3.5, "cpu") == 3.5
