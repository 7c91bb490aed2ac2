"""The N > 1 host logic of bench.py on CPU: two gloo ranks, each timing its
own replica, agree on the slowest rank's time and on the whole-job value
(bytes of all ranks over that time).  Every box has one GPU, so the path runs
as independent replicas; this is the only cross-rank step."""
import os
import socket
import sys

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ws, r, local = bench._dist()
        ms = [3.0, 5.0, 4.0][rank]
        mx = bench.max_over_ranks(ms)
        q.put((r, ws, local, mx, bench.whole_job_gbs(1e9, ws, mx)))
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _run(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in ps:
        p.start()
    out = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    return out


def test_two_ranks_agree_on_slowest_time_and_whole_job_value():
    out = _run(2)
    assert [o[0] for o in out] == [0, 1] and all(o[1] == 2 and o[2] == o[0] for o in out)
    assert all(o[3] == 5.0 for o in out)
    assert all(abs(o[4] - 2 * 1e9 / 5e-3 / 1e9) < 1e-9 for o in out)


def test_single_process_is_identity():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(7.5) == 7.5
    assert bench.whole_job_gbs(2e9, 1, 1.0) == 2000.0
