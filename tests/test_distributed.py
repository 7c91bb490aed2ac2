"""The block-row distribution of Section 7 on CPU: the oracle's sketches of
the blocks of a row partition (global row indices) add up to the sketch of the
whole matrix, and `ms_sketch_distributed`'s host logic (partition, local
sketch, one sum all-reduce) returns the whole matrix's multisketch on every
rank — two and three gloo ranks, the local sketch supplied by the oracle."""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
D, N, K, P, SEED = 5003, 6, 72, 24, 0x5EED0011


def _problem():
    A = inputs.integer_matrix(D, N, 17, lo=-6, hi=6).numpy()
    b = inputs.integer_matrix(D, 1, 18, lo=-6, hi=6).numpy()[:, 0].copy()
    return A, b


@pytest.mark.parametrize("world", [1, 2, 3, 7])
def test_partition_blocks_add_up_to_the_whole_sketch(orc, world):
    from paper_2508_14209_gb300.distributed import row_partition

    A, b = _problem()
    parts = [row_partition(D, world, r) for r in range(world)]
    assert parts[0][0] == 0 and sum(m for _, m in parts) == D
    assert all(parts[r][0] + parts[r][1] == parts[r + 1][0] for r in range(world - 1))
    Y = sum(orc.countsketch_rows(A[r0:r0 + m], K, SEED, r0, b=b[r0:r0 + m]) for r0, m in parts)
    assert np.array_equal(Y, orc.countsketch(A, K, SEED, b=b))


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist

    import oracle as orc
    from paper_2508_14209_gb300.distributed import ms_sketch_distributed, row_partition

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        A, b = _problem()
        r0, m = row_partition(D, world, rank)
        G = orc.gaussian(SEED, P, K).astype(np.float64)

        def local(Ab, bb, row0):
            return torch.from_numpy(orc.gemm(G, orc.countsketch_rows(Ab, K, SEED, row0, b=bb)))

        Z = ms_sketch_distributed(A[r0:r0 + m], r0, K, P, SEED, b_local=b[r0:r0 + m], local_sketch=local)
        q.put((rank, Z.numpy()))
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("world", [2, 3])
def test_distributed_multisketch_equals_whole_matrix_on_every_rank(orc, world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in ps:
        p.start()
    out = sorted((q.get(timeout=120) for _ in ps), key=lambda t: t[0])
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    A, b = _problem()
    Zo, Gu, Yu = orc.multisketch(A, K, P, SEED, b=b, gemm_prec="f64")
    # integer A: every block sketch is exact; each rank's G Y_r is compensated,
    # and the all-reduce adds world - 1 roundings
    bound = 4 * world * np.finfo(np.float64).eps * (np.abs(Gu) @ np.abs(Yu))
    for _, Z in out:
        assert np.all(np.abs(Z - Zo) <= bound)
        assert np.array_equal(Z, out[0][1])
