"""Multi-rank host logic on CPU (gloo, world size 2): row shards cover the
database exactly and their answers concatenate to the full answer; the
max-over-ranks timing and the whole-job rate follow the slowest rank."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_2510_03631_gb300 import inputs, replicas


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, R, C, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        D = inputs.db_digits(R, C, 256, seed=3)
        q = inputs.uniform_u32(C, seed=4, tag=inputs.TAG_MISC)
        r0, r1 = replicas.shard_rows(R, world, rank)
        part = torch.from_numpy(oracle.answer(np.ascontiguousarray(D[r0:r1]), q).view(np.int32))
        full = replicas.gather_row_shards(part, dist)
        # each rank reports a different step time; every rank must see the largest
        slowest = replicas.max_over_ranks(1.0 + rank, dist)
        rate = replicas.job_rate(R * C, world, slowest * 1e-3)
        if rank == 0:
            np.save(os.path.join(out_dir, "full.npy"), full.numpy().view(np.uint32))
            np.save(os.path.join(out_dir, "timing.npy"), np.array([slowest, rate]))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("R", [1000, 300, 129])
def test_row_shards_concatenate_to_the_full_answer(tmp_path, R):
    world, C = 2, 96
    mp.start_processes(_worker, args=(world, _free_port(), R, C, str(tmp_path)), nprocs=world,
                       start_method="spawn", join=True)
    D = inputs.db_digits(R, C, 256, seed=3)
    q = inputs.uniform_u32(C, seed=4, tag=inputs.TAG_MISC)
    assert np.array_equal(np.load(tmp_path / "full.npy"), oracle.answer(D, q))
    slowest, rate = np.load(tmp_path / "timing.npy")
    assert slowest == 2.0
    assert rate == pytest.approx(R * C * world / 2e-3)


@pytest.mark.parametrize("rows,world", [(0, 1), (1, 1), (127, 2), (128, 2), (1000, 3), (32768, 8),
                                        (65536 + 5, 7), (300, 8)])
def test_shard_rows_partition(rows, world):
    spans = [replicas.shard_rows(rows, world, r) for r in range(world)]
    assert spans[0][0] == 0 and spans[-1][1] == rows
    for (a0, a1), (b0, b1) in zip(spans, spans[1:]):
        assert a1 == b0   # contiguous, in rank order
    for r0, r1 in spans:
        assert r0 <= r1
        assert r0 % 128 == 0   # whole 128-row tiles except where the database ends
    sizes = [r1 - r0 for r0, r1 in spans]
    if rows >= 128 * world:
        assert max(sizes) - min(sizes) <= 128


def test_shard_rows_rejects_bad_arguments():
    from paper_2510_03631_gb300 import pir
    for world, rank in ((0, 0), (2, 2)):
        with pytest.raises(pir.QpadlError):
            replicas.shard_rows(100, world, rank)


def test_job_rate_and_single_rank_max():
    assert replicas.max_over_ranks(3.5) == 3.5
    assert replicas.job_rate(10, 4, 2.0) == 20.0
    with pytest.raises(ValueError):
        replicas.job_rate(10, 4, 0.0)
