"""The multi-process path of bench.py on CPU: two gloo ranks check the
max-over-ranks timing, the whole-job value (all ranks' pixels over the
slowest rank's time, weak scaling), distinct per-rank images, that the
reference arm runs on rank 0 alone, and that the row bands of the strong-
scaling split cover an image's output rows exactly once."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, results):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = [0.25, 0.40][rank]
        mx = bench.reduce_max(ms, world, "cpu")
        value = bench.whole_job_value(world, bench.H * bench.W, mx)

        class A:
            steps, warmup = 1, 0
        ref = bench.run_reference(A(), rank, world) if rank != 0 else "skipped"
        # rows split: the bands of all ranks cover the VALID rows exactly once
        bands = [None] * world
        dist.all_gather_object(bands, bench.row_band(8188, world, rank))
        results[rank] = (mx, value, bench.rank_image_seed(rank), ref, bands)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    port = _free_port()
    with mp.get_context("spawn").Manager() as mgr:  # no fork of a threaded process
        results = mgr.dict()
        mp.spawn(_worker, args=(2, port, results), nprocs=2, join=True)
        r = dict(results)
    assert r[0][0] == r[1][0] == 0.40  # every rank sees the slowest rank's time
    expect = 2 * 8192 * 8192 / 0.40e-3 / 1e6
    assert r[0][1] == pytest.approx(expect) and r[1][1] == pytest.approx(expect)
    assert r[0][2] != r[1][2]  # each rank has its own image
    assert r[1][3] is None  # the reference arm does no work on rank 1
    bands = r[0][4]
    assert bands == r[1][4] and bands[0][0] == 0 and bands[-1][1] == 8188
    assert all(a[1] == b[0] and a[0] < a[1] for a, b in zip(bands, bands[1:] + [(8188, 8189)]))


@pytest.mark.parametrize("world", [1, 2, 3, 7, 8])
def test_row_bands_partition(world):
    import bench
    for hv in (1, 7, 8188, 8189):
        bands = [bench.row_band(hv, world, r) for r in range(world)]
        assert bands[0][0] == 0 and bands[-1][1] == hv
        assert all(a[1] == b[0] for a, b in zip(bands, bands[1:]))
        sizes = [b - a for a, b in bands]
        assert max(sizes) - min(sizes) <= 1
