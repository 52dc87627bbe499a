"""Multi-GPU host logic on CPU: world-size-2 gloo ranks (replicas only, no
data-path collective; the only collective is the timing MAX)."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_2410_05095_b300.replicas import row_bands


@pytest.mark.parametrize("H,world", [(1080, 2), (1080, 8), (7, 3), (1, 1), (5, 8)])
def test_row_bands_partition(H, world):
    bands = row_bands(H, world)
    assert len(bands) == world
    rows = [r for a, b in bands for r in range(a, b)]
    assert rows == list(range(H))
    sizes = [b - a for a, b in bands]
    assert max(sizes) - min(sizes) <= 1


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    from paper_2410_05095_b300.replicas import job_ms_per_frame, max_over_ranks
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local = 100.0 + 50.0 * rank          # rank 1 is the slow one
        m = max_over_ranks(local)
        v = job_ms_per_frame(local, frames_per_rank=10)
        q.put((rank, m, v))
    finally:
        dist.destroy_process_group()


def test_gloo_two_ranks_max_timing():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, m, v in res:
        assert m == 150.0                     # max over ranks
        assert v == pytest.approx(150.0 / 20)  # slowest rank's time over all 20 frames
