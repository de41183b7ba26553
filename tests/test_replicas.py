"""The multi-GPU (replica) path's host logic on CPU processes with gloo,
world size 2: ranks sort their own units, the job's time is the slowest
rank's, and its throughput counts every rank's units."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2605_14419_gb300 import replicas  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank: int, world: int, port: int, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, lr = replicas.world_info()
        # each rank times its own work; the job waits for the slowest
        slowest = replicas.max_over_ranks(1.0 + rank)
        rate = replicas.job_rate(100 * (rank + 1), 2.0 + rank)  # 300 units over 3 s
        lo, hi = replicas.shard_range(20_000, r, w)
        out.put((r, w, lr, slowest, rate, lo, hi, replicas.rank_seed(5, r)))
    finally:
        dist.destroy_process_group()


def test_gloo_world_size_two():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, w0, l0, s0, rate0, lo0, hi0, seed0), (r1, w1, l1, s1, rate1, lo1, hi1, seed1) = res
    assert (r0, r1, w0, w1, l0, l1) == (0, 1, 2, 2, 0, 1)
    assert s0 == s1 == 2.0  # the slowest rank's time, on every rank
    assert rate0 == rate1 == pytest.approx(100.0)  # (100 + 200) units / 3 s
    assert (lo0, hi0, lo1, hi1) == (0, 10_000, 10_000, 20_000)
    assert seed0 != seed1


def test_shard_range_covers_every_unit_once():
    for n in (0, 1, 7, 20_000, 20_001):
        for world in (1, 2, 3, 8):
            spans = [replicas.shard_range(n, r, world) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(spans, spans[1:]))
            assert max(h - l for l, h in spans) - min(h - l for l, h in spans) <= 1
    with pytest.raises(ValueError):
        replicas.shard_range(10, 2, 2)


def test_single_process_needs_no_group():
    assert replicas.max_over_ranks(3.5) == 3.5
    assert replicas.job_rate(10, 2.0) == 5.0
