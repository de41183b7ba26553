"""Sample sort across ranks (paper_2605_14419_gb300.distributed): the
exchange logic runs as two gloo ranks on CPU tensors, with the oracle's zSort
passed in as each rank's local sort (the CUDA sort needs a GPU per rank).
The concatenation of the ranks' outputs must be the stable sort of the
concatenated inputs, bit for bit, in keys and payloads (payload = global
input index)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port() -> int:
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _oracle_local_sort(k, v):
    import oracle

    kk, vv = oracle.zsort_pairs(k.numpy().view(np.uint64), v.numpy().view(np.uint32))
    return torch.from_numpy(kk.view(np.int64).copy()), torch.from_numpy(vv.view(np.int32).copy())


def _shard(case, rank):
    rng = np.random.default_rng(100 + rank)
    if case == "duplicates":  # few values, all with the top bit in play, repeated across ranks
        n = [5000, 3000][rank]
        return rng.integers(0, 50, n).astype(np.uint64) * np.uint64(2 ** 58)
    if case == "empty_rank":
        n = [0, 4000][rank]
        return rng.integers(0, 2 ** 63, n, dtype=np.uint64) * np.uint64(2)
    if case == "all_equal":
        return np.full(7000, 12345, dtype=np.uint64)
    if case == "wide":
        return rng.integers(0, 2 ** 64 - 1, [20_000, 13_000][rank], dtype=np.uint64)
    raise ValueError(case)


def _worker(rank, world, port, case, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2605_14419_gb300 import distributed as D

        keys = _shard(case, rank)
        sizes = [None] * world
        dist.all_gather_object(sizes, int(keys.size))
        base = sum(sizes[:rank])
        vals = (np.arange(keys.size) + base).astype(np.uint32)
        k, v = D.sample_sort(torch.from_numpy(keys.view(np.int64)), torch.from_numpy(vals.view(np.int32)),
                             local_sort=_oracle_local_sort, sample=64)
        got_k, got_v, inputs = [None] * world, [None] * world, [None] * world
        dist.all_gather_object(got_k, k.numpy().view(np.uint64).tolist())
        dist.all_gather_object(got_v, v.numpy().view(np.uint32).tolist())
        dist.all_gather_object(inputs, keys.tolist())
        if rank == 0:
            inp = np.array(sum(inputs, []), dtype=np.uint64)
            order = np.argsort(inp, kind="stable")
            gk = np.array(sum(got_k, []), dtype=np.uint64)
            gv = np.array(sum(got_v, []), dtype=np.uint32)
            out.put((bool(np.array_equal(gk, inp[order])), bool(np.array_equal(gv, order.astype(np.uint32))),
                     [len(x) for x in got_k]))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("case", ["duplicates", "empty_rank", "all_equal", "wide"])
def test_sample_sort_two_ranks_is_the_global_stable_sort(case):
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, case, out)) for r in range(2)]
    for p in procs:
        p.start()
    keys_ok, vals_ok, sizes = out.get(timeout=180)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert keys_ok and vals_ok
    if case == "all_equal":  # every copy of a key goes to one rank
        assert sorted(sizes) == [0, 14000]
    if case == "wide":  # the splitters balance distinct keys
        assert min(sizes) > 0.3 * sum(sizes)


def test_splitters_are_sample_quantiles():
    from paper_2605_14419_gb300 import distributed as D

    g = torch.arange(100, dtype=torch.int64).flip(0)
    assert D.splitters_from_sample(g, 4).tolist() == [25, 50, 75]
    assert D.splitters_from_sample(g, 1).numel() == 0
    assert D.splitters_from_sample(torch.empty(0, dtype=torch.int64), 3).numel() == 0
