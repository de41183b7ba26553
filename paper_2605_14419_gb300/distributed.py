"""Sample sort across ranks: one globally sorted, stable order of every
rank's (key, payload) shard, with one exchange step.

The paper sorts on one CPU and names distributed sorting as future work
(section "Conclusion").  zSort partitions by a monotone map of the key, and
the same idea spans GPUs: ranks agree on a monotone map of the keys onto
P = world_size ranges, every rank sends each range to its rank, and every
rank sorts what it received.  The steps:

  1. every rank sorts its shard locally (stable, by key);
  2. every rank draws `sample` keys at evenly spaced ranks of its sorted
     shard; one all_gather gives every rank all of them; the P - 1 splitters
     are the sample keys at ranks j * m / P (j = 1 .. P-1) of the gathered
     sample, so every rank computes the same splitters;
  3. the sorted shard splits into P contiguous runs at the splitters: run r
     holds the keys with splitters[r-1] <= key < splitters[r], so all copies
     of a key go to one rank;
  4. one all_to_all of the run sizes, then one all_to_all of keys and one of
     payloads: rank r receives run r of every rank, in rank order;
  5. every rank sorts what it received, stably.  Equal keys arrive in source
     rank order and, within a rank, in that rank's input order, so the
     concatenation of the ranks' outputs in rank order is the stable sort of
     the concatenated inputs (rank-major input order).

The local sorts are this library's zsort_pairs on the rank's GPU
(`local_sort` defaults to it).  Keys are uint64 held in int64 tensors;
comparisons here flip the sign bit so that they follow unsigned order.
The multi-process tests run the exchange over gloo on CPU tensors with the
local sort passed in; this build's runs use one GPU, so the collective
path is not measured on hardware.
"""
from __future__ import annotations

import torch
import torch.distributed as dist

SIGN = -(2 ** 63)


def _as_signed_order(k: torch.Tensor) -> torch.Tensor:
    """int64 view of uint64 keys whose signed order is their unsigned order."""
    return k ^ torch.tensor(SIGN, dtype=torch.int64, device=k.device)


def _gpu_local_sort(keys: torch.Tensor, vals: torch.Tensor):
    from paper_2605_14419_gb300 import sort_pairs

    k, v = keys.clone(), vals.clone()
    if k.numel() > 1:
        sort_pairs(k, v)
    return k, v


def splitters_from_sample(gathered: torch.Tensor, world: int) -> torch.Tensor:
    """The P - 1 splitters (in signed-order form) from the gathered sample:
    its keys at ranks j * m / P, j = 1 .. P-1."""
    s, _ = torch.sort(gathered)
    m = s.numel()
    if m == 0:
        return torch.empty(0, dtype=torch.int64, device=gathered.device)
    idx = torch.tensor([j * m // world for j in range(1, world)], dtype=torch.int64, device=gathered.device)
    return s[idx.clamp(max=m - 1)]


def sample_sort(keys: torch.Tensor, vals: torch.Tensor, group=None, local_sort=None, sample: int = 4096):
    """Globally sorts the shards of all ranks of `group`; returns this rank's
    part of the sorted order (keys, vals): rank r holds the r-th contiguous
    piece.  keys: int64 tensor holding uint64 keys; vals: int32 payloads."""
    assert keys.dtype == torch.int64 and vals.dtype == torch.int32 and keys.shape == vals.shape
    local_sort = local_sort or _gpu_local_sort
    world = dist.get_world_size(group)
    dev = keys.device
    k, v = local_sort(keys, vals)  # 1. stable local sort
    if world == 1:
        return k, v
    so = _as_signed_order(k)
    n = so.numel()
    # 2. evenly spaced sample of the sorted shard, gathered on every rank
    m = min(sample, n)
    pos = (torch.arange(m, dtype=torch.int64, device=dev) * n + n // 2) // max(m, 1) if m else \
        torch.empty(0, dtype=torch.int64, device=dev)
    mine = so[pos] if m else torch.empty(0, dtype=torch.int64, device=dev)
    counts = [torch.zeros(1, dtype=torch.int64, device=dev) for _ in range(world)]
    dist.all_gather(counts, torch.tensor([m], dtype=torch.int64, device=dev), group=group)
    cmax = int(max(int(c.item()) for c in counts))
    padded = torch.full((cmax,), 0, dtype=torch.int64, device=dev)
    padded[:m] = mine
    parts = [torch.empty(cmax, dtype=torch.int64, device=dev) for _ in range(world)]
    dist.all_gather(parts, padded, group=group)
    gathered = torch.cat([p[: int(c.item())] for p, c in zip(parts, counts)])
    split = splitters_from_sample(gathered, world)
    # 3. runs of the sorted shard: run r = [bound[r], bound[r+1])
    inner = torch.searchsorted(so, split, right=False) if split.numel() else \
        torch.empty(0, dtype=torch.int64, device=dev)
    bounds = torch.cat([torch.zeros(1, dtype=torch.int64, device=dev), inner,
                        torch.tensor([n], dtype=torch.int64, device=dev)])
    send = (bounds[1:] - bounds[:-1]).to(torch.int64)
    # 4. the exchange: sizes, then keys and payloads
    recv = torch.empty(world, dtype=torch.int64, device=dev)
    dist.all_to_all_single(recv, send, group=group)
    send_l, recv_l = [int(x) for x in send.tolist()], [int(x) for x in recv.tolist()]
    rk = torch.empty(sum(recv_l), dtype=torch.int64, device=dev)
    rv = torch.empty(sum(recv_l), dtype=torch.int32, device=dev)
    dist.all_to_all_single(rk, k.contiguous(), recv_l, send_l, group=group)
    dist.all_to_all_single(rv, v.contiguous(), recv_l, send_l, group=group)
    # 5. stable sort of the received runs (in source rank order)
    return local_sort(rk, rv)
