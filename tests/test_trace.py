"""Task trace of the persistent kernel (ZSORT_FLAG_TRACE): the records
account for every task the call ran, lie inside the launch, never overlap
on one CTA, and tracing leaves the sorted output unchanged.  Also checks on
the host (no GPU) that the record layout of the binding matches the C
header's."""
import ctypes
import re
from pathlib import Path

import numpy as np
import pytest

import paper_2605_14419_gb300 as z
from paper_2605_14419_gb300 import inputs

ROOT = Path(__file__).resolve().parents[1]


def test_trace_record_layout_matches_the_header():
    text = (ROOT / "include" / "zsort.h").read_text()
    body = re.search(r"typedef struct \{([^}]*)\} zsort_trace_rec;", text).group(1)
    fields = re.findall(r"uint(\d+)_t\s+(\w+);", body)
    assert [name for _, name in fields] == [f for f, _ in z.TraceRec._fields_]
    sizes = {"8": 1, "16": 2, "32": 4, "64": 8}
    assert sum(sizes[b] for b, _ in fields) == ctypes.sizeof(z.TraceRec) == 32
    assert int(re.search(r"#define ZSORT_FLAG_TRACE (\d+)u", text).group(1)) == z.FLAG_TRACE
    assert re.search(r"#define ZSORT_TRACE_CAP \(1u << (\d+)\)", text).group(1) == "20"


torch = pytest.importorskip("torch")
gpu = pytest.mark.gpu
needs_cuda = pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")


def sort_traced(keys, vals, opts):
    import oracle

    dev = torch.device("cuda:0")
    k = torch.from_numpy(keys.view(np.int64)).to(dev)
    v = torch.from_numpy(vals.view(np.int32)).to(dev)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        z.sort_pairs(k, v, opts=opts, stream=stream)
        st = z.last_stats(stream)
        rec, count = z.last_trace(stream)
    ok, ov = oracle.zsort_pairs(keys, vals)
    assert np.array_equal(k.cpu().numpy().view(np.uint64), ok)
    assert np.array_equal(v.cpu().numpy().view(np.uint32), ov)
    return st, rec, count


@gpu
@needs_cuda
@pytest.mark.parametrize("family,mapper", [("lognormal", 1), ("zipf", 0), ("uniform", 0)])
def test_trace_accounts_for_every_task(family, mapper):
    gen = {"lognormal": inputs.lognormal, "zipf": inputs.zipf, "uniform": inputs.uniform}[family]
    keys = gen(3_000_000, 17)
    vals = inputs.index_payload(keys.size)
    opts = z.default_opts(mapper=mapper, flags=z.FLAG_TRACE)
    st, rec, count = sort_traced(keys, vals, opts)
    assert count == rec.size > 0
    # tiles / items of all records = the tasks the kernel counted
    assert int(rec["count"].astype(np.uint64).sum()) == st["tasks"]
    base = rec["type"] & (z.TRACE_HANDLER - 1)
    assert set(np.unique(base)) <= set(z.TASK_TYPES)
    hnd = (rec["type"] & z.TRACE_HANDLER) != 0
    assert np.all(rec["count"][hnd] == 0) and hnd.any()
    # a phase's completion work follows its last task on the same CTA
    assert np.any(base[hnd] == 4)
    assert np.all(rec["t_start_ns"] <= rec["t_end_ns"])
    assert np.all(rec["cta"] < st["persistent_ctas"])
    # per CTA the tasks run one after the other
    order = np.lexsort((rec["t_start_ns"], rec["cta"]))
    r = rec[order]
    same = r["cta"][1:] == r["cta"][:-1]
    assert np.all(r["t_end_ns"][:-1][same] <= r["t_start_ns"][1:][same])
    # every leaf is one finish item; partitions report their depth
    assert int(rec["count"][rec["type"] == 6].sum()) == st["leaves"]
    assert int(re.search(r"#define ZSORT_TRACE_HANDLER (\d+)u", (ROOT / "include" / "zsort.h").read_text()).group(1)) \
        == z.TRACE_HANDLER
    assert int(rec["level"].max()) <= st["max_level"] + 1
    if mapper == 1:
        assert np.any(rec["type"] == 9)  # the learned map was fitted
    # sub-arrays below the top took sampled statistics (one task each), or
    # the exact pass after a sample without spread
    assert int((rec["type"] == 10).sum()) >= st["sampled_stats"]


@gpu
@needs_cuda
def test_untraced_call_reports_no_trace():
    keys = inputs.uniform(200_000, 3)
    vals = inputs.index_payload(keys.size)
    _, rec, count = sort_traced(keys, vals, z.default_opts(flags=z.FLAG_TRACE))
    assert count > 0
    _, rec, count = sort_traced(keys, vals, z.default_opts())
    assert count == 0 and rec.size == 0


def _chunk_plan(n, ln, cpc, nctas, tile=z.TILE_PAIRS):
    """The chunk geometry of a large (sub)array: chunks of ct tiles, the last
    round's worth of tiles in chunks of a quarter of that size."""
    tiles = (ln + tile - 1) // tile
    target = max(1, (cpc * nctas * ln + n - 1) // n)
    ct = max(4, (tiles + target - 1) // target)
    whole = (tiles + ct - 1) // ct
    small = max(4, ct // 4)
    if whole > 2 * nctas and small < ct:
        big = (tiles - nctas * ct) // ct
        return big + (tiles - big * ct + small - 1) // small
    return whole


@gpu
@needs_cuda
@pytest.mark.parametrize("cpc", [3, 8])
def test_short_chunks_end_the_top_level_phases(cpc):
    """A top-level array spanning several rounds of chunks ends each phase
    with short chunks; the result stays the stable sort (duplicate-heavy keys,
    checked by properties at 2^24) and the trace shows the planned count."""
    n = 1 << 24
    keys = inputs.zipf(n, 29)
    dev = torch.device("cuda:0")
    k_in = torch.from_numpy(keys.view(np.int64)).to(dev)
    k = k_in.clone()
    v = torch.arange(n, dtype=torch.int32, device=dev)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        z.sort_pairs(k, v, opts=z.default_opts(chunks_per_cta=cpc, flags=z.FLAG_TRACE), stream=stream)
        st = z.last_stats(stream)
        rec, count = z.last_trace(stream)
    pos = v.to(torch.int64) & 0xFFFFFFFF
    assert bool(torch.equal(k_in[pos], k))
    assert bool((torch.bincount(pos, minlength=n) == 1).all())
    s = k ^ torch.tensor(-(2 ** 63), dtype=torch.int64, device=dev)
    assert bool((s[1:] >= s[:-1]).all())
    eq = s[1:] == s[:-1]
    assert bool((pos[1:][eq] > pos[:-1][eq]).all())
    top = (rec["level"] == 0) & (rec["type"] == 4)
    assert int(rec["count"][top].sum()) == _chunk_plan(n, n, cpc, st["persistent_ctas"])
