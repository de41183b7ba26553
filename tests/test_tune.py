"""Autotuner: call classes and the JSON cache on the host (no GPU), and a
tuning run on the GPU whose chosen options still give the oracle's output.

The tuner is not part of the method (the paper fixes its constants for one
CPU thread); any options it returns must leave the sorted output unchanged,
which the GPU tests check against the oracle."""
import ctypes
import json
import os

import numpy as np
import pytest

import paper_2605_14419_gb300 as z
from paper_2605_14419_gb300 import build as zbuild
from paper_2605_14419_gb300 import inputs


@pytest.fixture(scope="module")
def lib():
    zbuild.build()
    return z.load()


# ------------------------------------------------------------ classes (host)
def strided(keys, m=4096):
    n = keys.size
    m = min(m, n)
    return keys[(np.arange(m, dtype=np.uint64) * np.uint64(n) // np.uint64(m)).astype(np.int64)]


def test_class_string_format(lib):
    keys = inputs.uniform(1 << 20, 1)
    assert z.tune_class_host(strided(keys), keys.size, 0, 152) == "sm152/n20/s0/flat"
    # segmented: log2 of the segment count, rounded
    assert z.tune_class_host(strided(keys), 2_035_112_118, 20_000, 152) == "sm152/n31/s14/flat"
    assert z.tune_class_host(strided(keys), keys.size, 1, 148) == "sm148/n20/s0/flat"


def test_class_of_each_family(lib):
    n = 1 << 20
    assert z.tune_class_host(strided(inputs.zipf(n, 3)), n).endswith("/dup")
    assert z.tune_class_host(strided(np.sort(inputs.uniform(n, 4))), n).endswith("/sorted")
    assert z.tune_class_host(strided(inputs.descending(n, 5)), n).endswith("/reversed")
    assert z.tune_class_host(strided(inputs.nearly_sorted(n, 6)), n).endswith("/sorted")
    # Eq. 1 with scale k/4 spans [min, min + 4 sd): a uniform law (range
    # sqrt(12) sd) fits in it; a normal one (min near mean - 3.5 sd) puts
    # every key above mean + 0.5 sd into the last bucket, and the lognormal's
    # mass sits in a few buckets near the minimum
    assert z.tune_class_host(strided(inputs.uniform(n, 9)), n).endswith("/flat")
    assert z.tune_class_host(strided(inputs.normal(n, 8)), n).endswith("/skew")
    assert z.tune_class_host(strided(inputs.lognormal(n, 7)), n).endswith("/skew")


def test_class_rules_at_their_thresholds(lib):
    m = 4000
    # exactly half distinct is not "dup"; one fewer distinct is
    half = np.repeat(np.arange(1, 2001, dtype=np.uint64) * np.uint64(7919), 2)
    rng = np.random.default_rng(0)
    rng.shuffle(half)
    assert not z.tune_class_host(half, m).endswith("/dup")
    fewer = half.copy()
    fewer[fewer == fewer[0]] = fewer[1] if fewer[1] != fewer[0] else fewer[2]
    assert z.tune_class_host(fewer, m).endswith("/dup")
    # 90% of adjacent pairs ascending -> sorted (distinct keys, shuffled tail)
    base = np.arange(m, dtype=np.uint64) * np.uint64(1 << 40)
    keys = base.copy()
    tail = keys[3700:].copy()
    rng.shuffle(tail)
    keys[3700:] = tail
    asc = int(np.sum(keys[:-1] <= keys[1:]))
    expect = "sorted" if 10 * asc >= 9 * (m - 1) else None
    got = z.tune_class_host(keys, m).rsplit("/", 1)[1]
    if expect:
        assert got == expect
    else:
        assert got in ("flat", "skew")


def test_class_edge_inputs(lib):
    assert z.tune_class_host(np.zeros(0, np.uint64), 0) == "sm152/n0/s0/flat"
    assert z.tune_class_host(np.array([5], np.uint64), 1) == "sm152/n0/s0/flat"
    buf = ctypes.create_string_buffer(8)
    a = np.arange(10, dtype=np.uint64)
    assert lib.zsort_tune_class_host(a.ctypes.data, 10, 10, 0, 152, buf, 8) == z.ERR_INVALID


# ------------------------------------------------------------ cache (host)
def tuned(kmax=512, leaf_target=2048, leaf_cap=4096, large_min=65536, chunks=8, ipt=12):
    o = z.default_opts()
    o.kmax, o.leaf_target, o.leaf_cap, o.large_min, o.chunks_per_cta = kmax, leaf_target, leaf_cap, large_min, chunks
    o.ipt = ipt
    return o


def test_cache_missing_file_and_entry(lib, tmp_path):
    path = str(tmp_path / "tune.json")
    assert z.tune_cache_get(path, "sm152/n20/s0/flat") is None
    z.tune_cache_put(path, "sm152/n20/s0/flat", tuned(), 1.5)
    assert z.tune_cache_get(path, "sm152/n20/s0/skew") is None


def test_cache_round_trip_and_update(lib, tmp_path):
    path = str(tmp_path / "tune.json")
    z.tune_cache_put(path, "sm152/n28/s0/flat", tuned(kmax=512, chunks=16), 14.25)
    z.tune_cache_put(path, "sm152/n31/s14/flat", tuned(leaf_cap=3072, large_min=131072), 203.5)
    o, ms = z.tune_cache_get(path, "sm152/n28/s0/flat")
    assert (o.kmax, o.chunks_per_cta, o.leaf_cap, ms) == (512, 16, 4096, 14.25)
    # other fields come from the base, not the file
    assert o.mapper == z.MAP_ZSCORE and o.struct_size == ctypes.sizeof(z.Opts)
    z.tune_cache_put(path, "sm152/n28/s0/flat", tuned(kmax=256, leaf_target=1024, ipt=8), 13.0)
    o, ms = z.tune_cache_get(path, "sm152/n28/s0/flat")
    assert (o.kmax, o.leaf_target, o.chunks_per_cta, o.ipt, ms) == (256, 1024, 8, 8, 13.0)
    o2, ms2 = z.tune_cache_get(path, "sm152/n31/s14/flat")
    assert (o2.leaf_cap, o2.large_min, ms2) == (3072, 131072, 203.5)
    # the file is a JSON object of the two entries
    with open(path) as f:
        doc = json.load(f)
    assert set(doc) == {"sm152/n28/s0/flat", "sm152/n31/s14/flat"}
    assert doc["sm152/n28/s0/flat"] == {"kmax": 256, "leaf_target": 1024, "leaf_cap": 4096,
                                        "large_min": 65536, "chunks_per_cta": 8, "ipt": 8, "ms": 13.0}
    assert not os.path.exists(path + ".tmp")


def test_cache_rejects_bad_values(lib, tmp_path):
    path = str(tmp_path / "tune.json")
    with pytest.raises(z.ZsortError):
        z.tune_cache_put(path, "a", tuned(kmax=1000), 1.0)
    with pytest.raises(z.ZsortError):
        z.tune_cache_put(path, "a", tuned(leaf_cap=8192), 1.0)
    with pytest.raises(z.ZsortError):
        z.tune_cache_put(path, "a", tuned(ipt=10), 1.0)
    with pytest.raises(z.ZsortError):
        z.tune_cache_put(path, 'bad"name', tuned(), 1.0)
    assert not os.path.exists(path)


def test_cache_malformed_entry(lib, tmp_path):
    path = tmp_path / "tune.json"
    path.write_text('{\n"good": {"kmax": 256, "leaf_target": 2048, "leaf_cap": 4096, "large_min": 65536, '
                    '"chunks_per_cta": 8, "ms": 2.0},\n"broken": {"kmax": 300, "leaf_target": 2048},\n}\n')
    o, ms = z.tune_cache_get(str(path), "good")
    assert o.kmax == 256 and ms == 2.0
    with pytest.raises(z.ZsortError):
        z.tune_cache_get(str(path), "broken")


def test_default_opts_carry_the_new_knobs(lib):
    o = z.default_opts()
    assert (o.leaf_cap, o.chunks_per_cta) == (4096, 8)
    for field, bad in (("leaf_cap", 255), ("leaf_cap", 4097), ("chunks_per_cta", 0), ("chunks_per_cta", 65)):
        b = z.default_opts(**{field: bad})
        assert lib.zsort_pairs_ex(None, 0, None, 10, ctypes.byref(b), None) == z.ERR_INVALID


# ------------------------------------------------------------ GPU
torch = pytest.importorskip("torch")
gpu = pytest.mark.gpu
needs_cuda = pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")


@gpu
@needs_cuda
def test_autotune_single_array_keeps_parity(lib, tmp_path):
    import oracle

    path = str(tmp_path / "tune.json")
    keys = inputs.gaussian_mixture(1 << 20, 11)
    vals = inputs.index_payload(keys.size)
    dev = torch.device("cuda:0")
    k = torch.from_numpy(keys.view(np.int64)).to(dev)
    v = torch.from_numpy(vals.view(np.int32)).to(dev)
    o = z.autotune(k, v, cache_path=path, budget_ms=60_000, reps=1)
    # the inputs are untouched; the class is cached with the chosen fields
    assert np.array_equal(k.cpu().numpy().view(np.uint64), keys)
    assert np.array_equal(v.cpu().numpy().view(np.uint32), vals)
    cls = z.tune_class(k)
    got = z.tune_cache_get(path, cls)
    assert got is not None
    c, ms = got
    assert (c.kmax, c.leaf_target, c.leaf_cap, c.large_min, c.chunks_per_cta) == \
        (o.kmax, o.leaf_target, o.leaf_cap, o.large_min, o.chunks_per_cta)
    assert ms > 0
    # a second call is served from the cache; the lookup agrees
    o2 = z.autotune(k, v, cache_path=path, budget_ms=1)
    assert bytes(o2) == bytes(o)
    o3, found = z.tuned_opts(k, cache_path=path)
    assert found and bytes(o3) == bytes(o)
    # the tuned options sort exactly like the oracle
    z.sort_pairs(k, v, opts=o)
    ok, ov = oracle.zsort_pairs(keys, vals)
    assert np.array_equal(k.cpu().numpy().view(np.uint64), ok)
    assert np.array_equal(v.cpu().numpy().view(np.uint32), ov)


@gpu
@needs_cuda
def test_autotune_segmented_keeps_parity(lib, tmp_path):
    import oracle

    keys, vals, off, _ = inputs.segmented(200, 21, lo=32, hi=100_000)
    dev = torch.device("cuda:0")
    k = torch.from_numpy(keys.view(np.int64)).to(dev)
    v = torch.from_numpy(vals.view(np.int32)).to(dev)
    o_dev = torch.from_numpy(off.view(np.int64)).to(dev)
    o = z.autotune(k, v, offsets=o_dev, cache_path=str(tmp_path / "t.json"), budget_ms=60_000, reps=1)
    assert z.tune_class(k, nseg=200).startswith("sm") and "/s8/" in z.tune_class(k, nseg=200)
    z.sort_segmented(k, v, o_dev, opts=o)
    ok, ov = oracle.zsort_segmented(keys, vals, off)
    assert np.array_equal(k.cpu().numpy().view(np.uint64), ok)
    assert np.array_equal(v.cpu().numpy().view(np.uint32), ov)


@gpu
@needs_cuda
@pytest.mark.parametrize("leaf_cap,chunks", [(256, 1), (2048, 4), (3000, 64)])
def test_knob_extremes_keep_parity(lib, leaf_cap, chunks):
    import oracle

    keys = inputs.lognormal(600_000, 12)
    vals = inputs.index_payload(keys.size)
    dev = torch.device("cuda:0")
    k = torch.from_numpy(keys.view(np.int64)).to(dev)
    v = torch.from_numpy(vals.view(np.int32)).to(dev)
    z.sort_pairs(k, v, opts=z.default_opts(leaf_cap=leaf_cap, chunks_per_cta=chunks, large_min=65536))
    ok, ov = oracle.zsort_pairs(keys, vals)
    assert np.array_equal(k.cpu().numpy().view(np.uint64), ok)
    assert np.array_equal(v.cpu().numpy().view(np.uint32), ov)


def test_cache_entry_without_ipt_reads_as_the_default(lib, tmp_path):
    """Entries written before items per thread became a knob parse with the
    default of 12."""
    path = tmp_path / "tune.json"
    path.write_text('{\n"old": {"kmax": 256, "leaf_target": 2048, "leaf_cap": 4096, "large_min": 65536, '
                    '"chunks_per_cta": 8, "ms": 2.0}\n}\n')
    o, ms = z.tune_cache_get(str(path), "old")
    assert (o.kmax, o.ipt, ms) == (256, 12, 2.0)
