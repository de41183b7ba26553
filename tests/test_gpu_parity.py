"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

The result of a stable sort is unique, so the bar is bit-exact keys and
payloads.  At sizes the oracle finishes in seconds the two are compared
element by element; at the full 2^28 size the output is checked by
properties that pin it completely (keys non-decreasing, payload i is the
input position of output key i, and ties keep ascending positions).
"""
import numpy as np
import pytest

import oracle
from paper_2605_14419_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU machine
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2605_14419_gb300 as z  # noqa: E402
from paper_2605_14419_gb300 import build as zbuild  # noqa: E402

zbuild.build()
DEV = torch.device("cuda:0")


def to_dev(keys, vals):
    k = torch.from_numpy(np.ascontiguousarray(keys).view(np.int64)).to(DEV)
    v = torch.from_numpy(np.ascontiguousarray(vals).view(np.int32)).to(DEV)
    return k, v


def gpu_sort(keys, vals, opts=None, key_type="u64"):
    k, v = to_dev(keys, vals)
    z.sort_pairs(k, v, key_type=key_type, opts=opts)
    return k.cpu().numpy().view(keys.dtype), v.cpu().numpy().view(np.uint32)


def assert_same_as_oracle(keys, vals=None, opts=None):
    vals = inputs.index_payload(keys.size) if vals is None else vals
    gk, gv = gpu_sort(keys, vals, opts)
    ok, ov = oracle.zsort_pairs(keys, vals)
    assert np.array_equal(gk, ok), "keys differ"
    assert np.array_equal(gv, ov), "payloads differ"


FAMILIES = list(inputs.FAMILIES)
SIZES = [2, 3, 31, 255, 256, 257, 1000, 4095, 4096, 4097, 8193, 65535, 65536, 65537, 200_003]


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("family", FAMILIES)
def test_parity_sizes(family, n):
    assert_same_as_oracle(inputs.FAMILIES[family](n, seed=n + 1))


def test_config1_uniform_65536_seed0():
    assert_same_as_oracle(inputs.uniform(65_536, 0))


@pytest.mark.parametrize("family", FAMILIES)
def test_config2_paper_scale_1e7(family):
    assert_same_as_oracle(inputs.FAMILIES[family](10_000_000, seed=2))


@pytest.mark.parametrize("gen", [inputs.lognormal, inputs.gaussian_mixture, inputs.dense_interval_u64])
@pytest.mark.parametrize("mapper", [z.MAP_ZSCORE, z.MAP_LEARNED])
def test_skewed_both_mappers(gen, mapper):
    keys = gen(3_000_000, seed=4)
    assert_same_as_oracle(keys, opts=z.default_opts(mapper=mapper))


def test_edge_cases():
    # empty, single, all equal, two values, extremes, random payload
    for keys in (np.zeros(0, np.uint64), np.array([5], np.uint64), np.full(100_000, 7, np.uint64),
                 np.array([2 ** 64 - 1, 0] * 50_000, np.uint64),
                 np.array([2 ** 63 + 1, 2 ** 63] * 40_000, np.uint64)):
        vals = inputs.index_payload(keys.size)
        if keys.size <= 1:
            k, v = to_dev(keys, vals) if keys.size else (torch.zeros(0, dtype=torch.int64, device=DEV),
                                                          torch.zeros(0, dtype=torch.int32, device=DEV))
            z.sort_pairs(k, v)
            assert np.array_equal(k.cpu().numpy().view(np.uint64), keys)
            continue
        assert_same_as_oracle(keys)
    rng = np.random.default_rng(3)
    keys = rng.integers(0, 1000, 300_000).astype(np.uint64)
    vals = rng.integers(0, 2 ** 32, 300_000, dtype=np.uint64).astype(np.uint32)
    assert_same_as_oracle(keys, vals)


def test_small_kmax_forces_deep_recursion():
    keys = inputs.uniform(2_000_000, 5)
    assert_same_as_oracle(keys, opts=z.default_opts(kmax=16, leaf_target=64, large_min=8192))


def test_guard_level_range_map():
    keys = inputs.lognormal(1_000_000, 6)
    assert_same_as_oracle(keys, opts=z.default_opts(guard_level=1))


def test_int64_and_float64_keys():
    x = inputs.dense_interval_i64(500_000, 7)
    vals = inputs.index_payload(x.size)
    gk, gv = gpu_sort(x.astype(np.int64), vals, key_type="i64")
    u = oracle.key_from_i64(x)
    ok, ov = oracle.zsort_pairs(u, vals)
    assert np.array_equal(gv, ov) and np.array_equal(gk, oracle.key_to_i64(ok))
    f = inputs.normal_f64_specials(500_000, 8)
    gk, gv = gpu_sort(f, vals, key_type="f64")
    u = oracle.key_from_f64(f)
    ok, ov = oracle.zsort_pairs(u, vals)
    assert np.array_equal(gv, ov)
    assert np.array_equal(gk.view(np.uint64), oracle.key_to_f64(ok).view(np.uint64))


def test_segmented_matches_oracle():
    keys, vals, off, _ = inputs.segmented(300, 9, lo=1, hi=300_000)
    k, v = to_dev(keys, vals)
    offs = torch.from_numpy(off.view(np.int64)).to(DEV)
    z.sort_segmented(k, v, offs)
    ok, ov = oracle.zsort_segmented(keys, vals, off)
    assert np.array_equal(k.cpu().numpy().view(np.uint64), ok)
    assert np.array_equal(v.cpu().numpy().view(np.uint32), ov)


def test_segmented_empty_and_untouched_edges():
    keys = inputs.uniform(10_000, 10)
    vals = inputs.index_payload(keys.size)
    off = np.array([100, 100, 5000, 5000, 9000], dtype=np.uint64)  # empty segments; outside untouched
    k, v = to_dev(keys, vals)
    z.sort_segmented(k, v, torch.from_numpy(off.view(np.int64)).to(DEV))
    gk = k.cpu().numpy().view(np.uint64)
    assert np.array_equal(gk[:100], keys[:100]) and np.array_equal(gk[9000:], keys[9000:])
    ok, ov = oracle.zsort_segmented(keys, vals, off)
    assert np.array_equal(gk, ok)


def test_bad_offsets_reported_and_data_untouched_then_recovers():
    keys = inputs.uniform(10_000, 11)
    vals = inputs.index_payload(keys.size)
    k, v = to_dev(keys, vals)
    bad = torch.tensor([0, 6000, 5000, 10_000], dtype=torch.int64, device=DEV)
    with pytest.raises(z.ZsortError) as ei:
        z.sort_segmented(k, v, bad)
    assert ei.value.code == z.ERR_BAD_OFFSETS
    assert np.array_equal(k.cpu().numpy().view(np.uint64), keys)
    past_end = torch.tensor([0, 10_001], dtype=torch.int64, device=DEV)
    with pytest.raises(z.ZsortError):
        z.sort_segmented(k, v, past_end)
    assert_same_as_oracle(keys)  # the next call works


def _check_full_properties(k_in, k_out, v_out):
    """Sorted, stable, and payload = input position of the output key."""
    pos = v_out.to(torch.int64) & 0xFFFFFFFF
    # payload is a permutation and points at the same key in the input
    assert bool(torch.equal(k_in[pos], k_out))
    seen = torch.zeros(k_in.numel(), dtype=torch.int32, device=DEV)
    seen.index_add_(0, pos, torch.ones_like(pos, dtype=torch.int32))
    assert bool((seen == 1).all())
    # order: compare as unsigned by flipping the sign bit
    s = k_out ^ torch.tensor(-(2 ** 63), dtype=torch.int64, device=DEV)
    assert bool((s[1:] >= s[:-1]).all())
    eq = s[1:] == s[:-1]
    assert bool((pos[1:][eq] > pos[:-1][eq]).all())


@pytest.mark.parametrize("gen", [inputs.lognormal, inputs.gaussian_mixture])
@pytest.mark.parametrize("mapper", [z.MAP_ZSCORE, z.MAP_LEARNED])
def test_full_size_2p28_properties(gen, mapper):
    n = 1 << 28
    keys = gen(n, seed=3)
    k_in = torch.from_numpy(keys.view(np.int64)).to(DEV)
    k = k_in.clone()
    v = torch.arange(n, dtype=torch.int32, device=DEV)
    z.sort_pairs(k, v, opts=z.default_opts(mapper=mapper))
    _check_full_properties(k_in, k, v)
    del k_in, k, v
    torch.cuda.empty_cache()


# ---------------------------------------------------------------- map rows
def _map_case(gen, n, seed):
    keys = gen(n, seed)
    kd = torch.from_numpy(keys.view(np.int64)).to(DEV)
    return keys, kd


def _dense_i64_encoded(n, seed):
    """The int64 dense-interval law in the order-preserving unsigned encoding:
    most keys within 2^19 of 2^63, so binary32 normalisation collapses them."""
    return inputs.dense_interval_i64(n, seed).view(np.uint64) ^ np.uint64(2 ** 63)


def _sample_max_load(buckets, k):
    return int(np.bincount(buckets.astype(np.int64), minlength=k).max())


@pytest.mark.parametrize("gen", [inputs.lognormal, inputs.gaussian_mixture, inputs.uniform,
                                 inputs.dense_interval_u64, inputs.zipf, _dense_i64_encoded])
def test_learned_map_buckets_bit_exact(gen):
    """Learned map (training sample, breakpoints, buckets) against the oracle's
    definition, bit for bit; the Eq. 1 fallback decision is checked from the
    load-test numbers the device reports.  When the normalised map fails its
    load test the device tries the exact-key breakpoints: its buckets and
    its accept / reject decision are checked against the oracle's."""
    n, m = 400_000, 65536
    keys, kd = _map_case(gen, n, 13)
    opts = z.default_opts(mapper=z.MAP_LEARNED, learn_min=m, sample=m, kmax=512)
    gb, info = z.map_buckets(kd, opts)
    mn, mx = int(keys.min()), int(keys.max())
    assert info.min == mn and info.max == mx
    if mn == mx:
        assert np.all(gb.cpu().numpy() == 0)
        return
    assert info.trained == 1
    pos = oracle.sample_positions(opts.seed, n, m).astype(np.int64)
    q = oracle.pwl_train(keys[pos], mn, mx)
    assert np.array_equal(np.frombuffer(bytes(info.q), dtype=np.float32), q)
    k = info.k
    if info.map == z.MAPINFO_LEARNED:
        ob = oracle.pwl_buckets(keys, mn, mx, q, k)
        assert np.array_equal(gb.cpu().numpy().view(np.uint32), ob)
        return
    # rejected by the load test: its rule, from the reported loads
    assert (info.learned_max_load > opts.fallback_ratio * m / k
            or info.learned_max_load > info.zscore_max_load)
    b, r = oracle.split_train(keys[pos], mn, mx)
    split_load = _sample_max_load(oracle.split_buckets(keys[pos], b, r, k), k)
    split_ok = split_load <= opts.fallback_ratio * m / k and split_load <= info.zscore_max_load
    assert info.map == (z.MAPINFO_SPLIT if split_ok else z.MAPINFO_ZSCORE)
    if split_ok:
        ob = oracle.split_buckets(keys, b, r, k)
        assert np.array_equal(gb.cpu().numpy().view(np.uint32), ob)
    if gen is _dense_i64_encoded:
        assert info.map == z.MAPINFO_SPLIT


def _top_keys(n, seed):
    """Keys just below 2^64 with both 32-bit halves large: every limb of the
    exact sums carries."""
    rng = np.random.default_rng(seed)
    return (np.uint64(2**64 - 1) - rng.integers(0, 2**40, n, dtype=np.uint64)).astype(np.uint64)


@pytest.mark.parametrize("gen", [inputs.uniform, inputs.normal, inputs.lognormal, inputs.nearly_sorted, _top_keys])
def test_zscore_map_and_stats(gen):
    """Eq. 1 map on the device: exact statistics match the oracle's FP64
    loops (relative 1e-12), the map is monotone, covers [min, min + 4 sd)
    with k/4 buckets per sd, and every bucket equals the formula evaluated
    from the reported constants."""
    n = 500_000
    keys, kd = _map_case(gen, n, 21)
    gb, info = z.map_buckets(kd, z.default_opts())
    mn, mx, mean_d, sd = oracle.stats(keys)
    assert info.min == mn and info.max == mx
    assert abs(info.mean_d - mean_d) <= 1e-12 * max(1.0, mean_d)
    assert abs(info.sd - sd) <= 1e-12 * sd
    assert info.map == z.MAP_ZSCORE
    k = info.k
    assert abs(info.zc / 2.0 ** info.zsh - (k / 4.0) / sd) <= 1e-6 * (k / 4.0) / sd
    b = gb.cpu().numpy().view(np.uint32)
    d = ((keys - np.uint64(mn)) >> np.uint64(info.zsh)).astype(np.float64)  # < 2^32: exact
    f32 = d.astype(np.float32)  # round to nearest; the device converts toward zero
    f32 = np.where(f32.astype(np.float64) > d, np.nextafter(f32, np.float32(0)), f32)
    f = f32 * np.float32(info.zc)  # binary32 product, round to nearest
    expect = np.minimum(np.floor(f.astype(np.float64)).astype(np.int64), k - 1)
    assert np.array_equal(expect, b.astype(np.int64))
    order = np.argsort(keys, kind="stable")
    assert np.all(np.diff(b[order].astype(np.int64)) >= 0)  # monotone
    assert b[order[0]] == 0 and b[order[-1]] >= 1


# ---------------------------------------------------------------- graphs
def test_segmented_graph_capture_and_replays():
    """ZSORT_FLAG_GRAPH: the first call captures the launch sequence, the next
    ones replay it; every replay sorts fresh data exactly."""
    keys, vals, off, _ = inputs.segmented(250, 12, lo=1, hi=150_000)
    kp, vp = to_dev(keys, vals)
    offs = torch.from_numpy(off.view(np.int64)).to(DEV)
    ok, ov = oracle.zsort_segmented(keys, vals, off)
    stream = torch.cuda.Stream()
    opts = z.default_opts(flags=z.FLAG_GRAPH)
    kb, vb = torch.empty_like(kp), torch.empty_like(vp)
    with torch.cuda.stream(stream):
        for _ in range(3):
            kb.copy_(kp)
            vb.copy_(vp)
            z.sort_segmented(kb, vb, offs, opts=opts, stream=stream)
            assert np.array_equal(kb.cpu().numpy().view(np.uint64), ok)
            assert np.array_equal(vb.cpu().numpy().view(np.uint32), ov)


def test_pairs_graph_replays_with_learned_map():
    keys = inputs.gaussian_mixture(1_500_000, 14)
    vals = inputs.index_payload(keys.size)
    kp, vp = to_dev(keys, vals)
    ok, ov = oracle.zsort_pairs(keys, vals)
    stream = torch.cuda.Stream()
    opts = z.default_opts(flags=z.FLAG_GRAPH, mapper=z.MAP_LEARNED, learn_min=65536, sample=65536)
    kb, vb = torch.empty_like(kp), torch.empty_like(vp)
    with torch.cuda.stream(stream):
        for _ in range(3):
            kb.copy_(kp)
            vb.copy_(vp)
            z.sort_pairs(kb, vb, opts=opts, stream=stream)
            assert np.array_equal(kb.cpu().numpy().view(np.uint64), ok)
            assert np.array_equal(vb.cpu().numpy().view(np.uint32), ov)


# ---------------------------------------------------------------- key-only mode
def keys_only(keys, opts=None, key_type="u64"):
    k = torch.from_numpy(np.ascontiguousarray(keys).view(np.int64)).to(DEV)
    z.sort_pairs(k, None, key_type=key_type, opts=opts)
    return k.cpu().numpy().view(keys.dtype)


@pytest.mark.parametrize("n", [2, 255, 4097, 65537, 200_003, 3_000_000])
@pytest.mark.parametrize("family", FAMILIES)
def test_keys_only_matches_oracle(family, n):
    """vals = NULL: the keys alone, sorted exactly as the oracle sorts the pairs."""
    keys = inputs.FAMILIES[family](n, seed=n + 101)
    ok, _ = oracle.zsort_pairs(keys, inputs.index_payload(n))
    assert np.array_equal(keys_only(keys), ok)


@pytest.mark.parametrize("mapper", [z.MAP_ZSCORE, z.MAP_LEARNED])
def test_keys_only_skewed_and_graph(mapper):
    keys = inputs.lognormal(2_000_000, 31)
    ok, _ = oracle.zsort_pairs(keys, inputs.index_payload(keys.size))
    opts = z.default_opts(mapper=mapper, learn_min=65536, flags=z.FLAG_GRAPH)
    kp = torch.from_numpy(keys.view(np.int64)).to(DEV)
    kb = torch.empty_like(kp)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        for _ in range(2):
            kb.copy_(kp)
            z.sort_pairs(kb, None, opts=opts, stream=stream)
            assert np.array_equal(kb.cpu().numpy().view(np.uint64), ok)
    # 8-byte elements: the library counts 2/3 of the pairs' bytes per pass
    st = z.last_stats(stream)
    kb.copy_(kp)
    vb = torch.arange(keys.size, dtype=torch.int32, device=DEV)
    with torch.cuda.stream(stream):
        z.sort_pairs(kb, vb, opts=z.default_opts(mapper=mapper, learn_min=65536), stream=stream)
    st2 = z.last_stats(stream)
    assert st["bytes_algorithmic"] < st2["bytes_algorithmic"]


def test_keys_only_int64_float64_and_segmented():
    x = inputs.dense_interval_i64(400_000, 17)
    assert np.array_equal(keys_only(x.astype(np.int64), key_type="i64"), np.sort(x.astype(np.int64), kind="stable"))
    f = inputs.normal_f64_specials(400_000, 18)
    got = keys_only(f, key_type="f64")
    want = oracle.key_to_f64(np.sort(oracle.key_from_f64(f)))
    assert np.array_equal(got.view(np.uint64), want.view(np.uint64))
    keys, vals, off, _ = inputs.segmented(200, 19, lo=1, hi=200_000)
    k = torch.from_numpy(keys.view(np.int64)).to(DEV)
    z.sort_segmented(k, None, torch.from_numpy(off.view(np.int64)).to(DEV))
    ok, _ = oracle.zsort_segmented(keys, vals, off)
    assert np.array_equal(k.cpu().numpy().view(np.uint64), ok)


# ---------------------------------------------------------------- MLP map
@pytest.mark.parametrize("gen", [inputs.lognormal, inputs.gaussian_mixture, inputs.uniform,
                                 inputs.dense_interval_u64])
def test_mlp_map_bit_exact(gen):
    """MLP map: the device's trained parameters and every key's bucket equal
    the oracle's (same knots, same binary32 training steps in the same
    order); a rejected map is checked by the load-test rule."""
    n, m = 400_000, 65536
    keys, kd = _map_case(gen, n, 23)
    opts = z.default_opts(mapper=z.MAP_MLP, learn_min=m, sample=m, kmax=512)
    gb, info = z.map_buckets(kd, opts)
    mn, mx = int(keys.min()), int(keys.max())
    assert info.trained == 1
    pos = oracle.sample_positions(opts.seed, n, m).astype(np.int64)
    q = oracle.pwl_train(keys[pos], mn, mx)
    assert np.array_equal(np.frombuffer(bytes(info.q), dtype=np.float32), q)
    p = oracle.mlp_train(q, 128)
    H = oracle.MLP_H
    om, be, al = p[:H], p[H:2 * H], p[2 * H:3 * H]
    want = np.concatenate([om * om, be, al * al, p[3 * H:]]).astype(np.float32)
    assert np.array_equal(np.frombuffer(bytes(info.mlp), dtype=np.float32), want)
    k = info.k
    if info.map == z.MAPINFO_MLP:
        ob = oracle.mlp_buckets(keys, mn, mx, p, k)
        assert np.array_equal(gb.cpu().numpy().view(np.uint32), ob)
    else:  # rejected: then the exact-key map, or Eq. 1
        assert info.map in (z.MAPINFO_SPLIT, z.MAPINFO_ZSCORE)
        assert (info.learned_max_load > opts.fallback_ratio * m / k
                or info.learned_max_load > info.zscore_max_load)


@pytest.mark.parametrize("mapper", [z.MAP_LEARNED, z.MAP_MLP])
def test_exact_key_map_sorts_the_collapsing_int64_law(mapper):
    """Keys packed within 2^19 of 2^63 (the int64 dense interval, encoded):
    both normalised maps fail the load test, the exact-key map takes the top
    level, and the sort equals the oracle's, pairs and keys only."""
    keys = _dense_i64_encoded(3_000_000, 6)
    opts = z.default_opts(mapper=mapper, learn_min=1 << 20)
    vals = inputs.index_payload(keys.size)
    k, v = to_dev(keys, vals)
    z.sort_pairs(k, v, opts=opts)
    st = z.last_stats()
    assert st["top_map"] == z.MAPINFO_SPLIT
    ok, ov = oracle.zsort_pairs(keys, vals)
    assert np.array_equal(k.cpu().numpy().view(np.uint64), ok)
    assert np.array_equal(v.cpu().numpy().view(np.uint32), ov)
    kk = torch.from_numpy(keys.view(np.int64)).to(DEV)
    z.sort_keys(kk, opts=opts)
    assert np.array_equal(kk.cpu().numpy().view(np.uint64), ok)


@pytest.mark.parametrize("gen", [inputs.lognormal, inputs.uniform, inputs.gaussian_mixture])
def test_mlp_mapper_sorts_exactly(gen):
    keys = gen(3_000_000, 24)
    assert_same_as_oracle(keys, opts=z.default_opts(mapper=z.MAP_MLP, learn_min=1 << 20))


# ---------------------------------------------------------------- failure path
def test_bounded_wait_runs_out_and_the_context_recovers():
    """ZSORT_FLAG_TEST_STALL: every CTA waits for a queue entry that nothing
    publishes; after wait_limit_ms without progress the kernel records
    ZSORT_ERR_TIMEOUT and returns (no trap, no hang).  The data is untouched
    and the next call on the same stream sorts exactly."""
    import time

    keys = inputs.uniform(1 << 20, 41)
    vals = inputs.index_payload(keys.size)
    k, v = to_dev(keys, vals)
    t0 = time.perf_counter()
    with pytest.raises(z.ZsortError) as ei:
        z.sort_pairs(k, v, opts=z.default_opts(flags=z.FLAG_TEST_STALL, wait_limit_ms=50))
    assert ei.value.code == z.ERR_TIMEOUT
    assert time.perf_counter() - t0 < 10.0
    assert np.array_equal(k.cpu().numpy().view(np.uint64), keys)
    assert np.array_equal(v.cpu().numpy().view(np.uint32), vals)
    assert z.sync_status() == z.OK  # the status word was read and cleared
    z.sort_pairs(k, v)
    ok, ov = oracle.zsort_pairs(keys, vals)
    assert np.array_equal(k.cpu().numpy().view(np.uint64), ok)
    assert np.array_equal(v.cpu().numpy().view(np.uint32), ov)


@pytest.mark.parametrize("mode,code,when", [("alloc", z.ERR_NOMEM, "call"),
                                            ("timeout", z.ERR_TIMEOUT, "status"),
                                            ("badoffsets", z.ERR_BAD_OFFSETS, "status")])
@pytest.mark.parametrize("segmented", [False, True])
def test_fault_injection_env(monkeypatch, mode, code, when, segmented):
    """ZSORT_FAULT injects a failure on the host: the call (alloc) or the
    device status (timeout, bad offsets) reports it, the data is untouched,
    and the next call without the variable sorts exactly."""
    keys, vals, off, _ = inputs.segmented(40, 43, lo=32, hi=200_000) if segmented else \
        (inputs.uniform(300_000, 42), None, None, None)
    vals = inputs.index_payload(keys.size) if vals is None else vals
    k, v = to_dev(keys, vals)
    od = torch.from_numpy(off.view(np.int64)).to(DEV) if segmented else None

    def run():
        if segmented:
            z.sort_segmented(k, v, od)
        else:
            z.sort_pairs(k, v)

    monkeypatch.setenv("ZSORT_FAULT", mode)
    with pytest.raises(z.ZsortError) as ei:
        run()
    assert ei.value.code == code
    if when == "call":
        assert z.sync_status() == z.OK
    assert np.array_equal(k.cpu().numpy().view(np.uint64), keys)
    assert np.array_equal(v.cpu().numpy().view(np.uint32), vals)
    monkeypatch.delenv("ZSORT_FAULT")
    run()
    ok, ov = oracle.zsort_segmented(keys, vals, off) if segmented else oracle.zsort_pairs(keys, vals)
    assert np.array_equal(k.cpu().numpy().view(np.uint64), ok)
    assert np.array_equal(v.cpu().numpy().view(np.uint32), ov)


# ---------------------------------------------------------------- 128-bit keys
def u128_case(n, seed, hi_distinct=None, lo_distinct=None):
    rng = np.random.default_rng(seed)
    hi = rng.integers(0, 2 ** 64, n, dtype=np.uint64, endpoint=False)
    lo = rng.integers(0, 2 ** 64, n, dtype=np.uint64, endpoint=False)
    if hi_distinct is not None:
        hi = rng.choice(hi[:max(hi_distinct, 1)], n)
    if lo_distinct is not None:
        lo = rng.choice(lo[:max(lo_distinct, 1)], n)
    return hi, lo


@pytest.mark.parametrize("n,hi_d,lo_d", [(2, None, None), (1001, None, None), (300_001, None, None),
                                        (300_000, 7, None), (300_000, None, 5), (300_000, 1, 3),
                                        (2_000_001, 1000, 1000)])
@pytest.mark.parametrize("with_vals", [True, False])
def test_u128_keys_match_the_stable_order(n, hi_d, lo_d, with_vals):
    """(high, low) word pairs sorted as unsigned 128-bit numbers, stably: the
    oracle is the definition (numpy's stable lexsort on (high, low))."""
    hi, lo = u128_case(n, n + 3, hi_d, lo_d)
    words = np.empty(2 * n, dtype=np.uint64)
    words[0::2], words[1::2] = lo, hi
    k = torch.from_numpy(words.view(np.int64)).to(DEV)
    v = torch.arange(n, dtype=torch.int32, device=DEV) if with_vals else None
    z.sort_pairs_u128(k, v)
    order = np.lexsort((lo, hi))  # primary hi, then lo; stable on ties
    got = k.cpu().numpy().view(np.uint64)
    assert np.array_equal(got[0::2], lo[order]) and np.array_equal(got[1::2], hi[order])
    if with_vals:
        assert np.array_equal(v.cpu().numpy().view(np.uint32), order.astype(np.uint32))


def u128_window_case(n, s, nwin, seed, dup):
    """Keys min + (w << s | r) with w drawn from nwin windows (0 and 2^64 - 1
    among them, so that the range's bit length is 64 + s) and r below 2^s:
    runs of equal windows resolved by the bits below them; dup draws r from
    five values, so that equal keys repeat."""
    rng = np.random.default_rng(seed)
    wins = rng.integers(0, 2 ** 64, nwin, dtype=np.uint64, endpoint=False)
    wins[0] = 0
    if nwin > 1:
        wins[-1] = np.uint64(2 ** 64 - 1)
    w = rng.choice(wins, n)
    r = rng.integers(0, 2 ** s, n, dtype=np.uint64, endpoint=False) if s < 64 else \
        rng.integers(0, 2 ** 64, n, dtype=np.uint64, endpoint=False)
    if dup:
        r = r % np.uint64(5)
    if s == 64:
        dhi, dlo = w, r
        mn_lo = np.uint64(0)
    else:
        dlo = (w << np.uint64(s)) | r
        dhi = w >> np.uint64(64 - s)
        mn_lo = np.uint64(rng.integers(0, 2 ** 64, dtype=np.uint64, endpoint=False))
    lo = dlo + mn_lo
    hi = dhi + (lo < mn_lo).astype(np.uint64)
    return hi, lo


@pytest.mark.parametrize("s", [1, 17, 40, 63, 64])
@pytest.mark.parametrize("nwin,dup", [(2, False), (100, False), (150_000, False), (100, True)])
def test_u128_window_runs_resolved_below_the_window(s, nwin, dup):
    """The 128-bit path's tie resolution: many keys share a 64-bit window
    (two runs of half the keys each, 100 long runs, ~150,000 short ones, and
    equal keys repeated), at window shifts 1..64; the result is numpy's
    stable lexsort on (high, low), keys and payloads."""
    n = 300_001
    hi, lo = u128_window_case(n, s, nwin, 1000 * s + nwin, dup)
    words = np.empty(2 * n, dtype=np.uint64)
    words[0::2], words[1::2] = lo, hi
    k = torch.from_numpy(words.view(np.int64)).to(DEV)
    v = torch.arange(n, dtype=torch.int32, device=DEV)
    z.sort_pairs_u128(k, v)
    order = np.lexsort((lo, hi))
    got = k.cpu().numpy().view(np.uint64)
    assert np.array_equal(got[0::2], lo[order]) and np.array_equal(got[1::2], hi[order])
    assert np.array_equal(v.cpu().numpy().view(np.uint32), order.astype(np.uint32))


def test_u128_more_window_runs_than_one_launch_takes():
    """1,057,674 runs of equal windows, more than the 2^20 runs one launch
    takes (4 million keys over 2 million windows at shift 40): the runs are
    sorted in two slices; the result is still numpy's stable lexsort on
    (high, low)."""
    n = 4_000_001
    hi, lo = u128_window_case(n, 40, n // 2, 77, False)
    words = np.empty(2 * n, dtype=np.uint64)
    words[0::2], words[1::2] = lo, hi
    k = torch.from_numpy(words.view(np.int64)).to(DEV)
    v = torch.arange(n, dtype=torch.int32, device=DEV)
    z.sort_pairs_u128(k, v)
    order = np.lexsort((lo, hi))
    got = k.cpu().numpy().view(np.uint64)
    assert np.array_equal(got[0::2], lo[order]) and np.array_equal(got[1::2], hi[order])
    assert np.array_equal(v.cpu().numpy().view(np.uint32), order.astype(np.uint32))


def _repeated_key_leaves(distinct, seed):
    """40 leaves' worth of keys, far apart: in each, `distinct` adjacent keys
    repeated ~3000 / distinct times in random order, plus a few far keys that
    widen the leaf's range so that the adjacent keys share one sub-bucket."""
    rng = np.random.default_rng(seed)
    parts = []
    for g in range(40):
        base = np.uint64(g) << np.uint64(56)
        x = base + rng.integers(0, distinct, 3000).astype(np.uint64)
        x[::997] = base + np.uint64(1 << 40)
        parts.append(x)
    return np.concatenate(parts)


def _sort_and_fallbacks(keys):
    vals = inputs.index_payload(keys.size)
    k, v = to_dev(keys, vals)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        z.sort_pairs(k, v, stream=stream)
        fb = z.last_stats(stream)["leaf_fallbacks"]
    ok, ov = oracle.zsort_pairs(keys, vals)
    assert np.array_equal(k.cpu().numpy().view(np.uint64), ok)
    assert np.array_equal(v.cpu().numpy().view(np.uint32), ov)
    return fb


@pytest.mark.parametrize("distinct", [2, 7, 32])
def test_leaf_with_few_repeated_keys_takes_the_warp_counting_sort(distinct):
    """Leaves whose sub-buckets mix up to 32 distinct keys, each repeated
    many times in random order: sorted stably by a warp's counting sort over
    the distinct keys, with no sorting network."""
    assert _sort_and_fallbacks(_repeated_key_leaves(distinct, 51 + distinct)) == 0


def test_leaf_with_many_repeated_keys_takes_the_network():
    """Sub-buckets of 64 distinct keys, each repeated ~47 times in random
    order: more than a warp's counting sort takes, so sorted by the
    per-sub-bucket sorting network, stably."""
    assert _sort_and_fallbacks(_repeated_key_leaves(64, 52)) > 0


def _child_stress(n_bulk, n_run, n_out, seed):
    """Uniform keys over [0, 2^40) plus, inside one top-level bucket, a run
    of n_run copies of one value V with a few distinct keys right beside it
    and a few far outliers on both sides (still below the next bucket),
    shuffled: the sub-array of that bucket is large, its 4096-key sample
    sees V alone or a narrow spread, and its true min and max lie outside
    what the sample saw."""
    rng = np.random.default_rng(seed)
    V = 10 ** 11
    bulk = rng.integers(0, 2 ** 40, n_bulk, dtype=np.uint64)
    run = np.full(n_run, V, dtype=np.uint64)
    near = (V + rng.integers(1, 1000, n_out)).astype(np.uint64)
    far = np.array([V - 500, V - 499, V + 10 ** 6, V + 10 ** 6 + 1][: max(2, n_out)], dtype=np.uint64)
    keys = np.concatenate([bulk, run, near, far])
    return keys[rng.permutation(keys.size)]


@pytest.mark.parametrize("n_run,n_out", [(300_000, 3), (300_000, 0), (150_000, 40)])
def test_sampled_substats_with_unseen_extremes(n_run, n_out):
    """Sub-array statistics from a sample: a sample without spread falls
    back to the exact pass, and keys outside the sampled [min, max] are
    clamped into the end buckets; the output is the oracle's in every case,
    and the same as with exact statistics at every level."""
    keys = _child_stress(1_000_000, n_run, n_out, 7 + n_run + n_out)
    vals = inputs.index_payload(keys.size)
    ok_k, ok_v = oracle.zsort_pairs(keys, vals)
    for flags in (0, z.FLAG_EXACT_SUBSTATS):
        k, v = gpu_sort(keys, vals, z.default_opts(flags=flags))
        assert np.array_equal(k, ok_k) and np.array_equal(v, ok_v)


@pytest.mark.parametrize("gen", [inputs.uniform, inputs.lognormal, inputs.zipf, inputs.nearly_sorted])
def test_sampled_substats_count_and_bytes(gen):
    """Two partition levels: the second level's sub-arrays take sampled
    statistics (counted in zsort_stats.sampled_stats), which saves their
    8 B/pair statistics pass; ZSORT_FLAG_EXACT_SUBSTATS restores it; both
    outputs equal the oracle's."""
    n = 6_000_000
    keys = gen(n, 23)
    vals = inputs.index_payload(n)
    ok_k, ok_v = oracle.zsort_pairs(keys, vals)
    got = {}
    for flags in (0, z.FLAG_EXACT_SUBSTATS):
        kd, vd = to_dev(keys, vals)
        z.sort_pairs(kd, vd, opts=z.default_opts(flags=flags))
        st = z.last_stats()
        assert np.array_equal(kd.cpu().numpy().view(np.uint64), ok_k)
        assert np.array_equal(vd.cpu().numpy().view(np.uint32), ok_v)
        got[flags] = st
    assert got[z.FLAG_EXACT_SUBSTATS]["sampled_stats"] == 0
    if got[0]["partitions_large"] > 1:
        assert got[0]["sampled_stats"] >= 1
        assert got[0]["bytes_algorithmic"] < got[z.FLAG_EXACT_SUBSTATS]["bytes_algorithmic"]


def _signed_order(t, key_type):
    """int64 values whose signed order is the key order (int64 storage)."""
    sign = torch.tensor(-(2 ** 63), dtype=torch.int64, device=t.device)
    if key_type == "u64":
        return t ^ sign
    if key_type == "i64":
        return t
    return torch.where(t >= 0, t, t ^ torch.tensor(2 ** 63 - 1, dtype=torch.int64, device=t.device))


def _check_order_payload_stability(k_in, k_out, v_out, key_type):
    o = _signed_order(k_out, key_type)
    assert bool((o[1:] >= o[:-1]).all()), "not sorted"
    pos = v_out.to(torch.int64) & 0xFFFFFFFF
    assert bool(torch.equal(k_in[pos], k_out)), "a payload does not name its key"
    assert int(torch.bincount(pos, minlength=k_in.numel()).max()) == 1, "payloads are not a permutation"
    eq = k_out[1:] == k_out[:-1]
    assert bool((pos[1:][eq] > pos[:-1][eq]).all()), "equal keys out of input order"


@pytest.mark.parametrize("key_type,gen", [("u64", inputs.dense_interval_u64),
                                          ("i64", lambda n, s: inputs.dense_interval_i64(n, s).view(np.uint64)),
                                          ("f64", lambda n, s: inputs.normal_f64_specials(n, s).view(np.uint64))])
def test_config4_full_size_adversarial_1e8(key_type, gen):
    """The adversarial workload at its stated size: n = 10^8, learned map with
    the Eq. 1 fallback at 4x the mean bucket load; u64 with 90% of the keys in
    one interval of width 2^20, the int64 law recentred on 0, and float64
    N(0,1) with 1% +-inf and 1% signed zeros (IEEE totalOrder: -0.0 first).
    Checked at full size by the properties that fix the stable sort: order,
    the payloads a permutation that names each key, equal keys in input
    order.  The float64 specials are also checked by count and place."""
    n = 10 ** 8
    keys = gen(n, 4)
    kd = torch.from_numpy(keys.view(np.int64)).to(DEV)
    vd = torch.arange(n, dtype=torch.int32, device=DEV)
    kb, vb = kd.clone(), vd.clone()
    z.sort_pairs(kb, vb, key_type=key_type, opts=z.default_opts(mapper=z.MAP_LEARNED, fallback_ratio=4.0))
    st = z.last_stats()
    assert st["max_level"] <= 48
    _check_order_payload_stability(kd, kb, vb, key_type)
    if key_type == "f64":
        x = kb.view(torch.float64)
        ninf, pinf = int(torch.isneginf(x).sum()), int(torch.isposinf(x).sum())
        assert bool(torch.isneginf(x[:ninf]).all()) and bool(torch.isposinf(x[n - pinf:]).all())
        zeros = (x == 0).nonzero().flatten()
        zbits = kb[zeros]
        negz = int((zbits < 0).sum())  # -0.0 has the sign bit
        assert bool((zbits[:negz] < 0).all()) and bool((zbits[negz:] == 0).all())
    del kd, vd, kb, vb
    torch.cuda.empty_cache()


def test_config5_full_size_20000_segments():
    """The batched workload at its stated size: 20,000 arrays with
    log-uniform sizes 32..2^20 (about 2e9 pairs), each from one of the five
    laws, sorted by one persistent launch under a CUDA graph; every segment
    checked for order, payloads (within-segment index) naming their keys,
    and stability."""
    nseg = 20_000
    keys, vals, off, _ = inputs.segmented_parallel(nseg, 5)
    n = keys.size
    kd = torch.from_numpy(keys.view(np.int64)).to(DEV)
    vd = torch.from_numpy(vals.view(np.int32)).to(DEV)
    od = torch.from_numpy(off.view(np.int64)).to(DEV)
    del keys, vals
    kb, vb = kd.clone(), vd.clone()
    stream = torch.cuda.Stream(device=DEV)
    with torch.cuda.stream(stream):
        z.sort_segmented(kb, vb, od, opts=z.default_opts(flags=z.FLAG_GRAPH), stream=stream)
    stream.synchronize()
    starts = torch.zeros(n, dtype=torch.bool, device=DEV)
    starts[od[:-1][od[:-1] < n]] = True
    same = ~starts[1:]
    del starts
    o = kb ^ torch.tensor(-(2 ** 63), dtype=torch.int64, device=DEV)
    assert bool((o[1:] >= o[:-1])[same].all()), "a segment is not sorted"
    del o
    seg = torch.repeat_interleave(torch.arange(nseg, device=DEV, dtype=torch.int32), (od[1:] - od[:-1]))
    src = od[:-1][seg.to(torch.int64)] + (vb.to(torch.int64) & 0xFFFFFFFF)
    del seg
    assert bool(torch.equal(kd[src], kb)), "a payload does not name its key"
    del src
    eq = same & (kb[1:] == kb[:-1])
    assert bool((vb[1:][eq].to(torch.int64) > vb[:-1][eq].to(torch.int64)).all()), "equal keys out of input order"
    del kd, vd, kb, vb, od, eq, same
    torch.cuda.empty_cache()


def test_fresh_workspace_on_a_side_stream_sorts_at_once():
    """A workspace allocated by a call on a non-blocking stream is cleared
    in that stream's order: right after zsort_release, a first call on a
    new side stream (a workspace of several GB, so clearing it takes
    milliseconds) must see its own published work and sort exactly, with
    and without graph capture."""
    n = 1 << 27
    keys = inputs.uniform(n, 61)
    kd = torch.from_numpy(keys.view(np.int64)).to(DEV)
    vd = torch.arange(n, dtype=torch.int32, device=DEV)
    for flags in (0, z.FLAG_GRAPH):
        z.release()
        kb, vb = kd.clone(), vd.clone()
        stream = torch.cuda.Stream(device=DEV)
        with torch.cuda.stream(stream):
            z.sort_pairs(kb, vb, opts=z.default_opts(flags=flags), stream=stream)
        _check_order_payload_stability(kd, kb, vb, "u64")
    del kd, vd, kb, vb
    torch.cuda.empty_cache()


@pytest.mark.parametrize("family", ["uniform", "normal", "zipf", "nearly_sorted", "descending"])
@pytest.mark.parametrize("n", [4097, 65_537, 200_003, 3_000_001])
def test_eight_items_per_thread(family, n):
    """zsort_opts.ipt = 8 (tiles of 2048 pairs, the autotuner's other choice):
    the statistics, histogram and scatter passes run their 8-item
    instantiations, the scatter with ballots where k = 512 leaves no room
    for a warp's peer table; the output is the oracle's."""
    keys = inputs.FAMILIES[family](n, 70 + n)
    assert_same_as_oracle(keys, opts=z.default_opts(ipt=8))


@pytest.mark.parametrize("mapper", [z.MAP_ZSCORE, z.MAP_LEARNED, z.MAP_MLP])
def test_eight_items_per_thread_maps_keys_only_segmented(mapper):
    """ipt = 8 with every map (the learned maps' bucket ids are written per
    2048-pair tile), keys alone, and a segmented batch."""
    keys = inputs.lognormal(3_000_000, 71)
    opts = z.default_opts(ipt=8, mapper=mapper, learn_min=1 << 20)
    assert_same_as_oracle(keys, opts=opts)
    kd = torch.from_numpy(keys.view(np.int64)).to(DEV)
    z.sort_pairs(kd, None, opts=opts)
    assert np.array_equal(kd.cpu().numpy().view(np.uint64), np.sort(keys))
    sk, sv, off, _ = inputs.segmented(200, 72, lo=1, hi=300_000)
    kp, vp = to_dev(sk, sv)
    z.sort_segmented(kp, vp, torch.from_numpy(off.view(np.int64)).to(DEV), opts=opts)
    ok_k, ok_v = oracle.zsort_segmented(sk, sv, off)
    assert np.array_equal(kp.cpu().numpy().view(np.uint64), ok_k)
    assert np.array_equal(vp.cpu().numpy().view(np.uint32), ok_v)


def test_invalid_items_per_thread_is_rejected():
    kd = torch.zeros(100, dtype=torch.int64, device=DEV)
    with pytest.raises(z.ZsortError):
        z.sort_pairs(kd, None, opts=z.default_opts(ipt=10))
